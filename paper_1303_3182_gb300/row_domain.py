"""Least squares of one tall matrix whose rows are split across ranks (row domains).

Section 3.2.4's PlasmaTree zeroes a tile column with a flat tree inside each domain of
consecutive rows and merges the domain heads with a binary tree.  Lifted to GPUs, a
domain is the block of rows one rank holds:

1. every rank factors its own row block A_r = Q_r [R_r; 0] (any tree, on its GPU) and
   applies Q_r^T to its right-hand sides, b_r = Q_r [c_r; e_r]: the n x n triangle R_r
   and the n x nrhs block c_r summarize the rank's rows;
2. one exchange step gathers every rank's (R_r, c_r) - n (n + nrhs) numbers per rank;
3. the stacked triangles [R_0; ...; R_{P-1}] are reduced by a tiled QR whose
   eliminations zero the lower ranks' triangles (the merge of the domain heads), the
   same transformation applied to [c_0; ...; c_{P-1}], and R x = c is solved.

Because ||A x - b||^2 = sum_r ||R_r x - c_r||^2 + ||e_r||^2, the merged problem has the
same minimizer as the whole one.  The per-rank reduction and the merge are passed in as
functions, so the exchange protocol is the same whatever computes them: the GPU
functions below call the library (tqr_factor / tqr_apply_qt / tqr_lstsq).
"""
from __future__ import annotations


def row_blocks(m: int, world: int, nb: int):
    """[start, stop) rows of each rank: whole tiles of nb rows, spread as evenly as
    possible (the last rank takes the ragged end)."""
    tiles = -(-m // nb)
    out, t0 = [], 0
    for r in range(world):
        t1 = t0 + tiles // world + (1 if r < tiles % world else 0)
        out.append((min(t0 * nb, m), min(t1 * nb, m)))
        t0 = t1
    return out


def solve(A_local, B_local, local_reduce, merge):
    """Least-squares solution of the row-split problem on every rank.

    A_local (m_r x n) and B_local (m_r x nrhs) are this rank's rows; local_reduce(A, B)
    returns (R_r, c_r) as float64 torch tensors (n x n upper triangular, n x nrhs) on the
    device the process group communicates on; merge(S, D) solves the stacked problem
    min ||S x - D|| and returns (x, R).  With one rank (no process group) the exchange is
    the identity."""
    import torch
    import torch.distributed as dist
    R, c = local_reduce(A_local, B_local)
    R = R.contiguous()
    c = c.contiguous()
    if dist.is_initialized() and dist.get_world_size() > 1:
        world = dist.get_world_size()
        Rs = [torch.empty_like(R) for _ in range(world)]
        cs = [torch.empty_like(c) for _ in range(world)]
        dist.all_gather(Rs, R)
        dist.all_gather(cs, c)
    else:
        Rs, cs = [R], [c]
    return merge(torch.cat(Rs, 0), torch.cat(cs, 0))


def gpu_local_reduce(nb: int, ib: int, tree="greedy", bs: int = 1):
    """Per-rank reduction on the GPU: FP64 tiled QR of the row block, Q^T applied to B."""
    def run(A, B):
        import torch
        from . import apply_qt, colmajor, factor
        m, n = A.shape
        if m < n:
            raise ValueError("every row block needs at least n rows")
        Aw = colmajor(A.to(torch.float64).clone())
        Bw = colmajor(B.to(torch.float64).clone())
        T = factor(Aw, nb, ib, tree, bs, "fp64")
        apply_qt(Aw, T, Bw, nb, ib, tree, bs, "fp64", trans=0)
        return torch.triu(Aw[:n, :n]), Bw[:n].clone()
    return run


def gpu_merge(nb: int, ib: int, tree="greedy", bs: int = 1):
    """The merge on the GPU: FP64 tiled QR of the stacked triangles, the same Q^T applied
    to the stacked blocks, and the triangular solve with the merged triangle R."""
    def run(S, D):
        import torch
        from . import apply_qt, colmajor, factor, trsm
        n = S.shape[1]
        Sw = colmajor(S.to(torch.float64).clone())
        Dw = colmajor(D.to(torch.float64).clone())
        T = factor(Sw, nb, ib, tree, bs, "fp64")
        apply_qt(Sw, T, Dw, nb, ib, tree, bs, "fp64", trans=0)
        trsm(Sw, Dw, n, "fp64")
        return Dw[:n].clone(), torch.triu(Sw[:n, :n])
    return run
