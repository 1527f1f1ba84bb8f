"""The row-domain split of one tall least-squares problem (Section 3.2.4's PlasmaTree
lifted to ranks: a flat elimination inside each rank's row domain, then one merge of the
domain heads' triangles), run as gloo ranks on CPU.

Each rank reduces its own rows to (R_r, c_r); one all-gather exchanges them; the stacked
triangles are merged.  The exchange protocol is the library's (paper_1303_3182_gb300.
row_domain.solve); the per-rank reduction and the merge are the oracle's tiled QR here
(on GPUs they are the library's), so the result must equal the single-process oracle's:
|R| to FP64 rounding and the solution within the LS perturbation bound."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

M, N, NRHS, NB, IB, COND = 600, 80, 2, 32, 8, 1e3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_reduce(tree):
    def run(A, B):
        from oracle import elimlists as E
        from oracle import householder as H
        A = A.numpy()
        B = B.numpy()
        m, n = A.shape
        p, q = H.tile_grid(m, n, NB)
        elims = E.elimination_list(p, q, tree)
        F, Tg, Tt = H.tiled_qr(A, NB, IB, elims)
        QtB = H.apply_qt(F, Tg, Tt, NB, IB, elims, B)
        return torch.from_numpy(np.triu(F[:n, :n]).copy()), torch.from_numpy(QtB[:n].copy())
    return run


def _oracle_merge(S, D):
    from oracle import elimlists as E
    from oracle import householder as H
    S = S.numpy()
    D = D.numpy()
    m, n = S.shape
    p, q = H.tile_grid(m, n, NB)
    elims = E.elimination_list(p, q, E.BINARY)
    F, Tg, Tt = H.tiled_qr(S, NB, IB, elims)
    QtD = H.apply_qt(F, Tg, Tt, NB, IB, elims, D)
    R = np.triu(F[:n, :n])
    return torch.from_numpy(H.back_substitute(R, QtD[:n])), torch.from_numpy(R)


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import synthetic
    from oracle import elimlists as E
    from paper_1303_3182_gb300 import replicas, row_domain
    replicas.init("gloo")
    A, _, B = synthetic.least_squares_problem(M, N, COND, 1e-3, NRHS, seed=1303318206)
    r0, r1 = row_domain.row_blocks(M, world, NB)[rank]
    x, R = row_domain.solve(torch.from_numpy(A[r0:r1].copy()), torch.from_numpy(B[r0:r1].copy()),
                            _oracle_reduce(E.FLAT if rank % 2 else E.GREEDY), _oracle_merge)
    replicas.finalize()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"x": x.numpy().tolist(), "R": R.numpy().tolist(), "rows": [r0, r1]}, f)


@pytest.mark.parametrize("world", [2, 3])
def test_row_domain_split_matches_single_process(tmp_path, world):
    import synthetic
    from oracle import elimlists as E
    from oracle import householder as H
    from oracle import refine
    from paper_1303_3182_gb300 import row_domain
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    # the domains tile the rows exactly once, in whole tiles
    rows = [tuple(x["rows"]) for x in res]
    assert rows[0][0] == 0 and rows[-1][1] == M
    assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
    assert all(r0 % NB == 0 for r0, _ in rows)
    assert rows == row_domain.row_blocks(M, world, NB)
    A, _, B = synthetic.least_squares_problem(M, N, COND, 1e-3, NRHS, seed=1303318206)
    p, q = H.tile_grid(M, N, NB)
    Xo = H.lstsq(A, B, NB, IB, E.elimination_list(p, q, E.GREEDY))
    Ro = np.linalg.qr(A, mode="r")
    r = B - A @ Xo
    bound = 64 * 2.0 ** -53 * (COND + COND ** 2 * np.linalg.norm(r) / np.linalg.norm(Xo))
    for x in res:
        X = np.array(x["x"])
        R = np.array(x["R"])
        assert refine.rel_error(X, Xo) <= bound
        assert np.max(np.abs(np.abs(R) - np.abs(Ro))) <= 1e-13 * np.linalg.norm(A) * M
    # every rank computed the same merge
    assert all(np.array_equal(np.array(x["x"]), np.array(res[0]["x"])) for x in res)


def test_row_blocks_single_rank_and_ragged():
    from paper_1303_3182_gb300 import row_domain
    assert row_domain.row_blocks(1000, 1, 64) == [(0, 1000)]
    blocks = row_domain.row_blocks(1000, 3, 64)  # 16 tiles: 6, 5, 5
    assert blocks == [(0, 384), (384, 704), (704, 1000)]
