"""The allocation-free triangular solve (tqr_trsm_static) against tqr_trsm.

tqr_trsm_static exists for callers that must not allocate device memory: its scratch
lives in a fixed array inside the library.  Its results must equal those of tqr_trsm
(the same kernel, scratch from the library's allocator) on two calls in a row - the
second call reuses the array the first one left behind - and the calls must not change
the device's free memory.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1303_3182_gb300 as tqr  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1303_3182_gb300 import build
    build.build()


def to_dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).to(dtype).cuda().t()


@pytest.mark.parametrize("prec,rdtype", [("fp64", torch.float64), ("fp32", torch.float32)])
def test_static_trsm_matches_trsm_twice(prec, rdtype):
    n, nrhs = 333, 37
    R = np.triu(synthetic.gaussian(n, n, seed=2)) + 4 * np.eye(n)
    if prec == "fp32":
        R = R.astype(np.float32).astype(np.float64)
    Bm = synthetic.gaussian(n, nrhs, seed=3)
    Rd = to_dev(R, rdtype)
    ref = to_dev(Bm)
    tqr.trsm(Rd, ref, n, prec)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    scale = np.max(np.abs(ref))
    # the first call on this device does the one-time set-up (address lookup)
    tqr.trsm_static(Rd, to_dev(Bm), n, prec)
    torch.cuda.synchronize()
    b1, b2 = to_dev(Bm), to_dev(Bm)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    tqr.trsm_static(Rd, b1, n, prec)
    tqr.trsm_static(Rd, b2, n, prec)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    for out in (b1, b2):
        assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-12 * scale
    assert free_after == free_before


def test_static_trsm_rejects_sizes_beyond_its_scratch():
    """n above 4096 blocks of 64 rows is refused before any device work (dummy pointers
    are never touched)."""
    L = tqr.lib()
    vp = ctypes.c_void_p
    n = 4096 * 64 + 1
    assert L.tqr_trsm_static(n, 0, vp(16), n, vp(16), n, 1, None) == -1
    assert b"static scratch limit" in L.tqr_last_error()
    assert L.tqr_trsm_static(0, 0, vp(16), 1, vp(16), 1, 1, None) == -1
