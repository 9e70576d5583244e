"""bccb_solve_noalloc: the entry point for callers that cannot allocate device
memory, checked against the ordinary entry point through the C ABI.

Collected last on purpose (file name), so a run that stops at the first failure
has already run every other test.  It must also pass on its own in a fresh
process: the first call on a device performs that device's one-time set-up.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import REL_TOL, gpu_run, rel_err

pytestmark = pytest.mark.gpu

ALGO = {"ista": 0, "fista": 1, "admm": 2}


def _entry(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    f = so.bccb_solve_noalloc
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    f.argtypes = [i32, i32, vp, i32, i32, i32, dbl, vp, dbl, i32, i32, vp, vp]
    f.restype = i32
    return f


def _noalloc(lib, f, s, algo, lam, iters, rho, lam_is_frac=0, mask=None):
    import torch

    mask = torch.from_numpy(np.ascontiguousarray(s.mask if mask is None else mask, np.uint8)).cuda()
    y = torch.from_numpy(s.y.astype(np.complex64)).cuda()
    c = torch.full((s.L1 * s.L2,), 7.0 + 7.0j, dtype=torch.complex64, device="cuda")  # garbage on purpose
    st = f(s.M1, s.M2, mask.data_ptr(), s.L1, s.L2, ALGO[algo], rho, y.data_ptr(), lam, lam_is_frac, iters,
           c.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.bccb_status_string(st)
    torch.cuda.synchronize()
    return c.cpu().numpy()


def test_noalloc_matches_ordinary_entry_point_on_two_calls_in_a_row(lib):
    f = _entry(lib)
    s1 = synth.workload_snapshot("solve256", 1)  # 32x32 array, N=256, 256x256 grid
    s2 = synth.make_snapshot(77, 16, 32, 120, 64, 128, 4, 12.0)
    s3 = synth.make_snapshot(78, 12, 8, 40, 32, 64, 3, 15.0)
    # (snapshot, algorithm, iterations, rho, lam given as a fraction of ||A^H y||_inf)
    cases = [(s1, "fista", 300, 1.0, False), (s2, "admm", 150, 4.0, False), (s3, "ista", 200, 1.0, True)]
    for s, algo, iters, rho, frac in cases:
        lam = 0.05 * _lmax(s)
        ref = gpu_run(lib, [s], [lam], algo, iters, rho=rho, check=False)["c"][0]
        if frac:
            got = _noalloc(lib, f, s, algo, 0.05, iters, rho, lam_is_frac=1)
        else:
            got = _noalloc(lib, f, s, algo, lam, iters, rho)
        assert rel_err(got, ref) <= REL_TOL, (algo, rel_err(got, ref))
        assert np.array_equal(np.abs(got) > 0, np.abs(ref) > 0)


def test_noalloc_against_the_oracle(lib):
    """One case checked against the FP64 oracle directly, so the entry point is pinned
    independently of the ordinary one."""
    from gpu_util import assert_parity, oracle_run

    f = _entry(lib)
    s = synth.workload_snapshot("fista64", 0)  # 16x16 array, N = 64, 64x64 grid, 3 on-grid sources
    ref = oracle_run(s, "fista", 500)
    got = _noalloc(lib, f, s, "fista", ref["lam"], 500, 1.0)
    assert_parity(got, ref, what="noalloc FISTA 64x64")


def test_noalloc_empty_mask_returns_zero(lib):
    """No element kept: A has no rows, so c = 0 minimises the LASSO; the call returns it
    (and not the NaN that 1/max Lambda would give)."""
    f = _entry(lib)
    s = synth.make_snapshot(79, 8, 8, 10, 32, 32, 2, 10.0)
    for algo in ("fista", "admm"):
        got = _noalloc(lib, f, s, algo, 0.1, 20, 2.0, lam_is_frac=1, mask=np.zeros(64, np.uint8))
        assert np.all(got == 0), algo


def test_noalloc_rejects_sizes_beyond_its_limits(lib):
    import torch

    f = _entry(lib)
    dummy = torch.zeros(16, dtype=torch.complex64, device="cuda")
    m = torch.ones(16, dtype=torch.uint8, device="cuda")
    p = dummy.data_ptr()
    stream = torch.cuda.current_stream().cuda_stream
    assert f(4, 4, m.data_ptr(), 512, 16, 1, 1.0, p, 0.1, 0, 10, p, stream) == lib.ERR_UNSUPPORTED
    assert f(200, 100, m.data_ptr(), 64, 64, 1, 1.0, p, 0.1, 0, 10, p, stream) == lib.ERR_UNSUPPORTED
    assert f(4, 4, m.data_ptr(), 64, 64, 1, 1.0, p, 0.1, 0, 9000, p, stream) == lib.ERR_UNSUPPORTED
    assert f(4, 4, m.data_ptr(), 64, 64, 2, 0.0, p, 0.1, 0, 10, p, stream) == lib.ERR_INVALID_ARG


def _lmax(s):
    import oracle

    A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
    return oracle.lambda_max(A, s.y)
