"""Parity at the benchmark's full size and launch configuration: 4096 snapshots of the
256x256 workload (32x32 array, N = 256, 8 off-grid sources, 10 dB, lam = 0.05 ||A^H y||_inf),
FISTA x 1000 in one batched solve with the autotuned tile, captured and replayed as bench.py
times it.  The oracle solves 64 evenly spaced instances one by one; every one of them is held
to the parity bar (relative l2 error <= 1e-4, identical support apart from entries within
1e-5 of the threshold)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_parity, inst

pytestmark = pytest.mark.gpu

B, T = 4096, 1000
SAMPLES = tuple(range(0, B, B // 64))[:63] + (B - 1,)


def _snap(i):
    # the benchmark's generator: seed 20000 + instance
    return synth.make_snapshot(20000 + i, 32, 32, 256, 256, 256, 8, 10.0)


def test_full_size_batch_sampled_against_oracle(lib):
    import torch

    snaps = [_snap(i) for i in range(B)]
    stream = torch.cuda.Stream()
    solver = lib.BatchSolver([inst(s, 0.05, True) for s in snaps], "fista", stream=stream)
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    lib.bccb_batch_tune(solver.handle, y, 20, None)
    lib.bccb_batch_capture(solver.handle, y, T, None, c, None, True)
    lib.bccb_batch_replay(solver.handle)
    torch.cuda.synchronize()
    res = solver.results()
    grids = solver.unpack(c.cpu().numpy())
    assert np.all(np.isfinite(res["kkt"])) and np.all(res["kkt"] >= 0)
    errs = []
    for i in SAMPLES:
        s = snaps[i]
        A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
        lam = float(res["lam"][i])
        # both sides see the same measurements: the complex64 values the solver was given
        y32 = s.y.astype(np.complex64).astype(np.complex128)
        assert lam == pytest.approx(0.05 * oracle.lambda_max(A, y32), rel=1e-9)
        c_ref, u, kappa = oracle.fista(A, y32, lam, T, pre=True)
        got = grids[i].reshape(-1)
        errs.append(assert_parity(got, dict(c=c_ref, u=u, kappa=kappa), what=f"instance {i} of the full batch"))
        assert res["kkt"][i] == pytest.approx(oracle.kkt_residual(A, y32, got.astype(np.complex128), lam),
                                              rel=1e-6, abs=1e-9)
    print(f"relative errors over {len(errs)} instances: median {np.median(errs):.1e}, max {max(errs):.1e}")
