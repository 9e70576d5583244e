"""Parity of the dense ("regular") iteration engine, which applies the stored L x L
Gram matrix every iteration (eq:ista, eq:fista, eq:admm), with the FP64 oracle, on the
paper's experiment shape (Section III-C) and on small grids."""
import numpy as np
import pytest

from gpu_util import REL_TOL, assert_parity, inst, oracle_run
import synth

pytestmark = pytest.mark.gpu


def _run(lib, snaps, lams, algo, iters, rho=1.0, method="dense", capture=False):
    import torch

    stream = torch.cuda.Stream()
    solver = lib.BatchSolver([inst(s, l) for s, l in zip(snaps, lams)], algo, rho, stream=stream)
    solver.set_method(method)
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    aux = torch.zeros_like(c) if algo == "admm" else None
    if capture:
        lib.bccb_batch_capture(solver.handle, y, iters, None, c, aux, True)
        lib.bccb_batch_replay(solver.handle)
    else:
        solver.solve(y, iters, c, aux_out=aux, check=True)
    torch.cuda.synchronize()
    res = solver.results()
    out = [g.reshape(-1) for g in solver.unpack(c.cpu().numpy())]
    aux_out = None if aux is None else [g.reshape(-1) for g in solver.unpack(aux.cpu().numpy())]
    solver.close()
    return dict(c=out, aux=aux_out, res=res)


@pytest.mark.parametrize("algo", ["ista", "fista", "admm"])
@pytest.mark.parametrize("L1", [64, 256, 512])
def test_dense_paper_shape(lib, algo, L1):
    """M1=51, M2=16, N=40, L2=32, 15 dB, 200 iterations; ADMM with rho = N."""
    s = synth.paper_experiment_snapshot(1, L1)
    rho = float(s.N)
    ref = oracle_run(s, algo, 200, rho=rho)
    run = _run(lib, [s], [ref["lam"]], algo, 200, rho=rho)
    assert_parity(run["c"][0], ref, what=f"dense {algo} {L1}x32")
    if algo == "admm":
        ratio = np.linalg.norm(ref["u"] - ref["aux"]) / np.linalg.norm(ref["aux"])
        tol = max(REL_TOL, 16 * 2.0**-24 * ratio)
        assert_parity(run["aux"][0], ref, ref_c=ref["aux"], tol=tol, what="dense admm c^(T)")


def test_dense_ragged_batch_and_fold(lib):
    """Two shapes in one batch, one of them with a mask wider than its grid (M1 > L1:
    the Gram folds; FISTA's mu then comes from max Lambda, not from L)."""
    snaps = [synth.make_snapshot(31, 12, 6, 30, 64, 32, K=3, snr_db=20.0),
             synth.make_snapshot(32, 40, 5, 60, 32, 16, K=2, snr_db=25.0)]
    refs = [oracle_run(s, "fista", 150) for s in snaps]
    run = _run(lib, snaps, [r["lam"] for r in refs], "fista", 150)
    for i, (s, r) in enumerate(zip(snaps, refs)):
        assert_parity(run["c"][i], r, what=f"dense fista instance {i}")


def test_dense_matches_fft_engine_and_capture(lib):
    s = synth.paper_experiment_snapshot(2, 128)
    ref = oracle_run(s, "fista", 300)
    dense = _run(lib, [s], [ref["lam"]], "fista", 300)
    fft = _run(lib, [s], [ref["lam"]], "fista", 300, method="fft")
    cap = _run(lib, [s], [ref["lam"]], "fista", 300, capture=True)
    for r in (dense, fft, cap):
        assert_parity(r["c"][0], ref, what="fista 128x32")
    assert np.array_equal(cap["c"][0], dense["c"][0])  # same kernels, same order
    assert dense["res"]["kkt"][0] == pytest.approx(fft["res"]["kkt"][0], abs=1e-4)


def test_dense_unsupported_cases(lib):
    import torch

    s = synth.make_snapshot(41, 40, 5, 60, 32, 16, K=2, snr_db=25.0)  # M1 > L1
    solver = lib.BatchSolver([inst(s, 0.1, True)], "admm", 1.0)
    with pytest.raises(lib.BccbError):
        solver.set_method("dense")  # ADMM needs D D^H = L I
    solver.close()
    solver = lib.BatchSolver([inst(s, 0.1, True)], "fista", prec="f64")
    with pytest.raises(lib.BccbError):
        solver.set_method("dense")  # complex64 only
    solver.close()
    solver = lib.BatchSolver([inst(s, 0.1, True)], "fista")
    solver.set_method("dense")
    solver.set_method("fft")  # and back
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    solver.solve(y, 10, c)
    solver.close()
