"""Element spacings gamma != 1/2: the Gram is block Toeplitz (Section III-A) and the CUDA
path iterates on its 2L1 x 2L2 circulant embedding.  Parity with the FP64 oracle built on
the same dictionary (eq:uniform_grid with the given gamma)."""
import numpy as np
import pytest

import oracle
from oracle import peaks as opk
from gpu_util import REL_TOL, assert_parity, gpu_run, inst, oracle_run, rel_err
import synth

pytestmark = pytest.mark.gpu

GAM = (0.35, 0.8)


def _snap(seed, M1, M2, N, L1, L2, gamma=GAM, K=3, snr=20.0):
    return synth.make_snapshot(seed, M1, M2, N, L1, L2, K=K, snr_db=snr, gamma=gamma)


def _A(s):
    return oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2, *s.gamma)


def _run(lib, snaps, lams, algo, iters, prec="f32", c0=None, check=True):
    import torch

    solver = lib.BatchSolver([inst(s, l) for s, l in zip(snaps, lams)], algo, prec=prec, gamma=snaps[0].gamma)
    cdt = torch.complex128 if prec == "f64" else torch.complex64
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=cdt, device="cuda")
    c0_t = None if c0 is None else torch.from_numpy(np.asarray(c0, solver.dtype)).cuda()
    solver.solve(y, iters, c, c0=c0_t, check=check)
    torch.cuda.synchronize()
    res = solver.results() if check else None
    out = [g.reshape(-1) for g in solver.unpack(c.cpu().numpy())]
    return dict(c=out, res=res, solver=solver, c_dev=c)


@pytest.mark.parametrize("algo", ["ista", "fista"])
@pytest.mark.parametrize("L1,L2,M1,M2", [(32, 32, 8, 8), (64, 16, 16, 6), (128, 128, 20, 20), (256, 64, 24, 10)])
def test_toeplitz_parity(lib, algo, L1, L2, M1, M2):
    s = _snap(100 + L1 + L2, M1, M2, max(4, (M1 * M2) // 3), L1, L2)
    A = _A(s)
    ref = oracle_run(s, algo, 150, A=A)
    run = _run(lib, [s], [ref["lam"]], algo, 150)
    assert_parity(run["c"][0], ref, what=f"toeplitz {algo} {L1}x{L2}")
    res = run["res"]
    assert res["mu"][0] == pytest.approx(oracle.step_size(A), rel=1e-12)
    # the check sees the complex64 measurements the solver was given
    c = run["c"][0].astype(np.complex128)
    y32 = s.y.astype(np.complex64).astype(np.complex128)
    assert res["kkt"][0] == pytest.approx(oracle.kkt_residual(A, y32, c, ref["lam"]), rel=1e-6, abs=1e-9)
    assert res["objective"][0] == pytest.approx(oracle.objective(A, y32, c, ref["lam"]), rel=1e-9)


def test_toeplitz_batch_mixed_shapes_and_fp64(lib):
    snaps = [_snap(201, 8, 8, 20, 32, 32), _snap(202, 12, 5, 25, 64, 16), _snap(203, 6, 12, 30, 16, 64)]
    refs = [oracle_run(s, "fista", 120, A=_A(s)) for s in snaps]
    run = _run(lib, snaps, [r["lam"] for r in refs], "fista", 120)
    for i, r in enumerate(refs):
        assert_parity(run["c"][i], r, what=f"toeplitz batch instance {i}")
    run64 = _run(lib, snaps, [r["lam"] for r in refs], "fista", 120, prec="f64")
    for i, r in enumerate(refs):
        err = rel_err(run64["c"][i], r["c"])
        assert err <= 1e-10, f"FP64 toeplitz instance {i}: {err:.2e}"


def test_toeplitz_warm_start_ista(lib):
    s = _snap(301, 10, 10, 30, 64, 64)
    A = _A(s)
    ref = oracle_run(s, "ista", 150, A=A)
    first = _run(lib, [s], [ref["lam"]], "ista", 100, check=False)
    second = _run(lib, [s], [ref["lam"]], "ista", 50, c0=first["c"][0])
    assert_parity(second["c"][0], ref, what="ista 100 + 50 from the warm start")


def test_half_wavelength_through_gamma_entry_is_identical(lib):
    import torch

    s = synth.make_snapshot(401, 16, 16, 60, 64, 64, K=3, snr_db=20.0)
    a = gpu_run(lib, [s], [0.1], "fista", 100, check=False)["c"][0]
    solver = lib.BatchSolver([inst(s, 0.1)], "fista", gamma=(0.5, 0.5))
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    solver.solve(y, 100, c, check=False)
    assert np.array_equal(c.cpu().numpy(), a)


def test_toeplitz_peaks_use_the_spacing(lib):
    s = _snap(501, 12, 12, 50, 64, 64, K=4, snr=30.0)
    A = _A(s)
    ref = oracle_run(s, "fista", 200, A=A)
    run = _run(lib, [s], [ref["lam"]], "fista", 200, check=False)
    out = run["solver"].peaks(run["c_dev"], 8, 0.05)
    got = {k: v.cpu().numpy()[0] for k, v in out.items()}
    exp = opk.peaks(run["c"][0].reshape(64, 64), 8, 0.05, *GAM)
    assert np.array_equal(got["idx"], exp["idx"]) and got["count"] == exp["count"]
    assert np.array_equal(got["harm"], exp["harm"], equal_nan=True)
    nan = np.isnan(exp["ang"])
    assert np.array_equal(np.isnan(got["ang"]), nan)
    assert np.allclose(got["ang"][~nan], exp["ang"][~nan], rtol=0, atol=1e-14)


def test_toeplitz_unsupported(lib):
    import torch

    s = _snap(601, 8, 8, 20, 32, 32)
    with pytest.raises(lib.BccbError):
        lib.BatchSolver([inst(s, 0.1, True)], "admm", gamma=GAM)
    wide = _snap(602, 40, 8, 60, 32, 32)  # M1 > L1
    with pytest.raises(lib.BccbError):
        lib.BatchSolver([inst(wide, 0.1, True)], "fista", gamma=GAM)
    solver = lib.BatchSolver([inst(s, 0.1, True)], "fista", gamma=GAM)
    with pytest.raises(lib.BccbError):
        solver.set_method("dense")
    with pytest.raises(lib.BccbError):
        solver.get(0, torch.zeros(solver.total_c, dtype=torch.float64, device="cuda"))


def test_toeplitz_cached_setup_and_tuner(lib):
    """The mask-only setup (embedding spectrum, mu) runs once per solver; later solves and
    the autotuner reuse it and give identical results."""
    import torch

    s = _snap(701, 12, 12, 50, 128, 128)
    A = _A(s)
    ref = oracle_run(s, "fista", 100, A=A)
    solver = lib.BatchSolver([inst(s, ref["lam"])], "fista", gamma=GAM)
    y = torch.from_numpy(solver.y_host).cuda()
    c1 = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    c2 = torch.zeros_like(c1)
    solver.solve(y, 100, c1)
    mu1 = solver.results()["mu"][0]
    lib.bccb_batch_tune(solver.handle, y, 5, None)
    solver.solve(y, 100, c2)
    assert solver.results()["mu"][0] == mu1 == pytest.approx(oracle.step_size(A), rel=1e-12)
    assert np.array_equal(c1.cpu().numpy(), c2.cpu().numpy())
    assert_parity(c2.cpu().numpy(), ref, what="toeplitz after tuning")


def test_toeplitz_host_buffers_and_graph_replay(lib):
    """The host-buffer entry point and a captured graph give the caller's L1 x L2 packing."""
    import torch

    snaps = [_snap(801, 8, 8, 20, 32, 32), _snap(802, 10, 6, 24, 64, 32)]
    refs = [oracle_run(s, "fista", 80, A=_A(s)) for s in snaps]
    lams = [r["lam"] for r in refs]
    stream = torch.cuda.Stream()
    solver = lib.BatchSolver([inst(s, l) for s, l in zip(snaps, lams)], "fista", stream=stream, gamma=GAM)
    out = np.zeros(solver.total_c, dtype=np.complex64)
    solver.solve_host(solver.y_host, 80, out)
    for i, r in enumerate(refs):
        assert_parity(solver.unpack(out)[i].reshape(-1), r, what=f"host buffers instance {i}")
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    lib.bccb_batch_capture(solver.handle, y, 80, None, c, None, True)
    lib.bccb_batch_replay(solver.handle)
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy(), out)
