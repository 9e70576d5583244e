"""Grids beyond the on-chip kernel (up to 1024 x 1024) and the FP64 solve path, against the
FP64 oracle; at 1024 x 1024 the oracle is evaluated on sampled outputs."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_parity, gpu_run, oracle_run, rel_err

pytestmark = pytest.mark.gpu


def _snap(seed, M1, M2, N, L1, L2, K=3, snr=15.0, lam_frac=0.1):
    s = synth.make_snapshot(seed, M1, M2, N, L1, L2, K, snr)
    s.lam_frac = lam_frac
    return s


@pytest.mark.parametrize("algo", ["ista", "fista", "admm"])
@pytest.mark.parametrize("L1,L2", [(512, 32), (32, 512), (1024, 16), (512, 128)])
def test_multipass_fp32_matches_oracle(lib, algo, L1, L2):
    M1, M2 = max(2, L1 // 16), max(2, L2 // 8)
    s = _snap(11 * L1 + L2, M1, M2, max(4, (M1 * M2) // 4), L1, L2)
    ref = oracle_run(s, algo, 120, rho=8.0)
    run = gpu_run(lib, [s], [ref["lam"]], algo, 120, rho=8.0)
    assert_parity(run["c"][0], ref, what=f"{algo} {L1}x{L2} multipass")


@pytest.mark.parametrize("algo", ["ista", "fista", "admm"])
@pytest.mark.parametrize("L1,L2", [(32, 32), (64, 16), (256, 64), (16, 512)])
def test_fp64_path_matches_oracle_to_1e10(lib, algo, L1, L2):
    """The complex128 path (complex128 y in, complex128 c out) agrees with the dense FP64 oracle to
    1e-10 relative: the two differ only in the order of FP64 rounding (Table I's eps_r is at
    1e-14..1e-9 for the same comparison)."""
    M1, M2 = max(2, L1 // 4), max(2, L2 // 4)
    s = _snap(7 * L1 + 3 * L2, M1, M2, max(4, (M1 * M2) // 3), L1, L2)
    ref = oracle_run(s, algo, 200, rho=4.0)
    run = gpu_run(lib, [s], [ref["lam"]], algo, 200, rho=4.0, prec="f64")
    assert run["c"][0].dtype == np.complex128
    err = rel_err(run["c"][0], ref["c"])
    assert err <= 1e-10, (algo, L1, L2, err)
    assert np.array_equal(np.abs(run["c"][0]) > 0, np.abs(ref["c"]) > 0)
    if algo == "admm":
        assert rel_err(run["aux"][0], ref["aux"]) <= 1e-10


@pytest.mark.parametrize("algo", ["ista", "fista", "admm"])
@pytest.mark.parametrize("L1,L2,M1,M2", [(8, 8, 12, 10), (8, 32, 12, 6), (64, 8, 10, 4), (8, 1024, 5, 40)])
def test_side_of_8_runs_multipass(lib, algo, L1, L2, M1, M2):
    """Grids with a side of 8 (below the fused kernel's radix-16 stages) run on the multi-pass
    solver, FP32 to the parity bar and FP64 to 1e-10; masks wider than the grid fold (M_i > L_i)."""
    s = _snap(9 * L1 + L2, M1, M2, max(4, (M1 * M2) // 3), L1, L2, K=2)
    ref = oracle_run(s, algo, 150, rho=4.0)
    run = gpu_run(lib, [s], [ref["lam"]], algo, 150, rho=4.0)
    assert lib.bccb_batch_variant(run["solver"].handle, L1, L2) == (0, 0)  # not the on-chip kernel
    assert_parity(run["c"][0], ref, what=f"{algo} {L1}x{L2} fp32")
    run64 = gpu_run(lib, [s], [ref["lam"]], algo, 150, rho=4.0, prec="f64")
    assert rel_err(run64["c"][0], ref["c"]) <= 1e-10
    assert np.array_equal(np.abs(run64["c"][0]) > 0, np.abs(ref["c"]) > 0)


def test_ragged_batch_mixing_on_chip_and_multipass(lib):
    snaps = [_snap(71, 8, 8, 20, 64, 64), _snap(72, 16, 4, 20, 512, 32), _snap(73, 8, 8, 20, 256, 256),
             _snap(74, 4, 16, 20, 16, 1024), _snap(75, 6, 6, 12, 8, 16)]
    refs = [oracle_run(s, "fista", 100) for s in snaps]
    run = gpu_run(lib, snaps, [r["lam"] for r in refs], "fista", 100)
    for i, (c, r) in enumerate(zip(run["c"], refs)):
        assert_parity(c, r, what=f"mixed batch {i}")


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_1024x1024_two_ista_iterations_sampled(lib, prec):
    """Full 1024 x 1024 grid, 64 x 64 array with N = 1024 (the precision-study shape): two ISTA
    iterations from zero, checked at sampled grid cells.  The oracle forms b = A^H y from the
    Kronecker factors of D, c1 = S(mu b) exactly, and c2 = S(c1 - mu A^H A c1 + mu b) at the sampled cells from the
    columns on c1's support."""
    s = synth.workload_snapshot("admm1024", 0)
    L = s.L1 * s.L2
    b = oracle.adjoint_measurements_kron(s.mask, s.M1, s.M2, s.L1, s.L2, s.y)
    mu = 1.0 / L  # sigma_max(A)^2 = L1 L2: rows of the partial DFT are orthogonal (M_i <= L_i)
    lam = 0.05 * np.abs(b).max()
    c1 = oracle.soft_threshold(mu * b, mu * lam)
    supp = np.flatnonzero(c1)
    A_s = oracle.dictionary_columns(s.mask, s.M1, s.M2, s.L1, s.L2, supp)
    r = A_s @ c1[supp]  # A c1
    rng = np.random.default_rng(0)
    cells = np.unique(np.concatenate([rng.choice(L, 2000, replace=False), supp[:500],
                                      np.argsort(-np.abs(b))[:200]]))
    A_c = oracle.dictionary_columns(s.mask, s.M1, s.M2, s.L1, s.L2, cells)
    u2 = c1[cells] - mu * (A_c.conj().T @ r) + mu * b[cells]
    c2 = oracle.soft_threshold(u2, mu * lam)
    tol = 1e-10 if prec == "f64" else 1e-5
    for iters, ref in ((1, c1[cells]), (2, c2)):
        run = gpu_run(lib, [s], [lam], "ista", iters, check=False, prec=prec)
        got = run["c"][0][cells]
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (prec, iters, np.abs(got - ref).max())


def test_1024x1024_admm_fp32_vs_fp64_paths(lib):
    """Precision study at full size (64 x 64 array, N = 1024, 1024 x 1024 grid, 20 off-grid sources,
    15 dB, ADMM rho = 0.5): the FP32 path against the FP64 path after 300 iterations, both returned
    iterates and the FP64 KKT residuals."""
    s = synth.workload_snapshot("admm1024", 0)
    # lam as a fraction of ||A^H y||_inf is applied on the device by both paths
    r32 = gpu_run_frac(lib, s, "f32")
    r64 = gpu_run_frac(lib, s, "f64")
    c32, c64 = r32["c"], r64["c"]
    if np.linalg.norm(c64) > 0:
        assert rel_err(c32, c64) <= 1e-4, rel_err(c32, c64)
    else:
        assert np.count_nonzero(c32) == 0
    assert rel_err(r32["aux"], r64["aux"]) <= 1e-4
    assert abs(r32["kkt"] - r64["kkt"]) <= 1e-3 * max(1.0, r64["kkt"])


def gpu_run_frac(lib, s, prec, iters=300):
    import torch

    from gpu_util import inst

    solver = lib.BatchSolver([inst(s, 0.05, lam_is_frac=True)], "admm", 0.5, prec=prec)
    cdt = torch.complex128 if prec == "f64" else torch.complex64
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=cdt, device="cuda")
    aux = torch.zeros_like(c)
    solver.solve(y, iters, c, aux_out=aux, check=True)
    res = solver.results()
    out = dict(c=c.cpu().numpy().astype(np.complex128), aux=aux.cpu().numpy().astype(np.complex128),
               kkt=float(res["kkt"][0]))
    solver.close()
    return out


@pytest.mark.parametrize("L1,L2,M1,M2,N,seed", [(512, 512, 32, 32, 256, 31), (1024, 1024, 64, 64, 1024, 41)])
def test_multipass_fista_1000_iterations_against_oracle(lib, L1, L2, M1, M2, N, seed):
    """FISTA x 1000 on grids beyond the on-chip kernel, FP32: the multi-pass solver keeps its state in
    compensated form as the fused kernel does (plain FP32 state drifted to 2e-4 at 1024 x 1024).  The
    oracle applies D through its Kronecker factors (A would be 2 or 16 GiB)."""
    s = synth.make_snapshot(seed, M1, M2, N, L1, L2, 8, 10.0)
    y32 = s.y.astype(np.complex64).astype(np.complex128)  # what the FP32 path is given
    K = oracle.KronDictionary(s.mask, M1, M2, L1, L2)
    lam = 0.05 * float(np.abs(K.adjoint(y32)).max())
    c_ref, u, kappa = oracle.fista_kron(K, y32, lam, 1000, pre=True)
    run = gpu_run(lib, [s], [lam], "fista", 1000, check=False)
    assert_parity(run["c"][0], dict(c=c_ref, u=u, kappa=kappa), what=f"FISTA {L1}x{L2} x1000 multipass")
