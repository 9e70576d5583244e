"""Pins for the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle through a route other than its own code: the
signal model of Section II-A, the BCCB structure and eigenvalues of Section
III-A, the FFT identity of Section III-B computed with numpy.fft, Table I's
dense-versus-FFT agreement, closed-form LASSO solutions, an independent
coordinate-descent solver, a direct dense solve for the ADMM inverse, and
finite differences for the unrolled network.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_problem(seed=1, M1=5, M2=3, N=9, L1=8, L2=16, K=2, snr=None, on_grid=True):
    s = synth.make_snapshot(seed, M1, M2, N, L1, L2, K, snr, on_grid=on_grid, unit_amplitude=True)
    A = oracle.dictionary(s.mask, M1, M2, L1, L2)
    return s, A


# ------------------------------------------------------------------------------------------
# Dictionary against the signal model (Section II-A)
# ------------------------------------------------------------------------------------------


@pytest.mark.parametrize("M1,M2,L1,L2", [(5, 3, 8, 16), (4, 7, 32, 8), (6, 6, 16, 16)])
def test_dictionary_reproduces_noiseless_on_grid_snapshot(M1, M2, L1, L2):
    """A c_true equals the synthetic snapshot for on-grid sources (eq:signal_model vs
    eq:sparse_forward_model); a transposed index, wrong sign or wrong grid fails here."""
    s = synth.make_snapshot(11, M1, M2, min(M1 * M2, 10), L1, L2, 3, None, on_grid=True)
    A = oracle.dictionary(s.mask, M1, M2, L1, L2)
    c = np.zeros(L1 * L2, np.complex128)
    l1 = np.rint((s.freqs[:, 0] + 0.5) * L1).astype(int)
    l2 = np.rint((s.freqs[:, 1] + 0.5) * L2).astype(int)
    c[l1 + l2 * L1] = s.amps
    np.testing.assert_allclose(A @ c, s.y, rtol=0, atol=1e-12)


# ------------------------------------------------------------------------------------------
# BCCB structure (Section III-A, eq:bccb_sum, eq:diagonalization, eq:lambda)
# ------------------------------------------------------------------------------------------


@pytest.mark.parametrize("M1,M2,L1,L2", [(5, 3, 8, 16), (3, 4, 4, 8), (9, 2, 8, 4)])
def test_gram_is_bccb_bruteforce(M1, M2, L1, L2):
    """Every entry of the dense A^H A depends only on the cyclic 2D lag (BCCB), including
    a mask wider than the grid (M1 > L1), where positions fold."""
    rng = np.random.default_rng(3)
    mask = synth.make_mask(rng, M1, M2, max(2, (M1 * M2) // 2))
    A = oracle.dictionary(mask, M1, M2, L1, L2)
    G = A.conj().T @ A
    r = G[:, 0].reshape(L2, L1)
    for l in range(L1 * L2):
        for lp in range(L1 * L2):
            d1 = ((l % L1) - (lp % L1)) % L1
            d2 = ((l // L1) - (lp // L1)) % L2
            assert abs(G[l, lp] - r[d2, d1]) < 1e-10


@pytest.mark.parametrize("M1,M2,L1,L2", [(5, 3, 8, 16), (16, 16, 64, 32), (9, 6, 8, 4)])
def test_eigenvalues_closed_form(M1, M2, L1, L2):
    """eq:lambda applied to the first column gives L1*L2 times the number of kept elements
    with (m1, m2) = (p1, p2) modulo (L1, L2): a real, non-negative grid."""
    rng = np.random.default_rng(5)
    mask = synth.make_mask(rng, M1, M2, max(3, (M1 * M2) // 3))
    A = oracle.dictionary(mask, M1, M2, L1, L2)
    lam = oracle.gram_eigenvalues(A, L1, L2)
    m1, m2 = oracle.element_positions(mask, M1)
    count = np.zeros((L2, L1))
    np.add.at(count, (m2 % L2, m1 % L1), 1.0)
    np.testing.assert_allclose(lam, L1 * L2 * count, rtol=0, atol=1e-9 * L1 * L2)


def test_gram_product_equals_2d_fft_identity():
    """R c = vec(F^-1 (Omega . F C F^T) F^-T) (eq:Rc), computed here with numpy.fft."""
    s, A = _small_problem(M1=6, M2=5, N=14, L1=16, L2=8)
    lam = oracle.gram_eigenvalues(A, 16, 8)
    rng = np.random.default_rng(9)
    x = rng.standard_normal(128) + 1j * rng.standard_normal(128)
    dense = A.conj().T @ (A @ x)
    fast = np.fft.ifft2(lam * np.fft.fft2(x.reshape(8, 16))).reshape(-1)
    np.testing.assert_allclose(dense, fast, rtol=0, atol=1e-11 * np.abs(dense).max())


def test_rows_orthogonal_and_step_size():
    """With M_i <= L_i the rows of the partial 2D DFT are orthogonal: A A^H = L1 L2 I, so
    sigma_max^2 = L1 L2 and mu = 1/(L1 L2) (eq:ista)."""
    s, A = _small_problem(M1=7, M2=5, N=20, L1=16, L2=8)
    np.testing.assert_allclose(A @ A.conj().T, 128 * np.eye(20), atol=1e-10)
    assert abs(oracle.step_size(A) - 1.0 / 128) < 1e-15


def test_step_size_with_folding_is_top_eigenvalue():
    """With folding (M1 > L1) sigma_max^2 = max Omega, the largest BCCB eigenvalue."""
    rng = np.random.default_rng(2)
    mask = synth.make_mask(rng, 9, 3, 20)
    A = oracle.dictionary(mask, 9, 3, 4, 4)
    lam = oracle.gram_eigenvalues(A, 4, 4).real
    assert abs(oracle.step_size(A) * lam.max() - 1.0) < 1e-12
    assert abs(oracle.step_size(A) - 1.0 / np.linalg.norm(A, 2) ** 2) < 1e-12


# ------------------------------------------------------------------------------------------
# Soft threshold (eq:ista)
# ------------------------------------------------------------------------------------------


def test_soft_threshold_cases():
    u = np.array([0.0, 0.5, -2.0, 3j, 1 + 1j, 0.3 - 0.4j, 0.5 + 0j])
    out = oracle.soft_threshold(u, 0.5)
    exp = np.array([0, 0, -1.5, 2.5j, (1 + 1j) / np.sqrt(2) * (np.sqrt(2) - 0.5), 0, 0])
    np.testing.assert_allclose(out, exp, atol=1e-15)
    assert np.all(oracle.soft_threshold(u, 0.0) == u)


# ------------------------------------------------------------------------------------------
# Closed-form LASSO solutions and special cases
# ------------------------------------------------------------------------------------------


def test_lambda_zero_ista_reaches_min_norm_solution_in_one_step():
    """lam = 0: from c0 = 0, c1 = mu A^H y = A^H y/(L1 L2) = A^+ y (rows orthogonal);
    it interpolates y exactly and is a fixed point."""
    s, A = _small_problem(snr=10.0)
    c1 = oracle.ista(A, s.y, 0.0, 1)
    np.testing.assert_allclose(A @ c1, s.y, atol=1e-11)
    np.testing.assert_allclose(c1, np.linalg.pinv(A) @ s.y, atol=1e-12)
    c3 = oracle.ista(A, s.y, 0.0, 3)
    np.testing.assert_allclose(c3, c1, atol=1e-12)


@pytest.mark.parametrize("algo", ["ista", "fista", "admm"])
def test_single_on_grid_source_closed_form(algo):
    """One noiseless on-grid source a at column l*: the LASSO minimiser is
    c = e_{l*} a (1 - lam/(N|a|))_+ because |G(i, l*)| <= N = G(l*, l*)."""
    M1, M2, L1, L2, N = 6, 5, 16, 8, 12
    s = synth.make_snapshot(21, M1, M2, N, L1, L2, 1, None, on_grid=True, unit_amplitude=False)
    A = oracle.dictionary(s.mask, M1, M2, L1, L2)
    a = s.amps[0]
    lstar = int(round((s.freqs[0, 0] + 0.5) * L1)) + L1 * int(round((s.freqs[0, 1] + 0.5) * L2))
    lam = 0.3 * N * abs(a)
    exp = np.zeros(L1 * L2, np.complex128)
    exp[lstar] = a * (1 - lam / (N * abs(a)))
    if algo == "ista":
        c = oracle.ista(A, s.y, lam, 3000)
    elif algo == "fista":
        c = oracle.fista(A, s.y, lam, 600)
    else:
        c = oracle.admm(A, s.y, lam, 8.0, 600)[0]
    np.testing.assert_allclose(c, exp, atol=1e-8)


def _cd_lasso(A, y, lam, sweeps=4000):
    """Independent complex LASSO solver (cyclic coordinate descent) for tiny problems."""
    L = A.shape[1]
    c = np.zeros(L, np.complex128)
    norms = np.sum(np.abs(A) ** 2, axis=0)
    r = y.astype(np.complex128).copy()
    for _ in range(sweeps):
        for i in range(L):
            r = r + A[:, i] * c[i]
            rho = np.vdot(A[:, i], r)
            mag = abs(rho)
            c[i] = 0 if mag <= lam else rho / mag * (mag - lam) / norms[i]
            r = r - A[:, i] * c[i]
    return c


def test_all_solvers_match_coordinate_descent_and_kkt():
    """ISTA, FISTA and ADMM run long reach the coordinate-descent minimiser of the
    1/2-scaled LASSO, and the KKT conditions hold there."""
    s, A = _small_problem(seed=4, M1=4, M2=3, N=7, L1=4, L2=4, K=2, snr=15.0, on_grid=False)
    lam = 0.2 * oracle.lambda_max(A, s.y)
    ref = _cd_lasso(A, s.y, lam)
    c_i = oracle.ista(A, s.y, lam, 20000)
    c_f = oracle.fista(A, s.y, lam, 3000)
    z_a, c_a, _ = oracle.admm(A, s.y, lam, 1.0, 5000)
    for c in (c_i, c_f, z_a, c_a):
        np.testing.assert_allclose(c, ref, atol=1e-7)
        assert oracle.kkt_residual(A, s.y, c if c is not c_a else z_a, lam) < 1e-6
    f_ref = oracle.objective(A, s.y, ref, lam)
    assert abs(oracle.objective(A, s.y, c_f, lam) - f_ref) < 1e-10 * max(1.0, f_ref)


def test_admm_threshold_reading_changes_answer_for_rho_not_one():
    """kappa_2 = lam/rho gives the LASSO minimiser for any rho (reading of eq:admm); the
    literal rho*lam would not for rho = 0.5, so the test pins the reading."""
    s, A = _small_problem(seed=8, M1=4, M2=4, N=9, L1=8, L2=4, K=2, snr=20.0, on_grid=False)
    lam = 0.15 * oracle.lambda_max(A, s.y)
    ref = _cd_lasso(A, s.y, lam)
    z, _, _ = oracle.admm(A, s.y, lam, 0.5, 6000)
    np.testing.assert_allclose(z, ref, atol=1e-7)


def test_ista_objective_monotone():
    """ISTA with step 1/sigma_max^2 never increases the objective."""
    s, A = _small_problem(seed=6, M1=8, M2=8, N=20, L1=16, L2=16, K=3, snr=10.0, on_grid=False)
    lam = 0.1 * oracle.lambda_max(A, s.y)
    _, hist = oracle.ista(A, s.y, lam, 200, history=True)
    f = [oracle.objective(A, s.y, c, lam) for c in hist]
    assert all(f[t + 1] <= f[t] * (1 + 1e-13) + 1e-13 for t in range(len(f) - 1))


def test_fista_first_steps_and_rate():
    """With alpha_1 = 1 the first momentum weight is 0, so FISTA's c^(1), c^(2) equal ISTA's
    and c^(3) differs; F(c^(t)) - F* <= 2 ||c0 - c*||^2 / (mu (t+1)^2) (Beck-Teboulle)."""
    s, A = _small_problem(seed=7, M1=8, M2=8, N=24, L1=16, L2=8, K=3, snr=10.0, on_grid=False)
    lam = 0.1 * oracle.lambda_max(A, s.y)
    _, hi = oracle.ista(A, s.y, lam, 3, history=True)
    _, hf = oracle.fista(A, s.y, lam, 400, history=True)
    np.testing.assert_allclose(hf[1], hi[1], atol=1e-15)
    np.testing.assert_allclose(hf[2], hi[2], atol=1e-15)
    assert np.abs(hf[3] - hi[3]).max() > 1e-6
    beta = oracle.fista_momentum(50)
    assert beta[0] == 0.0 and np.all(np.diff(beta) > 0) and beta[-1] < 1
    c_star = oracle.fista(A, s.y, lam, 20000)
    f_star = oracle.objective(A, s.y, c_star, lam)
    mu = oracle.step_size(A)
    bound_c = np.vdot(c_star, c_star).real
    for t in range(1, 400):
        gap = oracle.objective(A, s.y, hf[t], lam) - f_star
        assert gap <= 2 * bound_c / (mu * (t + 1) ** 2) + 1e-9


def test_admm_inverse_matches_direct_dense_solve():
    """The Woodbury application of (A^H A + rho I)^{-1} equals a direct L x L solve."""
    s, A = _small_problem(M1=5, M2=3, N=9, L1=8, L2=4)
    rng = np.random.default_rng(1)
    w = rng.standard_normal(32) + 1j * rng.standard_normal(32)
    for rho in (0.5, 1.0, 3.0):
        direct = np.linalg.solve(A.conj().T @ A + rho * np.eye(32), w)
        np.testing.assert_allclose(oracle.admm_c_update(A, rho)(w), direct, atol=1e-12)


def test_shift_equivariance():
    """Modulating every measurement by exp(-j 2 pi m1/L1) (all harmonics move one grid step
    in f1) cyclically shifts the LASSO iterates by one in l1 (columns of A satisfy
    col(l1+1) = diag(exp(-j 2 pi m1/L1)) col(l1))."""
    M1, M2, L1, L2 = 6, 4, 16, 8
    s = synth.make_snapshot(31, M1, M2, 15, L1, L2, 3, 12.0)
    A = oracle.dictionary(s.mask, M1, M2, L1, L2)
    m1, _ = oracle.element_positions(s.mask, M1)
    y2 = s.y * np.exp(-2j * np.pi * m1 / L1)
    lam = 0.1 * oracle.lambda_max(A, s.y)
    for solve in (lambda y: oracle.fista(A, y, lam, 60), lambda y: oracle.admm(A, y, lam, 1.0, 60)[0]):
        c1 = solve(s.y).reshape(L2, L1)
        c2 = solve(y2).reshape(L2, L1)
        np.testing.assert_allclose(c2, np.roll(c1, 1, axis=1), atol=1e-11)


def test_noiseless_on_grid_sources_are_the_largest_peaks():
    """Config-1-shaped problem without noise: the K largest |c| sit on the true grid cells."""
    s = synth.workload_snapshot("fista64", 0, snr_db=None)
    A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
    lam = 0.1 * oracle.lambda_max(A, s.y)
    c = oracle.fista(A, s.y, lam, 500)
    l1 = np.rint((s.freqs[:, 0] + 0.5) * s.L1).astype(int)
    l2 = np.rint((s.freqs[:, 1] + 0.5) * s.L2).astype(int)
    top = set(np.argsort(-np.abs(c))[: len(l1)].tolist())
    assert top == set((l1 + l2 * s.L1).tolist())


# ------------------------------------------------------------------------------------------
# Table I: dense and FFT implementations agree to FP64 rounding
# ------------------------------------------------------------------------------------------


def _table1():
    rows = {}
    with open(os.path.join(GOLDEN, "table1_eps_r.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                algo, it, l1, eps = line.split()
                rows[(algo, int(it), int(l1))] = float(eps)
    return rows


def _fft_solver(s, lam, algo, iters, rho=1.0):
    """The paper's fast implementation written from eq:Rc with numpy.fft (test-only)."""
    L1, L2 = s.L1, s.L2
    m1, m2 = oracle.element_positions(s.mask, s.M1)
    count = np.zeros((L2, L1))
    np.add.at(count, (m2 % L2, m1 % L1), 1.0)
    lam_grid = L1 * L2 * count
    grid = np.zeros((L2, L1), np.complex128)
    np.add.at(grid, (m2 % L2, m1 % L1), (-1.0) ** (m1 + m2) * s.y)
    b = (L1 * L2) * np.fft.ifft2(grid)
    mu = 1.0 / lam_grid.max()
    gram = lambda x: np.fft.ifft2(lam_grid * np.fft.fft2(x))
    S = lambda u, k: oracle.soft_threshold(u.reshape(-1), k).reshape(L2, L1)
    if algo == "ista":
        c = np.zeros((L2, L1), np.complex128)
        for _ in range(iters):
            c = S(c - mu * gram(c) + mu * b, mu * lam)
        return c.reshape(-1)
    if algo == "fista":
        beta = oracle.fista_momentum(iters)
        c_prev = np.zeros((L2, L1), np.complex128)
        z = c_prev.copy()
        for t in range(iters):
            c = S(z - mu * gram(z) + mu * b, mu * lam)
            z = c + beta[t] * (c - c_prev)
            c_prev = c
        return c.reshape(-1)
    inv = lambda x: np.fft.ifft2(np.fft.fft2(x) / (lam_grid + rho))
    d = inv(b)
    z = np.zeros((L2, L1), np.complex128)
    v = np.zeros_like(z)
    for _ in range(iters):
        c = d + rho * inv(z - v)
        zn = S(c + v, lam / rho)
        v = v + c - zn
        z = zn
    return z.reshape(-1)


@pytest.mark.parametrize("algo", ["ista", "fista", "admm"])
@pytest.mark.parametrize("L1", [64, 128])
def test_table1_dense_vs_fft_agree_to_fp64_rounding(algo, L1):
    """On the paper's workload the dense oracle and an FFT implementation agree to within
    ten times the eps_r of Table I (Section III-C) after 50 and 100 iterations."""
    table = _table1()
    for trial in range(2):
        s = synth.paper_experiment_snapshot(trial, L1)
        A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
        lam = 0.1 * oracle.lambda_max(A, s.y)
        for iters in (50, 100):
            if algo == "ista":
                ref = oracle.ista(A, s.y, lam, iters)
            elif algo == "fista":
                ref = oracle.fista(A, s.y, lam, iters)
            else:
                # The paper gives no rho; rho = N (the Gram diagonal) keeps z nonzero within
                # 50 iterations, where rho = 1 leaves it at exactly 0 on this workload.
                ref = oracle.admm(A, s.y, lam, float(s.N), iters)[0]
            fast = _fft_solver(s, lam, algo, iters, rho=float(s.N))
            assert np.linalg.norm(ref) > 0
            eps = np.linalg.norm(ref - fast) / np.linalg.norm(ref)
            assert eps <= 10 * table[(algo, iters, L1)], (trial, iters, eps)


# ------------------------------------------------------------------------------------------
# Unrolled FISTA: analytic backward against central finite differences
# ------------------------------------------------------------------------------------------


def test_unrolled_backward_matches_finite_differences():
    s, A = _small_problem(seed=12, M1=5, M2=4, N=12, L1=8, L2=8, K=2, snr=15.0, on_grid=False)
    K = 5
    lam = 0.1 * oracle.lambda_max(A, s.y)
    mu0 = oracle.step_size(A)
    rng = np.random.default_rng(0)
    mu = mu0 * (0.7 + 0.5 * rng.random(K))
    th = mu0 * lam * (0.5 + rng.random(K))
    target = oracle.fista(A, s.y, lam, 300)

    def loss(m, t):
        c = oracle.unrolled_forward(A, s.y, m, t)
        return float(np.sum(np.abs(c - target) ** 2))

    c = oracle.unrolled_forward(A, s.y, mu, th)
    d_mu, d_th = oracle.unrolled_backward(A, s.y, mu, th, 2.0 * (c - target))
    for k in range(K):
        h = 1e-6 * mu[k]
        e = np.zeros(K)
        e[k] = h
        fd = (loss(mu + e, th) - loss(mu - e, th)) / (2 * h)
        assert abs(fd - d_mu[k]) <= 1e-5 * max(1.0, abs(fd)), (k, fd, d_mu[k])
        h = 1e-6 * th[k]
        e = np.zeros(K)
        e[k] = h
        fd = (loss(mu, th + e) - loss(mu, th - e)) / (2 * h)
        assert abs(fd - d_th[k]) <= 1e-5 * max(1.0, abs(fd)), (k, fd, d_th[k])


def test_unrolled_grad_y_matches_finite_differences():
    """dLoss/dy of the unrolled network (thresholds fixed) against central differences on the
    real and imaginary part of every measurement."""
    s, A = _small_problem(seed=13, M1=4, M2=4, N=9, L1=8, L2=8, K=2, snr=15.0, on_grid=False)
    K = 4
    lam = 0.1 * oracle.lambda_max(A, s.y)
    mu0 = oracle.step_size(A)
    rng = np.random.default_rng(1)
    mu = mu0 * (0.7 + 0.5 * rng.random(K))
    th = mu0 * lam * (0.5 + rng.random(K))
    target = oracle.fista(A, s.y, lam, 200)

    def loss(y):
        c = oracle.unrolled_forward(A, y, mu, th)
        return float(np.sum(np.abs(c - target) ** 2))

    c = oracle.unrolled_forward(A, s.y, mu, th)
    _, _, g_y = oracle.unrolled_backward(A, s.y, mu, th, 2.0 * (c - target), want_grad_y=True)
    h = 1e-7 * np.abs(s.y).max()
    for n in range(s.y.size):
        for unit in (1.0, 1j):
            e = np.zeros(s.y.size, np.complex128)
            e[n] = h * unit
            fd = (loss(s.y + e) - loss(s.y - e)) / (2 * h)
            got = g_y[n].real if unit == 1.0 else g_y[n].imag
            assert abs(fd - got) <= 1e-5 * max(1.0, abs(fd)), (n, unit, fd, got)


def test_column_and_kronecker_helpers_match_dense_dictionary():
    """The large-grid helpers (selected columns, b from the Kronecker factors) equal the dense
    construction on grids where both fit."""
    s, A = _small_problem(seed=13, M1=6, M2=5, N=17, L1=16, L2=32)
    cols = np.array([0, 1, 31, 200, 511])
    np.testing.assert_allclose(oracle.dictionary_columns(s.mask, 6, 5, 16, 32, cols), A[:, cols], atol=1e-13)
    np.testing.assert_allclose(oracle.adjoint_measurements_kron(s.mask, 6, 5, 16, 32, s.y), A.conj().T @ s.y,
                               atol=1e-12)
