"""Dense FP64 oracle: sensing matrix, ISTA, FISTA, ADMM, KKT, unrolled FISTA.

Test infrastructure only (see the package docstring).  Every function follows a
passage of "Fast Single-Snapshot Harmonic Recovery with 2D Sparse Arrays using
BCCB Matrices" (arXiv 2509.13592) and is written as the plain definition, with
NumPy/SciPy primitives (matrix products, an eigenvalue routine, a Cholesky
factorisation) as its only building blocks.

Notation.  lam is the LASSO weight (the paper's tau), N the number of kept
elements (the paper's M), L = L1*L2.  The unknown c is a length-L vector whose
entry l1 + l2*L1 belongs to the harmonic pair (f_{1,l1}, f_{2,l2}) (Section
II-A); viewed as a grid it is an (L2, L1) row-major array.

Readings of the paper used here:
  * objective 1/2 ||y - A c||^2 + lam ||c||_1: the ISTA step with mu =
    1/sigma_max^2 and threshold mu*tau (eq:ista) is proximal gradient for the
    1/2-scaled data term;
  * the soft-threshold of eq:ista uses its subscript kappa as threshold; an
    input with |u| <= kappa maps to exactly 0;
  * FISTA starts with alpha_1 = 1 and z^(1) = c^(0), so the first momentum
    weight (alpha_1 - 1)/alpha_2 is 0 (Beck and Teboulle's indexing);
  * ADMM thresholds with kappa_2 = lam/rho: at an ADMM fixed point rho*v =
    A^H(y - A c) and v lies in kappa_2 * d||c||_1, so the LASSO optimality
    condition needs rho*kappa_2 = lam (equal to the printed rho*tau for rho=1);
    the solve returns z^(T), the exactly sparse iterate, and also c^(T), v^(T);
  * the rows of Psi follow ascending linear index m1 + m2*M1.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

# ------------------------------------------------------------------------------------------
# Dictionary (Section II-A)
# ------------------------------------------------------------------------------------------


def harmonic_grid(L: int, gamma: float = 0.5) -> np.ndarray:
    """Uniform harmonic grid f_l = -gamma + l*2*gamma/L (eq:uniform_grid); gamma is the element
    spacing in wavelengths (Section II-A), 1/2 for the BCCB case of Section III."""
    return -gamma + np.arange(L, dtype=np.float64) * (2.0 * gamma / L)


def element_positions(mask, M1: int):
    """(m1, m2) for the rows of Psi: kept elements in ascending m1 + m2*M1 (Section II-A)."""
    lin = np.flatnonzero(np.asarray(mask).reshape(-1))
    return lin % M1, lin // M1


def dictionary(mask, M1: int, M2: int, L1: int, L2: int, gamma1: float = 0.5, gamma2: float = 0.5) -> np.ndarray:
    """Row-subsampled dictionary D_s = Psi (D2 kron D1) in complex128, shape (N, L1*L2).

    D_i(m, l) = exp(-j 2 pi f_{i,l} m) (eq:subdictionary) on the grids of eq:uniform_grid
    with spacings gamma1, gamma2 (1/2: half-wavelength, the BCCB case); the row of D for
    element (m1, m2) is row m1 + m2*M1 of D2 kron D1, i.e. kron(D2[m2], D1[m1])
    (eq:forward_model, eq:sparse_forward_model).
    """
    m1, m2 = element_positions(mask, M1)
    if np.any(m1 >= M1) or np.any(m2 >= M2):
        raise ValueError("mask larger than M1*M2")
    D1 = np.exp(-2j * np.pi * np.outer(np.arange(M1), harmonic_grid(L1, gamma1)))
    D2 = np.exp(-2j * np.pi * np.outer(np.arange(M2), harmonic_grid(L2, gamma2)))
    A = np.empty((m1.size, L1 * L2), dtype=np.complex128)
    for n in range(m1.size):
        A[n] = np.kron(D2[m2[n]], D1[m1[n]])
    return A


def dictionary_columns(mask, M1: int, M2: int, L1: int, L2: int, cols) -> np.ndarray:
    """Columns `cols` (indices l1 + l2*L1) of D_s, shape (N, len(cols)): entry (n, l) =
    D1(m1_n, l1) D2(m2_n, l2) (eq:subdictionary, eq:forward_model), for grids too large to
    form whole."""
    m1, m2 = element_positions(mask, M1)
    cols = np.asarray(cols)
    l1, l2 = cols % L1, cols // L1
    f1, f2 = harmonic_grid(L1)[l1], harmonic_grid(L2)[l2]
    return np.exp(-2j * np.pi * np.outer(m1, f1)) * np.exp(-2j * np.pi * np.outer(m2, f2))


def adjoint_measurements_kron(mask, M1: int, M2: int, L1: int, L2: int, y) -> np.ndarray:
    """b = A^H y for grids too large to form A, from D = D2 kron D1 (eq:forward_model): with the
    kept rows D1s = D1[m1_n, :] (N x L1) and D2s = D2[m2_n, :] (N x L2),
    b[l1 + l2 L1] = sum_n conj(D2s[n, l2]) y_n conj(D1s[n, l1]) = (D2s^H diag(y) conj(D1s))[l2, l1]."""
    m1, m2 = element_positions(mask, M1)
    D1s = np.exp(-2j * np.pi * np.outer(m1, harmonic_grid(L1)))
    D2s = np.exp(-2j * np.pi * np.outer(m2, harmonic_grid(L2)))
    y = np.asarray(y, np.complex128)
    return (D2s.conj().T @ (y[:, None] * D1s.conj())).reshape(-1)


class KronDictionary:
    """D_s = Psi (D2 kron D1) applied through its Kronecker factors, for grids too large to
    form (eq:forward_model, eq:sparse_forward_model): with a grid W[l2, l1] (the vector
    c[l1 + l2 L1]),
      (D_s c)_n   = (D2 W D1^T)[m2_n, m1_n],
      (D_s^H r)   = D2^H R conj(D1),  R[m2, m1] = sum of r_n over the elements at (m1, m2),
      (D_s D_s^H) = (D1 D1^H)[m1_n, m1_n'] * (D2 D2^H)[m2_n, m2_n']  (entrywise),
    with D_i the full M_i x L_i subdictionaries of eq:subdictionary.  These are the dense
    products regrouped by the Kronecker structure (matrix products only, no FFT)."""

    def __init__(self, mask, M1: int, M2: int, L1: int, L2: int):
        self.M1, self.M2, self.L1, self.L2 = M1, M2, L1, L2
        self.m1, self.m2 = element_positions(mask, M1)
        self.D1 = np.exp(-2j * np.pi * np.outer(np.arange(M1), harmonic_grid(L1)))
        self.D2 = np.exp(-2j * np.pi * np.outer(np.arange(M2), harmonic_grid(L2)))
        self.shape = (self.m1.size, L1 * L2)

    def forward(self, c):
        W = np.asarray(c, np.complex128).reshape(self.L2, self.L1)
        return (self.D2 @ W @ self.D1.T)[self.m2, self.m1]

    def adjoint(self, r):
        R = np.zeros((self.M2, self.M1), np.complex128)
        np.add.at(R, (self.m2, self.m1), np.asarray(r, np.complex128))
        return (self.D2.conj().T @ R @ self.D1.conj()).reshape(-1)

    def gram_rows(self):
        S1 = self.D1 @ self.D1.conj().T
        S2 = self.D2 @ self.D2.conj().T
        return S1[np.ix_(self.m1, self.m1)] * S2[np.ix_(self.m2, self.m2)]


def fista_kron(K: KronDictionary, y, lam, iters, pre=False):
    """FISTA (eq:fista) exactly as ``fista`` from c^(0) = 0, with the products with D_s taken through
    its Kronecker factors and mu = 1/lambda_max(A A^H) from the N x N matrix A A^H.  Returns c^(T)
    (with ``pre`` also the last soft-threshold argument and the threshold mu*lam)."""
    mu = 1.0 / float(np.linalg.eigvalsh(K.gram_rows())[-1])
    b = K.adjoint(y)
    L = K.shape[1]
    c_prev = np.zeros(L, np.complex128)
    z = c_prev.copy()
    beta = fista_momentum(iters)
    c = c_prev
    u = z
    for t in range(iters):
        u = z - mu * K.adjoint(K.forward(z)) + mu * b
        c = soft_threshold(u, mu * lam)
        z = c + beta[t] * (c - c_prev)
        c_prev = c
    return (c, u, mu * lam) if pre else c


def admm_kron(K: KronDictionary, y, lam, rho, iters):
    """ADMM (eq:admm) exactly as ``admm``, with every product with D_s taken through its
    Kronecker factors (``KronDictionary``) and the Woodbury form of (A^H A + rho I)^{-1} on
    the N x N matrix A A^H.  Returns (z^(T), c^(T), v^(T), u^(T)) with u^(T) = c^(T) + v^(T-1)
    the last soft-threshold argument (threshold lam/rho)."""
    rho = float(rho)
    G = K.gram_rows()
    G[np.diag_indices_from(G)] += rho
    factor = scipy.linalg.cho_factor(G, lower=True)

    def inv(w):
        return (w - K.adjoint(scipy.linalg.cho_solve(factor, K.forward(w)))) / rho

    d = inv(K.adjoint(y))
    L = K.shape[1]
    z = np.zeros(L, np.complex128)
    v = np.zeros(L, np.complex128)
    c = z
    u = z
    for _ in range(iters):
        c = d + rho * inv(z - v)
        u = c + v
        z_new = soft_threshold(u, lam / rho)
        v = v + c - z_new
        z = z_new
    return z, c, v, u


# ------------------------------------------------------------------------------------------
# Building blocks of Section II-B
# ------------------------------------------------------------------------------------------


def soft_threshold(u: np.ndarray, kappa: float) -> np.ndarray:
    """Complex soft-threshold S_kappa(u) = exp(j arg u) max(|u| - kappa, 0) (eq:ista)."""
    u = np.asarray(u, dtype=np.complex128)
    mag = np.abs(u)
    out = np.zeros_like(u)
    keep = mag > kappa
    out[keep] = u[keep] / mag[keep] * (mag[keep] - kappa)
    return out


def step_size(A: np.ndarray) -> float:
    """mu = 1 / sigma_max(A)^2 (eq:ista); sigma_max^2 is the top eigenvalue of A A^H."""
    AAh = A @ A.conj().T
    top = np.linalg.eigvalsh(AAh)[-1]  # ascending eigenvalues of the Hermitian N x N matrix
    return 1.0 / float(top)


def adjoint_measurements(A: np.ndarray, y: np.ndarray) -> np.ndarray:
    """b = A^H y, the constant term of eq:ista / eq:admm."""
    return A.conj().T @ np.asarray(y, dtype=np.complex128)


def lambda_max(A: np.ndarray, y: np.ndarray) -> float:
    """||A^H y||_inf: the smallest lam whose LASSO solution is c = 0."""
    return float(np.max(np.abs(adjoint_measurements(A, y))))


class _Gram:
    """A^H A x as two dense matrix-vector products (the paper's "regular" O(L^2)
    product); A^H is formed once."""

    def __init__(self, A):
        self.A = A
        self.Ah = np.ascontiguousarray(A.conj().T)

    def __call__(self, x):
        return self.Ah @ (self.A @ x)


def _gram_apply(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    return A.conj().T @ (A @ x)


def ista(A, y, lam, iters, mu=None, c0=None, history=False, pre=False):
    """ISTA (eq:ista): c^(t+1) = S_{mu lam}((I - mu A^H A) c^(t) + mu A^H y).

    Returns c^(T); with ``history`` also the list [c^(0), ..., c^(T)]; with ``pre``
    also the last soft-threshold argument u^(T) and the threshold mu*lam.
    """
    mu = step_size(A) if mu is None else float(mu)
    gram = _Gram(A)
    b = adjoint_measurements(A, y)
    c = np.zeros(A.shape[1], np.complex128) if c0 is None else np.array(c0, np.complex128)
    hist = [c.copy()] if history else None
    u = c
    for _ in range(iters):
        u = c - mu * gram(c) + mu * b
        c = soft_threshold(u, mu * lam)
        if history:
            hist.append(c.copy())
    out = (c,)
    if history:
        out += (hist,)
    if pre:
        out += (u, mu * lam)
    return out if len(out) > 1 else c


def fista_momentum(iters: int) -> np.ndarray:
    """Momentum weights beta_t = (alpha_t - 1)/alpha_(t+1), t = 1..T, with alpha_1 = 1 and
    alpha_(t+1) = (1 + sqrt(1 + 4 alpha_t^2))/2 (eq:fista)."""
    beta = np.empty(iters, dtype=np.float64)
    a = 1.0
    for t in range(iters):
        a_next = (1.0 + np.sqrt(1.0 + 4.0 * a * a)) / 2.0
        beta[t] = (a - 1.0) / a_next
        a = a_next
    return beta


def fista(A, y, lam, iters, mu=None, c0=None, history=False, pre=False):
    """FISTA (eq:fista).

    z^(1) = c^(0); for t = 1..T:
      c^(t)     = S_{mu lam}((I - mu A^H A) z^(t) + mu A^H y)
      z^(t+1)   = c^(t) + beta_t (c^(t) - c^(t-1)).
    T iterations are T Gram products.  Returns c^(T) (and the list of c^(t); with
    ``pre`` also the last soft-threshold argument and the threshold mu*lam).
    """
    mu = step_size(A) if mu is None else float(mu)
    gram = _Gram(A)
    b = adjoint_measurements(A, y)
    c_prev = np.zeros(A.shape[1], np.complex128) if c0 is None else np.array(c0, np.complex128)
    z = c_prev.copy()
    beta = fista_momentum(iters)
    hist = [c_prev.copy()] if history else None
    c = c_prev
    u = z
    for t in range(iters):
        u = z - mu * gram(z) + mu * b
        c = soft_threshold(u, mu * lam)
        z = c + beta[t] * (c - c_prev)
        c_prev = c
        if history:
            hist.append(c.copy())
    out = (c,)
    if history:
        out += (hist,)
    if pre:
        out += (u, mu * lam)
    return out if len(out) > 1 else c


class _AdmmInverse:
    """Applies (A^H A + rho I)^{-1} by the Woodbury identity with an N x N Cholesky:
    (A^H A + rho I)^{-1} w = (w - A^H (rho I_N + A A^H)^{-1} A w) / rho."""

    def __init__(self, A, rho):
        self.A = A
        self.Ah = np.ascontiguousarray(A.conj().T)
        self.rho = float(rho)
        K = A @ A.conj().T
        K[np.diag_indices_from(K)] += self.rho
        self.factor = scipy.linalg.cho_factor(K, lower=True)

    def __call__(self, w):
        Aw = self.A @ w
        return (w - self.Ah @ scipy.linalg.cho_solve(self.factor, Aw)) / self.rho


def admm_c_update(A, rho):
    """The operator w -> (A^H A + rho I)^{-1} w of eq:admm (dense Woodbury)."""
    return _AdmmInverse(A, rho)


def admm(A, y, lam, rho, iters, z0=None, v0=None, history=False, pre=False):
    """ADMM (eq:admm) with the precomputed term d = (A^H A + rho I)^{-1} A^H y:

      c^(t+1) = d + rho (A^H A + rho I)^{-1} (z^(t) - v^(t))
      z^(t+1) = S_{lam/rho}(c^(t+1) + v^(t))
      v^(t+1) = v^(t) + c^(t+1) - z^(t+1)

    Returns (z^(T), c^(T), v^(T)); with ``history`` also the list of z^(t); with
    ``pre`` also the last soft-threshold argument c^(T) + v^(T-1) and lam/rho.
    """
    inv = _AdmmInverse(A, rho)
    rho = float(rho)
    d = inv(adjoint_measurements(A, y))
    L = A.shape[1]
    z = np.zeros(L, np.complex128) if z0 is None else np.array(z0, np.complex128)
    v = np.zeros(L, np.complex128) if v0 is None else np.array(v0, np.complex128)
    c = np.zeros(L, np.complex128)
    hist = [z.copy()] if history else None
    u = z
    for _ in range(iters):
        c = d + rho * inv(z - v)
        u = c + v
        z_new = soft_threshold(u, lam / rho)
        v = v + c - z_new
        z = z_new
        if history:
            hist.append(z.copy())
    out = (z, c, v)
    if history:
        out = (out, hist)
    if pre:
        out = out + (u, lam / rho)
    return out


# ------------------------------------------------------------------------------------------
# Optimality (eq:lasso_objective with the 1/2 reading)
# ------------------------------------------------------------------------------------------


def objective(A, y, c, lam) -> float:
    """F(c) = 1/2 ||y - A c||_2^2 + lam ||c||_1."""
    r = np.asarray(y) - A @ c
    return 0.5 * float(np.vdot(r, r).real) + lam * float(np.sum(np.abs(c)))


def kkt_residual(A, y, c, lam) -> float:
    """Relative KKT residual of the LASSO at c, with r = A^H (y - A c):

      off the support: (|r_i| - lam)_+ ;  on the support: |r_i - lam c_i/|c_i||.

    Returns max over i of those, divided by lam (0 at an exact minimiser).
    """
    r = A.conj().T @ (np.asarray(y) - A @ c)
    mag = np.abs(c)
    on = mag > 0
    off_viol = np.maximum(np.abs(r[~on]) - lam, 0.0)
    on_viol = np.abs(r[on] - lam * c[on] / mag[on])
    worst = 0.0
    if off_viol.size:
        worst = max(worst, float(off_viol.max()))
    if on_viol.size:
        worst = max(worst, float(on_viol.max()))
    return worst / lam


# ------------------------------------------------------------------------------------------
# BCCB structure (Section III-A)
# ------------------------------------------------------------------------------------------


def gram_first_column(A) -> np.ndarray:
    """First column r of R = A^H A (property (iv)), as an (L2, L1) grid [l2, l1]."""
    L = A.shape[1]
    e0 = np.zeros(L, np.complex128)
    e0[0] = 1.0
    return _gram_apply(A, e0)


def gram_eigenvalues(A, L1: int, L2: int) -> np.ndarray:
    """Eigenvalue grid Omega of eq:lambda, returned as an (L2, L1) array [l2', l1'].

    lambda_{l2'} = F_{L1}( sum_{l2} r_{l2} exp(-j 2 pi l2 l2'/L2) ), with r_{l2}(l1) =
    r(l1 + l2 L1): the L2-point DFT across blocks followed by the L1-point DFT within a
    block.  Both DFTs are written as explicit DFT-matrix products.
    """
    r = gram_first_column(A).reshape(L2, L1)  # [l2, l1]
    F1 = np.exp(-2j * np.pi * np.outer(np.arange(L1), np.arange(L1)) / L1)
    F2 = np.exp(-2j * np.pi * np.outer(np.arange(L2), np.arange(L2)) / L2)
    across = F2 @ r  # [l2', l1] = sum_l2 r_{l2}(l1) e^{-j2pi l2 l2'/L2}
    return across @ F1.T  # apply F_{L1} to each block vector


# ------------------------------------------------------------------------------------------
# Unrolled FISTA (a network of K layers of eq:fista with per-layer step mu_k and
# threshold theta_k; the momentum schedule is FISTA's)
# ------------------------------------------------------------------------------------------


def unrolled_forward(A, y, mu, theta, save=False):
    """c_0 = 0, z_1 = c_0; for k = 1..K:
         u_k = z_k - mu_k A^H (A z_k - y)
         c_k = S_{theta_k}(u_k)
         z_(k+1) = c_k + beta_k (c_k - c_(k-1))      (beta from ``fista_momentum``)
    Returns c_K, and with ``save`` the lists (z_k, u_k) needed by the backward pass.
    """
    K = len(mu)
    b = adjoint_measurements(A, y)
    beta = fista_momentum(K)
    L = A.shape[1]
    gram = _Gram(A)
    c_prev = np.zeros(L, np.complex128)
    z = c_prev.copy()
    zs, us = [], []
    c = c_prev
    for k in range(K):
        u = z - mu[k] * (gram(z) - b)
        c = soft_threshold(u, theta[k])
        if save:
            zs.append(z.copy())
            us.append(u.copy())
        z = c + beta[k] * (c - c_prev)
        c_prev = c
    return (c, zs, us) if save else c


def unrolled_backward(A, y, mu, theta, grad_c, want_grad_y=False):
    """Reverse-mode derivative of a real loss through ``unrolled_forward``.

    Complex gradients use g = dLoss/dRe + j dLoss/dIm, so dLoss = Re(conj(g) dx).
    Returns (dLoss/dmu_k, dLoss/dtheta_k) as float64 arrays of length K; with ``want_grad_y``
    also dLoss/dy (the thresholds held fixed): every layer sees y through b = A^H y, with
    du_k/db = mu_k, so g_b = sum_k mu_k g_{u_k} and g_y = A g_b.
    Derivatives used:
      * S_theta at |u| > theta: with s = 1 - theta/|u|,
          g_u = s g_c + (theta/|u|^3) Re(conj(g_c) u) u,   dLoss/dtheta = -Re(conj(g_c) u)/|u|;
        zero for |u| <= theta;
      * u = z - mu (G z - b) with G = A^H A Hermitian:
          g_z += g_u - mu G g_u,  dLoss/dmu = Re<g_u, b - G z>;
      * z_(k+1) = (1 + beta_k) c_k - beta_k c_(k-1).
    """
    K = len(mu)
    b = adjoint_measurements(A, y)
    beta = fista_momentum(K)
    _, zs, us = unrolled_forward(A, y, mu, theta, save=True)
    gram = _Gram(A)
    L = A.shape[1]
    d_mu = np.zeros(K)
    d_th = np.zeros(K)
    g_c = np.array(grad_c, dtype=np.complex128)  # gradient w.r.t. c_k (current k)
    g_c_next = np.zeros(L, np.complex128)  # contribution to c_(k-1) from z_(k+1)
    g_b = np.zeros(L, np.complex128)
    for k in range(K - 1, -1, -1):
        u = us[k]
        mag = np.abs(u)
        act = mag > theta[k]
        g_u = np.zeros(L, np.complex128)
        s = 1.0 - theta[k] / mag[act]
        proj = np.real(np.conj(g_c[act]) * u[act])
        g_u[act] = s * g_c[act] + (theta[k] / mag[act] ** 3) * proj * u[act]
        d_th[k] = -float(np.sum(proj / mag[act]))
        Gz = gram(zs[k])
        d_mu[k] = float(np.real(np.vdot(g_u, b - Gz)))
        g_b += mu[k] * g_u
        g_z = g_u - mu[k] * gram(g_u)
        # z_k = (1 + beta_(k-1)) c_(k-1) - beta_(k-1) c_(k-2), with z_1 = c_0 = 0 constant.
        if k > 0:
            bk = beta[k - 1]
            g_c = (1.0 + bk) * g_z + g_c_next
            g_c_next = -bk * g_z
        else:
            g_c = np.zeros(L, np.complex128)
    if want_grad_y:
        return d_mu, d_th, A @ g_b
    return d_mu, d_th
