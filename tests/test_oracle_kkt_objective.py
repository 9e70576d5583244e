"""Closed-form pins for the oracle's optimality measures at points that are NOT minimisers.

The LASSO of Section II-A with the 1/2 reading of eq:lasso_objective,
F(c) = 1/2 ||y - A c||^2 + lam ||c||_1, and its relative KKT residual (off the support
(|r_i| - lam)_+, on it |r_i - lam c_i/|c_i||, r = A^H (y - A c), divided by lam) are the
yardsticks of the GPU's FP64 check.  Here every expected value comes from the signal model
alone: one noiseless on-grid source a at grid column l* gives y_n = a exp(-j 2 pi f*.m_n),
so |y_n| = |a|, ||y||^2 = N |a|^2 and, for c supported on {l*, j},
  A^H (y - A c) = (a - c_l*) g(. - l*) - c_j g(. - j),
with the cyclic Gram lag g(d) = sum_n exp(+j 2 pi (d1 m1_n/L1 + d2 m2_n/L2)) summed over the
element positions by hand (g(0) = N).  A dropped term, a missing 1/2, a sign error in the
on-support phase term or an l2 norm in place of the l1 norm each fails one of these.
"""
import numpy as np
import pytest

import oracle
import synth

M1, M2, L1, L2, N = 6, 5, 16, 8, 12


def _problem(seed=21):
    s = synth.make_snapshot(seed, M1, M2, N, L1, L2, 1, None, on_grid=True, unit_amplitude=False)
    A = oracle.dictionary(s.mask, M1, M2, L1, L2)
    a = complex(s.amps[0])
    l1 = int(round((s.freqs[0, 0] + 0.5) * L1))
    l2 = int(round((s.freqs[0, 1] + 0.5) * L2))
    m1, m2 = synth.element_positions(s.mask, M1)
    return s, A, a, l1, l2, m1, m2


def _lag(m1, m2, d1, d2):
    """g(d): the Gram entry between grid columns whose indices differ by (d1, d2)."""
    tot = 0j
    for p, q in zip(m1, m2):
        tot += np.exp(2j * np.pi * (d1 * p / L1 + d2 * q / L2))
    return tot


def _col(l1, l2):
    return l1 + l2 * L1


def test_objective_and_kkt_at_zero():
    """c = 0: F = N|a|^2/2 and the residual is (||A^H y||_inf - lam)_+/lam with
    ||A^H y||_inf = |a| g(0) = N|a| (|g(d)| <= N)."""
    s, A, a, *_ = _problem()
    c = np.zeros(L1 * L2, np.complex128)
    assert oracle.objective(A, s.y, c, 0.7) == pytest.approx(0.5 * N * abs(a) ** 2, rel=1e-13)
    for frac in (0.1, 0.5, 0.9):
        lam = frac * N * abs(a)
        assert oracle.kkt_residual(A, s.y, c, lam) == pytest.approx((N * abs(a) - lam) / lam, rel=1e-12)
    # above lambda_max the zero vector is the minimiser
    assert oracle.kkt_residual(A, s.y, c, 1.01 * N * abs(a)) == 0.0


@pytest.mark.parametrize("eps", [1e-3, -2e-3, 0.05])
def test_kkt_on_support_term_along_the_source(eps):
    """c = t a e_l*, t = t* + eps with t* = 1 - lam/(N|a|) the minimiser's shrink factor:
    on the support r = N a (1 - t), so the violation is |N|a|(1 - t) - lam| = N|a||eps|; off
    it |r_i| = |a|(1 - t)|g| stays below lam for these eps (largest off-peak |g| < N)."""
    s, A, a, l1, l2, m1, m2 = _problem()
    lam = 0.3 * N * abs(a)
    t = 1 - lam / (N * abs(a)) + eps
    c = np.zeros(L1 * L2, np.complex128)
    c[_col(l1, l2)] = t * a
    gmax = max(abs(_lag(m1, m2, d1, d2)) for d1 in range(L1) for d2 in range(L2) if (d1, d2) != (0, 0))
    assert abs(a) * (1 - t) * gmax < lam  # the off-support term is inactive here
    assert oracle.kkt_residual(A, s.y, c, lam) == pytest.approx(N * abs(a) * abs(eps) / lam, rel=1e-9)
    # F = N|a|^2 (1 - t)^2 / 2 + lam t |a|
    exp_f = 0.5 * N * abs(a) ** 2 * (1 - t) ** 2 + lam * t * abs(a)
    assert oracle.objective(A, s.y, c, lam) == pytest.approx(exp_f, rel=1e-12)


def test_kkt_off_support_term_decides_with_a_missed_source():
    """Two noiseless on-grid sources a1 at l1*, a2 at l2*; c holds only the first, at the
    single-source optimum c1 = a1 (1 - lam/(N|a1|)).  Then
      r = (a1 - c1) g(. - l1*) + a2 g(. - l2*),
    on the support |r_l1* - lam a1/|a1|| = |a2 g(l1* - l2*)|, and off it the missed source
    leaves |r_l2*| close to N|a2|, far above lam: the off-support term decides."""
    s = synth.make_snapshot(36, M1, M2, N, L1, L2, 2, None, on_grid=True, unit_amplitude=False)
    A = oracle.dictionary(s.mask, M1, M2, L1, L2)
    m1, m2 = synth.element_positions(s.mask, M1)
    (a1, a2) = (complex(s.amps[0]), complex(s.amps[1]))
    p = [(int(round((f1 + 0.5) * L1)), int(round((f2 + 0.5) * L2))) for f1, f2 in s.freqs]
    lam = 0.2 * N * abs(a1)
    c1 = a1 * (1 - lam / (N * abs(a1)))
    c = np.zeros(L1 * L2, np.complex128)
    c[_col(*p[0])] = c1

    def r_at(i1, i2):
        return (a1 - c1) * _lag(m1, m2, i1 - p[0][0], i2 - p[0][1]) + a2 * _lag(m1, m2, i1 - p[1][0], i2 - p[1][1])

    v_on = abs(r_at(*p[0]) - lam * c1 / abs(c1))
    v_off = max(max(abs(r_at(i1, i2)) - lam, 0.0) for i1 in range(L1) for i2 in range(L2) if (i1, i2) != p[0])
    assert v_on == pytest.approx(abs(a2 * _lag(m1, m2, p[0][0] - p[1][0], p[0][1] - p[1][1])), rel=1e-12)
    assert v_off > v_on  # the missed source dominates
    assert oracle.kkt_residual(A, s.y, c, lam) == pytest.approx(v_off / lam, rel=1e-9)
    # F = 1/2 ||(a1 - c1) A e_l1* + a2 A e_l2*||^2 + lam |c1|
    g21 = _lag(m1, m2, p[1][0] - p[0][0], p[1][1] - p[0][1])  # G(l2*, l1*)
    data = abs(a1 - c1) ** 2 * N + abs(a2) ** 2 * N + 2 * ((a1 - c1) * np.conj(a2) * g21).real
    assert oracle.objective(A, s.y, c, lam) == pytest.approx(0.5 * data + lam * abs(c1), rel=1e-12)


def test_kkt_and_objective_with_a_spurious_entry():
    """c = t* a e_l* + eta e_j (j != l*): data residual (1 - t*) a A e_l* - eta A e_j, so
      r_l* = N a (1 - t*) - eta g(l* - j),  r_j = a (1 - t*) g(j - l*) - eta N,
    on-support violations |r_l* - lam a/|a|| = |eta g(l* - j)| and |r_j - lam eta/|eta||, and
      F = ((1 - t*)^2 |a|^2 N + |eta|^2 N - 2 Re((1 - t*) a conj(eta) g(j - l*)))/2
          + lam (t* |a| + |eta|)."""
    s, A, a, l1, l2, m1, m2 = _problem()
    lam = 0.3 * N * abs(a)
    t = 1 - lam / (N * abs(a))
    j1, j2 = (l1 + 3) % L1, (l2 + 1) % L2
    eta = 0.05 * abs(a) * np.exp(1j * 0.7)
    c = np.zeros(L1 * L2, np.complex128)
    c[_col(l1, l2)] = t * a
    c[_col(j1, j2)] = eta
    g_lj = _lag(m1, m2, l1 - j1, l2 - j2)  # G(l*, j)
    g_jl = _lag(m1, m2, j1 - l1, j2 - l2)  # G(j, l*) = conj(G(l*, j))
    r_l = N * a * (1 - t) - eta * g_lj
    r_j = a * (1 - t) * g_jl - eta * N
    v_on = max(abs(r_l - lam * a / abs(a)), abs(r_j - lam * eta / abs(eta)))
    # every other column: |r_i| = |a (1 - t) g(i - l*) - eta g(i - j)| < lam here
    others = []
    for i1 in range(L1):
        for i2 in range(L2):
            if (i1, i2) in ((l1, l2), (j1, j2)):
                continue
            others.append(abs(a * (1 - t) * _lag(m1, m2, i1 - l1, i2 - l2) - eta * _lag(m1, m2, i1 - j1, i2 - j2)))
    v_off = max(max(others) - lam, 0.0)
    assert oracle.kkt_residual(A, s.y, c, lam) == pytest.approx(max(v_on, v_off) / lam, rel=1e-9)
    exp_f = 0.5 * (((1 - t) * abs(a)) ** 2 * N + abs(eta) ** 2 * N - 2 * ((1 - t) * a * np.conj(eta) * g_jl).real)
    exp_f += lam * (t * abs(a) + abs(eta))
    assert oracle.objective(A, s.y, c, lam) == pytest.approx(exp_f, rel=1e-12)
