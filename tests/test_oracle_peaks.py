"""Pins of the peak-extraction / harmonic-to-angle oracle (Section II-A) against
hand-derived expectations, closed forms and the signal model itself."""
import numpy as np
import pytest

import oracle
from oracle import peaks as opk


def _grid(L2, L1, entries, dtype=np.complex64):
    c = np.zeros((L2, L1), dtype=dtype)
    for (l2, l1), v in entries.items():
        c[l2, l1] = v
    return c


def test_planted_peaks_rule_by_hand():
    # magnitudes: 5 at (2,3); 3 at (5,10) beside 2 at (5,11); a plateau of two 4s at
    # (6,1),(6,2); 1 at the corner (0,0) whose cyclic neighbour (7,15) holds 0.5
    c = _grid(8, 16, {(2, 3): 5.0, (5, 10): 3.0j, (5, 11): 2.0, (6, 1): -4.0, (6, 2): 4.0j,
                      (0, 0): 1.0, (7, 15): 0.5})
    r = opk.peaks(c, K=6, rel_thresh=0.0)
    # expected ranking (hand-derived): 25 @ 35, 16 @ 97 (plateau: lower index), 9 @ 90, 1 @ 0
    assert r["count"] == 4
    assert list(r["idx"]) == [35, 97, 90, 0, -1, -1]
    assert list(r["mag"][:4]) == [5.0, 4.0, 3.0, 1.0]
    assert np.all(np.isnan(r["ang"][4:]))
    # the relative threshold drops the corner peak: 1 < 0.3^2 * 25
    r = opk.peaks(c, K=6, rel_thresh=0.3)
    assert r["count"] == 3 and list(r["idx"][:3]) == [35, 97, 90]


def test_plateau_keeps_only_lowest_index_and_all_equal_grid():
    c = np.full((8, 8), 1.0 + 1.0j, dtype=np.complex64)
    r = opk.peaks(c, K=4, rel_thresh=0.0)
    # every cell ties with its neighbours; only cell 0 has all 8 neighbours at larger indices
    assert r["count"] == 1 and r["idx"][0] == 0
    c = np.zeros((8, 8), dtype=np.complex64)
    assert opk.peaks(c, K=2, rel_thresh=0.0)["count"] == 0


def test_equal_isolated_peaks_break_ties_by_index():
    # equal peaks at even (l2, l1): 16 of them on an 8x8 grid; the K = 5 kept are the
    # five lowest linear indices 0, 2, 4, 6, 16
    c = np.zeros((8, 8), dtype=np.complex64)
    c[0::2, 0::2] = 2.0
    r = opk.peaks(c, K=5, rel_thresh=0.0)
    assert r["count"] == 16
    assert list(r["idx"]) == [0, 2, 4, 6, 16]


def test_harmonic_grid_and_angle_closed_forms():
    f1, f2 = opk.harmonics(np.array([0, 16, 20, 24]), np.array([16, 8, 16, 24]), 32, 32)
    assert np.array_equal(f1, [-0.5, 0.0, 0.125, 0.25]) and np.array_equal(f2, [0.0, -0.25, 0.0, 0.25])
    phi, theta = opk.angles(np.array([0.0, 0.25, 0.0, 0.25, 0.45]), np.array([0.0, 0.0, -0.25, 0.25, 0.45]))
    # broadside; sin(theta) = 1/2 along x; along -y; the 45-degree diagonal; outside the visible region
    assert theta[0] == 0.0 and phi[0] == 0.0
    assert np.isclose(theta[1], np.pi / 6, rtol=0, atol=1e-15) and phi[1] == 0.0
    assert np.isclose(theta[2], np.pi / 6, rtol=0, atol=1e-15) and np.isclose(phi[2], -np.pi / 2, rtol=0, atol=1e-15)
    assert np.isclose(theta[3], np.pi / 4, rtol=0, atol=1e-15) and np.isclose(phi[3], np.pi / 4, rtol=0, atol=1e-15)
    assert np.isnan(theta[4]) and np.isnan(phi[4])
    # the forward relation of Section II-A inverts it (gamma = 0.3 and 0.7 too)
    rng = np.random.default_rng(3)
    for g1, g2 in ((0.5, 0.5), (0.3, 0.7)):
        ph = rng.uniform(-np.pi, np.pi, 50)
        th = rng.uniform(0.0, np.pi / 2, 50)
        p2, t2 = opk.angles(g1 * np.cos(ph) * np.sin(th), g2 * np.sin(ph) * np.sin(th), g1, g2)
        assert np.allclose(t2, th, atol=1e-9) and np.allclose(np.angle(np.exp(1j * (p2 - ph))), 0, atol=1e-9)


def test_complex64_magnitude_uses_float32_rounding():
    # 1 + 2^-12 squared needs 25 bits: float32 rounds it, float64 does not
    x = np.float32(1.0 + 2.0**-12)
    m32 = opk.sq_magnitude(np.array([x + 0j], dtype=np.complex64))[0]
    m64 = opk.sq_magnitude(np.array([complex(float(x), 0.0)], dtype=np.complex128))[0]
    assert m32.dtype == np.float32 and m64.dtype == np.float64
    assert float(m32) == float(np.float32(float(x) * float(x))) and float(m64) == float(x) * float(x)
    assert float(m32) != float(m64)


def test_angles_recovered_from_the_signal_model():
    """Noiseless sources whose harmonics lie on the grid: the FISTA solution's three
    strongest peaks sit at their cells and map back to their angles (Section II-A)."""
    M1 = M2 = 8
    L1 = L2 = 32
    rng = np.random.default_rng(11)
    lin = np.sort(rng.choice(M1 * M2, size=40, replace=False))
    mask = np.zeros(M1 * M2, dtype=np.uint8)
    mask[lin] = 1
    m1, m2 = lin % M1, lin // M1
    # angles chosen so that f = (cos(phi) sin(theta), sin(phi) sin(theta)) / 2 is on the grid
    src = [(0.0, np.arcsin(0.25)), (-np.pi / 2, np.pi / 6), (np.pi / 4, np.pi / 4)]
    cells = [(20, 16), (16, 8), (24, 24)]  # (l1, l2)
    amps = [1.0, 0.8j, -0.9]
    y = np.zeros(lin.size, dtype=np.complex128)
    for (ph, th), a in zip(src, amps):
        f1, f2 = 0.5 * np.cos(ph) * np.sin(th), 0.5 * np.sin(ph) * np.sin(th)
        y += a * np.exp(-2j * np.pi * (m1 * f1 + m2 * f2))
    A = oracle.dictionary(mask, M1, M2, L1, L2)
    lam = 0.05 * oracle.lambda_max(A, y)
    c = oracle.fista(A, y, lam, 3000)
    r = opk.peaks(c.reshape(L2, L1), K=3, rel_thresh=0.1)
    assert sorted(r["idx"].tolist()) == sorted(l1 + L1 * l2 for (l1, l2) in cells)
    for k in range(3):
        j = [l1 + L1 * l2 for (l1, l2) in cells].index(int(r["idx"][k]))
        assert np.isclose(r["ang"][k, 1], src[j][1], atol=1e-12)
        assert np.isclose(np.angle(np.exp(1j * (r["ang"][k, 0] - src[j][0]))), 0.0, atol=1e-12)
