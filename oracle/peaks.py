"""Peak extraction and the harmonic-to-angle map (test infrastructure only).

Follows Section II-A of "Fast Single-Snapshot Harmonic Recovery with 2D Sparse
Arrays using BCCB Matrices" (arXiv 2509.13592): the support of the recovered c
marks harmonic pairs (f_{1,l1}, f_{2,l2}) on the uniform grids f_{i,l} =
-gamma_i + l * 2 gamma_i / L_i (eq:uniform_grid), and each pair gives the angles
through f_1 = gamma_1 cos(phi) sin(theta), f_2 = gamma_2 sin(phi) sin(theta)
with phi in [-pi, pi) and theta in [0, pi/2).

The paper states the map but no peak-picking rule; the rule written here (and
in the CUDA path) is:
  * m(p) = |c(p)|^2 in the precision of c (complex64 -> float32, each product
    and the sum rounded separately; complex128 -> float64);
  * p is a peak when m(p) > 0, m(p) >= rel_thresh^2 * max m, and for each of
    its 8 cyclic neighbours q: m(p) > m(q), or m(p) == m(q) and p < q (linear
    index l1 + l2*L1), so that of a plateau only its lowest index survives;
  * peaks are ranked by m descending, then index ascending, and the first K
    kept; |c| = sqrt(m) in the same precision.
Angles are FP64; a pair with (f1/gamma1)^2 + (f2/gamma2)^2 > 1 lies outside the
visible region and gets NaN angles.
"""
from __future__ import annotations

import numpy as np


def sq_magnitude(c: np.ndarray) -> np.ndarray:
    """|c|^2 with x*x and y*y rounded, then their sum rounded, in c's real precision."""
    c = np.asarray(c)
    dt = np.float32 if c.dtype == np.complex64 else np.float64
    x = np.ascontiguousarray(c.real, dtype=dt)
    y = np.ascontiguousarray(c.imag, dtype=dt)
    return (x * x) + (y * y)


def peak_mask(c_grid: np.ndarray, rel_thresh: float) -> np.ndarray:
    """Boolean (L2, L1) map of the peaks of one grid under the rule above."""
    m = sq_magnitude(c_grid)
    L2, L1 = m.shape
    top = float(m.max()) if m.size else 0.0
    thr = (rel_thresh * rel_thresh) * top
    lin = np.arange(L1 * L2).reshape(L2, L1)
    ok = (m > 0) & (m.astype(np.float64) >= thr)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            mq = np.roll(m, shift=(-dy, -dx), axis=(0, 1))  # mq[l2, l1] = m[l2+dy, l1+dx] (cyclic)
            q = np.roll(lin, shift=(-dy, -dx), axis=(0, 1))
            ok &= ~((mq > m) | ((mq == m) & (q < lin)))
    return ok


def harmonics(l1: np.ndarray, l2: np.ndarray, L1: int, L2: int, gamma1: float = 0.5, gamma2: float = 0.5):
    """(f1, f2) of grid indices on the uniform grids of eq:uniform_grid."""
    f1 = -gamma1 + np.asarray(l1, dtype=np.float64) * (2.0 * gamma1 / L1)
    f2 = -gamma2 + np.asarray(l2, dtype=np.float64) * (2.0 * gamma2 / L2)
    return f1, f2


def angles(f1, f2, gamma1: float = 0.5, gamma2: float = 0.5):
    """(phi, theta) from f1 = gamma1 cos(phi) sin(theta), f2 = gamma2 sin(phi) sin(theta).

    sin(theta) = sqrt(u1^2 + u2^2) with u_i = f_i / gamma_i and phi = atan2(u2, u1);
    NaN for both outside the visible region u1^2 + u2^2 > 1.
    """
    u1 = np.asarray(f1, dtype=np.float64) / gamma1
    u2 = np.asarray(f2, dtype=np.float64) / gamma2
    s = u1 * u1 + u2 * u2
    vis = s <= 1.0
    theta = np.where(vis, np.arcsin(np.sqrt(np.minimum(s, 1.0))), np.nan)
    phi = np.where(vis, np.arctan2(u2, u1), np.nan)
    return phi, theta


def peaks(c_grid: np.ndarray, K: int, rel_thresh: float, gamma1: float = 0.5, gamma2: float = 0.5):
    """Top-K peaks of one (L2, L1) grid.

    Returns dict(idx int32[K] (-1 past the peak count), mag float64[K] (|c|, 0
    past the count), harm float64[K, 2] (f1, f2), ang float64[K, 2] (phi, theta),
    both NaN past the count, count = number of peaks before the cut).
    """
    c_grid = np.asarray(c_grid)
    L2, L1 = c_grid.shape
    m = sq_magnitude(c_grid)
    pk = np.flatnonzero(peak_mask(c_grid, rel_thresh).reshape(-1))
    mv = m.reshape(-1)[pk]
    order = np.lexsort((pk, -mv.astype(np.float64)))  # m descending, then index ascending
    sel = pk[order][:K]
    n = sel.size
    idx = np.full(K, -1, dtype=np.int32)
    mag = np.zeros(K, dtype=np.float64)
    harm = np.full((K, 2), np.nan)
    ang = np.full((K, 2), np.nan)
    idx[:n] = sel
    mag[:n] = np.sqrt(m.reshape(-1)[sel]).astype(np.float64)  # sqrt in c's precision
    f1, f2 = harmonics(sel % L1, sel // L1, L1, L2, gamma1, gamma2)
    harm[:n, 0], harm[:n, 1] = f1, f2
    phi, theta = angles(f1, f2, gamma1, gamma2)
    ang[:n, 0], ang[:n, 1] = phi, theta
    return dict(idx=idx, mag=mag, harm=harm, ang=ang, count=int(pk.size))
