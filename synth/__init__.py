"""Seeded synthetic snapshots for the single-snapshot 2D harmonic-recovery workloads.

This module is shared by the FP64 oracle's tests, the GPU parity tests and the
benchmark.  It holds the *signal model* only (Section II-A, eq:signal_model and
the sparse-array subsampling of eq:sparse_forward_model): it draws element
masks, sources and noise and evaluates the array response at the element
positions.  It contains none of the recovery method's arithmetic (no
dictionary, no Gram matrix, no FFT, no LASSO step).

Conventions (Section II-A):
  * the full URA has M1 x M2 positions on a half-wavelength grid; a sparse
    array keeps N of them.  ``mask`` is a flat uint8 array of length M1*M2 with
    ``mask[m1 + m2*M1] = 1`` for a kept element (the subsampling matrix Psi);
  * the measurement vector ``y`` lists the kept elements in ascending order of
    the linear index m1 + m2*M1;
  * a source with harmonics (f1, f2) contributes exp(-j 2 pi (m1 f1 + m2 f2));
  * noise is circular complex Gaussian CN(0, sigma^2) per element with
    sigma^2 = P_s / 10^(SNR/10), P_s the mean clean power over the kept
    elements.

Every generator takes an explicit ``seed`` and uses NumPy's PCG64, so the same
call gives the same arrays on any machine.
"""
from __future__ import annotations

import dataclasses
from typing import Tuple, List, Optional

import numpy as np

__all__ = [
    "Snapshot",
    "make_mask",
    "element_positions",
    "on_grid_frequencies",
    "make_snapshot",
    "workload_snapshot",
    "workload_batch",
    "WORKLOADS",
]


@dataclasses.dataclass
class Snapshot:
    """One synthetic single-snapshot problem instance."""

    M1: int
    M2: int
    L1: int
    L2: int
    mask: np.ndarray  # uint8, length M1*M2, index m1 + m2*M1
    y: np.ndarray  # complex128, length N (ascending linear index)
    freqs: np.ndarray  # float64 (K, 2): (f1, f2) in [-1/2, 1/2)
    amps: np.ndarray  # complex128 (K,)
    snr_db: Optional[float]  # None = noiseless
    lam_frac: float = 0.1  # lambda = lam_frac * ||A^H y||_inf (applied by the caller)
    gamma: Tuple[float, float] = (0.5, 0.5)  # element spacings in wavelengths (Section II-A)

    @property
    def N(self) -> int:
        return int(self.mask.sum())


def make_mask(rng: np.random.Generator, M1: int, M2: int, N: int) -> np.ndarray:
    """Keep N of the M1*M2 URA positions, uniformly without replacement (Fig. 1)."""
    if not (1 <= N <= M1 * M2):
        raise ValueError("N must be in [1, M1*M2]")
    idx = rng.choice(M1 * M2, size=N, replace=False)
    mask = np.zeros(M1 * M2, dtype=np.uint8)
    mask[idx] = 1
    return mask


def element_positions(mask: np.ndarray, M1: int):
    """(m1, m2) of the kept elements in ascending linear index m1 + m2*M1."""
    lin = np.flatnonzero(np.asarray(mask).reshape(-1))
    return lin % M1, lin // M1


def on_grid_frequencies(rng: np.random.Generator, L1: int, L2: int, K: int,
                        gamma: Tuple[float, float] = (0.5, 0.5)) -> np.ndarray:
    """K distinct grid points f_{i,l} = -gamma_i + l 2 gamma_i / L_i (eq:uniform_grid)."""
    flat = rng.choice(L1 * L2, size=K, replace=False)
    l1 = flat % L1
    l2 = flat // L1
    g1, g2 = gamma
    return np.stack([-g1 + l1 * (2.0 * g1 / L1), -g2 + l2 * (2.0 * g2 / L2)], axis=1)


def _response(m1: np.ndarray, m2: np.ndarray, freqs: np.ndarray, amps: np.ndarray) -> np.ndarray:
    # eq:signal_model restricted to the kept elements.
    phase = np.outer(m1, freqs[:, 0]) + np.outer(m2, freqs[:, 1])
    return np.exp(-2j * np.pi * phase) @ amps


def make_snapshot(
    seed: int,
    M1: int,
    M2: int,
    N: int,
    L1: int,
    L2: int,
    K: int,
    snr_db: Optional[float],
    on_grid: bool = False,
    unit_amplitude: bool = False,
    mask: Optional[np.ndarray] = None,
    lam_frac: float = 0.1,
    gamma: Tuple[float, float] = (0.5, 0.5),
) -> Snapshot:
    """Draw one snapshot: mask (unless given), K sources, amplitudes, noise.

    ``on_grid`` puts the sources on the recovery grid; otherwise the harmonics
    are uniform on [-gamma_1, gamma_1) x [-gamma_2, gamma_2) (the range of
    f* = (gamma_1 cos(phi) sin(theta), gamma_2 sin(phi) sin(theta)), Section II-A;
    [-1/2, 1/2)^2 for half-wavelength spacing).  ``unit_amplitude`` gives
    |c_k| = 1 with a uniform phase; otherwise c_k ~ CN(0, 1).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if mask is None:
        mask = make_mask(rng, M1, M2, N)
    else:
        mask = np.asarray(mask, dtype=np.uint8).reshape(-1).copy()
    g1, g2 = gamma
    if on_grid:
        freqs = on_grid_frequencies(rng, L1, L2, K, gamma)
    elif gamma == (0.5, 0.5):
        freqs = rng.uniform(-0.5, 0.5, size=(K, 2))
    else:
        freqs = rng.uniform(0.0, 1.0, size=(K, 2)) * np.array([2 * g1, 2 * g2]) - np.array([g1, g2])
    if unit_amplitude:
        amps = np.exp(2j * np.pi * rng.uniform(0.0, 1.0, size=K))
    else:
        amps = (rng.standard_normal(K) + 1j * rng.standard_normal(K)) / np.sqrt(2.0)
    m1, m2 = element_positions(mask, M1)
    y = _response(m1, m2, freqs, amps)
    if snr_db is not None:
        p_s = float(np.mean(np.abs(y) ** 2))
        sigma2 = p_s / (10.0 ** (snr_db / 10.0))
        noise = (rng.standard_normal(y.size) + 1j * rng.standard_normal(y.size)) * np.sqrt(sigma2 / 2.0)
        y = y + noise
    return Snapshot(M1, M2, L1, L2, mask, y.astype(np.complex128), freqs, amps, snr_db, lam_frac,
                    (float(g1), float(g2)))


# --------------------------------------------------------------------------------------------
# Named workloads.  Each has a fixed seed base; instance i of a single-snapshot workload is drawn
# with seed base + i.
# --------------------------------------------------------------------------------------------
WORKLOADS = {
    # Plain FISTA, 16x16 array, N=64, 64x64 grid, 3 on-grid unit sources, 20 dB, 500 iterations.
    "fista64": dict(seed=1000, M1=16, M2=16, N=64, L1=64, L2=64, K=3, snr_db=20.0, on_grid=True,
                    unit_amplitude=True, lam_frac=0.1, iters=500),
    # ISTA / FISTA / ADMM(rho=1), 32x32 array, N=256, 256x256 grid, 8 off-grid CN(0,1) sources, 10 dB.
    "solve256": dict(seed=2000, M1=32, M2=32, N=256, L1=256, L2=256, K=8, snr_db=10.0, on_grid=False,
                     unit_amplitude=False, lam_frac=0.05, iters=1000, rho=1.0),
    # 64x64 array, N=1024, 1024x1024 grid, 20 off-grid sources, 15 dB, ADMM rho=0.5, 2000 iterations.
    "admm1024": dict(seed=4000, M1=64, M2=64, N=1024, L1=1024, L2=1024, K=20, snr_db=15.0, on_grid=False,
                     unit_amplitude=False, lam_frac=0.05, iters=2000, rho=0.5),
}


def workload_snapshot(name: str, instance: int = 0, **overrides) -> Snapshot:
    """Instance `instance` of a single-snapshot workload of WORKLOADS."""
    p = dict(WORKLOADS[name])
    p.update(overrides)
    return make_snapshot(
        p["seed"] + instance,
        p["M1"], p["M2"], p["N"], p["L1"], p["L2"], p["K"], p["snr_db"],
        on_grid=p["on_grid"], unit_amplitude=p["unit_amplitude"], lam_frac=p["lam_frac"],
    )


def workload_batch(name: str, count: int, first: int = 0, L_choices=(64, 128, 256),
                   fixed_mask_seed: Optional[int] = None, L: Optional[int] = None) -> List[Snapshot]:
    """Batched workloads.

    "ragged": per instance L1, L2 iid uniform on ``L_choices``, M_i = L_i/4, N =
    round(0.25*M1*M2) random elements, K ~ U{1..10} off-grid, SNR ~ U[0, 30] dB
    (instance i from seed 3000 + i).  ``L`` forces a square L x L grid.

    "learned": fixed 32x32 array with N=256 (mask from ``fixed_mask_seed``, default
    5000), 256x256 grid, K ~ U{1..8} off-grid, SNR ~ U[0, 30] dB (instance i from seed
    5001 + i).

    "solve256": every instance drawn like the single-snapshot workload (own mask,
    8 sources, 10 dB) with seed 2000 + instance.
    """
    out: List[Snapshot] = []
    if name == "ragged":
        for i in range(first, first + count):
            rng = np.random.Generator(np.random.PCG64(3000 + i))
            if L is None:
                L1 = int(rng.choice(L_choices))
                L2 = int(rng.choice(L_choices))
            else:
                L1 = L2 = int(L)
            M1, M2 = L1 // 4, L2 // 4
            N = int(round(0.25 * M1 * M2))
            K = int(rng.integers(1, 11))
            snr = float(rng.uniform(0.0, 30.0))
            sub = int(rng.integers(0, 2**62))
            out.append(make_snapshot(sub, M1, M2, N, L1, L2, K, snr, lam_frac=0.1))
    elif name == "learned":
        mseed = 5000 if fixed_mask_seed is None else fixed_mask_seed
        mask = make_mask(np.random.Generator(np.random.PCG64(mseed)), 32, 32, 256)
        for i in range(first, first + count):
            rng = np.random.Generator(np.random.PCG64(5001 + i))
            K = int(rng.integers(1, 9))
            snr = float(rng.uniform(0.0, 30.0))
            sub = int(rng.integers(0, 2**62))
            out.append(make_snapshot(sub, 32, 32, 256, 256, 256, K, snr, mask=mask, lam_frac=0.05))
    elif name == "solve256":
        for i in range(first, first + count):
            out.append(workload_snapshot("solve256", i))
    else:
        raise ValueError("batched workloads are 'ragged', 'learned' and 'solve256'")
    return out


def paper_experiment_snapshot(trial: int, L1: int, L2: int = 32) -> Snapshot:
    """The paper's experiment shape (Section III-C): M1=51, M2=16, 40 random elements,
    K uniform on {1..10}, harmonics uniform on [-1/2, 1/2)^2, 15 dB SNR."""
    rng = np.random.Generator(np.random.PCG64(7000 + trial))
    K = int(rng.integers(1, 11))
    sub = int(rng.integers(0, 2**62))
    return make_snapshot(sub, 51, 16, 40, L1, L2, K, 15.0, lam_frac=0.1)
