"""Pins for element spacings gamma != 1/2 (Section III-A): the Gram of the dictionary on
the uniform grid of eq:uniform_grid is then block Toeplitz with Toeplitz blocks, not
BCCB, and a product with it is the top-left block of a 2L1 x 2L2 circulant product."""
import numpy as np
import pytest

import oracle
import synth

G1, G2 = 0.35, 0.8


def _mask(seed, M1, M2, N):
    rng = np.random.default_rng(seed)
    mask = np.zeros(M1 * M2, np.uint8)
    mask[rng.choice(M1 * M2, size=N, replace=False)] = 1
    return mask


def _lag_sum(mask, M1, L1, L2, d1, d2, g1, g2):
    # sum over kept elements of exp(+j 2 pi (f-difference) . m) for grid steps d1, d2
    m1, m2 = oracle.element_positions(mask, M1)
    return np.sum(np.exp(2j * np.pi * (2 * g1 * d1 * m1 / L1 + 2 * g2 * d2 * m2 / L2)))


def test_half_wavelength_default_is_unchanged():
    mask = _mask(1, 5, 4, 11)
    A = oracle.dictionary(mask, 5, 4, 8, 16)
    assert np.array_equal(A, oracle.dictionary(mask, 5, 4, 8, 16, 0.5, 0.5))
    assert np.array_equal(oracle.harmonic_grid(8), -0.5 + np.arange(8) / 8)
    assert np.allclose(oracle.harmonic_grid(8, 0.3), np.linspace(-0.3, 0.3, 9)[:-1], rtol=0, atol=1e-15)


def test_gram_is_block_toeplitz_not_circulant():
    M1, M2, L1, L2 = 5, 3, 8, 4
    mask = _mask(2, M1, M2, 9)
    A = oracle.dictionary(mask, M1, M2, L1, L2, G1, G2)
    G = A.conj().T @ A
    worst = 0.0
    for l in range(L1 * L2):
        for lp in range(L1 * L2):
            d1, d2 = l % L1 - lp % L1, l // L1 - lp // L1
            worst = max(worst, abs(G[l, lp] - _lag_sum(mask, M1, L1, L2, d1, d2, G1, G2)))
    assert worst < 1e-12
    # wrapping the lag (a circulant) would be wrong for gamma != 1/2
    assert abs(G[1, 0] - G[0, L1 - 1]) > 1e-3


def test_circulant_embedding_reproduces_the_gram_product():
    M1, M2, L1, L2 = 6, 5, 16, 8
    mask = _mask(3, M1, M2, 17)
    A = oracle.dictionary(mask, M1, M2, L1, L2, G1, G2)
    G = A.conj().T @ A
    E1, E2 = 2 * L1, 2 * L2
    cext = np.zeros((E2, E1), np.complex128)
    for e2 in range(E2):
        for e1 in range(E1):
            if e1 == L1 or e2 == L2:
                continue  # the lag no pair of block entries uses
            d1 = e1 if e1 < L1 else e1 - E1
            d2 = e2 if e2 < L2 else e2 - E2
            cext[e2, e1] = _lag_sum(mask, M1, L1, L2, d1, d2, G1, G2)
    lam = np.fft.fft2(cext)
    assert np.max(np.abs(lam.imag)) < 1e-9 * np.max(np.abs(lam))  # Hermitian first column: real spectrum
    rng = np.random.default_rng(4)
    x = rng.standard_normal(L1 * L2) + 1j * rng.standard_normal(L1 * L2)
    pad = np.zeros((E2, E1), np.complex128)
    pad[:L2, :L1] = x.reshape(L2, L1)
    prod = np.fft.ifft2(lam * np.fft.fft2(pad))[:L2, :L1].reshape(-1)
    assert np.allclose(prod, G @ x, rtol=0, atol=1e-10 * np.linalg.norm(G @ x))
    # the step bound: the Gram's top eigenvalue never exceeds the embedding's (interlacing)
    assert np.linalg.eigvalsh(G)[-1] <= lam.real.max() * (1 + 1e-12)


def test_on_grid_sources_are_dictionary_columns():
    M1, M2, L1, L2 = 6, 5, 16, 8
    s = synth.make_snapshot(5, M1, M2, 18, L1, L2, K=3, snr_db=None, on_grid=True, gamma=(G1, G2))
    A = oracle.dictionary(s.mask, M1, M2, L1, L2, G1, G2)
    f1g, f2g = oracle.harmonic_grid(L1, G1), oracle.harmonic_grid(L2, G2)
    c = np.zeros(L1 * L2, np.complex128)
    for (f1, f2), a in zip(s.freqs, s.amps):
        l1 = int(np.argmin(np.abs(f1g - f1)))
        l2 = int(np.argmin(np.abs(f2g - f2)))
        c[l1 + L1 * l2] = a
    assert np.allclose(A @ c, s.y, rtol=0, atol=1e-12)


@pytest.mark.parametrize("algo", ["ista", "fista"])
def test_solvers_reach_kkt_for_toeplitz_gram(algo):
    s = synth.make_snapshot(6, 6, 5, 18, 16, 8, K=2, snr_db=20.0, gamma=(G1, G2))
    A = oracle.dictionary(s.mask, 6, 5, 16, 8, G1, G2)
    lam = 0.1 * oracle.lambda_max(A, s.y)
    c = oracle.ista(A, s.y, lam, 20000) if algo == "ista" else oracle.fista(A, s.y, lam, 4000)
    assert oracle.kkt_residual(A, s.y, c, lam) < 1e-6
