"""Pins for the oracle's Kronecker-factored dictionary (oracle.KronDictionary, oracle.admm_kron),
the form the 1024 x 1024 ADMM reference is computed with: on grids small enough to form A, every
product and the whole ADMM solve equal the dense oracle's (eq:forward_model: D = D2 kron D1)."""
import numpy as np
import pytest

import oracle
import synth

SHAPES = [(5, 3, 8, 16, 9), (9, 6, 8, 16, 30), (16, 8, 32, 16, 40), (7, 12, 16, 8, 50)]  # 2nd, 4th fold


@pytest.mark.parametrize("M1,M2,L1,L2,N", SHAPES)
def test_products_equal_the_dense_dictionary(M1, M2, L1, L2, N):
    s = synth.make_snapshot(17 + M1, M1, M2, N, L1, L2, 3, 10.0)
    A = oracle.dictionary(s.mask, M1, M2, L1, L2)
    K = oracle.KronDictionary(s.mask, M1, M2, L1, L2)
    rng = np.random.default_rng(M2)
    x = rng.standard_normal(L1 * L2) + 1j * rng.standard_normal(L1 * L2)
    np.testing.assert_allclose(K.forward(x), A @ x, rtol=0, atol=1e-12 * np.abs(A @ x).max())
    np.testing.assert_allclose(K.adjoint(s.y), A.conj().T @ s.y, rtol=0, atol=1e-12 * np.abs(s.y).sum())
    np.testing.assert_allclose(K.gram_rows(), A @ A.conj().T, rtol=0, atol=1e-11 * L1 * L2)
    assert K.shape == A.shape


@pytest.mark.parametrize("rho", [0.5, 3.0, 40.0])
def test_admm_equals_the_dense_oracle(rho):
    s = synth.make_snapshot(23, 9, 6, 30, 8, 16, 3, 10.0)  # M1 > L1: the rows fold
    A = oracle.dictionary(s.mask, 9, 6, 8, 16)
    K = oracle.KronDictionary(s.mask, 9, 6, 8, 16)
    lam = 0.1 * oracle.lambda_max(A, s.y)
    z1, c1, v1, u1, k1 = oracle.admm(A, s.y, lam, rho, 300, pre=True)
    z2, c2, v2, u2 = oracle.admm_kron(K, s.y, lam, rho, 300)
    for a, b in ((z1, z2), (c1, c2), (v1, v2), (u1, u2)):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-11 * max(1.0, np.abs(a).max()))
    assert k1 == pytest.approx(lam / rho)


def test_fista_equals_the_dense_oracle():
    s = synth.make_snapshot(29, 7, 12, 40, 16, 8, 3, 10.0)  # M2 > L2: the columns fold
    A = oracle.dictionary(s.mask, 7, 12, 16, 8)
    K = oracle.KronDictionary(s.mask, 7, 12, 16, 8)
    lam = 0.1 * oracle.lambda_max(A, s.y)
    ref = oracle.fista(A, s.y, lam, 250)
    np.testing.assert_allclose(oracle.fista_kron(K, s.y, lam, 250), ref, rtol=0, atol=1e-11 * np.abs(ref).max())
