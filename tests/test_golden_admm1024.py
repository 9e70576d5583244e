"""The stored 1024 x 1024 ADMM reference (tests/golden/admm1024_rho*.txt) is consistent with what the
oracle fixes cheaply: lam = 0.05 ||A^H y||_inf of the complex64-rounded measurements (A^H y through the
Kronecker factors of D), the sample indices from their seed, z^(T) = 0 at rho = 0.5 (rho far below the
Gram's nonzero eigenvalue L1 L2 keeps z at 0; see the readings), and the stored norm of z^(T) matching
its stored nonzeros."""
import os
import sys

import numpy as np
import pytest

import oracle
import synth

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_admm1024 as golden  # noqa: E402


@pytest.mark.parametrize("tag,rho", [("0p5", 0.5), ("1024", 1024.0)])
def test_reference_header_and_samples(tag, rho):
    ref = golden.read(tag)
    s = synth.workload_snapshot("admm1024", 0)
    y = s.y.astype(np.complex64).astype(np.complex128)
    K = oracle.KronDictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
    assert ref["lam"] == pytest.approx(0.05 * np.abs(K.adjoint(y)).max(), rel=1e-13)
    assert ref["rho"] == rho and ref["iters"] == golden.ITERS
    idx = np.sort(np.random.Generator(np.random.PCG64(4242)).choice(s.L1 * s.L2, golden.SAMPLES, replace=False))
    np.testing.assert_array_equal(ref["s_idx"], idx)
    assert np.all(np.isfinite(ref["s_c"])) and np.all(np.isfinite(ref["s_v"]))
    if rho == 0.5:
        assert ref["z_idx"].size == 0 and ref["norm_z"] == 0.0
    else:
        assert ref["z_idx"].size > 0
        assert np.linalg.norm(ref["z_val"]) == pytest.approx(ref["norm_z"], rel=1e-12)
