"""The bench's host timing leg for the paper's FFT method (Section III-B: Gram products as
IFFT2(Omega . FFT2(z)), Omega from eq:lambda) computes the same FISTA iterates as the dense
oracle, to FP64 rounding (the agreement Table I reports for the paper's two CPU
implementations)."""
import numpy as np

import bench
import oracle


def test_cpu_fft_leg_matches_dense_oracle():
    n, iters, first = 2, 25, 123
    rate, seconds, c = bench.cpu_fft_sample(n, iters, first=first)
    assert rate > 0 and seconds > 0
    L1, L2 = bench.WORKLOAD["L1"], bench.WORKLOAD["L2"]
    for i, s in enumerate(bench.make_batch(n, first)):
        A = oracle.dictionary(s.mask, s.M1, s.M2, L1, L2)
        lam = bench.WORKLOAD["lam_frac"] * oracle.lambda_max(A, s.y)
        ref = oracle.fista(A, s.y, lam, iters)
        assert np.count_nonzero(ref) > 0
        err = np.linalg.norm(c[i].reshape(-1) - ref) / np.linalg.norm(ref)
        assert err <= 1e-12, f"instance {i}: {err:.2e}"
