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


def test_algorithmic_flops_per_instance_iteration():
    """The roofline's unit: a forward and an inverse 2D FFT at 5 L log2 L flops each plus 18 L
    pointwise flops, L = L1 L2 (11.67 M on the 256 x 256 grid)."""
    assert bench.flops_per_inst_iter(256, 256) == (10 * 16 + 18) * 65536
    assert bench.flops_per_inst_iter(64, 64) == (10 * 12 + 18) * 4096
    assert bench.flops_per_inst_iter(1024, 1024) == (10 * 20 + 18) * 2**20
