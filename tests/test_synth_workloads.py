"""The seeded input generators draw what the workloads state (the signal model of Section II-A,
eq:signal_model, on a sparse half-wavelength array): masks, source counts and ranges, amplitudes,
noise at the stated SNR, the ragged batch's shape mix and the fixed array of the learned workload.
The generators hold none of the method's arithmetic; these checks keep the inputs honest."""
import numpy as np
import pytest

import synth


def _clean(s):
    """y without noise, from the snapshot's own sources (the model restated)."""
    m1, m2 = synth.element_positions(s.mask, s.M1)
    phase = np.outer(m1, s.freqs[:, 0]) + np.outer(m2, s.freqs[:, 1])
    return np.exp(-2j * np.pi * phase) @ s.amps


def test_same_seed_same_snapshot_and_distinct_seeds_differ():
    a = synth.make_snapshot(123, 8, 8, 20, 32, 32, 3, 15.0)
    b = synth.make_snapshot(123, 8, 8, 20, 32, 32, 3, 15.0)
    c = synth.make_snapshot(124, 8, 8, 20, 32, 32, 3, 15.0)
    assert np.array_equal(a.mask, b.mask) and np.array_equal(a.y, b.y)
    assert not np.array_equal(a.y, c.y)


def test_mask_keeps_n_positions_without_replacement():
    rng = np.random.Generator(np.random.PCG64(5))
    for M1, M2, N in ((16, 16, 64), (32, 32, 256), (51, 16, 40), (4, 4, 16)):
        m = synth.make_mask(rng, M1, M2, N)
        assert m.dtype == np.uint8 and m.size == M1 * M2 and int(m.sum()) == N
        assert set(np.unique(m)) <= {0, 1}
    with pytest.raises(ValueError):
        synth.make_mask(rng, 4, 4, 17)


def test_fista64_workload_sources_on_grid_with_unit_amplitude_at_20_db():
    s = synth.workload_snapshot("fista64", 0)
    assert (s.M1, s.M2, s.L1, s.L2, s.N) == (16, 16, 64, 64, 64)
    assert s.freqs.shape == (3, 2)
    # on the grid f = -1/2 + l/64, distinct points
    l = (s.freqs + 0.5) * 64
    assert np.allclose(l, np.round(l), atol=1e-12)
    assert len({tuple(x) for x in np.round(l).astype(int)}) == 3
    np.testing.assert_allclose(np.abs(s.amps), 1.0, rtol=0, atol=1e-12)
    # the noise is y - y_clean; its power over the signal's is 10^(-SNR/10) to within the sample
    # error of 64 complex Gaussian draws (relative std 1/8)
    clean = _clean(s)
    ratio = np.mean(np.abs(s.y - clean) ** 2) / np.mean(np.abs(clean) ** 2)
    assert 0.5 * 10 ** (-2.0) <= ratio <= 1.6 * 10 ** (-2.0)


def test_solve256_and_admm1024_workloads_off_grid_cn_amplitudes():
    for name, shape, K in (("solve256", (32, 32, 256, 256, 256), 8), ("admm1024", (64, 64, 1024, 1024, 1024), 20)):
        s = synth.workload_snapshot(name, 1)
        assert (s.M1, s.M2, s.L1, s.L2, s.N) == shape
        assert s.freqs.shape == (K, 2)
        assert np.all(s.freqs >= -0.5) and np.all(s.freqs < 0.5)
        l = (s.freqs + 0.5) * s.L1
        assert not np.allclose(l, np.round(l))  # off the grid
    # CN(0, 1) amplitudes: mean |c|^2 over many draws near 1
    p = np.mean([np.mean(np.abs(synth.workload_snapshot("solve256", i).amps) ** 2) for i in range(200)])
    assert 0.85 <= p <= 1.15


def test_ragged_batch_shape_mix():
    snaps = synth.workload_batch("ragged", 300)
    Ls = {(s.L1, s.L2) for s in snaps}
    assert Ls <= {(a, b) for a in (64, 128, 256) for b in (64, 128, 256)} and len(Ls) == 9
    for s in snaps:
        assert (s.M1, s.M2) == (s.L1 // 4, s.L2 // 4)
        assert s.N == int(round(0.25 * s.M1 * s.M2))
        assert 1 <= s.freqs.shape[0] <= 10
        assert 0.0 <= s.snr_db <= 30.0
        assert s.lam_frac == 0.1
    # a forced square grid (the homogeneous form)
    assert all((s.L1, s.L2) == (256, 256) for s in synth.workload_batch("ragged", 5, L=256))


def test_learned_batch_shares_one_array():
    snaps = synth.workload_batch("learned", 20)
    for s in snaps:
        assert np.array_equal(s.mask, snaps[0].mask)
        assert (s.M1, s.M2, s.L1, s.L2, s.N) == (32, 32, 256, 256, 256)
        assert 1 <= s.freqs.shape[0] <= 8 and 0.0 <= s.snr_db <= 30.0
    assert not np.array_equal(synth.workload_batch("learned", 1, fixed_mask_seed=9)[0].mask, snaps[0].mask)


def test_paper_experiment_shape():
    for L1 in (64, 128, 256, 512):
        s = synth.paper_experiment_snapshot(0, L1)
        assert (s.M1, s.M2, s.N, s.L1, s.L2, s.snr_db) == (51, 16, 40, L1, 32, 15.0)
        assert 1 <= s.freqs.shape[0] <= 10


def test_noiseless_snapshot_is_the_signal_model():
    s = synth.make_snapshot(7, 6, 5, 12, 16, 16, 2, None)
    np.testing.assert_allclose(s.y, _clean(s), rtol=0, atol=1e-12)
