"""Parity of the CUDA peak extraction / harmonic-to-angle map (Section II-A) with the
oracle: indices, counts, magnitudes and harmonics bit-exact, angles to FP64 rounding."""
import numpy as np
import pytest

from gpu_util import inst
from oracle import peaks as opk
import synth

pytestmark = pytest.mark.gpu

ANG_TOL = 1e-14  # two libm implementations of asin/atan2 in FP64


def _solver(lib, shapes, prec="f32", algo="fista"):
    snaps = []
    for k, (L1, L2) in enumerate(shapes):
        M1, M2 = max(2, L1 // 8), max(2, L2 // 8)
        snaps.append(synth.make_snapshot(900 + k, M1, M2, max(2, (M1 * M2) // 3), L1, L2, K=5, snr_db=20.0))
    return lib.BatchSolver([inst(s, 0.1, True) for s in snaps], algo, prec=prec), snaps


def _compare(solver, c_host, K, rel, out):
    import torch

    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    for i, grid in enumerate(solver.unpack(c_host)):
        ref = opk.peaks(grid, K, rel)
        assert got["count"][i] == ref["count"], f"instance {i}: count {got['count'][i]} vs {ref['count']}"
        assert np.array_equal(got["idx"][i], ref["idx"]), f"instance {i}: idx differ"
        assert np.array_equal(got["mag"][i], ref["mag"]), f"instance {i}: |c| differ"
        assert np.array_equal(got["harm"][i], ref["harm"], equal_nan=True), f"instance {i}: harmonics differ"
        nan_g, nan_r = np.isnan(got["ang"][i]), np.isnan(ref["ang"])
        assert np.array_equal(nan_g, nan_r), f"instance {i}: visible-region decisions differ"
        assert np.allclose(got["ang"][i][~nan_g], ref["ang"][~nan_r], rtol=0, atol=ANG_TOL)


@pytest.mark.parametrize("K,rel", [(16, 0.05), (1, 0.0), (1024, 0.0), (40, 1.0)])
def test_peaks_of_solved_batch(lib, K, rel):
    import torch

    solver, _ = _solver(lib, [(256, 256), (64, 128), (128, 64), (16, 16), (256, 32)])
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    solver.solve(y, 200, c, check=False)
    out = solver.peaks(c, K, rel)
    _compare(solver, c.cpu().numpy(), K, rel, out)


def _synthetic(kind, n, rng):
    if kind == "noise":
        return (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    if kind == "quantised":  # |c|^2 in {0, 1, 4, 9} exactly: ties among neighbours and at the K cut
        return (rng.integers(0, 4, n) * rng.choice(np.array([1, 1j, -1, -1j]), n)).astype(np.complex64)
    if kind == "equal":
        return np.full(n, 1.0 - 1.0j, dtype=np.complex64)
    if kind == "zero":
        return np.zeros(n, dtype=np.complex64)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["noise", "quantised", "equal", "zero"])
@pytest.mark.parametrize("K", [7, 300, 1024])
def test_peaks_synthetic_grids(lib, kind, K):
    import torch

    solver, _ = _solver(lib, [(256, 256), (128, 256), (32, 16)])
    rng = np.random.default_rng(5 + K)
    c_host = _synthetic(kind, solver.total_c, rng)
    out = solver.peaks(torch.from_numpy(c_host).cuda(), K, 0.0)
    _compare(solver, c_host, K, 0.0, out)


def test_checkerboard_of_equal_peaks_takes_lowest_indices(lib):
    import torch

    solver, _ = _solver(lib, [(64, 64)])
    g = np.zeros((64, 64), dtype=np.complex64)
    g[0::2, 0::2] = 3.0j  # 1024 isolated equal peaks
    out = solver.peaks(torch.from_numpy(g.reshape(-1)).cuda(), 100, 0.0)
    _compare(solver, g.reshape(-1), 100, 0.0, out)
    idx = out["idx"].cpu().numpy()[0]
    assert out["count"].cpu().numpy()[0] == 1024
    assert np.array_equal(idx, np.flatnonzero(np.abs(g.reshape(-1)) > 0)[:100])


def test_peaks_fp64_solver(lib):
    import torch

    solver, _ = _solver(lib, [(64, 64), (128, 32)], prec="f64")
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex128, device="cuda")
    solver.solve(y, 100, c, check=False)
    out = solver.peaks(c, 24, 0.02)
    _compare(solver, c.cpu().numpy(), 24, 0.02, out)


def test_peaks_invalid_arguments(lib):
    import torch

    solver, _ = _solver(lib, [(32, 32)])
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    for K, rel in ((0, 0.0), (1025, 0.0), (4, 1.5), (4, -0.1)):
        with pytest.raises(lib.BccbError):
            solver.peaks(c, K, rel)
