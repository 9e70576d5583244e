"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on the same
seeded inputs (complex64 on the GPU, complex128 in the oracle)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_parity, gpu_run, inst, oracle_run, rel_err

pytestmark = pytest.mark.gpu


def _snap(seed, M1, M2, N, L1, L2, K=3, snr=15.0, lam_frac=0.1, **kw):
    s = synth.make_snapshot(seed, M1, M2, N, L1, L2, K, snr, **kw)
    s.lam_frac = lam_frac
    return s


# ------------------------------------------------------------------------------------------
# setup rows: Lambda (eq:lambda), b = A^H y, mu (eq:ista), lam = frac ||A^H y||_inf
# ------------------------------------------------------------------------------------------


@pytest.mark.parametrize("M1,M2,N,L1,L2", [(16, 16, 64, 64, 64), (8, 4, 12, 16, 32), (24, 6, 50, 16, 64),
                                           (32, 32, 256, 256, 256), (20, 40, 300, 32, 32)])
def test_setup_lambda_b_mu(lib, M1, M2, N, L1, L2):
    import torch

    s = _snap(100 + L1 + L2, M1, M2, N, L1, L2)
    A = oracle.dictionary(s.mask, M1, M2, L1, L2)
    lam_ref = oracle.gram_eigenvalues(A, L1, L2).real.reshape(-1)
    b_ref = oracle.adjoint_measurements(A, s.y)
    run = gpu_run(lib, [s], [0.1], "fista", 1)
    solver = run["solver"]
    lam_gpu = torch.zeros(L1 * L2, dtype=torch.float64, device="cuda")
    b_gpu = torch.zeros(L1 * L2, dtype=torch.complex128, device="cuda")
    solver.get(lib.GET_LAMBDA, lam_gpu)
    solver.get(lib.GET_B, b_gpu)
    torch.cuda.synchronize()
    assert np.abs(lam_gpu.cpu().numpy() - lam_ref).max() <= 1e-9 * lam_ref.max()
    # y enters the GPU as complex64, so b carries that rounding (about 6e-8 relative)
    assert rel_err(b_gpu.cpu().numpy(), b_ref) <= 1e-6
    assert abs(run["res"]["mu"][0] * oracle.step_size(A) ** -1 - 1.0) <= 1e-12


def test_shared_mask_batch_shares_lambda(lib):
    """Instances with the same array and grid take Lambda from one transform: each one's
    Lambda, mu and solution equal those of a one-instance solve bit for bit, and instances
    on another mask or grid keep their own."""
    import torch

    rng = np.random.Generator(np.random.PCG64(77))
    shared = synth.make_mask(rng, 16, 12, 60)
    other = synth.make_mask(rng, 16, 12, 60)
    snaps = [_snap(700 + i, 16, 12, 60, 64, 32, mask=m, K=3, snr=20.0)
             for i, m in enumerate([shared, shared, other, shared, other])]
    snaps.append(_snap(706, 16, 12, 60, 32, 32, mask=shared, K=2, snr=20.0))  # same mask, other grid
    refs = [oracle_run(s, "fista", 60) for s in snaps]
    run = gpu_run(lib, snaps, [r["lam"] for r in refs], "fista", 60)
    lam_all = torch.zeros(run["solver"].total_c, dtype=torch.float64, device="cuda")
    run["solver"].get(lib.GET_LAMBDA, lam_all)
    lam_all = lam_all.cpu().numpy()
    for i, (s, r) in enumerate(zip(snaps, refs)):
        assert_parity(run["c"][i], r, what=f"shared-mask batch instance {i}")
        one = gpu_run(lib, [s], [r["lam"]], "fista", 60)
        lam_one = torch.zeros(s.L1 * s.L2, dtype=torch.float64, device="cuda")
        one["solver"].get(lib.GET_LAMBDA, lam_one)
        o, L1, L2 = run["solver"].offsets[i]
        assert np.array_equal(lam_all[o:o + L1 * L2], lam_one.cpu().numpy()), f"Lambda of instance {i}"
        assert run["res"]["mu"][i] == one["res"]["mu"][0]
        assert run["res"]["kkt"][i] == pytest.approx(one["res"]["kkt"][0], rel=1e-6, abs=1e-9)


def test_lambda_fraction_of_lmax(lib):
    s = synth.workload_snapshot("fista64", 3)
    A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
    run = gpu_run_frac(lib, s, 0.1)
    assert abs(run["res"]["lam"][0] / (0.1 * oracle.lambda_max(A, s.y)) - 1.0) <= 1e-6


def gpu_run_frac(lib, s, frac):
    import torch

    solver = lib.BatchSolver([inst(s, frac, lam_is_frac=True)], "fista")
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    solver.solve(y, 5, c)
    return dict(res=solver.results())


# ------------------------------------------------------------------------------------------
# full-size single-snapshot workloads
# ------------------------------------------------------------------------------------------


def test_fista_64x64_500_iterations(lib):
    """Plain FISTA, 16x16 array, N=64, 64x64 grid, 3 on-grid sources, 20 dB, 500 iterations."""
    s = synth.workload_snapshot("fista64", 0)
    ref = oracle_run(s, "fista", 500)
    run = gpu_run(lib, [s], [ref["lam"]], "fista", 500)
    assert_parity(run["c"][0], ref, what="fista 64x64")
    assert run["res"]["kkt"][0] == pytest.approx(oracle.kkt_residual(ref["A"], s.y, run["c"][0].astype(np.complex128), ref["lam"]), abs=1e-4)


@pytest.mark.parametrize("algo,rho", [("ista", 1.0), ("fista", 1.0), ("admm", 1.0), ("admm", 256.0)])
def test_256x256_1000_iterations(lib, algo, rho):
    """32x32 array, N=256, 256x256 grid, 8 off-grid sources, 10 dB, 1000 iterations (ADMM with
    rho = 1 as specified, and with rho = 256 = N, where ADMM actually moves z off 0)."""
    s = synth.workload_snapshot("solve256", 0)
    ref = oracle_run(s, algo, 1000, rho=rho)
    run = gpu_run(lib, [s], [ref["lam"]], algo, 1000, rho=rho)
    assert_parity(run["c"][0], ref, what=f"{algo} 256x256 rho={rho}")
    if algo == "admm":
        # c^(T) = u - v^(T-1) with |u| ~ |v|; at rho = 1 ||v||/||c|| is about T, so FP32 keeps
        # log2(T) fewer bits of c than of u and v: allow 16 ulps of ||v|| relative to ||c||.
        ratio = np.linalg.norm(ref["u"] - ref["aux"]) / np.linalg.norm(ref["aux"])
        tol = max(1e-4, 16 * 2.0**-24 * ratio)
        assert_parity(run["aux"][0], ref, ref_c=ref["aux"], tol=tol, what=f"admm c^(T) rho={rho} tol={tol:.1e}")


# ------------------------------------------------------------------------------------------
# every grid shape class (cluster sizes 1, 2, 4, 8) and non-square grids
# ------------------------------------------------------------------------------------------

SHAPES = [(16, 16), (32, 16), (16, 64), (64, 32), (128, 64), (256, 32), (32, 256), (128, 128), (256, 128),
          (128, 256), (64, 256)]


@pytest.mark.parametrize("algo", ["ista", "fista", "admm"])
@pytest.mark.parametrize("L1,L2", SHAPES)
def test_shapes(lib, algo, L1, L2):
    M1, M2 = max(2, L1 // 4), max(2, L2 // 4)
    s = _snap(7 * L1 + L2, M1, M2, max(1, (M1 * M2) // 4), L1, L2, K=4, snr=12.0, lam_frac=0.08)
    iters = 150
    ref = oracle_run(s, algo, iters, rho=4.0)
    run = gpu_run(lib, [s], [ref["lam"]], algo, iters, rho=4.0)
    assert_parity(run["c"][0], ref, what=f"{algo} {L1}x{L2}")


@pytest.mark.parametrize("algo", ["fista", "admm"])
@pytest.mark.parametrize("M1,L2", [(8, 32), (16, 64), (30, 32), (48, 128), (100, 32), (300, 16)])
def test_row256_active_column_counts(lib, algo, M1, L2):
    """Rows of 256 use a specialised transform whose work depends on how many 16-wide
    blocks of Fourier columns the element mask reaches (1, 2, 3, 7 and all 16; the
    last two masks are wider than the grid and fold)."""
    M2 = 4
    s = _snap(500 + M1 + L2, M1, M2, max(2, (M1 * M2) // 5), 256, L2, K=3, snr=15.0, lam_frac=0.08)
    ref = oracle_run(s, algo, 100, rho=16.0)
    run = gpu_run(lib, [s], [ref["lam"]], algo, 100, rho=16.0)
    assert_parity(run["c"][0], ref, what=f"{algo} M1={M1} 256x{L2}")


@pytest.mark.parametrize("algo", ["fista", "admm"])
@pytest.mark.parametrize("M2", [32, 40, 56, 72])
def test_middle_stage_row_support(lib, algo, M2, tmp_path):
    """The cross-CTA stage forms only the first two frequencies of its 16-point butterflies
    on a CTA whose spectrum lies in rows k2 < 32 of the 256-row grid, the full butterfly
    elsewhere: M2 = 32 puts every CTA on the short form, 40 mixes the two forms in one cluster
    (k2 < 40: the CTAs with k1 < 8 need q = 2), 56 and 72 put every CTA on the full form.
    Both tiles."""
    import torch

    s = _snap(800 + M2, 12, M2, (12 * M2) // 4, 256, 256, K=3, snr=15.0, lam_frac=0.08)
    ref = oracle_run(s, algo, 120, rho=16.0)
    for tile in (8192, 4096):
        cache = tmp_path / f"tiles_{tile}.txt"
        cache.write_text(f"{_gpu_name()} 256 256 {int(algo == 'admm')} {tile}\n")
        solver = lib.BatchSolver([inst(s, ref["lam"])], algo, 16.0)
        y = torch.from_numpy(solver.y_host).cuda()
        lib.bccb_batch_tune(solver.handle, y, 5, str(cache))
        assert lib.bccb_batch_tile(solver.handle, 256, 256) == tile
        c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
        solver.solve(y, 120, c, check=False)
        assert_parity(c.cpu().numpy(), ref, what=f"{algo} M2={M2} tile {tile}")


# ------------------------------------------------------------------------------------------
# batched, ragged shapes in one call
# ------------------------------------------------------------------------------------------


def test_ragged_batch_matches_oracle(lib):
    snaps = synth.workload_batch("ragged", 10)
    refs = [oracle_run(s, "fista", 200) for s in snaps]
    run = gpu_run(lib, snaps, [r["lam"] for r in refs], "fista", 200)
    for i, (c, r) in enumerate(zip(run["c"], refs)):
        assert_parity(c, r, what=f"batch instance {i} ({snaps[i].L1}x{snaps[i].L2})")
        assert run["res"]["kkt"][i] == pytest.approx(
            oracle.kkt_residual(r["A"], snaps[i].y, c.astype(np.complex128), r["lam"]), abs=1e-4)
        assert run["res"]["objective"][i] == pytest.approx(
            oracle.objective(r["A"], snaps[i].y, c.astype(np.complex128), r["lam"]), rel=1e-5)


# ------------------------------------------------------------------------------------------
# autotuned tiles and CUDA-graph replay
# ------------------------------------------------------------------------------------------


def _gpu_name():
    import torch

    return torch.cuda.get_device_name().replace(" ", "_")


@pytest.mark.parametrize("algo", ["fista", "admm"])
def test_both_tiles_match_oracle(lib, algo, tmp_path):
    """Every tile the autotuner may pick (8192 or 4096 grid elements per CTA) gives the
    oracle's iterates; the tile is forced through the tuner's cache file."""
    import torch

    snaps = [synth.workload_snapshot("solve256", 3), synth.make_snapshot(91, 16, 32, 128, 64, 128, 3, 15.0),
             synth.make_snapshot(92, 32, 16, 128, 256, 64, 3, 15.0)]
    refs = [oracle_run(s, algo, 120, rho=8.0) for s in snaps]
    for tile in (8192, 4096):
        cache = tmp_path / f"tiles_{tile}.txt"
        cache.write_text("".join(f"{_gpu_name()} {s.L1} {s.L2} {int(algo == 'admm')} {tile}\n" for s in snaps))
        solver = lib.BatchSolver([inst(s, r["lam"]) for s, r in zip(snaps, refs)], algo, 8.0)
        y = torch.from_numpy(solver.y_host).cuda()
        lib.bccb_batch_tune(solver.handle, y, 5, str(cache))
        for s in snaps:
            assert lib.bccb_batch_tile(solver.handle, s.L1, s.L2) == tile
        c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
        solver.solve(y, 120, c, check=False)
        for i, (g, r) in enumerate(zip(solver.unpack(c.cpu().numpy()), refs)):
            assert_parity(g.reshape(-1), r, what=f"{algo} tile {tile} instance {i}")


def test_tuner_measures_and_caches(lib, tmp_path):
    import torch

    snaps = synth.workload_batch("ragged", 12, first=40)
    solver = lib.BatchSolver([inst(s, 0.1, lam_is_frac=True) for s in snaps], "fista")
    y = torch.from_numpy(solver.y_host).cuda()
    cache = tmp_path / "tiles.txt"
    lib.bccb_batch_tune(solver.handle, y, 10, str(cache))
    lines = cache.read_text().split("\n")
    shapes = {(s.L1, s.L2) for s in snaps}
    assert len([ln for ln in lines if ln.strip()]) == len(shapes)
    for (L1, L2) in shapes:
        assert lib.bccb_batch_tile(solver.handle, L1, L2) in (8192, 4096)


def test_graph_replay_matches_direct_solve(lib):
    import torch

    snaps = synth.workload_batch("ragged", 9, first=60)
    solver = lib.BatchSolver([inst(s, 0.1, lam_is_frac=True) for s in snaps], "fista",
                             stream=torch.cuda.Stream())
    y = torch.from_numpy(solver.y_host).cuda()
    direct = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    replay = torch.full_like(direct, 3.0)
    torch.cuda.synchronize()  # the solver runs on its own stream
    solver.solve(y, 150, direct, check=True)
    res_direct = solver.results()
    lib.bccb_batch_capture(solver.handle, y, 150, None, replay, None, True)
    for _ in range(2):
        lib.bccb_batch_replay(solver.handle)
        res = solver.results()  # synchronises the solver's stream
        assert torch.equal(replay, direct)
        np.testing.assert_array_equal(res["kkt"], res_direct["kkt"])
        replay.fill_(5.0)
        torch.cuda.synchronize()
    lib.bccb_batch_replay(solver.handle)
    solver.results()
    assert torch.equal(replay, direct)


# ------------------------------------------------------------------------------------------
# edge cases
# ------------------------------------------------------------------------------------------


def test_single_element_and_full_mask(lib):
    s1 = _snap(41, 5, 4, 1, 16, 16, K=1, snr=None)
    s2 = _snap(42, 6, 5, 30, 32, 16, K=2, snr=20.0)
    for s in (s1, s2):
        for algo in ("fista", "admm"):
            ref = oracle_run(s, algo, 80, rho=2.0)
            run = gpu_run(lib, [s], [ref["lam"]], algo, 80, rho=2.0)
            assert_parity(run["c"][0], ref, what=f"{algo} N={s.N}")


def test_folded_mask_wider_than_grid(lib):
    """M1 > L1 and M2 > L2: the Gram is still BCCB with folded counts in Lambda."""
    s = _snap(43, 24, 20, 60, 16, 16, K=2, snr=20.0)
    for algo in ("ista", "fista", "admm"):
        ref = oracle_run(s, algo, 120, rho=50.0)
        run = gpu_run(lib, [s], [ref["lam"]], algo, 120, rho=50.0)
        assert_parity(run["c"][0], ref, what=f"{algo} folded")


def test_lambda_zero_and_above_lmax(lib):
    s = _snap(44, 8, 8, 20, 32, 32, K=2, snr=10.0)
    A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
    lmax = oracle.lambda_max(A, s.y)
    # lam = 0: one ISTA step gives A^H y / (L1 L2)
    ref = oracle_run(s, "ista", 1, lam=0.0, A=A)
    run = gpu_run(lib, [s], [0.0], "ista", 1)
    assert rel_err(run["c"][0], ref["c"]) <= 1e-5
    # lam above ||A^H y||_inf: the solution is exactly zero for every algorithm
    for algo in ("ista", "fista", "admm"):
        run = gpu_run(lib, [s], [1.01 * lmax], algo, 30)
        assert np.count_nonzero(run["c"][0]) == 0


def test_one_iteration_and_warm_start(lib):
    s = _snap(45, 8, 8, 24, 64, 16, K=3, snr=15.0)
    ref1 = oracle_run(s, "fista", 1)
    run1 = gpu_run(lib, [s], [ref1["lam"]], "fista", 1)
    assert_parity(run1["c"][0], ref1, what="fista 1 iteration")
    # ISTA is memoryless: 40 iterations warm-started from 60 equal 100 from zero
    ref = oracle_run(s, "ista", 100)
    first = gpu_run(lib, [s], [ref["lam"]], "ista", 60)
    second = gpu_run(lib, [s], [ref["lam"]], "ista", 40, c0=first["c"][0])
    assert_parity(second["c"][0], ref, what="ista warm start")


def test_host_entry_point_matches_device(lib):
    snaps = synth.workload_batch("ragged", 3, first=20)
    lams = [0.1 * oracle.lambda_max(oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2), s.y) for s in snaps]
    dev = gpu_run(lib, snaps, lams, "fista", 50)
    solver = dev["solver"]
    out = np.zeros(solver.total_c, np.complex64)
    solver.solve_host(solver.y_host, 50, out)
    np.testing.assert_array_equal(np.concatenate(dev["c"]), out)


def _solve_dev_and_host(lib, insts, masks, y, total_c, iters):
    """Device solve and host-buffer solves (pageable numpy, pinned torch) on one solver."""
    import torch

    h = lib.bccb_batch_create(insts, masks, lib.ALGOS["fista"])
    try:
        y_dev = torch.from_numpy(y).cuda()
        c_dev = torch.zeros(total_c, dtype=torch.complex64, device="cuda")
        lib.bccb_batch_solve(h, y_dev, iters, None, c_dev, None, True)
        torch.cuda.synchronize()
        dev = c_dev.cpu().numpy()
        kkt_dev = lib.bccb_batch_results(h, len(insts))["kkt"]
        pageable = np.full(total_c, np.nan, np.complex64)
        lib.bccb_batch_solve_host(h, y, iters, pageable, True)
        kkt_host = lib.bccb_batch_results(h, len(insts))["kkt"]
        y_pin = torch.from_numpy(y).pin_memory()
        c_pin = torch.full((total_c,), float("nan"), dtype=torch.complex64).pin_memory()
        lib.bccb_batch_solve_host_ptr(h, y_pin.data_ptr(), iters, c_pin.data_ptr(), True)
        return dev, pageable, c_pin.numpy().copy(), kkt_dev, kkt_host
    finally:
        lib.bccb_destroy(h)


@pytest.mark.parametrize("layout", ["packed", "reversed", "gaps"])
def test_host_entry_point_streams_chunks(lib, layout):
    """A batch of one shape class with at least 64 instances is solved in chunks whose results
    are copied back while later chunks run; every layout of c_out (packed, instances in reverse
    order, gaps between instances, which falls back to one copy) gives the device result."""
    snaps = [_snap(900 + i, 12, 12, 40, 64, 64, K=2, snr=20.0) for i in range(80)]
    insts, masks, y, total_c = lib.pack([inst(s, 0.1, True) for s in snaps])
    L = 64 * 64
    if layout == "reversed":
        for i, q in enumerate(insts):
            q.c_off = (len(insts) - 1 - i) * L
    elif layout == "gaps":
        for i, q in enumerate(insts):
            q.c_off = i * (L + 48)
        total_c = len(insts) * (L + 48)
    dev, pageable, pinned, kkt_dev, kkt_host = _solve_dev_and_host(lib, insts, masks, y, total_c, 40)
    cells = np.zeros(total_c, bool)
    for q in insts:
        cells[q.c_off:q.c_off + L] = True
    np.testing.assert_array_equal(pageable[cells], dev[cells])
    np.testing.assert_array_equal(pinned[cells], dev[cells])
    np.testing.assert_array_equal(kkt_host, kkt_dev)
    # spot parity with the oracle on two instances
    for i in (0, 79):
        ref = oracle_run(snaps[i], "fista", 40)
        q = insts[i]
        assert_parity(pinned[q.c_off:q.c_off + L], ref, what=f"{layout} instance {i}")


# ------------------------------------------------------------------------------------------
# argument checks (no kernel runs for these)
# ------------------------------------------------------------------------------------------


def test_invalid_arguments(lib):
    s = _snap(46, 4, 4, 6, 16, 16)
    good = inst(s, 0.1)
    for bad, status in [(dict(good, L1=48), lib.ERR_UNSUPPORTED), (dict(good, L2=2048), lib.ERR_UNSUPPORTED),
                        (dict(good, L1=4), lib.ERR_UNSUPPORTED),
                        (dict(good, mask=np.zeros(16, np.uint8)), lib.ERR_INVALID_ARG),
                        (dict(good, lam=-1.0), lib.ERR_INVALID_ARG)]:
        with pytest.raises(lib.BccbError) as e:
            lib.BatchSolver([bad], "fista")
        assert e.value.status == status
    with pytest.raises(lib.BccbError) as e:
        lib.BatchSolver([good], "admm", rho=0.0)
    assert e.value.status == lib.ERR_INVALID_ARG
    with pytest.raises(lib.BccbError) as e:
        lib.BatchSolver([good], 7)
    assert e.value.status == lib.ERR_INVALID_ARG
    import torch

    solver = lib.BatchSolver([good], "fista")
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.BccbError) as e:
        solver.solve(y, 0, c)
    assert e.value.status == lib.ERR_INVALID_ARG
