"""The boundary calls that report per-instance scalars and statuses, through the C ABI:
bccb_mu (eq:ista's step size, before any solve), bccb_create's precision argument, the
per-instance KKT status of bccb_batch_solve / bccb_batch_status (BCCB_ERR_KKT), and the
batch argument of the unrolled network."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_parity, inst, oracle_run

pytestmark = pytest.mark.gpu


def _folded_count_max(s):
    m1, m2 = oracle.element_positions(s.mask, s.M1)
    cnt = np.zeros((s.L2, s.L1))
    np.add.at(cnt, (m2 % s.L2, m1 % s.L1), 1.0)
    return cnt.max()


def test_mu_before_and_after_a_solve(lib):
    """mu = 1/max Lambda = 1/(L1 L2 max folded count) (eq:lambda closed form), read before any
    solve and equal to the value the solve reports."""
    import torch

    snaps = [synth.workload_snapshot("fista64", 0), synth.make_snapshot(91, 20, 6, 50, 16, 32, 2, 10.0)]  # 2nd folds
    solver = lib.BatchSolver([inst(s, 0.1, True) for s in snaps], "fista")
    mu = solver.mu()
    for i, s in enumerate(snaps):
        assert mu[i] == pytest.approx(1.0 / (s.L1 * s.L2 * _folded_count_max(s)), rel=1e-12)
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    solver.solve(y, 5, c)
    np.testing.assert_array_equal(solver.results()["mu"], mu)
    np.testing.assert_array_equal(solver.mu(), mu)


def test_create_with_fp64_precision(lib):
    """bccb_create(..., prec = BCCB_F64, ...) solves in complex128 to the FP64 path's bar."""
    import torch

    s = synth.workload_snapshot("fista64", 0)
    h = lib.bccb_create(s.M1, s.M2, s.mask, s.L1, s.L2, lib.FISTA, 1.0, None, lib.F64)
    try:
        y = torch.from_numpy(s.y.astype(np.complex128)).cuda()
        c = torch.zeros(s.L1 * s.L2, dtype=torch.complex128, device="cuda")
        kkt, _ = lib.bccb_solve(h, y, 0.1, True, 300, None, c)
        ref = oracle_run(s, "fista", 300)
        assert_parity(c.cpu().numpy(), ref, tol=1e-10, what="bccb_create FP64")
        assert kkt == pytest.approx(oracle.kkt_residual(ref["A"], s.y, c.cpu().numpy(), ref["lam"]), rel=1e-9)
    finally:
        lib.bccb_destroy(h)


def test_kkt_status_per_instance(lib):
    """status_out marks exactly the instances whose FP64 relative KKT residual exceeds the
    tolerance; the call returns BCCB_ERR_KKT and still writes every result."""
    import torch

    snaps = [synth.workload_snapshot("fista64", i) for i in range(4)]
    lams = [0.1 * oracle.lambda_max(oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2), s.y) for s in snaps]
    solver = lib.BatchSolver([inst(s, l) for s, l in zip(snaps, lams)], "fista")
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    solver.solve(y, 60, c)
    kkt = solver.results()["kkt"]
    ks = np.sort(kkt)
    assert ks[0] < ks[-1]
    tol = float(np.sqrt(ks[1] * ks[2]))  # two instances on each side
    lib.bccb_set_kkt_tol(solver.handle, tol)
    status = np.full(4, -1, np.int32)
    c2 = torch.zeros_like(c)
    st = lib.bccb_batch_solve(solver.handle, y, 60, None, c2, None, False, status)
    exp = np.where(kkt <= tol, lib.OK, lib.ERR_KKT)
    np.testing.assert_array_equal(status, exp)
    assert st == lib.ERR_KKT
    assert torch.equal(c, c2)  # results written as without the status
    np.testing.assert_array_equal(lib.bccb_batch_status(solver.handle, 4), exp)
    # every instance passes a loose tolerance: OK overall
    lib.bccb_set_kkt_tol(solver.handle, 10.0 * ks[-1])
    assert lib.bccb_batch_solve(solver.handle, y, 60, None, c2, None, False, status) == lib.OK
    assert np.all(status == lib.OK)
    with pytest.raises(lib.BccbError) as e:
        lib.bccb_set_kkt_tol(solver.handle, 0.0)
    assert e.value.status == lib.ERR_INVALID_ARG


def test_status_refused_inside_capture_and_without_check(lib):
    import torch

    s = synth.workload_snapshot("fista64", 0)
    stream = torch.cuda.Stream()
    solver = lib.BatchSolver([inst(s, 0.1, True)], "fista", stream=stream)
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    solver.solve(y, 10, c, check=False)
    with pytest.raises(lib.BccbError) as e:
        lib.bccb_batch_status(solver.handle, 1)
    assert e.value.status == lib.ERR_INVALID_ARG
    status = np.zeros(1, np.int32)
    with torch.cuda.stream(stream):
        g = torch.cuda.CUDAGraph()
        with pytest.raises(lib.BccbError) as e:
            with torch.cuda.graph(g, stream=stream):
                lib.bccb_batch_solve(solver.handle, y, 10, None, c, None, True, status)
        assert e.value.status == lib.ERR_INVALID_ARG


def test_unrolled_batch_argument_checked(lib):
    import torch

    s = synth.workload_snapshot("fista64", 0)
    solver = lib.BatchSolver([inst(s, 0.1, True)] * 2, "fista")
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=torch.complex64, device="cuda")
    ones = torch.ones(4, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.BccbError) as e:
        lib.bccb_unrolled_fwd(solver.handle, y, 3, 4, ones, ones, c)
    assert e.value.status == lib.ERR_INVALID_ARG
    lib.bccb_unrolled_fwd(solver.handle, y, 2, 4, ones, ones, c, None, True)
    assert lib.bccb_batch_status(solver.handle, 2).shape == (2,)
    plain = torch.zeros_like(c)
    solver.solve(y, 4, plain, check=False)
    assert torch.equal(c, plain)  # unit multipliers: plain FISTA
