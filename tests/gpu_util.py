"""Helpers shared by the GPU parity tests: run the oracle and the CUDA path on the
same seeded snapshot and compare element by element."""
import numpy as np

import oracle

# Parity bar for the FP32 path against the FP64 oracle: relative l2 error of the
# returned iterate, and identical support apart from entries whose oracle
# soft-threshold argument is within 1e-5 (relative to its max) of the threshold.
REL_TOL = 1e-4
NEAR_THRESHOLD = 1e-5


def inst(s, lam, lam_is_frac=False):
    return dict(M1=s.M1, M2=s.M2, L1=s.L1, L2=s.L2, mask=s.mask, y=s.y, lam=lam, lam_is_frac=lam_is_frac)


def oracle_run(s, algo, iters, lam=None, rho=1.0, A=None):
    """Returns dict(c, u, kappa, A, lam, aux) from the FP64 oracle (c: flat L1*L2)."""
    A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2) if A is None else A
    if lam is None:
        lam = s.lam_frac * oracle.lambda_max(A, s.y)
    aux = None
    if algo == "ista":
        c, u, kappa = oracle.ista(A, s.y, lam, iters, pre=True)
    elif algo == "fista":
        c, u, kappa = oracle.fista(A, s.y, lam, iters, pre=True)
    else:
        c, aux, _v, u, kappa = oracle.admm(A, s.y, lam, rho, iters, pre=True)
    return dict(c=c, u=u, kappa=kappa, A=A, lam=lam, aux=aux)


def gpu_run(lib, snaps, lams, algo, iters, rho=1.0, check=True, c0=None, prec="f32"):
    import torch

    solver = lib.BatchSolver([inst(s, l) for s, l in zip(snaps, lams)], algo, rho, prec=prec)
    cdt = torch.complex128 if prec == "f64" else torch.complex64
    y = torch.from_numpy(solver.y_host).cuda()
    c = torch.zeros(solver.total_c, dtype=cdt, device="cuda")
    aux = torch.zeros_like(c) if algo == "admm" else None
    c0_t = None if c0 is None else torch.from_numpy(np.asarray(c0, solver.dtype)).cuda()
    solver.solve(y, iters, c, c0=c0_t, aux_out=aux, check=check)
    torch.cuda.synchronize()
    res = solver.results() if check else None
    out = [g.reshape(-1) for g in solver.unpack(c.cpu().numpy())]
    aux_out = None if aux is None else [g.reshape(-1) for g in solver.unpack(aux.cpu().numpy())]
    return dict(c=out, aux=aux_out, res=res, solver=solver)


def rel_err(a, b):
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def assert_parity(gpu_c, ref, tol=REL_TOL, ref_c=None, what=""):
    ref_c = ref["c"] if ref_c is None else ref_c
    gpu_c = np.asarray(gpu_c, np.complex128)
    if np.linalg.norm(ref_c) == 0:
        assert np.count_nonzero(gpu_c) == 0, f"{what}: oracle result is 0, GPU has {np.count_nonzero(gpu_c)} nonzeros"
        return 0.0
    err = rel_err(gpu_c, ref_c)
    assert err <= tol, f"{what}: relative l2 error {err:.3e} > {tol:.1e}"
    if ref_c is ref["c"]:
        u = ref["u"]
        near = np.abs(np.abs(u) - ref["kappa"]) <= NEAR_THRESHOLD * np.abs(u).max()
        mismatch = ((np.abs(gpu_c) > 0) != (np.abs(ref_c) > 0)) & ~near
        assert not mismatch.any(), f"{what}: support differs at {np.flatnonzero(mismatch)[:10]}"
    return err
