"""Writes the FP64 reference of the 1024 x 1024 ADMM precision study (tests/golden/admm1024_rho*.txt).

Workload: 64 x 64 half-wavelength array, N = 1024 random elements, L1 = L2 = 1024, K = 20
off-grid sources, 15 dB (synth.workload_snapshot("admm1024", 0), seed 4000), lam = 0.05 ||A^H y||_inf,
ADMM (eq:admm) for 2000 iterations at rho = 0.5 (the stated value) and rho = N = 1024 (a
well-scaled one).  The measurements are the complex64-rounded y, as the GPU paths receive
them.  Only oracle/ computes: oracle.admm_kron, the dense ADMM with the products taken through
the Kronecker factors of D (A would be 16 GiB), pinned against the dense oracle by
tests/test_oracle_kron.py.

Each file stores the norms of z, c, v, every nonzero of z^(T), the entries whose threshold
argument lies within 1e-5 max|u| of lam/rho (reading A13), and 1024 seeded sample entries of
c^(T) and v^(T).  Run: python tests/golden/make_admm1024.py  (about 3 minutes per rho on 8 cores)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402

ITERS, LAM_FRAC, SAMPLES = 2000, 0.05, 1024


def read(rho_tag):
    """The stored reference for rho_tag '0p5' or '1024' as a dict: lam, rho, iters, the norms
    norm_z / norm_c / norm_v, z_idx / z_val (every nonzero of z^(T)), near (entries within 1e-5
    max|u| of the threshold), s_idx / s_c / s_v (the sampled entries of c^(T) and v^(T))."""
    ref = {}
    with open(os.path.join(HERE, f"admm1024_rho{rho_tag}.txt")) as f:
        lines = [ln.split() for ln in f if not ln.startswith("#")]
    it = iter(lines)
    for key in ("lam", "rho", "iters", "norm_z", "norm_c", "norm_v"):
        k, v = next(it)
        assert k == key, (k, key)
        ref[key] = float(v)
    k, n = next(it)
    assert k == "z_nonzeros"
    rows = [next(it) for _ in range(int(n))]
    ref["z_idx"] = np.array([int(r[0]) for r in rows], np.int64)
    ref["z_val"] = np.array([float(r[1]) + 1j * float(r[2]) for r in rows])
    k, n = next(it)
    assert k == "near_threshold"
    ref["near"] = np.array([int(next(it)[0]) for _ in range(int(n))], np.int64)
    k, n = next(it)
    assert k == "samples"
    rows = [next(it) for _ in range(int(n))]
    ref["s_idx"] = np.array([int(r[0]) for r in rows], np.int64)
    ref["s_c"] = np.array([float(r[1]) + 1j * float(r[2]) for r in rows])
    ref["s_v"] = np.array([float(r[3]) + 1j * float(r[4]) for r in rows])
    return ref


def errors(z, c, ref):
    """Relative errors of a solve's z^(T) (in full) and c^(T) (on the samples, and in norm)."""
    z_ref = np.zeros(z.size, np.complex128)
    z_ref[ref["z_idx"]] = ref["z_val"]
    nz = np.linalg.norm(z_ref)
    ez = np.linalg.norm(z - z_ref) / nz if nz > 0 else float(np.linalg.norm(z))
    ec = np.linalg.norm(c[ref["s_idx"]] - ref["s_c"]) / np.linalg.norm(ref["s_c"])
    en = abs(np.linalg.norm(c) - ref["norm_c"]) / ref["norm_c"]
    return dict(z=float(ez), c_samples=float(ec), c_norm=float(en))


def reference(rho):
    import oracle

    s = synth.workload_snapshot("admm1024", 0)
    y = s.y.astype(np.complex64).astype(np.complex128)
    K = oracle.KronDictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
    lam = LAM_FRAC * float(np.abs(K.adjoint(y)).max())
    z, c, v, u = oracle.admm_kron(K, y, lam, rho, ITERS)
    return s, lam, z, c, v, u


def write(rho, path):
    s, lam, z, c, v, u = reference(rho)
    kappa = lam / rho
    near = np.flatnonzero(np.abs(np.abs(u) - kappa) <= 1e-5 * np.abs(u).max())
    idx = np.sort(np.random.Generator(np.random.PCG64(4242)).choice(c.size, SAMPLES, replace=False))
    with open(path, "w") as f:
        f.write(f"# FP64 ADMM reference, 1024x1024 precision study, rho = {rho!r}; written by make_admm1024.py\n")
        f.write(f"# seed 4000 (synth.workload_snapshot('admm1024', 0)), iters {ITERS}, lam = {LAM_FRAC} ||A^H y||_inf\n")
        f.write(f"lam {float(lam)!r}\nrho {float(rho)!r}\niters {ITERS}\n")
        for name, x in (("z", z), ("c", c), ("v", v)):
            f.write(f"norm_{name} {float(np.linalg.norm(x))!r}\n")
        nz = np.flatnonzero(z)
        f.write(f"z_nonzeros {nz.size}\n")
        for i in nz:
            f.write(f"{int(i)} {float(z[i].real)!r} {float(z[i].imag)!r}\n")
        f.write(f"near_threshold {near.size}\n")
        for i in near:
            f.write(f"{int(i)}\n")
        f.write(f"samples {idx.size}\n")
        for i in idx:
            f.write(f"{int(i)} {float(c[i].real)!r} {float(c[i].imag)!r} {float(v[i].real)!r} {float(v[i].imag)!r}\n")


if __name__ == "__main__":
    for rho, tag in ((0.5, "0p5"), (1024.0, "1024")):
        write(rho, os.path.join(HERE, f"admm1024_rho{tag}.txt"))
        print("wrote rho", rho, flush=True)
