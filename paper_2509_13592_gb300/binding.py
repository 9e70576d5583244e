"""Python binding of ``libbccb.so`` (the C ABI declared in include/bccb.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  PyTorch supplies device memory and the CUDA stream.  Importing this
package fails loudly when the library has not been built; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbccb.so")

ISTA, FISTA, ADMM = 0, 1, 2
F32, F64 = 0, 1
FFT, DENSE = 0, 1
ALGOS = {"ista": ISTA, "fista": FISTA, "admm": ADMM}
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_KKT, ERR_TIMEOUT = range(6)
GET_LAMBDA, GET_B, GET_MULT, GET_CTERM = 0, 1, 2, 3


class BccbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class bccb_inst_t(ctypes.Structure):
    _fields_ = [
        ("M1", ctypes.c_int32), ("M2", ctypes.c_int32), ("L1", ctypes.c_int32), ("L2", ctypes.c_int32),
        ("mask_off", ctypes.c_int64), ("y_off", ctypes.c_int64), ("c_off", ctypes.c_int64),
        ("lam", ctypes.c_double), ("lam_is_frac", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2509_13592_gb300.build` "
            "(nvcc, sm_103a). There is no CPU fallback.")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    lib.bccb_batch_create.argtypes = [P(vp), P(bccb_inst_t), i32, vp, i32, dbl, vp]
    lib.bccb_batch_create2.argtypes = [P(vp), P(bccb_inst_t), i32, vp, i32, dbl, i32, vp]
    lib.bccb_batch_create_gamma.argtypes = [P(vp), P(bccb_inst_t), i32, vp, i32, dbl, i32, dbl, dbl, vp]
    lib.bccb_batch_solve.argtypes = [vp, vp, i32, vp, vp, vp, i32, vp]
    lib.bccb_set_kkt_tol.argtypes = [vp, dbl]
    lib.bccb_mu.argtypes = [vp, vp]
    lib.bccb_batch_status.argtypes = [vp, vp]
    lib.bccb_batch_solve_host.argtypes = [vp, vp, i32, vp, i32]
    lib.bccb_batch_results.argtypes = [vp, vp, vp, vp, vp]
    lib.bccb_batch_get.argtypes = [vp, i32, vp]
    lib.bccb_create.argtypes = [P(vp), i32, i32, vp, i32, i32, i32, dbl, i32, vp]
    lib.bccb_solve.argtypes = [vp, vp, dbl, i32, i32, vp, vp, vp, P(dbl), P(dbl)]
    lib.bccb_set_timing.argtypes = [vp, i32]
    lib.bccb_last_timing.argtypes = [vp, P(ctypes.c_float), P(ctypes.c_float), P(ctypes.c_float),
                                     P(ctypes.c_int64)]
    lib.bccb_batch_capture.argtypes = [vp, vp, i32, vp, vp, vp, i32]
    lib.bccb_batch_replay.argtypes = [vp]
    lib.bccb_batch_tune.argtypes = [vp, vp, i32, ctypes.c_char_p]
    lib.bccb_batch_tile.argtypes = [vp, i32, i32, P(i32)]
    lib.bccb_batch_variant.argtypes = [vp, i32, i32, P(i32), P(i32)]
    lib.bccb_unrolled_fwd.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, i32]
    lib.bccb_unrolled_bwd.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp]
    lib.bccb_batch_peaks.argtypes = [vp, vp, i32, dbl, vp, vp, vp, vp, vp]
    lib.bccb_batch_set_method.argtypes = [vp, i32]
    lib.bccb_batch_size.argtypes = [vp, P(i32)]
    lib.bccb_instance_shape.argtypes = [vp, i32, P(i32), P(i32), P(i32)]
    lib.bccb_destroy.argtypes = [vp]
    lib.bccb_fp32_fma_rate.argtypes = [i32, i32, vp, P(dbl)]
    lib.bccb_status_string.argtypes = [i32]
    lib.bccb_status_string.restype = ctypes.c_char_p
    lib.bccb_last_error.argtypes = [vp]
    lib.bccb_last_error.restype = ctypes.c_char_p
    for name in ("bccb_batch_create", "bccb_batch_create2", "bccb_batch_solve", "bccb_batch_solve_host", "bccb_batch_results",
                 "bccb_batch_get", "bccb_create", "bccb_solve", "bccb_batch_size", "bccb_instance_shape",
                 "bccb_destroy", "bccb_set_timing", "bccb_last_timing", "bccb_batch_capture", "bccb_batch_replay",
                 "bccb_batch_tune", "bccb_batch_tile", "bccb_unrolled_fwd", "bccb_unrolled_bwd", "bccb_batch_peaks",
                 "bccb_batch_set_method", "bccb_batch_create_gamma", "bccb_set_kkt_tol", "bccb_mu", "bccb_batch_status", "bccb_batch_variant",
                 "bccb_fp32_fma_rate"):
        getattr(lib, name).restype = i32
    return lib


_lib = _load()


def _raise(status: int, handle) -> None:
    if status != OK:
        msg = _lib.bccb_last_error(handle).decode(errors="replace")
        what = _lib.bccb_status_string(status).decode()
        raise BccbError(status, f"{what}: {msg}")


def _ptr(t) -> Optional[int]:
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


# ------------------------------------------------------------------------------------------
# thin wrappers with the C names
# ------------------------------------------------------------------------------------------


def bccb_batch_create(insts: Sequence[bccb_inst_t], masks_host: np.ndarray, algo: int, rho: float = 1.0,
                      stream=None, prec: int = F32, gamma=(0.5, 0.5)) -> int:
    arr = (bccb_inst_t * len(insts))(*insts)
    masks = np.ascontiguousarray(masks_host, dtype=np.uint8)
    h = ctypes.c_void_p()
    st = _lib.bccb_batch_create_gamma(ctypes.byref(h), arr, len(insts), masks.ctypes.data_as(ctypes.c_void_p),
                                      int(algo), float(rho), int(prec), float(gamma[0]), float(gamma[1]),
                                      _stream(stream))
    _raise(st, None)
    return h.value


def bccb_batch_solve(h: int, y_dev, iters: int, c0_dev, c_out_dev, aux_out_dev=None, check: bool = True,
                     status_out: Optional[np.ndarray] = None) -> int:
    """With ``status_out`` (int32 numpy array of n entries) the per-instance KKT status is
    written there and the call returns BCCB_ERR_KKT instead of raising when only that failed."""
    sp = None
    if status_out is not None:
        if not (isinstance(status_out, np.ndarray) and status_out.dtype == np.int32 and status_out.flags.c_contiguous):
            raise ValueError("status_out must be a C-contiguous int32 numpy array")
        sp = status_out.ctypes.data_as(ctypes.c_void_p)
    st = _lib.bccb_batch_solve(h, _ptr(y_dev), int(iters), _ptr(c0_dev), _ptr(c_out_dev), _ptr(aux_out_dev),
                               1 if check else 0, sp)
    if st == ERR_KKT and status_out is not None:
        return st
    _raise(st, h)
    return st


def bccb_set_kkt_tol(h: int, tol: float) -> None:
    _raise(_lib.bccb_set_kkt_tol(h, float(tol)), h)


def bccb_batch_status(h: int, n: int) -> np.ndarray:
    """Per-instance status (OK or ERR_KKT) of the last checked solve, as int32 (n,)."""
    st = np.zeros(n, np.int32)
    r = _lib.bccb_batch_status(h, st.ctypes.data_as(ctypes.c_void_p))
    if r != ERR_KKT:
        _raise(r, h)
    return st


def bccb_mu(h: int, n: int) -> np.ndarray:
    mu = np.zeros(n)
    _raise(_lib.bccb_mu(h, mu.ctypes.data_as(ctypes.c_void_p)), h)
    return mu


def bccb_batch_solve_host(h: int, y_host: np.ndarray, iters: int, c_out_host: np.ndarray, check: bool = True) -> None:
    for a in (y_host, c_out_host):
        if not (isinstance(a, np.ndarray) and a.flags.c_contiguous and a.dtype in (np.complex64, np.complex128)):
            raise ValueError("host buffers must be C-contiguous complex numpy arrays of the solver's precision")
    _raise(_lib.bccb_batch_solve_host(h, y_host.ctypes.data_as(ctypes.c_void_p), int(iters),
                                      c_out_host.ctypes.data_as(ctypes.c_void_p), 1 if check else 0), h)


def bccb_batch_results(h: int, n: int):
    kkt, obj, lam, mu = (np.zeros(n) for _ in range(4))
    vp = ctypes.c_void_p
    _raise(_lib.bccb_batch_results(h, kkt.ctypes.data_as(vp), obj.ctypes.data_as(vp), lam.ctypes.data_as(vp),
                                   mu.ctypes.data_as(vp)), h)
    return {"kkt": kkt, "objective": obj, "lam": lam, "mu": mu}


def bccb_batch_get(h: int, what: int, dst_dev) -> None:
    _raise(_lib.bccb_batch_get(h, int(what), _ptr(dst_dev)), h)


def bccb_create(M1: int, M2: int, mask_host: np.ndarray, L1: int, L2: int, algo: int, rho: float = 1.0,
                stream=None, prec: int = F32) -> int:
    m = np.ascontiguousarray(mask_host, dtype=np.uint8).reshape(-1)
    if m.size != M1 * M2:
        raise ValueError("mask must have M1*M2 entries")
    h = ctypes.c_void_p()
    _raise(_lib.bccb_create(ctypes.byref(h), int(M1), int(M2), m.ctypes.data_as(ctypes.c_void_p), int(L1),
                            int(L2), int(algo), float(rho), int(prec), _stream(stream)), None)
    return h.value


def bccb_solve(h: int, y_dev, lam: float, lam_is_frac: bool, iters: int, c0_dev, c_out_dev, aux_out_dev=None,
               check: bool = True):
    kkt, obj = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = _lib.bccb_solve(h, _ptr(y_dev), float(lam), 1 if lam_is_frac else 0, int(iters), _ptr(c0_dev),
                         _ptr(c_out_dev), _ptr(aux_out_dev), ctypes.byref(kkt) if check else None,
                         ctypes.byref(obj) if check else None)
    _raise(st, h)
    return (kkt.value, obj.value) if check else None


def bccb_batch_capture(h: int, y_dev, iters: int, c0_dev, c_out_dev, aux_out_dev=None, check: bool = True) -> None:
    _raise(_lib.bccb_batch_capture(h, _ptr(y_dev), int(iters), _ptr(c0_dev), _ptr(c_out_dev), _ptr(aux_out_dev),
                                   1 if check else 0), h)


def bccb_batch_replay(h: int) -> None:
    _raise(_lib.bccb_batch_replay(h), h)


def bccb_batch_tune(h: int, y_dev, probe_iters: int = 20, cache_path: Optional[str] = None) -> None:
    _raise(_lib.bccb_batch_tune(h, _ptr(y_dev), int(probe_iters),
                                None if cache_path is None else cache_path.encode()), h)


def bccb_batch_tile(h: int, L1: int, L2: int) -> int:
    t = ctypes.c_int(0)
    _raise(_lib.bccb_batch_tile(h, int(L1), int(L2), ctypes.byref(t)), h)
    return t.value


def bccb_batch_variant(h: int, L1: int, L2: int):
    """(tile, sparse_state) of the fused kernel chosen for the (L1, L2) class."""
    t, sp = ctypes.c_int(0), ctypes.c_int(0)
    _raise(_lib.bccb_batch_variant(h, int(L1), int(L2), ctypes.byref(t), ctypes.byref(sp)), h)
    return t.value, sp.value


def bccb_unrolled_fwd(h: int, y_dev, batch: int, layers: int, scale_dev, thresh_dev, c_out_dev, saved_dev=None,
                      check: bool = False) -> None:
    _raise(_lib.bccb_unrolled_fwd(h, _ptr(y_dev), int(batch), int(layers), _ptr(scale_dev), _ptr(thresh_dev),
                                  _ptr(c_out_dev), _ptr(saved_dev), 1 if check else 0), h)


def bccb_unrolled_bwd(h: int, batch: int, layers: int, scale_dev, thresh_dev, saved_dev, grad_c_dev,
                      grad_scale_dev, grad_thresh_dev, grad_y_dev=None) -> None:
    _raise(_lib.bccb_unrolled_bwd(h, int(batch), int(layers), _ptr(scale_dev), _ptr(thresh_dev), _ptr(saved_dev),
                                  _ptr(grad_c_dev), _ptr(grad_y_dev), _ptr(grad_scale_dev), _ptr(grad_thresh_dev)),
           h)


def bccb_batch_set_method(h: int, method) -> None:
    m = {"fft": FFT, "dense": DENSE}[method] if isinstance(method, str) else int(method)
    _raise(_lib.bccb_batch_set_method(h, m), h)


def bccb_batch_peaks(h: int, c_dev, K: int, rel_thresh: float, idx_dev, mag_dev, harm_dev, ang_dev,
                     count_dev=None) -> None:
    _raise(_lib.bccb_batch_peaks(h, _ptr(c_dev), int(K), float(rel_thresh), _ptr(idx_dev), _ptr(mag_dev),
                                 _ptr(harm_dev), _ptr(ang_dev), _ptr(count_dev)), h)


def bccb_set_timing(h: int, enable: bool) -> None:
    _raise(_lib.bccb_set_timing(h, 1 if enable else 0), h)


def bccb_last_timing(h: int):
    f = [ctypes.c_float(0.0) for _ in range(3)]
    n = ctypes.c_int64(0)
    _raise(_lib.bccb_last_timing(h, ctypes.byref(f[0]), ctypes.byref(f[1]), ctypes.byref(f[2]),
                                 ctypes.byref(n)), h)
    return {"setup_ms": f[0].value, "iterate_ms": f[1].value, "check_ms": f[2].value, "launches": n.value}


def bccb_fp32_fma_rate(paired: bool = False, iters: int = 20000, stream=None) -> float:
    """Measured FP32 multiply-add rate of the current device in TFLOP/s (scalar, or paired f32x2)."""
    out = ctypes.c_double(0.0)
    _raise(_lib.bccb_fp32_fma_rate(1 if paired else 0, int(iters), _stream(stream), ctypes.byref(out)), None)
    return out.value


def bccb_batch_solve_host_ptr(h: int, y_host_ptr: int, iters: int, c_out_host_ptr: int, check: bool = True) -> None:
    """Host-buffer entry point on raw host pointers (e.g. pinned torch CPU tensors)."""
    _raise(_lib.bccb_batch_solve_host(h, y_host_ptr, int(iters), c_out_host_ptr, 1 if check else 0), h)


def bccb_destroy(h: int) -> None:
    _lib.bccb_destroy(h)


def bccb_status_string(status: int) -> str:
    return _lib.bccb_status_string(int(status)).decode()


# ------------------------------------------------------------------------------------------
# packing helper and a small owner object (still marshalling only)
# ------------------------------------------------------------------------------------------


def pack(instances, dtype=np.complex64):
    """Pack instances given as dicts with keys M1, M2, L1, L2, mask (uint8, M1*M2),
    y (complex, N), lam, lam_is_frac into (inst table, masks, y of `dtype`, total c).

    Instance i's measurements start at y_off = sum of previous N; its solution at
    c_off = sum of previous L1*L2.
    """
    insts, masks, ys = [], [], []
    m_off = y_off = c_off = 0
    for d in instances:
        mask = np.ascontiguousarray(d["mask"], dtype=np.uint8).reshape(-1)
        y = np.asarray(d["y"]).reshape(-1)
        q = bccb_inst_t(d["M1"], d["M2"], d["L1"], d["L2"], m_off, y_off, c_off, float(d["lam"]),
                        1 if d.get("lam_is_frac", False) else 0, 0)
        insts.append(q)
        masks.append(mask)
        ys.append(y.astype(dtype))
        m_off += mask.size
        y_off += y.size
        c_off += d["L1"] * d["L2"]
    return insts, np.concatenate(masks), np.concatenate(ys), c_off


class BatchSolver:
    """Owns one solver handle.  ``instances`` as for :func:`pack`."""

    def __init__(self, instances, algo="fista", rho: float = 1.0, stream=None, prec="f32", gamma=(0.5, 0.5)):
        self.algo = ALGOS[algo] if isinstance(algo, str) else int(algo)
        self.prec = {"f32": F32, "f64": F64}[prec] if isinstance(prec, str) else int(prec)
        self.dtype = np.complex128 if self.prec == F64 else np.complex64
        self.insts, self.masks, self.y_host, self.total_c = pack(instances, self.dtype)
        self.n = len(self.insts)
        self.offsets = [(q.c_off, q.L1, q.L2) for q in self.insts]
        self.handle = bccb_batch_create(self.insts, self.masks, self.algo, rho, stream, self.prec, gamma)

    def solve(self, y_dev, iters, c_out, c0=None, aux_out=None, check=True, status_out=None):
        bccb_batch_solve(self.handle, y_dev, iters, c0, c_out, aux_out, check, status_out)
        return c_out

    def mu(self):
        return bccb_mu(self.handle, self.n)

    def solve_host(self, y_host, iters, c_out_host, check=True):
        bccb_batch_solve_host(self.handle, y_host, iters, c_out_host, check)
        return c_out_host

    def results(self):
        return bccb_batch_results(self.handle, self.n)

    def set_method(self, method):
        """'fft' (default) or 'dense' (the stored L x L Gram, bccb_batch_set_method)."""
        bccb_batch_set_method(self.handle, method)

    def peaks(self, c_dev, K: int, rel_thresh: float = 0.0):
        """Top-K peaks of every instance (bccb_batch_peaks); device tensors
        idx (n, K) int32, mag (n, K), harm (n, K, 2), ang (n, K, 2) float64, count (n,) int32."""
        import torch

        dev = c_dev.device
        idx = torch.empty((self.n, K), dtype=torch.int32, device=dev)
        mag = torch.empty((self.n, K), dtype=torch.float64, device=dev)
        harm = torch.empty((self.n, K, 2), dtype=torch.float64, device=dev)
        ang = torch.empty((self.n, K, 2), dtype=torch.float64, device=dev)
        count = torch.empty((self.n,), dtype=torch.int32, device=dev)
        bccb_batch_peaks(self.handle, c_dev, K, rel_thresh, idx, mag, harm, ang, count)
        return dict(idx=idx, mag=mag, harm=harm, ang=ang, count=count)

    def get(self, what, dst_dev):
        bccb_batch_get(self.handle, what, dst_dev)
        return dst_dev

    def unpack(self, flat: np.ndarray):
        """Split a packed solution (numpy, complex) into per-instance (L2, L1) grids."""
        return [flat[o:o + L1 * L2].reshape(L2, L1) for (o, L1, L2) in self.offsets]

    def close(self):
        if self.handle:
            bccb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
