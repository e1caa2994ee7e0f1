"""Python binding of the GB300 Kernel K-means library (``libpopcorn.so``).

Argument marshalling only: every step of the method runs in the CUDA library
behind the C ABI of ``include/popcorn.h``.  Functions carry the C names:

* ``popcorn_kernel_matrix`` -- K = kappa(P P^T) and diag(K) (Sec. 3.2).
* ``popcorn_assign_step``   -- one pass of the loop body of Alg. 2 on a given K.
* ``popcorn_fit``           -- Kernel K-means (Alg. 2) from points and labels.
* ``popcorn_kmeanspp``      -- K-means++ seeding (Sec. 2.1) in the kernel's feature space.

Device buffers are torch CUDA tensors (PyTorch supplies memory and streams);
``popcorn_fit`` also accepts host buffers (CPU tensors or numpy arrays), which
the library copies inside the call.  Importing this module fails loudly when
the compiled library is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "LIBRARY_PATH",
    "PopcornError",
    "popcorn_kernel_matrix",
    "popcorn_assign_step",
    "popcorn_fit",
    "popcorn_fit_batched",
    "popcorn_kmeanspp",
    "popcorn_assign_step_noalloc",
    "NOALLOC_SCRATCH_BYTES",
    "popcorn_version",
    "popcorn_autotune_entries",
    "popcorn_autotune_clear",
    "kernel_spec",
    "EXPORTED_SYMBOLS",
]

LIBRARY_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpopcorn.so")

if not os.path.exists(LIBRARY_PATH):
    raise ImportError(
        f"{LIBRARY_PATH} is missing: build it with `python paper_2501_05587_gb300/build.py` "
        "(nvcc, sm_103a). There is no CPU fallback.")

_lib = ctypes.CDLL(LIBRARY_PATH)

# names declared in include/popcorn.h
EXPORTED_SYMBOLS = (
    "popcorn_status_string",
    "popcorn_last_error_message",
    "popcorn_version",
    "popcorn_kernel_matrix",
    "popcorn_kernel_matrix_ex",
    "popcorn_kernel_matrix_ex",
    "popcorn_assign_step",
    "popcorn_fit",
    "popcorn_assign_step_noalloc",
    "popcorn_fit_batched",
    "popcorn_kmeanspp",
    "popcorn_autotune_entries",
    "popcorn_autotune_clear",
    "popcorn_allocation_count",
)

KIND = {"linear": 0, "polynomial": 1, "gaussian": 2}
PRECISION = {"fp32": 0, "bf16": 1, "bf16x3": 2, "fp8": 3}


class _Kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("degree", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("coef0", ctypes.c_double), ("sigma", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("store_k", ctypes.c_int32),
                ("check_convergence", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("k_storage", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("k_pass", ctypes.c_int32), ("sym_tile", ctypes.c_int32),
                ("reserved", ctypes.c_int64 * 4)]


K_STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
K_PASS = {"auto": 0, "symmetric": 1, "full": 2}


class _FitInfo(ctypes.Structure):
    _fields_ = [("kbuild_ms", ctypes.c_double), ("loop_ms", ctypes.c_double),
                ("reduce_ms", ctypes.c_double), ("assign_ms", ctypes.c_double),
                ("eval_ms", ctypes.c_double), ("reduce_launches", ctypes.c_int32),
                ("assign_launches", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("h2d_bytes", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64), ("J_history", ctypes.POINTER(ctypes.c_double)),
                ("changed_history", ctypes.POINTER(ctypes.c_int32)), ("tune_cache_hit", ctypes.c_int32),
                ("tune_candidates", ctypes.c_int32), ("tune_ms", ctypes.c_double),
                ("schedule", ctypes.c_int32 * 4), ("fold_ms", ctypes.c_double),
                ("k_pass_used", ctypes.c_int32), ("sym_form", ctypes.c_int32),
                ("E_out", ctypes.c_void_p)]


class _Instance(ctypes.Structure):
    _fields_ = [("P", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("ldp", ctypes.c_int64),
                ("k", ctypes.c_int32), ("kern", _Kernel), ("init_labels", ctypes.c_void_p),
                ("labels_out", ctypes.c_void_p)]


_vp, _i64, _i32, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
_lib.popcorn_status_string.restype = ctypes.c_char_p
_lib.popcorn_status_string.argtypes = [ctypes.c_int]
_lib.popcorn_last_error_message.restype = ctypes.c_char_p
_lib.popcorn_last_error_message.argtypes = []
_lib.popcorn_version.restype = _i32
_lib.popcorn_allocation_count.restype = ctypes.c_int64
_lib.popcorn_allocation_count.argtypes = []
_lib.popcorn_version.argtypes = []
_lib.popcorn_kernel_matrix.restype = ctypes.c_int
_lib.popcorn_kernel_matrix.argtypes = [_vp, _i64, _i32, _i64, _Kernel, _i32, _vp, _i64, _vp, _vp]
_lib.popcorn_kernel_matrix_ex.restype = ctypes.c_int
_lib.popcorn_kernel_matrix_ex.argtypes = [_vp, _i64, _i32, _i64, _Kernel, _i32, _i32, _vp, _i64, _vp, _vp]
_lib.popcorn_assign_step.restype = ctypes.c_int
_lib.popcorn_assign_step.argtypes = [_vp, _i64, _vp, _i64, _i32, _vp, _vp, _vp, _vp, _vp,
                                     ctypes.POINTER(_dbl), ctypes.POINTER(_i32), _vp]
_lib.popcorn_assign_step_noalloc.restype = ctypes.c_int
_lib.popcorn_assign_step_noalloc.argtypes = _lib.popcorn_assign_step.argtypes
_lib.popcorn_fit_batched.restype = ctypes.c_int
_lib.popcorn_fit_batched.argtypes = [_i32, ctypes.POINTER(_Instance), _i32, _dbl, ctypes.POINTER(_Options),
                                     ctypes.POINTER(_dbl), ctypes.POINTER(_i32), ctypes.POINTER(_FitInfo), _vp]
_lib.popcorn_autotune_entries.restype = _i32
_lib.popcorn_autotune_entries.argtypes = []
_lib.popcorn_autotune_clear.restype = None
_lib.popcorn_autotune_clear.argtypes = []
_lib.popcorn_kmeanspp.restype = ctypes.c_int
_lib.popcorn_kmeanspp.argtypes = [_vp, _i64, _i32, _i64, _i32, _Kernel, _vp, _vp, _vp, _vp]
_lib.popcorn_fit.restype = ctypes.c_int
_lib.popcorn_fit.argtypes = [_vp, _i64, _i32, _i64, _i32, _Kernel, _vp, _i32, _dbl,
                             ctypes.POINTER(_Options), _vp, ctypes.POINTER(_dbl), ctypes.POINTER(_i32),
                             ctypes.POINTER(_FitInfo), _vp]


class PopcornError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        name = _lib.popcorn_status_string(status).decode()
        msg = _lib.popcorn_last_error_message().decode()
        super().__init__(f"{where}: {name}: {msg}")


def _check(status: int, where: str) -> None:
    if status != 0:
        raise PopcornError(status, where)


def popcorn_version() -> int:
    return int(_lib.popcorn_version())


def kernel_spec(kind: str = "gaussian", *, gamma: float = 1.0, coef0: float = 1.0, degree: int = 2,
                sigma: float = 1.0) -> dict:
    return {"kind": kind, "gamma": float(gamma), "coef0": float(coef0), "degree": int(degree),
            "sigma": float(sigma)}


def _kernel(kern: dict) -> _Kernel:
    return _Kernel(KIND[kern["kind"]], int(kern.get("degree", 1)), float(kern.get("gamma", 1.0)),
                   float(kern.get("coef0", 0.0)), float(kern.get("sigma", 1.0)))


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(x):
    """Address of a tensor or a numpy array (no copy)."""
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


SCHEDULE = {"auto": 0, "symmetric": 1, "full": 2, "tune": 3}


def popcorn_kernel_matrix(P, kernel: dict, precision: str = "fp32", K=None, kdiag=None, stream=None,
                          schedule: str = "auto"):
    """K = kappa(P P^T) (full square, FP32) and diag(K) on the device of P.

    P is an (n, d) float32 CUDA tensor (rows may be strided: ldp = P.stride(0)).
    ``schedule`` ("auto", "symmetric", "full", "tune") picks the tile schedule
    (popcorn_kernel_matrix_ex).  Returns (K, kdiag); K has a leading dimension
    rounded up to a multiple of 4 (the returned tensor is the (n, n) view).
    """
    torch = _torch()
    assert P.is_cuda and P.dtype == torch.float32 and P.dim() == 2 and P.stride(1) == 1
    n, d = P.shape
    ldk = (n + 3) // 4 * 4
    if K is None:
        K = torch.empty((n, ldk), dtype=torch.float32, device=P.device)[:, :n]
    if kdiag is None:
        kdiag = torch.empty(n, dtype=torch.float32, device=P.device)
    _check(_lib.popcorn_kernel_matrix_ex(_ptr(P), n, d, P.stride(0), _kernel(kernel), PRECISION[precision],
                                         SCHEDULE[schedule], _ptr(K), K.stride(0), _ptr(kdiag), _stream(stream)),
           "popcorn_kernel_matrix_ex")
    return K, kdiag


def _assign_step(fn, where, K, kdiag, labels, k, want_E, stream):
    torch = _torch()
    n = K.shape[0]
    dev = K.device
    labels = labels.to(device=dev, dtype=torch.int32).contiguous()
    new = torch.empty(n, dtype=torch.int32, device=dev)
    counts = torch.empty(k, dtype=torch.int32, device=dev)
    cnorm = torch.empty(k, dtype=torch.float64, device=dev)
    E = torch.empty((n, k), dtype=torch.float32, device=dev) if want_E else None
    J = ctypes.c_double(0.0)
    ch = ctypes.c_int32(0)
    _check(fn(_ptr(K), K.stride(0), _ptr(kdiag), n, int(k), _ptr(labels), _ptr(new), _ptr(counts),
              _ptr(E) if E is not None else None, _ptr(cnorm), ctypes.byref(J), ctypes.byref(ch),
              _stream(stream)), where)
    return {"labels": new, "counts": counts, "cnorm": cnorm, "J": J.value, "changed": ch.value, "E": E}


def popcorn_assign_step(K, kdiag, labels, k: int, want_E: bool = False, stream=None) -> dict:
    """One pass of Alg. 2's loop body from ``labels`` on the device K.

    Returns new labels, counts of the new labels, centroid norms ||c_j||^2,
    J(labels), the number of changed labels and, with want_E, E = K V^T.
    """
    return _assign_step(_lib.popcorn_assign_step, "popcorn_assign_step", K, kdiag, labels, k, want_E, stream)


# size of the static device scratch array of popcorn_assign_step_noalloc (include/popcorn.h)
NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def popcorn_assign_step_noalloc(K, kdiag, labels, k: int, want_E: bool = False, stream=None) -> dict:
    """popcorn_assign_step for callers that may not allocate device memory.

    Same results and arguments; the library's temporaries live in one static
    device array of NOALLOC_SCRATCH_BYTES (calls must not overlap on the GPU).
    The output tensors this wrapper returns are allocated here by torch for
    convenience; a caller that cannot allocate passes its own buffers to the
    C entry point directly.
    """
    return _assign_step(_lib.popcorn_assign_step_noalloc, "popcorn_assign_step_noalloc", K, kdiag, labels, k,
                        want_E, stream)


def _info_dict(info) -> dict:
    out = {f: getattr(info, f) for f, _ in _FitInfo._fields_
           if f not in ("J_history", "changed_history", "schedule", "E_out")}
    out["schedule"] = list(info.schedule)
    return out


def popcorn_autotune_entries() -> int:
    """Workload signatures with a tuned schedule in this process's cache."""
    return int(_lib.popcorn_autotune_entries())


def popcorn_autotune_clear() -> None:
    """Forget every tuned schedule of this process (a cache file is left alone)."""
    _lib.popcorn_autotune_clear()


def popcorn_fit(P, k: int, kernel: dict, init_labels, max_iter: int, tol: float = 0.0,
                precision: str = "fp32", check_convergence: bool = True, timing: bool = False,
                history: bool = False, labels_out=None, store_k: bool = True, k_storage: str = "fp32",
                autotune: bool = False, k_pass: str = "auto", sym_tile: int = 0, E_out=None,
                stream=None) -> dict:
    """Kernel K-means (Alg. 2).  P and init_labels may live on the host or the device.

    ``store_k=False`` selects the recompute path (K never stored; precision
    "bf16" or "fp8").  ``k_storage`` ("fp32", "fp16", "bf16") is the element
    type of a stored K.  ``k_pass`` ("auto", "symmetric", "full") is how a pass
    reads a stored FP32 K; ``timing`` (False, True / "kernels", "phases") records CUDA-event
    times per phase and kernel, or per phase only (which leaves a fixed-iteration fit's passes
    in one CUDA graph); ``sym_tile`` (0 = automatic, else 1..8) is the super-tile edge of
    the symmetric pass.  ``E_out`` (an (n, k) float32 CUDA tensor) receives E = K V^T of the
    labels the last pass started from (stored-K fits).  Returns {"labels", "objective",
    "iterations", "info"};
    labels land where ``labels_out`` lives (default: same place as init_labels).
    """
    torch = _torch()
    host = isinstance(P, np.ndarray) or not P.is_cuda
    if isinstance(P, np.ndarray):
        P = np.ascontiguousarray(P, dtype=np.float32)
        n, d = P.shape
        ldp = d
    else:
        assert P.dtype == torch.float32 and P.dim() == 2 and P.stride(1) == 1
        n, d = P.shape
        ldp = P.stride(0)
    if isinstance(init_labels, np.ndarray):
        init_labels = np.ascontiguousarray(init_labels, dtype=np.int32)
    else:
        init_labels = init_labels.to(torch.int32).contiguous()
    if labels_out is None:
        if isinstance(init_labels, np.ndarray):
            labels_out = np.empty(n, dtype=np.int32)
        else:
            labels_out = torch.empty(n, dtype=torch.int32, device=init_labels.device)
    timing = {False: 0, True: 1, "kernels": 1, "phases": 2}[timing]
    opt = _Options(PRECISION[precision], 1 if store_k else 0, 1 if check_convergence else 0, timing,
                   K_STORAGE[k_storage], 1 if autotune else 0, K_PASS[k_pass], int(sym_tile),
                   (ctypes.c_int64 * 4)())
    info = _FitInfo()
    if E_out is not None:
        assert E_out.is_cuda and E_out.dtype == torch.float32 and E_out.is_contiguous()
        assert tuple(E_out.shape) == (n, int(k))
        info.E_out = E_out.data_ptr()
    Jh = (ctypes.c_double * max(1, max_iter))() if history else None
    Ch = (ctypes.c_int32 * max(1, max_iter))() if history else None
    if history:
        info.J_history = ctypes.cast(Jh, ctypes.POINTER(ctypes.c_double))
        info.changed_history = ctypes.cast(Ch, ctypes.POINTER(ctypes.c_int32))
    obj = ctypes.c_double(0.0)
    its = ctypes.c_int32(0)
    _check(_lib.popcorn_fit(_ptr(P), n, d, ldp, int(k), _kernel(kernel), _ptr(init_labels), int(max_iter),
                            float(tol), ctypes.byref(opt), _ptr(labels_out), ctypes.byref(obj),
                            ctypes.byref(its), ctypes.byref(info), _stream(stream)),
           "popcorn_fit")
    out_info = _info_dict(info)
    if history:
        out_info["J_history"] = list(Jh[: its.value])
        out_info["changed_history"] = list(Ch[: its.value])
    out_info["host_inputs"] = host
    return {"labels": labels_out, "objective": obj.value, "iterations": its.value, "info": out_info}


def popcorn_fit_batched(instances, max_iter: int, tol: float = 0.0, precision: str = "fp32",
                        check_convergence: bool = True, timing: bool = False, autotune: bool = False,
                        k_storage: str = "fp32", stream=None) -> dict:
    """Many independent fits in one captured CUDA graph.

    ``instances``: list of dicts {"P": (n, d) float32 CUDA tensor, "k": int, "kernel": dict,
    "init_labels": (n,) int32 CUDA tensor, optional "labels_out"}.  ``k_storage`` ("fp32",
    "fp16", "bf16"): the element type every instance's stored K is rounded to.  Returns
    {"labels": [tensor], "objectives": [float], "iterations": [int], "info": dict}.
    """
    torch = _torch()
    arr = (_Instance * len(instances))()
    outs = []
    keep = []
    for t, x in enumerate(instances):
        P = x["P"]
        assert P.is_cuda and P.dtype == torch.float32 and P.dim() == 2 and P.stride(1) == 1
        lab = x["init_labels"].to(torch.int32).contiguous()
        out = x.get("labels_out")
        if out is None:
            out = torch.empty(P.shape[0], dtype=torch.int32, device=P.device)
        keep += [P, lab, out]
        outs.append(out)
        arr[t] = _Instance(P.data_ptr(), P.shape[0], P.shape[1], P.stride(0), int(x["k"]), _kernel(x["kernel"]),
                           lab.data_ptr(), out.data_ptr())
    opt = _Options(PRECISION[precision], 1, 1 if check_convergence else 0, 1 if timing else 0, K_STORAGE[k_storage],
                   1 if autotune else 0, 0, 0, (ctypes.c_int64 * 4)())
    objs = (ctypes.c_double * len(instances))()
    its = (ctypes.c_int32 * len(instances))()
    info = _FitInfo()
    _check(_lib.popcorn_fit_batched(len(instances), arr, int(max_iter), float(tol), ctypes.byref(opt), objs, its,
                                    ctypes.byref(info), _stream(stream)), "popcorn_fit_batched")
    out_info = _info_dict(info)
    return {"labels": outs, "objectives": list(objs), "iterations": list(its), "info": out_info}


def popcorn_kmeanspp(P, k: int, kernel: dict, u, labels_out=None, stream=None) -> dict:
    """K-means++ seeding (Sec. 2.1) in the kernel's feature space with the caller's k draws
    ``u`` (values in [0, 1); a numpy array or a CUDA float64 tensor).  P may live on the host
    or the device; the labels land on P's side unless ``labels_out`` is given.  Returns
    {"labels": n initial labels, "centers": the k chosen points in order (numpy)}."""
    torch = _torch()
    if isinstance(P, np.ndarray):
        P = np.ascontiguousarray(P, dtype=np.float32)
        n, d = P.shape
        ldp = d
        on_host = True
    else:
        assert P.dtype == torch.float32 and P.dim() == 2 and P.stride(1) == 1
        n, d = P.shape
        ldp = P.stride(0)
        on_host = not P.is_cuda
    if isinstance(u, np.ndarray) or not hasattr(u, "data_ptr"):
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    else:
        u = u.to(torch.float64).contiguous()
    if labels_out is None:
        labels_out = (np.empty(n, dtype=np.int32) if on_host
                      else torch.empty(n, dtype=torch.int32, device=P.device))
    centers = np.empty(int(k), dtype=np.int32)
    _check(_lib.popcorn_kmeanspp(_ptr(P), n, d, ldp, int(k), _kernel(kernel), _ptr(u), _ptr(labels_out),
                                 _ptr(centers), _stream(stream)),
           "popcorn_kmeanspp")
    return {"labels": labels_out, "centers": centers}
