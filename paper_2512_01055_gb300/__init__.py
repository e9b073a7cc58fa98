"""Python binding of libtc (include/tc.h): argument marshalling only.

Every step of the (T) computation runs in the CUDA library; this module loads
``libtc.so`` (built in-tree by ``paper_2512_01055_gb300.build``) and converts
numpy arrays / torch tensors into the pointers and sizes of the C ABI.  There
is no fallback: if the library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc.so")

TC_OK, TC_EINVAL, TC_ENOMEM, TC_ECUDA, TC_ENOTREADY, TC_ETIMEOUT, TC_EBUSY, TC_ECANCELLED, TC_EINTERNAL = range(9)
TC_FP64, TC_SPLIT_BF16 = 0, 1

#: Every symbol include/tc.h declares (the CPU test checks the library exports them).
EXPORTS = ("tc_init", "tc_energy", "tc_energy_dev", "tc_workspace_bytes", "tc_status_str",
           "tc_last_error", "tc_finalize", "tc_energy_dev_noalloc", "tc_triplets_dev", "tc_submit", "tc_poll",
           "tc_wait", "tc_cancel", "tc_serve_stats_get", "tc_inject_fault", "tc_energy_df_dev", "tc_energy_df",
           "tc_shard_range", "tc_energy_shard_dev", "tc_sum_parts", "tc_combine_parts")
TC_JOB_DEVICE_INPUTS = 1
TC_FAULT_ALLOC, TC_FAULT_STALL = 1, 2

#: TC_NOALLOC_SCRATCH_BYTES of include/tc.h
NOALLOC_SCRATCH_BYTES = 8 << 20


class tc_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t),
                ("default_prec", ctypes.c_int), ("default_slices", ctypes.c_int),
                ("timeout_ms", ctypes.c_int), ("max_inflight", ctypes.c_int), ("max_queue", ctypes.c_int),
                ("iteration_ms", ctypes.c_int)]


class tc_ints(ctypes.Structure):
    _fields_ = [("ovvv", ctypes.c_void_p), ("ovoo", ctypes.c_void_p), ("ovov", ctypes.c_void_p)]


class tc_job(ctypes.Structure):
    _fields_ = [("o", ctypes.c_int), ("v", ctypes.c_int), ("eps", ctypes.c_void_p), ("t1", ctypes.c_void_p),
                ("t2", ctypes.c_void_p), ("ints", tc_ints), ("prec", ctypes.c_int), ("slices", ctypes.c_int),
                ("flags", ctypes.c_int), ("nq", ctypes.c_int), ("B", ctypes.c_void_p)]


class tc_serve_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "cancelled", "queued", "inflight",
                                               "iterations", "graph_launches", "batched_jobs")] + \
               [("reserved_bytes", ctypes.c_size_t)]


class tc_result(ctypes.Structure):
    _fields_ = [("e_t", ctypes.c_double), ("seconds", ctypes.c_double), ("tflops_alg", ctypes.c_double),
                ("prec", ctypes.c_int), ("slices", ctypes.c_int), ("o", ctypes.c_int), ("v", ctypes.c_int),
                ("queue_seconds", ctypes.c_double), ("kernel_seconds", ctypes.c_double),
                ("prep_seconds", ctypes.c_double), ("n_items", ctypes.c_longlong),
                ("launches", ctypes.c_int), ("reserved", ctypes.c_int), ("wterm_seconds", ctypes.c_double),
                ("e_t5", ctypes.c_double), ("df_seconds", ctypes.c_double), ("df_digits", ctypes.c_int),
                ("reserved2", ctypes.c_int)]


class TcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_str(status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libtc.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with `python -m paper_2512_01055_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    lib.tc_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(tc_options)]
    lib.tc_init.restype = i
    lib.tc_energy.argtypes = [vp, i, i, vp, vp, vp, ctypes.POINTER(tc_ints), i, i, vp, ctypes.POINTER(tc_result)]
    lib.tc_energy.restype = i
    lib.tc_energy_dev.argtypes = [vp, i, i, vp, vp, vp, ctypes.POINTER(tc_ints), i, i, vp, vp,
                                  ctypes.POINTER(tc_result)]
    lib.tc_energy_dev.restype = i
    lib.tc_workspace_bytes.argtypes = [i, i, i, i]
    lib.tc_workspace_bytes.restype = sz
    lib.tc_status_str.argtypes = [i]
    lib.tc_status_str.restype = ctypes.c_char_p
    lib.tc_last_error.argtypes = [vp]
    lib.tc_last_error.restype = ctypes.c_char_p
    lib.tc_finalize.argtypes = [vp]
    lib.tc_finalize.restype = None
    lib.tc_energy_dev_noalloc.argtypes = [i, i, vp, vp, vp, ctypes.POINTER(tc_ints), vp, vp, vp,
                                          ctypes.c_char_p, sz]
    lib.tc_energy_dev_noalloc.restype = i
    lib.tc_triplets_dev.argtypes = [vp, i, i, vp, vp, vp, ctypes.POINTER(tc_ints), i, i, vp, i, vp, vp,
                                    ctypes.POINTER(tc_result)]
    lib.tc_triplets_dev.restype = i
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.tc_submit.argtypes = [vp, ctypes.POINTER(tc_job), u64p]
    lib.tc_submit.restype = i
    lib.tc_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(tc_result)]
    lib.tc_poll.restype = i
    lib.tc_wait.argtypes = [vp, ctypes.c_uint64, i, ctypes.POINTER(tc_result)]
    lib.tc_wait.restype = i
    lib.tc_cancel.argtypes = [vp, ctypes.c_uint64]
    lib.tc_cancel.restype = i
    lib.tc_serve_stats_get.argtypes = [vp, ctypes.POINTER(tc_serve_stats)]
    lib.tc_serve_stats_get.restype = i
    lib.tc_inject_fault.argtypes = [vp, i, i]
    lib.tc_inject_fault.restype = i
    lib.tc_energy_df_dev.argtypes = [vp, i, i, i, vp, vp, vp, vp, i, i, vp, vp, ctypes.POINTER(tc_result)]
    lib.tc_energy_df_dev.restype = i
    lib.tc_energy_df.argtypes = [vp, i, i, i, vp, vp, vp, vp, i, i, vp, ctypes.POINTER(tc_result)]
    lib.tc_energy_df.restype = i
    llp = ctypes.POINTER(ctypes.c_longlong)
    lib.tc_shard_range.argtypes = [i, i, i, llp, llp]
    lib.tc_shard_range.restype = i
    lib.tc_energy_shard_dev.argtypes = [vp, i, i, vp, vp, vp, ctypes.POINTER(tc_ints), i, i, i, i, dp, vp,
                                        ctypes.POINTER(tc_result)]
    lib.tc_energy_shard_dev.restype = i
    lib.tc_sum_parts.argtypes = [dp, ctypes.c_longlong, dp]
    lib.tc_sum_parts.restype = i
    lib.tc_combine_parts.argtypes = [dp, i, dp]
    lib.tc_combine_parts.restype = i
    del d
    _lib = lib
    return lib


def status_str(s: int) -> str:
    return load().tc_status_str(s).decode()


# ---------------------------------------------------------------------------
# Same-named thin wrappers
# ---------------------------------------------------------------------------

def tc_init(device: int = 0, hbm_budget_bytes: int = 0, default_prec: int = TC_FP64,
            default_slices: int = 3, timeout_ms: int = 0, max_inflight: int = 0, max_queue: int = 0,
            iteration_ms: int = 0) -> ctypes.c_void_p:
    lib = load()
    ctx = ctypes.c_void_p()
    opt = tc_options(device, hbm_budget_bytes, default_prec, default_slices, timeout_ms, max_inflight, max_queue,
                     iteration_ms)
    s = lib.tc_init(ctypes.byref(ctx), ctypes.byref(opt))
    if s != TC_OK:
        raise TcError(s, "tc_init failed")
    return ctx


def tc_finalize(ctx) -> None:
    load().tc_finalize(ctx)


def tc_last_error(ctx) -> str:
    return load().tc_last_error(ctx).decode()


def tc_workspace_bytes(o: int, v: int, prec: int = TC_FP64, slices: int = 0) -> int:
    return int(load().tc_workspace_bytes(o, v, prec, slices))


def _ptr_np(a):
    import numpy as np
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError("host arrays must be C-contiguous float64 numpy arrays")
    return a.ctypes.data


def _ptr_dev(t):
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("device arrays must be contiguous float64 CUDA tensors")
    return t.data_ptr()


def _check(ctx, s):
    if s != TC_OK:
        raise TcError(s, tc_last_error(ctx))


def tc_energy(ctx, o, v, eps, t1, t2, ovvv, ovoo, ovov, prec=TC_FP64, slices=0, e_ijk=None) -> tc_result:
    """E_(T) from host numpy arrays (layouts of include/tc.h).  e_ijk: optional [o,o,o] float64 output."""
    ints = tc_ints(_ptr_np(ovvv), _ptr_np(ovoo), _ptr_np(ovov))
    res = tc_result()
    s = load().tc_energy(ctx, o, v, _ptr_np(eps), _ptr_np(t1), _ptr_np(t2), ctypes.byref(ints), prec, slices,
                         _ptr_np(e_ijk), ctypes.byref(res))
    _check(ctx, s)
    return res


def tc_energy_dev(ctx, o, v, eps, t1, t2, ovvv, ovoo, ovov, prec=TC_FP64, slices=0, e_ijk=None,
                  stream=None) -> tc_result:
    """E_(T) from device torch tensors read in place; ``stream``: a torch.cuda.Stream or None (current)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    ints = tc_ints(_ptr_dev(ovvv), _ptr_dev(ovoo), _ptr_dev(ovov))
    res = tc_result()
    s = load().tc_energy_dev(ctx, o, v, _ptr_dev(eps), _ptr_dev(t1), _ptr_dev(t2), ctypes.byref(ints), prec,
                             slices, _ptr_dev(e_ijk), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(res))
    _check(ctx, s)
    return res


def tc_energy_df_dev(ctx, o, v, B, eps, t1, t2, prec=TC_FP64, slices=0, e_ijk=None, stream=None) -> tc_result:
    """E_(T) with the integrals given as DF factors: B a device tensor [nq, o+v, o+v] (occupied first)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if not (isinstance(B, torch.Tensor) and B.dim() == 3 and B.shape[1] == o + v and B.shape[2] == o + v):
        raise TypeError("B must be a [nq, o+v, o+v] tensor")
    res = tc_result()
    s = load().tc_energy_df_dev(ctx, o, v, int(B.shape[0]), _ptr_dev(eps), _ptr_dev(t1), _ptr_dev(t2), _ptr_dev(B),
                                prec, slices, _ptr_dev(e_ijk), ctypes.c_void_p(stream.cuda_stream),
                                ctypes.byref(res))
    _check(ctx, s)
    return res


def tc_energy_df(ctx, o, v, B, eps, t1, t2, prec=TC_FP64, slices=0, e_ijk=None) -> tc_result:
    """E_(T) from host numpy arrays with the integrals given as DF factors B [nq, o+v, o+v] (occupied first)."""
    import numpy as np
    if not (isinstance(B, np.ndarray) and B.ndim == 3 and B.shape[1] == o + v and B.shape[2] == o + v):
        raise TypeError("B must be a [nq, o+v, o+v] array")
    res = tc_result()
    s = load().tc_energy_df(ctx, o, v, int(B.shape[0]), _ptr_np(eps), _ptr_np(t1), _ptr_np(t2), _ptr_np(B), prec,
                            slices, _ptr_np(e_ijk), ctypes.byref(res))
    _check(ctx, s)
    return res


def tc_triplets_dev(ctx, o, v, eps, t1, t2, ovvv, ovoo, ovov, triplets, prec=TC_FP64, slices=0,
                    stream=None):
    """Weighted contributions of the listed (i, j, k), i >= j >= k; returns (numpy array [n], tc_result)."""
    import numpy as np
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    trip = np.ascontiguousarray(np.asarray(triplets, dtype=np.int32).reshape(-1, 3))
    e_out = np.zeros(trip.shape[0], dtype=np.float64)
    ints = tc_ints(_ptr_dev(ovvv), _ptr_dev(ovoo), _ptr_dev(ovov))
    res = tc_result()
    s = load().tc_triplets_dev(ctx, o, v, _ptr_dev(eps), _ptr_dev(t1), _ptr_dev(t2), ctypes.byref(ints), prec, slices,
                               trip.ctypes.data, trip.shape[0], e_out.ctypes.data,
                               ctypes.c_void_p(stream.cuda_stream), ctypes.byref(res))
    _check(ctx, s)
    return e_out, res


def tc_energy_dev_noalloc(o, v, eps, t1, t2, ovvv, ovoo, ovov, e_t, e_ijk=None, stream=None) -> None:
    """FP64 E_(T) into the device tensor ``e_t`` (one float64) without any device allocation.

    For callers that may not allocate device memory: scratch lives in the
    library's static device array (NOALLOC_SCRATCH_BYTES).  Only enqueues work
    on ``stream`` (default: torch's current stream); calls that overlap on the
    GPU race on the shared array.
    """
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    ints = tc_ints(_ptr_dev(ovvv), _ptr_dev(ovoo), _ptr_dev(ovov))
    buf = ctypes.create_string_buffer(256)
    s = load().tc_energy_dev_noalloc(o, v, _ptr_dev(eps), _ptr_dev(t1), _ptr_dev(t2), ctypes.byref(ints),
                                     _ptr_dev(e_t), _ptr_dev(e_ijk), ctypes.c_void_p(stream.cuda_stream), buf, 256)
    if s != TC_OK:
        raise TcError(s, buf.value.decode())


# ---------------------------------------------------------------------------
# One energy over several ranks
# ---------------------------------------------------------------------------

def tc_shard_range(o, rank, world):
    """(first, count) of rank's contiguous range of the occupied triplets i >= j >= k (all-equal excluded)."""
    first, count = ctypes.c_longlong(), ctypes.c_longlong()
    s = load().tc_shard_range(o, rank, world, ctypes.byref(first), ctypes.byref(count))
    if s != TC_OK:
        raise TcError(s, f"invalid shard (o={o}, rank={rank}, world={world})")
    return first.value, count.value


def tc_energy_shard_dev(ctx, o, v, eps, t1, t2, ovvv, ovoo, ovov, rank, world, prec=TC_FP64, slices=0, stream=None):
    """This rank's (sum, compensation) pair of E_(T) from device tensors; returns (pair, tc_result)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    ints = tc_ints(_ptr_dev(ovvv), _ptr_dev(ovoo), _ptr_dev(ovov))
    part = (ctypes.c_double * 2)()
    res = tc_result()
    s = load().tc_energy_shard_dev(ctx, o, v, _ptr_dev(eps), _ptr_dev(t1), _ptr_dev(t2), ctypes.byref(ints), prec,
                                   slices, rank, world, part, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(res))
    _check(ctx, s)
    return (part[0], part[1]), res


def tc_sum_parts(x):
    """(sum, compensation) of the host values x in order."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    part = (ctypes.c_double * 2)()
    s = load().tc_sum_parts(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.size, part)
    if s != TC_OK:
        raise TcError(s, "tc_sum_parts")
    return part[0], part[1]


def tc_combine_parts(parts):
    """E_(T) from the (sum, compensation) pairs of ranks 0 .. n-1."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(parts, dtype=np.float64).reshape(-1, 2))
    e = ctypes.c_double()
    s = load().tc_combine_parts(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.shape[0], ctypes.byref(e))
    if s != TC_OK:
        raise TcError(s, "tc_combine_parts")
    return e.value


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------

def tc_submit(ctx, o, v, eps, t1, t2, ovvv=None, ovoo=None, ovov=None, prec=TC_FP64, slices=0, device_inputs=False,
              B=None) -> int:
    """Queue one job; host numpy arrays are copied before return, device tensors stay resident (caller keeps them).

    With B ([nq, o+v, o+v] density-fitting factors) the service assembles the
    integrals itself when it admits the job, and ovvv / ovoo / ovov are not given.
    """
    ptr = _ptr_dev if device_inputs else _ptr_np
    nq = 0 if B is None else int(B.shape[0])
    ints = tc_ints(None, None, None) if B is not None else tc_ints(ptr(ovvv), ptr(ovoo), ptr(ovov))
    job = tc_job(o, v, ptr(eps), ptr(t1), ptr(t2), ints, prec, slices,
                 TC_JOB_DEVICE_INPUTS if device_inputs else 0, nq, ptr(B) if B is not None else None)
    ticket = ctypes.c_uint64()
    s = load().tc_submit(ctx, ctypes.byref(job), ctypes.byref(ticket))
    if s != TC_OK:
        raise TcError(s, "tc_submit refused the job")
    return ticket.value


def tc_poll(ctx, ticket):
    """(status, tc_result); status TC_ENOTREADY while the job is pending."""
    res = tc_result()
    return load().tc_poll(ctx, ticket, ctypes.byref(res)), res


def tc_wait(ctx, ticket, timeout_ms=-1):
    res = tc_result()
    return load().tc_wait(ctx, ticket, timeout_ms, ctypes.byref(res)), res


def tc_cancel(ctx, ticket) -> int:
    return load().tc_cancel(ctx, ticket)


def tc_serve_stats_get(ctx) -> tc_serve_stats:
    st = tc_serve_stats()
    _check(ctx, load().tc_serve_stats_get(ctx, ctypes.byref(st)))
    return st


def tc_inject_fault(ctx, kind, param=0) -> int:
    return load().tc_inject_fault(ctx, kind, param)
