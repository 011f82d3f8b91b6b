"""Thin Python binding of liblgt (include/lgt.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Links are numpy
complex128 arrays of shape ``(N_t, N_3, N_2, N_1, 4, 3, 3)`` in host memory,
or torch CUDA tensors with the same bytes (complex128 of that shape, or
float64 with a trailing axis of 2) in device memory.  Error statuses raise
``LgtError`` with the library's message, except the informational ones
(``LGT_ENOTCONV``, ``LGT_EAGAIN``), which are returned.

The CUDA library must be built (``paper_1305_3440_gb300.build.build()``);
importing this module without it raises ImportError -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblgt.so")

LGT_OK, LGT_EINVAL, LGT_ENOMEM, LGT_ECUDA, LGT_ENOTCONV, LGT_EAGAIN, LGT_ETIMEOUT, LGT_EBUSY, \
    LGT_ECANCELLED, LGT_ENOTFOUND = range(10)
LGT_LANDAU, LGT_COULOMB, LGT_MAG = 0, 1, 2
LGT_OR, LGT_SR = 0, 1
LGT_FP64, LGT_FP32_18, LGT_FP32_12 = 0, 1, 2
LGT_POLISH_PAIR, LGT_POLISH_FP64, LGT_POLISH_ANCHOR = 0, 1, 2
LGT_POLISH_SAME, LGT_POLISH_OR = 0, 1  # lgt_params.polish_algo

STATUS_NAMES = {0: "LGT_OK", 1: "LGT_EINVAL", 2: "LGT_ENOMEM", 3: "LGT_ECUDA", 4: "LGT_ENOTCONV",
                5: "LGT_EAGAIN", 6: "LGT_ETIMEOUT", 7: "LGT_EBUSY", 8: "LGT_ECANCELLED", 9: "LGT_ENOTFOUND"}


class lgt_params(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("gauge", ctypes.c_int32), ("algo", ctypes.c_int32),
                ("bulk", ctypes.c_int32), ("transform_temporal", ctypes.c_int32), ("omega", ctypes.c_double),
                ("p", ctypes.c_double), ("seed", ctypes.c_uint64), ("sweep_offset", ctypes.c_uint64),
                ("theta_tol", ctypes.c_double), ("theta_switch", ctypes.c_double),
                ("max_sweeps", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("reunit_every", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("polish", ctypes.c_int32), ("launch_config", ctypes.c_int32), ("omega_polish", ctypes.c_double),
                ("sa_sweeps", ctypes.c_int32), ("polish_algo", ctypes.c_int32), ("sa_beta0", ctypes.c_double),
                ("sa_beta1", ctypes.c_double), ("omega_late", ctypes.c_double), ("theta_omega", ctypes.c_double)]


class lgt_result(ctypes.Structure):
    _fields_ = [("F", ctypes.c_double), ("theta", ctypes.c_double), ("plaquette", ctypes.c_double),
                ("seconds", ctypes.c_double), ("sweeps_bulk", ctypes.c_int64),
                ("sweeps_fp64", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class lgt_stats(ctypes.Structure):
    _fields_ = [("sweep_ms", ctypes.c_double * 2), ("sweep_launches", ctypes.c_int64 * 2),
                ("site_updates", ctypes.c_int64 * 2), ("launches", ctypes.c_int64),
                ("measure_ms", ctypes.c_double), ("measure_launches", ctypes.c_int64),
                ("launch_config", ctypes.c_int32 * 2), ("loop_launches", ctypes.c_int64),
                ("loop_chunks", ctypes.c_int64)]

    def as_dict(self):
        return dict(sweep_ms=list(self.sweep_ms), sweep_launches=list(self.sweep_launches),
                    site_updates=list(self.site_updates), launches=self.launches,
                    measure_ms=self.measure_ms, measure_launches=self.measure_launches,
                    launch_config=list(self.launch_config), loop_launches=self.loop_launches,
                    loop_chunks=self.loop_chunks)


class LgtError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)
_P = ctypes.POINTER
_vp = ctypes.c_void_p
_sigs = {
    "lgt_params_default": ([_P(lgt_params)], ctypes.c_int),
    "lgt_create": ([_P(lgt_params), _vp, ctypes.c_int, _vp, _P(_vp)], ctypes.c_int),
    "lgt_sweep": ([_vp, ctypes.c_int32], ctypes.c_int),
    "lgt_half_sweep": ([_vp, ctypes.c_int32], ctypes.c_int),
    "lgt_measure": ([_vp, _P(ctypes.c_double), _P(ctypes.c_double), _P(ctypes.c_double)], ctypes.c_int),
    "lgt_measure_slices": ([_vp, _vp, _vp], ctypes.c_int),
    "lgt_estimate": ([_vp, _P(ctypes.c_double), _P(ctypes.c_double), _vp, _vp], ctypes.c_int),
    "lgt_fix": ([_vp, _P(lgt_result)], ctypes.c_int),
    "lgt_promote": ([_vp], ctypes.c_int),
    "lgt_get_links": ([_vp, _vp, ctypes.c_int], ctypes.c_int),
    "lgt_get_working_links": ([_vp, _vp, ctypes.c_int], ctypes.c_int),
    "lgt_get_progress": ([_vp, _P(ctypes.c_int64), _P(ctypes.c_int64), _P(ctypes.c_int32)], ctypes.c_int),
    "lgt_load": ([_vp, _vp, ctypes.c_int], ctypes.c_int),
    "lgt_get_stats": ([_vp, _P(lgt_stats)], ctypes.c_int),
    "lgt_destroy": ([_vp], None),
    "lgt_inject_stream_stall": ([_vp, ctypes.c_uint64, ctypes.c_uint32], ctypes.c_int),
    "lgt_slab_create": ([_P(lgt_params), ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int, _vp, _P(_vp)],
                        ctypes.c_int),
    "lgt_slab_half_sweep": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "lgt_slab_boundary_bytes": ([_vp, _P(ctypes.c_size_t)], ctypes.c_int),
    "lgt_slab_boundary": ([_vp, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int32], ctypes.c_int),
    "lgt_slab_sync": ([_vp], ctypes.c_int),
    "lgt_measure_slice_sums": ([_vp, _vp], ctypes.c_int),
    "lgt_measure_noalloc": ([_P(ctypes.c_int32), _vp, _vp, _vp], ctypes.c_int),
    "lgt_server_create": ([ctypes.c_size_t, ctypes.c_int, _P(_vp)], ctypes.c_int),
    "lgt_submit": ([_vp, _P(lgt_params), _vp, _P(ctypes.c_uint64)], ctypes.c_int),
    "lgt_poll": ([_vp, ctypes.c_uint64, _P(lgt_result), _vp], ctypes.c_int),
    "lgt_cancel": ([_vp, ctypes.c_uint64], ctypes.c_int),
    "lgt_server_stats": ([_vp, _P(ctypes.c_uint64), _P(ctypes.c_uint64), _P(ctypes.c_size_t)], ctypes.c_int),
    "lgt_server_counters": ([_vp] + [_P(ctypes.c_uint64)] * 4, ctypes.c_int),
    "lgt_server_destroy": ([_vp], None),
    "lgt_last_error": ([], ctypes.c_char_p),
    "lgt_version": ([], ctypes.c_char_p),
}
for _name, (_args, _res) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def lgt_last_error() -> str:
    return _lib.lgt_last_error().decode()


def lgt_version() -> str:
    return _lib.lgt_version().decode()


def _check(status, allowed=(LGT_OK,)):
    if status not in allowed:
        raise LgtError(status, lgt_last_error())
    return status


def lgt_params_default(**overrides) -> lgt_params:
    """Defaults of the library, then the given fields (dims as a 4-sequence)."""
    p = lgt_params()
    _check(_lib.lgt_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        if k == "dims":
            p.dims[:] = [int(d) for d in v]
        else:
            setattr(p, k, v)
    return p


def _links_arg(links, dims=None):
    """(pointer, on_device, keepalive) for a numpy or torch links buffer."""
    if isinstance(links, np.ndarray):
        if links.dtype != np.complex128 or not links.flags.c_contiguous:
            raise TypeError("host links must be C-contiguous complex128")
        return links.ctypes.data, 0, links
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(links, torch.Tensor):
        if not links.is_cuda:
            a = links.numpy()
            return _links_arg(np.ascontiguousarray(a))
        if links.dtype not in (torch.complex128, torch.float64) or not links.is_contiguous():
            raise TypeError("device links must be contiguous complex128 or float64")
        return links.data_ptr(), 1, links
    raise TypeError(f"unsupported links type {type(links)}")


def _stream_arg(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def lgt_create(params: lgt_params, links, stream=None):
    """Context handle (c_void_p) for ``links`` (numpy host array or torch CUDA tensor)."""
    ptr, on_dev, _keep = _links_arg(links)
    out = _vp()
    _check(_lib.lgt_create(ctypes.byref(params), ptr, on_dev, _stream_arg(stream), ctypes.byref(out)))
    return out


def lgt_slab_create(params: lgt_params, nt_global: int, t0: int, links, stream=None):
    """Context of a temporal slab: params.dims[0] owned slices starting at global slice t0."""
    ptr, on_dev, _keep = _links_arg(links)
    out = _vp()
    _check(_lib.lgt_slab_create(ctypes.byref(params), int(nt_global), int(t0), ptr, on_dev, _stream_arg(stream),
                                ctypes.byref(out)))
    return out


def lgt_slab_half_sweep(ctx, parity: int, first: int, count: int) -> None:
    _check(_lib.lgt_slab_half_sweep(ctx, int(parity), int(first), int(count)))


def lgt_slab_boundary_bytes(ctx) -> int:
    n = ctypes.c_size_t()
    _check(_lib.lgt_slab_boundary_bytes(ctx, ctypes.byref(n)))
    return n.value


def lgt_slab_boundary(ctx, slice_: int, parity: int, buf, into_slab: bool) -> None:
    """Copy U_0 of one parity on one owned slice (-1: the halo) to / from buf, a
    contiguous torch CUDA tensor of lgt_slab_boundary_bytes bytes."""
    _check(_lib.lgt_slab_boundary(ctx, int(slice_), int(parity), buf.data_ptr(), 1 if into_slab else 0))


def lgt_slab_sync(ctx) -> None:
    _check(_lib.lgt_slab_sync(ctx))


def lgt_measure_slice_sums(ctx, nt: int):
    """Exact per-slice sums, shape (nt, 5) (see lgt.h); nt = the owned slices of a slab."""
    out = np.zeros((int(nt), 5))
    _check(_lib.lgt_measure_slice_sums(ctx, out.ctypes.data))
    return out


def lgt_sweep(ctx, n: int) -> None:
    _check(_lib.lgt_sweep(ctx, int(n)))


def lgt_half_sweep(ctx, parity: int) -> None:
    _check(_lib.lgt_half_sweep(ctx, int(parity)))


def lgt_measure(ctx):
    """(F, theta, plaquette) of the working field."""
    F, th, pl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.lgt_measure(ctx, ctypes.byref(F), ctypes.byref(th), ctypes.byref(pl)))
    return F.value, th.value, pl.value


def lgt_measure_slices(ctx, nt: int):
    F_t = np.zeros(int(nt))
    th_t = np.zeros(int(nt))
    _check(_lib.lgt_measure_slices(ctx, F_t.ctypes.data, th_t.ctypes.data))
    return F_t, th_t


def lgt_estimate(ctx, nt: int):
    """(F, theta, F_t, theta_t) of the sweeps' fused estimate of the last full sweep."""
    F, th = ctypes.c_double(), ctypes.c_double()
    F_t = np.zeros(int(nt))
    th_t = np.zeros(int(nt))
    _check(_lib.lgt_estimate(ctx, ctypes.byref(F), ctypes.byref(th), F_t.ctypes.data, th_t.ctypes.data))
    return F.value, th.value, F_t, th_t


def lgt_inject_stream_stall(ctx, wait_ns: int, skip_items: int) -> None:
    """Test support: bounded-wait fault injection for streaming launches (see lgt.h)."""
    _check(_lib.lgt_inject_stream_stall(ctx, int(wait_ns), int(skip_items)))


def lgt_fix(ctx):
    """(status, lgt_result); status is LGT_OK or LGT_ENOTCONV."""
    res = lgt_result()
    st = _check(_lib.lgt_fix(ctx, ctypes.byref(res)), (LGT_OK, LGT_ENOTCONV))
    return st, res


def lgt_promote(ctx) -> None:
    _check(_lib.lgt_promote(ctx))


def _out_arg(out, dims):
    if out is None:
        out = np.empty(tuple(dims) + (4, 3, 3), np.complex128)
    ptr, on_dev, _ = _links_arg(out)
    return out, ptr, on_dev


def lgt_get_links(ctx, dims=None, out=None):
    """The current field (FP64); into ``out`` (numpy or torch CUDA) or a new numpy array."""
    out, ptr, on_dev = _out_arg(out, dims)
    _check(_lib.lgt_get_links(ctx, ptr, on_dev))
    return out


def lgt_get_working_links(ctx, dims=None, out=None):
    out, ptr, on_dev = _out_arg(out, dims)
    _check(_lib.lgt_get_working_links(ctx, ptr, on_dev))
    return out


def lgt_get_progress(ctx):
    """(sweeps_bulk, sweeps_fp64, phase)."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(_lib.lgt_get_progress(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def lgt_load(ctx, links) -> None:
    """Replace the context's field (numpy host array or torch CUDA tensor) and restart."""
    ptr, on_dev, _keep = _links_arg(links)
    _check(_lib.lgt_load(ctx, ptr, on_dev))


def lgt_get_stats(ctx) -> lgt_stats:
    st = lgt_stats()
    _check(_lib.lgt_get_stats(ctx, ctypes.byref(st)))
    return st


def lgt_measure_noalloc(dims, links_device, out_device, stream=None) -> None:
    """Asynchronous exact measurement of device links into a device buffer of at
    least 8 + 2*N_t doubles (see include/lgt.h); nothing is allocated."""
    d = (ctypes.c_int32 * 4)(*[int(x) for x in dims])
    ptr, on_dev, _ = _links_arg(links_device)
    if not on_dev:
        raise TypeError("lgt_measure_noalloc takes device links")
    if not getattr(out_device, "is_cuda", False):
        raise TypeError("lgt_measure_noalloc writes a device buffer")
    optr = out_device.data_ptr()
    _check(_lib.lgt_measure_noalloc(d, ptr, optr, _stream_arg(stream)))


def lgt_destroy(ctx) -> None:
    _lib.lgt_destroy(ctx)


def lgt_server_create(hbm_budget_bytes: int, device: int = 0):
    out = _vp()
    _check(_lib.lgt_server_create(int(hbm_budget_bytes), int(device), ctypes.byref(out)))
    return out


def lgt_submit(server, params: lgt_params, links: np.ndarray) -> int:
    ptr, on_dev, _keep = _links_arg(links)
    if on_dev:
        raise TypeError("lgt_submit takes host links")
    jid = ctypes.c_uint64()
    _check(_lib.lgt_submit(server, ctypes.byref(params), ptr, ctypes.byref(jid)))
    return jid.value


def lgt_poll(server, job_id: int, links_out: np.ndarray | None = None):
    """(status, lgt_result); status LGT_EAGAIN while the job runs, else the job's final
    status (LGT_OK, LGT_ENOTCONV, LGT_ECANCELLED, or the error that ended it)."""
    res = lgt_result()
    ptr = None
    if links_out is not None:
        ptr, on_dev, _ = _links_arg(links_out)
        if on_dev:
            raise TypeError("lgt_poll writes host links")
    st = _lib.lgt_poll(server, int(job_id), ctypes.byref(res), ptr)
    if st == LGT_ENOTFOUND:
        raise LgtError(st, lgt_last_error())
    return st, res


def lgt_cancel(server, job_id: int) -> None:
    _check(_lib.lgt_cancel(server, int(job_id)))


def lgt_server_stats(server):
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_size_t()
    _check(_lib.lgt_server_stats(server, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def lgt_server_counters(server) -> dict:
    """Ticks run, ticks replayed from captured CUDA graphs, graphs captured, kernel launches."""
    v = [ctypes.c_uint64() for _ in range(4)]
    _check(_lib.lgt_server_counters(server, *[ctypes.byref(x) for x in v]))
    return dict(zip(("ticks", "graph_launches", "graph_captures", "kernel_launches"), (x.value for x in v)))


def lgt_server_destroy(server) -> None:
    _lib.lgt_server_destroy(server)
