"""Thin ctypes binding of ``liblcs_gb300.so`` (declared in ``include/lcs.h``).

Every function here has the name of the C entry point it calls and does
argument marshalling only (torch tensors -> device pointers, sizes, strides,
the current CUDA stream); every step of the computation runs in the library's
CUDA kernels.  There is no fallback: if the library is missing or fails to
load, :func:`load` raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblcs_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "lcs.h")

LCS_OK, LCS_EINVAL, LCS_ENOMEM, LCS_ETIMEOUT, LCS_ECUDA, LCS_EAGAIN, LCS_EOVERFLOW = range(7)
LCS_I32, LCS_I16 = 0, 1


class LcsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s (status %d): %s" % (fn_strerror(status), status, message))
        self.status = status


class lcs_stats(ctypes.Structure):
    _fields_ = [
        ("workspace_bytes", ctypes.c_int64),
        ("peak_workspace_bytes", ctypes.c_int64),
        ("strip_height", ctypes.c_int32),
        ("strips", ctypes.c_int32),
        ("merges", ctypes.c_int32),
        ("tree_levels", ctypes.c_int32),
        ("kernel_launches", ctypes.c_int32),
        ("tile", ctypes.c_int32),
        ("depth_first", ctypes.c_int32),
        ("chunk_strips", ctypes.c_int32),
        ("plan_bytes", ctypes.c_int64),
    ]


class lcs_kernel_profile(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("launches", ctypes.c_int32),
        ("ms", ctypes.c_double),
        ("bytes", ctypes.c_double),
        ("ops", ctypes.c_double),
    ]


class lcs_plan_info(ctypes.Structure):
    _fields_ = [
        ("workspace_bytes", ctypes.c_int64),
        ("fits", ctypes.c_int32),
        ("strip_height", ctypes.c_int32),
        ("strips", ctypes.c_int32),
        ("nodes", ctypes.c_int32),
        ("levels", ctypes.c_int32),
        ("depth_first", ctypes.c_int32),
        ("chunk", ctypes.c_int32),
        ("launches", ctypes.c_int32),
        ("root", ctypes.c_int32),
        ("tile", ctypes.c_int32),
    ]


class lcs_plan_node(ctypes.Structure):
    _fields_ = [
        ("row0", ctypes.c_int64),
        ("rows", ctypes.c_int64),
        ("offset", ctypes.c_int64),
        ("bytes", ctypes.c_int64),
        ("grid_offset", ctypes.c_int64),
        ("grid_bytes", ctypes.c_int64),
        ("upper", ctypes.c_int32),
        ("lower", ctypes.c_int32),
        ("parent", ctypes.c_int32),
        ("level", ctypes.c_int32),
        ("made_by", ctypes.c_int32),
        ("last_use", ctypes.c_int32),
        ("grid_last_use", ctypes.c_int32),
    ]


LCS_WANT_STRING = 1


class lcs_pair(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_void_p),
        ("m", ctypes.c_int64),
        ("b", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("flags", ctypes.c_uint32),
    ]


class lcs_result(ctypes.Structure):
    _fields_ = [
        ("len", ctypes.c_int64),
        ("string_offset", ctypes.c_int64),
        ("status", ctypes.c_int),
        ("t_submit", ctypes.c_double),
        ("t_done", ctypes.c_double),
    ]


KERNEL_KINDS = {0: "strip", 1: "coarse", 2: "merge_tile", 3: "traceback_level", 4: "traceback_leaf",
                5: "compact", 6: "fill"}

_lib = None
_lock = threading.Lock()


def declared_symbols(header: str = HEADER):
    """Names of the entry points declared in include/lcs.h."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lcs_[a-z_0-9]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load the library (building it first if it is absent and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            from . import build as _build
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError("liblcs_gb300.so is missing: run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        st = ctypes.c_int
        sig = {
            "lcs_create": ([ctypes.POINTER(vp), ctypes.c_int, sz], st),
            "lcs_destroy": ([vp], st),
            "lcs_strerror": ([st], ctypes.c_char_p),
            "lcs_last_error": ([vp], ctypes.c_char_p),
            "lcs_set_strip_height": ([vp, i32], st),
            "lcs_set_merge_kernel": ([vp, i32], st),
            "lcs_set_graphs": ([vp, i32], st),
            "lcs_set_fault_injection": ([vp, i32, i64], st),
            "lcs_set_schedule": ([vp, i32, i32], st),
            "lcs_plan": ([i64, i64, i32, i32, i32, sz, i32, st, ctypes.POINTER(lcs_plan_info),
                          ctypes.POINTER(lcs_plan_node), i64], st),
            "lcs_autotune": ([vp, vp, i64, vp, i64, i32, vp, i64, vp, i64, vp, ctypes.POINTER(i32),
                              ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)], st),
            "lcs_get_stats": ([vp, ctypes.POINTER(lcs_stats)], st),
            "lcs_sync": ([vp, vp], st),
            "lcs_set_profiling": ([vp, i32], st),
            "lcs_get_profile": ([vp, ctypes.POINTER(lcs_kernel_profile), i32, ctypes.POINTER(i32)], st),
            "lcs_measure_int32_peak": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)], st),
            "lcs_strip_dist": ([vp, vp, i32, vp, i64, st, vp, i64, vp], st),
            "lcs_merge": ([vp, vp, vp, i64, st, i64, vp, vp, vp], st),
            "lcs_merge_static": ([vp, vp, i64, st, i64, vp, vp, vp], st),
            "lcs_dist": ([vp, vp, i64, vp, i64, st, vp, i64, vp], st),
            "lcs_length": ([vp, vp, i64, vp, i64, ctypes.POINTER(i64), vp], st),
            "lcs_traceback": ([vp, vp, i64, vp, i64, vp, i64, ctypes.POINTER(i64), vp], st),
            "lcs_path": ([vp, vp, i64, vp, i64, vp, i64, ctypes.POINTER(i64), vp], st),
            "lcs_strip_dform": ([vp, vp, i64, i32, vp, i64, i32, vp, i64, vp], st),
            "lcs_dform_merge": ([vp, vp, i32, i64, vp, i32, i64, i64, i32, vp, i64, vp], st),
            "lcs_solve": ([vp, vp, i64, vp, i64, st, vp, i64, vp, i64, vp, vp, vp], st),
            "lcs_solve_host": ([vp, vp, i64, vp, i64, st, vp, i64, vp, i64, ctypes.POINTER(i64), vp], st),
            "lcs_batch_submit": ([vp, ctypes.POINTER(lcs_pair), i64, ctypes.POINTER(ctypes.c_uint64)], st),
            "lcs_batch_poll": ([vp, ctypes.c_uint64, ctypes.POINTER(lcs_result), i64, ctypes.POINTER(i64), i32], st),
            "lcs_batch_strings": ([vp, ctypes.c_uint64, vp, i64, ctypes.POINTER(i64)], st),
            "lcs_batch_release": ([vp, ctypes.c_uint64], st),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def fn_strerror(status: int) -> str:
    try:
        return load().lcs_strerror(int(status)).decode()
    except Exception:  # noqa: BLE001 - message only
        return "status"


# ------------------------------------------------------------------ marshalling helpers
def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_of(t) -> int:
    import torch
    if t.dtype == torch.int32:
        return LCS_I32
    if t.dtype == torch.int16:
        return LCS_I16
    raise ValueError("DIST tensors are int32 or int16")


def _ld(t) -> int:
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("DIST tensors are 2-D with unit column stride")
    return int(t.stride(0))


def _place(t, name: str, device: bool) -> None:
    if device and not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not device and t.is_cuda:
        raise ValueError("%s must be a host (CPU) tensor" % name)


def _seq(t, name: str, device: bool = True):
    """A string: contiguous uint8 bytes on the device (or the host)."""
    import torch
    if t.dtype != torch.uint8 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous uint8 tensor" % name)
    _place(t, name, device)
    return _ptr(t), int(t.numel())


def _out(t, name: str, dtype, device: bool = True):
    """An output buffer of one element type, contiguous; None passes through."""
    if t is None:
        return None
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError("%s must be a contiguous %s tensor" % (name, str(dtype).replace("torch.", "")))
    _place(t, name, device)
    return _ptr(t)


def _mat(t, name: str, device: bool = True) -> int:
    """A DIST / breakout matrix: 2-D, unit column stride; returns ld."""
    ld = _ld(t)
    _dtype_of(t)
    _place(t, name, device)
    return ld


def _check(ctx, status):
    if status != LCS_OK:
        msg = load().lcs_last_error(ctx)
        raise LcsError(status, msg.decode() if msg else "")


# ------------------------------------------------------------------ entry points
def lcs_create(device: int = 0, mem_budget_bytes: int = 0):
    ctx = ctypes.c_void_p()
    _check(None, load().lcs_create(ctypes.byref(ctx), int(device), int(mem_budget_bytes)))
    return ctx


def lcs_destroy(ctx) -> None:
    _check(ctx, load().lcs_destroy(ctx))


def lcs_strerror(status: int) -> str:
    return load().lcs_strerror(int(status)).decode()


def lcs_last_error(ctx) -> str:
    return load().lcs_last_error(ctx).decode()


def lcs_set_strip_height(ctx, h: int) -> None:
    _check(ctx, load().lcs_set_strip_height(ctx, int(h)))


LCS_MERGE_AUTO, LCS_MERGE_EXACT, LCS_MERGE_DPX = 0, 1, 2


def lcs_set_merge_kernel(ctx, kind: int) -> None:
    _check(ctx, load().lcs_set_merge_kernel(ctx, int(kind)))


LCS_SCHED_AUTO, LCS_SCHED_RETAIN, LCS_SCHED_DEPTH = 0, 1, 2


def lcs_set_schedule(ctx, mode: int, chunk: int = 0) -> None:
    _check(ctx, load().lcs_set_schedule(ctx, int(mode), int(chunk)))


def lcs_plan(m: int, n: int, h: int = 0, schedule: int = LCS_SCHED_AUTO, chunk: int = 0, budget_bytes: int = 0,
             want_lcs: bool = True, dtype: int = LCS_I32):
    """The tree plan a solve of an m x n pair would use (host only, no
    device): (info dict, list of node dicts)."""
    lib = load()
    info = lcs_plan_info()
    st = lib.lcs_plan(int(m), int(n), int(h), int(schedule), int(chunk), int(budget_bytes), 1 if want_lcs else 0,
                      int(dtype), ctypes.byref(info), None, 0)
    if st != LCS_OK:
        raise LcsError(st, "lcs_plan arguments")
    recs = (lcs_plan_node * max(1, info.nodes))()
    st = lib.lcs_plan(int(m), int(n), int(h), int(schedule), int(chunk), int(budget_bytes), 1 if want_lcs else 0,
                      int(dtype), ctypes.byref(info), recs, int(info.nodes))
    if st != LCS_OK:
        raise LcsError(st, "lcs_plan arguments")
    nodes = [{name: getattr(recs[v], name) for name, _ in lcs_plan_node._fields_} for v in range(info.nodes)]
    return {name: getattr(info, name) for name, _ in info._fields_}, nodes


def lcs_set_fault_injection(ctx, hold_band: bool, wait_limit_ns: int = 0) -> None:
    _check(ctx, load().lcs_set_fault_injection(ctx, 1 if hold_band else 0, int(wait_limit_ns)))


def lcs_set_graphs(ctx, enable: bool) -> None:
    _check(ctx, load().lcs_set_graphs(ctx, 1 if enable else 0))


def lcs_autotune(ctx, a, b, dist=None, out_lcs=None, stream=None) -> dict:
    """Time the candidate strip heights / merge kernels on this call's shape
    and outputs; returns the choice kept for the size bucket."""
    import torch
    (pa, m), (pb, n) = _seq(a, "a"), _seq(b, "b")
    dtype = _dtype_of(dist) if dist is not None else LCS_I32
    ld = _mat(dist, "dist") if dist is not None else 0
    cap = int(out_lcs.numel()) if out_lcs is not None else 0
    h, mk, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(ctx, load().lcs_autotune(ctx, pa, m, pb, n, dtype, _ptr(dist), ld,
                                    _out(out_lcs, "out_lcs", torch.uint8), cap, _stream(stream), ctypes.byref(h),
                                    ctypes.byref(mk), ctypes.byref(ms)))
    return {"strip_height": h.value, "merge_kernel": mk.value, "ms": ms.value}


def lcs_get_stats(ctx) -> dict:
    s = lcs_stats()
    _check(ctx, load().lcs_get_stats(ctx, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in s._fields_}


def lcs_set_profiling(ctx, enable: bool) -> None:
    _check(ctx, load().lcs_set_profiling(ctx, 1 if enable else 0))


def lcs_get_profile(ctx) -> dict:
    """{kind name: {launches, ms, bytes, ops}} accumulated since profiling was enabled."""
    arr = (lcs_kernel_profile * 8)()
    cnt = ctypes.c_int32()
    _check(ctx, load().lcs_get_profile(ctx, arr, 8, ctypes.byref(cnt)))
    out = {}
    for k in range(cnt.value):
        e = arr[k]
        out[KERNEL_KINDS.get(e.kind, str(e.kind))] = {"launches": e.launches, "ms": e.ms, "bytes": e.bytes,
                                                      "ops": e.ops}
    return out


def lcs_measure_int32_peak(device: int = 0):
    """(10^9 INT32 ops/s, SM MHz seen by the kernel)."""
    g, mhz = ctypes.c_double(), ctypes.c_double()
    _check(None, load().lcs_measure_int32_peak(int(device), ctypes.byref(g), ctypes.byref(mhz)))
    return g.value, mhz.value


def lcs_sync(ctx, stream=None) -> None:
    _check(ctx, load().lcs_sync(ctx, _stream(stream)))


def lcs_strip_dist(ctx, a_strip, b, dist, stream=None) -> None:
    """dist[i, j] = LCS(a_strip, b[i:j]) (dense (n+1) x ld int32/int16)."""
    (pa, h), (pb, n) = _seq(a_strip, "a_strip"), _seq(b, "b")
    ld = _mat(dist, "dist")
    _check(ctx, load().lcs_strip_dist(ctx, pa, h, pb, n, _dtype_of(dist), _ptr(dist), ld, _stream(stream)))


def _merge_args(dist_u, dist_l, dist_out, argmax_out):
    """(n, ld) of a merge's matrices: one dtype and one ld, on the device."""
    import torch
    ld = _mat(dist_u, "dist_u")
    _mat(dist_l, "dist_l")
    _mat(dist_out, "dist_out")
    if dist_l.dtype != dist_u.dtype or dist_out.dtype != dist_u.dtype or dist_l.stride(0) != ld \
            or dist_out.stride(0) != ld:
        raise ValueError("dist_u, dist_l and dist_out share one dtype and one ld")
    if argmax_out is not None:
        if argmax_out.dtype != torch.int32 or argmax_out.dim() != 2 or argmax_out.stride(1) != 1 \
                or argmax_out.stride(0) != ld:
            raise ValueError("argmax_out must be int32 with the matrices' ld")
        _place(argmax_out, "argmax_out", True)
    return int(dist_u.shape[0]) - 1, ld


def lcs_merge(ctx, dist_u, dist_l, dist_out, argmax_out=None, stream=None) -> None:
    """dist_out[i, j] = max_k dist_u[i, k] + dist_l[k, j]; argmax_out = smallest k."""
    n, ld = _merge_args(dist_u, dist_l, dist_out, argmax_out)
    _check(ctx, load().lcs_merge(ctx, _ptr(dist_u), _ptr(dist_l), n, _dtype_of(dist_u), ld,
                                 _ptr(dist_out), _ptr(argmax_out), _stream(stream)))


def lcs_merge_static(dist_u, dist_l, dist_out, argmax_out=None, stream=None) -> None:
    """lcs_merge with all scratch in the library's static device array (no
    allocation, n <= 1024, synchronous)."""
    n, ld = _merge_args(dist_u, dist_l, dist_out, argmax_out)
    _check(None, load().lcs_merge_static(_ptr(dist_u), _ptr(dist_l), n, _dtype_of(dist_u), ld,
                                         _ptr(dist_out), _ptr(argmax_out), _stream(stream)))


def lcs_dist(ctx, a, b, dist, stream=None) -> None:
    (pa, m), (pb, n) = _seq(a, "a"), _seq(b, "b")
    ld = _mat(dist, "dist")
    _check(ctx, load().lcs_dist(ctx, pa, m, pb, n, _dtype_of(dist), _ptr(dist), ld, _stream(stream)))


def lcs_length(ctx, a, b, stream=None) -> int:
    (pa, m), (pb, n) = _seq(a, "a"), _seq(b, "b")
    out = ctypes.c_int64()
    _check(ctx, load().lcs_length(ctx, pa, m, pb, n, ctypes.byref(out), _stream(stream)))
    return out.value


def lcs_traceback(ctx, a, b, out_lcs, stream=None) -> int:
    import torch
    (pa, m), (pb, n) = _seq(a, "a"), _seq(b, "b")
    out = ctypes.c_int64()
    _check(ctx, load().lcs_traceback(ctx, pa, m, pb, n, _out(out_lcs, "out_lcs", torch.uint8),
                                     int(out_lcs.numel()), ctypes.byref(out), _stream(stream)))
    return out.value


def lcs_strip_dform(ctx, a, b, dform, h=None, stream=None) -> None:
    """Breakout matrices of a's strips of h rows (default: one strip of all of
    a) into ``dform``: shape (S, n+1, ldf) or, for one strip, (n+1, ldf);
    int32 or int16."""
    (pa, m), (pb, n) = _seq(a, "a"), _seq(b, "b")
    h = m if h is None else int(h)
    if dform.dim() not in (2, 3):
        raise ValueError("dform is (n+1, ldf) or (S, n+1, ldf)")
    d2 = dform if dform.dim() == 2 else dform[0]
    _mat(d2, "dform")
    if dform.dim() == 3 and dform.stride(0) != (int(b.numel()) + 1) * d2.stride(0):
        raise ValueError("strips of dform must be contiguous (n+1) x ldf blocks")
    _check(ctx, load().lcs_strip_dform(ctx, pa, m, h, pb, n, _dtype_of(d2), _ptr(dform), _ld(d2),
                                       _stream(stream)))


def lcs_dform_merge(ctx, du, hu, dl, hl, out, stream=None) -> None:
    """Combination of two breakout matrices (rows = top vertices) into ``out``."""
    n = int(du.shape[0]) - 1
    ldu, ldl, ldo = _mat(du, "du"), _mat(dl, "dl"), _mat(out, "out")
    if du.dtype != out.dtype or dl.dtype != out.dtype:
        raise ValueError("du, dl and out share one dtype")
    _check(ctx, load().lcs_dform_merge(ctx, _ptr(du), int(hu), ldu, _ptr(dl), int(hl), ldl, n,
                                       _dtype_of(out), _ptr(out), ldo, _stream(stream)))


def lcs_path(ctx, a, b, path, stream=None) -> int:
    """Vertices of the leftmost heaviest path into ``path`` (int32, shape
    (cap, 2) of (row, col) pairs); returns their number."""
    import torch
    (pa, m), (pb, n) = _seq(a, "a"), _seq(b, "b")
    out = ctypes.c_int64()
    cap = int(path.numel()) // 2 if path is not None else 0
    _check(ctx, load().lcs_path(ctx, pa, m, pb, n, _out(path, "path", torch.int32), cap,
                                ctypes.byref(out), _stream(stream)))
    return out.value


def lcs_solve(ctx, a, b, dist=None, out_lcs=None, cross=None, out_len=None, stream=None) -> None:
    """Asynchronous whole path; any output may be None (see lcs.h)."""
    import torch
    (pa, m), (pb, n) = _seq(a, "a"), _seq(b, "b")
    dtype = _dtype_of(dist) if dist is not None else LCS_I32
    ld = _mat(dist, "dist") if dist is not None else 0
    cap = int(out_lcs.numel()) if out_lcs is not None else 0
    _check(ctx, load().lcs_solve(ctx, pa, m, pb, n, dtype, _ptr(dist), ld,
                                 _out(out_lcs, "out_lcs", torch.uint8), cap, _out(cross, "cross", torch.int32),
                                 _out(out_len, "out_len", torch.int64), _stream(stream)))


def lcs_solve_host(ctx, a_host, b_host, dist_host=None, lcs_host=None, dtype=LCS_I32, stream=None) -> int:
    """Whole path on host (ideally pinned) tensors; returns the LCS length."""
    import torch
    (pa, m), (pb, n) = _seq(a_host, "a_host", device=False), _seq(b_host, "b_host", device=False)
    out = ctypes.c_int64()
    if dist_host is not None:
        dtype = _dtype_of(dist_host)
    ld = _mat(dist_host, "dist_host", device=False) if dist_host is not None else 0
    cap = int(lcs_host.numel()) if lcs_host is not None else 0
    _check(ctx, load().lcs_solve_host(ctx, pa, m, pb, n, dtype, _ptr(dist_host), ld,
                                      _out(lcs_host, "lcs_host", torch.uint8, device=False), cap,
                                      ctypes.byref(out), _stream(stream)))
    return out.value


def lcs_batch_submit(ctx, pairs) -> int:
    """Queue pairs [(a, b) or (a, b, want_string)] of device uint8 tensors;
    returns the ticket.  The tensors must stay alive until the batch is done."""
    arr = (lcs_pair * max(1, len(pairs)))()
    for k, pr in enumerate(pairs):
        a, b = pr[0], pr[1]
        _seq(a, "a of pair %d" % k)
        _seq(b, "b of pair %d" % k)
        want = pr[2] if len(pr) > 2 else True
        arr[k].a = a.data_ptr() if a.numel() else None
        arr[k].m = int(a.numel())
        arr[k].b = b.data_ptr() if b.numel() else None
        arr[k].n = int(b.numel())
        arr[k].flags = LCS_WANT_STRING if want else 0
    ticket = ctypes.c_uint64()
    _check(ctx, load().lcs_batch_submit(ctx, arr, len(pairs), ctypes.byref(ticket)))
    return ticket.value


def lcs_batch_poll(ctx, ticket: int, count: int, timeout_ms: int = -1):
    """List of result dicts when the batch is done within timeout_ms, else None."""
    arr = (lcs_result * max(1, count))()
    done = ctypes.c_int64()
    _check(ctx, load().lcs_batch_poll(ctx, ticket, arr, count, ctypes.byref(done), int(timeout_ms)))
    if done.value == 0 and count > 0:
        return None
    return [{"len": r.len, "string_offset": r.string_offset, "status": r.status, "t_submit": r.t_submit,
             "t_done": r.t_done} for r in arr[:count]]


def lcs_batch_strings(ctx, ticket: int) -> bytes:
    """The batch's string buffer (each pair's LCS at its string_offset)."""
    import torch
    size = ctypes.c_int64()
    probe = ctypes.c_int64()
    status = load().lcs_batch_strings(ctx, ticket, None, 0, ctypes.byref(probe))
    if status not in (LCS_OK, LCS_EOVERFLOW):
        _check(ctx, status)
    buf = torch.empty(max(1, probe.value), dtype=torch.uint8)
    _check(ctx, load().lcs_batch_strings(ctx, ticket, _ptr(buf), int(probe.value), ctypes.byref(size)))
    return bytes(buf[: size.value].numpy().tobytes())


def lcs_batch_release(ctx, ticket: int) -> None:
    _check(ctx, load().lcs_batch_release(ctx, ticket))


class Context:
    """Owns one lcs_ctx (one per host thread)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.handle = lcs_create(device, mem_budget_bytes)

    def close(self):
        if self.handle is not None:
            lcs_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
