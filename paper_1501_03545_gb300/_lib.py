"""ctypes binding of libhrg.so (include/hrg.h).  Argument marshalling only.

The functions keep the C names.  Device buffers are torch CUDA tensors (used
for allocation and streams only); every step of the generator runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is missing
or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

HRG_OK, HRG_EINVAL, HRG_ENOMEM, HRG_EOVERFLOW, HRG_ECUDA, HRG_ESTATE, HRG_EINTERNAL, HRG_ETIMEOUT = range(8)
HRG_FLAG_FP64_ONLY = 0x1

# every symbol declared in include/hrg.h
EXPORTS = (
    "hrg_solve_radius", "hrg_expected_degree", "hrg_create", "hrg_destroy", "hrg_generate_begin",
    "hrg_generate_from_points_begin", "hrg_generate_finish", "hrg_job_stats", "hrg_job_release",
    "hrg_generate", "hrg_generate_host", "hrg_last_error", "hrg_version", "hrg_row_offsets_noalloc",
    "hrg_generate_batch_begin", "hrg_server_create", "hrg_server_submit", "hrg_server_wait", "hrg_server_release",
    "hrg_server_stats", "hrg_server_last_error", "hrg_server_destroy", "hrg_graph_props", "hrg_degree_histogram",
    "hrg_add_random_edges", "hrg_bfs", "hrg_diameter_bounds", "hrg_set_limits", "hrg_update_begin",
    "hrg_workspace_bytes", "hrg_release_workspace",
)
HRG_PROPS_TRIANGLES = 0x1


class HrgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hrg error %d: %s" % (code, msg))
        self.code = code


class hrg_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("alpha", ctypes.c_double), ("avg_degree", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("R_override", ctypes.c_double), ("flags", ctypes.c_uint32),
                ("bands", ctypes.c_int32), ("hub_candidates", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class hrg_stats(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("n_entries", ctypes.c_int64), ("candidates", ctypes.c_uint64),
                ("rechecks", ctypes.c_uint64), ("bands", ctypes.c_int32), ("hub_bands", ctypes.c_int32),
                ("buckets", ctypes.c_int64), ("hub_queries", ctypes.c_int32), ("mid_rows", ctypes.c_int32),
                ("big_rows", ctypes.c_int32), ("reserved", ctypes.c_int32), ("mu", ctypes.c_float),
                ("stage_ms", ctypes.c_float * 8), ("launches", ctypes.c_int32), ("ties", ctypes.c_uint64),
                ("rows_no_room", ctypes.c_int64), ("hub_rows_retraversed", ctypes.c_int32),
                ("heavy_retries", ctypes.c_int32), ("write_chunks", ctypes.c_int32), ("d2h_ms", ctypes.c_float)]

    STAGES = ("sample", "bands", "count_hub", "count_rim", "offsets", "write_hub", "write_rim", "rowsort")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("reserved", "stage_ms")}
        d["stage_ms"] = {s: float(self.stage_ms[i]) for i, s in enumerate(self.STAGES)}
        return d


class hrg_limits(ctypes.Structure):
    _fields_ = [("row_buffer_ids", ctypes.c_int64), ("hub_pool_ids", ctypes.c_int64), ("hub_runs", ctypes.c_int32),
                ("heavy_segments", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64)]


class hrg_props(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("entries", ctypes.c_int64), ("max_degree", ctypes.c_int64),
                ("d_min", ctypes.c_int64), ("tail_count", ctypes.c_int64), ("tail_log_sum", ctypes.c_double),
                ("gamma", ctypes.c_double), ("triads", ctypes.c_int64), ("triangles", ctypes.c_int64),
                ("clustering", ctypes.c_double), ("avg_local_clustering", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_PI64 = ctypes.POINTER(ctypes.c_int64)


def library_path() -> str:
    return _build.SO


def load(build_if_missing: bool = True):
    """Loads libhrg.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.SO):
            raise RuntimeError("libhrg.so is not built (python -m paper_1501_03545_gb300.build)")
        L = ctypes.CDLL(_build.SO)
        L.hrg_solve_radius.argtypes = [_I64, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
        L.hrg_expected_degree.argtypes = [_I64, ctypes.c_double, ctypes.c_double]
        L.hrg_expected_degree.restype = ctypes.c_double
        L.hrg_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int]
        L.hrg_destroy.argtypes = [_P]
        L.hrg_generate_begin.argtypes = [_P, ctypes.POINTER(hrg_params), _P, _P, _P, _P, ctypes.POINTER(_P), _PI64]
        L.hrg_generate_from_points_begin.argtypes = [_P, _I64, ctypes.c_double, _P, _P, ctypes.c_uint32,
                                                     ctypes.c_int32, _P, _P, ctypes.POINTER(_P), _PI64]
        L.hrg_generate_finish.argtypes = [_P, _P]
        L.hrg_job_stats.argtypes = [_P, ctypes.POINTER(hrg_stats)]
        L.hrg_job_release.argtypes = [_P]
        L.hrg_generate.argtypes = [_P, ctypes.POINTER(hrg_params), _P, _P, _P, _P, _P, _I64, _PI64,
                                   ctypes.POINTER(hrg_stats)]
        L.hrg_generate_host.argtypes = [_P, ctypes.POINTER(hrg_params), _P, _P, _P, _P, _I64, _PI64,
                                        ctypes.POINTER(hrg_stats)]
        L.hrg_last_error.argtypes = [_P]
        L.hrg_last_error.restype = ctypes.c_char_p
        L.hrg_version.restype = ctypes.c_char_p
        L.hrg_row_offsets_noalloc.argtypes = [_P, _I64, _P, _P]
        L.hrg_generate_batch_begin.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(hrg_params), ctypes.c_uint32, _P,
                                               _P, _P, _P, ctypes.POINTER(_P), _PI64]
        L.hrg_server_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int32, _I64]
        L.hrg_server_submit.argtypes = [_P, ctypes.POINTER(hrg_params), _PI64]
        L.hrg_server_wait.argtypes = [_P, _I64, ctypes.c_double, ctypes.POINTER(hrg_result)]
        L.hrg_server_release.argtypes = [_P, _I64]
        L.hrg_server_stats.argtypes = [_P, ctypes.POINTER(hrg_server_counters)]
        L.hrg_server_last_error.argtypes = [_P]
        L.hrg_server_last_error.restype = ctypes.c_char_p
        L.hrg_server_destroy.argtypes = [_P]
        L.hrg_graph_props.argtypes = [_P, _I64, _P, _P, _I64, ctypes.c_uint32, _P, ctypes.POINTER(hrg_props)]
        L.hrg_degree_histogram.argtypes = [_P, _I64, _P, _I64, _P, _P]
        L.hrg_bfs.argtypes = [_P, _I64, _P, _P, _I64, _P, _P, ctypes.POINTER(ctypes.c_int32), _PI64, _PI64, _PI64]
        L.hrg_diameter_bounds.argtypes = [_P, _I64, _P, _P, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32), _PI64, _PI64]
        L.hrg_set_limits.argtypes = [_P, ctypes.POINTER(hrg_limits)]
        L.hrg_workspace_bytes.argtypes = [_P, _PI64]
        L.hrg_release_workspace.argtypes = [_P]
        L.hrg_update_begin.argtypes = [_P, _I64, ctypes.c_double, _P, _P, _P, _P, _I64, _P, _P, _P, ctypes.c_uint32,
                                       ctypes.c_int32, _P, _P, ctypes.POINTER(_P), _PI64]
        L.hrg_add_random_edges.argtypes = [_P, _I64, _P, _P, _I64, ctypes.c_uint64, _P, _P, _P, _I64, _PI64, _PI64]
        for name in EXPORTS:
            getattr(L, name).restype = getattr(L, name).restype or ctypes.c_int
        _lib = L
        return L


class hrg_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch_size", ctypes.c_int32), ("n", ctypes.c_int64),
                ("n_entries", ctypes.c_int64), ("r", ctypes.c_void_p), ("phi", ctypes.c_void_p),
                ("row_off", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("submit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class hrg_server_counters(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("completed", "batches", "batched_requests", "queued", "max_running",
                                               "in_use_bytes", "peak_in_use_bytes", "budget_bytes",
                                               "resident_bytes")]


def hrg_solve_radius(n: int, alpha: float, avg_degree: float) -> float:
    out = ctypes.c_double()
    rc = load().hrg_solve_radius(int(n), float(alpha), float(avg_degree), ctypes.byref(out))
    if rc != HRG_OK:
        raise HrgError(rc, "no radius for n=%r alpha=%r avg_degree=%r" % (n, alpha, avg_degree))
    return out.value


def hrg_expected_degree(n: int, alpha: float, R: float) -> float:
    return float(load().hrg_expected_degree(int(n), float(alpha), float(R)))


def hrg_version() -> str:
    return load().hrg_version().decode()


class Context:
    """An hrg_ctx on one device (hrg_create / hrg_destroy)."""

    def __init__(self, device: int = 0):
        L = load()
        h = _P()
        rc = L.hrg_create(ctypes.byref(h), int(device))
        if rc != HRG_OK:
            raise HrgError(rc, "hrg_create(device=%d) failed" % device)
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            load().hrg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return load().hrg_last_error(self.h).decode()

    def check(self, rc):
        if rc != HRG_OK:
            raise HrgError(rc, self.last_error())

    def workspace_bytes(self) -> int:
        """hrg_workspace_bytes: device bytes of the context's workspace."""
        v = ctypes.c_int64()
        self.check(load().hrg_workspace_bytes(self.h, ctypes.byref(v)))
        return v.value

    def release_workspace(self):
        """hrg_release_workspace: free the context's workspace."""
        self.check(load().hrg_release_workspace(self.h))

    def set_limits(self, row_buffer_ids=0, hub_pool_ids=0, hub_runs=0, heavy_segments=0, workspace_bytes=0):
        """hrg_set_limits: capacities of the count pass's buffers for later
        jobs (0: automatic) and a cap on the context's workspace (0: none)."""
        lim = hrg_limits(int(row_buffer_ids), int(hub_pool_ids), int(hub_runs), int(heavy_segments),
                         int(workspace_bytes))
        self.check(load().hrg_set_limits(self.h, ctypes.byref(lim)))


def params(n, alpha, avg_degree, seed, R_override=0.0, fp64_only=False, bands=0, hub_candidates=0) -> hrg_params:
    return hrg_params(int(n), float(alpha), float(avg_degree), int(seed), float(R_override),
                      HRG_FLAG_FP64_ONLY if fp64_only else 0, int(bands), int(hub_candidates), 0)


def _dptr(t) -> int:
    return t.data_ptr()


def generate(ctx: Context, n, alpha, avg_degree, seed, R_override=0.0, fp64_only=False, bands=0, stream=None,
             hub_candidates=0):
    """Device generation through hrg_generate_begin / hrg_generate_finish.
    Returns dict of torch tensors (r, phi, row_off, col_idx) and stats."""
    import torch

    L = load()
    dev = torch.device("cuda", ctx.device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    r = torch.empty(n, dtype=torch.float64, device=dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    p = params(n, alpha, avg_degree, seed, R_override, fp64_only, bands, hub_candidates)
    job = _P()
    ne = ctypes.c_int64()
    ctx.check(L.hrg_generate_begin(ctx.h, ctypes.byref(p), _P(st.cuda_stream), _P(_dptr(r)), _P(_dptr(phi)),
                                   _P(_dptr(off)), ctypes.byref(job), ctypes.byref(ne)))
    try:
        col = torch.empty(max(ne.value, 1), dtype=torch.int32, device=dev)
        ctx.check(L.hrg_generate_finish(job, _P(_dptr(col))))
        s = hrg_stats()
        L.hrg_job_stats(job, ctypes.byref(s))
    finally:
        L.hrg_job_release(job)
    return {"r": r, "phi": phi, "row_off": off, "col_idx": col[: ne.value], "stats": s.as_dict()}


def graph_props(ctx: Context, row_off, col_idx=None, d_min=1, triangles=True, stream=None) -> dict:
    """hrg_graph_props on a device CSR (torch tensors: row_off int64[n+1],
    col_idx int32): degree tail exponent, triads, triangles, clustering."""
    import torch

    L = load()
    dev = torch.device("cuda", ctx.device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    n = row_off.numel() - 1
    out = hrg_props()
    col = _P(_dptr(col_idx)) if col_idx is not None and col_idx.numel() > 0 else _P(None)
    ctx.check(L.hrg_graph_props(ctx.h, n, _P(_dptr(row_off)), col, int(d_min),
                                HRG_PROPS_TRIANGLES if triangles else 0, _P(st.cuda_stream), ctypes.byref(out)))
    return out.as_dict()


def degree_histogram(ctx: Context, row_off, max_degree: int, stream=None):
    """hrg_degree_histogram: int64 tensor hist[max_degree + 1] on the device."""
    import torch

    L = load()
    dev = torch.device("cuda", ctx.device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    hist = torch.empty(max_degree + 1, dtype=torch.int64, device=dev)
    ctx.check(L.hrg_degree_histogram(ctx.h, row_off.numel() - 1, _P(_dptr(row_off)), int(max_degree),
                                     _P(_dptr(hist)), _P(st.cuda_stream)))
    return hist


def add_random_edges(ctx: Context, row_off, col_idx, count: int, seed: int, stream=None) -> dict:
    """hrg_add_random_edges: the CSR with ``count`` random vertex pairs added
    as edges (Sec. 4.2's long-range edges).  Returns row_off, col_idx (torch
    tensors) and the number of added edges."""
    import torch

    L = load()
    dev = torch.device("cuda", ctx.device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    n = row_off.numel() - 1
    old = int(row_off[-1].item() - row_off[0].item())
    cap = old + 2 * int(count)
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    ne = ctypes.c_int64()
    added = ctypes.c_int64()
    src = _P(_dptr(col_idx)) if col_idx is not None and col_idx.numel() > 0 else _P(None)
    ctx.check(L.hrg_add_random_edges(ctx.h, n, _P(_dptr(row_off)), src, int(count), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                     _P(st.cuda_stream), _P(_dptr(off)), _P(_dptr(col)), cap, ctypes.byref(ne),
                                     ctypes.byref(added)))
    return {"row_off": off, "col_idx": col[: ne.value], "added": added.value}


def bfs(ctx: Context, row_off, col_idx, source: int, stream=None):
    """hrg_bfs: (dist int32 tensor, eccentricity, component size, farthest
    vertex, source used); source -1 starts at the highest-degree vertex."""
    import torch

    L = load()
    dev = torch.device("cuda", ctx.device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    n = row_off.numel() - 1
    dist = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ecc = ctypes.c_int32()
    reached, far, src = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    col = _P(_dptr(col_idx)) if col_idx is not None and col_idx.numel() > 0 else _P(None)
    ctx.check(L.hrg_bfs(ctx.h, n, _P(_dptr(row_off)), col, int(source), _P(st.cuda_stream), _P(_dptr(dist)),
                        ctypes.byref(ecc), ctypes.byref(reached), ctypes.byref(far), ctypes.byref(src)))
    return dist[:n], ecc.value, reached.value, far.value, src.value


def diameter_bounds(ctx: Context, row_off, col_idx, sweeps: int = 4, stream=None):
    """hrg_diameter_bounds: (lower, upper, roots, component size)."""
    import torch

    L = load()
    dev = torch.device("cuda", ctx.device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    n = row_off.numel() - 1
    lo, hi = ctypes.c_int32(), ctypes.c_int32()
    size = ctypes.c_int64()
    roots = (ctypes.c_int64 * sweeps)()
    col = _P(_dptr(col_idx)) if col_idx is not None and col_idx.numel() > 0 else _P(None)
    ctx.check(L.hrg_diameter_bounds(ctx.h, n, _P(_dptr(row_off)), col, int(sweeps), _P(st.cuda_stream),
                                    ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(size), roots))
    return lo.value, hi.value, [r for r in roots if r >= 0], size.value


class BatchItems:
    """The hrg_params array of a batch, built once: items is a sequence of
    (n, alpha, avg_degree, seed) or dicts with those keys (plus optional
    R_override, bands, hub_candidates)."""

    def __init__(self, items):
        self.arr = (hrg_params * len(items))()
        self.goff = [0]
        for k, it in enumerate(items):
            if isinstance(it, dict):
                self.arr[k] = params(it["n"], it["alpha"], it["avg_degree"], it["seed"], it.get("R_override", 0.0),
                                     False, it.get("bands", 0), it.get("hub_candidates", 0))
            else:
                self.arr[k] = params(*it)
            self.goff.append(self.goff[-1] + int(self.arr[k].n))

    def __len__(self):
        return len(self.arr)


def generate_batch(ctx: Context, items, fp64_only=False, stream=None):
    """hrg_generate_batch_begin + hrg_generate_finish on items (a sequence as
    in BatchItems, or a BatchItems).  Returns the concatenated outputs (r,
    phi, row_off global, col_idx with local ids), the graph offsets
    goff[count+1] (host list) and stats."""
    import torch

    L = load()
    dev = torch.device("cuda", ctx.device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    prepared = items if isinstance(items, BatchItems) else BatchItems(items)
    arr, goff = prepared.arr, prepared.goff
    N = goff[-1]
    r = torch.empty(N, dtype=torch.float64, device=dev)
    phi = torch.empty(N, dtype=torch.float64, device=dev)
    off = torch.empty(N + 1, dtype=torch.int64, device=dev)
    job = _P()
    ne = ctypes.c_int64()
    ctx.check(L.hrg_generate_batch_begin(ctx.h, len(arr), arr, HRG_FLAG_FP64_ONLY if fp64_only else 0,
                                         _P(st.cuda_stream), _P(_dptr(r)), _P(_dptr(phi)), _P(_dptr(off)),
                                         ctypes.byref(job), ctypes.byref(ne)))
    try:
        col = torch.empty(max(ne.value, 1), dtype=torch.int32, device=dev)
        ctx.check(L.hrg_generate_finish(job, _P(_dptr(col))))
        s = hrg_stats()
        L.hrg_job_stats(job, ctypes.byref(s))
    finally:
        L.hrg_job_release(job)
    return {"r": r, "phi": phi, "row_off": off, "col_idx": col[: ne.value], "goff": goff, "stats": s.as_dict()}


def generate_from_points(ctx: Context, r, phi, R, fp64_only=False, bands=0, stream=None):
    """hrg_generate_from_points_begin + finish on caller device tensors r, phi."""
    import torch

    L = load()
    r = r.contiguous()
    phi = phi.contiguous()
    n = r.numel()
    dev = r.device
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    job = _P()
    ne = ctypes.c_int64()
    ctx.check(L.hrg_generate_from_points_begin(ctx.h, n, float(R), _P(_dptr(r)), _P(_dptr(phi)),
                                               HRG_FLAG_FP64_ONLY if fp64_only else 0, int(bands),
                                               _P(st.cuda_stream), _P(_dptr(off)), ctypes.byref(job),
                                               ctypes.byref(ne)))
    try:
        col = torch.empty(max(ne.value, 1), dtype=torch.int32, device=dev)
        ctx.check(L.hrg_generate_finish(job, _P(_dptr(col))))
        s = hrg_stats()
        L.hrg_job_stats(job, ctypes.byref(s))
    finally:
        L.hrg_job_release(job)
    return {"row_off": off, "col_idx": col[: ne.value], "stats": s.as_dict()}


def update_points(ctx: Context, r, phi, row_off, col_idx, R, ids, r_new, phi_new, fp64_only=False, bands=0,
                  stream=None):
    """hrg_update_begin + hrg_generate_finish: k = len(ids) vertices move to
    (r_new, phi_new).  r, phi (device float64[n]) are updated in place;
    row_off, col_idx are the current CSR.  Returns the new row_off, col_idx
    (torch tensors) and stats."""
    import torch

    L = load()
    n = r.numel()
    dev = r.device
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    ids = ids.to(device=dev, dtype=torch.int32).contiguous()
    r_new = r_new.to(device=dev, dtype=torch.float64).contiguous()
    phi_new = phi_new.to(device=dev, dtype=torch.float64).contiguous()
    k = ids.numel()
    if r_new.numel() != k or phi_new.numel() != k:
        raise ValueError("ids, r_new and phi_new must have the same length")
    if not (r.is_contiguous() and phi.is_contiguous() and r.dtype == torch.float64 and phi.dtype == torch.float64):
        raise ValueError("r and phi must be contiguous float64 device tensors")
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    job = _P()
    ne = ctypes.c_int64()
    col_in = _P(_dptr(col_idx)) if col_idx.numel() > 0 else _P(None)
    ctx.check(L.hrg_update_begin(ctx.h, n, float(R), _P(_dptr(r)), _P(_dptr(phi)), _P(_dptr(row_off)), col_in, k,
                                 _P(_dptr(ids)) if k else _P(None), _P(_dptr(r_new)) if k else _P(None),
                                 _P(_dptr(phi_new)) if k else _P(None), HRG_FLAG_FP64_ONLY if fp64_only else 0,
                                 int(bands), _P(st.cuda_stream), _P(_dptr(off)), ctypes.byref(job), ctypes.byref(ne)))
    try:
        col = torch.empty(max(ne.value, 1), dtype=torch.int32, device=dev)
        ctx.check(L.hrg_generate_finish(job, _P(_dptr(col))))
        s = hrg_stats()
        L.hrg_job_stats(job, ctypes.byref(s))
    finally:
        L.hrg_job_release(job)
    return {"row_off": off, "col_idx": col[: ne.value], "stats": s.as_dict()}


def generate_host(ctx: Context, n, alpha, avg_degree, seed, r_host, phi_host, off_host, col_host, fp64_only=False,
                  bands=0):
    """hrg_generate_host into caller host tensors (pinned for full speed).
    Returns (n_entries, stats)."""
    L = load()
    p = params(n, alpha, avg_degree, seed, 0.0, fp64_only, bands)
    ne = ctypes.c_int64()
    s = hrg_stats()
    rc = L.hrg_generate_host(ctx.h, ctypes.byref(p), _P(r_host.data_ptr()), _P(phi_host.data_ptr()),
                             _P(off_host.data_ptr()), _P(col_host.data_ptr()), int(col_host.numel()),
                             ctypes.byref(ne), ctypes.byref(s))
    ctx.check(rc)
    return ne.value, s.as_dict()


def hrg_row_offsets_noalloc(deg, row_off, stream=None) -> int:
    """Row offsets from int32 degrees (device tensors) using the library's
    static scratch; returns the status code.  deg: contiguous int32[n];
    row_off: contiguous int64 with at least n + 1 elements, on deg's device
    (ValueError otherwise).  The call runs with that device current."""
    import torch

    if not (deg.is_cuda and row_off.is_cuda and deg.device == row_off.device):
        raise ValueError("deg and row_off must be CUDA tensors on one device")
    if deg.dtype != torch.int32 or row_off.dtype != torch.int64:
        raise ValueError("deg must be int32 and row_off int64")
    if not (deg.is_contiguous() and row_off.is_contiguous()):
        raise ValueError("deg and row_off must be contiguous")
    if row_off.numel() < deg.numel() + 1:
        raise ValueError("row_off needs n + 1 = %d elements, has %d" % (deg.numel() + 1, row_off.numel()))
    with torch.cuda.device(deg.device):
        st = stream if stream is not None else torch.cuda.current_stream(deg.device)
        return int(load().hrg_row_offsets_noalloc(_P(deg.data_ptr()), int(deg.numel()), _P(row_off.data_ptr()),
                                                  _P(st.cuda_stream)))


class Server:
    """hrg_server: queued generation requests with continuous batching."""

    def __init__(self, device: int = 0, slots: int = 2, mem_budget_bytes: int = 0):
        L = load()
        h = _P()
        rc = L.hrg_server_create(ctypes.byref(h), int(device), int(slots), int(mem_budget_bytes))
        if rc != HRG_OK:
            raise HrgError(rc, "hrg_server_create failed")
        self.h = h
        self.device = device

    def submit(self, n, alpha, avg_degree, seed, bands=0, hub_candidates=0) -> int:
        p = params(n, alpha, avg_degree, seed, 0.0, False, bands, hub_candidates)
        t = ctypes.c_int64()
        rc = load().hrg_server_submit(self.h, ctypes.byref(p), ctypes.byref(t))
        if rc != HRG_OK:
            raise HrgError(rc, self.last_error())
        return t.value

    def wait(self, ticket: int, timeout_s: float = -1.0) -> hrg_result:
        """Blocks (GIL released) until the request is done; returns the
        hrg_result (status may be non-zero) or raises on HRG_ETIMEOUT."""
        res = hrg_result()
        rc = load().hrg_server_wait(self.h, int(ticket), float(timeout_s), ctypes.byref(res))
        if rc == HRG_ETIMEOUT:
            raise TimeoutError("request %d not done" % ticket)
        if rc == HRG_EINVAL and res.n == 0:
            raise HrgError(rc, "unknown ticket %d" % ticket)
        return res

    def fetch(self, res: hrg_result):
        """Host copies (numpy) of a finished request: r, phi, row_off
        (rebased to 0), col_idx."""
        import numpy as np
        import torch

        n, ne = int(res.n), int(res.n_entries)
        dev = torch.device("cuda", self.device)
        torch.cuda.synchronize(dev)
        r = np.empty(n, dtype=np.float64)
        phi = np.empty(n, dtype=np.float64)
        off = np.empty(n + 1, dtype=np.int64)
        _memcpy_d2h(r, res.r)
        _memcpy_d2h(phi, res.phi)
        _memcpy_d2h(off, res.row_off)
        col = np.empty(ne, dtype=np.int32)
        if ne:
            _memcpy_d2h(col, res.col_idx + 4 * int(off[0]))
        return r, phi, off - off[0], col

    def release(self, ticket: int):
        rc = load().hrg_server_release(self.h, int(ticket))
        if rc != HRG_OK:
            raise HrgError(rc, "release of %d failed" % ticket)

    def counters(self) -> dict:
        c = hrg_server_counters()
        load().hrg_server_stats(self.h, ctypes.byref(c))
        return {k: getattr(c, k) for k, _ in c._fields_}

    def last_error(self) -> str:
        return load().hrg_server_last_error(self.h).decode()

    def close(self):
        if self.h:
            load().hrg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _memcpy_d2h(arr, dptr):
    """Device-to-host copy into a numpy array through the CUDA runtime."""
    rt = _cudart()
    rc = rt.cudaMemcpy(ctypes.c_void_p(arr.ctypes.data), ctypes.c_void_p(dptr), ctypes.c_size_t(arr.nbytes), 2)
    if rc != 0:
        raise HrgError(HRG_ECUDA, "cudaMemcpy failed (%d)" % rc)


_rt = None


def _cudart():
    global _rt
    if _rt is None:
        import torch  # noqa: F401  (loads the CUDA runtime the library links)

        for name in ("libcudart.so.13", "libcudart.so.12", "libcudart.so"):
            try:
                _rt = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if _rt is None:
            raise HrgError(HRG_ECUDA, "CUDA runtime library not found")
    return _rt
