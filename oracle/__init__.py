"""CPU oracle for the threshold random hyperbolic graph -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The generator library never loads it,
and it never loads the generator: the two share no code.  It wraps the plain C
restatement in ``hrg_oracle.c`` with ctypes and numpy.

Functions and the passage each follows (von Looz, Meyerhenke, Prutkin, Staudt,
"Fast generation of complex networks with underlying hyperbolic geometry"):

* ``philox``            -- Philox4x32-10 (Salmon et al., SC'11); the paper names no
                           generator, this is the chosen one.
* ``expected_degree``   -- Krioukov et al. Eq. (22) restated in Appendix B.1
                           (reading: middle term (pi-1)(zeta/alpha), zeta = 1).
* ``solve_radius``      -- Appendix B.1 binary search; Algorithm 1, first line.
* ``sample``            -- Algorithm 1, the two "draw" lines; Eq. (1).
* ``cosh_dist``         -- Sec. 2.1 edge rule, hyperbolic law of cosines.
* ``brute_csr``         -- the plain definition: all pairs, edge iff dist < R.
* ``band_csr`` / ``band_rows`` -- an independent band algorithm for large n.
* ``ties``              -- pairs within 1e-12 relative of the threshold.
* ``graph_props``       -- Sec. 4.1 properties of a CSR: the degree tail's
                           power-law exponent (discrete MLE approximation of
                           Clauset, Shalizi and Newman, Eq. 3.7), triads,
                           triangles, and the clustering coefficient as the
                           fraction of closed triads; the mean local
                           coefficient beside it.
* ``quadtree_csr``      -- the paper's own generator (Algorithm 1, the polar
                           quadtree of Sec. 3, Proposition 1, Eq. (3)) from
                           ``hrg_quadtree.c``: a second CPU baseline, checked
                           against brute force, not the parity reference.
* ``bfs`` / ``diameter_bounds`` -- hop distances from one vertex; the
                           diameter of a vertex's component bracketed by
                           repeated double sweeps (Sec. 4.1's longest
                           shortest path, which Sec. 4.2's long-range edges
                           shorten).
* ``random_pairs`` / ``add_random_edges`` -- Sec. 4.2's graph with random
                           long-range edges: uniform vertex pairs from a
                           Philox stream of their own, merged into the CSR.

Every function here is pinned by ``tests/test_oracle*.py`` to something other
than itself (an independent Philox, mpmath, scipy quadrature, the paper's
worked example, Lemma 4 cell masses, exhaustive checks).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hrg_oracle.c")
_SRC_QT = os.path.join(_HERE, "hrg_quadtree.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I64 = ctypes.c_int64
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_QT))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, _SRC_QT, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            L.orc_philox4x32_10.argtypes = [_P, _P, _P]
            L.orc_expected_degree.argtypes = [_D, _D, _D]
            L.orc_expected_degree.restype = _D
            L.orc_solve_radius.argtypes = [_I64, _D, _D, _P]
            L.orc_solve_radius.restype = ctypes.c_int
            L.orc_uniforms.argtypes = [ctypes.c_uint64, _I64, _P, _P]
            L.orc_sample.argtypes = [_I64, _D, _D, ctypes.c_uint64, _P, _P]
            for f in ("orc_cosh_dist", "orc_cosh_dist_textbook", "orc_cosh_dist_poincare"):
                getattr(L, f).argtypes = [_D, _D, _D, _D]
                getattr(L, f).restype = _D
            L.orc_in_circle_prop1.argtypes = [_D, _D, _D, _D, _D]
            L.orc_in_circle_prop1.restype = ctypes.c_int
            L.orc_brute_degrees.argtypes = [_I64, _P, _P, _D, _P]
            L.orc_brute_degrees.restype = _I64
            L.orc_brute_fill.argtypes = [_I64, _P, _P, _D, _P, _P]
            L.orc_brute_ties.argtypes = [_I64, _P, _P, _D, _D, _I64, _P]
            L.orc_brute_rows.argtypes = [_I64, _P, _P, _D, _I64, _P, _P, _P, _P]
            L.orc_brute_ties.restype = _I64
            L.orc_bands_build.argtypes = [_I64, _P, _P, _D]
            L.orc_bands_build.restype = _P
            L.orc_bands_free.argtypes = [_P]
            L.orc_bands_degrees.argtypes = [_P, _P, _P, _P]
            L.orc_bands_degrees.restype = _I64
            L.orc_bands_fill.argtypes = [_P, _P, _P, _P, _P]
            L.orc_bands_rows.argtypes = [_P, _P, _P, _I64, _P, _P, _P, _P]
            L.orc_bands_ties.argtypes = [_P, _P, _P, _D, _I64, _P]
            L.orc_bands_ties.restype = _I64
            L.orc_degree_stats.argtypes = [_I64, _P, _I64, _P, _P]
            L.orc_random_pairs.argtypes = [_I64, _I64, ctypes.c_uint64, _P, _P]
            L.orc_quadtree_build.argtypes = [_I64, _P, _P, _D, _D, ctypes.c_int32]
            L.orc_quadtree_build.restype = _P
            L.orc_quadtree_free.argtypes = [_P]
            L.orc_quadtree_degrees.argtypes = [_P, _P]
            L.orc_quadtree_degrees.restype = _I64
            L.orc_quadtree_fill.argtypes = [_P, _P, _P]
            L.orc_quadtree_circle.argtypes = [_D, _D, _D, _P]
            L.orc_bfs.argtypes = [_I64, _P, _P, _I64, _P]
            L.orc_bfs.restype = ctypes.c_int32
            L.orc_quadtree_depth_counts.argtypes = [_I64, _P, _P, _D, _D, ctypes.c_int32, ctypes.c_int32, _P]
            L.orc_quadtree_depth_counts.restype = ctypes.c_int32
            L.orc_triangles.argtypes = [_I64, _P, _P, _P]
            L.orc_triangles.restype = _I64
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def philox(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: ctr = 4 uint32 words, key = 2 uint32 words."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def uniforms(seed: int, vid: int):
    a = ctypes.c_double()
    b = ctypes.c_double()
    lib().orc_uniforms(ctypes.c_uint64(seed), vid, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def expected_degree(n, alpha, R) -> float:
    return float(lib().orc_expected_degree(float(n), float(alpha), float(R)))


def solve_radius(n: int, alpha: float, kbar: float) -> float:
    out = ctypes.c_double()
    rc = lib().orc_solve_radius(int(n), float(alpha), float(kbar), ctypes.byref(out))
    if rc != 0:
        raise ValueError("invalid parameters for Eq. (22): n=%r alpha=%r kbar=%r" % (n, alpha, kbar))
    return out.value


def sample(n: int, alpha: float, R: float, seed: int):
    r = np.empty(n, dtype=np.float64)
    phi = np.empty(n, dtype=np.float64)
    lib().orc_sample(int(n), float(alpha), float(R), ctypes.c_uint64(seed), _ptr(r), _ptr(phi))
    return r, phi


def cosh_dist(r1, phi1, r2, phi2) -> float:
    return float(lib().orc_cosh_dist(r1, phi1, r2, phi2))


def cosh_dist_textbook(r1, phi1, r2, phi2) -> float:
    return float(lib().orc_cosh_dist_textbook(r1, phi1, r2, phi2))


def cosh_dist_poincare(r1, phi1, r2, phi2) -> float:
    return float(lib().orc_cosh_dist_poincare(r1, phi1, r2, phi2))


def in_circle_prop1(R, rq, phiq, rc, phic) -> bool:
    return bool(lib().orc_in_circle_prop1(R, rq, phiq, rc, phic))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _offsets(deg: np.ndarray) -> np.ndarray:
    off = np.zeros(len(deg) + 1, dtype=np.int64)
    np.cumsum(deg, out=off[1:])
    return off


def brute_csr(r, phi, R):
    """All-pairs CSR (row_off int64[n+1], col_idx int32[2m]), rows ascending."""
    r = _f64(r)
    phi = _f64(phi)
    n = len(r)
    deg = np.zeros(n, dtype=np.int64)
    lib().orc_brute_degrees(n, _ptr(r), _ptr(phi), float(R), _ptr(deg))
    off = _offsets(deg)
    col = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
    lib().orc_brute_fill(n, _ptr(r), _ptr(phi), float(R), _ptr(off), _ptr(col))
    return off, col[: int(off[-1])]


def brute_rows(r, phi, R, qids):
    """Sorted neighbour lists of the vertices ``qids`` by scanning all points:
    (cnt, off, rows)."""
    r = _f64(r)
    phi = _f64(phi)
    q = np.ascontiguousarray(np.asarray(qids, dtype=np.int64))
    cnt = np.zeros(len(q), dtype=np.int64)
    lib().orc_brute_rows(len(r), _ptr(r), _ptr(phi), float(R), len(q), _ptr(q), _ptr(cnt), None, None)
    off = _offsets(cnt)
    rows = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
    lib().orc_brute_rows(len(r), _ptr(r), _ptr(phi), float(R), len(q), _ptr(q), _ptr(cnt), _ptr(off), _ptr(rows))
    return cnt, off, rows[: int(off[-1])]


class Bands:
    """The CPU band algorithm's structure over one point set."""

    def __init__(self, r, phi, R):
        self.r = _f64(r)
        self.phi = _f64(phi)
        self.R = float(R)
        self.n = len(self.r)
        self.h = lib().orc_bands_build(self.n, _ptr(self.r), _ptr(self.phi), self.R)

    def close(self):
        if self.h:
            lib().orc_bands_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def degrees(self):
        deg = np.zeros(self.n, dtype=np.int64)
        lib().orc_bands_degrees(self.h, _ptr(self.r), _ptr(self.phi), _ptr(deg))
        return deg

    def csr(self):
        deg = self.degrees()
        off = _offsets(deg)
        col = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
        lib().orc_bands_fill(self.h, _ptr(self.r), _ptr(self.phi), _ptr(off), _ptr(col))
        return off, col[: int(off[-1])]

    def rows(self, qids):
        """Sorted neighbour lists of the vertices ``qids``: (cnt, off, rows)."""
        q = np.ascontiguousarray(np.asarray(qids, dtype=np.int64))
        cnt = np.zeros(len(q), dtype=np.int64)
        lib().orc_bands_rows(self.h, _ptr(self.r), _ptr(self.phi), len(q), _ptr(q), _ptr(cnt), None, None)
        off = _offsets(cnt)
        rows = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
        lib().orc_bands_rows(self.h, _ptr(self.r), _ptr(self.phi), len(q), _ptr(q), _ptr(cnt), _ptr(off), _ptr(rows))
        return cnt, off, rows[: int(off[-1])]

    def ties(self, tol=1e-12, cap=1 << 16):
        pairs = np.zeros(2 * cap, dtype=np.int64)
        k = lib().orc_bands_ties(self.h, _ptr(self.r), _ptr(self.phi), float(tol), cap, _ptr(pairs))
        return int(k), pairs[: 2 * min(int(k), cap)].reshape(-1, 2)


def band_csr(r, phi, R):
    b = Bands(r, phi, R)
    try:
        return b.csr()
    finally:
        b.close()


def brute_ties(r, phi, R, tol=1e-12, cap=1 << 16):
    r = _f64(r)
    phi = _f64(phi)
    pairs = np.zeros(2 * cap, dtype=np.int64)
    k = lib().orc_brute_ties(len(r), _ptr(r), _ptr(phi), float(R), float(tol), cap, _ptr(pairs))
    return int(k), pairs[: 2 * min(int(k), cap)].reshape(-1, 2)


def generate(n: int, alpha: float, kbar: float, seed: int, method: str = "auto", R: float | None = None):
    """Whole oracle pipeline: R (Eq. (22) unless given), points, CSR."""
    if R is None:
        R = solve_radius(n, alpha, kbar)
    r, phi = sample(n, alpha, R, seed)
    if method == "auto":
        method = "brute" if n <= 20000 else "bands"
    off, col = brute_csr(r, phi, R) if method == "brute" else band_csr(r, phi, R)
    return {"R": R, "r": r, "phi": phi, "row_off": off, "col_idx": col}


def graph_props(row_off, col_idx, d_min: int, triangles: bool = True) -> dict:
    """Sec. 4.1 properties of a canonical CSR (rows ascending, both directions).

    gamma = 1 + tail_count / tail_log_sum over the vertices of degree >=
    d_min (NaN for an empty tail); clustering = 3 triangles / triads (NaN
    without triads); avg_local_clustering = the mean over all vertices of
    t_v / (d_v (d_v - 1) / 2), vertices of degree < 2 counting 0."""
    off = np.ascontiguousarray(np.asarray(row_off, dtype=np.int64))
    col = np.ascontiguousarray(np.asarray(col_idx, dtype=np.int32))
    n = len(off) - 1
    oi = np.zeros(4, dtype=np.int64)
    od = np.zeros(1, dtype=np.float64)
    lib().orc_degree_stats(n, _ptr(off), int(d_min), _ptr(oi), _ptr(od))
    res = {"n": n, "entries": int(oi[0]), "max_degree": int(oi[1]), "d_min": int(d_min),
           "tail_count": int(oi[2]), "tail_log_sum": float(od[0]), "triads": int(oi[3])}
    res["gamma"] = 1.0 + res["tail_count"] / res["tail_log_sum"] if res["tail_count"] > 0 else float("nan")
    res["triangles"] = -1
    res["clustering"] = float("nan")
    res["avg_local_clustering"] = float("nan")
    if triangles:
        t = np.zeros(max(n, 1), dtype=np.int64)
        colp = col if len(col) else np.zeros(1, dtype=np.int32)
        T = int(lib().orc_triangles(n, _ptr(off), _ptr(colp), _ptr(t)))
        t = t[:n]
        res["triangles"] = T
        res["triangles_per_vertex"] = t
        if res["triads"] > 0:
            res["clustering"] = 3.0 * T / res["triads"]
        d = np.diff(off)
        pairs = d * (d - 1) // 2
        local = np.where(pairs > 0, t / np.maximum(pairs, 1), 0.0)
        res["avg_local_clustering"] = float(local.sum() / n) if n > 0 else float("nan")
    return res


def random_pairs(n: int, count: int, seed: int):
    """The vertex pairs (u[count], v[count]) of the long-range edges."""
    u = np.zeros(max(count, 1), dtype=np.int64)
    v = np.zeros(max(count, 1), dtype=np.int64)
    lib().orc_random_pairs(int(n), int(count), int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(u), _ptr(v))
    return u[:count], v[:count]


def add_random_edges(row_off, col_idx, count: int, seed: int):
    """The CSR with the long-range edges of ``random_pairs`` added: the union
    of the graph's edges and the drawn pairs (self-pairs dropped; a pair
    drawn twice or already present is one edge).  Returns (row_off,
    col_idx, added) with ``added`` the new undirected edges."""
    off = np.asarray(row_off, dtype=np.int64)
    col = np.asarray(col_idx, dtype=np.int64)
    n = len(off) - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    u, v = random_pairs(n, count, seed)
    keep = u != v
    a = np.minimum(u[keep], v[keep])
    b = np.maximum(u[keep], v[keep])
    old = set(zip(rows[rows < col].tolist(), col[rows < col].tolist()))
    new = set(zip(a.tolist(), b.tolist())) - old
    if new:
        na = np.fromiter((p[0] for p in new), dtype=np.int64, count=len(new))
        nb = np.fromiter((p[1] for p in new), dtype=np.int64, count=len(new))
        src = np.concatenate([rows, na, nb])
        dst = np.concatenate([col, nb, na])
    else:
        src, dst = rows, col
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    out_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=out_off[1:])
    return out_off, dst.astype(np.int32), len(new)


def quadtree_csr(r, phi, R: float, alpha: float, capacity: int = 64):
    """CSR of the paper's quadtree generator on the given points: (row_off,
    col_idx, seconds) with seconds = (tree build, degree queries, row queries)."""
    import time

    r = _f64(r)
    phi = _f64(phi)
    n = len(r)
    L = lib()
    t0 = time.perf_counter()
    h = L.orc_quadtree_build(n, _ptr(r), _ptr(phi), float(R), float(alpha), int(capacity))
    try:
        t1 = time.perf_counter()
        deg = np.zeros(max(n, 1), dtype=np.int64)
        L.orc_quadtree_degrees(h, _ptr(deg))
        off = _offsets(deg[:n])
        t2 = time.perf_counter()
        col = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
        L.orc_quadtree_fill(h, _ptr(off), _ptr(col))
        t3 = time.perf_counter()
    finally:
        L.orc_quadtree_free(h)
    return off, col[: int(off[-1])], (t1 - t0, t2 - t1, t3 - t2)


def quadtree_depth_counts(r, phi, R: float, alpha: float, depth: int, capacity: int = 1):
    """Points per cell of the quadtree's complete level ``depth`` (Lemma 4)."""
    r = _f64(r)
    phi = _f64(phi)
    counts = np.zeros(4 ** depth, dtype=np.int64)
    lib().orc_quadtree_depth_counts(len(r), _ptr(r), _ptr(phi), float(R), float(alpha), int(capacity), int(depth),
                                    _ptr(counts))
    return counts


def quadtree_circle(R: float, phi: float, rh: float):
    """Proposition 1: (centre radius, circle radius) in the Poincare disk of
    the hyperbolic circle of radius R around (phi, rh)."""
    out = np.zeros(2, dtype=np.float64)
    lib().orc_quadtree_circle(float(R), float(phi), float(rh), _ptr(out))
    return float(out[0]), float(out[1])


def bfs(row_off, col_idx, source: int):
    """(dist int32[n] with -1 where unreached, eccentricity of source)."""
    off = np.ascontiguousarray(np.asarray(row_off, dtype=np.int64))
    col = np.ascontiguousarray(np.asarray(col_idx, dtype=np.int32))
    n = len(off) - 1
    dist = np.zeros(max(n, 1), dtype=np.int32)
    colp = col if len(col) else np.zeros(1, dtype=np.int32)
    ecc = int(lib().orc_bfs(n, _ptr(off), _ptr(colp), int(source), _ptr(dist)))
    return dist[:n], ecc


def diameter_bounds(row_off, col_idx, sweeps: int = 4, bfs_fn=None):
    """Bounds on the diameter of the component of the highest-degree vertex
    (lowest id among ties) by repeated double sweeps: BFS from a root gives
    ecc(root) <= diameter <= 2 ecc(root); the next root is the farthest
    vertex (lowest id among ties).  Returns (lower, upper, roots, component
    size).  bfs_fn(source) -> (dist, ecc) may replace the oracle's BFS, so
    that the device's search is driven by the same rule."""
    off = np.asarray(row_off, dtype=np.int64)
    if bfs_fn is None:
        bfs_fn = lambda s: bfs(row_off, col_idx, s)  # noqa: E731
    deg = np.diff(off)
    root = int(np.argmax(deg))
    lower, upper, roots, size = 0, None, [], 0
    for _ in range(sweeps):
        dist, ecc = bfs_fn(root)
        dist = np.asarray(dist)
        roots.append(root)
        size = int((dist >= 0).sum())
        lower = max(lower, ecc)
        upper = 2 * ecc if upper is None else min(upper, 2 * ecc)
        far = int(np.flatnonzero(dist == ecc)[0])
        if far == root:
            break
        root = far
    return lower, upper, roots, size
