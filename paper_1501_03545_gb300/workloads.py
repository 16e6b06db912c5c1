"""Seeded synthetic workloads shared by the tests, the smoke check and the bench.

This module holds inputs only: parameter sets and numpy-seeded point sets.  It
contains none of the generator's arithmetic (no radius solve, no sampler, no
predicate), so both the CUDA path and the CPU oracle can take their inputs
from it without sharing any of the method's code.

The paper measures on graphs it generates itself (Sec. 4.4); there is no
public dataset.  The four parameter sets below are the workloads this library
is measured and checked on:

* ``SMALL``    n = 1e4,  alpha = 1.0  (gamma = 3),   kbar = 6,  seed 1
* ``MEDIUM``   n = 1e6,  alpha = 0.75 (gamma = 2.5), kbar = 10, seed 2
* ``LARGE``    n = 1e8,  alpha = 0.55 (gamma = 2.1), kbar = 16, seed 3
* ``EXAMPLE``  n = 500,  alpha = 0.8, R = 5.08 -- the illustrative graph of
  Sec. 2.1 (its R is printed, its kbar is not).

``moves`` draws the vertex movements that the dynamic update takes as input
(the paper defines no movement law).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    alpha: float
    kbar: float
    seed: int


SMALL = Workload("rhg_n1e4_a1.0_k6", 10_000, 1.0, 6.0, 1)
MEDIUM = Workload("rhg_n1e6_a0.75_k10", 1_000_000, 0.75, 10.0, 2)
LARGE = Workload("rhg_n1e8_a0.55_k16", 100_000_000, 0.55, 16.0, 3)

ALL = (SMALL, MEDIUM, LARGE)

# Sec. 2.1: "500 vertices, R ~ 5.08 and alpha = 0.8"
EXAMPLE_N = 500
EXAMPLE_ALPHA = 0.8
EXAMPLE_R = 5.08


def scaled(w: Workload, n: int, seed: int | None = None) -> Workload:
    """Same alpha and kbar at another size (for parity at oracle-friendly n)."""
    return Workload("%s@n%d" % (w.name, n), int(n), w.alpha, w.kbar, w.seed if seed is None else seed)


def random_points(n: int, R: float, seed: int, r_lo: float = 0.0):
    """Point sets for the injected-geometry entry point: r uniform on
    [r_lo, R), phi uniform on [0, 2pi).  Not the model's radial law -- these
    exercise the query path on arbitrary inputs."""
    g = np.random.default_rng(seed)
    r = g.uniform(r_lo, R, size=n)
    phi = g.uniform(0.0, 2.0 * np.pi, size=n)
    phi = np.where(phi >= 2.0 * np.pi, 0.0, phi)
    return r.astype(np.float64), phi.astype(np.float64)


def clustered_points(n: int, R: float, seed: int, clusters: int = 4, spread: float = 1e-6):
    """Many points packed into a few tiny angular clusters near the rim:
    stresses windows, ties in angle and wrap-around at phi = 0."""
    g = np.random.default_rng(seed)
    centres = g.uniform(0.0, 2.0 * np.pi, size=clusters)
    centres[0] = 0.0  # one cluster straddles the wrap point
    which = g.integers(0, clusters, size=n)
    phi = np.mod(centres[which] + g.normal(0.0, spread, size=n), 2.0 * np.pi)
    phi = np.where(phi >= 2.0 * np.pi, 0.0, phi)
    r = R - g.exponential(1.0, size=n)
    r = np.clip(r, 0.0, np.nextafter(R, 0.0))
    return r.astype(np.float64), phi.astype(np.float64)


# ---------------------------------------------------------------------------
# Many small graphs in one call, and a stream of requests of mixed size.
# ---------------------------------------------------------------------------
BATCH_COUNT = 4096
BATCH_DRAW_SEED = 42
BATCH_KBARS = (4.0, 8.0, 16.0, 32.0)


def batch_items(count: int = BATCH_COUNT, draw_seed: int = BATCH_DRAW_SEED, n_lo: float = 1e3, n_hi: float = 1e5,
                first_seed: int = 1000):
    """The batched workload: ``count`` independent graphs with n log-uniform
    in [n_lo, n_hi], alpha uniform in [0.55, 1.5], kbar drawn from
    {4, 8, 16, 32}, Philox seeds first_seed, first_seed + 1, ...  The
    per-graph parameters come from numpy's generator seeded with draw_seed.
    Returns a list of (n, alpha, kbar, seed)."""
    g = np.random.default_rng(draw_seed)
    n = np.exp(g.uniform(np.log(n_lo), np.log(n_hi), size=count)).astype(np.int64)
    alpha = g.uniform(0.55, 1.5, size=count)
    kbar = np.asarray(BATCH_KBARS)[g.integers(0, len(BATCH_KBARS), size=count)]
    return [(int(n[k]), float(alpha[k]), float(kbar[k]), first_seed + k) for k in range(count)]


SERVE_RATE = 200.0
SERVE_DRAW_SEED = 7


def serving_requests(count: int, rate: float = SERVE_RATE, draw_seed: int = SERVE_DRAW_SEED, n_lo: float = 1e3,
                     n_hi: float = 3e7, first_seed: int = 10000):
    """The serving workload: Poisson arrivals at ``rate`` requests/s, n
    log-uniform in [n_lo, n_hi], alpha uniform in [0.55, 1.5], kbar uniform
    in [4, 32], seed first_seed + request index.  Returns a list of
    (arrival_s, n, alpha, kbar, seed)."""
    g = np.random.default_rng(draw_seed)
    t = np.cumsum(g.exponential(1.0 / rate, size=count))
    n = np.exp(g.uniform(np.log(n_lo), np.log(n_hi), size=count)).astype(np.int64)
    alpha = g.uniform(0.55, 1.5, size=count)
    kbar = g.uniform(4.0, 32.0, size=count)
    return [(float(t[k]), int(n[k]), float(alpha[k]), float(kbar[k]), first_seed + k) for k in range(count)]


# ---------------------------------------------------------------------------
# Vertex movement: the paper leaves the law of motion open, so the moves of a
# dynamic update are synthetic inputs.
# ---------------------------------------------------------------------------
def moves(r, phi, R: float, k: int, seed: int, jumps: float = 0.15):
    """k distinct vertices and their new coordinates, from the current points
    (numpy arrays r, phi) and numpy's generator seeded with ``seed``: 10 % to
    just beside phi = 0 on either side (through the wrap point), a fraction
    ``jumps`` (default 15 %) to a radius uniform on [0, R) (across bands,
    some to the centre, where a vertex sees most of the graph), 15 % to the
    rim (R - Exp(1)), the rest small steps (r + N(0, 0.3), phi + N(0,
    1e-3)).  Returns (ids int32, r_new, phi_new) with 0 <= r_new < R and
    0 <= phi_new < 2 pi."""
    g = np.random.default_rng(seed)
    n = len(r)
    ids = np.sort(g.choice(n, size=k, replace=False)).astype(np.int32)
    kind = g.uniform(size=k)
    r0, p0 = np.asarray(r, dtype=np.float64)[ids], np.asarray(phi, dtype=np.float64)[ids]
    rn = r0 + g.normal(0.0, 0.3, size=k)
    pn = p0 + g.normal(0.0, 1e-3, size=k)
    wrap = (kind >= 0.60) & (kind < 0.70)
    pn = np.where(wrap, g.normal(0.0, 1e-4, size=k), pn)
    jump = (kind >= 0.70) & (kind < 0.70 + jumps)
    rn = np.where(jump, g.uniform(0.0, R, size=k), rn)
    rim = kind >= 0.85
    rn = np.where(rim, R - g.exponential(1.0, size=k), rn)
    rn = np.clip(rn, 0.0, np.nextafter(R, 0.0))
    pn = np.mod(pn, 2.0 * np.pi)
    pn = np.where(pn >= 2.0 * np.pi, 0.0, pn)
    return ids, rn.astype(np.float64), pn.astype(np.float64)
