"""Seeded synthetic Matryoshka-like embeddings (shared input generator).

This module only draws random numbers; it holds none of the search method's
arithmetic (no normalisation, no distances, no clustering).  Both the FP64
oracle and the GPU library read the arrays it returns.

Generative model (stands in for the paper's ImageNet-1K / NQ embeddings,
Sec. 3 "Datasets"; those corpora and the trained MRL encoders are not
available, so only their shapes are reproduced):

* K mixture components with uniform weights;
* per-dimension scale sigma_j = (j + 1) ** -0.5, so early coordinates carry
  most of the energy, like a nested (Matryoshka) representation (Sec. 3 "MR");
* component means mu_c[j] ~ N(0, sigma_j^2);
* points x = mu_c + alpha * sigma_j * eps, eps ~ N(0, 1), alpha = 0.5.

Database and queries share the component means (drawn from `mix_seed`) and
draw their points from independent streams.  Rows are generated in chunks,
each chunk from its own PCG64 stream keyed by (seed, chunk index), so the
result does not depend on how many threads generate it.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

CHUNK_ROWS = 1 << 14
ALPHA = 0.5


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


def dim_scale(d: int) -> np.ndarray:
    return (np.arange(d, dtype=np.float64) + 1.0) ** -0.5


def mixture_means(K: int, d: int, mix_seed: int) -> np.ndarray:
    """Component means, float32 [K, d]."""
    g = _rng(mix_seed, 0)
    return (g.standard_normal((K, d)) * dim_scale(d)).astype(np.float32)


def sample_points(n: int, d: int, means: np.ndarray, seed: int, alpha: float = ALPHA,
                  threads: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Draw n points of the mixture.  Returns (x float32 [n, d], label int32 [n])."""
    K = means.shape[0]
    x = np.empty((n, d), dtype=np.float32)
    lab = np.empty(n, dtype=np.int32)
    spread = (alpha * dim_scale(d)).astype(np.float32)
    nchunks = (n + CHUNK_ROWS - 1) // CHUNK_ROWS

    def work(c: int) -> None:
        lo, hi = c * CHUNK_ROWS, min(n, (c + 1) * CHUNK_ROWS)
        g = _rng(seed, c + 1)
        lc = g.integers(0, K, size=hi - lo, dtype=np.int64)
        eps = g.standard_normal((hi - lo, d), dtype=np.float32)
        np.multiply(eps, spread, out=eps)
        np.add(eps, means[lc], out=x[lo:hi])
        lab[lo:hi] = lc

    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    if nchunks <= 1 or threads <= 1:
        for c in range(nchunks):
            work(c)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(work, range(nchunks)))
    return x, lab


@dataclass(frozen=True)
class Workload:
    """Shape of one synthetic workload (database, queries, mixture)."""
    name: str
    N: int
    B: int
    d: int
    K: int
    db_seed: int
    q_seed: int
    mix_seed: int


# The paper's workloads, by shape.  Tiny: 10k x 64; ImageNet-1K-shaped:
# 1,281,167 x 2048 with 50,000 queries (Sec. 3, App. "Evaluation Metrics");
# NQ-shaped: 21,015,324 x 768 with 8,000 queries.
WORKLOADS = {
    "tiny": Workload("tiny", 10_000, 200, 64, 64, 1000, 2000, 3000),
    "imagenet": Workload("imagenet", 1_281_167, 50_000, 2048, 1000, 1001, 2001, 3001),
    "nq": Workload("nq", 21_015_324, 8_000, 768, 4096, 1003, 2003, 3003),
}


def make(workload: str | Workload, n: int | None = None, b: int | None = None,
         threads: int | None = None):
    """Database and queries of a workload (optionally truncated to n / b rows).

    Returns dict(db, db_label, queries, q_label, means).  Truncation keeps the
    leading rows of the full draw, so a prefix of the large workload is the
    same data at any n.
    """
    w = WORKLOADS[workload] if isinstance(workload, str) else workload
    n = w.N if n is None else n
    b = w.B if b is None else b
    means = mixture_means(w.K, w.d, w.mix_seed)
    db, dl = sample_points(n, w.d, means, w.db_seed, threads=threads)
    q, ql = sample_points(b, w.d, means, w.q_seed, threads=threads)
    return {"db": db, "db_label": dl, "queries": q, "q_label": ql, "means": means}


def small(n: int, b: int, d: int, K: int, seed: int):
    """A small ad-hoc workload for tests (same generative model)."""
    means = mixture_means(K, d, seed + 7)
    db, dl = sample_points(n, d, means, seed + 11, threads=1)
    q, ql = sample_points(b, d, means, seed + 13, threads=1)
    return {"db": db, "db_label": dl, "queries": q, "q_label": ql, "means": means}
