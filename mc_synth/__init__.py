"""Seeded synthetic inputs for matrix completion (observed entries P_Phi(M)).

This module is shared by the tests, the benchmark, the CPU oracle's callers and
the GPU path's callers.  It only draws inputs: it holds none of the completion
method's arithmetic (no SVD, no thresholding, no products with the iterate).

Every generator is driven by ``numpy.random.Generator(numpy.random.Philox(seed))``
so a (recipe, sizes, seed) triple always yields the same matrix on any machine.

Workload recipes (the paper's own data -- a 2048x2048 landscape photo and the
MovieLens 10M/20M rating sets of Sec. V.B-V.C -- are not available, so these
stand in for them with the same shapes and structure):

* ``lowrank_uniform``   M = U V^T with Gaussian factors, observed set drawn
                        uniformly without replacement (the synthetic test of
                        Sec. II.C / Alg. 2 style problems).
* ``smooth_image``      an image-like matrix: rank-r product of factors that are
                        Gaussian-smoothed along their rows (sigma px), min-max
                        scaled to [0, 255]; pixels observed uniformly (Sec. V.B
                        stand-in).
* ``ratings``           rating-like matrix: Zipf(1.1) row and column popularity,
                        half-star values from a rank-20 Gaussian model plus noise,
                        clipped to [0.5, 5]; optional held-out fraction (Sec. V.C
                        stand-in, MovieLens-20M shape 138,000 x 27,000).
* ``serving_jobs``      a Poisson stream of mixed-size low-rank completion jobs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Observed",
    "rng_for",
    "lowrank_uniform",
    "smooth_image",
    "ratings",
    "zipf_pairs",
    "serving_jobs",
    "to_csr",
]


@dataclasses.dataclass
class Observed:
    """Observed entries of an m x n matrix in CSR order (rows ascending, columns
    ascending within a row, no duplicates).

    ``row_ptr`` int64[m+1], ``col`` int32[nnz], ``val`` float32[nnz].
    ``test_*`` hold held-out entries (same layout, may be empty) and ``truth``
    optionally a callable/array to evaluate M at arbitrary (i, j).
    """

    m: int
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    test_rows: np.ndarray | None = None
    test_cols: np.ndarray | None = None
    test_val: np.ndarray | None = None
    dense: np.ndarray | None = None  # full M when small enough to keep
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col.size)

    @property
    def rows(self) -> np.ndarray:
        """Row index of every stored entry (expanded from row_ptr)."""
        return np.repeat(np.arange(self.m, dtype=np.int64), np.diff(self.row_ptr))


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def to_csr(m: int, n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray):
    """Sort (row, col) pairs into CSR arrays; pairs must be unique."""
    key = rows.astype(np.int64) * n + cols.astype(np.int64)
    order = np.argsort(key, kind="stable")
    key = key[order]
    if key.size > 1 and np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate (row, col) pairs")
    r = (key // n).astype(np.int64)
    c = (key % n).astype(np.int32)
    v = np.asarray(vals, dtype=np.float32)[order]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=m), out=row_ptr[1:])
    return row_ptr, c, v


def _sample_without_replacement(total: int, count: int, rng: np.random.Generator) -> np.ndarray:
    if count > total:
        raise ValueError("cannot observe more entries than the matrix has")
    return np.sort(rng.choice(total, size=count, replace=False))


def lowrank_uniform(m: int = 500, n: int = 500, rank: int = 10, nobs: int | None = None,
                    frac: float = 0.2, seed: int = 0) -> Observed:
    """M = U V^T, U (m x rank), V (n x rank) i.i.d. N(0,1); exactly ``nobs``
    positions (default round(frac*m*n)) drawn uniformly without replacement."""
    rng = rng_for(seed)
    U = rng.standard_normal((m, rank))
    V = rng.standard_normal((n, rank))
    M = U @ V.T
    if nobs is None:
        nobs = int(round(frac * m * n))
    flat = _sample_without_replacement(m * n, nobs, rng)
    rows, cols = flat // n, flat % n
    row_ptr, col, val = to_csr(m, n, rows, cols, M[rows, cols])
    return Observed(m, n, row_ptr, col, val, dense=M.astype(np.float32),
                    meta=dict(recipe="lowrank_uniform", rank=rank, seed=seed, nobs=nobs))


def smooth_image(m: int = 1024, n: int = 1024, rank: int = 40, sigma_px: float = 8.0,
                 frac: float = 0.5, seed: int = 0) -> Observed:
    """Image-like matrix: factors N(0,1) smoothed along their row index with a
    Gaussian of ``sigma_px`` pixels (reflect boundary, truncated at 4 sigma),
    M = U V^T min-max scaled to [0, 255]; ``frac`` of the pixels observed."""
    from scipy.ndimage import gaussian_filter1d

    rng = rng_for(seed)
    U = gaussian_filter1d(rng.standard_normal((m, rank)), sigma_px, axis=0, mode="reflect", truncate=4.0)
    V = gaussian_filter1d(rng.standard_normal((n, rank)), sigma_px, axis=0, mode="reflect", truncate=4.0)
    M = U @ V.T
    M = (M - M.min()) * (255.0 / (M.max() - M.min()))
    nobs = int(round(frac * m * n))
    flat = _sample_without_replacement(m * n, nobs, rng)
    rows, cols = flat // n, flat % n
    row_ptr, col, val = to_csr(m, n, rows, cols, M[rows, cols])
    return Observed(m, n, row_ptr, col, val, dense=M.astype(np.float32),
                    meta=dict(recipe="smooth_image", rank=rank, sigma_px=sigma_px, seed=seed, nobs=nobs))


def _alias_table(w: np.ndarray):
    """Walker/Vose alias table for sampling index i with probability w_i/sum(w)."""
    n = w.size
    p = (w * (n / w.sum())).tolist()
    prob = np.ones(n)
    alias = np.arange(n, dtype=np.int64)
    small = [i for i in range(n) if p[i] < 1.0]
    large = [i for i in range(n) if p[i] >= 1.0]
    while small and large:
        s = small.pop()
        l = large.pop()
        prob[s] = p[s]
        alias[s] = l
        p[l] = p[l] + p[s] - 1.0
        (small if p[l] < 1.0 else large).append(l)
    return prob, alias


def _alias_draw(prob, alias, size, rng):
    u = rng.random(size) * prob.size
    idx = u.astype(np.int64)
    np.minimum(idx, prob.size - 1, out=idx)
    return np.where(u - idx < prob[idx], idx, alias[idx])


def zipf_pairs(m: int, n: int, N: int, s: float, rng: np.random.Generator, batch: int = 1 << 23) -> np.ndarray:
    """N distinct (row, col) keys row*n+col, sorted.

    Row and column popularities follow Zipf(s) over random permutations of the
    ids; pairs are drawn independently from the product distribution and the
    first N distinct pairs in draw order are kept (heavy rows/columns saturate,
    as they do in rating data)."""
    if N > m * n:
        raise ValueError("N exceeds m*n")
    pr_, al_r = _alias_table(np.arange(1, m + 1, dtype=np.float64) ** (-s))
    pc_, al_c = _alias_table(np.arange(1, n + 1, dtype=np.float64) ** (-s))
    perm_r = rng.permutation(m).astype(np.int64)
    perm_c = rng.permutation(n).astype(np.int64)
    seen = np.zeros((m * n + 7) // 8, dtype=np.uint8)
    out, have = [], 0
    batch = max(1024, min(batch, 4 * N + 1024))
    while have < N:
        key = perm_r[_alias_draw(pr_, al_r, batch, rng)] * n + perm_c[_alias_draw(pc_, al_c, batch, rng)]
        fresh = (seen[key >> 3] & (np.uint8(1) << (key & 7).astype(np.uint8))) == 0
        key = key[fresh]
        u, first = np.unique(key, return_index=True)
        b = u >> 3
        bit = (np.uint8(1) << (u & 7).astype(np.uint8)).astype(np.int64)
        if u.size:
            starts = np.flatnonzero(np.r_[True, b[1:] != b[:-1]])
            seen[b[starts]] |= np.add.reduceat(bit, starts).astype(np.uint8)
        take = u[np.argsort(first, kind="stable")][: N - have]
        out.append(take)
        have += take.size
    return np.sort(np.concatenate(out))


def ratings(m: int = 138_000, n: int = 27_000, N: int = 20_000_000, rank: int = 20,
            zipf_s: float = 1.1, noise_sd: float = 0.5, holdout: float = 0.0,
            seed: int = 0) -> Observed:
    """Rating-like matrix (MovieLens-20M shape by default).

    value = clip(round_to_half(3.5 + (U V^T)_ij / sqrt(rank) + eta), 0.5, 5),
    U, V ~ N(0,1) (rank columns), eta ~ N(0, noise_sd^2).  ``holdout`` of the N
    pairs (seeded) are kept apart as test entries; the rest are observed."""
    rng = rng_for(seed)
    keys = zipf_pairs(m, n, N, zipf_s, rng)
    U = rng.standard_normal((m, rank)).astype(np.float64)
    V = rng.standard_normal((n, rank)).astype(np.float64)
    vals = np.empty(N, dtype=np.float32)
    chunk = 1 << 21
    scale = 1.0 / math.sqrt(rank)
    for a in range(0, N, chunk):
        kk = keys[a:a + chunk]
        r, c = kk // n, kk % n
        x = 3.5 + np.einsum("ij,ij->i", U[r], V[c]) * scale + noise_sd * rng.standard_normal(kk.size)
        vals[a:a + chunk] = np.clip(np.round(x * 2.0) / 2.0, 0.5, 5.0)
    test = np.zeros(N, dtype=bool)
    if holdout > 0:
        test[rng.choice(N, size=int(round(holdout * N)), replace=False)] = True
    tr = ~test
    ktr = keys[tr]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(ktr // n, minlength=m), out=row_ptr[1:])
    obs = Observed(m, n, row_ptr, (ktr % n).astype(np.int32), vals[tr],
                   meta=dict(recipe="ratings", rank=rank, zipf_s=zipf_s, N=N, holdout=holdout, seed=seed))
    if holdout > 0:
        kte = keys[test]
        obs.test_rows = (kte // n).astype(np.int64)
        obs.test_cols = (kte % n).astype(np.int64)
        obs.test_val = vals[test]
    return obs


def serving_jobs(num_jobs: int = 2000, dim_lo: int = 256, dim_hi: int = 8192, frac_lo: float = 0.05,
                 frac_hi: float = 0.5, rank_lo: int = 5, rank_hi: int = 50, rate: float = 1.0,
                 seed: int = 0):
    """Arrival stream of completion jobs: m, n log-uniform in [dim_lo, dim_hi],
    observed fraction uniform in [frac_lo, frac_hi], true rank uniform in
    {rank_lo..rank_hi}, Poisson arrivals at ``rate`` jobs/s.  Returns a list of
    dicts with the job shape, its arrival time and its own seed; the matrix of
    job j is ``lowrank_uniform(m, n, rank, nobs, seed=job_seed)``."""
    rng = rng_for(seed)
    t = 0.0
    jobs = []
    for j in range(num_jobs):
        t += rng.exponential(1.0 / rate)
        m = int(round(math.exp(rng.uniform(math.log(dim_lo), math.log(dim_hi)))))
        n = int(round(math.exp(rng.uniform(math.log(dim_lo), math.log(dim_hi)))))
        frac = float(rng.uniform(frac_lo, frac_hi))
        rank = int(rng.integers(rank_lo, rank_hi + 1))
        jobs.append(dict(job=j, arrival=t, m=m, n=n, rank=rank, frac=frac,
                         nobs=int(round(frac * m * n)), seed=int(rng.integers(0, 2**31 - 1))))
    return jobs
