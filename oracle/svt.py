"""Singular value thresholding for matrix completion (CPU oracle; test
infrastructure).

* ``svt_exact``  -- Alg. 2 (SVT of Cai, Candes & Shen as stated in Sec. II.C),
  with a dense LAPACK SVD in place of svds for small problems.
* ``svt_fast``   -- Alg. 6 (fast SVT, Sec. IV.C): rSVD-BKI, subspace recycling
  (Sec. IV.B strategies 1 and 2, plus an optional warm-started Omega) and the
  adaptive power parameter p.
* ``spectral_norm`` -- ||P_Phi(M)||_2 for the constant c of Sec. II.C.

Readings taken where the paper is silent, ambiguous or inconsistent:
  * tau defaults to 5*sqrt(m n) (Sec. II.C says 5n for the column count n; the
    two agree for square matrices); delta is a caller parameter, held constant.
  * ||P_Phi(M)||_2 is estimated by float64 power iteration on A^T A, started
    from column 0 of the Philox Omega of call 0, stopped at relative change
    < 1e-10 (at most 1000 steps).  c = ceil(tau / (delta ||P_Phi(M)||_2)).
  * Step 16 of Alg. 6 writes P_Omega(Y); Y is supported on Phi, so it is read
    as Y^i = Y^{i-1} + delta P_Phi(M - X^i).
  * The repeat test uses the last computed singular value, kept when > tau
    (strictly); r_i = #{j : sigma_j > tau}; comparisons in float64.
  * q counts SVD calls (it is advanced inside the repeat loop as printed).
  * A recycled SVD cannot deliver more values than its basis holds: when the
    recycled basis is narrower than k_i, or a recycled result fails the repeat
    test, the next attempt is a fresh rSVD-BKI.
  * p adaptation: after each iteration's error e_i, p += 1 if e_i > e_{i-1}
    (strict) and the decrease streak restarts; after 10 consecutive
    e_i < e_{i-1} p -= 1 and the streak restarts; an equal error ends the
    streak; p stays within [p_min, p_max] = [3, 20] by default.
  * Each rSVD-BKI call draws a fresh Omega from the Philox stream with call id
    1, 2, 3, ... (call 0 is the power-iteration start vector).
  * When the loop breaks on the tolerance, the result is X^i; Y is not
    advanced further.
  * recycle=3 (warm start): a fresh rSVD-BKI whose Omega has the previous
    right singular vectors V^{i-1}(:, 1:min(r_{i-1}, k+s)) in its leading
    columns and Philox columns after them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

from .philox import omega
from .rsvd import as_csr64, clamp_rank, recycle_q, recycle_u, rsvd_bki, rsvd_pi


def default_tau(m: int, n: int) -> float:
    return 5.0 * math.sqrt(float(m) * float(n))


def spectral_norm(A: sp.csr_matrix, seed: int = 0, rtol: float = 1e-10, max_iter: int = 1000) -> float:
    """||A||_2 by power iteration on A^T A (float64)."""
    m, n = A.shape
    v = omega(n, 1, seed, 0)[:, 0]
    v /= np.linalg.norm(v)
    lam_old = 0.0
    for _ in range(max_iter):
        w = A.T @ (A @ v)
        lam = float(np.linalg.norm(w))
        if lam == 0.0:
            return 0.0
        v = w / lam
        if abs(lam - lam_old) <= rtol * lam:
            break
        lam_old = lam
    return math.sqrt(lam)


def adapt_p(p: int, streak: int, err: float, prev_err: float, p_min: int = 3, p_max: int = 20):
    """The power-parameter rule stated after Alg. 6 (Sec. IV.C): p grows by one
    when the relative error of step 16 increases, and falls by one after the
    error has decreased ten times in a row.  Readings: both comparisons are
    strict, an unchanged error ends the streak, every change of p restarts it,
    and p stays within [p_min, p_max].  Returns the new (p, streak)."""
    if err > prev_err:
        return min(p + 1, p_max), 0
    if err < prev_err:
        streak += 1
        if streak == 10:
            return max(p - 1, p_min), 0
        return p, streak
    return p, 0


def sample_lowrank(rows: np.ndarray, cols: np.ndarray, Us: np.ndarray, V: np.ndarray,
                   chunk: int = 1 << 20) -> np.ndarray:
    """Entries (Us V^T)_{ij} at the listed positions (the X^i of Alg. 6 step 15
    evaluated only where it is used)."""
    out = np.empty(rows.size, dtype=np.float64)
    for a in range(0, rows.size, chunk):
        out[a:a + chunk] = np.einsum("ij,ij->i", Us[rows[a:a + chunk]], V[cols[a:a + chunk]])
    return out


@dataclasses.dataclass
class SvtResult:
    Us: np.ndarray  # m x r, columns u_j * (sigma_j - tau)
    V: np.ndarray   # n x r
    sigma: np.ndarray  # r leading singular values of the last Y (before shrink)
    iters: int
    err: float
    converged: bool
    history: list


def svt_fast(m, n, row_ptr, col, val, tau=None, delta=1.2, eps=1e-4, l=5, s=10, p0=3, p_min=3,
             p_max=20, i_max=1000, i_reuse=50, q_reuse=10, recycle=1, seed=0, callback=None,
             on_factors=None, on_update=None, inner=0) -> SvtResult:
    """Alg. 6.  ``recycle``: 0 none, 1 reuse Q, 2 reuse U, 3 warm-started Omega.
    ``inner``: the SVD of a fresh call, 0 rSVD-BKI (Alg. 5, as Alg. 6 states)
    or 1 rSVD-PI (Alg. 4, one block of k + s columns whatever p).
    ``callback(rec)`` receives each iteration's record; ``on_factors(rec, Us,
    V)`` also the factors of X^i (for metrics that need the estimate);
    ``on_update(rec, y)`` the values of Y^i on Phi (CSR order) after step 16."""
    A = as_csr64(m, n, row_ptr, col, val)
    M = A.data.copy()
    rows = np.repeat(np.arange(m), np.diff(np.asarray(row_ptr)))
    cols = np.asarray(col, np.int64)
    if tau is None:
        tau = default_tau(m, n)
    normF = float(np.linalg.norm(M))
    norm2 = spectral_norm(A, seed)
    c = math.ceil(tau / (delta * norm2))
    Y = A.copy()
    Y.data = c * delta * M
    r = 0
    q = 0
    p = p0
    prev_err = math.inf
    streak = 0
    call_id = 1
    basis = None
    Vprev = None
    history = []
    Us = np.zeros((m, 0))
    Vr = np.zeros((n, 0))
    sig = np.zeros(0)
    err = math.inf
    it = 0
    for it in range(1, i_max + 1):
        k = r + 1
        force_fresh = False
        nsvd = 0
        used_recycle = False
        margin = math.inf  # closest any computed sigma came to tau, relative (a conditioning record only)
        while True:
            if inner == 1:
                kk, _ = clamp_rank(m, n, k, s, 0)
                pp = p
            else:
                kk, pp = clamp_rank(m, n, k, s, p)
            width_ok = basis is not None and (recycle != 2 or basis.shape[1] >= kk) and \
                (recycle != 1 or basis.shape[1] >= kk)
            fresh = (recycle in (0, 3) or it < i_reuse or q == q_reuse or not width_ok or force_fresh)
            if fresh:
                Om = omega(n, kk + s, seed, call_id)
                if recycle == 3 and Vprev is not None and r > 0:
                    w = min(r, kk + s, Vprev.shape[1])
                    Om[:, :w] = Vprev[:, :w]
                U, S, V, Q = (rsvd_pi if inner == 1 else rsvd_bki)(Y, kk, pp, s, Om=Om)
                call_id += 1
                q = 0
                basis = Q if recycle == 1 else U
                recycled = False
            else:
                if recycle == 1:
                    U, S, V = recycle_q(Y, basis, kk)
                else:
                    U, S, V = recycle_u(Y, basis)
                    basis = U
                q += 1
                recycled = True
                used_recycle = True
            nsvd += 1
            if S.size:
                margin = min(margin, float(np.min(np.abs(S - tau))) / tau)
            k += l
            if S.size == 0 or S[-1] <= tau:
                break
            if kk >= min(m, n) - s:  # cannot grow further
                break
            if recycled:
                force_fresh = True
        r = int(np.count_nonzero(S > tau))
        sig = S[:r].copy()
        Us = U[:, :r] * (S[:r] - tau)
        Vr = V[:, :r].copy()
        Vprev = V
        x = sample_lowrank(rows, cols, Us, Vr)
        err = float(np.linalg.norm(x - M)) / normF
        rec = dict(i=it, k=int(kk), r=r, p=int(p), err=err, nsvd=nsvd, recycled=used_recycle,
                   sigma_last=float(S[-1]) if S.size else 0.0, sigma_max=float(S[0]) if S.size else 0.0, c=c, norm2=norm2, tau_margin=margin)
        history.append(rec)
        if callback is not None:
            callback(rec)
        if on_factors is not None:
            on_factors(rec, Us, Vr)
        if err < eps:
            return SvtResult(Us, Vr, sig, it, err, True, history)
        Y.data = Y.data + delta * (M - x)
        if on_update is not None:
            on_update(rec, Y.data)
        p, streak = adapt_p(p, streak, err, prev_err, p_min, p_max)
        prev_err = err
    return SvtResult(Us, Vr, sig, it, err, False, history)


def svt_exact(m, n, row_ptr, col, val, tau=None, delta=1.2, eps=1e-4, l=5, i_max=1000,
              seed=0, norm2=None) -> SvtResult:
    """Alg. 2 with an exact (dense LAPACK) truncated SVD standing in for svds.
    The repeat loop of steps 4-7 is kept: k grows by l until the k-th singular
    value is <= tau.  Only for matrices that fit densely in memory."""
    A = as_csr64(m, n, row_ptr, col, val)
    M = A.data.copy()
    rows = np.repeat(np.arange(m), np.diff(np.asarray(row_ptr)))
    cols = np.asarray(col, np.int64)
    if tau is None:
        tau = default_tau(m, n)
    normF = float(np.linalg.norm(M))
    if norm2 is None:
        norm2 = spectral_norm(A, seed)
    c = math.ceil(tau / (delta * norm2))
    y = c * delta * M
    r = 0
    history = []
    lim = min(m, n)
    Us = np.zeros((m, 0))
    Vr = np.zeros((n, 0))
    sig = np.zeros(0)
    err = math.inf
    it = 0
    for it in range(1, i_max + 1):
        Yd = np.zeros((m, n))
        Yd[rows, cols] = y
        Uf, Sf, Vtf = np.linalg.svd(Yd, full_matrices=False)
        k = r + 1
        while True:
            kk = min(k, lim)
            k += l
            if Sf[kk - 1] <= tau or kk == lim:
                break
        r = int(np.count_nonzero(Sf[:kk] > tau))
        sig = Sf[:r].copy()
        Us = Uf[:, :r] * (Sf[:r] - tau)
        Vr = Vtf[:r].T.copy()
        x = sample_lowrank(rows, cols, Us, Vr)
        err = float(np.linalg.norm(x - M)) / normF
        history.append(dict(i=it, k=int(kk), r=r, err=err))
        if err < eps:
            return SvtResult(Us, Vr, sig, it, err, True, history)
        y = y + delta * (M - x)
    return SvtResult(Us, Vr, sig, it, err, False, history)
