"""Randomized SVD algorithms of Feng, Yu & Li (CPU oracle; test infrastructure).

Plain float64 restatements of Sec. II.B (Alg. 1) and Sec. III (Alg. 3, 4, 5,
Lemma 3) and of the two subspace-recycling strategies of Sec. IV.B, following
the paper's steps and notation.  LAPACK (through NumPy/SciPy) does the dense
steps the paper delegates to built-ins: qr for orth(), eigh for eig(), pivoted
getrf for lu(), and SciPy's sparse products for A*X.

Readings taken where the paper is silent or inconsistent:
  * Alg. 5 never assigns H_p ("if i < p" guards the only assignment) although
    H has p+1 blocks; H_i = A (A^T H_{i-1}) is formed for every i <= p and lu()
    is applied only while i < p, the last block entering orth(H) as is.
  * The output V is n x k (the listing prints k x n).  eigSVD(B^T) returns
    [V, S, W] with W = the k x k right factor.
  * eigSVD returns ascending singular values (Sec. III.A after Lemma 1); the
    callers take the last k and reverse them so results are descending.
  * eigSVD needs full column rank; eigenpairs with lambda <= K*eps*lambda_max
    are dropped, so a rank-deficient input yields fewer columns.
  * The power/Krylov count is clamped so (p+1)(k+s) <= min(m, n); if k+s
    exceeds min(m, n), k is reduced to min(m, n) - s.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .philox import omega

EPS64 = np.finfo(np.float64).eps


def as_csr64(m, n, row_ptr, col, val) -> sp.csr_matrix:
    return sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col, np.int64),
                          np.asarray(row_ptr, np.int64)), shape=(m, n))


def lu_basis(K: np.ndarray) -> np.ndarray:
    """First output of lu(K): the row-permuted unit lower factor P^T L, whose
    column space equals that of K (Lemma 3, eq. (9))."""
    PL, _U = sla.lu(K, permute_l=True)
    return PL


def orth(H: np.ndarray) -> np.ndarray:
    """orth() of Alg. 1: orthonormal basis of range(H) by Householder QR."""
    Q, _R = np.linalg.qr(H, mode="reduced")
    return Q


def eig_svd(A: np.ndarray):
    """eigSVD (Alg. 3): B = A^T A, [V, D] = eig(B), S = sqrt(D), U = A V S^-1.

    Returns (U, S, V) with S ascending (Lemma 1 gives the economic SVD).  Needs
    m >= n; eigen-directions with lambda <= n*eps*lambda_max are dropped."""
    m, n = A.shape
    if m < n:
        raise ValueError("eigSVD needs m >= n")
    B = A.T @ A
    lam, V = np.linalg.eigh(B)  # ascending
    keep = lam > n * EPS64 * max(lam[-1], 0.0)
    lam, V = lam[keep], V[:, keep]
    S = np.sqrt(lam)
    U = (A @ V) / S
    return U, S, V


def clamp_rank(m: int, n: int, k: int, s: int, p: int):
    """Clamp (k, p) so that one Krylov block fits and (p+1)(k+s) <= min(m, n)."""
    lim = min(m, n)
    if k + s > lim:
        k = max(1, lim - s)
    kb = k + s
    if kb > lim:
        raise ValueError("k + s exceeds min(m, n) even at k = 1")
    p = max(0, min(p, lim // kb - 1))
    return k, p


def rsvd_basic(A, k: int, p: int, s: int = 10, seed: int = 0, call_id: int = 0, Om=None):
    """Basic rSVD with power iteration (Alg. 1): orth after every product."""
    m, n = A.shape
    if Om is None:
        Om = omega(n, k + s, seed, call_id)
    Q = orth(A @ Om)
    for _ in range(p):
        G = orth(A.T @ Q)
        Q = orth(A @ G)
    B = Q.T @ A  # (k+s) x n
    B = np.asarray(B)
    Ub, S, Vt = np.linalg.svd(B, full_matrices=False)
    U = Q @ Ub
    return U[:, :k], S[:k], Vt[:k].T


def rsvd_pi(A, k: int, p: int, s: int = 10, seed: int = 0, call_id: int = 0, Om=None):
    """rSVD-PI (Alg. 4): LU in the power loop, eigSVD for the last orth and for
    the SVD of B.  Returns U (m x k), S (k, descending), V (n x k), Q."""
    m, n = A.shape
    if Om is None:
        Om = omega(n, k + s, seed, call_id)
    Q = A @ Om
    for i in range(p + 1):
        if i < p:
            Q = lu_basis(Q)
        else:
            Q, _S, _V = eig_svd(Q)
            break
        Q = A @ (A.T @ Q)
    Bt = np.asarray(A.T @ Q)  # B^T = A^T Q, n x (k+s)
    V, S, W = eig_svd(Bt)
    kk = min(k, S.size)
    # ind = s+1 : k+s of the ascending list, i.e. its last k entries
    V, S, W = V[:, -kk:], S[-kk:], W[:, -kk:]
    U = Q @ W
    return U[:, ::-1].copy(), S[::-1].copy(), V[:, ::-1].copy(), Q


def rsvd_bki(A, k: int, p: int, s: int = 10, seed: int = 0, call_id: int = 0, Om=None):
    """rSVD-BKI (Alg. 5).  Returns U (m x k), S (k, descending), V (n x k) and
    the Krylov basis Q (m x (p+1)(k+s)) kept for subspace recycling."""
    m, n = A.shape
    if Om is None:
        Om = omega(n, k + s, seed, call_id)
    blocks = [lu_basis(A @ Om)]
    for i in range(1, p + 1):
        Hi = A @ (A.T @ blocks[-1])
        blocks.append(lu_basis(Hi) if i < p else Hi)
    Q = orth(np.hstack(blocks))
    S, U, V = _ritz_from_basis(A, Q, k)
    return U, S, V, Q


def _ritz_from_basis(A, Q, k):
    """Steps 8-11 of Alg. 5: B = Q^T A, eigSVD(B^T), keep the last k (largest)."""
    Bt = np.asarray(A.T @ Q)
    V, S, W = eig_svd(Bt)
    kk = min(k, S.size)
    V, S, W = V[:, -kk:], S[-kk:], W[:, -kk:]
    U = Q @ W
    return S[::-1].copy(), U[:, ::-1].copy(), V[:, ::-1].copy()


def recycle_q(A, Q, k):
    """Recycling strategy 1 (Sec. IV.B): restart Alg. 5 at step 8 with the
    previous Krylov basis Q.  Returns U, S (descending), V."""
    S, U, V = _ritz_from_basis(A, Q, k)
    return U, S, V


def recycle_u(A, Uprev):
    """Recycling strategy 2 (Sec. IV.B): B = U_prev^T Y, eigSVD(B^T),
    U = U_prev W.  Returns all k_prev triplets, descending."""
    Bt = np.asarray(A.T @ Uprev)
    V, S, W = eig_svd(Bt)
    U = Uprev @ W
    return U[:, ::-1].copy(), S[::-1].copy(), V[:, ::-1].copy()
