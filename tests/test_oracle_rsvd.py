"""Pins for the CPU oracle's random generator and randomized SVDs.

Each check ties the oracle to something other than itself: published
known-answer vectors, the N(0,1) law, LAPACK's SVD, the equivalences of
Lemmas 1-3 and Theorems 1-2 (exact-arithmetic statements, so they hold to
rounding), closed-form spectra and the error bound (4)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy import stats

from oracle import metrics
from oracle.philox import omega, philox4x32_10, philox_words
from oracle.rsvd import (clamp_rank, eig_svd, lu_basis, orth, recycle_q, recycle_u, rsvd_basic,
                         rsvd_bki, rsvd_pi)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers():
    for r in _kat():
        out = philox4x32_10(*r[:6])
        assert [int(x) for x in out] == r[6:]


def test_philox_vectorised_matches_scalar():
    i = np.arange(7)[:, None]
    j = np.arange(5)[None, :]
    vec = philox4x32_10(i, j, 3, 0, 0xDEADBEEF, 1)
    for a in range(7):
        for b in range(5):
            sc = philox4x32_10(a, b, 3, 0, 0xDEADBEEF, 1)
            assert all(int(v[a, b]) == int(s) for v, s in zip(vec, sc))


def test_omega_is_standard_normal():
    z = omega(20000, 8, seed=12345, call_id=7).ravel()
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.02
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # columns independent of each other
    c = np.corrcoef(omega(20000, 4, seed=1, call_id=0).T)
    assert np.abs(c - np.eye(4)).max() < 0.05


def test_omega_prefix_columns_and_streams():
    a = omega(300, 5, seed=9, call_id=2)
    b = omega(300, 12, seed=9, call_id=2)
    assert np.array_equal(a, b[:, :5])
    assert np.array_equal(omega(300, 3, 9, 2, col0=5), b[:, 5:8])
    assert not np.allclose(omega(300, 5, 9, 3), a)
    assert not np.allclose(omega(300, 5, 10, 2), a)
    x0, x1 = philox_words(4, 2, seed=(5 << 32) | 6, call_id=(7 << 32) | 8)
    r = philox4x32_10(3, 1, 8, 7, 6, 5)
    assert int(x0[3, 1]) == int(r[0]) and int(x1[3, 1]) == int(r[1])


def test_omega_box_muller_edge_words():
    # u1 = (x0+1) 2^-32 is 1 for x0 = 2^32-1, making the sample exactly 0; the
    # transform is finite for every word (no log(0)).
    z = omega(5000, 50, seed=3, call_id=1)
    assert np.all(np.isfinite(z))


def _rand_tall(m, n, cond, rng):
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.logspace(0, -np.log10(cond), n)
    return U @ np.diag(s) @ V.T, s


def test_eig_svd_matches_lapack_svd():
    rng = np.random.default_rng(0)
    A, s = _rand_tall(200, 30, 100.0, rng)
    U, S, V = eig_svd(A)
    assert np.all(np.diff(S) >= 0), "eigSVD returns ascending values"
    ref = np.linalg.svd(A, compute_uv=False)[::-1]
    assert np.max(np.abs(S - ref) / ref) < 1e-10
    assert np.allclose(U @ np.diag(S) @ V.T, A, atol=1e-12)
    assert np.allclose(U.T @ U, np.eye(30), atol=1e-9)
    assert np.allclose(V.T @ V, np.eye(30), atol=1e-12)


def test_eig_svd_drops_rank_deficient_directions():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((50, 4)) @ rng.standard_normal((4, 8))
    U, S, V = eig_svd(A)
    assert S.size == 4
    assert np.allclose(U @ np.diag(S) @ V.T, A, atol=1e-10)


def test_lu_basis_spans_same_space_and_is_unit_lower():
    rng = np.random.default_rng(2)
    K = rng.standard_normal((40, 6))
    PL = lu_basis(K)
    assert metrics.max_principal_angle(PL, K) < 1e-10
    # P^T L: some row permutation of a unit lower-triangular matrix
    ones = np.isclose(np.abs(PL), 1.0).sum()
    assert ones >= 6
    assert np.abs(PL).max() <= 1.0 + 1e-12  # partial pivoting bounds |L| by 1


def test_orth_is_orthonormal_basis():
    rng = np.random.default_rng(3)
    H = rng.standard_normal((80, 10))
    Q = orth(H)
    assert np.allclose(Q.T @ Q, np.eye(10), atol=1e-13)
    assert metrics.max_principal_angle(Q, H) < 1e-10


def _sparse_test_matrix(m, n, density, seed, decay=None):
    rng = np.random.default_rng(seed)
    A = sp.random(m, n, density=density, random_state=rng, format="csr")
    A.data = rng.standard_normal(A.nnz)
    return A


def test_theorem1_rsvd_pi_equals_basic_rsvd():
    # Same Omega -> same result (exact-arithmetic equivalence, Thm. 1).
    A = _sparse_test_matrix(300, 200, 0.05, 4)
    for p in (0, 2):
        Om = omega(200, 15 + 5, seed=11, call_id=0)
        U1, S1, V1 = rsvd_basic(A, 15, p, s=5, Om=Om)
        U2, S2, V2, _ = rsvd_pi(A, 15, p, s=5, Om=Om)
        assert np.max(np.abs(S1 - S2) / S1) < 1e-10
        X1 = U1 @ np.diag(S1) @ V1.T
        X2 = U2 @ np.diag(S2) @ V2.T
        assert np.linalg.norm(X1 - X2) / np.linalg.norm(X1) < 1e-9


def _bki_by_qr(A, Om, p, k):
    """Block Krylov subspace with plain QR (the scheme Thm. 2 compares with)."""
    blocks = [A @ Om]
    for _ in range(p):
        blocks.append(A @ (A.T @ blocks[-1]))
    K = np.hstack(blocks)
    K = K / np.linalg.norm(K, axis=0)
    Q, _ = np.linalg.qr(K)
    B = np.asarray((A.T @ Q).T)
    Ub, S, Vt = np.linalg.svd(B, full_matrices=False)
    return Q @ Ub[:, :k], S[:k], Vt[:k].T


def test_theorem2_rsvd_bki_equals_block_krylov():
    A = _sparse_test_matrix(400, 300, 0.03, 5)
    Om = omega(300, 12, seed=2, call_id=5)
    U1, S1, V1, Q = rsvd_bki(A, 8, 2, s=4, Om=Om)
    U2, S2, V2 = _bki_by_qr(A, Om, 2, 8)
    assert Q.shape == (400, 36)
    assert np.max(np.abs(S1 - S2) / S2) < 1e-9
    assert metrics.max_principal_angle(U1, U2) < 1e-6
    assert metrics.max_principal_angle(V1, V2) < 1e-6


def test_lemma2_result_independent_of_basis_choice():
    # Replacing orth(H) by another orthonormal basis of range(H) changes nothing.
    A = _sparse_test_matrix(250, 180, 0.05, 6)
    Om = omega(180, 10, seed=0, call_id=1)
    _, S1, _, Q = rsvd_bki(A, 6, 1, s=4, Om=Om)
    Rot, _ = np.linalg.qr(np.random.default_rng(7).standard_normal((Q.shape[1],) * 2))
    U2, S2, V2 = recycle_q(A, Q @ Rot, 6)
    assert np.max(np.abs(S1 - S2) / S1) < 1e-11


def test_closed_form_spectrum_recovered():
    # A = U diag(0.9^j) V^T, full rank: with a Krylov space as wide as the
    # matrix the rSVD must return the exact leading singular values.
    rng = np.random.default_rng(8)
    m, n = 120, 60
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = 0.9 ** np.arange(1, n + 1)
    A = sp.csr_matrix(U @ np.diag(sig) @ V.T)
    Ub, S, Vb, _ = rsvd_bki(A, 10, 2, s=10, seed=1)  # K_t = 60 = n
    assert np.max(np.abs(S - sig[:10]) / sig[:10]) < 1e-9
    Up, Sp, Vp, _ = rsvd_pi(A, 10, 30, s=10, seed=1)
    assert np.max(np.abs(Sp - sig[:10]) / sig[:10]) < 1e-6
    assert metrics.max_principal_angle(Ub, U[:, :10]) < 1e-6


def test_error_bound_eq4():
    rng = np.random.default_rng(9)
    m, n = 300, 200
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = 1.0 / np.arange(1, n + 1) ** 0.7
    A = sp.csr_matrix(U @ np.diag(sig) @ V.T)
    k = 20
    best = np.sqrt(np.sum(sig[k:] ** 2))
    Ub, S, Vb, _ = rsvd_bki(A, k, 4, s=10, seed=2)
    err = np.linalg.norm(A.toarray() - Ub @ np.diag(S) @ Vb.T)
    assert err <= 1.05 * best
    # the rank-k result never beats the optimum (Eckart-Young)
    assert err >= best * (1 - 1e-12)


def test_brute_force_tiny():
    rng = np.random.default_rng(10)
    for m, n in ((8, 6), (7, 7), (5, 8)):
        D = rng.standard_normal((m, n))
        D[rng.random((m, n)) < 0.3] = 0.0
        A = sp.csr_matrix(D)
        k, p = clamp_rank(m, n, 2, 2, 3)
        U, S, V, _ = rsvd_bki(A, k, p, s=2, seed=3)
        ref = np.linalg.svd(D, compute_uv=False)
        # the clamped Krylov space covers min(m, n) directions only when it is
        # full; compare where it is (rank of the Krylov space >= min(m,n)).
        if (p + 1) * (k + 2) >= min(m, n):
            assert np.allclose(S, ref[:k], rtol=1e-9)


def test_clamp_rank():
    assert clamp_rank(500, 500, 11, 10, 3) == (11, 3)
    assert clamp_rank(100, 1000, 20, 10, 5) == (20, 2)
    assert clamp_rank(12, 40, 10, 10, 3) == (2, 0)


def test_recycle_q_same_matrix_is_identity_restart():
    A = _sparse_test_matrix(200, 150, 0.06, 11)
    U, S, V, Q = rsvd_bki(A, 7, 2, s=5, seed=4)
    U2, S2, V2 = recycle_q(A, Q, 7)
    assert np.allclose(S, S2, rtol=1e-12)


def test_recycle_u_with_exact_vectors_is_exact():
    A = _sparse_test_matrix(200, 150, 0.06, 12)
    Uf, Sf, Vtf = np.linalg.svd(A.toarray(), full_matrices=False)
    U, S, V = recycle_u(A, Uf[:, :9])
    assert np.allclose(S, Sf[:9], rtol=1e-10)
    assert metrics.max_principal_angle(V, Vtf[:9].T) < 1e-6


def test_rsvd_pi_index_set_takes_largest():
    A = _sparse_test_matrix(300, 200, 0.05, 13)
    U, S, V, _ = rsvd_pi(A, 10, 6, s=10, seed=5)
    ref = np.linalg.svd(A.toarray(), compute_uv=False)[:10]
    assert np.all(np.diff(S) <= 0)
    assert np.max(np.abs(S - ref) / ref) < 2e-2
    # S equals the singular values of the rank-k product it returns
    assert np.allclose(np.linalg.svd(U @ np.diag(S) @ V.T, compute_uv=False)[:10], S, rtol=1e-10)
