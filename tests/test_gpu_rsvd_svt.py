"""Parity of the GPU rSVD-PI / rSVD-BKI (Alg. 4/5) and fast SVT (Alg. 6) with
the float64 CPU oracle on the same seeded inputs and the same Philox Omega.

Tolerances (plain float32 path): leading singular values within 1e-5
relative; SVT: the same iteration count +-1, the same ranks, and the relative
completion error on Phi within 1e-4 of the oracle's."""
import math

import numpy as np
import pytest

import mc_synth
from oracle import metrics
from oracle import rsvd as orsvd
from oracle import svt as osvt
from oracle.rsvd import as_csr64

pytestmark = pytest.mark.gpu

SIG_TOL = 1e-5


@pytest.fixture(scope="module")
def mc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_06860_gb300 as mc

    return mc


def _A(o):
    return as_csr64(o.m, o.n, o.row_ptr, o.col, o.val)


@pytest.fixture(scope="module")
def ratings_small():
    return mc_synth.ratings(m=4000, n=1200, N=150_000, seed=2)


@pytest.mark.parametrize("k,p", [(20, 3), (50, 2), (5, 0)])
def test_rsvd_bki_matches_oracle(mc, ratings_small, k, p):
    o = ratings_small
    with mc.Handle.from_observed(o) as h:
        U, S, V = h.rsvd_bki(k, s=10, p=p, seed=11, call_id=4)
    Uo, So, Vo, _ = orsvd.rsvd_bki(_A(o), k, p, s=10, seed=11, call_id=4)
    assert S.shape == (k,)
    assert metrics.sigma_rel_err(S, So) < SIG_TOL
    # well-separated leading directions agree
    gap = np.flatnonzero(np.diff(So) / So[1:] < -0.05)
    j = int(gap[0]) + 1 if gap.size else 1
    assert metrics.max_principal_angle(U[:, :j], Uo[:, :j]) < 1e-3
    assert metrics.max_principal_angle(V[:, :j], Vo[:, :j]) < 1e-3
    # U S V^T is the Ritz triple: A v_j = sigma_j u_j (restricted to the basis)
    A = _A(o)
    r = np.linalg.norm(A.T @ U.astype(np.float64) - V.astype(np.float64) * S, axis=0) / S
    assert np.max(r) < 1e-4


def test_rsvd_pi_matches_oracle(mc, ratings_small):
    o = ratings_small
    with mc.Handle.from_observed(o) as h:
        U, S, V = h.rsvd_pi(30, s=10, p=3, seed=5, call_id=0)
    _, So, _, _ = orsvd.rsvd_pi(_A(o), 30, 3, s=10, seed=5, call_id=0)
    assert metrics.sigma_rel_err(S, So) < SIG_TOL


def test_rsvd_basic_matches_oracle(mc, ratings_small):
    """Basic rSVD (Alg. 1): an orthonormalisation after every product; same
    Omega, same singular values as the oracle's Alg. 1 (and, by Theorem 1, as
    rSVD-PI's)."""
    o = ratings_small
    with mc.Handle.from_observed(o) as h:
        U, S, V = h.rsvd_basic(30, s=10, p=3, seed=5, call_id=0)
        _, Spi, _ = h.rsvd_pi(30, s=10, p=3, seed=5, call_id=0)
    _, So, Vo = orsvd.rsvd_basic(_A(o), 30, 3, s=10, seed=5, call_id=0)
    assert metrics.sigma_rel_err(S, So) < SIG_TOL
    assert metrics.sigma_rel_err(Spi, So) < SIG_TOL
    gap = np.flatnonzero(np.diff(So) / So[1:] < -0.05)
    j = int(gap[0]) + 1 if gap.size else 1
    assert metrics.max_principal_angle(V[:, :j], Vo[:, :j]) < 1e-3


def test_rsvd_on_lowrank_exact(mc):
    o = mc_synth.lowrank_uniform(400, 300, 6, frac=1.0, seed=4)  # fully observed rank-6 matrix
    with mc.Handle.from_observed(o) as h:
        U, S, V = h.rsvd_bki(6, s=10, p=2, seed=1)
    ref = np.linalg.svd(o.dense.astype(np.float64), compute_uv=False)[:6]
    assert metrics.sigma_rel_err(S, ref) < SIG_TOL
    X = (U * S) @ V.T
    assert np.linalg.norm(X - o.dense) / np.linalg.norm(o.dense) < 1e-5


def test_rsvd_clamps_and_empty(mc):
    o = mc_synth.lowrank_uniform(30, 20, 2, frac=0.5, seed=1)
    with mc.Handle.from_observed(o) as h:
        U, S, V = h.rsvd_bki(50, s=10, p=5, seed=0)  # k+s > min(m,n): k clamped to 10, p to 1
        assert S.size == 10
        _, So, _, _ = orsvd.rsvd_bki(_A(o), *orsvd.clamp_rank(30, 20, 50, 10, 5), s=10, seed=0)
        assert metrics.sigma_rel_err(S, So) < SIG_TOL
    empty = mc.Handle(5, 30, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    U, S, V = empty.rsvd_bki(3, s=2, p=1)
    assert S.size == 0
    empty.close()


def _svt_compare(mc, o, prm_kw, i_max=1000, tol_iters=1):
    kw = dict(prm_kw)
    prm = mc.params(**kw, i_max=i_max)
    okw = {k: v for k, v in kw.items() if k not in ("precision",)}
    ref = osvt.svt_fast(o.m, o.n, o.row_ptr, o.col, o.val, i_max=i_max, **okw)
    hist = []
    with mc.Handle.from_observed(o) as h:
        for _ in range(i_max):
            info = h.svt_step(prm)
            hist.append(info)
            if info["converged"]:
                break
        Us, V, sg = h.factors()
    return ref, hist, (Us, V, sg)


def test_svt_config1_matches_oracle(mc):
    """500 x 500 rank 10, 20% observed, tau = 5 sqrt(mn), delta = 1.2/0.2,
    eps = 1e-4, l = 5, warm-started Omega."""
    o = mc_synth.lowrank_uniform(500, 500, 10, frac=0.2, seed=0)
    ref, hist, (Us, V, sg) = _svt_compare(mc, o, dict(tau=2500.0, delta=6.0, eps=1e-4, recycle=3, seed=0))
    assert ref.converged and hist[-1]["converged"]
    assert abs(len(hist) - ref.iters) <= 1
    assert hist[0]["c"] == ref.history[0]["c"]
    n = min(len(hist), ref.iters)
    assert [x["r"] for x in hist[:n]] == [x["r"] for x in ref.history[:n]]
    for a, b in zip(hist[:n], ref.history[:n]):
        assert abs(a["err"] - b["err"]) <= 1e-4 * max(1.0, b["err"]), (a, b)
    X = Us.astype(np.float64) @ V.astype(np.float64).T
    Xo = ref.Us @ ref.V.T
    assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) < 1e-3
    assert np.linalg.norm(X - o.dense) / np.linalg.norm(o.dense) < 1e-3


@pytest.mark.parametrize("case", ["config1", "zipf"])
def test_svt_iterate_matches_oracle_elementwise(mc, case):
    """Y^i on Phi (Alg. 6 step 16) entry by entry against the oracle's after
    1, 5 and 20 iterations.  Bound: each step adds delta (M - x^i) on Phi, and
    the per-iteration parity of the estimate on Phi is 1e-4 of the data
    (the error tolerance of the trajectory tests), so after i steps an entry
    may differ by delta * i * 1e-4 * max|M| and the whole vector by
    delta * i * 1e-4 * ||P_Phi M||_F.  A wrong sign, a dropped term or a
    misplaced entry in the fused update exceeds that at the first step."""
    if case == "config1":
        o = mc_synth.lowrank_uniform(500, 500, 10, frac=0.2, seed=0)
        kw = dict(tau=2500.0, delta=6.0, eps=1e-4, recycle=3, seed=0)
    else:
        o = mc_synth.ratings(m=4000, n=1200, N=150_000, seed=2)
        kw = dict(tau=5.0 * 1200, delta=1.9, eps=1e-4, recycle=3, seed=4)
    checks = (1, 5, 20)
    ys = {}

    def keep(rec, y):
        if rec["i"] in checks:
            ys[rec["i"]] = y.copy()

    osvt.svt_fast(o.m, o.n, o.row_ptr, o.col, o.val, i_max=max(checks), on_update=keep, **kw)
    m_max = float(np.max(np.abs(o.val)))
    m_fro = float(np.linalg.norm(o.val.astype(np.float64)))
    prm = mc.params(**kw, i_max=1000)
    with mc.Handle.from_observed(o) as h:
        for i in range(1, max(checks) + 1):
            info = h.svt_step(prm)
            assert not info["converged"]
            if i in checks:
                got = h.get_values().astype(np.float64)
                want = ys[i]
                assert got.shape == want.shape
                d = np.abs(got - want)
                assert np.max(d) <= kw["delta"] * i * 1e-4 * m_max, (i, float(np.max(d)))
                assert np.linalg.norm(got - want) <= kw["delta"] * i * 1e-4 * m_fro, i


def test_svt_inner_rsvd_pi_matches_oracle(mc):
    """Alg. 6 with rSVD-PI (Alg. 4) as the inner SVD (mc_params.inner = 1),
    warm-started Omega: the whole solve against the oracle's, iteration by
    iteration."""
    o = mc_synth.lowrank_uniform(500, 500, 10, frac=0.2, seed=0)
    ref, hist, (Us, V, _) = _svt_compare(mc, o, dict(tau=2500.0, delta=6.0, eps=1e-4, recycle=3, seed=0, inner=1))
    assert ref.converged and hist[-1]["converged"]
    assert abs(len(hist) - ref.iters) <= 1
    n = min(len(hist), ref.iters)
    assert [x["r"] for x in hist[:n]] == [x["r"] for x in ref.history[:n]]
    for a, b in zip(hist[:n], ref.history[:n]):
        assert abs(a["err"] - b["err"]) <= 1e-4 * max(1.0, b["err"]), (a, b)
    X = Us.astype(np.float64) @ V.astype(np.float64).T
    assert np.linalg.norm(X - o.dense) / np.linalg.norm(o.dense) < 1e-3


def test_svt_recycle_q_matches_oracle(mc):
    o = mc_synth.lowrank_uniform(500, 500, 10, frac=0.2, seed=0)
    ref, hist, _ = _svt_compare(mc, o, dict(tau=2500.0, delta=6.0, eps=1e-4, recycle=1, i_reuse=50, q_reuse=2,
                                            seed=0))
    assert ref.converged and hist[-1]["converged"]
    assert abs(len(hist) - ref.iters) <= 1
    n = min(len(hist), ref.iters)
    assert [x["recycled"] for x in hist[:n]] == [int(x["recycled"]) for x in ref.history[:n]]
    for a, b in zip(hist[:n], ref.history[:n]):
        assert abs(a["err"] - b["err"]) <= 1e-4 * max(1.0, b["err"]), (a, b)


# A rank decision (sigma > tau, Alg. 6) whose oracle sigma lies within this
# relative distance of tau is not fixed by float32 arithmetic: eigSVD (Alg. 3)
# squares the spectrum and the Krylov basis of rSVD-BKI is ill-conditioned, so
# trailing Ritz values of a clustered tail carry errors of 1e-4 relative and
# more.  Trajectories are compared up to the first such decision.
TAU_MARGIN = 1e-3


def _compare_trajectory(hist, ref_hist, min_iters):
    n = next((j for j, b in enumerate(ref_hist) if b["tau_margin"] < TAU_MARGIN), len(ref_hist))
    assert n >= min_iters and any(b["recycled"] for b in ref_hist[:n]), n
    assert len(hist) >= n
    for a, b in zip(hist[:n], ref_hist[:n]):
        assert a["r"] == b["r"] and a["k"] == b["k"] and a["recycled"] == int(b["recycled"]), (a, b)
        assert abs(a["err"] - b["err"]) <= 1e-4 * max(1.0, b["err"]), (a, b)


def test_svt_recycle_u_first_iterations(mc):
    """Image-like 256 x 256 with a clustered tail near tau: the ranks swing
    between 45 and 175, so recycled U bases of K > 128 columns are exercised."""
    o = mc_synth.smooth_image(256, 256, 10, sigma_px=4.0, frac=0.5, seed=3)
    kw = dict(tau=5 * 256.0, delta=1.2 / 0.5, eps=1e-4, recycle=2, i_reuse=4, q_reuse=3, seed=1)
    ref, hist, _ = _svt_compare(mc, o, kw, i_max=12)
    _compare_trajectory(hist, ref.history, 5)


def test_svt_recycle_u_lowrank(mc):
    """500 x 500 rank 10: a fresh rSVD every fourth iteration, recycled U
    bases in between; every decision lies well clear of tau."""
    o = mc_synth.lowrank_uniform(500, 500, 10, frac=0.2, seed=0)
    kw = dict(tau=2500.0, delta=6.0, eps=1e-4, recycle=2, i_reuse=4, q_reuse=3, seed=0)
    ref, hist, _ = _svt_compare(mc, o, kw, i_max=12)
    _compare_trajectory(hist, ref.history, 12)


def test_svt_sample_and_values(mc):
    o = mc_synth.lowrank_uniform(120, 90, 3, frac=0.4, seed=9)
    with mc.Handle.from_observed(o) as h:
        prm = mc.params(tau=5 * math.sqrt(120 * 90), delta=1.2 / 0.4, eps=1e-4, recycle=0)
        for _ in range(3):
            h.svt_step(prm)
        Us, V, sg = h.factors()
        rows = np.array([0, 5, 119, 7], np.int64)
        cols = np.array([0, 89, 3, 7], np.int64)
        got = h.sample(rows, cols)
        want = np.einsum("ij,ij->i", Us[rows].astype(np.float64), V[cols].astype(np.float64))
        assert np.allclose(got, want, rtol=1e-5, atol=1e-5)
        y = h.get_values()
        assert y.shape == (o.nnz,) and np.all(np.isfinite(y))


def test_products_after_step_see_updated_iterate(mc):
    """After an SVT step the copy of Y into CSC order runs on the handle's
    second stream; a Y^T X product issued right after must wait for it and
    agree with the product of the updated values in CSR order."""
    o = mc_synth.ratings(m=6000, n=2500, N=400000, seed=11)
    rng = np.random.default_rng(5)
    with mc.Handle.from_observed(o) as h:
        prm = mc.params(tau=5 * math.sqrt(o.m * o.n), delta=1.9, eps=1e-4, recycle=1, seed=3)
        for step in range(3):
            h.svt_step(prm)
            Xt = rng.standard_normal((o.m, 12)).astype(np.float32)
            got = h.spmm(Xt, trans=True)      # reads the CSC copy immediately
            y = h.get_values().astype(np.float64)
            A = as_csr64(o.m, o.n, o.row_ptr, o.col, y)
            want = A.T @ Xt.astype(np.float64)
            assert np.max(np.abs(got - want)) < 1e-4 * max(1.0, np.abs(want).max()), step
        h.join()
        X = rng.standard_normal((o.n, 12)).astype(np.float32)
        assert np.array_equal(h.spmm(X), h.spmm(X))
