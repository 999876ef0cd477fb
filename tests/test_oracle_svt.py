"""Pins for the CPU oracle's SVT (Alg. 2 / Alg. 6), spectral norm and metrics."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import mc_synth
from oracle import metrics, svt
from oracle.rsvd import as_csr64


def test_spectral_norm_matches_dense():
    o = mc_synth.lowrank_uniform(120, 90, 4, frac=0.3, seed=1)
    A = as_csr64(o.m, o.n, o.row_ptr, o.col, o.val)
    assert abs(svt.spectral_norm(A, seed=0) - np.linalg.norm(A.toarray(), 2)) < 1e-8 * np.linalg.norm(A.toarray(), 2)


def test_sample_lowrank_matches_dense_product():
    rng = np.random.default_rng(0)
    Us, V = rng.standard_normal((30, 4)), rng.standard_normal((20, 4))
    r, c = rng.integers(0, 30, 100), rng.integers(0, 20, 100)
    assert np.allclose(svt.sample_lowrank(r, c, Us, V, chunk=7), (Us @ V.T)[r, c])


def _diag_case(d, tau, delta):
    n = d.size
    row_ptr = np.arange(n + 1, dtype=np.int64)
    col = np.arange(n, dtype=np.int32)
    c = math.ceil(tau / (delta * d.max()))
    x = np.maximum(c * delta * d - tau, 0.0)
    return row_ptr, col, c, np.linalg.norm(x - d) / np.linalg.norm(d), int(np.count_nonzero(c * delta * d > tau))


def test_first_iteration_shrinks_diagonal():
    # Y^0 = c*delta*diag(d) on a diagonal observed set: shrink(Y, tau) is the
    # soft threshold of the diagonal, so X^1 = diag(max(c delta d - tau, 0)).
    d = np.array([9.0, 7.5, 6.0, 3.0, 2.0, 1.0, 0.5, 0.25])
    tau, delta = 10.0, 1.5
    row_ptr, col, c, want, r = _diag_case(d, tau, delta)
    res = svt.svt_exact(d.size, d.size, row_ptr, col, d.astype(np.float32), tau=tau, delta=delta,
                        eps=1e-12, i_max=1)
    assert res.history[0]["r"] == r == 2
    assert abs(res.history[0]["err"] - want) < 1e-12
    assert np.allclose(np.sort(np.abs(res.sigma)), np.sort(c * delta * d[:2]))


def test_first_iteration_shrinks_diagonal_fast_svt():
    # Alg. 6 on a 16 x 16 diagonal: the final repeat (k = 6, s = 10) has a
    # Krylov space of dimension 16 = n, so its SVD -- and the shrink -- is exact.
    d = np.array([9, 4, 3.5, 3, 2.5, 2, 1.5, 1, .9, .8, .7, .6, .5, .4, .3, .2])
    tau, delta = 10.0, 1.5
    row_ptr, col, c, want, r = _diag_case(d, tau, delta)
    res = svt.svt_fast(16, 16, row_ptr, col, d.astype(np.float32), tau=tau, delta=delta, eps=1e-12,
                       i_max=1, s=10, p0=3)
    h = res.history[0]
    assert h["r"] == r == 1 and h["k"] == 6 and h["nsvd"] == 2
    assert abs(h["err"] - want) < 1e-10


def test_tau_margin_records_closest_sigma():
    # As above with sigma_2 = 1.5 * 6.6 = 9.9 just below tau = 10: the exact
    # final repeat (k = 6) holds the closest sigma; the first repeat (k = 1,
    # an 11-column sketch) only approximates sigma_1 = 13.5, far from tau.
    d = np.array([9, 6.6, 3.5, 3, 2.5, 2, 1.5, 1, .9, .8, .7, .6, .5, .4, .3, .2])
    tau, delta = 10.0, 1.5
    row_ptr, col, c, _, r = _diag_case(d, tau, delta)
    res = svt.svt_fast(16, 16, row_ptr, col, d.astype(np.float32), tau=tau, delta=delta, eps=1e-12,
                       i_max=1, s=10, p0=3)
    h = res.history[0]
    assert c == 1 and h["r"] == r == 1 and h["k"] == 6 and h["nsvd"] == 2
    assert abs(h["tau_margin"] - abs(1.5 * float(np.float32(6.6)) - tau) / tau) < 1e-12


def test_svt_exact_recovers_low_rank_matrix():
    o = mc_synth.lowrank_uniform(200, 200, 5, frac=0.3, seed=3)
    res = svt.svt_exact(o.m, o.n, o.row_ptr, o.col, o.val, tau=5 * 200, delta=1.2 / 0.3, eps=1e-4)
    assert res.converged
    X = res.Us @ res.V.T
    assert np.linalg.norm(X - o.dense) / np.linalg.norm(o.dense) < 1e-3
    assert res.V.shape[1] == 5


@pytest.fixture(scope="module")
def c1():
    return mc_synth.lowrank_uniform(500, 500, 10, frac=0.2, seed=0)


@pytest.fixture(scope="module")
def c1_exact(c1):
    """Alg. 2 with an exact SVD on config 1 (the reference for the Alg. 6 pins)."""
    return svt.svt_exact(c1.m, c1.n, c1.row_ptr, c1.col, c1.val, tau=2500.0, delta=6.0, eps=1e-4, seed=0)


def test_alg6_matches_alg2_on_config1(c1, c1_exact):
    """Sec. IV.C / V.B: fast SVT behaves as SVT with an exact truncated SVD --
    same iteration count and error, and exact recovery of the rank-10 M."""
    kw = dict(tau=2500.0, delta=6.0, eps=1e-4, seed=0)
    ex = c1_exact
    fa = svt.svt_fast(c1.m, c1.n, c1.row_ptr, c1.col, c1.val, recycle=3, **kw)
    assert ex.converged and fa.converged
    assert abs(ex.iters - fa.iters) <= 2
    for res in (ex, fa):
        X = res.Us @ res.V.T
        assert np.linalg.norm(X - c1.dense) / np.linalg.norm(c1.dense) < 1e-3
        assert res.V.shape[1] == 10
    # Y stays supported on Phi: the iterate is only ever stored there, and the
    # completion error is measured there.
    assert fa.err < 1e-4


def test_p_adaptation_and_recycling_bookkeeping(c1):
    res = svt.svt_fast(c1.m, c1.n, c1.row_ptr, c1.col, c1.val, tau=2500.0, delta=6.0, eps=1e-4,
                       recycle=1, i_reuse=5, q_reuse=2, i_max=40)
    h = res.history
    assert not any(x["recycled"] for x in h[:4])
    assert any(x["recycled"] for x in h[4:])
    errs = [x["err"] for x in h]
    ps = [x["p"] for x in h]
    for i in range(1, len(h) - 1):
        if errs[i] > errs[i - 1]:
            assert ps[i + 1] == min(ps[i] + 1, 20)
        assert 3 <= ps[i] <= 20


def test_metrics():
    assert metrics.mae(np.array([1.0, 2.0]), np.array([0.0, 4.0])) == 1.5
    assert abs(metrics.rmse(np.array([1.0, 2.0]), np.array([0.0, 4.0])) - math.sqrt(2.5)) < 1e-15
    th = 0.3
    A = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    B = np.array([[1.0, 0.0], [0.0, math.cos(th)], [0.0, math.sin(th)]])
    assert abs(metrics.max_principal_angle(A, B) - th) < 1e-12
    assert metrics.sigma_rel_err(np.array([1.0, 2.2]), np.array([1.0, 2.0])) == pytest.approx(0.1)
    assert metrics.completion_error(np.array([0.0, 0.0]), np.array([3.0, 4.0])) == 1.0


@pytest.fixture(scope="module")
def c1_recycle_q(c1):
    return svt.svt_fast(c1.m, c1.n, c1.row_ptr, c1.col, c1.val, tau=2500.0, delta=6.0, eps=1e-4, seed=0,
                        recycle=1, i_reuse=5, q_reuse=2)


def test_recycle_q_matches_alg2_on_config1(c1, c1_exact, c1_recycle_q):
    """Sec. IV.B strategy 1 (restart Alg. 5 at step 8 with the stored Q) inside
    Alg. 6: with recycling from iteration 5, two recycled calls per fresh
    basis, the iteration count, the recovered matrix and its rank are those of
    Alg. 2 with an exact SVD (the claim of Sec. IV.C and Sec. V that recycling
    does not change the result)."""
    fa = c1_recycle_q
    ex = c1_exact
    assert ex.converged and fa.converged
    assert abs(fa.iters - ex.iters) <= 2
    h = fa.history
    assert not any(x["recycled"] for x in h[:4])
    rec = [x["recycled"] for x in h[4:]]
    assert sum(rec) >= len(rec) // 2  # two recycled calls per fresh basis
    # after each fresh basis, at most q_reuse recycled iterations in a row
    run = best = 0
    for x in rec:
        run = run + 1 if x else 0
        best = max(best, run)
    assert best <= 2
    X = fa.Us @ fa.V.T
    assert np.linalg.norm(X - c1.dense) / np.linalg.norm(c1.dense) < 1e-3
    assert fa.V.shape[1] == ex.V.shape[1] == 10
    Xe = ex.Us @ ex.V.T
    assert np.linalg.norm(X - Xe) / np.linalg.norm(Xe) < 1e-3


def test_alg6_with_rsvd_pi_matches_alg2(c1, c1_exact):
    """Alg. 6 with rSVD-PI (Alg. 4) as the SVD of each call reaches the exact
    SVD's result on the rank-10 case: iteration count within 2, the same
    recovered matrix."""
    fa = svt.svt_fast(c1.m, c1.n, c1.row_ptr, c1.col, c1.val, tau=2500.0, delta=6.0, eps=1e-4, seed=0, recycle=3,
                      inner=1)
    ex = c1_exact
    assert fa.converged and abs(fa.iters - ex.iters) <= 2
    X, Xe = fa.Us @ fa.V.T, ex.Us @ ex.V.T
    assert np.linalg.norm(X - Xe) / np.linalg.norm(Xe) < 1e-3
    assert np.linalg.norm(X - c1.dense) / np.linalg.norm(c1.dense) < 1e-3


def test_p_rule_on_error_sequence():
    """The p rule after Alg. 6 (Sec. IV.C) on a hand-written error sequence:
    +1 on every increase, -1 after ten strict decreases in a row, the streak
    broken by an increase or an unchanged error, p kept in [p_min, p_max]."""
    def run(errs, p=5, p_min=3, p_max=7):
        streak, prev, ps = 0, math.inf, []
        for e in errs:
            p, streak = svt.adapt_p(p, streak, e, prev, p_min, p_max)
            prev = e
            ps.append(p)
        return ps

    dec = [1.0 - 0.01 * j for j in range(31)]  # 31 strict decreases after the first (inf -> 1.0 counts too)
    ps = run(dec)
    # decreases number 10, 20 and 30 (counting the first from inf) lower p by one each, down to p_min = 3
    assert ps[8] == 5 and ps[9] == 4 and ps[18] == 4 and ps[19] == 3 and ps[29] == 3 and ps[30] == 3
    # an increase raises p and restarts the streak
    ps = run([1.0, 0.9, 0.95] + [0.9 - 0.01 * j for j in range(10)])
    assert ps[:3] == [5, 5, 6] and ps[11] == 6 and ps[12] == 5
    # an unchanged error ends the streak without changing p
    head = [1.0] + [0.9 - 0.01 * j for j in range(8)]  # nine strict decreases (from inf)
    ps = run(head + [head[-1]] + [0.8 - 0.01 * j for j in range(9)])
    assert ps == [5] * 19
    ps = run(head + [head[-1]] + [0.8 - 0.01 * j for j in range(10)])
    assert ps[-1] == 4 and ps[:-1] == [5] * 19
    # increases saturate at p_max
    assert run([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])[-1] == 7


def test_svt_fast_follows_p_rule(c1_recycle_q):
    """The p recorded per iteration of Alg. 6 replays the rule from the
    recorded errors, and the trajectory exercises both branches."""
    h = c1_recycle_q.history
    p, streak, prev = h[0]["p"], 0, math.inf
    ups = downs = 0
    for a, b in zip(h[:-1], h[1:]):
        assert a["p"] == p
        p2, streak = svt.adapt_p(p, streak, a["err"], prev, 3, 20)
        ups += p2 > p
        downs += p2 < p
        p, prev = p2, a["err"]
        assert b["p"] == p
    assert ups >= 1 and downs >= 1


def test_stored_image_solve_reproduces():
    """The stored image-inpainting solve (tests/golden/image_svt_oracle.json)
    is the current oracle's: its first iterations replay exactly."""
    import json
    import os

    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "image_svt_oracle.json")) as f:
        ref = json.load(f)
    w = ref["workload"]
    o = mc_synth.smooth_image(w["size"], w["size"], w["rank"], sigma_px=w["sigma_px"], frac=w["frac"],
                              seed=w["seed"])
    kw = dict(ref["params"])
    kw["i_max"] = 4
    res = svt.svt_fast(o.m, o.n, o.row_ptr, o.col, o.val, **kw)
    for a, b in zip(res.history, ref["history"][:4]):
        assert (a["k"], a["r"], a["p"]) == (b["k"], b["r"], b["p"])
        assert a["err"] == pytest.approx(b["err"], rel=1e-12)
    assert ref["converged"] and ref["rank"] == 41 and ref["recovery_rel_err"] < 1e-3
