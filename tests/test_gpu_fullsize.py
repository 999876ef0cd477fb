"""Parity at the full rating workload the bench times: 138,000 x 27,000 with
2e7 pairs (10 % held out for the SVT, 1.8e7 observed), against the oracle
on the same inputs.  About a minute of oracle work on the host, plus the
oracle's stored trajectory of the benchmark's SVT run
(tests/golden/rating_svt_oracle.json, written from the oracle alone by
tests/golden/make_rating_svt_oracle.py)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import mc_synth
from oracle import rsvd as orsvd
from oracle import svt as osvt
from oracle.philox import omega

pytestmark = pytest.mark.gpu

M, N, PAIRS = 138_000, 27_000, 20_000_000


@pytest.fixture(scope="module")
def mc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_06860_gb300 as mc

    return mc


@pytest.fixture(scope="module")
def rating():
    return mc_synth.ratings(M, N, PAIRS, holdout=0.1, seed=0)


def test_rsvd_bki_full_size(mc, rating):
    """rSVD-BKI at k = 50, s = 10, p = 3 on all 2e7 pairs (the bench's rSVD
    leg): the top 50 singular values within 1e-5 of the oracle's on the same
    Omega, the leading singular vectors equal up to sign."""
    o = rating
    rows = np.concatenate([o.rows, o.test_rows])
    cols = np.concatenate([o.col.astype(np.int64), o.test_cols])
    vals = np.concatenate([o.val, o.test_val])
    A = sp.csr_matrix((vals.astype(np.float64), (rows, cols)), shape=(M, N))
    A.sort_indices()
    k, s, p, seed, call = 50, 10, 3, 11, 4
    with mc.Handle(M, N, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float32)) as h:
        U, S, V = h.rsvd_bki(k, s=s, p=p, seed=seed, call_id=call)
    Uo, So, Vo, _ = orsvd.rsvd_bki(A, k, p, s, Om=omega(N, k + s, seed, call))
    assert np.max(np.abs(S.astype(np.float64) - So) / So) < 1e-5
    for j in range(3):  # well separated at the top (7105, 4465, 2476)
        assert abs(abs(np.dot(U[:, j].astype(np.float64), Uo[:, j])) - 1.0) < 1e-5
        assert abs(abs(np.dot(V[:, j].astype(np.float64), Vo[:, j])) - 1.0) < 1e-5
    G = U.astype(np.float64).T @ U.astype(np.float64)
    assert np.max(np.abs(G - np.eye(k))) < 1e-4


def test_svt_first_iterations_full_size(mc, rating):
    """The first SVT iterations with the bench's parameters on the 1.8e7
    observed entries: the same c, k and r as the oracle, the error on the
    observed set within 1e-4 (relative) of the oracle's."""
    o = rating
    kw = dict(tau=5.0 * math.sqrt(M * N), delta=1.9, eps=1e-4, recycle=1, i_reuse=50, q_reuse=10, seed=0)
    ref = osvt.svt_fast(o.m, o.n, o.row_ptr, o.col, o.val, i_max=3, **kw)
    assert all(b["tau_margin"] > 1e-3 for b in ref.history)
    with mc.Handle.from_observed(o) as h:
        prm = mc.params(**kw)
        hist = [h.svt_step(prm) for _ in range(3)]
    assert hist[0]["c"] == ref.history[0]["c"]
    for a, b in zip(hist, ref.history):
        assert a["r"] == b["r"] and a["k"] == b["k"], (a, b)
        assert abs(a["err"] - b["err"]) <= 1e-4 * b["err"], (a, b)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rating_svt_oracle.json")


@pytest.fixture(scope="module")
def stored():
    with open(GOLDEN) as f:
        return json.load(f)


def _heldout_rmse(h, o):
    pred = h.sample(o.test_rows, o.test_cols).astype(np.float64)
    return float(np.sqrt(np.mean((pred - o.test_val.astype(np.float64)) ** 2)))


def test_svt_window_matches_stored_oracle(mc, rating, stored):
    """The benchmark's SVT run (tau = 5n, delta = 1.9, warm-started Omega)
    through every iteration the oracle stored (past the timed window, where
    the rank is about 50): the same k, r and p at every iteration, the error
    on Phi within 1e-4 (relative) of the oracle's, and the held-out RMSE of
    X^i within 1e-3 of the oracle's wherever it was stored."""
    o = rating
    ref = stored["history"]
    rmse = {int(k): v for k, v in stored["heldout_rmse"].items()}
    assert ref[-1]["r"] >= 40 and rmse
    prm = mc.params(**stored["params"])
    worst = worst_err = 0.0
    with mc.Handle.from_observed(o) as h:
        for b in ref:
            a = h.svt_step(prm)
            assert a["i"] == b["i"]
            assert (a["k"], a["r"], a["p"]) == (b["k"], b["r"], b["p"]), (a, b)
            worst_err = max(worst_err, abs(a["err"] - b["err"]) / b["err"])
            assert abs(a["err"] - b["err"]) <= 1e-4 * b["err"], (a, b)
            if b["i"] == 1:
                assert a["c"] == b["c"]
            if b["i"] in rmse:
                d = abs(_heldout_rmse(h, o) - rmse[b["i"]])
                worst = max(worst, d)
                assert d <= 1e-3, (b["i"], d)
    print(f"largest held-out RMSE difference from the oracle: {worst:.2e}; "
          f"largest relative error difference on Phi: {worst_err:.2e}")


def test_svt_window_mixed_form_heldout_rmse(mc, rating, stored):
    """The mixed-precision form (bf16 panels in the Krylov products) on the
    same run: held-out RMSE within 1e-3 of the float64 oracle's at the last
    stored iteration."""
    o = rating
    rmse = {int(k): v for k, v in stored["heldout_rmse"].items()}
    last = max(rmse)
    prm = mc.params(**stored["params"], precision=1)
    with mc.Handle.from_observed(o) as h:
        for _ in range(last):
            info = h.svt_step(prm)
        assert info["i"] == last
        d = abs(_heldout_rmse(h, o) - rmse[last])
    assert d <= 1e-3, d
