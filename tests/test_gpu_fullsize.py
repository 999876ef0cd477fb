"""Parity at the full rating workload the bench times: 138,000 x 27,000 with
2e7 pairs (10 % held out for the SVT, 1.8e7 observed), against the oracle
on the same inputs.  About a minute of oracle work on the host."""
import math

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
