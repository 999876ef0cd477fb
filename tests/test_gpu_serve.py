"""Serving form on the GPU: a job's result is the same alone and in a mix of
concurrent jobs, the same as through a single handle, and matches the oracle
at the plain form's tolerances."""
import math

import numpy as np
import pytest

import mc_synth
from oracle import svt as osvt

pytestmark = pytest.mark.gpu

# (m, n, rank, observed fraction, seed): shapes of different aspect, size and rank
JOBS = [(300, 200, 5, 0.3, 1), (500, 500, 10, 0.2, 2), (800, 400, 8, 0.25, 3), (256, 1000, 6, 0.3, 4),
        (1500, 900, 12, 0.12, 5), (700, 700, 10, 0.2, 6)]


@pytest.fixture(scope="module")
def mc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_06860_gb300 as mc

    return mc


def _prm(mc, o, frac, seed):
    # warm-started Omega (recycle = 3): converges on these jobs in 80-130 iterations
    return mc.params(tau=5.0 * math.sqrt(o.m * o.n), delta=1.2 / frac, eps=1e-4, i_max=500, seed=seed, recycle=3)


def _unobserved_rel_err(o, Us, V):
    X = Us.astype(np.float64) @ V.astype(np.float64).T
    mask = np.ones((o.m, o.n), bool)
    mask[o.rows, o.col] = False
    d = (X - o.dense)[mask]
    return float(np.linalg.norm(d) / np.linalg.norm(o.dense[mask]))


def test_served_result_same_alone_and_in_mix(mc):
    obs = [mc_synth.lowrank_uniform(m, n, r, frac=f, seed=s) for (m, n, r, f, s) in JOBS]
    prms = [_prm(mc, o, f, s) for o, (_, _, _, f, s) in zip(obs, JOBS)]
    alone = []
    with mc.Server(max_active=1) as srv:
        for o, p in zip(obs, prms):
            alone.append(srv.wait(srv.submit_observed(o, p), 900))
    with mc.Server(max_active=len(JOBS)) as srv:
        ids = [srv.submit_observed(o, p) for o, p in zip(obs, prms)]
        mix = [srv.wait(j, 900) for j in ids]
        st = srv.stats()
    assert st["peak_active"] >= 2 and st["completed"] == len(JOBS)
    # the jobs ran at the same time: the last admitted started before the first finished
    assert max(r["queue_s"] for r in mix) < min(r["latency_s"] for r in mix)
    for a, b, o in zip(alone, mix, obs):
        assert a["status"] == 0 and b["status"] == 0, (a["status"], b["status"], a["message"], b["message"])
        assert a["iters"] == b["iters"] and a["r"] == b["r"]
        # every kernel is deterministic: bit-identical factors
        assert np.array_equal(a["Us"], b["Us"]) and np.array_equal(a["V"], b["V"])
        assert np.array_equal(a["sigma"], b["sigma"])
        assert b["device_bytes_peak"] <= b["footprint_bytes"]
        assert _unobserved_rel_err(o, b["Us"], b["V"]) < 5e-3


def test_served_equals_handle_and_oracle(mc):
    o = mc_synth.lowrank_uniform(500, 500, 10, frac=0.2, seed=0)
    prm = mc.params(tau=2500.0, delta=6.0, eps=1e-4, recycle=3, seed=0, i_max=1000)
    with mc.Server(max_active=2) as srv:
        j = srv.submit_observed(o, prm)
        res = srv.wait(j, 900)
    with mc.Handle.from_observed(o) as h:
        info = h.svt_solve(prm)
        Us, V, sg = h.factors()
    assert res["iters"] == info["i"] and res["r"] == Us.shape[1]
    assert np.array_equal(res["Us"], Us) and np.array_equal(res["V"], V) and np.array_equal(res["sigma"], sg)
    ref = osvt.svt_fast(o.m, o.n, o.row_ptr, o.col, o.val, tau=2500.0, delta=6.0, eps=1e-4, recycle=3, seed=0,
                        i_max=1000)
    assert ref.converged and abs(res["iters"] - ref.iters) <= 1
    e_gpu = _unobserved_rel_err(o, res["Us"], res["V"])
    e_ref = _unobserved_rel_err(o, ref.Us.astype(np.float32), ref.V.astype(np.float32))
    assert abs(e_gpu - e_ref) < 1e-3


def test_served_cancel_and_bad_job(mc):
    o = mc_synth.lowrank_uniform(600, 600, 10, frac=0.2, seed=7)
    with mc.Server(max_active=1) as srv:
        a = srv.submit_observed(o, _prm(mc, o, 0.2, 7))
        bad = srv.submit(3, 3, np.array([0, 2, 1, 1], np.int64), np.array([0, 1], np.int32),
                         np.ones(2, np.float32), mc.params())
        b = srv.submit_observed(o, _prm(mc, o, 0.2, 8))
        srv.cancel(b)
        ra, rbad, rb = srv.wait(a, 900), srv.wait(bad, 900), srv.wait(b, 900)
    assert ra["status"] == 0
    assert rbad["status"] == 1  # MC_EINVAL: row_ptr not monotone
    assert rb["status"] == 8 and rb["iters"] == 0
