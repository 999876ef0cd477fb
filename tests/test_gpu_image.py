"""Parity of the image-inpainting solve with the float64 oracle's stored solve
(tests/golden/image_svt_oracle.json, written from the oracle alone by
tests/golden/make_image_svt_oracle.py).

Workload: a 1024 x 1024 image of rank 40 (Gaussian-smoothed factors, 8 px,
min-max scaled to [0, 255]; the offset makes the matrix rank 41), half of the
pixels observed.  The solve is Alg. 6 with the second recycling strategy of
Sec. IV.B (recycled left singular vectors, i_reuse = 100, q_reuse = 10, the
paper's image settings) run to its stopping tolerance, in the plain float32
form and in the mixed form (bf16 panels in the Krylov products).

Plain form: the same k, r and recycled flag at every iteration, the error on
Phi within 1e-4 of the oracle's at every iteration, the same iteration count
+-1, and at the end the relative error against the full image and the RMSE
over the unobserved pixels within 1e-4 (relative) and 1e-3 (pixel units) of
the oracle's.  Mixed form: the same iteration count +-2 and the same two
end-point errors within the same bounds."""
import json
import os

import numpy as np
import pytest

import mc_synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "image_svt_oracle.json")


@pytest.fixture(scope="module")
def mc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_06860_gb300 as mc

    return mc


@pytest.fixture(scope="module")
def stored():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def image(stored):
    w = stored["workload"]
    return mc_synth.smooth_image(w["size"], w["size"], w["rank"], sigma_px=w["sigma_px"], frac=w["frac"],
                                 seed=w["seed"])


def _solve(mc, o, params, precision):
    kw = dict(params)
    i_max = kw.pop("i_max")
    prm = mc.params(**kw, i_max=i_max, precision=precision)
    hist = []
    with mc.Handle.from_observed(o) as h:
        for _ in range(i_max):
            info = h.svt_step(prm)
            hist.append(info)
            if info["converged"]:
                break
        Us, V, _ = h.factors()
    X = Us.astype(np.float64) @ V.astype(np.float64).T
    M = o.dense.astype(np.float64)
    observed = np.zeros(M.shape, bool)
    observed[np.repeat(np.arange(o.m), np.diff(o.row_ptr)), o.col] = True
    rec = float(np.linalg.norm(X - M) / np.linalg.norm(M))
    rmse = float(np.sqrt(np.mean((X - M)[~observed] ** 2)))
    return hist, rec, rmse


def _endpoint(stored, hist, rec, rmse, tol_iters):
    assert stored["converged"] and hist[-1]["converged"]
    assert abs(len(hist) - stored["iterations"]) <= tol_iters
    assert any(b["recycled"] for b in stored["history"])
    assert abs(hist[-1]["err"] - stored["err"]) <= 1e-4
    assert abs(rec - stored["recovery_rel_err"]) <= 1e-4, (rec, stored["recovery_rel_err"])
    assert abs(rmse - stored["unobserved_rmse"]) <= 1e-3, (rmse, stored["unobserved_rmse"])


def test_image_solve_plain_matches_oracle(mc, image, stored):
    hist, rec, rmse = _solve(mc, image, stored["params"], 0)
    n = min(len(hist), len(stored["history"]))
    for a, b in zip(hist[:n], stored["history"][:n]):
        assert (a["k"], a["r"], a["recycled"]) == (b["k"], b["r"], int(b["recycled"])), (a, b)
        assert abs(a["err"] - b["err"]) <= 1e-4 * max(1.0, b["err"]), (a, b)
    _endpoint(stored, hist, rec, rmse, 1)


def test_image_solve_mixed_matches_oracle(mc, image, stored):
    hist, rec, rmse = _solve(mc, image, stored["params"], 1)
    _endpoint(stored, hist, rec, rmse, 2)
