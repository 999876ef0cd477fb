"""Writes image_svt_oracle.json: the float64 oracle's fast-SVT solve (Alg. 6,
strategy 2: recycled left singular vectors, Sec. IV.B) of the image-inpainting
workload, the reference for the GPU parity test of that solve.

Workload: mc_synth.smooth_image(1024, 1024, rank 40, sigma 8 px, 50 % of the
pixels observed, seed 0).  Parameters: tau = 25 sqrt(mn) = 25,600, delta =
1.2 / 0.5 = 2.4, eps = 7e-4, l = 5, s = 10, p0 = p_min = 3, p_max = 20,
recycle = 2 with i_reuse = 100 and q_reuse = 10 (the paper's image
settings), Philox seed 0.  Recorded: per iteration k, r, p, the error on Phi,
the SVD calls and whether one was recycled; at the end the iteration count,
the relative error of X against the full image and the RMSE over the
unobserved pixels.  Calls only mc_synth and oracle/ (a few minutes):

    python tests/golden/make_image_svt_oracle.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import mc_synth  # noqa: E402
from oracle import svt  # noqa: E402

SIZE, RANK, SIGMA_PX, FRAC, SEED = 1024, 40, 8.0, 0.5, 0
PARAMS = dict(tau=25.0 * SIZE, delta=1.2 / FRAC, eps=7e-4, l=5, s=10, p0=3, p_min=3, p_max=20, recycle=2,
              i_reuse=100, q_reuse=10, seed=SEED, i_max=300)


def main():
    o = mc_synth.smooth_image(SIZE, SIZE, RANK, sigma_px=SIGMA_PX, frac=FRAC, seed=SEED)
    t0 = time.time()
    hist = []
    res = svt.svt_fast(o.m, o.n, o.row_ptr, o.col, o.val,
                       callback=lambda r: hist.append({k: r[k] for k in ("i", "k", "r", "p", "err", "nsvd",
                                                                         "recycled", "sigma_max", "sigma_last", "c")}),
                       **PARAMS)
    X = res.Us @ res.V.T
    M = o.dense.astype(np.float64)
    observed = np.zeros(M.shape, bool)
    observed[np.repeat(np.arange(o.m), np.diff(o.row_ptr)), o.col] = True
    out = {"workload": {"size": SIZE, "rank": RANK, "sigma_px": SIGMA_PX, "frac": FRAC, "seed": SEED,
                        "generator": "mc_synth.smooth_image"},
           "params": PARAMS, "iterations": int(res.iters), "converged": bool(res.converged), "err": float(res.err),
           "rank": int(res.V.shape[1]), "history": hist,
           "recovery_rel_err": float(np.linalg.norm(X - M) / np.linalg.norm(M)),
           "unobserved_rmse": float(np.sqrt(np.mean((X - M)[~observed] ** 2))),
           "sigma_final": [float(x) for x in res.sigma], "seconds": round(time.time() - t0, 1)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "image_svt_oracle.json")
    with open(path + ".tmp", "w") as f:
        json.dump(out, f, indent=0)
    os.replace(path + ".tmp", path)
    print("wrote", path, out["iterations"], out["converged"], out["recovery_rel_err"], out["unobserved_rmse"],
          flush=True)


if __name__ == "__main__":
    main()
