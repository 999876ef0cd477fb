"""Writes rating_svt_oracle.json: the float64 oracle's fast-SVT trajectory
(Alg. 6) on the rating workload, the reference for the full-size GPU parity
test and for the held-out RMSE the benchmark reports beside its own.

Workload: mc_synth.ratings(138000, 27000, 2e7 pairs, 10% held out, seed 0).
Parameters: tau = 5n (Sec. II.C, n the column count), delta = 1.9, eps =
1e-4 (not reached in this window), l = 5, s = 10, p0 = p_min = 3, p_max = 20,
Omega warm-started with the previous right singular block (recycle = 3),
Philox seed 0.  Per iteration: k, r, p, the error on Phi and the leading and
last singular values; every 5 iterations from 380 the held-out RMSE of X^i.
Calls only mc_synth and oracle/ (about an hour on a few host cores):

    python tests/golden/make_rating_svt_oracle.py [iterations]
"""
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import mc_synth  # noqa: E402
from oracle import svt  # noqa: E402

M_ROWS, N_COLS, N_PAIRS, HOLDOUT, SEED = 138_000, 27_000, 20_000_000, 0.1, 0
PARAMS = dict(tau=5.0 * N_COLS, delta=1.9, eps=1e-4, l=5, s=10, p0=3, p_min=3, p_max=20, recycle=3, seed=SEED)
RMSE_FROM, RMSE_EVERY = 380, 5


def main():
    iters = int(sys.argv[1]) if len(sys.argv) > 1 else 440
    o = mc_synth.ratings(M_ROWS, N_COLS, N_PAIRS, holdout=HOLDOUT, seed=SEED)
    hist, rmse = [], {}
    t0 = time.time()

    def on_factors(rec, Us, V):
        hist.append({k: rec[k] for k in ("i", "k", "r", "p", "err", "nsvd", "sigma_max", "sigma_last", "c", "norm2")})
        i = rec["i"]
        if i >= RMSE_FROM and i % RMSE_EVERY == 0:
            pred = svt.sample_lowrank(o.test_rows, o.test_cols, Us, V)
            rmse[str(i)] = float(np.sqrt(np.mean((pred - o.test_val.astype(np.float64)) ** 2)))
        if i % 10 == 0:
            print(f"i={i} k={rec['k']} r={rec['r']} p={rec['p']} err={rec['err']:.6f} t={time.time() - t0:.0f}s",
                  flush=True)

    res = svt.svt_fast(o.m, o.n, o.row_ptr, o.col, o.val, i_max=iters, on_factors=on_factors, **PARAMS)
    out = {"workload": {"m": M_ROWS, "n": N_COLS, "pairs": N_PAIRS, "holdout": HOLDOUT, "seed": SEED,
                        "generator": "mc_synth.ratings"},
           "params": PARAMS, "iterations": len(hist), "converged": bool(res.converged), "history": hist,
           "heldout_rmse": rmse, "sigma_final": [float(x) for x in res.sigma],
           "seconds": round(time.time() - t0, 1)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rating_svt_oracle.json")
    with open(path + ".tmp", "w") as f:
        json.dump(out, f, indent=0)
    os.replace(path + ".tmp", path)
    print("wrote", path, flush=True)


if __name__ == "__main__":
    main()
