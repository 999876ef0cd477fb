"""The mixed-precision form (bf16 panels in the Krylov products, float32
orthonormalisation and final projection) against the float64 oracle: errors
are stated per result -- singular values, largest principal angle of the
leading subspace, and completion / held-out error of SVT."""
import math

import numpy as np
import pytest

import mc_synth
from oracle import metrics
from oracle import rsvd as orsvd
from oracle import svt as osvt
from oracle.rsvd import as_csr64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_06860_gb300 as mc

    return mc


def test_mixed_rsvd_bki_errors(mc):
    o = mc_synth.ratings(m=4000, n=1200, N=150_000, seed=2)
    A = as_csr64(o.m, o.n, o.row_ptr, o.col, o.val)
    Uo, So, Vo, _ = orsvd.rsvd_bki(A, 20, 3, s=10, seed=11, call_id=4)
    res = {}
    for prec in (0, 1):
        with mc.Handle.from_observed(o) as h:
            h.set_precision(prec)
            U, S, V = h.rsvd_bki(20, s=10, p=3, seed=11, call_id=4)
        gap = np.flatnonzero(np.diff(So) / So[1:] < -0.05)
        j = int(gap[0]) + 1 if gap.size else 1
        res[prec] = (metrics.sigma_rel_err(S, So), metrics.max_principal_angle(V[:, :j], Vo[:, :j]))
    print("sigma rel err / leading angle: plain %.2e / %.2e, mixed %.2e / %.2e" % (*res[0], *res[1]))
    assert res[0][0] < 1e-5
    assert res[1][0] < 1e-3 and res[1][1] < 1e-2


def test_mixed_svt_config1(mc):
    o = mc_synth.lowrank_uniform(500, 500, 10, frac=0.2, seed=0)
    kw = dict(tau=2500.0, delta=6.0, eps=1e-4, recycle=3, seed=0)
    ref = osvt.svt_fast(o.m, o.n, o.row_ptr, o.col, o.val, **kw)
    Xo = ref.Us @ ref.V.T
    unobs = np.ones((500, 500), bool)
    unobs[o.rows, o.col] = False
    scale = float(np.std(o.dense))
    out = {}
    for prec in (0, 1):
        prm = mc.params(**kw, precision=prec)
        with mc.Handle.from_observed(o) as h:
            hist = []
            for _ in range(1000):
                hist.append(h.svt_step(prm))
                if hist[-1]["converged"]:
                    break
            Us, V, sg = h.factors()
        X = Us.astype(np.float64) @ V.astype(np.float64).T
        rmse = float(np.sqrt(np.mean((X - o.dense)[unobs] ** 2))) / scale
        out[prec] = (len(hist), hist[-1]["err"], rmse)
    rmse_o = float(np.sqrt(np.mean((Xo - o.dense)[unobs] ** 2))) / scale
    print("iters/err/held-out relative RMSE: oracle %d/%.2e/%.2e plain %d/%.2e/%.2e mixed %d/%.2e/%.2e"
          % (ref.iters, ref.err, rmse_o, *out[0], *out[1]))
    assert abs(out[0][0] - ref.iters) <= 1
    assert out[1][1] < 1e-4  # converged
    # the stated target of the mixed form: held-out error within 1e-3 of the
    # oracle's; the bf16 panels perturb the Krylov spaces, which costs some
    # iterations (measured: 151 against 128)
    assert abs(out[1][2] - rmse_o) < 1e-3
    assert out[1][0] <= 1.4 * ref.iters
