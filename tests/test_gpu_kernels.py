"""Kernel-level parity of the CUDA library (through the C ABI) against the CPU
oracle and plain float64 references on the same seeded inputs."""
import numpy as np
import pytest
import scipy.sparse as sp

import mc_synth
from oracle.philox import omega as omega_ref
from oracle.philox import philox_words

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_06860_gb300 as mc

    return mc


@pytest.mark.parametrize("n,k,seed,call,col0", [(1, 1, 0, 0, 0), (1000, 13, 5, 3, 0), (4097, 64, (7 << 32) | 9, (3 << 32) | 1, 11)])
def test_omega_words_bit_exact_and_values(mc, n, k, seed, call, col0):
    z, w = mc.omega(n, k, seed, call, col0, words=True)
    x0, x1 = philox_words(n, k, seed, call, col0)
    assert np.array_equal(w[..., 0], x0) and np.array_equal(w[..., 1], x1)
    ref = omega_ref(n, k, seed, call, col0)
    assert np.max(np.abs(z - ref) / (1.0 + np.abs(ref))) < 4e-6


def _spd(K, spectrum, rng):
    Qm, _ = np.linalg.qr(rng.standard_normal((K, K)))
    return (Qm * spectrum) @ Qm.T


@pytest.mark.parametrize("K,kw,kind", [(1, 1, "rand"), (2, 2, "rand"), (8, 5, "rand"), (60, 50, "decay"),
                                        (64, 64, "cluster"), (65, 20, "decay"), (100, 30, "cluster"),
                                        (129, 3, "rating"), (240, 50, "rating"), (252, 60, "zeros"),
                                        (300, 80, "decay"), (400, 100, "decay"), (1024, 40, "decay")])
def test_eig_topk(mc, K, kw, kind):
    rng = np.random.default_rng(K * 7 + kw)
    if kind == "rand":
        B = rng.standard_normal((K, K))
        A = B @ B.T
    elif kind == "decay":
        A = _spd(K, 1e4 * 0.97 ** np.arange(K), rng)
    elif kind == "cluster":
        s = np.repeat([100.0, 50.0, 49.9999, 10.0], K // 4)
        A = _spd(K, s, rng)
    elif kind == "rating":
        s = np.concatenate([[5e5], np.linspace(8000, 6000, 60), np.linspace(6000, 100, K - 61)])
        A = _spd(K, s, rng)
    else:  # zero rows/columns from padding
        A = _spd(K, np.concatenate([np.linspace(1e3, 1, K - 12), np.zeros(12)]), rng)
        P = np.eye(K)[rng.permutation(K)]
        A = P @ A @ P.T
        A[:, :12] = 0
        A[:12, :] = 0
    A = A.astype(np.float32)
    lam, W = mc.eig_sym(A, kw)
    A64 = A.astype(np.float64)
    ref = np.linalg.eigvalsh(A64)[::-1][:kw]
    scale = max(abs(ref[0]), 1e-30)
    assert np.max(np.abs(lam - ref)) <= 2e-5 * scale * max(1.0, np.sqrt(K) / 8)
    W64 = W.astype(np.float64)
    assert np.max(np.abs(W64.T @ W64 - np.eye(kw))) < 1e-4
    res = np.linalg.norm(A64 @ W64 - W64 * lam.astype(np.float64), axis=0)
    assert np.max(res) <= 1e-4 * scale * max(1.0, np.sqrt(K) / 8)


@pytest.mark.parametrize("R,K", [(1, 1), (37, 5), (1000, 60), (5000, 64), (20000, 100), (3000, 256), (1200, 300)])
def test_gram(mc, R, K):
    rng = np.random.default_rng(R + K)
    X = rng.standard_normal((R, K)).astype(np.float32)
    G = mc.gram(X)
    ref = X.astype(np.float64).T @ X.astype(np.float64)
    assert np.max(np.abs(G - ref)) <= 1e-5 * np.max(np.abs(ref)) * max(1, np.sqrt(R / 1000))


def _rand_csr(m, n, density, rng, heavy_row=None, heavy_col=None):
    A = sp.random(m, n, density=density, random_state=np.random.RandomState(rng.integers(1 << 30)), format="lil")
    if heavy_row is not None:
        A[heavy_row, :] = rng.standard_normal(n)
    if heavy_col is not None:
        A[:, heavy_col] = rng.standard_normal((m, 1))
    A = A.tocsr()
    A.sort_indices()
    A.data = rng.standard_normal(A.nnz).astype(np.float32)
    return A


@pytest.mark.parametrize("K", [1, 3, 4, 8, 12, 20, 32, 60, 64, 100, 128, 240, 300, 1024])
def test_spmm_both_ways(mc, K):
    rng = np.random.default_rng(K)
    m, n = 700, 900
    A = _rand_csr(m, n, 0.01, rng, heavy_row=5, heavy_col=17)  # rows/cols longer than one segment
    A[10:20, :] = 0  # empty rows
    A.eliminate_zeros()
    A.sort_indices()
    with mc.Handle(m, n, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float32)) as h:
        X = rng.standard_normal((n, K)).astype(np.float32)
        Xt = rng.standard_normal((m, K)).astype(np.float32)
        A64 = A.astype(np.float64)
        Y1 = h.spmm(X)
        Y2 = h.spmm(Xt, trans=True)
        r1 = A64 @ X.astype(np.float64)
        r2 = A64.T @ Xt.astype(np.float64)
        assert np.max(np.abs(Y1 - r1)) < 1e-4 * max(1, np.abs(r1).max())
        assert np.max(np.abs(Y2 - r2)) < 1e-4 * max(1, np.abs(r2).max())
        # deterministic
        assert np.array_equal(Y1, h.spmm(X))


def test_create_rejects_bad_input(mc):
    rp = np.array([0, 2, 3], np.int64)
    with pytest.raises(mc.McError) as e:
        mc.Handle(2, 4, rp, np.array([1, 1, 0], np.int32), np.ones(3, np.float32))
    assert e.value.status == 1
    with pytest.raises(mc.McError):
        mc.Handle(2, 4, rp, np.array([0, 5, 0], np.int32), np.ones(3, np.float32))
    with pytest.raises(mc.McError):
        mc.Handle(2, 4, rp, np.array([0, 1, 0], np.int32), np.array([1, np.nan, 1], np.float32))
    with pytest.raises(mc.McError):
        mc.Handle(2, 4, np.array([0, 3, 2], np.int64), np.array([0, 1, 0], np.int32), np.ones(3, np.float32))
    with pytest.raises(mc.McError):
        mc.Handle(0, 4, np.array([0], np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))


def test_csc_copy_matches_transpose(mc):
    o = mc_synth.ratings(m=3000, n=800, N=60000, seed=1)
    with mc.Handle.from_observed(o) as h:
        rng = np.random.default_rng(0)
        Xt = rng.standard_normal((o.m, 8)).astype(np.float32)
        A = sp.csr_matrix((o.val.astype(np.float64), o.col, o.row_ptr), shape=(o.m, o.n))
        got = h.spmm(Xt, trans=True)
        assert np.max(np.abs(got - A.T @ Xt.astype(np.float64))) < 1e-4 * np.abs(got).max()


@pytest.mark.parametrize("R,K", [(1, 32), (37, 60), (1000, 64), (5000, 100), (3000, 128), (2000, 129),
                                 (20000, 200), (138000, 240), (777, 256)])
def test_gram_tensor_cores(mc, R, K):
    rng = np.random.default_rng(R * 3 + K)
    X = rng.standard_normal((R, K)).astype(np.float32)
    X[:, ::7] *= 30.0  # uneven column scales
    G = mc.gram(X, tensor_cores=True)
    ref = X.astype(np.float64).T @ X.astype(np.float64)
    # three TF32 products: about float32 accuracy relative to the entries' scale
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.max(np.abs(G - ref) / scale) < 2e-5


def test_eig_rank_deficient_krylov_gram(mc):
    """Gram of a Krylov basis whose later blocks lost their leading columns
    (they repeat a converged invariant subspace): 90 of 176 rows are exactly
    zero and the trailing block of the reduction is pure rounding residue.
    Reflecting that residue divides by a denormal; the solver must skip it."""
    rng = np.random.default_rng(31)
    K, kw, n = 176, 31, 2658
    live = np.ones(K, bool)
    for b in range(1, 4):
        live[b * 44: b * 44 + 30] = False
    nl = int(live.sum())
    s = np.concatenate([27300 - 40 * np.arange(30), 5200 - 10 * np.arange(nl - 30)])
    U, _ = np.linalg.qr(rng.standard_normal((n, nl)))
    Vq, _ = np.linalg.qr(rng.standard_normal((nl, nl)))
    B = np.zeros((n, K))
    B[:, live] = (U * s) @ Vq.T
    B = B.astype(np.float32).astype(np.float64)
    G = (B.T @ B).astype(np.float32)
    lam, W = mc.eig_sym(G, kw)
    G64 = G.astype(np.float64)
    ref = np.linalg.eigvalsh(G64)[::-1][:kw]
    assert np.all(np.isfinite(lam)) and np.all(np.isfinite(W))
    assert np.max(np.abs(np.sqrt(lam) - np.sqrt(ref))) <= 1e-5 * np.sqrt(ref[0])
    W64 = W.astype(np.float64)
    assert np.max(np.abs(W64.T @ W64 - np.eye(kw))) < 1e-4
    assert np.max(np.linalg.norm(G64 @ W64 - W64 * lam.astype(np.float64), axis=0)) <= 1e-4 * ref[0]


_SHAPE_PROBE = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import mc_synth, paper_1810_06860_gb300 as mc
o = mc_synth.ratings(m=4000, n=1500, N=150000, seed=2)
rng = np.random.default_rng(0)
out = []
with mc.Handle.from_observed(o) as h:
    for K in (4, 12, 60, 200):
        out.append(h.spmm(rng.standard_normal((o.n, K)).astype(np.float32)))
        out.append(h.spmm(rng.standard_normal((o.m, K)).astype(np.float32), trans=True))
np.savez({path!r}, *out)
"""


def test_spmm_launch_shapes_bit_identical(mc, tmp_path):
    """Every SpMM launch shape the autotuner may pick (gathers in flight, CTA
    size, column chunk) gives the same bits."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = []
    for force in ("1,128,128", "4,256,32", "2,256,64", "1,128,16"):
        path = str(tmp_path / f"s{len(res)}.npz")
        env = dict(os.environ, MC_SPMM_FORCE=force)
        subprocess.run([sys.executable, "-c", _SHAPE_PROBE.format(root=root, path=path)], env=env, check=True,
                       timeout=600)
        z = np.load(path)
        res.append([z[f"arr_{i}"] for i in range(len(z.files))])
    for other in res[1:]:
        for a, b in zip(res[0], other):
            assert np.array_equal(a, b)


_PDL_PROBE = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import mc_synth, paper_1810_06860_gb300 as mc
o = mc_synth.ratings(m=6000, n=2000, N=240000, seed=5)
prm = mc.params(tau=5.0 * np.sqrt(o.m * o.n), delta=1.9, eps=1e-6, recycle=3, seed=1)
out = []
with mc.Handle.from_observed(o) as h:
    for _ in range(6):
        h.svt_step(prm)
    out.append(h.get_values())
    s, U, V = h.rsvd_bki(50, s=10, p=3, seed=3)
    out += [s, U, V]
np.savez({path!r}, *out)
"""


def test_dependent_launches_bit_identical(mc, tmp_path):
    """Programmatic dependent launches (each kernel waits for its predecessor
    in griddepcontrol.wait) give the same bits as ordinary launches: six SVT
    iterations and an rSVD-BKI at k = 50 (60-column blocks through the
    tensor-core Gram and product, the blocked Cholesky, the SpMM and the
    eigensolver chain), run with MC_PDL unset and with MC_PDL=0."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = []
    for flag in (None, "0"):
        path = str(tmp_path / f"p{len(res)}.npz")
        env = dict(os.environ)
        env.pop("MC_PDL", None)
        if flag is not None:
            env["MC_PDL"] = flag
        subprocess.run([sys.executable, "-c", _PDL_PROBE.format(root=root, path=path)], env=env, check=True,
                       timeout=600)
        z = np.load(path)
        res.append([z[f"arr_{i}"] for i in range(len(z.files))])
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


def test_coo_ingest_matches_csr(mc):
    """Coordinates in a shuffled order give the same iterate, bit for bit, as
    the CSR ingest; a repeated pair and an index out of range are refused."""
    o = mc_synth.ratings(m=3000, n=900, N=80000, seed=4)
    rng = np.random.default_rng(1)
    order = rng.permutation(o.nnz)
    rows = o.rows[order]
    cols = o.col[order]
    vals = o.val[order]
    with mc.Handle.from_observed(o) as h1, mc.Handle.from_coo(o.m, o.n, rows, cols, vals) as h2:
        assert np.array_equal(h1.get_values(), h2.get_values())
        X = rng.standard_normal((o.n, 12)).astype(np.float32)
        Xt = rng.standard_normal((o.m, 12)).astype(np.float32)
        assert np.array_equal(h1.spmm(X), h2.spmm(X))
        assert np.array_equal(h1.spmm(Xt, trans=True), h2.spmm(Xt, trans=True))
    with pytest.raises(mc.McError) as e:
        mc.Handle.from_coo(4, 4, np.array([0, 1, 1], np.int64), np.array([2, 3, 3], np.int32), np.ones(3, np.float32))
    assert e.value.status == 1
    with pytest.raises(mc.McError):
        mc.Handle.from_coo(4, 4, np.array([0, 4], np.int64), np.array([2, 3], np.int32), np.ones(2, np.float32))
    empty = mc.Handle.from_coo(5, 3, np.zeros(0, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    empty.close()


@pytest.mark.parametrize("R,K,N", [(138_000, 60, 60), (27_000, 240, 52), (50_001, 180, 60), (300, 7, 13),
                                   (129, 32, 16), (5_000, 256, 64), (1_000, 64, 256), (777, 40, 33)])
def test_panel_gemm_tensor_cores(mc, R, K, N):
    """Z = X W on the tensor cores (3xTF32) against a float64 product: every
    entry within 1e-5 of max |X| |W| (the bound of a float32 sum over K terms
    with the TF32 split's error of about 2^-22 per product), and against the
    SIMT kernels.  Ragged R (not a multiple of the 128-row tile), K and N (not
    multiples of the 32-column box or 16-column MMA) are covered; at 777 x 33
    the last 32-row output block starts past R (no store issued) and the
    second 32-column store box holds one column."""
    rng = np.random.default_rng(R + K + N)
    X = rng.standard_normal((R, K)).astype(np.float32)
    W = (rng.standard_normal((K, N)) / np.sqrt(K)).astype(np.float32)
    Z = mc.panel_gemm(X, W, tensor_cores=True)
    ref = X.astype(np.float64) @ W.astype(np.float64)
    bound = np.abs(X).astype(np.float64) @ np.abs(W).astype(np.float64)
    assert np.all(np.abs(Z - ref) <= 1e-5 * bound.max())
    Zs = mc.panel_gemm(X, W, tensor_cores=False)
    assert np.max(np.abs(Z - Zs)) <= 2e-5 * bound.max()


def test_panel_gemm_tensor_cores_rejects_wide(mc):
    X = np.zeros((10, 256), np.float32)
    W = np.zeros((256, 128), np.float32)  # 256 x 128 > 16384
    with pytest.raises(mc.McError):
        mc.panel_gemm(X, W, tensor_cores=True)


def test_gather_rate_probe(mc):
    """mc_gather_rate runs the products' gathers alone and reports a positive
    rate for both index streams; bad arguments are rejected."""
    o = mc_synth.ratings(m=4000, n=1500, N=150000, seed=2)
    with mc.Handle.from_observed(o) as h:
        for trans in (False, True):
            g = h.gather_rate(60, trans=trans, reps=3)
            assert np.isfinite(g) and g > 0
        with pytest.raises(mc.McError):
            h.gather_rate(256)


@pytest.mark.parametrize("R,K1,K2,same", [(138_000, 60, 60, True), (138_000, 180, 60, False), (27_000, 240, 240, True),
                                          (1_000, 17, 33, False), (300, 256, 32, False), (129, 64, 20, False)])
def test_panel_gram_tensor_cores(mc, R, K1, K2, same):
    """C = X1^T X2 on the tensor cores (3xTF32) against float64 and against the
    SIMT kernels: every entry within 1e-5 of max |X1|^T |X2|, scaled by
    sqrt(R / 1000) for the float32 sums over R rows (the Gram tests' bound);
    ragged R (not a multiple of the 32-row stage), K1 and K2 (not multiples of
    the 32-column box) are covered."""
    rng = np.random.default_rng(R + K1 + K2)
    X1 = rng.standard_normal((R, K1)).astype(np.float32)
    X2 = X1 if same else rng.standard_normal((R, K2)).astype(np.float32)
    Ct = mc.panel_gram(X1, X2, tensor_cores=True)
    ref = X1.astype(np.float64).T @ X2.astype(np.float64)
    bound = (np.abs(X1).astype(np.float64).T @ np.abs(X2).astype(np.float64)).max()
    tol = 1e-5 * bound * max(1.0, np.sqrt(R / 1000))
    assert np.max(np.abs(Ct - ref)) <= tol
    Cs = mc.panel_gram(X1, X2, tensor_cores=False)
    assert np.max(np.abs(Ct - Cs)) <= 2 * tol


def test_panel_gram_tensor_cores_rejects_two_wide_panels(mc):
    """Two different 256-column panels need more shared memory per stage than
    the kernel's two-stage minimum: rejected with nothing run (the library's
    products fall back to SIMT for them)."""
    X = np.zeros((10, 256), np.float32)
    Y = np.zeros((10, 256), np.float32)
    with pytest.raises(mc.McError):
        mc.panel_gram(X, Y, tensor_cores=True)
