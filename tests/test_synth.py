"""Input generators: structure of the synthetic workloads."""
import numpy as np

import mc_synth


def _check_csr(o):
    assert o.row_ptr.shape == (o.m + 1,) and o.row_ptr[0] == 0 and o.row_ptr[-1] == o.nnz
    assert o.col.dtype == np.int32 and o.val.dtype == np.float32
    for i in range(o.m):
        c = o.col[o.row_ptr[i]:o.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    assert o.col.min() >= 0 and o.col.max() < o.n


def test_lowrank_uniform():
    o = mc_synth.lowrank_uniform(60, 40, 3, nobs=500, seed=2)
    _check_csr(o)
    assert o.nnz == 500
    assert np.allclose(o.val, o.dense[o.rows, o.col])
    assert np.linalg.matrix_rank(o.dense.astype(np.float64), tol=1e-3) == 3
    o2 = mc_synth.lowrank_uniform(60, 40, 3, nobs=500, seed=2)
    assert np.array_equal(o.col, o2.col) and np.array_equal(o.val, o2.val)


def test_smooth_image():
    o = mc_synth.smooth_image(64, 48, 5, sigma_px=3.0, frac=0.5, seed=1)
    _check_csr(o)
    assert o.dense.min() >= 0 and o.dense.max() <= 255.0 + 1e-3
    assert abs(o.nnz - 0.5 * 64 * 48) <= 1


def test_ratings_structure():
    o = mc_synth.ratings(m=2000, n=500, N=40000, holdout=0.1, seed=0)
    _check_csr(o)
    assert o.nnz == 36000 and o.test_val.size == 4000
    allv = np.concatenate([o.val, o.test_val])
    assert set(np.unique(allv * 2).astype(int)) <= set(range(1, 11))
    tr = set((o.rows * o.n + o.col).tolist())
    te = set((o.test_rows * o.n + o.test_cols).tolist())
    assert not (tr & te)
    deg = np.diff(o.row_ptr)
    assert deg.max() > 20 * np.median(deg)  # heavy-tailed rows


def test_serving_jobs():
    js = mc_synth.serving_jobs(50, seed=3)
    assert all(256 <= j["m"] <= 8192 and 5 <= j["rank"] <= 50 for j in js)
    t = [j["arrival"] for j in js]
    assert np.all(np.diff(t) > 0)
