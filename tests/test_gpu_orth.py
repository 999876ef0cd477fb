"""Block orthonormalisation of the Krylov basis (mc_orth_block: the orth() of
Alg. 5 one block at a time) against a float64 Householder QR of the same
projected block."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_06860_gb300 as mc

    return mc


def _basis(R, cols, rng):
    if cols == 0:
        return np.zeros((R, 0), np.float32)
    q, _ = np.linalg.qr(rng.standard_normal((R, cols)))
    return q.astype(np.float32)


def _reference(X, Qp, keep):
    """float64: X projected against Qp twice, then QR with a positive
    diagonal of the kept columns; dropped columns are zero."""
    Y = X.astype(np.float64)
    Q64 = Qp.astype(np.float64)
    for _ in range(2):
        Y = Y - Q64 @ (Q64.T @ Y)
    q, r = np.linalg.qr(Y[:, keep])
    q = q * np.sign(np.diag(r))
    out = np.zeros_like(Y)
    out[:, keep] = q
    return out


def _run(mc, X, Qp):
    Xd = torch.from_numpy(X.copy()).cuda()
    Qd = torch.from_numpy(Qp.copy()).cuda() if Qp.shape[1] else None
    out = mc.orth_block(Xd, Qd)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _check(got, want, Qp, keep, drop):
    K = got.shape[1]
    assert np.all(got[:, drop] == 0.0)
    g = got[:, keep].astype(np.float64)
    assert np.linalg.norm(g - want[:, keep]) / np.sqrt(len(keep)) < 2e-5
    assert np.max(np.abs(g.T @ g - np.eye(len(keep)))) < 2e-5
    if Qp.shape[1]:
        assert np.max(np.abs(Qp.astype(np.float64).T @ g)) < 2e-5
    assert got.shape[1] == K


# (R, K, cols, padding columns): narrow blocks take the one-launch path
# (K <= 32), K = 60 the separate kernels; 1001 and 7 rows leave ragged CTAs;
# at 138,000 x 16 / 48 and 138,000 x 32 / 96 the earlier columns do not fit
# the CTAs' shared memory and are read from global memory
@pytest.mark.parametrize("R,K,cols,pad", [(7, 4, 0, 0), (1001, 12, 0, 2), (1001, 12, 36, 0), (138000, 12, 36, 2),
                                          (50000, 32, 96, 0), (138000, 16, 48, 2), (138000, 32, 96, 0),
                                          (20000, 60, 120, 3), (20000, 60, 0, 0)])
def test_orth_block_matches_qr(mc, R, K, cols, pad):
    rng = np.random.default_rng(R + K + cols)
    Qp = _basis(R, cols, rng)
    X = rng.standard_normal((R, K)).astype(np.float32)
    if pad:
        X[:, K - pad:] = 0.0  # zero columns padding a block to a multiple of 4
    keep = list(range(K - pad))
    want = _reference(X, Qp, keep)
    got = _run(mc, X, Qp)
    _check(got, want, Qp, keep, list(range(K - pad, K)))


@pytest.mark.parametrize("R,K,cols", [(5000, 12, 24), (20000, 60, 120)])
def test_orth_block_drops_dependent_column(mc, R, K, cols):
    """A column inside span(Qp) keeps ~1e-7 of its norm through the
    projection, far below the 1e-10 (squared) dependence threshold: it comes
    out as a zero column and the others as the QR of the remaining ones."""
    rng = np.random.default_rng(3)
    Qp = _basis(R, cols, rng)
    X = rng.standard_normal((R, K)).astype(np.float32)
    X[:, 3] = Qp @ rng.standard_normal(cols).astype(np.float32)
    keep = [j for j in range(K) if j != 3]
    want = _reference(X, Qp, keep)
    got = _run(mc, X, Qp)
    _check(got, want, Qp, keep, [3])


def test_orth_block_rejects_bad_shapes(mc):
    X = torch.zeros((100, 6), device="cuda")
    with pytest.raises(mc.McError) as e:
        mc.orth_block(X)
    assert e.value.status == 1
    X = torch.zeros((100, 8), device="cuda")
    Q = torch.zeros((100, 6), device="cuda")
    with pytest.raises(mc.McError):
        mc.orth_block(X, Q)


@pytest.mark.skipif(__import__("os").environ.get("MC_ORTH_FUSED") == "0", reason="already the separate kernels")
def test_orth_block_separate_kernels(mc):
    """The same cases with the one-launch path switched off (MC_ORTH_FUSED=0):
    narrow blocks then go through the separate Gram, Cholesky and panel
    product kernels (the narrow-output panel product with beta = 1 in the
    projection)."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MC_ORTH_FUSED="0")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(root, "tests", "test_gpu_orth.py"), "-q", "-x",
                        "-p", "no:cacheprovider", "-k", "matches_qr or dependent"], env=env, cwd=root,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
