"""mc_gram_noalloc: the Gram entry point that allocates no device memory.

It serves callers that cannot allocate while they call the library (inside a
CUDA stream capture, in host callbacks or allocator hooks, or in hosts whose
device memory all belongs to their own pool).  Its output must agree with the
allocating entry point mc_gram and with a float64 X^T X, over two calls in a
row that share the library's fixed scratch array.  This file sorts last so
that a run stopping at the first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_06860_gb300 as mc

    return mc


def _noalloc(lib, X, G, stream, K=None, ld=None):
    R = X.shape[0]
    K = X.shape[1] if K is None else K
    ld = X.shape[1] if ld is None else ld
    return lib.mc_gram_noalloc(R, K, ctypes.c_void_p(X.data_ptr()), ld, ctypes.c_void_p(G.data_ptr()), K,
                               ctypes.c_void_p(stream.cuda_stream))


def _tol(R, ref):
    # the allocating Gram's own parity tolerance: float32 sums over R rows
    return 1e-5 * np.max(np.abs(ref)) * max(1.0, np.sqrt(R / 1000))


def test_gram_noalloc_matches_gram_twice(mc):
    import torch

    lib = mc.load()
    stream = torch.cuda.Stream()
    # two calls in a row: different shapes, same shared scratch
    for R, K, seed in ((60_000, 60, 0), (20_000, 256, 1)):
        g = torch.Generator(device="cpu").manual_seed(seed)
        Xh = torch.randn(R, K, generator=g, dtype=torch.float32)
        X = Xh.cuda()
        G = torch.full((K, K), float("nan"), device="cuda")
        torch.cuda.synchronize()
        assert _noalloc(lib, X, G, stream) == 0, lib.mc_last_error()
        stream.synchronize()
        got = G.cpu().numpy()
        ref = mc.gram(Xh.numpy())  # the allocating entry point
        x64 = Xh.numpy().astype(np.float64)
        exact = x64.T @ x64
        assert np.max(np.abs(got - ref)) <= _tol(R, ref)
        assert np.max(np.abs(got - exact)) <= _tol(R, exact)
        assert np.array_equal(got, got.T)


def test_gram_noalloc_ignores_padding_columns(mc):
    """K = 62 columns inside rows of 64: the two padding columns hold NaN and
    must not reach G (the kernel reads whole float4 groups of a row)."""
    import torch

    lib = mc.load()
    stream = torch.cuda.Stream()
    R, K, ld = 30_000, 62, 64
    g = torch.Generator(device="cpu").manual_seed(5)
    Xh = torch.randn(R, ld, generator=g, dtype=torch.float32)
    Xh[:, K:] = float("nan")
    X = Xh.cuda()
    G = torch.zeros((K, K), device="cuda")
    torch.cuda.synchronize()
    for _ in range(2):
        assert _noalloc(lib, X, G, stream, K=K, ld=ld) == 0, lib.mc_last_error()
        stream.synchronize()
        got = G.cpu().numpy()
        assert np.all(np.isfinite(got))
        x64 = Xh[:, :K].numpy().astype(np.float64)
        exact = x64.T @ x64
        assert np.max(np.abs(got - exact)) <= _tol(R, exact)


def test_gram_noalloc_rejects_oversized_and_bad_args(mc):
    import torch

    lib = mc.load()
    X = torch.zeros(8, 1028, device="cuda")
    G = torch.zeros(1028, 1028, device="cuda")
    st = lib.mc_gram_noalloc(8, 1028, ctypes.c_void_p(X.data_ptr()), 1028, ctypes.c_void_p(G.data_ptr()), 1028, None)
    assert st == 1 and b"1024" in lib.mc_last_error()
    st = lib.mc_gram_noalloc(8, 6, ctypes.c_void_p(X.data_ptr()), 6, ctypes.c_void_p(G.data_ptr()), 6, None)
    assert st == 1
    # a base address one float past an aligned one is rejected on the host
    st = lib.mc_gram_noalloc(8, 4, ctypes.c_void_p(X.data_ptr() + 4), 1028, ctypes.c_void_p(G.data_ptr()), 4, None)
    assert st == 1 and b"aligned" in lib.mc_last_error()
    # host memory is rejected on the host
    Xh = np.zeros((8, 4), np.float32)
    st = lib.mc_gram_noalloc(8, 4, Xh.ctypes.data_as(ctypes.c_void_p), 4, ctypes.c_void_p(G.data_ptr()), 4, None)
    assert st == 1 and b"device" in lib.mc_last_error()
    torch.cuda.synchronize()
