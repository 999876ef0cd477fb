"""Failure paths of the C ABI, injected on the host: an allocator hook that
refuses the n-th device allocation.  Every call must return MC_ENOMEM (no
exception, no crash), and every allocation the library obtained before the
failure must be returned to the hook once the handle is destroyed (or, for a
failed mc_create, before it returns).  No GPU fault is involved: the hook
simply returns NULL."""
import ctypes as C
import math

import numpy as np
import pytest

import mc_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_06860_gb300 as mc

    return mc


class FailingAllocator:
    """Counts allocations through torch's caching allocator and returns NULL
    for the fail_at-th one (1-based; 0 never fails)."""

    def __init__(self, fail_at: int):
        import torch

        from paper_1810_06860_gb300 import _native

        self.torch = torch
        self.fail_at = fail_at
        self.count = 0
        self.live = {}
        self.alloc_cb = _native.ALLOC_FN(self._alloc)
        self.free_cb = _native.FREE_FN(self._free)
        self.struct = _native.McAllocator(None, self.alloc_cb, self.free_cb)

    def _alloc(self, ctx, nbytes, stream):
        self.count += 1
        if self.count == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        self.live[int(p)] = int(nbytes)
        return p

    def _free(self, ctx, ptr, nbytes, stream):
        assert int(ptr) in self.live, "free of a pointer the hook did not hand out"
        del self.live[int(ptr)]
        self.torch.cuda.caching_allocator_delete(int(ptr))


def _sequence(mc, lib, obs, alloc):
    """mc_create, two SVT steps and one rSVD-BKI through the allocator hook.
    Returns (status of the first failing call or 0, handle or None)."""
    rp = np.ascontiguousarray(obs.row_ptr, np.int64)
    ci = np.ascontiguousarray(obs.col, np.int32)
    va = np.ascontiguousarray(obs.val, np.float32)
    h = C.c_void_p()
    st = lib.mc_create(C.byref(h), obs.m, obs.n, obs.nnz, rp.ctypes.data_as(C.c_void_p),
                       ci.ctypes.data_as(C.c_void_p), va.ctypes.data_as(C.c_void_p), None, C.byref(alloc.struct))
    if st != 0:
        assert not h.value, "a failed mc_create must not return a handle"
        return st, None
    prm = mc.params(tau=5 * math.sqrt(obs.m * obs.n), delta=1.2 / 0.3, eps=1e-4, recycle=1, i_reuse=2, q_reuse=1,
                    seed=0)
    info = mc._native.McIterInfo()
    for _ in range(3):
        st = lib.mc_svt_step(h, C.byref(prm), C.byref(info))
        if st != 0:
            return st, h
    U = np.zeros((obs.m, 12), np.float32)
    S = np.zeros(12, np.float32)
    V = np.zeros((obs.n, 12), np.float32)
    kout = C.c_int(0)
    st = lib.mc_rsvd_bki(h, 12, 10, 2, 0, 5, U.ctypes.data_as(C.c_void_p), S.ctypes.data_as(C.c_void_p),
                         V.ctypes.data_as(C.c_void_p), C.byref(kout))
    return st, h


def test_allocation_failure_at_every_point_returns_enomem_without_leak(mc):
    import torch

    lib = mc.load()
    obs = mc_synth.lowrank_uniform(300, 200, 6, frac=0.3, seed=2)
    ok = FailingAllocator(0)
    st, h = _sequence(mc, lib, obs, ok)
    assert st == 0, lib.mc_last_error()
    total = ok.count
    lib.mc_destroy(h)
    torch.cuda.synchronize()
    assert not ok.live
    assert total >= 10
    for n in range(1, total + 1):
        a = FailingAllocator(n)
        st, h = _sequence(mc, lib, obs, a)
        assert st == 2, (n, st, lib.mc_last_error())  # MC_ENOMEM
        assert b"NULL" in lib.mc_last_error()
        if h is not None:
            lib.mc_destroy(h)
        torch.cuda.synchronize()
        assert not a.live, f"allocation {n} failed: {len(a.live)} buffers not returned"
    # the library is still usable afterwards
    st, h = _sequence(mc, lib, obs, FailingAllocator(0))
    assert st == 0
    lib.mc_destroy(h)
