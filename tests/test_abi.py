"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/mc.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(mc_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_06860_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mc_create", "mc_rsvd_pi", "mc_rsvd_bki", "mc_svt_step", "mc_svt_solve", "mc_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1810_06860_gb300 import _native

    assert set(_declared()) <= set(_native.exported_symbols())


def test_params_default_and_status_strings(lib):
    import paper_1810_06860_gb300 as mc

    p = mc.params()
    assert (p.l, p.s, p.p0, p.p_min, p.p_max, p.i_max, p.i_reuse, p.q_reuse) == (5, 10, 3, 3, 20, 1000, 50, 10)
    assert mc.load().mc_status_str(1) == b"MC_EINVAL"
    with pytest.raises(KeyError):
        mc.params(nonsense=1)
