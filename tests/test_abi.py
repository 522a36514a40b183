"""The C ABI library loads and exports every entry point of include/ridgesketch.h;
host-side argument checks answer without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ridgesketch.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    import paper_2105_05565_gb300 as rs

    if not os.path.exists(rs.LIB_PATH):
        import __graft_entry__

        __graft_entry__.build()
    return rs.lib()


def test_header_declares_the_boundary():
    names = declared()
    for must in ("rs_create", "rs_solve", "rs_destroy", "rs_last_error", "rs_dump_sketch"):
        assert must in names


def test_every_declared_symbol_is_exported(L):
    import paper_2105_05565_gb300 as rs

    for name in declared():
        assert hasattr(L, name), name
    assert set(declared()) == set(rs.EXPORTED)


def test_null_arguments_are_rejected_without_a_device(L):
    import paper_2105_05565_gb300 as rs

    ctx = ctypes.c_void_p()
    st = L.rs_create(None, None, 0, 1.0, 0, 0, 0, None, 0, None, ctypes.byref(ctx))
    assert st == rs.RS_EINVAL and ctx.value is None
    assert b"null" in L.rs_last_error(None)
    st = L.rs_solve(None, 1e-6, 10, None, 0, None, None)
    assert st == rs.RS_EINVAL
    assert L.rs_iter_plan(None, None, None) == rs.RS_EINVAL
    L.rs_destroy(None)
    # no pool exists before the first context: nothing to trim, no CUDA call
    assert L.rs_trim_memory(-1) == rs.RS_EINVAL and L.rs_trim_memory(64) == rs.RS_EINVAL
    assert L.rs_trim_memory(0) == rs.RS_OK


def test_bad_enums_rejected(L):
    import numpy as np

    import paper_2105_05565_gb300 as rs

    X = np.zeros((4, 3))
    y = np.zeros(4)
    mat = rs.Matrix(0, 0, 4, 3, 0, X.ctypes.data, None, None, 0)
    ctx = ctypes.c_void_p()
    for args in [(-1.0, 0, 1), (1.0, 5, 1), (1.0, 0, 9)]:
        lam, form, sketch = args
        st = L.rs_create(ctypes.byref(mat), y.ctypes.data, 0, lam, form, sketch, 0, None, 0, None,
                         ctypes.byref(ctx))
        assert st == rs.RS_EINVAL


def test_default_options(L):
    import paper_2105_05565_gb300 as rs

    o = rs.Opts()
    L.rs_default_opts(ctypes.byref(o))
    assert o.precision == 0 and o.refresh_every == 50 and o.chol_fp64 == 1
    assert o.iter_ctas == 0 and o.setup_tc == 1
    m = rs.Mom()
    L.rs_default_mom(ctypes.byref(m), 3)
    assert m.kind == 3 and m.eta == 0.995 and m.beta_switch == 0.5
