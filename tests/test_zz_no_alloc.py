"""rs_gram_apply_noalloc: X^T (X v) without any allocation, for callers that are not
allowed to allocate device memory (its work space is a fixed array inside the
library). Checked through the C ABI against the library's allocating path
(rs_true_residual of a solver context, which runs the same product) and against
FP64 numpy, on two calls in a row that reuse the shared work space."""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,d", [(3000, 700), (2500, 4096)])
def test_noalloc_matches_allocating_path(n, d):
    import torch

    import paper_2105_05565_gb300 as rs

    L = rs.lib()
    g = np.random.default_rng(n + d)
    X = g.standard_normal((n, d)).astype(np.float32)
    y = g.standard_normal(n)
    lam = 0.3
    X64 = X.astype(np.float64)
    b = X64.T @ y
    Xd = torch.from_numpy(X).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    with rs.Solver(X, y, lam, sketch="count", tau=16, seed=1, precision="mixed") as s:
        for call in range(2):  # two calls in a row share the work space
            v = g.standard_normal(d) * (1.0 + call)
            vd = torch.from_numpy(v).cuda()
            out = torch.full((d,), float("nan"), dtype=torch.float64, device="cuda")
            st = L.rs_gram_apply_noalloc(ctypes.c_void_p(Xd.data_ptr()), n, d,
                                         ctypes.c_void_p(vd.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
            assert st == rs.RS_OK, L.rs_last_error(None)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            ref_vec = X64.T @ (X64 @ v)
            assert np.linalg.norm(got - ref_vec) <= 1e-12 * np.linalg.norm(ref_vec)
            rel = np.linalg.norm(got + lam * v - b) / np.linalg.norm(b)
            ref = s.true_residual(v)  # the allocating path of the library
            assert abs(rel - ref) <= 1e-12 * ref
            assert abs(ref - oracle.true_residual(X64, y, lam, v)) <= 1e-12 * ref


def test_noalloc_rejects_sizes_beyond_its_work_space():
    import torch

    import paper_2105_05565_gb300 as rs

    L = rs.lib()
    X = torch.zeros((4, 4097), dtype=torch.float32, device="cuda")
    v = torch.zeros(4097, dtype=torch.float64, device="cuda")
    out = torch.zeros(4097, dtype=torch.float64, device="cuda")
    st = L.rs_gram_apply_noalloc(ctypes.c_void_p(X.data_ptr()), 4, 4097,
                                 ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 None)
    assert st == rs.RS_EINVAL
    assert b"4096" in L.rs_last_error(None)


def test_noalloc_small_problems_after_a_large_one():
    """A large call fills all 64 block slots of the shared work space; the smaller
    calls after it (fewer rows than blocks, one row, a narrower d) must not pick up
    any of its stale block sums."""
    import torch

    import paper_2105_05565_gb300 as rs

    L = rs.lib()
    g = np.random.default_rng(7)
    stream = torch.cuda.current_stream().cuda_stream
    for n, d in [(2500, 4096), (10, 300), (1, 4096), (63, 1025), (2500, 4096), (1, 1)]:
        X = g.standard_normal((n, d)).astype(np.float32)
        v = g.standard_normal(d)
        Xd = torch.from_numpy(X).cuda()
        vd = torch.from_numpy(v).cuda()
        out = torch.full((d,), float("nan"), dtype=torch.float64, device="cuda")
        st = L.rs_gram_apply_noalloc(ctypes.c_void_p(Xd.data_ptr()), n, d,
                                     ctypes.c_void_p(vd.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == rs.RS_OK, L.rs_last_error(None)
        torch.cuda.synchronize()
        X64 = X.astype(np.float64)
        ref = X64.T @ (X64 @ v)
        got = out.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), (n, d)
