"""GB300-native sketch-and-project ridge regression (arXiv 2105.05565, "RidgeSketch").

Thin Python binding of the C ABI declared in ``include/ridgesketch.h``. Every
step of the iteration runs in the CUDA kernels of ``libridgesketch.so``; this
module only marshals arguments (numpy arrays or torch tensors, host or device)
into the ABI calls. There is no CPU fallback: importing the solver without the
built library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["Solver", "Batch", "CSR", "MLP", "RidgeSketch", "RSError", "lib", "SKETCHES", "MOMENTA"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libridgesketch.so")

RS_OK, RS_EINVAL, RS_ENOMEM, RS_ECUDA, RS_ENUMERIC, RS_ETIMEOUT, RS_ENOTCONV, RS_EUNSUPPORTED = range(8)
STATUS_NAMES = ["RS_OK", "RS_EINVAL", "RS_ENOMEM", "RS_ECUDA", "RS_ENUMERIC", "RS_ETIMEOUT",
                "RS_ENOTCONV", "RS_EUNSUPPORTED"]
SKETCHES = {"gaussian": 0, "subsample": 1, "count": 2, "subcount": 3, "srht": 4}
MOMENTA = {"none": 0, "const": 1, "theory": 2, "heuristic": 3}
FORMS = {"primal": 0, "dual": 1}
PRECISIONS = {"fp64": 0, "mixed": 1}


class RSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class Mom(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("uncapped", ctypes.c_int32), ("eta", ctypes.c_double),
                ("beta_switch", ctypes.c_double), ("gamma_c", ctypes.c_double),
                ("beta_c", ctypes.c_double)]


class Matrix(ctypes.Structure):
    _fields_ = [("is_csr", ctypes.c_int32), ("dtype", ctypes.c_int32), ("n", ctypes.c_int64),
                ("d", ctypes.c_int64), ("nnz", ctypes.c_int64), ("val", ctypes.c_void_p),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p),
                ("on_device", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("refresh_every", ctypes.c_int32),
                ("sub_s", ctypes.c_int64), ("cuda_stream", ctypes.c_void_p),
                ("device", ctypes.c_int32), ("chol_fp64", ctypes.c_int32), ("chunk", ctypes.c_int64),
                ("setup_tc", ctypes.c_int32), ("iter_ctas", ctypes.c_int32),
                ("spin_limit_ns", ctypes.c_int64), ("stall_ns", ctypes.c_int64),
                ("tune_cache", ctypes.c_char_p)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double), ("iters", ctypes.c_int64)]


_LIB = None
_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "rs_default_opts": (None, [ctypes.POINTER(Opts)]),
    "rs_default_mom": (None, [ctypes.POINTER(Mom), _I32]),
    "rs_create": (_I32, [ctypes.POINTER(Matrix), _P, _I32, _D, _I32, _I32, _I64,
                         ctypes.POINTER(Mom), ctypes.c_uint64, ctypes.POINTER(Opts),
                         ctypes.POINTER(_P)]),
    "rs_solve": (_I32, [_P, _D, _I64, _P, _I32, _P, ctypes.POINTER(_I64)]),
    "rs_destroy": (None, [_P]),
    "rs_trim_memory": (_I32, [_I32]),
    "rs_last_error": (ctypes.c_char_p, [_P]),
    "rs_get_dims": (_I32, [_P] + [ctypes.POINTER(_I64)] * 5),
    "rs_iter_plan": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
    "rs_chunking": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "rs_set_sampling": (_I32, [_P, _I32]),
    "rs_create_kernel": (_I32, [ctypes.POINTER(Matrix), _P, _I32, _D, _D, _I32, _I64,
                                ctypes.POINTER(Mom), ctypes.c_uint64, ctypes.POINTER(Opts),
                                ctypes.POINTER(_P)]),
    "rs_get_kernel": (_I32, [_P, _P]),
    "rs_set_acceleration": (_I32, [_P, _D, _D]),
    "rs_solve_cg": (_I32, [_P, _D, _I64, _P, _I32, _P, ctypes.POINTER(_I64)]),
    "rs_collect": (_I32, [_P, _P, _I64, _D, _P, _P, ctypes.POINTER(_I64)]),
    "rs_set_averaging": (_I32, [_P, _I32]),
    "rs_get_average": (_I32, [_P, _P, _I32]),
    "rs_dump_sketch": (_I32, [_P, _I64, _P, _P, _P]),
    "rs_dump_gaussian": (_I32, [_P, _I64, _P]),
    "rs_get_state": (_I32, [_P, _P, _P, _P, _P, ctypes.POINTER(_I64)]),
    "rs_set_state": (_I32, [_P, _P, _P, _P, _P, _I64]),
    "rs_probe_step": (_I32, [_P, _P, _P, _P]),
    "rs_step": (_I32, [_P, _I64, _P]),
    "rs_true_residual": (_I32, [_P, _P, ctypes.POINTER(_D)]),
    "rs_timings": (_I32, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "rs_profile_iteration": (_I32, [_P, _I64, ctypes.POINTER(KernelStat), _I32,
                                    ctypes.POINTER(_I32)]),
    "rs_gram_apply_noalloc": (_I32, [_P, _I64, _I64, _P, _P, _P]),
    "rs_create_batch": (_I32, [_I32, ctypes.POINTER(Matrix), ctypes.POINTER(_P), _I32, _I32,
                               ctypes.POINTER(_D), _I32, ctypes.POINTER(_I64), ctypes.POINTER(Mom),
                               ctypes.c_uint64, ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "rs_solve_batch": (_I32, [_P, _D, _I64, ctypes.POINTER(_P), _P, _P]),
    "rs_destroy_batch": (None, [_P]),
    "rs_batch_last_error": (ctypes.c_char_p, [_P]),
    "rs_batch_info": (_I32, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D),
                             ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "rs_batch_set_launch": (_I32, [_P, _I32, _I32]),
    "rs_batch_profile": (_I32, [_P, _I32, _P]),
    "rs_set_proposal": (_I32, [_P, _P, _D]),
    "rs_proposal_features": (_I32, [_P, _P]),
    "rs_mlp_create": (_I32, [_P, _I32, _P, ctypes.POINTER(_P)]),
    "rs_mlp_grad": (_I32, [_P, _P, _P, _I64, _P, ctypes.POINTER(_D)]),
    "rs_mlp_step": (_I32, [_P, _P, _P, _I64, _D, ctypes.POINTER(_D)]),
    "rs_mlp_scores": (_I32, [_P, _P, _I64, _P]),
    "rs_mlp_get": (_I32, [_P, _P, _P]),
    "rs_mlp_destroy": (None, [_P]),
    "rs_mlp_last_error": (ctypes.c_char_p, [_P]),
}
EXPORTED = tuple(_SIGS)


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
                " (the solver has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _buf(x, dtype):
    """(pointer, on_device, keepalive) of a contiguous array of ``dtype`` (numpy dtype)."""
    if _is_torch(x):
        import torch

        tdt = {np.float64: torch.float64, np.float32: torch.float32}[np.dtype(dtype).type]
        t = x.detach()
        if t.dtype != tdt:
            t = t.to(tdt)
        t = t.contiguous()
        return t.data_ptr(), int(t.is_cuda), t
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, 0, a


def trim_memory(device: int = 0) -> None:
    """Return the unused device memory the library's pool keeps after destroyed
    contexts (rs_trim_memory)."""
    st = lib().rs_trim_memory(int(device))
    if st != RS_OK:
        raise RSError(st, lib().rs_last_error(None).decode())


class CSR:
    """Sparse X in compressed rows for the matrix-free path: rowptr (n + 1, int64),
    colidx (nnz, int32), vals (nnz; float64, float32, or bfloat16 given as the
    float values, which must be representable in bfloat16, with ``bf16=True``)."""

    def __init__(self, rowptr, colidx, vals, shape, bf16=False):
        self.n, self.d = (int(v) for v in shape)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        v = np.ascontiguousarray(vals)
        if bf16:
            bits = v.astype(np.float32).view(np.uint32)
            if np.any(bits & 0xFFFF):
                raise ValueError("CSR values are not representable in bfloat16")
            self.vals = np.ascontiguousarray((bits >> 16).astype(np.uint16))
            self.dtype = 2
        elif v.dtype == np.float32:
            self.vals, self.dtype = v, 1
        else:
            self.vals, self.dtype = np.ascontiguousarray(v, dtype=np.float64), 0
        self.nnz = int(self.colidx.shape[0])
        self.shape = (self.n, self.d)

    @classmethod
    def from_scipy(cls, A, bf16=False):
        A = A.tocsr()
        return cls(A.indptr, A.indices, A.data, A.shape, bf16=bf16)


def _default_stream(device):
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream
    except Exception:  # pragma: no cover
        pass
    return None


class Solver:
    """One ridge problem on the GPU (rs_create / rs_solve / rs_destroy).

    X: (n, d) float32 or float64 array or tensor (host or CUDA); y: (n,) targets.
    """

    def __init__(self, X, y, lam, form="primal", sketch="count", tau=0, momentum="none", seed=0,
                 precision="fp64", refresh_every=50, sub_s=0, chol_fp64=True, chunk=0,
                 eta=0.995, beta_switch=0.5, gamma_c=1.0, beta_c=0.5, uncapped=False,
                 device=0, stream=None, setup_tc=True, iter_ctas=0, spin_limit_ns=0,
                 stall_ns=0, kernel_sigma=None):
        L = lib()
        self._ctx = None
        yp, ydev, self._ykeep = _buf(y, np.float64)
        if isinstance(X, CSR):
            self._xkeep = X
            n, d = X.n, X.d
            mat = Matrix(1, X.dtype, n, d, X.nnz, X.vals.ctypes.data, X.rowptr.ctypes.data,
                         X.colidx.ctypes.data, 0)
        else:
            xdt = np.float32 if str(getattr(X, "dtype", "")).endswith("float32") else np.float64
            xp, xdev, self._xkeep = _buf(X, xdt)
            n, d = (int(s) for s in X.shape)
            mat = Matrix(0, 1 if xdt == np.float32 else 0, n, d, 0, xp, None, None, xdev)
        mom = Mom()
        L.rs_default_mom(ctypes.byref(mom), MOMENTA[momentum])
        mom.eta, mom.beta_switch, mom.gamma_c, mom.beta_c = eta, beta_switch, gamma_c, beta_c
        mom.uncapped = int(bool(uncapped))
        opts = Opts()
        L.rs_default_opts(ctypes.byref(opts))
        opts.precision = PRECISIONS[precision]
        opts.refresh_every = int(refresh_every)
        opts.sub_s = int(sub_s)
        opts.device = int(device)
        opts.chol_fp64 = int(bool(chol_fp64))
        opts.chunk = int(chunk)
        opts.setup_tc = int(bool(setup_tc))
        opts.iter_ctas = int(iter_ctas)
        opts.spin_limit_ns = int(spin_limit_ns)
        opts.stall_ns = int(stall_ns)
        st = stream if stream is not None else _default_stream(device)
        opts.cuda_stream = st
        ctx = _P()
        if kernel_sigma is not None:
            # kernel ridge (Section 2.2): X holds the n points; the system is n x n
            status = L.rs_create_kernel(ctypes.byref(mat), yp, ydev, float(lam),
                                        float(kernel_sigma), SKETCHES[sketch], int(tau),
                                        ctypes.byref(mom), ctypes.c_uint64(int(seed)),
                                        ctypes.byref(opts), ctypes.byref(ctx))
            d = n
        else:
            status = L.rs_create(ctypes.byref(mat), yp, ydev, float(lam), FORMS[form],
                                 SKETCHES[sketch], int(tau), ctypes.byref(mom),
                                 ctypes.c_uint64(int(seed)), ctypes.byref(opts),
                                 ctypes.byref(ctx))
        if status != RS_OK:
            raise RSError(status, L.rs_last_error(None).decode())
        self._ctx = ctx
        self.n, self.d, self.form, self.sketch = n, d, form, sketch
        dims = [_I64() for _ in range(5)]
        L.rs_get_dims(ctx, *[ctypes.byref(v) for v in dims])
        self.m, self.tau, self.s, self.k_sum, self.m_pad = (v.value for v in dims)
        ctas, q = _I32(), _I64()
        L.rs_iter_plan(ctx, ctypes.byref(ctas), ctypes.byref(q))
        self.iter_ctas, self.iter_rows = ctas.value, q.value

    # -- helpers --
    def _check(self, status, allow=(RS_OK,)):
        if status not in allow:
            raise RSError(status, lib().rs_last_error(self._ctx).decode())
        return status

    def close(self):
        if self._ctx is not None:
            lib().rs_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- API --
    def solve(self, tol=1e-6, max_iters=10000, w_out=None):
        """Run from w = 0 to tol or max_iters. Returns (w, hist, iters, converged).
        ``w_out`` may be a CUDA float64 tensor of d entries to receive w on the device."""
        hist = np.empty(int(max_iters) + 1)
        iters = _I64()
        if w_out is not None:
            wp, wdev, _keep = w_out.data_ptr(), int(w_out.is_cuda), w_out
            w_ret = w_out
        else:
            w_ret = np.empty(self.d)
            wp, wdev = w_ret.ctypes.data, 0
        st = self._check(lib().rs_solve(self._ctx, float(tol), int(max_iters), wp, wdev,
                                        hist.ctypes.data, ctypes.byref(iters)),
                         allow=(RS_OK, RS_ENOTCONV))
        k = iters.value
        return w_ret, hist[: k + 1].copy(), k, st == RS_OK

    def solve_cg(self, tol=1e-6, max_iters=10000, w_out=None):
        """Conjugate Gradients on the same system from w = 0 (rs_solve_cg). Returns
        (w, hist, iters, converged) like solve."""
        hist = np.empty(int(max_iters) + 1)
        iters = _I64()
        if w_out is not None:
            wp, wdev, _keep = w_out.data_ptr(), int(w_out.is_cuda), w_out
            w_ret = w_out
        else:
            w_ret = np.empty(self.d)
            wp, wdev = w_ret.ctypes.data, 0
        st = self._check(lib().rs_solve_cg(self._ctx, float(tol), int(max_iters), wp, wdev,
                                           hist.ctypes.data, ctypes.byref(iters)),
                         allow=(RS_OK, RS_ENOTCONV))
        return w_ret, hist[: iters.value + 1], iters.value, st == RS_OK

    def dump_sketch(self, k):
        cap = max(self.m, self.s, self.tau, 1)
        idx = np.zeros(cap, np.int32)
        sign = np.zeros(cap, np.int8)
        bucket = np.zeros(cap, np.int32)
        self._check(lib().rs_dump_sketch(self._ctx, int(k), idx.ctypes.data, sign.ctypes.data,
                                         bucket.ctypes.data))
        return idx, sign, bucket

    def dump_gaussian(self, k):
        S = np.empty((self.m, self.tau))
        self._check(lib().rs_dump_gaussian(self._ctx, int(k), S.ctypes.data))
        return S

    def get_state(self):
        m = self.m
        w, wp, r, rp = (np.empty(m) for _ in range(4))
        k = _I64()
        self._check(lib().rs_get_state(self._ctx, w.ctypes.data, wp.ctypes.data, r.ctypes.data,
                                       rp.ctypes.data, ctypes.byref(k)))
        return w, wp, r, rp, k.value

    def set_state(self, w, w_prev, r, r_prev, k):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (w, w_prev, r, r_prev)]
        self._check(lib().rs_set_state(self._ctx, *[a.ctypes.data for a in arrs], int(k)))

    def probe_step(self):
        t = self.tau
        M = np.empty((t, t))
        rS = np.empty(t)
        delta = np.empty(t)
        self._check(lib().rs_probe_step(self._ctx, M.ctypes.data, rS.ctypes.data, delta.ctypes.data))
        return M, rS, delta

    def step(self, n_iters):
        hist = np.empty(max(int(n_iters), 1))
        self._check(lib().rs_step(self._ctx, int(n_iters), hist.ctypes.data))
        return hist[: int(n_iters)]

    def true_residual(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = _D()
        self._check(lib().rs_true_residual(self._ctx, v.ctypes.data, ctypes.byref(out)))
        return out.value

    def chunking(self):
        """(iterations per chunk, FP64 refresh period or 0, 1 if M^+ comes from the fused
        factor-inverse-product kernel)."""
        ch, ref, fu = _I64(), _I32(), _I32()
        self._check(lib().rs_chunking(self._ctx, ctypes.byref(ch), ctypes.byref(ref),
                                      ctypes.byref(fu)))
        return ch.value, ref.value, fu.value

    def profile_iteration(self, reps):
        """Per kernel group: dict(name -> (mean ms per launch, launches, bytes, flops))."""
        cap = 16
        arr = (KernelStat * cap)()
        n = _I32()
        self._check(lib().rs_profile_iteration(self._ctx, int(reps), arr, cap, ctypes.byref(n)))
        return {arr[i].name.decode(): (arr[i].ms, arr[i].launches, arr[i].bytes, arr[i].flops,
                                       arr[i].iters)
                for i in range(n.value)}

    def set_acceleration(self, mu, nu):
        """Accelerated sketch-and-project (Algorithm 3) with parameters mu, nu; (0, 0)
        returns to the momentum form."""
        self._check(lib().rs_set_acceleration(self._ctx, float(mu), float(nu)))

    def kernel_matrix(self):
        """The n x n kernel matrix of a kernel ridge solver (host array)."""
        K = np.empty((self.n, self.n))
        self._check(lib().rs_get_kernel(self._ctx, K.ctypes.data))
        return K

    def set_averaging(self, on=True):
        """Keep the mean of the iterates of each solve (Section 5.2)."""
        self._check(lib().rs_set_averaging(self._ctx, int(bool(on))))

    def average(self):
        """Mean of the iterates w^0..w^t of the last solve (host array)."""
        out = np.empty(self.d)
        self._check(lib().rs_get_average(self._ctx, out.ctypes.data, 0))
        return out

    def collect(self, w_star, n_iters, tol=1e-10):
        """Features and targets of the rows drawn along up to n_iters iterations from the
        current state (rs_collect): (Z (n, 4) float32, y (n,) float32)."""
        ws = np.ascontiguousarray(w_star, dtype=np.float64)
        Z = np.empty((int(n_iters) * self.tau, 4), np.float32)
        y = np.empty(int(n_iters) * self.tau, np.float32)
        n = _I64()
        self._check(lib().rs_collect(self._ctx, ws.ctypes.data, int(n_iters), float(tol),
                                     Z.ctypes.data, y.ctypes.data, ctypes.byref(n)))
        return Z[:n.value].copy(), y[:n.value].copy()

    def set_sampling(self, kind="diag"):
        """Subsample rows drawn in proportion to A_jj ("diag", Section 7) or uniformly
        ("uniform", the default)."""
        self._check(lib().rs_set_sampling(self._ctx, {"uniform": 0, "diag": 1}[kind]))

    def set_proposal(self, weights_bf16=None, eps=0.1):
        """Draw the subsample rows from the learned proposal: ``weights_bf16`` (4545
        uint16 bfloat16 bit patterns) or None for the uniform proposal; eps < 0
        switches back to the plain sampler."""
        if weights_bf16 is None:
            ptr = None
        else:
            self._wkeep = np.ascontiguousarray(weights_bf16, dtype=np.uint16)
            if self._wkeep.size != MLP_PARAMS:
                raise ValueError(f"weights_bf16 must hold {MLP_PARAMS} values")
            ptr = self._wkeep.ctypes.data
        self._check(lib().rs_set_proposal(self._ctx, ptr, float(eps)))

    def proposal_features(self):
        """(m, 4) float32 standardised features at the current state."""
        Z = np.empty((self.m, 4), np.float32)
        self._check(lib().rs_proposal_features(self._ctx, Z.ctypes.data))
        return Z

    def timings(self):
        a, b = _D(), _D()
        self._check(lib().rs_timings(self._ctx, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value


MLP_PARAMS = 4545


class MLP:
    """The proposal's 4 -> 64 -> 64 -> 1 network on the GPU for training: FP32
    master weights, Adam, and the bfloat16 copy the proposal reads
    (rs_mlp_create / rs_mlp_grad / rs_mlp_step / rs_mlp_get)."""

    def __init__(self, theta0, device=0, stream=None):
        L = lib()
        self._h = None
        th = np.ascontiguousarray(theta0, dtype=np.float32)
        if th.size != MLP_PARAMS:
            raise ValueError(f"theta0 must hold {MLP_PARAMS} values")
        h = _P()
        st = stream if stream is not None else _default_stream(device)
        status = L.rs_mlp_create(th.ctypes.data, int(device), st, ctypes.byref(h))
        if status != RS_OK:
            raise RSError(status, L.rs_mlp_last_error(None).decode())
        self._h = h
        self.device = device

    def _check(self, status):
        if status != RS_OK:
            raise RSError(status, lib().rs_mlp_last_error(self._h).decode())

    @staticmethod
    def _dev(x, dtype):
        import torch

        t = torch.as_tensor(x)
        return t.to(device="cuda", dtype=dtype).contiguous()

    def grad(self, Z, y):
        """(loss, gradient (4545,) float32) of mean((s - y)^2) / 2."""
        import torch

        Zd, yd = self._dev(Z, torch.float32), self._dev(y, torch.float32)
        g = np.empty(MLP_PARAMS, np.float32)
        loss = _D()
        self._check(lib().rs_mlp_grad(self._h, Zd.data_ptr(), yd.data_ptr(), int(yd.numel()),
                                      g.ctypes.data, ctypes.byref(loss)))
        return loss.value, g

    def step(self, Z, y, lr=1e-3):
        """One Adam step; returns the loss before it."""
        import torch

        Zd, yd = self._dev(Z, torch.float32), self._dev(y, torch.float32)
        loss = _D()
        self._check(lib().rs_mlp_step(self._h, Zd.data_ptr(), yd.data_ptr(), int(yd.numel()),
                                      float(lr), ctypes.byref(loss)))
        return loss.value

    def scores(self, Z):
        import torch

        Zd = self._dev(Z, torch.float32)
        n = Zd.shape[0]
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        self._check(lib().rs_mlp_scores(self._h, Zd.data_ptr(), int(n), out.data_ptr()))
        torch.cuda.synchronize()
        return out.cpu().numpy()

    def params(self):
        th = np.empty(MLP_PARAMS, np.float32)
        self._check(lib().rs_mlp_get(self._h, th.ctypes.data, None))
        return th

    def weights_bf16(self):
        w = np.empty(MLP_PARAMS, np.uint16)
        self._check(lib().rs_mlp_get(self._h, None, w.ctypes.data))
        return w

    def close(self):
        if self._h is not None:
            lib().rs_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """P independent primal ridge problems, nrhs right-hand sides each, solved together
    (rs_create_batch / rs_solve_batch / rs_destroy_batch).

    Xs: P dense (n_p, d_p) arrays (float32 for ``precision="mixed"``); Ys: P arrays of
    shape (nrhs, n_p); lams: P regularisers; taus: P sketch sizes (0 = default rule)
    or None. Problem p draws its sketches with seed + p.
    """

    def __init__(self, Xs, Ys, lams, sketch="count", taus=None, momentum="none", seed=0,
                 precision="fp64", refresh_every=300, sub_s=0, chunk=0, eta=0.995,
                 beta_switch=0.5, gamma_c=1.0, beta_c=0.5, uncapped=False, device=0, stream=None,
                 setup_tc=True, chol_fp64=True, tune_cache=None):
        L = lib()
        self._b = None
        P = len(Xs)
        if not (len(Ys) == P and len(lams) == P):
            raise ValueError("Xs, Ys and lams must have one entry per problem")
        xdt = np.float32 if precision == "mixed" else np.float64
        mats = (Matrix * P)()
        self._keep = []
        yptrs = (_P * P)()
        nrhs = None
        self.dims = []
        ydev = None
        for p in range(P):
            xp, xdev, xk = _buf(Xs[p], xdt)
            n, d = (int(v) for v in Xs[p].shape)
            mats[p] = Matrix(0, 1 if xdt == np.float32 else 0, n, d, 0, xp, None, None, xdev)
            Y = Ys[p]
            if Y.ndim == 1:
                Y = Y[None, :]
            if tuple(Y.shape)[1] != n:
                raise ValueError(f"Ys[{p}] must have shape (nrhs, {n})")
            yp, ydv, yk = _buf(Y, np.float64)
            if ydev is None:
                ydev = ydv
            elif ydv != ydev:
                raise ValueError("Ys must be all host arrays or all CUDA tensors")
            if nrhs is None:
                nrhs = int(Y.shape[0])
            elif int(Y.shape[0]) != nrhs:
                raise ValueError("every problem needs the same number of right-hand sides")
            yptrs[p] = yp
            self._keep += [xk, yk]
            self.dims.append(d)
        lam_a = (_D * P)(*[float(v) for v in lams])
        tau_a = (_I64 * P)(*[int(v) for v in (taus if taus is not None else [0] * P)])
        mom = Mom()
        L.rs_default_mom(ctypes.byref(mom), MOMENTA[momentum])
        mom.eta, mom.beta_switch, mom.gamma_c, mom.beta_c = eta, beta_switch, gamma_c, beta_c
        mom.uncapped = int(bool(uncapped))
        opts = Opts()
        L.rs_default_opts(ctypes.byref(opts))
        opts.precision = PRECISIONS[precision]
        opts.refresh_every = int(refresh_every)
        opts.sub_s = int(sub_s)
        opts.device = int(device)
        opts.chunk = int(chunk)
        opts.setup_tc = int(bool(setup_tc))
        opts.chol_fp64 = int(bool(chol_fp64))
        self._tune_cache = None if tune_cache is None else str(tune_cache).encode()
        opts.tune_cache = self._tune_cache
        opts.cuda_stream = stream if stream is not None else _default_stream(device)
        b = _P()
        status = L.rs_create_batch(P, mats, yptrs, int(ydev), int(nrhs), lam_a, SKETCHES[sketch], tau_a,
                                   ctypes.byref(mom), ctypes.c_uint64(int(seed)), ctypes.byref(opts),
                                   ctypes.byref(b))
        if status != RS_OK:
            raise RSError(status, L.rs_batch_last_error(None).decode())
        self._b = b
        self.P, self.nrhs = P, int(nrhs)

    def _check(self, status, allow=(RS_OK,)):
        if status not in allow:
            raise RSError(status, lib().rs_batch_last_error(self._b).decode())
        return status

    def close(self):
        if self._b is not None:
            lib().rs_destroy_batch(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, tol=1e-6, max_iters=10000):
        """Returns (W, iters, resid, converged): W[p] of shape (nrhs, d_p); iters and resid
        of shape (P, nrhs); converged is True when every pair reached tol."""
        W = [np.empty((self.nrhs, d)) for d in self.dims]
        wptr = (_P * self.P)(*[w.ctypes.data for w in W])
        iters = np.empty(self.P * self.nrhs, np.int64)
        resid = np.empty(self.P * self.nrhs)
        st = self._check(lib().rs_solve_batch(self._b, float(tol), int(max_iters), wptr,
                                              iters.ctypes.data, resid.ctypes.data),
                         allow=(RS_OK, RS_ENOTCONV))
        return (W, iters.reshape(self.P, self.nrhs), resid.reshape(self.P, self.nrhs),
                st == RS_OK)

    def set_launch(self, iter_threads=0, phase1_streams=0):
        """Fix the iteration kernel's CTA size and the phase-1 streams (0, 0: autotune)."""
        self._check(lib().rs_batch_set_launch(self._b, int(iter_threads), int(phase1_streams)))

    def profile(self, chunks=2):
        """Mean ms per chunk of each part (plans, rows, msys, inverse: phase 1; iterate;
        refresh); overwrites the state."""
        out = np.zeros(6)
        self._check(lib().rs_batch_profile(self._b, int(chunks), out.ctypes.data))
        names = ["plan_ms", "rows_ms", "msys_ms", "inverse_ms", "iterate_ms", "refresh_ms"]
        r = dict(zip(names, out.tolist()))
        r["phase1_ms"] = float(out[:4].sum())
        return r

    def info(self):
        """dict: setup_ms, solve_ms, tune_ms, iter_threads, phase1_streams."""
        a, b, c = _D(), _D(), _D()
        t, ns = _I32(), _I32()
        self._check(lib().rs_batch_info(self._b, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                        ctypes.byref(t), ctypes.byref(ns)))
        return {"setup_ms": a.value, "solve_ms": b.value, "tune_ms": c.value,
                "iter_threads": t.value, "phase1_streams": ns.value}


class RidgeSketch:
    """Estimator with the paper's interface (Appendix B): RidgeSketch(alpha,
    algo_mode, solver, sketch_size).fit(X, y) -> coef_."""

    def __init__(self, alpha=1.0, algo_mode="mom", solver="subsample", sketch_size=0, tol=1e-6,
                 max_iter=10000, seed=0, precision="fp64", form=None):
        self.alpha, self.algo_mode, self.solver, self.sketch_size = alpha, algo_mode, solver, sketch_size
        self.tol, self.max_iter, self.seed, self.precision, self.form = tol, max_iter, seed, precision, form

    def fit(self, X, y):
        n, d = X.shape
        form = self.form or ("primal" if d <= n else "dual")  # Section 2.1
        mom = {"mom": "heuristic", "no_mom": "none", "auto": "heuristic"}.get(self.algo_mode, self.algo_mode)
        with Solver(X, y, self.alpha, form=form, sketch=self.solver, tau=self.sketch_size,
                    momentum=mom, seed=self.seed, precision=self.precision) as s:
            w, hist, iters, conv = s.solve(self.tol, self.max_iter)
        self.coef_, self.residuals_, self.n_iter_, self.converged_ = w, hist, iters, conv
        return self

    def predict(self, X):
        return np.asarray(X) @ self.coef_
