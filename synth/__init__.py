"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only draws data (design matrices, targets, sparse patterns). It holds
none of the sketch-and-project arithmetic: no sketch, no projection, no residual.
Every generator is deterministic in its ``seed``.

Shapes and distributions follow the workloads the solver is meant for: dense
Gaussian designs, dense designs with a prescribed singular spectrum (Haar-random
singular vectors), Zipf-distributed sparse designs and batches of uneven problems.
The paper's own datasets (California Housing, Boston, RCV1, YearPredictionMSD;
Section 9) are not used; these generators stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "gaussian_problem",
    "haar_columns",
    "spectrum_problem",
    "spectrum_problem_torch",
    "zipf_csr",
    "batched_specs",
    "batched_problem",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian_problem(n: int, d: int, seed: int, noise: float = 0.1, dtype=np.float64):
    """X iid N(0,1) (n x d), w* ~ N(0,1), y = X w* + noise * N(0,1).

    ``dtype`` is the storage type of X; y is computed from the stored X in float64.
    Returns (X, y, w_true).
    """
    g = _rng(seed)
    X = g.standard_normal((n, d)).astype(dtype)
    w_true = g.standard_normal(d)
    y = X.astype(np.float64) @ w_true + noise * g.standard_normal(n)
    return X, y, w_true


def haar_columns(g: np.random.Generator, n: int, d: int) -> np.ndarray:
    """n x d matrix with orthonormal columns, Haar distributed (QR of a Gaussian
    matrix with the signs of R's diagonal moved into Q; Mezzadri 2007)."""
    G = g.standard_normal((n, d))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def spectrum_problem(n: int, d: int, sigma: np.ndarray, seed: int, noise: float = 0.01,
                     dtype=np.float64):
    """X = U diag(sigma) V^T with Haar U (n x d) and V (d x d); y = X w* + noise.

    Returns (X, y, w_true). Small sizes only (numpy QR on the CPU)."""
    g = _rng(seed)
    U = haar_columns(g, n, d)
    V = haar_columns(g, d, d)
    X = ((U * np.asarray(sigma)[None, :]) @ V.T).astype(dtype)
    w_true = g.standard_normal(d)
    y = X.astype(np.float64) @ w_true + noise * g.standard_normal(n)
    return X, y, w_true


def _preload_torch_linalg():
    """Load torch's lazily opened CUDA linear-algebra library by full path, so that
    the QR below also works under tools that change the library search path."""
    import ctypes
    import os

    import torch

    p = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(p):
        try:
            ctypes.CDLL(p, mode=ctypes.RTLD_GLOBAL)
        except OSError:
            pass


def spectrum_problem_torch(n: int, d: int, sigma, seed: int, noise: float = 0.01,
                           device="cuda"):
    """Large-size version of ``spectrum_problem`` drawn with torch on ``device``.

    X is float32 (n x d, row-major) and is the problem's data as stored; y is
    computed from that stored X in float64. Returns torch tensors (X, y, w_true).
    """
    import torch

    _preload_torch_linalg()
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    sig = torch.as_tensor(np.asarray(sigma), dtype=torch.float32, device=device)

    def haar(rows, cols):
        G = torch.randn(rows, cols, generator=gen, device=device, dtype=torch.float32)
        Q, R = torch.linalg.qr(G)
        return Q * torch.sign(torch.diagonal(R))[None, :]

    U = haar(n, d)
    V = haar(d, d)
    X = (U * sig[None, :]) @ V.T
    del U
    w_true = torch.randn(d, generator=gen, device=device, dtype=torch.float64)
    eps = torch.randn(n, generator=gen, device=device, dtype=torch.float64)
    y = X.double() @ w_true + noise * eps
    return X.contiguous(), y.contiguous(), w_true


def geometric_sigma(d: int, lo: float = 1e-3) -> np.ndarray:
    """sigma_i geometric from 1 down to ``lo`` over d values."""
    if d == 1:
        return np.ones(1)
    return lo ** (np.arange(d) / (d - 1))


def power_sigma(d: int, p: float = 0.8) -> np.ndarray:
    """sigma_i = i^-p, i = 1..d."""
    return np.arange(1, d + 1, dtype=np.float64) ** (-p)


__all__ += ["geometric_sigma", "power_sigma"]


def zipf_csr(n: int, d: int, nnz_target: int, seed: int, alpha: float = 1.1):
    """Sparse n x d design in CSR form.

    (row, col) pairs are drawn with col ~ Zipf(alpha) truncated to [0, d) and row
    uniform on [0, n); duplicate pairs keep their first draw; values are
    lognormal(0, 1). Returns (rowptr int64[n+1], colidx int32[nnz], vals f64[nnz]);
    columns are sorted within each row.
    """
    g = _rng(seed)
    ranks = np.arange(1, d + 1, dtype=np.float64)
    p = ranks ** (-alpha)
    p /= p.sum()
    cols = g.choice(d, size=nnz_target, p=p).astype(np.int64)
    rows = g.integers(0, n, size=nnz_target, dtype=np.int64)
    vals = g.lognormal(0.0, 1.0, size=nnz_target)
    key = rows * d + cols
    _, first = np.unique(key, return_index=True)
    first.sort()
    rows, cols, vals, key = rows[first], cols[first], vals[first], key[first]
    order = np.argsort(key, kind="stable")
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols.astype(np.int32), vals


def batched_specs(P: int, seed: int, dmin: int = 256, dmax: int = 4096):
    """Per-problem sizes and regularisers of a batch of uneven ridge problems:
    d log-uniform in [dmin, dmax], n = 4 d, lambda log-uniform in [1e-4, 1]."""
    g = _rng(seed)
    d = np.floor(np.exp(g.uniform(math.log(dmin), math.log(dmax), size=P))).astype(np.int64)
    d = np.clip(d, dmin, dmax)
    lam = np.exp(g.uniform(math.log(1e-4), 0.0, size=P))
    return d, 4 * d, lam


def batched_problem(n: int, d: int, nrhs: int, seed: int, noise: float = 0.1,
                    dtype=np.float32):
    """X = N(0,1) diag(c), c_j log-uniform in [1e-2, 1]; nrhs targets
    y_r = X w*_r + noise N(0,1). Returns (X (n x d), Y (nrhs x n) f64)."""
    g = _rng(seed)
    c = np.exp(g.uniform(math.log(1e-2), 0.0, size=d))
    X = (g.standard_normal((n, d)) * c[None, :]).astype(dtype)
    W = g.standard_normal((nrhs, d))
    Y = (X.astype(np.float64) @ W.T).T + noise * g.standard_normal((nrhs, n))
    return X, Y


def batched_problem_torch(n: int, d: int, nrhs: int, seed: int, noise: float = 0.1,
                          device="cuda"):
    """Large-batch version of ``batched_problem`` drawn with torch on ``device``:
    X float32 (n x d, row-major, the stored data), Y float64 (nrhs x n) computed from
    that stored X. Returns torch tensors (X, Y)."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    u = torch.rand(d, generator=gen, device=device, dtype=torch.float64)
    c = torch.exp(math.log(1e-2) * (1.0 - u))
    X = (torch.randn(n, d, generator=gen, device=device, dtype=torch.float32)
         * c.float()[None, :]).contiguous()
    W = torch.randn(nrhs, d, generator=gen, device=device, dtype=torch.float64)
    eps = torch.randn(nrhs, n, generator=gen, device=device, dtype=torch.float64)
    Y = (X.double() @ W.T).T + noise * eps
    return X, Y.contiguous()


def bf16_round(x) -> np.ndarray:
    """Values of x rounded to the nearest bfloat16 (ties to even), as float64: the
    stored data of a bfloat16 design matrix."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def sparse_problem(n: int, d: int, nnz_target: int, seed: int, noise: float = 0.1,
                   alpha: float = 1.1, bf16: bool = True):
    """Zipf-sparse design (``zipf_csr``), values rounded to bfloat16 when ``bf16``;
    w* ~ N(0,1), y = X w* + noise * N(0,1) from the stored values.
    Returns (rowptr, colidx, vals, y, w_true)."""
    import scipy.sparse as sp

    rowptr, colidx, vals = zipf_csr(n, d, nnz_target, seed, alpha)
    if bf16:
        vals = bf16_round(vals)
    g = _rng(seed + 7919)
    w_true = g.standard_normal(d)
    X = sp.csr_matrix((vals, colidx, rowptr), shape=(n, d))
    y = X @ w_true + noise * g.standard_normal(n)
    return rowptr, colidx, vals, y, w_true


__all__ += ["bf16_round", "sparse_problem"]


def mlp_init(seed: int) -> np.ndarray:
    """Initial parameters of the 4 -> 64 -> 64 -> 1 scoring network (flat, 4545
    entries: W1 64 x 4, b1, W2 64 x 64, b2, w3, b3): He-normal weights
    (std sqrt(2 / fan_in); sqrt(1 / 64) for the output layer), zero biases."""
    g = _rng(seed)
    W1 = g.standard_normal((64, 4)) * np.sqrt(2.0 / 4)
    W2 = g.standard_normal((64, 64)) * np.sqrt(2.0 / 64)
    w3 = g.standard_normal(64) * np.sqrt(1.0 / 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [0.0]])


__all__ += ["mlp_init"]
