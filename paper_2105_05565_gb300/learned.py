"""Training the learned sketch proposal (offline, on solver trajectories).

``collect`` runs a solver (subsample sketch, no momentum, a proposal set with
``Solver.set_proposal``) through the library's rs_collect, which records on the
device, for every drawn row, its standardised features and the target

    y_p = (1/2) ln(m max(a_p, 0) / ||e_k||_A^2 + 1e-3),   a_p = (r_C)_p delta_p,

where r_C . delta is the exact decrease of ||w - w*||_A^2 of the step (the
projection identity of Section 3) and ||e_k||_A^2 = (w_k - w*) . r_k. ``train``
fits the network to those pairs with the library's Adam kernels. The arithmetic
of both runs in the CUDA library; this module only drives it.
"""
from __future__ import annotations

import numpy as np

from . import MLP, MLP_PARAMS


def init_params(seed: int) -> np.ndarray:
    """He-normal initial weights (std sqrt(2 / fan_in), sqrt(1 / 64) for the output
    layer), zero biases, in the library's parameter layout."""
    g = np.random.default_rng(seed)
    W1 = g.standard_normal((64, 4)) * np.sqrt(0.5)
    W2 = g.standard_normal((64, 64)) * np.sqrt(2.0 / 64)
    w3 = g.standard_normal(64) * np.sqrt(1.0 / 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [0.0]])


def collect(solver, w_star, n_iters: int, tol: float = 1e-10):
    """(features (n, 4) float32, targets (n,) float32) of the rows drawn along
    n_iters iterations of ``solver`` from its current state (stops early once the
    relative residual is below tol); the library forms both on the device
    (rs_collect)."""
    return solver.collect(w_star, n_iters, tol)


def train(Z, y, steps: int = 2000, batch: int = 512, lr: float = 3e-3, seed: int = 0,
          theta0=None, device: int = 0):
    """Adam on minibatches of (Z, y); returns (bfloat16 weights (4545,) uint16,
    FP32 weights, losses)."""
    import torch

    Zd = torch.as_tensor(np.ascontiguousarray(Z, dtype=np.float32)).to(f"cuda:{device}")
    yd = torch.as_tensor(np.ascontiguousarray(y, dtype=np.float32)).to(f"cuda:{device}")
    n = yd.numel()
    g = torch.Generator(device=f"cuda:{device}")
    g.manual_seed(int(seed))
    theta0 = init_params(seed) if theta0 is None else np.asarray(theta0)
    assert theta0.size == MLP_PARAMS
    losses = []
    with MLP(theta0, device=device) as net:
        for _ in range(int(steps)):
            sel = torch.randint(0, n, (min(batch, n),), generator=g, device=Zd.device)
            losses.append(net.step(Zd[sel], yd[sel], lr))
        return net.weights_bf16(), net.params(), np.asarray(losses)
