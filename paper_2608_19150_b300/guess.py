"""Training of the learned initial guess on trajectories the solver itself generates.

All arithmetic runs in the library's kernels (features, targets, forward, backward,
Adam); this module only orders the calls and keeps the data in device memory (torch
tensors used as buffers).  Batches are drawn with a seeded torch generator.
"""
from __future__ import annotations

import numpy as np

from . import bgk


def collect(solver: "bgk.Solver", steps: int, X_out: list, Y_out: list):
    """Advance `solver` by `steps` steps, recording for every step the features of the
    stage start and the converged change of (log n, u, log theta) at every node, less the
    previous step's change (what the network learns to correct)."""
    import torch
    F, O = solver.guess_dims()
    iters = []
    for _ in range(steps):
        X = torch.empty((solver.nnode, F), dtype=torch.float32, device="cuda")
        Y = torch.empty((solver.nnode, O), dtype=torch.float32, device="cuda")
        U0 = torch.empty((solver.nnode, O), dtype=torch.float64, device="cuda")
        solver.guess_features(X.data_ptr())
        solver.get_moments_device(U0.data_ptr())
        st = solver.step(1)
        iters.append(int(sum(st.iterations[:st.n_stages])))
        solver.guess_targets(U0.data_ptr(), X.data_ptr(), Y.data_ptr())
        X_out.append(X)
        Y_out.append(Y)
    return iters


def train(mlp: "bgk.MLP", X, Y, iters=2000, batch=4096, lr=1e-3, seed=0, lr_final=None):
    """Adam on random mini-batches of the rows of (X, Y); returns the loss history."""
    import torch
    n = X.shape[0]
    mlp.fit_norm(X.data_ptr(), Y.data_ptr(), n)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    xb = torch.empty((batch, X.shape[1]), dtype=torch.float32, device="cuda")
    yb = torch.empty((batch, Y.shape[1]), dtype=torch.float32, device="cuda")
    losses = []
    for k in range(iters):
        idx = torch.randint(0, n, (batch,), generator=gen, device="cuda")
        torch.index_select(X, 0, idx, out=xb)
        torch.index_select(Y, 0, idx, out=yb)
        torch.cuda.synchronize()
        rate = lr if lr_final is None else lr * (lr_final / lr) ** (k / max(1, iters - 1))
        losses.append(mlp.train_step(xb.data_ptr(), yb.data_ptr(), batch, rate))
    return np.array(losses)
