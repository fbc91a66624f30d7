"""Training and use of the learned proposal (host orchestration only).

The network, its gradient and the optimiser run in the library's kernels
(maxsat_mp_*); this module batches formulas into contexts, labels them with
the solver's own best assignments, loops over epochs, and turns the
network's output into the chains' initial distribution (maxsat_reset_probs).
"""
from __future__ import annotations

import numpy as np

from . import binding as ms


def _chunks(seq, size):
    for i in range(0, len(seq), size):
        yield seq[i:i + size]


def label_with_solver(formulas, params, restarts=256, steps=200, seed=0, batch=256, stream=None):
    """Best assignment of each formula ((n, off, lits, weights) tuples) after
    `steps` Gibbs rounds of `restarts` chains, solved `batch` formulas per
    context."""
    labels = []
    for chunk in _chunks(list(formulas), batch):
        ctx = ms.maxsat_create_batch(chunk, params, stream)
        _, assign = ms.maxsat_solve(ctx, restarts, steps, seed)
        vb = ctx.var_base
        labels += [assign[vb[k]:vb[k + 1]].copy() for k in range(len(chunk))]
        ms.maxsat_destroy(ctx)
    return labels


def train(model, formulas, labels, params, epochs=4, batch=64, lr=3e-3, seed=0, stream=None):
    """Adam on the mean binary cross entropy against the labels, one step per
    batch of `batch` formulas (a batch context), batches in a seeded random
    order every epoch. Returns the loss of every step."""
    import torch
    groups = []
    for idx in _chunks(list(range(len(formulas))), batch):
        ctx = ms.maxsat_create_batch([formulas[i] for i in idx], params, stream)
        y = torch.tensor(np.concatenate([labels[i] for i in idx]).astype(np.uint8), device="cuda")
        groups.append((ctx, y))
    torch.cuda.synchronize()  # the labels are on the device before any library stream uses them
    rng = np.random.default_rng(seed)
    losses = []
    for _ in range(epochs):
        for g in rng.permutation(len(groups)):
            ctx, y = groups[g]
            losses.append(ms.maxsat_mp_gradient(model, ctx, y))
            ms.maxsat_mp_adam(model, ctx, lr)
    for ctx, _ in groups:
        ms.maxsat_destroy(ctx)
    return losses


def propose(model, ctx, stream=None):
    """p(x_v = 1) for every variable of the context's formula (host FP32)."""
    import torch
    p = torch.zeros(ctx.n, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    ms.maxsat_mp_forward(model, ctx, p)
    torch.cuda.synchronize()
    return p.cpu().numpy()
