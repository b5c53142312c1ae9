"""TT entry evaluation and its exact gradient (test infrastructure only).

Entry formula (Section 2.3): a(i_1..i_d) = G_1[i_1] G_2[i_2] ... G_d[i_d],
where G_k[i_k] is the r_{k-1} x r_k slice of core k at mode index i_k.

For a loss L = sum_e g_e a(i^e) the gradient of slice G_k[i] is
  dL/dG_k[i] = sum_{e: i^e_k = i} g_e * L_{k-1}(e)^T R_{k+1}(e)
with the left partial product L_{k-1} = G_1[i_1]..G_{k-1}[i_{k-1}] (1 x r_{k-1})
and the right one R_{k+1} = G_{k+1}[i_{k+1}]..G_d[i_d] (r_k x 1).
"""
from __future__ import annotations

import numpy as np


def tt_eval_at(cores, idx):
    """a(i^e) for every column e of idx (d, m), in FP64, one entry at a time."""
    idx = np.asarray(idx, dtype=np.int64)
    m = idx.shape[1]
    out = np.empty(m)
    for e in range(m):
        v = np.ones((1, 1))
        for k, G in enumerate(cores):
            v = v @ G[:, idx[k, e], :].astype(np.float64)
        out[e] = v[0, 0]
    return out


def tt_eval_at_batched(cores, idx):
    """Same values, vectorised over entries (a batch of vector-matrix chains)."""
    idx = np.asarray(idx, dtype=np.int64)
    v = np.ones((idx.shape[1], 1))
    for k, G in enumerate(cores):
        v = np.einsum("ea,aeb->eb", v, G[:, idx[k], :].astype(np.float64))
    return v[:, 0]


def tt_eval_grad(cores, idx, g):
    """dL/dG_k for L = sum_e g[e] * a(i^e), by the closed form in the module docstring."""
    idx = np.asarray(idx, dtype=np.int64)
    g = np.asarray(g, dtype=np.float64)
    d = len(cores)
    m = idx.shape[1]
    cores = [G.astype(np.float64) for G in cores]
    # left partials L[k] = product of slices 0..k-1, shape (m, r_k)
    L = [np.ones((m, 1))]
    for k in range(d - 1):
        L.append(np.einsum("ea,aeb->eb", L[-1], cores[k][:, idx[k], :]))
    # right partials Rp[k] = product of slices k..d-1, shape (m, r_{k-1}); Rp[d] = ones
    Rp = [None] * (d + 1)
    Rp[d] = np.ones((m, 1))
    for k in range(d - 1, 0, -1):
        Rp[k] = np.einsum("aeb,eb->ea", cores[k][:, idx[k], :], Rp[k + 1])
    grads = []
    for k in range(d):
        dG = np.zeros_like(cores[k])
        contrib = g[:, None, None] * L[k][:, :, None] * Rp[k + 1][:, None, :]
        np.add.at(dG, (slice(None), idx[k], slice(None)), np.transpose(contrib, (1, 0, 2)))
        grads.append(dG)
    return grads


def tt_fit_loss(cores, idx, vals):
    """L = 1/2 sum_e (a(i^e) - v_e)^2 over the given entries (math.fsum of the squares)."""
    import math
    r = tt_eval_at_batched(cores, idx) - np.asarray(vals, dtype=np.float64)
    return 0.5 * math.fsum((r * r).tolist())


def tt_fit_gd(cores, idx, vals, steps, lr):
    """Fixed-rank fitting of a TT to entries (the completion use of fixed-rank TTs,
    Section 3.4) by plain gradient descent with the adjoint of the entry formula:
    every step evaluates the residual r_e = a(i^e) - v_e, takes the gradient of
    L = 1/2 sum r_e^2, which is the adjoint with upstream weights g_e = r_e, and moves
    all cores at once, G_k <- G_k - lr dL/dG_k.  Returns the new cores (FP64) and the
    steps + 1 losses (before every step and after the last)."""
    cores = [np.array(G, dtype=np.float64, copy=True) for G in cores]
    v = np.asarray(vals, dtype=np.float64)
    losses = []
    for _ in range(steps):
        r = tt_eval_at_batched(cores, idx) - v
        losses.append(tt_fit_loss(cores, idx, v))
        grads = tt_eval_grad(cores, idx, r)
        cores = [G - lr * dG for G, dG in zip(cores, grads)]
    losses.append(tt_fit_loss(cores, idx, v))
    return cores, losses
