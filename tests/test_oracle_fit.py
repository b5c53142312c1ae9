"""Pins for the oracle's fixed-rank TT fitting by gradient descent with the adjoint
(oracle.tteval.tt_fit_gd), checked against closed forms and finite differences
rather than against the oracle's own formulas."""
import math

import numpy as np

from oracle import tteval as T


def test_one_mode_tt_has_the_closed_form_trajectory():
    """d = 1: a(i) = g_i, so each observed entry follows g_t = v + (1 - lr)^t (g_0 - v)
    and unobserved entries never move; L_t = 1/2 (1 - lr)^(2t) sum (g_0 - v)^2."""
    rng = np.random.default_rng(3)
    n, lr, steps = 12, 0.3, 7
    g0 = rng.standard_normal((1, n, 1))
    obs = np.array([0, 2, 3, 7, 11])
    v = rng.standard_normal(obs.size)
    cores, losses = T.tt_fit_gd([g0], obs[None, :], v, steps, lr)
    want = g0[0, :, 0].copy()
    want[obs] = v + (1 - lr) ** steps * (g0[0, obs, 0] - v)
    assert np.allclose(cores[0][0, :, 0], want, rtol=0, atol=1e-14)
    base = 0.5 * np.sum((g0[0, obs, 0] - v) ** 2)
    for t, L in enumerate(losses):
        assert math.isclose(L, base * (1 - lr) ** (2 * t), rel_tol=1e-13)


def test_step_is_minus_lr_times_the_loss_gradient():
    """(G_0 - G_1) / lr equals the central finite difference of the reported loss."""
    rng = np.random.default_rng(5)
    dims, ranks = [4, 3, 5], [1, 2, 3, 1]
    cores = [rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(3)]
    idx = np.stack([rng.integers(0, n, 25) for n in dims])
    v = rng.standard_normal(25)
    lr = 1e-3
    new, _ = T.tt_fit_gd(cores, idx, v, 1, lr)
    h = 1e-6
    for k in range(3):
        step = (cores[k] - new[k]) / lr
        for pos in [(0, 0, 0), tuple(s - 1 for s in cores[k].shape), (0, 1, 0)]:
            plus = [c.copy() for c in cores]
            minus = [c.copy() for c in cores]
            plus[k][pos] += h
            minus[k][pos] -= h
            fd = (T.tt_fit_gd(plus, idx, v, 0, lr)[1][0] - T.tt_fit_gd(minus, idx, v, 0, lr)[1][0]) / (2 * h)
            assert math.isclose(step[pos], fd, rel_tol=1e-6, abs_tol=1e-7)


def test_exact_fit_is_a_fixed_point():
    """Rank-1 TT with small integer factors reproduces integer data exactly: the
    residual, the loss and the gradient are exactly zero and nothing moves."""
    x = np.array([1.0, -2.0, 3.0, 4.0])
    y = np.array([2.0, 5.0, -1.0])
    cores = [x[None, :, None], y[None, :, None]]
    idx = np.array([[0, 1, 2, 3, 3], [0, 2, 1, 1, 0]])
    v = x[idx[0]] * y[idx[1]]
    new, losses = T.tt_fit_gd(cores, idx, v, 5, 0.5)
    assert losses == [0.0] * 6
    assert all(np.array_equal(a, b) for a, b in zip(new, cores))


def test_small_steps_decrease_the_loss():
    rng = np.random.default_rng(7)
    dims, ranks = [6, 5, 7, 4], [1, 2, 3, 2, 1]
    planted = [rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(4)]
    idx = np.stack([rng.integers(0, n, 200) for n in dims])
    v = T.tt_eval_at(planted, idx)
    start = [G + 0.1 * rng.standard_normal(G.shape) for G in planted]
    _, losses = T.tt_fit_gd(start, idx, v, 30, 2e-3)
    assert all(b < a for a, b in zip(losses, losses[1:]))
    assert losses[-1] < 0.5 * losses[0]
