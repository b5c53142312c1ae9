"""Fixed-rank TT fitting by gradient descent with the adjoint (tt_fit_gd) through
the C ABI against the oracle (oracle.tteval.tt_fit_gd) on seeded inputs.

Bars: FP64 trajectories agree with the oracle's to 1e-10 relative (losses) and
1e-10 of the largest core entry (cores) after 20 steps; the sums and the atomic
accumulation of the adjoint only reorder FP64 roundings.  FP32 cores: losses
within 1e-4 relative of the FP64 oracle's.  The closed-form and exact cases hold to
rounding or bit for bit."""
import numpy as np
import pytest
import torch

from oracle import tteval as T
from paper_1908_02721_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1908_02721_gb300 import fasttt
    return fasttt


def _problem(dims, ranks, m, seed, noise=0.1):
    planted = W.random_tt(dims, ranks, seed=seed)
    rng = np.random.Generator(np.random.Philox(key=seed + 1))
    idx = np.stack([rng.integers(0, n, m) for n in dims]).astype(np.int32)
    vals = T.tt_eval_at_batched(planted, idx)
    start = [G + noise * rng.standard_normal(G.shape) for G in planted]
    return start, idx, vals


def _run(F, cores, idx, vals, steps, lr, dtype):
    dev = [torch.from_numpy(np.ascontiguousarray(G)).to("cuda", dtype) for G in cores]
    losses = F.tt_fit_gd(dev, torch.from_numpy(idx), torch.from_numpy(vals), steps, lr)
    return [G.cpu().double().numpy() for G in dev], losses


def test_fp64_trajectory_matches_the_oracle(F):
    start, idx, vals = _problem([6, 5, 7, 4], [1, 2, 3, 2, 1], 300, seed=11)
    got, losses = _run(F, start, idx, vals, 20, 2e-3, torch.float64)
    ref, ref_losses = T.tt_fit_gd(start, idx, vals, 20, 2e-3)
    assert np.allclose(losses, ref_losses, rtol=1e-10, atol=0)
    for G, R in zip(got, ref):
        assert np.max(np.abs(G - R)) <= 1e-10 * np.max(np.abs(R))
    assert losses[-1] < losses[0]


def test_fp32_cores(F):
    start, idx, vals = _problem([6, 5, 7, 4], [1, 2, 3, 2, 1], 300, seed=13)
    start32 = [G.astype(np.float32).astype(np.float64) for G in start]
    vals32 = vals.astype(np.float32)
    _, losses = _run(F, start32, idx, vals32, 20, 2e-3, torch.float32)
    _, ref_losses = T.tt_fit_gd(start32, idx, vals32.astype(np.float64), 20, 2e-3)
    assert np.allclose(losses, ref_losses, rtol=1e-4, atol=0)


def test_larger_entry_set(F):
    """3e4 entries of an 8-way 100^8 rank-8 TT (ranks and mode sizes of the Zipf
    workload), five steps, FP64."""
    start, idx, vals = _problem([100] * 8, [1] + [8] * 7 + [1], 30_000, seed=17, noise=0.02)
    start = [G / np.sqrt(8.0) for G in start]
    vals = T.tt_eval_at_batched([G for G in start], idx) + 0.01   # a nearby target
    got, losses = _run(F, start, idx, vals, 5, 1e-4, torch.float64)
    ref, ref_losses = T.tt_fit_gd(start, idx, vals, 5, 1e-4)
    assert np.allclose(losses, ref_losses, rtol=1e-10, atol=0)
    for G, R in zip(got, ref):
        assert np.max(np.abs(G - R)) <= 1e-10 * np.max(np.abs(R))


def test_one_mode_closed_form(F):
    rng = np.random.default_rng(19)
    g0 = rng.standard_normal((1, 12, 1))
    obs = np.array([[0, 2, 3, 7, 11]], dtype=np.int32)
    v = rng.standard_normal(5)
    got, losses = _run(F, [g0], obs, v, 7, 0.3, torch.float64)
    want = g0[0, :, 0].copy()
    want[obs[0]] = v + 0.7 ** 7 * (g0[0, obs[0], 0] - v)
    assert np.allclose(got[0][0, :, 0], want, rtol=0, atol=1e-14)
    base = 0.5 * np.sum((g0[0, obs[0], 0] - v) ** 2)
    assert np.allclose(losses, base * 0.49 ** np.arange(8), rtol=1e-13, atol=0)


def test_exact_fit_is_a_fixed_point(F):
    x = np.array([1.0, -2.0, 3.0, 4.0])
    y = np.array([2.0, 5.0, -1.0])
    cores = [x[None, :, None], y[None, :, None]]
    idx = np.array([[0, 1, 2, 3, 3], [0, 2, 1, 1, 0]], dtype=np.int32)
    v = x[idx[0]] * y[idx[1]]
    got, losses = _run(F, cores, idx, v, 5, 0.5, torch.float64)
    assert np.array_equal(losses, np.zeros(6))
    assert all(np.array_equal(a, b) for a, b in zip(got, cores))


def test_zero_steps_and_bad_arguments(F):
    start, idx, vals = _problem([4, 5, 3], [1, 2, 2, 1], 40, seed=23)
    got, losses = _run(F, start, idx, vals, 0, 0.1, torch.float64)
    assert losses.shape == (1,)
    assert np.isclose(losses[0], T.tt_fit_loss(start, idx, vals), rtol=1e-13)
    assert all(np.array_equal(a, b) for a, b in zip(got, start))
    bad = idx.copy()
    bad[1, 3] = 5
    with pytest.raises(F.FastTTError) as e:
        _run(F, start, bad, vals, 2, 0.1, torch.float64)
    assert e.value.code == F.EINVAL
    with pytest.raises(F.FastTTError):
        _run(F, start, idx, vals, -1, 0.1, torch.float64)
