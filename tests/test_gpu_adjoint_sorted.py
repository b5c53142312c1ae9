"""Entry evaluation and its adjoint on the index-sorted batched path (ranks 16 to
1024), against the FP64 oracle's entry formula and closed-form gradient (Sec. 2.3).

The cases cross the 64-wide tiles (ranks 16..70), put most entries on one hot
index per mode (as Zipf-distributed data does) next to many indices with one or
two entries (tiles that span several runs), and run the stored and the
recomputed (checkpointed) left partials.  Bars: FP64 within 1e-12 of the largest
reference value; FP32 within 1e-4 relative (FP32 products, FP32 chunk sums, FP64
cross-chunk sums).  The gradients are deterministic: two calls give the same bits.
"""
import math

import numpy as np
import pytest
import torch

from oracle import tteval as OT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1908_02721_gb300 import fasttt
    return fasttt


def _tt(dims, ranks, seed):
    rng = np.random.Generator(np.random.Philox(key=seed))
    return [rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) / math.sqrt(ranks[k]) for k in range(len(dims))]


def _skewed_indices(dims, m, seed):
    """40 % of the entries on index 0 of every mode, the rest uniform."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    idx = np.stack([rng.integers(0, n, m) for n in dims])
    hot = rng.random((len(dims), m)) < 0.4
    idx[hot] = 0
    return np.ascontiguousarray(idx.astype(np.int32))


CASES = {
    "r16-70": ([7, 9, 5, 6, 8], [1, 16, 70, 33, 64, 1], 20000),
    "many-runs": ([3000, 40, 2500], [1, 24, 17, 1], 6000),
    "d2-r40": ([50, 60], [1, 40, 1], 5000),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_sorted_eval_and_adjoint_fp64(F, case):
    dims, ranks, m = CASES[case]
    cores = _tt(dims, ranks, 801)
    idx = _skewed_indices(dims, m, 802)
    g = np.random.Generator(np.random.Philox(key=803)).standard_normal(m)
    tc = [torch.from_numpy(c).cuda() for c in cores]
    a = F.tt_eval_at(tc, idx).cpu().numpy()
    ref = OT.tt_eval_at_batched(cores, idx)
    assert np.max(np.abs(a - ref)) <= 1e-12 * np.abs(ref).max()
    grads_ref = OT.tt_eval_grad(cores, idx, g)
    gd = torch.from_numpy(g).cuda()
    first = None
    for recompute in (False, True):
        grads = F.tt_eval_backward(tc, idx, gd, recompute=recompute)
        for gg, gr in zip(grads, grads_ref):
            assert np.max(np.abs(gg.cpu().numpy() - gr)) <= 1e-12 * max(1.0, np.abs(gr).max())
        if first is None:
            first = [x.clone() for x in grads]
    again = F.tt_eval_backward(tc, idx, gd, recompute=False)
    assert all(torch.equal(x, y) for x, y in zip(again, first))


def test_sorted_eval_and_adjoint_fp32(F):
    dims, ranks, m = CASES["r16-70"]
    cores = _tt(dims, ranks, 811)
    idx = _skewed_indices(dims, m, 812)
    g = np.random.Generator(np.random.Philox(key=813)).standard_normal(m)
    tc = [torch.from_numpy(c.astype(np.float32)).cuda() for c in cores]
    c32 = [c.astype(np.float32).astype(np.float64) for c in cores]
    a = F.tt_eval_at(tc, idx).cpu().numpy().astype(np.float64)
    ref = OT.tt_eval_at_batched(c32, idx)
    assert np.max(np.abs(a - ref)) <= 1e-4 * np.abs(ref).max()
    grads_ref = OT.tt_eval_grad(c32, idx, g.astype(np.float32).astype(np.float64))
    for recompute in (False, True):
        grads = F.tt_eval_backward(tc, idx, torch.from_numpy(g.astype(np.float32)).cuda(), recompute=recompute)
        for gg, gr in zip(grads, grads_ref):
            assert np.max(np.abs(gg.cpu().numpy().astype(np.float64) - gr)) <= 1e-4 * max(1.0, np.abs(gr).max())


def test_sorted_path_reports_bad_index(F):
    dims, ranks = [5, 6], [1, 20, 1]
    tc = [torch.from_numpy(c).cuda() for c in _tt(dims, ranks, 821)]
    idx = np.array([[0, 4], [2, 6]], dtype=np.int32)     # 6 is outside mode 2
    with pytest.raises(F.FastTTError) as e:
        F.tt_eval_at(tc, idx)
    assert e.value.code == F.EINVAL
    with pytest.raises(F.FastTTError) as e:
        F.tt_eval_backward(tc, idx, torch.ones(2, dtype=torch.float64, device="cuda"))
    assert e.value.code == F.EINVAL
