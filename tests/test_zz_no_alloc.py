"""tt_eval_backward_noalloc: the adjoint for callers that cannot allocate device
memory, such as a framework that owns all device memory through its own pool or
a runtime with a fixed memory budget.  The library works in its fixed scratch
array instead.  Its gradients must match the FP64 oracle's closed form
(oracle.tteval.tt_eval_grad) and the allocating entry point's, on two calls in a
row: the scratch keeps the previous call's contents, which must not leak into
the next result.  One case has rank sums large enough that the scratch, not the
work, caps the number of warps (the grid sizing by what fits).

Kept in its own file, named to be collected last.
"""
import math

import numpy as np
import pytest
import torch

from oracle import tteval as OT

pytestmark = pytest.mark.gpu


def _tt(dims, ranks, seed, dtype):
    rng = np.random.Generator(np.random.Philox(key=seed))
    return [torch.from_numpy((rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) / math.sqrt(ranks[k]))
                             .astype(dtype)).cuda() for k in range(len(dims))]


def _check(F, cores, idx, g, tol):
    out = [torch.zeros_like(c) for c in cores]
    F.tt_eval_backward_noalloc(cores, idx, g, out)
    ref_lib = F.tt_eval_backward(cores, idx, g, recompute=False)
    torch.cuda.synchronize()
    ref = OT.tt_eval_grad([c.cpu().numpy().astype(np.float64) for c in cores], idx.cpu().numpy(),
                          g.cpu().numpy().astype(np.float64))
    for a, b, r in zip(out, ref_lib, ref):
        scale = max(1.0, float(np.abs(r).max()))
        assert float(np.abs(a.cpu().numpy().astype(np.float64) - r).max()) <= tol * scale
        assert (a - b).abs().max().item() <= tol * scale


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 1e-5)])
def test_noalloc_backward_matches_oracle(dtype, tol):
    from paper_1908_02721_gb300 import fasttt as F
    dims = [7, 9, 5, 6]
    rng = np.random.Generator(np.random.Philox(key=503))
    for call, ranks in enumerate([[1, 6, 12, 4, 1], [1, 30, 17, 45, 1]]):   # two calls in a row
        cores = _tt(dims, ranks, 501 + call, dtype)
        m = 2000
        idx = torch.from_numpy(np.stack([rng.integers(0, n, m) for n in dims]).astype(np.int32)).cuda()
        g = torch.from_numpy(rng.standard_normal(m).astype(dtype)).cuda()
        _check(F, cores, idx, g, tol)


def test_noalloc_grid_capped_by_scratch():
    """64 modes of size 2 at ranks 16: a warp's left partials take (1 + 63 x 16) x 8 B,
    so about 4,150 warps fit in the 32 MiB scratch, fewer than 6,000 entries would use."""
    from paper_1908_02721_gb300 import fasttt as F
    d, r = 64, 16
    dims = [2] * d
    ranks = [1] + [r] * (d - 1) + [1]
    cores = _tt(dims, ranks, 701, np.float64)
    rng = np.random.Generator(np.random.Philox(key=702))
    m = 6000
    idx = torch.from_numpy(np.stack([rng.integers(0, 2, m) for _ in dims]).astype(np.int32)).cuda()
    g = torch.from_numpy(rng.standard_normal(m)).cuda()
    _check(F, cores, idx, g, 1e-12)


def test_noalloc_reports_bad_index():
    from paper_1908_02721_gb300 import fasttt as F
    dims, ranks = [3, 4], [1, 2, 1]
    cores = _tt(dims, ranks, 601, np.float64)
    idx = torch.tensor([[0, 2], [1, 4]], dtype=torch.int32, device="cuda")   # 4 is out of range
    g = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FastTTError) as e:
        F.tt_eval_backward_noalloc(cores, idx, g, [torch.zeros_like(c) for c in cores])
    assert e.value.code == F.EINVAL
