"""tt_eval_backward_noalloc: the adjoint for callers that cannot allocate device
memory (the library uses its fixed scratch array instead).  Its result must
match tt_eval_backward's, on two calls in a row (the scratch keeps the previous
call's contents, which must not leak into the next result).

Kept in its own file, named to be collected last.
"""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _tt(dims, ranks, seed, dtype):
    rng = np.random.Generator(np.random.Philox(key=seed))
    return [torch.from_numpy((rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) / math.sqrt(ranks[k]))
                             .astype(dtype)).cuda() for k in range(len(dims))]


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 1e-5)])
def test_noalloc_backward_matches_allocating_entry_point(dtype, tol):
    from paper_1908_02721_gb300 import fasttt as F
    dims = [7, 9, 5, 6]
    rng = np.random.Generator(np.random.Philox(key=503))
    for call, ranks in enumerate([[1, 6, 12, 4, 1], [1, 30, 17, 45, 1]]):   # two calls in a row
        cores = _tt(dims, ranks, 501 + call, dtype)
        m = 5000
        idx = torch.from_numpy(np.stack([rng.integers(0, n, m) for n in dims]).astype(np.int32)).cuda()
        g = torch.from_numpy(rng.standard_normal(m).astype(dtype)).cuda()
        ref = F.tt_eval_backward(cores, idx, g, recompute=False)
        out = [torch.zeros_like(c) for c in cores]
        F.tt_eval_backward_noalloc(cores, idx, g, out)
        torch.cuda.synchronize()
        for a, b in zip(out, ref):
            scale = max(1.0, b.abs().max().item())
            assert (a - b).abs().max().item() <= tol * scale


def test_noalloc_reports_bad_index():
    from paper_1908_02721_gb300 import fasttt as F
    dims, ranks = [3, 4], [1, 2, 1]
    cores = _tt(dims, ranks, 601, np.float64)
    idx = torch.tensor([[0, 2], [1, 4]], dtype=torch.int32, device="cuda")   # 4 is out of range
    g = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FastTTError) as e:
        F.tt_eval_backward_noalloc(cores, idx, g, [torch.zeros_like(c) for c in cores])
    assert e.value.code == F.EINVAL
