"""Block-sparse bonds of the first SVD sweep (Alg. 6, bonds p+1..d-1) against
the FP64 oracle and against the dense route of the same library.

The block-sparse bond never forms G_k = W_{k-1} x_1 P_k: its Gram Z Z^T and its
projection U^T Z come from the nonzero blocks.  Its singular values come from
the Gram's eigenvalues, so they are compared on the squared scale the Gram
fixes: |s_gpu^2 - s^2| <= 2e-12 s_1^2 (the K-term FP64 sums of the Gram, K the
number of right groups, and the eigensolver's n u lambda error, both far below
that for the sizes here); TT products within 1e-12 relative.
"""
import math

import numpy as np
import pytest

from oracle import dense as D
from oracle import fasttt as O
from paper_1908_02721_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12
SQ_TOL = 2e-12
MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def F():
    from paper_1908_02721_gb300 import fasttt
    return fasttt


def _cores(tt):
    return [G.detach().cpu().numpy() for G in tt.cores()]


def _cases():
    return [
        W.random_sparse([9, 8, 7, 6], 700, 17, "normal"),
        W.random_sparse([40, 30, 20], 3000, 18, "uniform"),
        W.random_sparse([6, 7, 5, 6, 4], 1500, 21, "normal"),
        W.zipf_tt(seed=22, nnz=4000, d=6, n=9, rank=3, noise=1e-3, eps=1e-3, max_rank=12),
    ]


def _sparse_check(F, w, eps, p, max_rank=0):
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, eps, p=p, max_rank=max_rank, keep_intermediates=True,
                            sparse_sweep="sparse")
    res = O.fasttt(w.idx, w.vals, w.dims, eps, p=p, max_rank=max_rank)
    st = tt.stats
    assert st["p"] == p
    assert st["sparse_bonds"] == max(0, w.d - 1 - p)
    assert tt.ranks == res.ranks
    for b, s in res.sigmas.items():
        g = tt.array("sigma", b).cpu().numpy()
        assert g.size == s.size
        assert np.all(np.abs(g * g - s * s) <= SQ_TOL * s[0] * s[0]), b
    nA = math.sqrt(res.norm2)
    diff = D.tt_diff_norm(_cores(tt), res.cores)
    assert diff <= TOL * nA, diff / nA
    assert abs(st["err2"] - res.err2) <= 1e-9 * max(res.err2, 1e-30) + 1e-20 * res.norm2
    tt.free()


@pytest.mark.parametrize("case", range(4))
@pytest.mark.parametrize("eps", [1e-3, 0.1])
def test_sparse_bonds_match_oracle(F, case, eps):
    w = _cases()[case]
    for p in range(1, w.d - 1):
        _sparse_check(F, w, eps, p, max_rank=w.max_rank)


def test_sparse_bonds_with_rank_cap_and_dynamic_rounding(F):
    w = _cases()[2]
    _sparse_check(F, w, 0.0 + 1e-2, 1, max_rank=4)
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, 0.2, p=1, rounding="dynamic", sparse_sweep="sparse")
    res = O.fasttt(w.idx, w.vals, w.dims, 0.2, p=1, rounding="dynamic")
    assert tt.ranks == res.ranks
    assert D.tt_diff_norm(_cores(tt), res.cores) <= TOL * math.sqrt(res.norm2)
    tt.free()


def test_sparse_and_dense_routes_agree(F):
    w = W.random_sparse([12, 12, 12, 12, 12], 6000, 23, "normal")
    for p in (1, 2):
        a = F.fasttt_decompose(w.idx, w.vals, w.dims, 1e-2, p=p, sparse_sweep="sparse")
        b = F.fasttt_decompose(w.idx, w.vals, w.dims, 1e-2, p=p, sparse_sweep="dense")
        assert a.stats["sparse_bonds"] == w.d - 1 - p and b.stats["sparse_bonds"] == 0
        assert a.ranks == b.ranks
        nA = math.sqrt(a.stats["norm2"])
        assert D.tt_diff_norm(_cores(a), _cores(b)) <= TOL * nA
        a.free()
        b.free()


def test_sparse_bonds_mixed_precision(F):
    w = _cases()[2]
    res = O.fasttt(w.idx, w.vals, w.dims, 1e-3, p=1)
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, 1e-3, p=1, precision="mixed", sparse_sweep="sparse")
    assert tt.stats["sparse_bonds"] == w.d - 2
    assert tt.ranks == res.ranks
    assert D.tt_diff_norm(_cores(tt), res.cores) <= MIXED_TOL * math.sqrt(res.norm2)
    tt.free()


def test_sparse_sweep_mode_is_validated(F):
    w = _cases()[0]
    with pytest.raises(F.FastTTError):
        F.fasttt_decompose(w.idx, w.vals, w.dims, 0.1, sparse_sweep="blocks")


@pytest.mark.parametrize("case", [1, 3])
def test_rank_cap_partial_spectrum_matches_oracle(F, case):
    """A rank cap of 4 on block-sparse bonds whose Grams have order 120 (case 1) or 36
    (case 3), intermediates not kept: the FP64 tridiagonal route computes only the 20
    largest eigenvalues (the others stand in as their mean, from the trace) and the
    vectors kept.  Ranks, the TT and err2 (a tail
    sum, exact through the trace up to the Gram's rounding) match the oracle."""
    w = _cases()[case]
    for p in range(1, w.d - 1):
        tt = F.fasttt_decompose(w.idx, w.vals, w.dims, 1e-3, p=p, max_rank=4, sparse_sweep="sparse")
        res = O.fasttt(w.idx, w.vals, w.dims, 1e-3, p=p, max_rank=4)
        st = tt.stats
        assert st["sparse_bonds"] == max(0, w.d - 1 - p)
        assert tt.ranks == res.ranks
        nA = math.sqrt(res.norm2)
        assert D.tt_diff_norm(_cores(tt), res.cores) <= TOL * nA
        assert abs(st["err2"] - res.err2) <= 1e-9 * max(res.err2, 1e-30) + 1e-13 * res.norm2
        tt.free()
