"""Bit-exact grouping and value Depar at the full sizes of the two large-nnz
workloads, against the oracle (S2-S6: Alg. 4 with Alg. 5, Alg. 3):

  * the banded 2^20 x 2^20 matrix as a 20-way QTT (1.05e7 nonzeros), split at
    p = 10 (the split Alg. 9 takes for it), r~ up to about 1e6: its exact ranks are
    too large for the rounding, so the decomposition stops after value Depar;
  * the Zipf(1.2) 8-way 100^8 tensor (1e7 nonzeros, FP32 values upcast exactly),
    split at p = 1 as its decomposition is, r~ up to 9.4e6.

These sizes take wider keys (more radix passes) and r~ in the millions.  Group
maps, r~, R, the middle unfolding's COO, Depar classes, prefactors and D' must be
equal bit for bit; Lambda (an exactly rounded sum in the oracle, a sequential
sum on the GPU) within that sum's error bound for each class's size.  The oracle
takes a few minutes here.
"""
import numpy as np
import pytest

from oracle import fasttt as O
from paper_1908_02721_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def F():
    from paper_1908_02721_gb300 import fasttt
    return fasttt


def _np(t):
    return t.detach().cpu().numpy()


def _check(F, w, p):
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, w.eps, p=p, stage="depar", keep_intermediates=True)
    st = tt.stats
    idx, v, dropped = O.ingest(w.idx, w.vals.astype(np.float64), w.dims)
    assert st["nnz"] == idx.shape[1] and st["dropped"] == dropped
    ex = O.exact_tt(idx, v, w.dims, p)
    assert st["p"] == p and st["R"] == ex.R and st["rt"] == ex.rt
    for k in range(1, p):
        parent, i = ex.left[k - 1]
        assert np.array_equal(_np(tt.array("left_parent", k)), parent)
        assert np.array_equal(_np(tt.array("left_index", k)), i)
    for k in range(p + 1, w.d + 1):
        i, child = ex.right[k - p - 1]
        assert np.array_equal(_np(tt.array("right_index", k)), i)
        assert np.array_equal(_np(tt.array("right_child", k)), child)
    order = np.lexsort((ex.mid_cols, ex.mid_rows))
    assert np.array_equal(_np(tt.array("mid_row")), ex.mid_rows[order])
    assert np.array_equal(_np(tt.array("mid_col")), ex.mid_cols[order])
    assert np.array_equal(_np(tt.array("mid_val")), ex.mid_vals[order])
    dp = O.value_depar(ex.mid_rows, ex.mid_cols, ex.mid_vals)
    assert st["beta_r"] == dp.beta_r and st["beta_c"] == dp.beta_c
    for name, ref in (("row_id", dp.row_ids), ("row_class", dp.row_class), ("row_pref", dp.row_pref),
                      ("col_id", dp.col_ids), ("col_class", dp.col_class), ("col_pref", dp.col_pref)):
        assert np.array_equal(_np(tt.array(name)), ref), name
    g_r, g_c, g_v = _np(tt.array("dp_row")), _np(tt.array("dp_col")), _np(tt.array("dp_val"))
    o1, o2 = np.lexsort((g_r, g_c)), np.lexsort((dp.dp_rows, dp.dp_cols))
    assert np.array_equal(g_r[o1], dp.dp_rows[o2])
    assert np.array_equal(g_c[o1], dp.dp_cols[o2])
    assert np.array_equal(g_v[o1], dp.dp_vals[o2])
    # Lambda: the oracle's sum of squares is exactly rounded, the GPU's a sequential FMA sum
    # of a class's K squares in ascending member order (relative error <= (K - 1) u for
    # positive terms); the square root halves it, and each side rounds its square root (u each)
    for name, lam, cls, beta in (("lam_s", dp.lam_s, dp.row_class, dp.beta_r),
                                 ("lam_t", dp.lam_t, dp.col_class, dp.beta_c)):
        size = np.bincount(cls, minlength=beta)
        bound = (0.5 * np.maximum(size - 1, 0) + 2.0) * 2.0 ** -53
        got = _np(tt.array(name))
        assert np.all(np.abs(got - lam) <= bound * lam), name
    tt.free()


def test_banded_qtt_2p20_grouping_and_depar_bit_exact(F):
    _check(F, W.banded_qtt(20), 10)


def test_zipf_1e7_grouping_and_depar_bit_exact(F):
    _check(F, W.zipf_tt(), 1)
