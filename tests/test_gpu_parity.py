"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer outputs (group maps, r~, R, p, middle COO, Depar classes) and copied
floating-point factors (prefactors, normalised values) must match bit for bit.
Floating-point results: singular values within 1e-12 relative, TT products
within 1e-12 relative Frobenius error (computed as a TT difference, Lemma 2).
"""
import math

import numpy as np
import pytest
import torch

from oracle import dense as D
from oracle import fasttt as O
from oracle import tteval as OT
from paper_1908_02721_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def F():
    from paper_1908_02721_gb300 import fasttt
    return fasttt


def _np(t):
    return t.detach().cpu().numpy()


def _cases():
    return [
        W.random_sparse([4, 5, 3], 25, 11, "normal"),
        W.random_sparse([3, 4, 5, 2], 40, 12, "normal"),
        W.random_sparse([6, 6, 6], 80, 13, "uniform"),
        W.random_sparse([2, 3, 4, 3, 2], 60, 14, "normal"),
        W.random_sparse([5, 7], 12, 15, "signed"),
        W.random_sparse([3, 3, 3, 3], 81, 16, "normal"),
        W.random_sparse([9, 8, 7, 6], 700, 17, "normal"),
        W.random_sparse([40, 30, 20], 3000, 18, "uniform"),
    ]


# ---------------------------------------------------------------- S2-S5: bit-exact grouping

@pytest.mark.parametrize("case", range(8))
def test_grouping_bit_exact(F, case):
    w = _cases()[case]
    for p in range(1, w.d + 1):
        tt = F.fasttt_decompose(w.idx, w.vals, w.dims, 0.0, p=p, stage="exact", keep_intermediates=True)
        ex = O.exact_tt(w.idx.astype(np.int64), w.vals, w.dims, p)
        st = tt.stats
        assert st["p"] == p and st["R"] == ex.R
        assert st["rt"] == ex.rt
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
        tt.free()


@pytest.mark.parametrize("case", [0, 1, 3, 6, 7])
def test_alg9_split_selection(F, case):
    w = _cases()[case]
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, 0.0, stage="exact")
    Rs = [O.fiber_ids(w.idx.astype(np.int64), q)[0] for q in range(1, w.d + 1)]
    p, _ = O.select_p(w.dims, Rs)
    assert tt.stats["Rs"] == Rs
    assert tt.stats["p"] == p


def _golden(name):
    import os
    rec, rows = {}, {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        if not line.strip() or line.startswith("#"):
            continue
        tag, *rest = line.split()
        rows.setdefault(tag, []).append(rest)
    return rows


def test_grouping_hand_worked_example_on_gpu(F):
    """The hand-derived ids, P-core maps, r~, R and middle unfolding of
    tests/golden/grouping_example.txt, bit for bit."""
    g = _golden("grouping_example.txt")
    dims = [int(x) for x in g["DIMS"][0]]
    p = int(g["P"][0][0])
    idx = np.ascontiguousarray(np.array([[int(x) for x in r[:4]] for r in g["NZ"]], dtype=np.int32).T)
    vals = np.array([float(r[4]) for r in g["NZ"]])
    tt = F.fasttt_decompose(idx, vals, dims, 0.0, p=p, stage="exact", keep_intermediates=True)
    ints = lambda tag: [int(x) for x in g[tag][0]]
    assert tt.stats["R"] == ints("R")[0] and tt.stats["rt"] == ints("RT")
    l1, l2, r4 = ints("LEFT1"), ints("LEFT2"), ints("RIGHT4")
    assert _np(tt.array("left_parent", 1)).tolist() == l1[:2] and _np(tt.array("left_index", 1)).tolist() == l1[2:]
    assert _np(tt.array("left_parent", 2)).tolist() == l2[:4] and _np(tt.array("left_index", 2)).tolist() == l2[4:]
    assert _np(tt.array("right_index", 4)).tolist() == r4[:3] and _np(tt.array("right_child", 4)).tolist() == r4[3:]
    mid = sorted((int(r[0]), int(r[1]), float(r[2])) for r in g["MID"])
    got = list(zip(_np(tt.array("mid_row")).tolist(), _np(tt.array("mid_col")).tolist(),
                   _np(tt.array("mid_val")).tolist()))
    assert got == mid
    tt.free()


def test_value_depar_hand_worked_example_on_gpu(F):
    """The 6 x 5 matrix of tests/golden/depar_example.txt as a 2-way tensor at p = 1 (its
    middle unfolding is the matrix itself): classes, prefactors, D' and Lambda as
    derived by hand, bit for bit."""
    g = _golden("depar_example.txt")
    idx = np.ascontiguousarray(np.array([[int(r[0]), int(r[1])] for r in g["X"]], dtype=np.int32).T)
    vals = np.array([float(r[2]) for r in g["X"]])
    tt = F.fasttt_decompose(idx, vals, [6, 5], 0.1, p=1, keep_intermediates=True)
    ints = lambda tag: [int(x) for x in g[tag][0]]
    flts = lambda tag: [float(x) for x in g[tag][0]]
    assert _np(tt.array("row_id")).tolist() == ints("ROWS")
    assert _np(tt.array("row_class")).tolist() == ints("ROW_CLASS")
    assert _np(tt.array("row_pref")).tolist() == flts("ROW_PREF")
    assert _np(tt.array("col_id")).tolist() == ints("COLS")
    assert _np(tt.array("col_class")).tolist() == ints("COL_CLASS")
    assert _np(tt.array("col_pref")).tolist() == flts("COL_PREF")
    dp = sorted(zip(_np(tt.array("dp_row")).tolist(), _np(tt.array("dp_col")).tolist(),
                    _np(tt.array("dp_val")).tolist()))
    assert dp == sorted((int(r[0]), int(r[1]), float(r[2])) for r in g["DP"])
    assert _np(tt.array("lam_s")).tolist() == flts("LAM_S")
    assert _np(tt.array("lam_t")).tolist() == flts("LAM_T")
    tt.free()


# ---------------------------------------------------------------- S6: bit-exact value Depar

def _depar_check(F, w, p):
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, 0.1, p=p, keep_intermediates=True)
    ex = O.exact_tt(w.idx.astype(np.int64), w.vals, w.dims, p)
    dp = O.value_depar(ex.mid_rows, ex.mid_cols, ex.mid_vals)
    assert tt.stats["beta_r"] == dp.beta_r and tt.stats["beta_c"] == dp.beta_c
    assert np.array_equal(_np(tt.array("row_id")), dp.row_ids)
    assert np.array_equal(_np(tt.array("row_class")), dp.row_class)
    assert np.array_equal(_np(tt.array("row_pref")), dp.row_pref)
    assert np.array_equal(_np(tt.array("col_id")), dp.col_ids)
    assert np.array_equal(_np(tt.array("col_class")), dp.col_class)
    assert np.array_equal(_np(tt.array("col_pref")), dp.col_pref)
    g_r, g_c, g_v = _np(tt.array("dp_row")), _np(tt.array("dp_col")), _np(tt.array("dp_val"))
    o1 = np.lexsort((g_r, g_c))
    o2 = np.lexsort((dp.dp_rows, dp.dp_cols))
    assert np.array_equal(g_r[o1], dp.dp_rows[o2])
    assert np.array_equal(g_c[o1], dp.dp_cols[o2])
    assert np.array_equal(g_v[o1], dp.dp_vals[o2])
    assert np.allclose(_np(tt.array("lam_s")), dp.lam_s, rtol=1e-15, atol=0)
    assert np.allclose(_np(tt.array("lam_t")), dp.lam_t, rtol=1e-15, atol=0)
    tt.free()


@pytest.mark.parametrize("case", range(8))
def test_value_depar_bit_exact(F, case):
    w = _cases()[case]
    for p in range(1, w.d + 1):
        _depar_check(F, w, p)


def test_value_depar_planted_parallel_rows(F):
    """Rows that are exact power-of-two multiples of each other must share a class."""
    rng = np.random.Generator(np.random.Philox(key=101))
    dims = [16, 8, 8]
    base = rng.standard_normal((4, 8))
    idx, vals = [], []
    for i0 in range(16):
        pat = base[i0 % 4]
        mult = [1.0, -2.0, 0.5, 8.0][i0 // 4]
        for i1 in range(8):
            for i2 in range(8):
                if (i1 + i2 + i0 % 4) % 3 == 0:
                    idx.append((i0, i1, i2))
                    vals.append(pat[i2] * mult * (1 + i1))
    idx = np.ascontiguousarray(np.array(idx, dtype=np.int32).T)
    w = W.Workload("planted", dims, idx, np.array(vals), 0.0)
    _depar_check(F, w, 1)
    _depar_check(F, w, 3)


# ---------------------------------------------------------------- S7-S12: full decomposition

def _cores_np(tt):
    return [_np(G) for G in tt.cores()]


def _full_check(F, w, eps, p=0, max_rank=0, rounding="static", depar=True):
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, eps, p=p, max_rank=max_rank, rounding=rounding,
                            depar_values=depar, keep_intermediates=True)
    res = O.fasttt(w.idx, w.vals, w.dims, eps, p=p, max_rank=max_rank, rounding=rounding, depar_values=depar)
    st = tt.stats
    assert st["p"] == res.p
    assert tt.ranks == res.ranks
    assert abs(st["norm2"] - res.norm2) <= 1e-14 * res.norm2
    for b, s in res.sigmas.items():
        g = _np(tt.array("sigma", b))
        assert g.size == s.size
        assert np.allclose(g, s, rtol=0, atol=TOL * s[0])
    nA = math.sqrt(res.norm2)
    diff = D.tt_diff_norm(_cores_np(tt), res.cores)
    assert diff <= TOL * nA, diff / nA
    assert abs(st["err2"] - res.err2) <= 1e-10 * max(res.err2, 1e-30) + 1e-24 * res.norm2
    tt.free()
    return res


@pytest.mark.parametrize("case", range(8))
@pytest.mark.parametrize("eps", [0.0, 1e-8, 0.1, 0.4])
def test_fasttt_matches_oracle(F, case, eps):
    w = _cases()[case]
    for p in range(1, w.d + 1):
        _full_check(F, w, eps, p=p)
    _full_check(F, w, eps, p=0)


@pytest.mark.parametrize("case", [1, 5, 6])
def test_variants_match_oracle(F, case):
    w = _cases()[case]
    for p in (1, 2, w.d):
        _full_check(F, w, 0.2, p=p, rounding="dynamic")
        _full_check(F, w, 0.0, p=p, max_rank=3)
        _full_check(F, w, 1e-6, p=p, depar=False)


def test_exact_small_eps0(F):
    """4-way 20^4, 1e3 nnz, eps = 0: exact TT, ranks = unfolding ranks."""
    w = W.exact_small()
    res = _full_check(F, w, w.eps)
    A = D.full_from_coo(w.idx, w.vals, w.dims)
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, 0.0)
    B = D.tt_full(_cores_np(tt))
    assert np.linalg.norm(A - B) <= 1e-13 * np.linalg.norm(A)
    assert tt.ranks == [1] + [int(np.linalg.matrix_rank(D.unfold(A, k))) for k in (1, 2, 3)] + [1]
    assert res.ranks == tt.ranks


@pytest.mark.parametrize("coeffs", ["pattern", "random"])
def test_fdm_table2_on_gpu(F, coeffs):
    """Table 2 structure (n = 20): R = 1920, r~ = 58, 58, r = 2, 2 (pattern) / 58, 58 (random)."""
    w = W.fdm7(20, coeffs)
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, w.eps, p=2)
    assert tt.stats["R"] == 1920
    assert tt.stats["rt"][1:3] == [58, 58]
    assert tt.ranks[1:3] == ([2, 2] if coeffs == "pattern" else [58, 58])
    _full_check(F, w, w.eps, p=2)


def test_float32_values_upcast_exactly(F):
    w = W.random_sparse([6, 5, 7, 4], 300, 19, "normal")
    v32 = w.vals.astype(np.float32)
    tt = F.fasttt_decompose(w.idx, torch.from_numpy(v32), w.dims, 1e-3, p=2, keep_intermediates=True)
    res = O.fasttt(w.idx, v32, w.dims, 1e-3, p=2)
    assert tt.ranks == res.ranks
    assert D.tt_diff_norm(_cores_np(tt), res.cores) <= TOL * math.sqrt(res.norm2)


# ---------------------------------------------------------------- input errors

def test_input_errors(F):
    with pytest.raises(F.FastTTError) as e:
        F.fasttt_decompose(np.array([[0, 1, 1], [2, 0, 0]]), np.array([1.0, 2.0, 3.0]), [2, 3], 0.1)
    assert e.value.code == F.EDUP
    with pytest.raises(F.FastTTError) as e:
        F.fasttt_decompose(np.array([[0, 2], [0, 0]]), np.array([1.0, 2.0]), [2, 3], 0.1)
    assert e.value.code == F.EINVAL
    with pytest.raises(F.FastTTError) as e:
        F.fasttt_decompose(np.array([[0, 1], [0, 0]]), np.array([1.0, np.inf]), [2, 3], 0.1)
    assert e.value.code == F.EINVAL
    with pytest.raises(F.FastTTError) as e:
        F.fasttt_decompose(np.array([[0, 1], [0, 0]]), np.array([0.0, -0.0]), [2, 3], 0.1)
    assert e.value.code == F.EINVAL
    tt = F.fasttt_decompose(np.array([[0, 1, 1], [0, 0, 2]]), np.array([1.0, 0.0, 2.0]), [2, 3], 0.0)
    assert tt.stats["dropped"] == 1
    A = np.zeros((2, 3)); A[0, 0] = 1.0; A[1, 2] = 2.0
    assert np.allclose(D.tt_full(_cores_np(tt)), A, atol=1e-15)


def test_allocation_failure_is_reported_and_recoverable(F):
    w = _cases()[6]
    for n in (1, 5, 40):
        F.debug_fail_alloc_after(n)
        with pytest.raises(F.FastTTError) as e:
            F.fasttt_decompose(w.idx, w.vals, w.dims, 0.1)
        assert e.value.code == F.ENOMEM
    F.debug_fail_alloc_after(0)
    _full_check(F, w, 0.1)


# ---------------------------------------------------------------- E3: evaluation and adjoint

def _random_tt(dims, ranks, seed, dtype=np.float64):
    rng = np.random.Generator(np.random.Philox(key=seed))
    return [(rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) / math.sqrt(ranks[k])).astype(dtype)
            for k in range(len(dims))]


@pytest.mark.parametrize("ranks", [[1, 3, 4, 2, 1], [1, 40, 33, 64, 1], [1, 100, 1, 70, 1]])
def test_tt_eval_and_adjoint(F, ranks):
    dims = [7, 9, 5, 6]
    cores = _random_tt(dims, ranks, 201)
    rng = np.random.Generator(np.random.Philox(key=202))
    m = 3000
    idx = np.stack([rng.integers(0, n, m) for n in dims]).astype(np.int32)
    g = rng.standard_normal(m)
    tc = [torch.from_numpy(c).cuda() for c in cores]
    a = _np(F.tt_eval_at(tc, idx))
    ref = OT.tt_eval_at_batched(cores, idx)
    assert np.allclose(a, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    grads_ref = OT.tt_eval_grad(cores, idx, g)
    for recompute in (False, True):
        grads = F.tt_eval_backward(tc, idx, torch.from_numpy(g).cuda(), recompute=recompute)
        for gg, gr in zip(grads, grads_ref):
            assert np.allclose(_np(gg), gr, rtol=0, atol=1e-12 * max(1.0, np.abs(gr).max()))


def test_autograd_function_and_finite_differences(F):
    dims, ranks = [5, 4, 6], [1, 3, 2, 1]
    cores = [torch.from_numpy(c).cuda().requires_grad_(True) for c in _random_tt(dims, ranks, 301)]
    rng = np.random.Generator(np.random.Philox(key=302))
    idx = torch.from_numpy(np.stack([rng.integers(0, n, 50) for n in dims]).astype(np.int32)).cuda()
    w = torch.from_numpy(rng.standard_normal(50)).cuda()
    loss = (F.tt_eval(cores, idx) * w).sum()
    loss.backward()
    h = 1e-6
    for k in range(3):
        for flat in range(0, cores[k].numel(), 3):
            cp = [c.detach().clone() for c in cores]
            cm = [c.detach().clone() for c in cores]
            cp[k].view(-1)[flat] += h
            cm[k].view(-1)[flat] -= h
            fd = ((F.tt_eval_at(cp, idx) * w).sum() - (F.tt_eval_at(cm, idx) * w).sum()).item() / (2 * h)
            assert abs(fd - cores[k].grad.view(-1)[flat].item()) <= 1e-6 * max(1.0, abs(fd))


def test_eval_float32_and_bad_index(F):
    dims, ranks = [4, 4, 4], [1, 5, 5, 1]
    cores = _random_tt(dims, ranks, 401, np.float32)
    idx = np.array([[0, 3], [1, 2], [3, 0]], dtype=np.int32)
    tc = [torch.from_numpy(c).cuda() for c in cores]
    a = _np(F.tt_eval_at(tc, idx))
    assert np.allclose(a, OT.tt_eval_at(cores, idx), rtol=1e-5, atol=1e-6)
    with pytest.raises(F.FastTTError) as e:
        F.tt_eval_at(tc, np.array([[0], [1], [4]], dtype=np.int32))
    assert e.value.code == F.EINVAL


def test_banded_qtt_m10(F):
    """2^10 x 2^10 band + off-band matrix as a 10-way QTT tensor (eps = 1e-6): grouping
    bit-exact (Alg. 9 picks p), ranks equal, products within 1e-12."""
    w = W.banded_qtt(10)
    res = _full_check(F, w, w.eps)
    assert max(res.ranks) > 900    # the random off-band entries keep the ranks high


def test_uniform5_full_size_properties(F):
    """The bench workload (50^5, 1e5 nonzeros, eps = 1e-8) at full size: ranks, r~, beta and R
    against the oracle's grouping, and B reproduces A at sampled nonzeros and zeros."""
    w = W.uniform5()
    tt = F.fasttt_decompose(w.idx, w.vals, w.dims, w.eps)
    ex = O.exact_tt(w.idx.astype(np.int64), w.vals, w.dims, tt.stats["p"])
    Rs = [O.fiber_ids(w.idx.astype(np.int64), q)[0] for q in range(1, w.d + 1)]
    p, _ = O.select_p(w.dims, Rs)
    assert tt.stats["p"] == p and tt.stats["Rs"] == Rs and tt.stats["rt"] == ex.rt
    dp = O.value_depar(ex.mid_rows, ex.mid_cols, ex.mid_vals)
    assert (tt.stats["beta_r"], tt.stats["beta_c"]) == (dp.beta_r, dp.beta_c)
    # every bond is well conditioned and eps = 1e-8: the TT keeps the full unfolding ranks
    assert tt.ranks == [1, 50, 2500, 2500, 50, 1]
    cores = tt.cores()
    rng = np.random.Generator(np.random.Philox(key=701))
    pick = rng.choice(w.nnz, 20000, replace=False)
    a = _np(F.tt_eval_at(cores, w.idx[:, pick]))
    nA = math.sqrt(tt.stats["norm2"])
    assert np.linalg.norm(a - w.vals[pick]) <= 1e-8 * nA
    zeros = np.stack([rng.integers(0, 50, 20000) for _ in range(5)]).astype(np.int32)
    lin = lambda I: sum(I[k].astype(np.int64) * 50 ** (4 - k) for k in range(5))
    zeros = zeros[:, ~np.isin(lin(zeros), lin(w.idx))]
    z = _np(F.tt_eval_at(cores, zeros))
    assert np.linalg.norm(z) <= 1e-8 * nA
    # cores 2..d are right-orthonormal after Alg. 6 (second sweep / QR sweep)
    for k in range(2, 6):
        G = cores[k - 1].reshape(cores[k - 1].shape[0], -1)
        I = G @ G.T
        assert torch.allclose(I, torch.eye(I.shape[0], dtype=I.dtype, device=I.device), atol=1e-12)
    tt.free()




# ---------------------------------------------------------------- Alg. 8 on the hand-worked input

def _read_alg8_golden():
    import os
    rows = []
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "alg8_example.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("row", _read_alg8_golden())
def test_alg8_hand_worked_on_gpu(F, row):
    """Alg. 8 (and the static schedule) on the superdiagonal tensor whose ranks were
    derived by hand (tests/golden/alg8_example.txt): ranks and err2 exact, products
    within 1e-12 of the oracle's."""
    s = np.array([8.0, 4.0, 2.0, 1.0, 0.5])
    idx = np.tile(np.arange(5, dtype=np.int32), (4, 1))
    dims = [5, 5, 5, 5]
    eps = 1.2 / math.sqrt(float(np.sum(s * s)))
    p, rounding = int(row[0]), row[1]
    tt = F.fasttt_decompose(idx, s, dims, eps, p=p, rounding=rounding)
    assert tt.ranks == [int(x) for x in row[2:7]]
    assert abs(tt.stats["err2"] - float(row[7])) <= 1e-12
    res = O.fasttt(idx, s, dims, eps, p=p, rounding=rounding)
    assert D.tt_diff_norm(_cores_np(tt), res.cores) <= TOL * math.sqrt(res.norm2)
    tt.free()
