"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: the paper's printed
numbers (Table 2, the Sec. 3.6 flop example), closed forms (Theorem of Sec. 3.1:
the rank-R TT is exact; quasi-permutation unfoldings are orthonormal), library
routines for special cases (numpy.linalg.matrix_rank at eps = 0, LAPACK SVD of
the dense unfoldings), the error bound of the Alg. 6 correctness theorem, and
brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

from oracle import dense as D
from oracle import fasttt as F
from oracle import tteval as T
from paper_1908_02721_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _small_cases():
    cases = []
    for seed, dims, nnz in [(11, [4, 5, 3], 25), (12, [3, 4, 5, 2], 40), (13, [6, 6, 6], 80),
                            (14, [2, 3, 4, 3, 2], 60), (15, [5, 7], 12), (16, [3, 3, 3, 3], 81)]:
        cases.append(W.random_sparse(dims, nnz, seed, "normal"))
    return cases


# ---------------------------------------------------------------- Theorem (Sec. 3.1) + Alg. 4/5

def _dense_exact(ex, dims):
    """Contract the exact TT of Alg. 4: left P-cores, the fiber core V, right P-cores."""
    d = len(dims)
    p = ex.p
    cores = []
    for k in range(1, p):
        parent, i = ex.left[k - 1]
        cores.append(F.left_pcore(parent, i, ex.rt[k - 1], dims[k - 1]))
    V = np.zeros((ex.rt[p - 1], dims[p - 1], ex.rt[p]))
    if p < d:
        M = V.reshape(-1, ex.rt[p])
        M[ex.mid_rows, ex.mid_cols] = ex.mid_vals
    else:
        V[ex.mid_cols, ex.mid_rows, 0] = ex.mid_vals
    cores.append(V)
    for k in range(p + 1, d + 1):
        i, child = ex.right[k - p - 1]
        cores.append(F.right_pcore(i, child, dims[k - 1], ex.rt[k]))
    return cores


@pytest.mark.parametrize("case", range(6))
def test_exact_tt_reconstructs_A_bit_exactly(case):
    """T1: the TT of Alg. 4 equals A exactly, for every split point p."""
    w = _small_cases()[case]
    A = D.full_from_coo(w.idx, w.vals, w.dims)
    for p in range(1, w.d + 1):
        ex = F.exact_tt(w.idx.astype(np.int64), w.vals, w.dims, p)
        B = D.tt_full(_dense_exact(ex, w.dims))
        assert np.array_equal(A, B)


@pytest.mark.parametrize("case", range(6))
def test_pcores_orthonormal_and_ranks_characterised(case):
    """T2-T4: deduplicated quasi-permutation unfoldings satisfy Q^T Q = I exactly
    (Lemma 'quasi-permutation => orthonormal', Cor. of Alg. 4); r~_k obeys eq. (10)
    and equals the number of nonzero rows (k < p) / columns (k >= p) of unfold_k(A)."""
    w = _small_cases()[case]
    A = D.full_from_coo(w.idx, w.vals, w.dims)
    d = w.d
    for p in range(1, d + 1):
        ex = F.exact_tt(w.idx.astype(np.int64), w.vals, w.dims, p)
        R, _ = F.fiber_ids(w.idx.astype(np.int64), p)
        rb = F.rank_bounds(w.dims, R, p)
        cores = _dense_exact(ex, w.dims)
        for k in range(1, d):
            assert ex.rt[k] <= rb[k]
            Ak = D.unfold(A, k)
            if k < p:
                assert ex.rt[k] == np.count_nonzero(np.any(Ak != 0, axis=1))
            else:
                assert ex.rt[k] == np.count_nonzero(np.any(Ak != 0, axis=0))
        for k in range(1, d + 1):
            G = cores[k - 1]
            if k < p:
                M = G.reshape(-1, G.shape[2])
                assert np.array_equal(M.T @ M, np.eye(G.shape[2]))
            elif k > p:
                M = G.reshape(G.shape[0], -1)
                assert np.array_equal(M @ M.T, np.eye(G.shape[0]))


def test_fiber_count_brute_force():
    """R of eq. (4): brute-force count of nonzero p-fibers of the dense tensor."""
    w = W.random_sparse([4, 3, 5, 2], 30, 21, "uniform")
    A = D.full_from_coo(w.idx, w.vals, w.dims)
    for p in range(1, 5):
        R, _ = F.fiber_ids(w.idx.astype(np.int64), p)
        Am = np.moveaxis(A, p - 1, -1)
        assert R == np.count_nonzero(np.any(Am != 0, axis=-1))


# ---------------------------------------------------------------- paper's printed numbers

@pytest.mark.parametrize("row", _read_golden("fdm_table2.txt")[:3])
def test_fdm_table2(row):
    """T7: R, r~ and r of Table 2 for the 7-point FDM matrices (eps = 1e-14, p = 2)."""
    n, coeffs, R, rt1, rt2, r1, r2 = row[0], row[1], *map(int, row[2:])
    n = int(n)
    w = W.fdm7(n, coeffs)
    res = F.fasttt(w.idx, w.vals, w.dims, w.eps, p=2)
    assert res.R == R
    assert res.rt[1:3] == [rt1, rt2]
    assert res.ranks[1:3] == [r1, r2]
    A_err = math.sqrt(res.err2) / math.sqrt(res.norm2)
    assert A_err < 1e-14
    # the paper-exact grouping (no value Depar) gives the same R and r~
    ex = F.exact_tt(w.idx.astype(np.int64), w.vals, w.dims, 2)
    assert (ex.R, ex.rt[1], ex.rt[2]) == (R, rt1, rt2)


def test_alg9_flop_example():
    """T8: the rank bounds and flop estimate of the Sec. 3.6 worked example."""
    dims = [10, 20, 20, 10, 15, 20, 3]
    for row in _read_golden("alg9_example.txt"):
        R, rank, p = int(row[0]), int(row[1]), int(row[2])
        rbar = [int(x) for x in row[3:9]]
        f_exact, f_paper = int(row[9]), float(row[10])
        rt = F.rank_bounds(dims, R, p)
        assert rt[1:7] == rbar
        r = [min(x, rank) if 0 < k < 7 else x for k, x in enumerate(rt)]
        f = F.flop_estimate(dims, rt, p, r)
        assert f == f_exact
        assert abs(f - f_paper) / f_paper < 0.01


def test_alg9_paper_terms():
    """The individual terms the paper prints for the R = 12000 case."""
    r = 10
    assert F.f_svd(3, 12000) == 108000
    assert F.f_svd(20 * r, 12000) == 480_000_000
    assert F.f_svd(15 * r, 12000) == 270_000_000
    assert F.f_svd(10 * r, 4000) == 40_000_000
    assert F.f_svd(20 * r, 200) == 8_000_000


# ---------------------------------------------------------------- eps = 0, error bounds, plain definition

def test_eps0_ranks_match_matrix_rank_and_exact():
    """T6: at eps = 0 the ranks are the unfolding ranks (numpy.linalg.matrix_rank)
    and the TT reproduces A to rounding (Sec. 3.3, remark after Alg. 7)."""
    w = W.exact_small()
    res = F.fasttt(w.idx, w.vals, w.dims, 0.0)
    A = D.full_from_coo(w.idx, w.vals, w.dims)
    for k in range(1, w.d):
        assert res.ranks[k] == np.linalg.matrix_rank(D.unfold(A, k))
    B = D.tt_full(res.cores)
    assert np.linalg.norm(A - B) <= 1e-13 * np.linalg.norm(A)
    # and equal to Alg. 1's ranks
    _, rk, _ = D.tt_svd(A, 0.0)
    assert rk == res.ranks


@pytest.mark.parametrize("case", range(6))
@pytest.mark.parametrize("eps", [0.0, 1e-8, 0.05, 0.3])
def test_error_bound_and_plain_definition(case, eps):
    """T5 + the plain definition: ||A - B|| <= eps ||A|| (Alg. 6 correctness theorem),
    and B equals the sequential truncation of the unfoldings with the same deltas
    (bonds p..d-1, then p-1..1) computed with LAPACK on the dense tensor."""
    w = _small_cases()[case]
    A = D.full_from_coo(w.idx, w.vals, w.dims)
    nA = np.linalg.norm(A)
    for p in range(1, w.d + 1):
        for depar in (True, False):
            res = F.fasttt(w.idx, w.vals, w.dims, eps, p=p, depar_values=depar)
            B = D.tt_full(res.cores)
            err = np.linalg.norm(A - B)
            assert err <= eps * nA + 1e-12 * nA
            Bref, rref = D.sequential_projection(A, eps, p)
            assert res.ranks == rref
            assert np.linalg.norm(B - Bref) <= 1e-12 * nA
            if p in (1, w.d):  # errors add in quadrature exactly (proof of the theorem)
                assert abs(err ** 2 - res.err2) <= 1e-12 * nA ** 2


def test_p1_equals_alg1_ttsvd():
    """At p = 1 eq. (11) gives Alg. 1's delta and FastTT reproduces TT-SVD."""
    w = W.random_sparse([5, 4, 6, 3], 70, 31, "normal")
    A = D.full_from_coo(w.idx, w.vals, w.dims)
    for eps in (1e-10, 0.1, 0.4):
        res = F.fasttt(w.idx, w.vals, w.dims, eps, p=1)
        cores, rk, _ = D.tt_svd(A, eps)
        assert res.ranks == rk
        assert D.tt_diff_norm(res.cores, cores) <= 1e-12 * np.linalg.norm(A)


def test_fixed_rank_cap():
    """Sec. 3.4 fixed-rank variant: ranks never exceed the cap."""
    w = W.random_sparse([6, 6, 6, 6], 300, 41, "normal")
    res = F.fasttt(w.idx, w.vals, w.dims, 0.0, max_rank=4)
    assert max(res.ranks) <= 4
    A = D.full_from_coo(w.idx, w.vals, w.dims)
    B = D.tt_full(res.cores)
    assert abs(np.linalg.norm(A - B) ** 2 - res.err2) <= 1e-9 * np.linalg.norm(A) ** 2 or res.p not in (1, 4)


def test_dynamic_alg8_bound():
    """Alg. 8 (appendix theorem): the dynamic budget still guarantees eps ||A||."""
    w = W.random_sparse([5, 5, 5, 5], 200, 51, "normal")
    A = D.full_from_coo(w.idx, w.vals, w.dims)
    nA = np.linalg.norm(A)
    for eps in (0.05, 0.2, 0.5):
        for p in (1, 2, 3, 4):
            st = F.fasttt(w.idx, w.vals, w.dims, eps, p=p)
            dy = F.fasttt(w.idx, w.vals, w.dims, eps, p=p, rounding="dynamic")
            assert np.linalg.norm(A - D.tt_full(dy.cores)) <= eps * nA * (1 + 1e-12)
            assert sum(dy.ranks) <= sum(st.ranks) + 2 * w.d


def superdiagonal_alg8_workload():
    """The hand-worked Alg. 8 input of tests/golden/alg8_example.txt: 4 modes of size
    5, A(i,i,i,i) = (8, 4, 2, 1, 1/2)_i, eps ||A|| = 1.2."""
    s = np.array([8.0, 4.0, 2.0, 1.0, 0.5])
    idx = np.tile(np.arange(5, dtype=np.int32), (4, 1))
    return idx, s, [5, 5, 5, 5], 1.2 / math.sqrt(float(np.sum(s * s)))


@pytest.mark.parametrize("row", _read_golden("alg8_example.txt"))
def test_alg8_hand_worked_ranks(row):
    """Alg. 8 pinned by hand: delta_right / sqrt(d-k) (and delta_left / sqrt(k-1)) on a
    superdiagonal tensor whose spectra are known in closed form.  The schedule
    delta / (d-k), or the static eq. (11), gives other ranks on the same input."""
    p, rounding = int(row[0]), row[1]
    ranks = [int(x) for x in row[2:7]]
    err2 = float(row[7])
    idx, vals, dims, eps = superdiagonal_alg8_workload()
    res = F.fasttt(idx, vals, dims, eps, p=p, rounding=rounding)
    assert res.ranks == ranks
    assert abs(res.err2 - err2) <= 1e-12
    A = D.full_from_coo(idx, vals, dims)
    assert abs(np.linalg.norm(A - D.tt_full(res.cores)) ** 2 - err2) <= 1e-12


# ---------------------------------------------------------------- value Depar (S6)

def test_value_depar_factorisation_and_planted_parallels():
    """S6: X = Q_S C Q_T with orthonormal Q_S, Q_T; rows/columns that are exact
    power-of-two multiples of each other fall into one class with the multiplier
    as prefactor ratio (the parallel test of Alg. 3)."""
    rng = np.random.Generator(np.random.Philox(key=61))
    base = rng.standard_normal(5)
    rows, cols, vals = [], [], []
    for r, mult in enumerate([1.0, -2.0, 0.5, 4.0]):   # four parallel rows
        for c in range(5):
            rows.append(r); cols.append(c + 1); vals.append(base[c] * mult)
    rows += [4, 4]; cols += [0, 3]; vals += [1.5, -0.25]           # a different row
    rows += [6]; cols += [2]; vals += [3.0]                          # single entry rows
    rows += [7]; cols += [2]; vals += [-7.0]
    X = (np.array(rows), np.array(cols), np.array(vals))
    dp = F.value_depar(*X)
    cls = dict(zip(dp.row_ids.tolist(), dp.row_class.tolist()))
    assert cls[0] == cls[1] == cls[2] == cls[3] == 0
    assert cls[4] == 1 and cls[6] == cls[7] == 2
    assert dp.beta_r == 3
    pref = dict(zip(dp.row_ids.tolist(), dp.row_pref.tolist()))
    assert pref[1] == base[0] * -2.0 and pref[7] == -7.0
    C = F.depar_dense_C(dp)
    Xd = np.zeros((8, 6))
    Xd[X[0], X[1]] = X[2]
    QS = np.zeros((8, dp.beta_r))
    QS[dp.row_ids, dp.row_class] = dp.row_pref / dp.lam_s[dp.row_class]
    QT = np.zeros((dp.beta_c, 6))
    QT[dp.col_class, dp.col_ids] = dp.col_pref / dp.lam_t[dp.col_class]
    assert np.allclose(QS.T @ QS, np.eye(dp.beta_r), atol=1e-15)
    assert np.allclose(QT @ QT.T, np.eye(dp.beta_c), atol=1e-15)
    assert np.allclose(QS @ C @ QT, Xd, rtol=0, atol=1e-14 * np.abs(Xd).max())


# ---------------------------------------------------------------- input edge cases

def test_input_errors_and_zero_dropping():
    idx = np.array([[0, 1, 1], [2, 0, 0]], dtype=np.int32)
    with pytest.raises(F.FastTTError) as e:
        F.fasttt(idx, np.array([1.0, 2.0, 3.0]), [2, 3], 0.1)
    assert e.value.code == F.EDUP
    with pytest.raises(F.FastTTError) as e:
        F.fasttt(np.array([[0, 2], [0, 0]]), np.array([1.0, 2.0]), [2, 3], 0.1)
    assert e.value.code == F.EINVAL
    with pytest.raises(F.FastTTError) as e:
        F.fasttt(np.array([[0, 1], [0, 0]]), np.array([1.0, np.nan]), [2, 3], 0.1)
    assert e.value.code == F.EINVAL
    with pytest.raises(F.FastTTError) as e:
        F.fasttt(np.array([[0, 1], [0, 0]]), np.array([0.0, -0.0]), [2, 3], 0.1)
    assert e.value.code == F.EINVAL
    res = F.fasttt(np.array([[0, 1, 1], [0, 0, 2]]), np.array([1.0, 0.0, 2.0]), [2, 3], 0.0)
    assert res.dropped == 1
    A = np.zeros((2, 3)); A[0, 0] = 1.0; A[1, 2] = 2.0
    assert np.allclose(D.tt_full(res.cores), A, atol=1e-15)


def test_matrix_case_is_svd():
    """d = 2: the TT is a truncated SVD of the matrix (Alg. 1 with one bond)."""
    w = W.random_sparse([30, 20], 150, 71, "normal")
    A = D.full_from_coo(w.idx, w.vals, w.dims)
    s = np.linalg.svd(A, compute_uv=False)
    for eps in (0.0, 0.2):
        for p in (1, 2):
            res = F.fasttt(w.idx, w.vals, w.dims, eps, p=p)
            assert np.allclose(res.sigmas[1][: len(s)], s[: len(res.sigmas[1])], rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- TT evaluation and gradient

def test_tt_eval_and_gradient_finite_differences():
    rng = np.random.Generator(np.random.Philox(key=81))
    dims, ranks = [4, 3, 5, 2], [1, 3, 4, 2, 1]
    cores = [rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(4)]
    idx = np.stack([rng.integers(0, n, 40) for n in dims])
    full = D.tt_full(cores)
    a = T.tt_eval_at(cores, idx)
    assert np.allclose(a, full[tuple(idx)], rtol=1e-14, atol=1e-14)
    assert np.allclose(T.tt_eval_at_batched(cores, idx), a, rtol=1e-14, atol=1e-14)
    g = rng.standard_normal(40)
    grads = T.tt_eval_grad(cores, idx, g)
    h = 1e-6
    for k in range(4):
        for flat in rng.choice(cores[k].size, min(6, cores[k].size), replace=False):
            pos = np.unravel_index(flat, cores[k].shape)
            cp = [c.copy() for c in cores]
            cm = [c.copy() for c in cores]
            cp[k][pos] += h
            cm[k][pos] -= h
            fd = (g @ T.tt_eval_at_batched(cp, idx) - g @ T.tt_eval_at_batched(cm, idx)) / (2 * h)
            assert abs(fd - grads[k][pos]) <= 1e-7 * max(1.0, abs(fd))


def test_tt_sum_and_diff_norm():
    rng = np.random.Generator(np.random.Philox(key=91))
    dims = [3, 4, 2, 3]
    a = [rng.standard_normal((r0, n, r1)) for r0, n, r1 in zip([1, 2, 3, 2], dims, [2, 3, 2, 1])]
    b = [rng.standard_normal((r0, n, r1)) for r0, n, r1 in zip([1, 3, 1, 2], dims, [3, 1, 2, 1])]
    assert np.allclose(D.tt_full(D.tt_sum(a, b)), D.tt_full(a) + D.tt_full(b), atol=1e-13)
    ref = np.linalg.norm(D.tt_full(a) - D.tt_full(b))
    assert abs(D.tt_diff_norm(a, b) - ref) <= 1e-13 * ref


def test_value_depar_hand_worked_example():
    """S6 on the hand-worked example of tests/golden/depar_example.txt (Alg. 3 with exact
    parallelism on the rows of X, then on the columns of D): classes, prefactors, D',
    Lambda_S, Lambda_T and C exactly as derived by hand."""
    rec = {}
    X, DP, C = [], [], []
    path = os.path.join(os.path.dirname(__file__), "golden", "depar_example.txt")
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        tag, *rest = line.split()
        if tag == "X":
            X.append((int(rest[0]), int(rest[1]), float(rest[2])))
        elif tag == "DP":
            DP.append((int(rest[0]), int(rest[1]), float(rest[2])))
        elif tag == "C":
            C.append((int(rest[0]), int(rest[1]), float(rest[2])))
        else:
            rec[tag] = [float(x) for x in rest]
    rows = np.array([x[0] for x in X])
    cols = np.array([x[1] for x in X])
    vals = np.array([x[2] for x in X])
    dp = F.value_depar(rows, cols, vals)
    assert dp.row_ids.tolist() == [int(x) for x in rec["ROWS"]]
    assert dp.row_class.tolist() == [int(x) for x in rec["ROW_CLASS"]]
    assert dp.row_pref.tolist() == rec["ROW_PREF"]
    assert dp.col_ids.tolist() == [int(x) for x in rec["COLS"]]
    assert dp.col_class.tolist() == [int(x) for x in rec["COL_CLASS"]]
    assert dp.col_pref.tolist() == rec["COL_PREF"]
    got_dp = sorted(zip(dp.dp_rows.tolist(), dp.dp_cols.tolist(), dp.dp_vals.tolist()))
    assert got_dp == sorted(DP)
    assert dp.lam_s.tolist() == rec["LAM_S"] and dp.lam_t.tolist() == rec["LAM_T"]
    Cd = F.depar_dense_C(dp)
    want = np.zeros((3, 3))
    for i, j, v in C:
        want[i, j] = v
    assert np.array_equal(Cd, want)


def test_grouping_hand_worked_example():
    """S2-S5 on the hand-worked example of tests/golden/grouping_example.txt: the
    lexicographic-rank ids of both sweeps, the P-cores' (parent, index) and
    (index, child) maps, r~, R (eq. (4)) and the middle unfolding."""
    rec, nz, mid = {}, [], []
    path = os.path.join(os.path.dirname(__file__), "golden", "grouping_example.txt")
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        tag, *rest = line.split()
        if tag == "NZ":
            nz.append(([int(x) for x in rest[:4]], float(rest[4])))
        elif tag == "MID":
            mid.append((int(rest[0]), int(rest[1]), float(rest[2])))
        else:
            rec[tag] = [int(x) for x in rest]
    dims, p = rec["DIMS"], rec["P"][0]
    idx = np.array([i for i, _ in nz]).T
    v = np.array([x for _, x in nz])
    tt = F.exact_tt(idx, v, dims, p)
    assert tt.R == rec["R"][0]
    assert list(tt.rt) == rec["RT"]
    l1, l2 = rec["LEFT1"], rec["LEFT2"]
    assert tt.left[0][0].tolist() == l1[:2] and tt.left[0][1].tolist() == l1[2:]
    assert tt.left[1][0].tolist() == l2[:4] and tt.left[1][1].tolist() == l2[4:]
    r4 = rec["RIGHT4"]
    assert tt.right[0][0].tolist() == r4[:3] and tt.right[0][1].tolist() == r4[3:]
    assert tt.alpha_left.tolist() == rec["ALPHA_L"] and tt.alpha_right.tolist() == rec["ALPHA_R"]
    got = sorted(zip(tt.mid_rows.tolist(), tt.mid_cols.tolist(), tt.mid_vals.tolist()))
    assert got == sorted(mid)
    assert tuple(tt.mid_shape) == (rec["RT"][2] * dims[2], rec["RT"][3])
