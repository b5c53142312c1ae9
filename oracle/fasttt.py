"""FastTT in plain numpy/scipy FP64 (test infrastructure only).

Follows the paper's steps in its order and notation (0-based indices here):

S1  ingest               input checks; A as the sum over its nonzeros (Sec. 3.1)
S2  select_p             Alg. 9 with the rank bounds of eq. (10) and the flop model of eq. (13)
S3  left sweep           Alg. 4 (k = 1..p-1) with Alg. 5 on quasi-permutation unfoldings
S4  right sweep          Alg. 4 (k = d..p+1) with Alg. 5
S5  middle core          the fiber core V of Theorem (sparse tensor -> rank-R TT), eq. (7)
S6  value Depar          Alg. 3 with exact (bit-equal after normalisation) parallelism on the
                         rows, then the columns, of V's unfolding
S7-S10 rounding          Alg. 6 (first SVD sweep, QR sweep, second SVD sweep) or Alg. 8
S11 rank rule            delta_k of eq. (11); smallest r whose tail is <= delta_k
S12 output               dense cores r_{k-1} x n_k x r_k

Readings of places where the paper is silent or ambiguous (each one also
listed in the design notes):
 * "parallel" (Alg. 3) means bit-equal after dividing a vector by its first
   nonzero with IEEE round-to-nearest; the kept vector is that normalised
   vector and the prefactor is the first nonzero itself.
 * Alg. 3's else-branch appends a column only when no kept column is parallel.
 * classes are numbered by first occurrence in ascending row (column) order;
   Alg. 5 ids follow ascending row order of the quasi-permutation unfolding.
 * eps = 0 means the numerical rank: s_i > max(M, N) * 2^-52 * s_1 with M x N
   the dims of the k-unfolding of A (numpy.linalg.matrix_rank's default).
 * duplicate coordinates are an error (EDUP); explicit zeros are dropped.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg

from .dense import truncation_rank, unfolding_rank_tol

EINVAL, EDUP, ENOMEM, ETIMEOUT, ENUMERIC, ERANK = -1, -2, -3, -4, -5, -6


class FastTTError(Exception):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


# ------------------------------------------------------------------------ S1

def ingest(idx, vals, dims):
    """Validate the COO input; drop explicit zeros; upcast values to FP64 exactly."""
    dims = [int(n) for n in dims]
    d = len(dims)
    idx = np.asarray(idx)
    if d < 2 or any(n < 1 for n in dims):
        raise FastTTError(EINVAL, "need d >= 2 and positive mode sizes")
    if idx.ndim != 2 or idx.shape[0] != d:
        raise FastTTError(EINVAL, "indices must have shape (d, nnz)")
    idx = idx.astype(np.int64)
    v = np.asarray(vals).astype(np.float64)
    if v.shape != (idx.shape[1],):
        raise FastTTError(EINVAL, "values must have shape (nnz,)")
    if idx.size and ((idx < 0).any() or (idx >= np.asarray(dims)[:, None]).any()):
        raise FastTTError(EINVAL, "index out of range")
    if not np.isfinite(v).all():
        raise FastTTError(EINVAL, "non-finite value")
    keep = v != 0.0
    idx, v = idx[:, keep], v[keep]
    if v.size == 0:
        raise FastTTError(EINVAL, "the tensor has no nonzero entry")
    return idx, v, int((~keep).sum())


def frobenius2(v):
    """||A||_F^2 as the exactly rounded sum of the (rounded) squares."""
    return math.fsum((v * v).tolist())


# ------------------------------------------------------------------------ fibers, S2

def fiber_ids(idx, p):
    """p-fibers (eq. (2)): the distinct index tuples without mode p, ranked
    lexicographically.  Returns (R, fiber id of every nonzero)."""
    d = idx.shape[0]
    others = [k for k in range(d) if k != p - 1]
    uniq, inv = np.unique(idx[others].T, axis=0, return_inverse=True)
    return uniq.shape[0], inv.reshape(-1)


def rank_bounds(dims, R, p):
    """r_bar_k of eq. (10), k = 0..d (r_bar_0 = r_bar_d = 1), as Python ints."""
    d = len(dims)
    rb = [1] * (d + 1)
    for k in range(1, d):
        if k < p:
            rb[k] = min(R, math.prod(dims[:k]))
        else:
            rb[k] = min(R, math.prod(dims[k:]))
    return rb


def f_svd(m, n):
    """FLOP count of an economic m x n SVD up to the constant C_svd (below eq. (1))."""
    return m * n * min(m, n)


def flop_estimate(dims, rt, p, r=None):
    """eq. (13): the SVD cost of Alg. 6 for split point p, in units of C_svd.
    rt: ranks before rounding (k = 0..d); r: ranks after (defaults to rt)."""
    d = len(dims)
    n = [None] + list(dims)          # 1-based mode sizes
    r = rt if r is None else r
    f = f_svd(rt[p - 1] * n[p], rt[p])
    for i in range(p + 1, d):
        f += f_svd(r[i - 1] * n[i], rt[i])
    for i in range(2, p + 1):
        f += f_svd(rt[i - 1], n[i] * r[i])
    return f


def select_p(dims, Rs, max_rank=0):
    """Alg. 9: the p in 1..d with the smallest estimate of eq. (13), using the
    bounds of eq. (10) for r~ and, for r, the bounds capped at max_rank (the
    ranks 'specified by users').  Ties go to the smallest p."""
    d = len(dims)
    best, best_f, fs = None, None, []
    for p in range(1, d + 1):
        rt = rank_bounds(dims, Rs[p - 1], p)
        r = [min(x, max_rank) if max_rank and 0 < k < d else x for k, x in enumerate(rt)]
        f = flop_estimate(dims, rt, p, r)
        fs.append(f)
        if best_f is None or f < best_f:
            best, best_f = p, f
    return best, fs


# ------------------------------------------------------------------------ S3-S5

def depar_quasi_permutation(rowpos):
    """Alg. 5 on a quasi-permutation matrix M given by the row of the single 1
    in each column.  Scanning rows in ascending order, every nonzero row opens a
    new column beta of N (N[:, beta] = e_row) and T[beta, :] = M[row, :].
    Returns (kept rows in ascending order, beta of every column of M)."""
    kept = np.unique(rowpos)
    return kept, np.searchsorted(kept, rowpos)


@dataclasses.dataclass
class ExactTT:
    """Output of Alg. 4 (sparse -> exact TT, Theorem of Sec. 3.1)."""
    dims: list
    p: int
    R: int
    rt: list              # r~_0..r~_d
    left: list            # k = 1..p-1: (parent alpha_{k-1}, i_k) per alpha_k
    right: list           # k = p+1..d: (i_k, child alpha_k) per alpha_{k-1}
    alpha_left: np.ndarray   # alpha_{p-1} of every nonzero
    alpha_right: np.ndarray  # alpha_p of every nonzero
    mid_rows: np.ndarray  # middle unfolding X: row of every nonzero
    mid_cols: np.ndarray  # column of every nonzero
    mid_vals: np.ndarray
    mid_shape: tuple


def exact_tt(idx, v, dims, p):
    """Alg. 4 with Depar = Alg. 5.  The rank-R TT of Theorem (Sec. 3.1) is held
    by the fibers: fiber j contributes e_{i_1} o ... o v_j o ... o e_{i_d}
    (eq. (4)); its P-core columns are the standard basis vectors e_{i_k(j)}."""
    d = len(dims)
    R, fib = fiber_ids(idx, p)
    # one representative nonzero per fiber gives the fiber's indices i_k (k != p)
    first = np.full(R, -1, dtype=np.int64)
    order = np.arange(fib.size)[::-1]
    first[fib[order]] = order
    fidx = idx[:, first]                       # (d, R), mode p entry unused
    rt = [1] * (d + 1)
    # left sweep k = 1..p-1: M = unfold_2(G_k), rows (alpha_{k-1}, i_k)
    alpha = np.zeros(R, dtype=np.int64)
    left = []
    for k in range(1, p):
        n = dims[k - 1]
        rowpos = alpha * n + fidx[k - 1]
        kept, alpha = depar_quasi_permutation(rowpos)
        rt[k] = kept.size
        left.append((kept // n, kept % n))
    alpha_l = alpha
    # right sweep k = d..p+1: M = unfold_1^T(G_k), rows (i_k, alpha_k)
    alpha = np.zeros(R, dtype=np.int64)
    right = [None] * (d - p)
    for k in range(d, p, -1):
        rk = rt[k]
        rowpos = fidx[k - 1] * rk + alpha
        kept, alpha = depar_quasi_permutation(rowpos)
        rt[k - 1] = kept.size
        right[k - p - 1] = (kept // rk, kept % rk)
    alpha_r = alpha
    # fiber core V (r~_{p-1} x n_p x r~_p): V[alpha_l(j), i_p, alpha_r(j)] = A entry
    al, ar = alpha_l[fib], alpha_r[fib]
    n_p = dims[p - 1]
    if p < d:
        rows, cols = al * n_p + idx[p - 1], ar
        shape = (rt[p - 1] * n_p, rt[p])
    else:  # p = d: Alg. 6 starts on unfold_1^T(G_d), rows i_d, columns alpha_{d-1}
        rows, cols = idx[p - 1].copy(), al
        shape = (n_p, rt[p - 1])
    key = rows * shape[1] + cols
    if np.unique(key).size != key.size:
        raise FastTTError(EDUP, "duplicate coordinate")
    return ExactTT(list(dims), p, R, rt, left, right, al, ar, rows, cols, v.copy(), shape)


# ------------------------------------------------------------------------ S6

def depar_rows(rows, cols, vals):
    """Alg. 3 applied to the rows of a sparse matrix X (the columns of X^T) with
    exact parallelism.  Every nonzero row is divided by its first nonzero (the
    one in the smallest column) with IEEE round-to-nearest; two rows are
    parallel when their column patterns and normalised value bits are equal.
    Classes are numbered by first occurrence in ascending row order.

    Returns (nonzero rows ascending, class of each, prefactor of each,
             class representatives as a list of (cols, normalised values))."""
    order = np.lexsort((cols, rows))
    r_s, c_s, v_s = rows[order], cols[order], vals[order]
    starts = np.flatnonzero(np.r_[True, r_s[1:] != r_s[:-1]])
    ends = np.r_[starts[1:], r_s.size]
    classes = {}
    reps = []
    row_ids = r_s[starts]
    row_class = np.empty(starts.size, dtype=np.int64)
    row_pref = np.empty(starts.size, dtype=np.float64)
    for t, (a, b) in enumerate(zip(starts, ends)):
        v0 = v_s[a]
        norm = v_s[a:b] / v0
        key = (c_s[a:b].tobytes(), norm[1:].view(np.uint64).tobytes())
        g = classes.get(key)
        if g is None:
            g = len(reps)
            classes[key] = g
            reps.append((c_s[a:b].copy(), norm))
        row_class[t] = g
        row_pref[t] = v0
    return row_ids, row_class, row_pref, reps


@dataclasses.dataclass
class Depar:
    row_ids: np.ndarray
    row_class: np.ndarray
    row_pref: np.ndarray
    col_ids: np.ndarray
    col_class: np.ndarray
    col_pref: np.ndarray
    beta_r: int
    beta_c: int
    dp_rows: np.ndarray   # D' entries (beta_r x beta_c), normalised twice
    dp_cols: np.ndarray
    dp_vals: np.ndarray
    lam_s: np.ndarray     # Lambda_S (beta_r)
    lam_t: np.ndarray     # Lambda_T (beta_c)


def value_depar(X_rows, X_cols, X_vals, enabled=True):
    """S6: X = S D (row pass), D = D' T (column pass of D), S = Q_S Lambda_S,
    T = Lambda_T Q_T, so X = Q_S C Q_T with C = Lambda_S D' Lambda_T."""
    if not enabled:  # identity factors: every nonzero row/column is its own class
        rid = np.unique(X_rows)
        cid = np.unique(X_cols)
        rc = np.searchsorted(rid, X_rows)
        cc = np.searchsorted(cid, X_cols)
        return Depar(rid, np.arange(rid.size), np.ones(rid.size), cid, np.arange(cid.size),
                     np.ones(cid.size), rid.size, cid.size, rc, cc, X_vals.copy(),
                     np.ones(rid.size), np.ones(cid.size))
    row_ids, row_class, row_pref, reps = depar_rows(X_rows, X_cols, X_vals)
    beta_r = len(reps)
    # D as COO: class-row g, column c, normalised value
    d_rows = np.concatenate([np.full(c.size, g, dtype=np.int64) for g, (c, _) in enumerate(reps)])
    d_cols = np.concatenate([c for c, _ in reps])
    d_vals = np.concatenate([v for _, v in reps])
    # column pass = row pass on D^T
    col_ids, col_class, col_pref, creps = depar_rows(d_cols, d_rows, d_vals)
    beta_c = len(creps)
    dp_rows = np.concatenate([g for g, _ in creps])
    dp_cols = np.concatenate([np.full(g.size, h, dtype=np.int64) for h, (g, _) in enumerate(creps)])
    dp_vals = np.concatenate([w for _, w in creps])
    lam_s = class_norms(row_class, row_pref, beta_r)
    lam_t = class_norms(col_class, col_pref, beta_c)
    return Depar(row_ids, row_class, row_pref, col_ids, col_class, col_pref, beta_r, beta_c,
                 dp_rows, dp_cols, dp_vals, lam_s, lam_t)


def class_norms(cls, pref, beta):
    """Lambda: the 2-norm of the prefactors of every class (exactly rounded sum of squares)."""
    order = np.argsort(cls, kind="stable")
    c_s, sq = cls[order], (pref[order] ** 2)
    bounds = np.searchsorted(c_s, np.arange(beta + 1))
    return np.array([math.sqrt(math.fsum(sq[bounds[g]:bounds[g + 1]].tolist())) for g in range(beta)])


def depar_dense_C(dp: Depar):
    """C = Lambda_S D' Lambda_T as a dense beta_r x beta_c array, each entry
    formed as (lambda_s * d') * lambda_t."""
    C = np.zeros((dp.beta_r, dp.beta_c))
    C[dp.dp_rows, dp.dp_cols] = (dp.lam_s[dp.dp_rows] * dp.dp_vals) * dp.lam_t[dp.dp_cols]
    return C


# ------------------------------------------------------------------------ S7-S12

def svd(M):
    return scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")


@dataclasses.dataclass
class Result:
    cores: list
    ranks: list
    p: int
    R: int
    Rs: list
    rt: list
    norm2: float
    err2: float
    deltas: list
    sigmas: dict          # bond -> singular values
    exact: ExactTT
    depar: Depar
    dropped: int


def _rank_at(s, delta, dims, bond, max_rank, eps):
    tol = unfolding_rank_tol(dims, bond, s[0] if s.size else 0.0) if eps == 0.0 else None
    return truncation_rank(s, delta if eps > 0 else 0.0, tol, max_rank)


def left_pcore(parent, i, r_prev, n):
    """Dense 0/1 core r~_{k-1} x n_k x r~_k of a left quasi-permutation core."""
    G = np.zeros((r_prev, n, parent.size))
    G[parent, i, np.arange(parent.size)] = 1.0
    return G


def right_pcore(i, child, n, r_next):
    """Dense 0/1 core r~_{k-1} x n_k x r~_k of a right quasi-permutation core."""
    G = np.zeros((i.size, n, r_next))
    G[np.arange(i.size), i, child] = 1.0
    return G


def fasttt(idx, vals, dims, eps, p=0, max_rank=0, depar_values=True, rounding="static"):
    """Alg. 7 (FastTT): Alg. 4 (with Alg. 5), value Depar of the middle
    unfolding, then Alg. 6 (rounding='static') or Alg. 8 (rounding='dynamic')."""
    dims = [int(n) for n in dims]
    d = len(dims)
    idx, v, dropped = ingest(idx, vals, dims)
    norm2 = frobenius2(v)
    normA = math.sqrt(norm2)
    Rs = []
    if p == 0:
        Rs = [fiber_ids(idx, q)[0] for q in range(1, d + 1)]
        p, _ = select_p(dims, Rs, max_rank)
    if not 1 <= p <= d:
        raise FastTTError(EINVAL, "p out of range")
    ex = exact_tt(idx, v, dims, p)
    dp = value_depar(ex.mid_rows, ex.mid_cols, ex.mid_vals, depar_values)

    # truncation parameters: eq. (11) (static) or Alg. 8 (dynamic)
    c = math.sqrt(p - 1) + math.sqrt(d - p)
    deltas = [eps * normA / c] * (d + 1)
    d_right = math.sqrt(d - p) / c * eps * normA
    d_left = math.sqrt(p - 1) / c * eps * normA

    def delta_for(bond, right_side):
        if rounding == "static":
            return deltas[bond]
        return (d_right / math.sqrt(d - bond)) if right_side else (d_left / math.sqrt(bond))

    # dense cores: left P-cores, (middle filled below), right P-cores
    G = [None] * d
    for k in range(1, p):
        parent, i = ex.left[k - 1]
        G[k - 1] = left_pcore(parent, i, ex.rt[k - 1], dims[k - 1])
    for k in range(p + 1, d + 1):
        i, child = ex.right[k - p - 1]
        G[k - 1] = right_pcore(i, child, dims[k - 1], ex.rt[k])
    ranks = list(ex.rt)
    sig = {}
    err2 = 0.0
    used = {}

    # the first SVD of Alg. 6 on the value-deparallelised middle unfolding
    C = depar_dense_C(dp)
    U, s, Vt = svd(C)
    bond = p if p < d else d - 1
    dl = delta_for(bond, p < d)
    r = _rank_at(s, dl, dims, bond, max_rank, eps)
    e2 = float(np.sum(s[r:] ** 2))
    err2 += e2
    sig[bond] = s
    used[bond] = dl
    # rows of X: Q_S U; columns of X: Q_T^T V
    Xrows, Xcols = ex.mid_shape
    Ufull = np.zeros((Xrows, r))
    Ufull[dp.row_ids] = (dp.row_pref / dp.lam_s[dp.row_class])[:, None] * U[dp.row_class, :r]
    Vfull = np.zeros((Xcols, r))
    Vfull[dp.col_ids] = (dp.col_pref / dp.lam_t[dp.col_class])[:, None] * Vt[:r, dp.col_class].T
    if p < d:
        G[p - 1] = Ufull.reshape(ex.rt[p - 1], dims[p - 1], r)
        W = s[:r, None] * Vfull.T                                  # Sigma V^T: r x r~_p
        r1 = G[p].shape
        G[p] = (W @ G[p].reshape(r1[0], -1)).reshape(r, r1[1], r1[2])
        ranks[p] = r
        if rounding == "dynamic":
            d_right = math.sqrt(max(d_right ** 2 - e2, 0.0))
        # first SVD sweep, k = p+1..d-1
        for k in range(p + 1, d):
            r0, n, r1 = G[k - 1].shape
            U, s, Vt = svd(G[k - 1].reshape(r0 * n, r1))
            dl = delta_for(k, True)
            r = _rank_at(s, dl, dims, k, max_rank, eps)
            e2 = float(np.sum(s[r:] ** 2))
            err2 += e2
            sig[k] = s
            used[k] = dl
            G[k - 1] = U[:, :r].reshape(r0, n, r)
            W = s[:r, None] * Vt[:r]
            q0, qn, q1 = G[k].shape
            G[k] = (W @ G[k].reshape(q0, -1)).reshape(r, qn, q1)
            ranks[k] = r
            if rounding == "dynamic":
                d_right = math.sqrt(max(d_right ** 2 - e2, 0.0))
        # QR sweep, k = d..p+1
        for k in range(d, p, -1):
            r0, n, r1 = G[k - 1].shape
            Q, Rm = np.linalg.qr(G[k - 1].reshape(r0, n * r1).T, mode="reduced")
            q = Q.shape[1]
            G[k - 1] = Q.T.reshape(q, n, r1)
            a0, an, a1 = G[k - 2].shape
            G[k - 2] = (G[k - 2].reshape(a0 * an, a1) @ Rm.T).reshape(a0, an, q)
            ranks[k - 1] = q
        start = p
    else:
        # p = d: the middle SVD is the k = d step of the second sweep
        G[d - 1] = Ufull.T.reshape(r, dims[d - 1], 1)
        VS = Vfull * s[:r]
        a0, an, a1 = G[d - 2].shape
        G[d - 2] = (G[d - 2].reshape(a0 * an, a1) @ VS).reshape(a0, an, r)
        ranks[d - 1] = r
        if rounding == "dynamic":
            d_left = math.sqrt(max(d_left ** 2 - e2, 0.0))
        start = d - 1
    # second SVD sweep, k = start..2
    for k in range(start, 1, -1):
        r0, n, r1 = G[k - 1].shape
        U, s, Vt = svd(G[k - 1].reshape(r0, n * r1).T)
        dl = delta_for(k - 1, False)
        r = _rank_at(s, dl, dims, k - 1, max_rank, eps)
        e2 = float(np.sum(s[r:] ** 2))
        err2 += e2
        sig[k - 1] = s
        used[k - 1] = dl
        G[k - 1] = U[:, :r].T.reshape(r, n, r1)
        VS = Vt[:r].T * s[:r]
        a0, an, a1 = G[k - 2].shape
        G[k - 2] = (G[k - 2].reshape(a0 * an, a1) @ VS).reshape(a0, an, r)
        ranks[k - 1] = r
        if rounding == "dynamic":
            d_left = math.sqrt(max(d_left ** 2 - e2, 0.0))
    ranks = [1] + [G[k].shape[2] for k in range(d - 1)] + [1]
    return Result(G, ranks, p, ex.R, Rs, list(ex.rt), norm2, err2,
                  [used.get(k) for k in range(d + 1)], sig, ex, dp, dropped)
