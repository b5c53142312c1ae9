"""Dense brute force for small tensors (test infrastructure only).

Conventions follow Section 2.2 of the paper: row-major vectorisation with the
last index fastest; the k-unfolding has rows (i_1..i_k) and columns
(i_{k+1}..i_d); TT core k has shape r_{k-1} x n_k x r_k with r_0 = r_d = 1
(Section 2.3).  Indices are 0-based here.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

EPS_MACH = 2.0 ** -52   # numpy's float64 eps, the unit used by matrix_rank's default tolerance


def full_from_coo(idx, vals, dims):
    """The dense tensor A with A[idx[:, e]] = vals[e] (Section 2.1)."""
    A = np.zeros(tuple(int(n) for n in dims), dtype=np.float64)
    A[tuple(np.asarray(idx, dtype=np.int64))] = np.asarray(vals, dtype=np.float64)
    return A


def unfold(A, k):
    """k-unfolding (Section 2.2, Definition of unfolding): prod(n_1..n_k) x prod(n_{k+1}..n_d)."""
    rows = int(np.prod(A.shape[:k], dtype=object))
    return A.reshape(rows, -1)


def tt_full(cores):
    """Contract TT cores into the dense tensor (entry formula of Section 2.3)."""
    T = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])
    shape = [cores[0].shape[1]]
    for G in cores[1:]:
        r0, n, r1 = G.shape
        T = T.reshape(-1, r0) @ G.reshape(r0, n * r1)
        shape.append(n)
    return T.reshape(shape)


def truncation_rank(s, delta, numerical_tol=None, max_rank=0):
    """Smallest r >= 1 whose discarded tail sqrt(sum_{i>r} s_i^2) is <= delta
    (delta-truncated SVD, Alg. 1 / Alg. 6).  With delta == 0 the tail test is
    replaced by the numerical rank s_i > numerical_tol (the paper's eps = 0 case,
    Section 3.3).  A positive max_rank caps the result (fixed-rank variant,
    Section 3.4).  Tail sums run from the smallest singular value upwards."""
    s = np.asarray(s, dtype=np.float64)
    n = s.size
    if n == 0:
        return 0
    if delta > 0.0:
        tail = np.zeros(n + 1)
        acc = 0.0
        for i in range(n - 1, -1, -1):
            acc += s[i] * s[i]
            tail[i] = acc          # tail[i] = sum_{j>=i} s_j^2 (0-based)
        d2 = delta * delta
        r = n
        for cand in range(1, n + 1):
            if tail[cand] <= d2:   # tail[n] = 0
                r = cand
                break
    else:
        tol = 0.0 if numerical_tol is None else numerical_tol
        r = max(1, int(np.count_nonzero(s > tol)))
    if max_rank and max_rank > 0:
        r = min(r, max_rank)
    return r


def unfolding_rank_tol(dims, k, sigma1):
    """numpy.linalg.matrix_rank's default tolerance for the k-unfolding of A."""
    m = int(np.prod([int(n) for n in dims[:k]], dtype=object))
    n = int(np.prod([int(n) for n in dims[k:]], dtype=object))
    return max(m, n) * EPS_MACH * sigma1


def tt_svd(A, eps, max_rank=0):
    """Alg. 1 (TT-SVD): d-1 sequential delta-truncated SVDs, delta = eps*||A||/sqrt(d-1)."""
    dims = A.shape
    d = len(dims)
    normA = math.sqrt(math.fsum((A * A).ravel()))
    delta = eps / math.sqrt(d - 1) * normA if d > 1 else 0.0
    C = A.copy()
    r_prev = 1
    cores, ranks, err2 = [], [1], 0.0
    for k in range(d - 1):
        C = C.reshape(r_prev * dims[k], -1)
        U, s, Vt = scipy.linalg.svd(C, full_matrices=False, lapack_driver="gesvd")
        tol = unfolding_rank_tol(dims, k + 1, s[0] if s.size else 0.0)
        r = truncation_rank(s, delta, tol, max_rank)
        err2 += float(np.sum(s[r:] ** 2))
        cores.append(U[:, :r].reshape(r_prev, dims[k], r))
        C = s[:r, None] * Vt[:r]
        ranks.append(r)
        r_prev = r
    cores.append(C.reshape(r_prev, dims[-1], 1))
    ranks.append(1)
    return cores, ranks, err2


def sequential_projection(A, eps, p, max_rank=0):
    """The plain definition FastTT reaches in exact arithmetic: best truncation of
    the k-unfoldings of the current tensor for bonds p..d-1 (left-to-right), then
    bonds p-1..1 (right-to-left), each with delta_k of eq. (11).  Returns the
    approximating dense tensor and the bond ranks."""
    dims = A.shape
    d = len(dims)
    normA = math.sqrt(math.fsum((A * A).ravel()))
    delta = eps * normA / (math.sqrt(p - 1) + math.sqrt(d - p))
    B = A.copy()
    ranks = [1] + [0] * (d - 1) + [1]
    order = list(range(p, d)) + list(range(p - 1, 0, -1))
    for k in order:
        M = unfold(B, k)
        U, s, Vt = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
        tol = unfolding_rank_tol(dims, k, s[0] if s.size else 0.0)
        r = truncation_rank(s, delta, tol, max_rank)
        B = ((U[:, :r] * s[:r]) @ Vt[:r]).reshape(dims)
        ranks[k] = r
    return B, ranks


def tt_round(cores, eps, max_rank=0):
    """Alg. 2 (TT-rounding of a TT given by its cores), Section 2.4.

    1. Right-to-left orthogonalisation: for k = d..2 the QR factorisation of the
       transposed 1-unfolding of core k, unfold_1(G_k)^T = Q R; core k becomes Q^T
       (its rows orthonormal) and R^T is absorbed into core k-1 (mode-3 product).
    2. Afterwards ||A||_F = ||G_1||_F, and delta = eps ||A||_F / sqrt(d-1).
    3. Left-to-right compression: for k = 1..d-1 the delta-truncated SVD of the
       2-unfolding of core k, U S V^T; core k becomes U and S V^T is absorbed into
       core k+1 (mode-1 product).
    The rank rule is truncation_rank's, with eps = 0 meaning the numerical rank of
    the k-unfolding of A (the tolerance numpy.linalg.matrix_rank uses for it).
    Returns (cores, ranks, err2) with err2 the sum of the discarded sigma^2."""
    G = [np.array(c, dtype=np.float64, copy=True) for c in cores]
    d = len(G)
    dims = [c.shape[1] for c in G]
    for k in range(d - 1, 0, -1):
        r0, n, r1 = G[k].shape
        Q, R = np.linalg.qr(G[k].reshape(r0, n * r1).T, mode="reduced")   # (n r1) x q, q x r0
        q = Q.shape[1]
        G[k] = Q.T.reshape(q, n, r1)
        a0, an, _ = G[k - 1].shape
        G[k - 1] = (G[k - 1].reshape(a0 * an, r0) @ R.T).reshape(a0, an, q)
    normA = math.sqrt(math.fsum((G[0] * G[0]).ravel()))
    delta = eps * normA / math.sqrt(d - 1) if d > 1 else 0.0
    ranks, err2 = [1], 0.0
    for k in range(d - 1):
        r0, n, r1 = G[k].shape
        U, s, Vt = scipy.linalg.svd(G[k].reshape(r0 * n, r1), full_matrices=False, lapack_driver="gesvd")
        tol = unfolding_rank_tol(dims, k + 1, s[0] if s.size else 0.0)
        r = truncation_rank(s, delta, tol, max_rank)
        err2 += float(np.sum(s[r:] ** 2))
        G[k] = U[:, :r].reshape(r0, n, r)
        b0, bn, b1 = G[k + 1].shape
        G[k + 1] = ((s[:r, None] * Vt[:r]) @ G[k + 1].reshape(b0, bn * b1)).reshape(r, bn, b1)
        ranks.append(r)
    ranks.append(1)
    return G, ranks, err2


def tt_sum(a_cores, b_cores, beta=1.0):
    """Cores of A + beta*B by the block construction of Lemma 2 (eq. (6))."""
    d = len(a_cores)
    out = []
    for k, (Ga, Gb) in enumerate(zip(a_cores, b_cores)):
        ra0, n, ra1 = Ga.shape
        rb0, _, rb1 = Gb.shape
        if d == 1:
            out.append(Ga + beta * Gb)
        elif k == 0:
            C = np.zeros((1, n, ra1 + rb1))
            C[:, :, :ra1] = Ga
            C[:, :, ra1:] = beta * Gb
            out.append(C)
        elif k == d - 1:
            C = np.zeros((ra0 + rb0, n, 1))
            C[:ra0] = Ga
            C[ra0:] = Gb
            out.append(C)
        else:
            C = np.zeros((ra0 + rb0, n, ra1 + rb1))
            C[:ra0, :, :ra1] = Ga
            C[ra0:, :, ra1:] = Gb
            out.append(C)
    return out


def tt_norm(cores):
    """Frobenius norm of a TT by a left-to-right QR sweep; the norm of the last
    core is the answer (no squared-norm cancellation)."""
    R = np.ones((1, 1))
    for G in cores:
        r0, n, r1 = G.shape
        M = (R @ G.reshape(r0, n * r1)).reshape(-1, r1)
        Q, R = np.linalg.qr(M, mode="reduced")
    return float(abs(R).reshape(-1)[0]) if R.size == 1 else float(np.linalg.norm(R))


def tt_diff_norm(a_cores, b_cores):
    """||A - B||_F for two TTs, through the TT difference of Lemma 2."""
    return tt_norm(tt_sum(a_cores, b_cores, -1.0))
