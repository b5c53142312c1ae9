"""Seeded synthetic sparse tensors shaped like the FastTT paper's workloads.

This module only draws inputs: COO coordinates and values.  It holds none of
the decomposition's arithmetic, so both the CUDA path and the CPU oracle can
take their inputs from here.  Every generator uses numpy's counter-based
Philox4x32-10 bit generator (Salmon et al., SC'11), keyed by a fixed seed.

Coordinates come back as a C-contiguous ``int32`` array of shape ``(d, nnz)``
(0-based, structure-of-arrays: mode k's indices are row k) and values as a 1-D
``float64`` (or ``float32``) array.  Coordinates are always distinct: draws are
deduplicated keeping the first occurrence and topped up until ``nnz`` distinct
positions exist.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    dims: list
    idx: np.ndarray          # (d, nnz) int32, 0-based
    vals: np.ndarray         # (nnz,) float64 or float32
    eps: float
    max_rank: int = 0        # 0 = no cap
    p: int = 0               # 0 = choose by the flop model (Alg. 9)
    note: str = ""

    @property
    def d(self) -> int:
        return len(self.dims)

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[1])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=seed))


def _split_modes(dims):
    """Split the modes into groups whose mixed-radix products fit in 62 bits."""
    groups, cur, bits = [], [], 0.0
    for k, n in enumerate(dims):
        b = math.log2(max(n, 2))
        if cur and bits + b > 62:
            groups.append(cur)
            cur, bits = [], 0.0
        cur.append(k)
        bits += b
    groups.append(cur)
    return groups


def first_occurrence_mask(idx: np.ndarray, dims) -> np.ndarray:
    """Boolean mask selecting the first occurrence of every distinct coordinate."""
    d, n = idx.shape
    if n == 0:
        return np.zeros(0, dtype=bool)
    keys = []
    for g in _split_modes(dims):
        key = np.zeros(n, dtype=np.int64)
        for k in g:
            key = key * int(dims[k]) + idx[k].astype(np.int64)
        keys.append(key)
    pos = np.arange(n, dtype=np.int64)
    order = np.lexsort([pos] + keys[::-1])
    same = np.ones(n, dtype=bool)
    for key in keys:
        ks = key[order]
        same[1:] &= ks[1:] == ks[:-1]
    same[0] = False
    mask = np.zeros(n, dtype=bool)
    mask[order[~same]] = True
    return mask


def _distinct_draw(draw, dims, nnz, rng, oversample=1.1, max_rounds=64):
    """Call ``draw(rng, count) -> (d, count)`` until ``nnz`` distinct coordinates exist."""
    d = len(dims)
    have = np.zeros((d, 0), dtype=np.int64)
    for _ in range(max_rounds):
        need = nnz - have.shape[1]
        if need <= 0:
            break
        extra = draw(rng, max(16, int(need * oversample)))
        cand = np.concatenate([have, extra.astype(np.int64)], axis=1)
        have = cand[:, first_occurrence_mask(cand, dims)]
    if have.shape[1] < nnz:
        raise RuntimeError("could not draw enough distinct coordinates")
    return np.ascontiguousarray(have[:, :nnz].astype(np.int32))


def uniform_positions(dims, nnz, rng):
    def draw(r, count):
        return np.stack([r.integers(0, n, size=count) for n in dims])
    return _distinct_draw(draw, dims, nnz, rng)


def random_sparse(dims, nnz, seed, dist="uniform", eps=0.0, p=0, max_rank=0, name=None):
    """Distinct uniform positions; values U(0,1) ('uniform'), N(0,1) ('normal') or U(-1,1) ('signed')."""
    rng = _rng(seed)
    idx = uniform_positions(dims, nnz, rng)
    if dist == "uniform":
        vals = rng.random(nnz)
    elif dist == "normal":
        vals = rng.standard_normal(nnz)
    elif dist == "signed":
        vals = rng.uniform(-1.0, 1.0, nnz)
    elif dist == "ones":
        vals = np.ones(nnz)
    else:
        raise ValueError(dist)
    return Workload(name or f"random{tuple(dims)}x{nnz}", list(dims), idx, vals.astype(np.float64),
                    eps, max_rank, p)


# ---------------------------------------------------------------- paper-shaped workloads

def exact_small(seed: int = 1) -> Workload:
    """4-way 20^4 tensor, 1,000 distinct uniform positions, U(0,1) values, eps = 0."""
    w = random_sparse([20] * 4, 1000, seed, "uniform", eps=0.0)
    w.name = "4-way 20^4, 1e3 nnz, U(0,1), eps=0"
    return w


def uniform5(seed: int = 2, nnz: int = 100_000, n: int = 50) -> Workload:
    """5-way 50^5 tensor, 1e5 distinct uniform positions, N(0,1) values, eps = 1e-8."""
    w = random_sparse([n] * 5, nnz, seed, "normal", eps=1e-8)
    w.name = f"5-way {n}^5, {nnz:.0e} nnz, N(0,1), eps=1e-8"
    return w


def banded_qtt(m: int = 20, seed: int = 3, offband: int = 5, band: int = 2, eps: float = 1e-6) -> Workload:
    """2^m x 2^m matrix: a (2*band+1)-diagonal band plus ``offband`` uniform
    off-band entries per row, U(-1,1) values; row and column bits interleaved
    (most significant first) into an m-way tensor of mode size 4, mode index
    = 2*row_bit + col_bit."""
    rng = _rng(seed)
    N = 1 << m
    rows, cols = [], []
    r = np.arange(N, dtype=np.int64)
    for off in range(-band, band + 1):
        c = r + off
        ok = (c >= 0) & (c < N)
        rows.append(r[ok])
        cols.append(c[ok])
    # off-band: per row, `offband` distinct columns with |col - row| > band
    picked = np.full((N, offband), -1, dtype=np.int64)
    for j in range(offband):
        todo = np.arange(N, dtype=np.int64)
        for _ in range(64):
            if todo.size == 0:
                break
            c = rng.integers(0, N, size=todo.size)
            bad = np.abs(c - todo) <= band
            for jj in range(j):
                bad |= c == picked[todo, jj]
            picked[todo[~bad], j] = c[~bad]
            todo = todo[bad]
        if todo.size:
            raise RuntimeError("off-band draw did not converge")
    rows.append(np.repeat(r, offband))
    cols.append(picked.reshape(-1))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = rng.uniform(-1.0, 1.0, rows.size)
    idx = np.empty((m, rows.size), dtype=np.int32)
    for k in range(m):
        shift = m - 1 - k
        idx[k] = (((rows >> shift) & 1) * 2 + ((cols >> shift) & 1)).astype(np.int32)
    return Workload(f"QTT 2^{m}x2^{m} band{2*band+1}+{offband}/row, U(-1,1), eps={eps:g}", [4] * m,
                    np.ascontiguousarray(idx), vals, eps)


def zipf_tt(seed: int = 4, nnz: int = 10_000_000, d: int = 8, n: int = 100, rank: int = 8,
            s: float = 1.2, noise: float = 1e-3, eps: float = 1e-4, max_rank: int = 64) -> Workload:
    """d-way n^d tensor; indices per mode truncated Zipf(s) on 1..n (mapped to 0..n-1);
    values = a random rank-``rank`` TT (cores N(0, 1/sqrt(rank))) at those positions
    plus ``noise``*N(0,1), stored as float32."""
    rng = _rng(seed)
    k = np.arange(1, n + 1, dtype=np.float64)
    pmf = k ** (-s)
    pmf /= pmf.sum()

    def draw(r, count):
        return np.stack([r.choice(n, size=count, p=pmf) for _ in range(d)])

    idx = _distinct_draw(draw, [n] * d, nnz, rng, oversample=1.25)
    ranks = [1] + [rank] * (d - 1) + [1]
    cores = [rng.standard_normal((ranks[j], n, ranks[j + 1])) / math.sqrt(rank) for j in range(d)]
    # synthesis of the values from the planted cores (input preparation only)
    acc = cores[0][0, idx[0], :]
    for j in range(1, d):
        acc = np.einsum("ea,aeb->eb", acc, cores[j][:, idx[j], :])
    vals = acc[:, 0] + noise * rng.standard_normal(nnz)
    return Workload(f"Zipf({s}) {d}-way {n}^{d}, {nnz:.0e} nnz, rank-{rank} TT + noise, f32",
                    [n] * d, idx, vals.astype(np.float32), eps, max_rank)


def clustered(seed: int = 5, nnz: int = 50_000_000, d: int = 12, n: int = 64, clusters: int = 1000,
              sigma: float = 4.0, eps: float = 1e-5, max_rank: int = 128) -> Workload:
    """d-way n^d tensor, nnz positions in Gaussian clusters (centres uniform,
    offsets round(N(0, sigma)) per mode, clipped to [0, n-1]), U(0,1) values."""
    rng = _rng(seed)
    centres = rng.uniform(0, n, size=(d, clusters))

    def draw(r, count):
        c = r.integers(0, clusters, size=count)
        pos = np.rint(centres[:, c] + r.normal(0.0, sigma, size=(d, count)))
        return np.clip(pos, 0, n - 1).astype(np.int64)

    idx = _distinct_draw(draw, [n] * d, nnz, rng, oversample=1.05)
    vals = rng.random(nnz)
    return Workload(f"clustered {d}-way {n}^{d}, {nnz:.0e} nnz, {clusters} clusters, U(0,1)",
                    [n] * d, idx, vals, eps, max_rank)


def fdm7(n: int, coeffs: str = "pattern", seed: int = 6, eps: float = 1e-14) -> Workload:
    """7-point finite-difference matrix of an n x n x n grid as a 3-way MPO-ordered
    tensor: mode k has size n*n and index row_k*n + col_k (grid coordinate k of
    the row and of the column).  'pattern': 6 on the diagonal, -1 off it;
    'random': U(0,1) coefficients."""
    rng = _rng(seed)
    g = np.arange(n)
    I1, I2, I3 = np.meshgrid(g, g, g, indexing="ij")
    I = np.stack([I1.ravel(), I2.ravel(), I3.ravel()])
    rows, cols = [I], [I]
    vals = [np.full(I.shape[1], 6.0)]
    for ax in range(3):
        for s in (-1, 1):
            J = I.copy()
            J[ax] += s
            ok = (J[ax] >= 0) & (J[ax] < n)
            rows.append(I[:, ok])
            cols.append(J[:, ok])
            vals.append(np.full(ok.sum(), -1.0))
    R = np.concatenate(rows, axis=1)
    C = np.concatenate(cols, axis=1)
    v = np.concatenate(vals)
    if coeffs == "random":
        v = rng.random(v.size)
    idx = (R * n + C).astype(np.int32)
    return Workload(f"FDM 7-point {n}^3 -> 3-way MPO, {coeffs}", [n * n] * 3,
                    np.ascontiguousarray(idx), v, eps)


CONFIGS = {
    1: exact_small,
    2: uniform5,
}


def random_tt(dims, ranks, seed: int, decay: float = 1.0):
    """Cores of a random TT (r_{k-1}, n_k, r_k), N(0,1) entries, FP64.  decay < 1
    scales slice j of every core's right bond by decay**j, so the unfoldings'
    singular values fall off geometrically (well-separated truncation points)."""
    rng = _rng(seed)
    cores = []
    for k, n in enumerate(dims):
        G = rng.standard_normal((ranks[k], n, ranks[k + 1]))
        if decay != 1.0:
            G = G * (decay ** np.arange(ranks[k + 1]))[None, None, :]
        cores.append(G)
    return cores


def sample_positions(w: Workload, n_nonzero: int, n_uniform: int, seed: int) -> np.ndarray:
    """Positions at which two TTs of the workload's shape are compared entry by
    entry: ``n_nonzero`` of the workload's nonzero coordinates (drawn without
    replacement) followed by ``n_uniform`` uniform coordinates of the whole
    index space.  (d, n_nonzero + n_uniform) int32."""
    rng = _rng(seed)
    pick = rng.choice(w.nnz, size=min(n_nonzero, w.nnz), replace=False)
    uni = np.stack([rng.integers(0, n, size=n_uniform) for n in w.dims]) if n_uniform else \
        np.zeros((w.d, 0), dtype=np.int64)
    return np.ascontiguousarray(np.concatenate([w.idx[:, pick].astype(np.int64), uni], axis=1).astype(np.int32))
