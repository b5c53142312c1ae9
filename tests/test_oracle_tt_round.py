"""Pins for the oracle's TT-rounding (Alg. 2) and TT sum (Lemma 2, eq. (6)), checked
against what the mathematics fixes rather than against the oracle's own code:
LAPACK TT-SVD (Alg. 1) of the dense tensor, exact ranks of constructed TTs, the
error identity of orthogonal truncations, and dense addition."""
import math

import numpy as np
import pytest

from oracle import dense as D


def _random_tt(dims, ranks, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(len(dims))]


def test_tt_sum_is_dense_addition():
    a = _random_tt([3, 4, 5, 2], [1, 2, 3, 2, 1], 1)
    b = _random_tt([3, 4, 5, 2], [1, 3, 1, 4, 1], 2)
    s = D.tt_sum(a, b, beta=-0.5)
    assert [c.shape[0] for c in s] + [1] == [1, 5, 4, 6, 1]
    assert np.allclose(D.tt_full(s), D.tt_full(a) - 0.5 * D.tt_full(b), rtol=0, atol=1e-13)


def test_rounding_a_doubled_tt_recovers_its_ranks():
    """A + A has TT ranks at most those of A; the sum's block construction doubles
    them, and rounding at eps = 1e-12 (or the numerical rank, eps = 0) returns the
    ranks of A and the tensor 2A."""
    dims, ranks = [4, 5, 6, 3], [1, 3, 4, 2, 1]
    a = _random_tt(dims, ranks, 3)
    s = D.tt_sum(a, a)
    for eps in (1e-12, 0.0):
        cores, r, err2 = D.tt_round(s, eps)
        assert r == ranks
        full = D.tt_full(cores)
        ref = 2.0 * D.tt_full(a)
        assert np.linalg.norm(full - ref) <= 1e-12 * np.linalg.norm(ref)


def test_rounding_error_identity_and_bound():
    """Truncations against orthonormal complements are orthogonal: ||A - B||^2 equals
    the sum of the discarded sigma^2, and it stays within (eps ||A||)^2."""
    dims, ranks = [5, 6, 7, 5], [1, 6, 8, 6, 1]
    a = _random_tt(dims, ranks, 4)
    A = D.tt_full(a)
    nA = np.linalg.norm(A)
    for eps in (0.05, 0.3):
        cores, r, err2 = D.tt_round(a, eps)
        B = D.tt_full(cores)
        e2 = np.linalg.norm(A - B) ** 2
        assert abs(e2 - err2) <= 1e-9 * nA * nA
        assert math.sqrt(e2) <= eps * nA * (1 + 1e-12)
        assert all(ri <= r0 for ri, r0 in zip(r, ranks))
        if eps == 0.3:
            assert sum(r) < sum(ranks)   # the tolerance truncates


@pytest.mark.parametrize("eps", [1e-3, 0.05, 0.2])
def test_rounding_of_the_exact_tt_equals_tt_svd(eps):
    """From the exact TT of a dense tensor, TT-rounding performs the same sequential
    delta-truncations as Alg. 1 on the tensor itself: same ranks, same tensor."""
    rng = np.random.default_rng(5)
    dims = [4, 6, 5, 4]
    A = D.tt_full(_random_tt(dims, [1, 3, 5, 3, 1], 6)) + 1e-2 * rng.standard_normal(dims)
    exact, r0, _ = D.tt_svd(A, 0.0)
    assert r0 == [1, 4, 20, 4, 1]
    cores, r, err2 = D.tt_round(exact, eps)
    ref, rr, err2_ref = D.tt_svd(A, eps)
    assert r == rr
    assert np.linalg.norm(D.tt_full(cores) - D.tt_full(ref)) <= 1e-12 * np.linalg.norm(A)
    assert abs(err2 - err2_ref) <= 1e-12 * np.linalg.norm(A) ** 2


def test_rounding_respects_the_rank_cap():
    a = _random_tt([5, 6, 7, 5], [1, 5, 8, 5, 1], 7)
    cores, r, err2 = D.tt_round(a, 0.0, max_rank=3)
    assert r == [1, 3, 3, 3, 1]
    B = D.tt_full(cores)
    assert abs(np.linalg.norm(D.tt_full(a) - B) ** 2 - err2) <= 1e-9 * np.linalg.norm(D.tt_full(a)) ** 2
