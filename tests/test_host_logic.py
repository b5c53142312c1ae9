"""The library's host-side decisions against the oracle, with no device: Alg. 9's
choice of p (eq. (10) bounds, eq. (13) flop model, 128-bit exact) and the rank rule of
the rounding (delta tail rule, eps = 0 numerical rank, max_rank cap), through the
host-only hooks fasttt_debug_select_p / fasttt_debug_rank_rule."""
import math

import numpy as np
import pytest

from oracle import dense as D
from oracle import fasttt as O


@pytest.fixture(scope="module")
def F():
    from paper_1908_02721_gb300 import fasttt
    return fasttt


def test_select_p_matches_the_oracle_on_random_cases(F):
    rng = np.random.default_rng(2024)
    for trial in range(400):
        d = int(rng.integers(2, 9))
        big = trial % 4 == 0
        dims = [int(x) for x in rng.integers(1, (2 ** 31 - 1) if big else 200, d)]
        Rs = [int(x) for x in rng.integers(1, (2 ** 31 - 1) if big else 5000, d)]
        max_rank = int(rng.choice([0, 0, 1, 8, 64, 1000]))
        want, _ = O.select_p(dims, Rs, max_rank)
        assert F.debug_select_p(dims, Rs, max_rank) == want, (dims, Rs, max_rank)


def test_select_p_on_the_alg9_example(F):
    """The tensor of the Sec. 3.6 worked example with every R equal to 12000 or 120000."""
    dims = [10, 20, 20, 10, 15, 20, 3]
    for R in (12000, 120000):
        want, _ = O.select_p(dims, [R] * 7, 10)
        assert F.debug_select_p(dims, [R] * 7, 10) == want


def test_select_p_ties_go_to_the_smallest_p(F):
    # a symmetric problem: p and d + 1 - p have equal estimates
    dims, Rs = [7, 7, 7, 7], [50, 50, 50, 50]
    want, fs = O.select_p(dims, Rs)
    assert F.debug_select_p(dims, Rs) == want == fs.index(min(fs)) + 1


def _oracle_rank(s, delta, eps_zero, dims, bond, max_rank):
    tol = D.unfolding_rank_tol(dims, bond, s[0]) if eps_zero else None
    return D.truncation_rank(s, 0.0 if eps_zero else delta, tol, max_rank)


def test_rank_rule_matches_the_oracle(F):
    rng = np.random.default_rng(7)
    for trial in range(600):
        d = int(rng.integers(2, 7))
        dims = [int(x) for x in rng.integers(1, 60, d)]
        bond = int(rng.integers(1, d))
        n = int(rng.integers(1, 80))
        kind = trial % 3
        if kind == 0:
            s = np.sort(rng.random(n))[::-1]
        elif kind == 1:
            s = np.sort(10.0 ** -rng.uniform(0, 18, n))[::-1]
        else:   # exact zeros and repeated values
            s = np.sort(np.round(rng.random(n), 1))[::-1]
        s = np.ascontiguousarray(s)
        eps_zero = trial % 5 == 0
        if eps_zero:
            delta = 0.0
        else:
            # delta at, just below or just above a tail, to exercise the inclusive comparison
            c = int(rng.integers(0, n + 1))
            tail = math.sqrt(sum(float(x) ** 2 for x in s[c:][::-1]))
            delta = [tail, np.nextafter(tail, 0.0), np.nextafter(tail, 1.0), float(rng.random())][trial % 4]
            if delta <= 0.0:
                delta = float(s[0]) * 1e-3
        max_rank = int(rng.choice([0, 0, 1, 3, 10]))
        want = _oracle_rank(s, delta, eps_zero, dims, bond, max_rank)
        got = F.debug_rank_rule(s, delta, eps_zero, dims, bond, max_rank)
        assert got == want, (s, delta, eps_zero, dims, bond, max_rank)


def test_hooks_reject_bad_arguments(F):
    with pytest.raises(F.FastTTError):
        F.debug_select_p([3], [1])
    with pytest.raises(F.FastTTError):
        F.debug_select_p([3, 0], [1, 1])
    with pytest.raises(F.FastTTError):
        F.debug_select_p([3, 4], [1, 2 ** 31])
    with pytest.raises(F.FastTTError):
        F.debug_rank_rule([1.0], 0.1, False, [3, 4], 2)
    with pytest.raises(F.FastTTError):
        F.debug_rank_rule([], 0.1, False, [3, 4], 1)
