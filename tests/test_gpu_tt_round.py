"""GPU TT-rounding (Alg. 2) and TT sum (Lemma 2) through the C ABI
(fasttt_tt_round, fasttt_tt_add) against the oracle (oracle.dense.tt_round,
oracle.dense.tt_sum) on seeded random TTs.

Bars: the sum is a copy and one product per entry, compared bit for bit.  Rounding
results are unique only as tensors (the cores carry an orthogonal gauge), so the
ranks must be equal, the rounded tensors must agree to 1e-12 of ||A|| in FP64
(1e-6 in mixed precision), ||A||^2 to twice that relative, and err2 (the discarded
sigma^2) to 1e-10 relative or 1e-24 ||A||^2 absolute."""
import numpy as np
import pytest
import torch

from oracle import dense as D
from paper_1908_02721_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1908_02721_gb300 import fasttt
    return fasttt


def _cuda(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def _host(tt):
    return [c.cpu().numpy() for c in tt.cores()]


def _tt_dist(a, b):
    """||A - B||_F of two TTs through the oracle's sum and QR-sweep norm."""
    return D.tt_norm(D.tt_sum(a, b, beta=-1.0))


def _check_round(F, cores, eps, max_rank=0, tol=1e-12, precision="fp64"):
    ref, ref_ranks, ref_err2 = D.tt_round(cores, eps, max_rank)
    out = F.tt_round(_cuda(cores), eps, max_rank=max_rank, precision=precision)
    assert out.ranks == ref_ranks
    got = _host(out)
    for k, G in enumerate(got):
        assert G.shape == ref[k].shape
    normA = D.tt_norm(cores)
    assert _tt_dist(got, ref) <= tol * normA
    # ||A||^2 from the first bond's singular values.  Backward-stable factorisations
    # commit errors of order u prod_k ||G_k||_F, which exceeds u ||A||_F by the
    # cancellation factor prod_k ||G_k|| / ||A|| of the input TT (560 for the rank-300 case)
    cond = float(np.prod([np.linalg.norm(G) for G in cores])) / normA
    rel = abs(out.stats["norm2"] - normA ** 2) / normA ** 2
    assert rel <= max(2 * tol, 64 * 2.0 ** -53 * cond), (rel, cond)
    if precision == "fp64":
        assert abs(out.stats["err2"] - ref_err2) <= max(1e-10 * ref_err2, 1e-24 * normA ** 2)
    # the first d-1 cores come out left-orthonormal
    for G in got[:-1]:
        U = G.reshape(-1, G.shape[2])
        assert np.linalg.norm(U.T @ U - np.eye(U.shape[1])) <= (1e-12 if precision == "fp64" else 1e-5)
    return out


@pytest.mark.parametrize("dims,ranks", [([4, 5, 6, 5, 4], [1, 3, 7, 6, 3, 1]),
                                        ([7, 3, 9], [1, 5, 4, 1]),
                                        ([2, 2, 2, 2, 2, 2, 2], [1, 2, 4, 8, 8, 4, 2, 1]),
                                        ([11, 13], [1, 9, 1])])
def test_numerical_ranks_at_eps0(F, dims, ranks):
    _check_round(F, W.random_tt(dims, ranks, seed=71 + len(dims)), 0.0)


@pytest.mark.parametrize("eps", [1e-3, 1e-1, 0.5])
def test_truncation_matches_the_oracle(F, eps):
    cores = W.random_tt([6, 7, 8, 7, 6], [1, 6, 20, 20, 6, 1], seed=81, decay=0.5)
    out = _check_round(F, cores, eps)
    assert out.stats["err2"] <= eps ** 2 * out.stats["norm2"] * (1 + 1e-12)


def test_rank_cap(F):
    cores = W.random_tt([5, 6, 7, 6], [1, 5, 12, 6, 1], seed=83, decay=0.6)
    out = _check_round(F, cores, 1e-12, max_rank=4)
    assert max(out.ranks) == 4


def test_sum_is_bit_exact(F):
    a = W.random_tt([3, 4, 5, 2], [1, 2, 3, 2, 1], seed=85)
    b = W.random_tt([3, 4, 5, 2], [1, 3, 1, 4, 1], seed=86)
    for beta in (1.0, -0.37):
        s = F.tt_add(_cuda(a), _cuda(b), beta=beta)
        ref = D.tt_sum(a, b, beta=beta)
        assert s.ranks == [1, 5, 4, 6, 1]
        for G, R in zip(_host(s), ref):
            assert np.array_equal(G, R)


def test_sum_of_one_mode_tts(F):
    a = W.random_tt([9], [1, 1], seed=87)
    b = W.random_tt([9], [1, 1], seed=88)
    s = F.tt_add(_cuda(a), _cuda(b), beta=-2.5)
    assert np.array_equal(_host(s)[0], D.tt_sum(a, b, beta=-2.5)[0])
    r = F.tt_round(s, 0.0)
    assert r.ranks == [1, 1]
    assert np.array_equal(_host(r)[0], _host(s)[0])


def test_doubled_tt_rounds_back_to_its_ranks(F):
    """A + A: the block construction doubles the ranks; rounding (Alg. 2) returns A's
    ranks and the tensor 2A, as the oracle does."""
    dims, ranks = [5, 6, 7, 6, 5], [1, 4, 9, 8, 3, 1]
    a = W.random_tt(dims, ranks, seed=89)
    s = F.tt_add(_cuda(a), _cuda(a))
    assert s.ranks == [1, 8, 18, 16, 6, 1]
    r = F.tt_round(s, 1e-12)
    assert r.ranks == ranks
    two_a = [2.0 * a[0]] + a[1:]
    assert _tt_dist(_host(r), two_a) <= 1e-12 * D.tt_norm(two_a)
    _check_round(F, D.tt_sum(a, a), 1e-12)


def test_difference_of_close_tts(F):
    """A - B with B = A + 1e-6 C: rounding the Lemma 2 difference at eps = 1e-8 keeps
    the small difference to the accuracy the FP64 cores allow (absolute u ||A||)."""
    dims = [6, 5, 7, 5]
    a = W.random_tt(dims, [1, 4, 5, 3, 1], seed=91)
    c = W.random_tt(dims, [1, 2, 2, 2, 1], seed=92)
    b = D.tt_sum(a, c, beta=1e-6)
    diff = F.tt_add(_cuda(a), _cuda(b), beta=-1.0)
    r = F.tt_round(diff, 1e-8)
    ref, ref_ranks, _ = D.tt_round(D.tt_sum(a, b, beta=-1.0), 1e-8)
    target = [-1e-6 * c[0]] + c[1:]
    nA = D.tt_norm(a)
    assert _tt_dist(_host(r), target) <= 1e-13 * nA
    assert _tt_dist(ref, target) <= 1e-13 * nA
    assert r.ranks == ref_ranks


def test_rounding_a_handle_in_place_of_cores(F):
    a = W.random_tt([4, 5, 6], [1, 3, 4, 1], seed=93)
    s = F.tt_add(_cuda(a), _cuda(a), beta=0.5)
    r = F.tt_round(s, 0.0)
    ref, ref_ranks, _ = D.tt_round(D.tt_sum(a, a, beta=0.5), 0.0)
    assert r.ranks == ref_ranks
    assert _tt_dist(_host(r), ref) <= 1e-12 * D.tt_norm(ref)


def test_large_ranks_take_the_tensor_core_products(F):
    """Rank 300 at mode size 32: the products multiplying the factors into the
    neighbouring cores (1024 x 300 x 300) run on the tensor cores; checked as tensors
    through the oracle's TT arithmetic."""
    dims, ranks = [32, 32, 32, 32], [1, 32, 300, 32, 1]
    cores = W.random_tt(dims, ranks, seed=95, decay=0.98)
    out = _check_round(F, cores, 1e-3)
    assert 32 < out.ranks[2] < 300


def test_mixed_precision(F):
    cores = W.random_tt([6, 7, 8, 7, 6], [1, 6, 20, 20, 6, 1], seed=97, decay=0.5)
    _check_round(F, cores, 1e-3, tol=1e-6, precision="mixed")


def test_rejects_bad_arguments(F):
    a = _cuda(W.random_tt([3, 4], [1, 2, 1], seed=99))
    with pytest.raises(F.FastTTError) as e:
        F.tt_round([torch.zeros((2, 3, 2), dtype=torch.float64, device="cuda"),
                    torch.zeros((2, 4, 1), dtype=torch.float64, device="cuda")], 0.1)
    assert e.value.code == F.EINVAL
    with pytest.raises(F.FastTTError):
        F.tt_round(a, -1.0)
    b = _cuda(W.random_tt([3, 5], [1, 2, 1], seed=100))
    with pytest.raises(F.FastTTError):
        F.tt_add(a, b)
