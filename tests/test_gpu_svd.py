"""The dense SVD of the rounding sweeps (S7-S10), through the fasttt_debug_svd
test hook, against LAPACK (numpy) on matrices with chosen singular values.

Shapes cover the three routes: one-sided Jacobi on the matrix (short side small,
long side short), Householder TSQR + Jacobi on R (tall-skinny and wide-short,
the long side cut into several row blocks and tree levels, with a ragged last
block), and the Gram route (both sides large).  Bounds (backward-stable SVD):
  singular values  |sigma - sigma_ref| <= 8 max(M, N) u sigma_1
  reconstruction   ||Z - U diag(sigma) Vt||_F <= 8 max(M, N) u ||Z||_F
  orthogonality    ||U^T U - I||_F, ||Vt Vt^T - I||_F <= 32 max(M, N) u  (r <= rank;
                   the Jacobi rotations accumulate over the sweeps)
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def F():
    from paper_1908_02721_gb300 import fasttt
    return fasttt


def _orth(m, n, rng):
    q, r = np.linalg.qr(rng.standard_normal((m, n)))
    return q * np.sign(np.diag(r))


def _matrix(M, N, kind, seed):
    rng = np.random.default_rng(seed)
    r = min(M, N)
    if kind == "gaussian":
        return rng.standard_normal((M, N))
    if kind == "graded":                     # sigma from 1 down to 1e-14
        sig = 10.0 ** -np.linspace(0.0, 14.0, r)
    elif kind == "rank_deficient":           # half of the singular values exactly zero
        sig = np.concatenate([np.linspace(2.0, 1.0, r - r // 2), np.zeros(r // 2)])
    else:
        raise ValueError(kind)
    return (_orth(M, r, rng) * sig) @ _orth(N, r, rng).T


def _check(F, Z, full_rank=True):
    M, N = Z.shape
    sigma, Uf, Vt = F.debug_svd(torch.from_numpy(Z).cuda())
    Uf, Vt = Uf.cpu().numpy(), Vt.cpu().numpy()
    ref = np.linalg.svd(Z, compute_uv=False)
    s1 = ref[0]
    tol = 8 * max(M, N) * U
    assert np.all(np.diff(sigma) <= 0)
    assert np.max(np.abs(sigma - ref)) <= tol * s1
    assert np.linalg.norm(Z - (Uf * sigma) @ Vt) <= tol * np.linalg.norm(Z)
    k = len(sigma) if full_rank else int(np.sum(ref > 1e-8 * s1))
    assert np.linalg.norm(Uf[:, :k].T @ Uf[:, :k] - np.eye(k)) <= 4 * tol
    assert np.linalg.norm(Vt[:k] @ Vt[:k].T - np.eye(k)) <= 4 * tol


TSQR_SHAPES = [(125000, 50), (50, 125000), (1024, 2), (5000, 64), (70000, 33), (2048 + 7, 17),
               # 64 < n <= 128: blocks of 224 rows, tree stopped at <= 4n stacked rows
               (12800, 128), (128, 12800), (1024, 65), (30000 + 13, 100)]


@pytest.mark.parametrize("shape", TSQR_SHAPES)
def test_tall_skinny_gaussian(F, shape):
    _check(F, _matrix(*shape, "gaussian", seed=shape[0] + shape[1]))


@pytest.mark.parametrize("shape", [(20000, 40), (40, 20000), (3000, 64), (12800, 128)])
def test_tall_skinny_graded(F, shape):
    """Singular values over 14 decades: the small ones are resolved to u sigma_1."""
    _check(F, _matrix(*shape, "graded", seed=7 + shape[0]))


@pytest.mark.parametrize("shape", [(20000, 40), (3000, 60), (5000, 120)])
def test_tall_skinny_rank_deficient(F, shape):
    _check(F, _matrix(*shape, "rank_deficient", seed=9 + shape[0]), full_rank=False)


@pytest.mark.parametrize("shape", [(300, 200), (65, 2000), (900, 100)])
def test_jacobi_route(F, shape):
    _check(F, _matrix(*shape, "gaussian", seed=3 + shape[0]))


def test_gram_route(F):
    """Both sides large: Gram route (singular values well above sqrt(u) sigma_1)."""
    rng = np.random.default_rng(5)
    Z = rng.standard_normal((3000, 1500))
    sigma, Uf, Vt = F.debug_svd(torch.from_numpy(Z).cuda())
    ref = np.linalg.svd(Z, compute_uv=False)
    assert np.max(np.abs(sigma - ref)) <= 1e-12 * ref[0]
    Uf, Vt = Uf.cpu().numpy(), Vt.cpu().numpy()
    assert np.linalg.norm(Z - (Uf * sigma) @ Vt) <= 1e-12 * np.linalg.norm(Z)


def test_svd_hook_rejects_bad_arguments(F):
    with pytest.raises(F.FastTTError):
        F.debug_svd(torch.zeros((3, 4), dtype=torch.float64, device="cuda"), precision="bf16")
