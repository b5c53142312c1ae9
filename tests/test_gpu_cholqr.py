"""CholeskyQR2 (the QR factorisation of Alg. 6's right-to-left sweep and the
re-orthonormalisation of the mixed precision), through the fasttt_debug_cholqr
test hook, on matrices with chosen condition numbers.

A QR factorisation Z = R^T Q of the rows of Z is fixed by three properties, each
checked against bounds of backward-stable arithmetic at the products' precision:
  orthogonality   ||Q Q^T - I||_F <= 16 M u
  residual        ||Z - R^T Q||_F <= 16 M u ||Z||_F   (a substitution, not an inverse:
                  independent of kappa(Z))
  R upper triangular with a positive diagonal, and equal to LAPACK's R of Z^T
  (signs fixed) within kappa(Z) * 16 M u (the conditioning of the QR factor).
u = 2^-53 in FP64, 2^-24 for the FP32-level products of the mixed precision.
Shapes span one 64 x 64 Cholesky leaf, ragged splits and several levels, and a solve
wide enough for 128 columns per block.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1908_02721_gb300 import fasttt
    return fasttt


def _matrix(M, N, kappa, seed):
    rng = np.random.default_rng(seed)
    qa, _ = np.linalg.qr(rng.standard_normal((M, M)))
    qb, _ = np.linalg.qr(rng.standard_normal((N, M)))
    sig = kappa ** -np.linspace(0.0, 1.0, M)
    return (qa * sig) @ qb.T


def _check(F, Z, kappa, precision):
    M, N = Z.shape
    u = 2.0 ** -53 if precision == "fp64" else 2.0 ** -24
    Q, R = F.debug_cholqr(torch.from_numpy(Z).cuda(), precision)
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    tol = 16 * M * u
    assert np.linalg.norm(Q @ Q.T - np.eye(M)) <= tol
    assert np.linalg.norm(Z - R.T @ Q) <= tol * np.linalg.norm(Z)
    assert np.array_equal(np.triu(R), R)
    assert np.all(np.diag(R) > 0)
    _, Rref = np.linalg.qr(Z.T)
    Rref = Rref * np.sign(np.diag(Rref))[:, None]
    assert np.linalg.norm(R - Rref) <= kappa * tol * np.linalg.norm(Rref)


@pytest.mark.parametrize("M,N", [(1, 5), (64, 64), (100, 300), (257, 1000), (1030, 2100), (100, 40000)])
@pytest.mark.parametrize("kappa", [1.0, 1e3, 1e6])
def test_cholqr2_fp64(F, M, N, kappa):
    _check(F, _matrix(M, N, kappa, M + N), kappa, "fp64")


@pytest.mark.parametrize("M,N", [(64, 200), (300, 2000), (1030, 2100)])
def test_cholqr2_mixed_well_conditioned(F, M, N):
    _check(F, _matrix(M, N, 10.0, M * 7 + N), 10.0, "mixed")


@pytest.mark.parametrize("precision,kappa", [("fp64", 1e12), ("mixed", 1e6)])
def test_cholqr2_reports_breakdown(F, precision, kappa):
    # beyond u^{-1/2} of the Gram's precision the factorisation must fail loudly
    Z = _matrix(200, 400, kappa, 5)
    with pytest.raises(F.FastTTError) as e:
        F.debug_cholqr(torch.from_numpy(Z).cuda(), precision)
    assert e.value.code == F.ENUMERIC
    # the library stays usable after the failure
    _check(F, _matrix(100, 300, 10.0, 6), 10.0, "fp64")
