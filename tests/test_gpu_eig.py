"""The dense symmetric eigensolver behind the Gram route of the rounding SVDs
(S7-S10), through the fasttt_debug_sym_eig test hook, on matrices with chosen
spectra.  Bounds (backward-stable solver, n u ||G|| scale):
  eigenvalues   |lam - lam_ref| <= 8 n u ||G||_2   (lam_ref: LAPACK syevd, FP64)
  residual      ||G V^T - V^T diag(lam)||_F <= 8 n u ||G||_2
  orthogonality ||V V^T - I||_F <= 8 n u
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


def _orth(n, rng):
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    return q * np.sign(np.diag(r))


def _spectrum(kind, n, rng):
    if kind == "separated":
        lam = np.linspace(0.1, 100.0, n) + 1e-3 * rng.random(n)
    elif kind == "clusters":
        lam = np.repeat(rng.uniform(1.0, 10.0, 10), n // 10 + 1)[:n]
    elif kind == "graded":
        lam = 10.0 ** -np.linspace(0.0, 12.0, n)
    else:
        raise ValueError(kind)
    q = _orth(n, rng)
    G = (q * lam) @ q.T
    return 0.5 * (G + G.T)


def _matrix(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind in ("separated", "clusters", "graded"):
        return _spectrum(kind, n, rng)
    if kind == "rank_deficient":
        B = rng.standard_normal((n // 2, n))
        return B.T @ B
    if kind == "sparse_gram":   # Gram of a sparse N(0,1) matrix, as in the TT-rounding SVDs
        B = rng.standard_normal((4 * n, n)) * (rng.random((4 * n, n)) < 0.02)
        return B.T @ B
    raise ValueError(kind)


def _check(F, G, method):
    n = G.shape[0]
    lam, V = F.debug_sym_eig(torch.from_numpy(G).cuda(), method=method)
    V = V.cpu().numpy()
    ref = np.linalg.eigvalsh(G)
    g2 = np.abs(ref).max()
    bound = 8 * n * U * g2
    assert np.max(np.abs(np.sort(lam) - ref)) <= bound
    res = np.linalg.norm(G @ V.T - V.T * lam)
    assert res <= bound, res / g2
    orth = np.linalg.norm(V @ V.T - np.eye(n))
    assert orth <= 8 * n * U, orth


KINDS = ["separated", "clusters", "graded", "rank_deficient", "sparse_gram"]


@pytest.mark.parametrize("n", [300, 1100])
@pytest.mark.parametrize("kind", KINDS)
def test_library_eigensolver(F, kind, n):
    _check(F, _matrix(kind, n, seed=31 + n), "auto")


@pytest.mark.parametrize("n", [700, 1500])
@pytest.mark.parametrize("kind", ["separated", "graded", "sparse_gram"])
def test_tridiagonal_route_takes_well_separated_spectra(F, kind, n):
    """n = 700: two blocked panels of 64 columns (panel updates on the DFMA GEMM), the
    rest unblocked; n = 1500: fifteen panels, updates on the tensor-core slice GEMM."""
    _check(F, _matrix(kind, n, seed=41), "tridiagonal")


@pytest.mark.parametrize("kind", ["clusters", "rank_deficient"])
def test_tridiagonal_route_meets_the_bounds_or_declines(F, kind):
    G = _matrix(kind, 700, seed=43)
    try:
        _check(F, G, "tridiagonal")
    except F.FastTTError as e:
        assert e.code == F.ENUMERIC


def test_iterative_route(F):
    _check(F, _matrix("sparse_gram", 500, seed=47), "iterative")


def test_eig_hook_rejects_bad_arguments(F):
    with pytest.raises(F.FastTTError):
        F.debug_sym_eig(torch.zeros((3, 4), dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("kind,n", [("separated", 300), ("separated", 1100), ("separated", 2500),
                                    ("sparse_gram", 300), ("sparse_gram", 1100), ("sparse_gram", 2500),
                                    ("clusters", 300)])
def test_fast_route(F, kind, n):
    """FP32 tridiagonal start + FP64-level refinement + Rayleigh-Ritz on close runs."""
    _check(F, _matrix(kind, n, seed=53 + n), "fast")


@pytest.mark.parametrize("kind,n", [("graded", 300), ("graded", 1100), ("rank_deficient", 300),
                                    ("rank_deficient", 1100), ("clusters", 1100)])
def test_fast_route_meets_the_bounds_or_declines(F, kind, n):
    """Spectra with a large cluster below the FP32 start's resolution: the route may
    decline (the library then takes the FP64 tridiagonal route), never answer wrongly."""
    G = _matrix(kind, n, seed=57 + n)
    try:
        _check(F, G, "fast")
    except F.FastTTError as e:
        assert e.code == F.ENUMERIC, e


def test_fast_route_near_clusters(F):
    """Pairs of eigenvalues 1e-9 apart (below the FP32 start's resolution, above the
    FP64 bound): the Rayleigh-Ritz step must separate them."""
    rng = np.random.default_rng(59)
    n = 600
    base = np.linspace(1.0, 10.0, n // 2)
    lam = np.sort(np.concatenate([base, base + 1e-9 * base]))
    q = _orth(n, rng)
    G = (q * lam) @ q.T
    _check(F, 0.5 * (G + G.T), "fast")


def test_fast_route_zero_matrix(F):
    lam, V = F.debug_sym_eig(torch.zeros((50, 50), dtype=torch.float64, device="cuda"), method="fast")
    assert np.all(lam == 0.0)
    assert np.array_equal(V.cpu().numpy(), np.eye(50))
