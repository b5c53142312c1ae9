"""The GEMM engines of the dense rounding contractions (S7-S10), through the
fasttt_debug_gemm test hook, against numpy's FP64 product.

tensor_f64 (tcgen05, 7 exact bf16 slices) is held to the FP64 bound
||C - C_ref||_F <= 4 K u ||A||_F ||B||_F; the FP32-level engines (tcgen05 on 3
slices, split-TF32 mma.sync) to 1e-6 ||A||_F ||B||_F.  Shapes run from one tile
and one K chunk to ragged multi-tile cases and a 2500^3 product.
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


SHAPES = [(128, 64, 64), (128, 64, 1000), (300, 200, 1000), (257, 129, 65), (1, 1, 70), (1000, 37, 2500),
          (2500, 2500, 2500)]


def _mats(M, N, K, seed, graded=False):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    if graded:
        A *= 10.0 ** rng.uniform(-6, 6, size=(M, 1))
        B *= 10.0 ** rng.uniform(-6, 6, size=(1, N))
    return A, B


def _err(F, A, B, engine):
    C = F.debug_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), engine).cpu().numpy()
    ref = A @ B
    return np.linalg.norm(C - ref) / (np.linalg.norm(A) * np.linalg.norm(B))


@pytest.mark.parametrize("shape", SHAPES)
def test_tensor_core_fp64_engine(F, shape):
    M, N, K = shape
    A, B = _mats(M, N, K, seed=M + 7 * N + 13 * K)
    assert _err(F, A, B, "tensor_f64") <= 4 * K * U


@pytest.mark.parametrize("shape", SHAPES[:4])
def test_tensor_core_fp64_engine_graded_rows(F, shape):
    """Rows and columns scaled over 12 decades: each row and column carries its own exponent."""
    M, N, K = shape
    A, B = _mats(M, N, K, seed=3 * M + N + K, graded=True)
    C = F.debug_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), "tensor_f64").cpu().numpy()
    ref = A @ B
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :] * K
    assert np.max(np.abs(C - ref) / scale) <= 8 * U


@pytest.mark.parametrize("engine", ["tensor_f32", "tf32x3"])
@pytest.mark.parametrize("shape", SHAPES[:6])
def test_fp32_level_engines(F, shape, engine):
    M, N, K = shape
    A, B = _mats(M, N, K, seed=M + N + K + 1)
    assert _err(F, A, B, engine) <= 1e-6


def test_dfma_engine(F):
    A, B = _mats(300, 200, 1000, seed=5)
    assert _err(F, A, B, "dfma") <= 4 * 1000 * U


@pytest.mark.parametrize("shape", [(64, 64), (300, 1000), (257, 4100), (1, 70), (1500, 3000)])
@pytest.mark.parametrize("engine", ["tensor_f64", "dfma"])
def test_gram_fp64_engines(F, shape, engine):
    """C = A A^T through the symmetric path (upper tiles only; the tensor engine splits A once)."""
    M, K = shape
    A, _ = _mats(M, 1, K, seed=11 * M + K)
    C = F.debug_gram(torch.from_numpy(A).cuda(), engine).cpu().numpy()
    ref = A @ A.T
    assert np.array_equal(C, C.T)
    assert np.linalg.norm(C - ref) / np.linalg.norm(A) ** 2 <= 4 * K * U


@pytest.mark.parametrize("engine", ["tensor_f32", "tf32x3"])
def test_gram_fp32_level_engines(F, engine):
    A, _ = _mats(400, 1, 2000, seed=17)
    C = F.debug_gram(torch.from_numpy(A).cuda(), engine).cpu().numpy()
    assert np.linalg.norm(C - A @ A.T) / np.linalg.norm(A) ** 2 <= 1e-6


def test_tensor_core_fp64_engine_extreme_rows(F):
    """Rows of zeros, subnormal rows, rows near the top of the exponent range and
    subnormals inside normal rows: the slicing is exact integer work on the bits."""
    rng = np.random.default_rng(23)
    M, N, K = 200, 130, 300
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    A[3] = 0.0
    A[5] *= 1e-310                                   # a whole row of subnormals
    A[7] *= 1e300
    A[9, ::7] = 4e-320                               # subnormals among normal entries
    A[11] = rng.standard_normal(K) * 2.0 ** rng.integers(-1000, -960, size=K)
    B[:, 2] = 0.0
    B[:, 4] *= 1e-300
    C = F.debug_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), "tensor_f64").cpu().numpy()
    ref = A @ B
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :] * K
    scale[scale == 0] = 1.0
    # the dropped bits are below 2^-56 of each row's (column's) maximum; subnormal
    # inputs carry their own absolute rounding of 2^-1075
    err = np.abs(C - ref) - 4.0 * K * 2.0 ** -1074 * (np.abs(B).max(axis=0)[None, :] + np.abs(A).max(axis=1)[:, None])
    assert np.all(err <= 8 * U * scale)
    assert np.all(C[3] == 0.0) and np.all(C[:, 2] == 0.0)
