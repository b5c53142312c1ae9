// FP64 Cholesky factorisation on the GPU and CholeskyQR2, plus the probe that
// measures how far an FP32-level Gram matrix is from the exact one.
//
// Alg. 6 needs, in its right-to-left sweep, a QR factorisation of unfold_1^T(G_k)
// (any Q with orthonormal columns serves), and the mixed-precision rounding needs
// the factor that a low-precision projection leaves nearly orthonormal made
// orthonormal again.  Both are CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa,
// Yamamoto, 2014): for the rows of Z (M x N, M <= N),
//     H = Z Z^T,  H = R^T R (Cholesky, R upper),  Z <- R^-T Z,      twice,
// so that Z_in = (R_2 R_1)^T Q with Q's rows orthonormal to rounding level when
// kappa(Z) stays below about u^{-1/2} of the Gram's precision.  The Cholesky
// factorisation and the triangular solves are recursive (halving to 64 x 64
// leaves): the off-diagonal work is GEMMs (FP64-level slice GEMMs, or FP32-level
// ones in mixed precision for the Gram and the solve updates), the leaves run in
// one block's shared memory in FP64 (64 x 64 Cholesky leaves, 32 x 32 solve
// leaves).  The triangular solve is a substitution (never an explicit inverse), so
// the residual Z - R^T Q stays at the rounding level of the products whatever R's
// condition number.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "dense.cuh"

namespace fasttt {

namespace {

constexpr int kLeaf = 64;        // Cholesky leaves
constexpr int kSolveLeaf = 32;   // triangular-solve leaves: a leaf's FP64 work per column is
                                 // kSolveLeaf^2 / 2 on one warp, the rest goes to GEMMs
constexpr int kMaxDevices = 64;

#define CHOL_GRID_STRIDE(i, n)                                                     \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

// Upper Cholesky factor of the nb x nb (nb <= 64) symmetric block at H (leading
// dimension ld, upper triangle read), in place: H's upper triangle <- R with
// block = R^T R, strict lower triangle <- 0.  A pivot at or below `tiny` (or not
// finite) sets *info; the factorisation then carries on with pivot 1 so that
// nothing below turns into NaN (the caller discards the result).
__global__ void chol_leaf_kernel(double* H, int64_t ld, int nb, double tiny, int* info) {
  __shared__ double A[kLeaf][kLeaf + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    A[i][j] = (j >= i) ? H[(int64_t)i * ld + j] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    double piv = A[k][k];
    if (!(piv > tiny) || !isfinite(piv)) {
      if (threadIdx.x == 0) atomicExch(info, 1);
      piv = 1.0;
    }
    const double rk = sqrt(piv);
    __syncthreads();   // every thread has read A[k][k]
    for (int j = k + threadIdx.x; j < nb; j += blockDim.x) A[k][j] = (j == k) ? rk : A[k][j] / rk;
    __syncthreads();
    // trailing update of the upper triangle: a warp per row, lanes along it
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = k + 1 + warp; i < nb; i += nw) {
      const double aki = A[k][i];
      for (int j = i + lane; j < nb; j += 32) A[i][j] -= aki * A[k][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    H[(int64_t)i * ld + j] = (j >= i) ? A[i][j] : 0.0;
  }
}

// Forward substitution R^T X = B for the nb x nb upper R at R (leading dimension
// ldr), B (nb rows x ncols, row stride ldb, unit column stride) overwritten by X.
// One thread per column of B; the block's NB x TC tile of B is staged in shared
// memory with all its loads in flight at once, so the substitution chain reads
// shared memory only; the solution overwrites the tile row by row.
constexpr int kTrsmCols = 128;
template <int NB, int TC>
__global__ void __launch_bounds__(TC) trsm_leaf_kernel(const double* R, int64_t ldr, int nb, double* B,
                                                       int64_t ldb, int64_t ncols) {
  extern __shared__ double tsm[];
  double(*L)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(tsm);            // L = R^T, identity-padded
  double(*T)[TC + 1] = reinterpret_cast<double(*)[TC + 1]>(tsm + NB * (NB + 1));
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int j = e / NB, i = e % NB;   // consecutive threads read along row j of R
    double v;
    if (i < nb && j < nb) v = (j <= i) ? R[(int64_t)j * ldr + i] : 0.0;
    else v = (i == j) ? 1.0 : 0.0;
    L[i][j] = v;
  }
  __shared__ double rd[NB];   // reciprocal pivots: one division per row for the whole block
  const int64_t c0 = (int64_t)blockIdx.x * TC;
  const int64_t c = c0 + threadIdx.x;
  for (int i = 0; i < nb; ++i) T[i][threadIdx.x] = (c < ncols) ? B[(int64_t)i * ldb + c] : 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < NB; i += blockDim.x) rd[i] = 1.0 / L[i][i];
  __syncthreads();
  if (c >= ncols) return;
  // row i of the solution overwrites row i of the tile; the loop over i stays rolled (a
  // fully unrolled 64-step solve is thousands of instructions that every thread runs
  // once, and fetching them, not the arithmetic, then sets the pace)
#pragma unroll 1
  for (int i = 0; i < nb; ++i) {
    // four interleaved partial sums keep the dependent chain a quarter as long
    double a0 = T[i][threadIdx.x], a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int j = 0;
#pragma unroll 2
    for (; j + 3 < i; j += 4) {
      a0 -= L[i][j] * T[j][threadIdx.x];
      a1 -= L[i][j + 1] * T[j + 1][threadIdx.x];
      a2 -= L[i][j + 2] * T[j + 2][threadIdx.x];
      a3 -= L[i][j + 3] * T[j + 3][threadIdx.x];
    }
    for (; j < i; ++j) a0 -= L[i][j] * T[j][threadIdx.x];
    T[i][threadIdx.x] = ((a0 + a1) + (a2 + a3)) * rd[i];
  }
  for (int i = 0; i < nb; ++i) B[(int64_t)i * ldb + c] = T[i][threadIdx.x];
}

// max_i H[i][i] (all >= 0 for a Gram; NaN orders above +inf as bits), as bits
__global__ void diag_max_kernel(const double* H, int64_t n, int64_t ld, unsigned long long* out) {
  unsigned long long m = 0;
  CHOL_GRID_STRIDE(i, n) {
    const double v = fabs(H[i * ld + i]);
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_down_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// sum over the n x n H of (H - I)^2 (block partial sums added atomically; a
// check value, so the order of the additions does not matter)
__global__ void dev_identity_kernel(const double* H, int64_t n, double* out) {
  double acc = 0.0;
  CHOL_GRID_STRIDE(e, n * n) {
    const int64_t i = e / n, j = e % n;
    const double v = H[e] - (i == j ? 1.0 : 0.0);
    acc += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// zero the strict lower triangle of the n x n row-major H
__global__ void zero_lower_kernel(double* H, int64_t n) {
  CHOL_GRID_STRIDE(e, n * n) {
    if (e / n > e % n) H[e] = 0.0;
  }
}

__global__ void unit_diag_kernel(double* V, int64_t n) {
  CHOL_GRID_STRIDE(i, n) V[i * n + i] = 1.0;
}

// ---------------------------------------------------------------- Gram error probes

constexpr int kProbes = 4;

// X (n x kProbes, row-major): independent +-1 entries from a splitmix64 hash of
// (seed, index); E ||D x||^2 = ||D||_F^2 for such x and any matrix D.
__global__ void rademacher_kernel(double* X, int64_t n, uint64_t seed) {
  CHOL_GRID_STRIDE(e, n * kProbes) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(e + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    X[e] = (z >> 63) ? 1.0 : -1.0;
  }
}

// Y (rows x kProbes) = A (rows x cols, leading dimension lda) X (cols x kProbes):
// one warp per row of A, FP64.
__global__ void rows_times_probes_kernel(const double* A, int64_t rows, int64_t cols, int64_t lda, const double* X,
                                         double* Y) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < rows; i += nw) {
    double acc[kProbes] = {};
    const double* a = A + i * lda;
    for (int64_t j = lane; j < cols; j += 32) {
      const double v = a[j];
#pragma unroll
      for (int p = 0; p < kProbes; ++p) acc[p] = fma(v, X[j * kProbes + p], acc[p]);
    }
#pragma unroll
    for (int p = 0; p < kProbes; ++p) {
      double t = acc[p];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) Y[i * kProbes + p] = t;
    }
  }
}

// Y (cols x kProbes) += A^T X, A (rows x cols, lda), X (rows x kProbes): a thread per
// column of A over a chunk of rows, partial sums added atomically (Y zeroed first).
constexpr int kColChunk = 512;
__global__ void cols_times_probes_kernel(const double* A, int64_t rows, int64_t cols, int64_t lda, const double* X,
                                         double* Y) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= cols) return;
  const int64_t i0 = (int64_t)blockIdx.y * kColChunk, i1 = min(rows, i0 + kColChunk);
  double acc[kProbes] = {};
  for (int64_t i = i0; i < i1; ++i) {
    const double v = A[i * lda + j];
#pragma unroll
    for (int p = 0; p < kProbes; ++p) acc[p] = fma(v, X[i * kProbes + p], acc[p]);
  }
#pragma unroll
  for (int p = 0; p < kProbes; ++p) atomicAdd(&Y[j * kProbes + p], acc[p]);
}

// sum of (a - b)^2 over n values
__global__ void diff_sumsq_kernel(const double* a, const double* b, int64_t n, double* out) {
  double acc = 0.0;
  CHOL_GRID_STRIDE(e, n) {
    const double v = a[e] - b[e];
    acc += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

void rows_times_probes(const double* A, int64_t rows, int64_t cols, int64_t lda, const double* X, double* Y,
                       cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>(ceil_div(rows, 8), (int64_t)kNumSMs * 16);
  rows_times_probes_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(A, rows, cols, lda, X, Y);
  FTT_LAUNCH();
}

void cols_times_probes(const double* A, int64_t rows, int64_t cols, int64_t lda, const double* X, double* Y,
                       cudaStream_t s) {
  FTT_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * cols * kProbes, s));
  const int64_t gy = ceil_div(rows, kColChunk);
  if (gy > 65535) fail(FASTTT_ERANK, "Gram probe: too many rows");
  dim3 grid((unsigned)ceil_div(cols, 256), (unsigned)gy);
  cols_times_probes_kernel<<<grid, 256, 0, s>>>(A, rows, cols, lda, X, Y);
  FTT_LAUNCH();
}

// ---------------------------------------------------------------- recursive Cholesky / solve

int64_t split_point(int64_t n, int64_t leaf = kLeaf) { return std::max<int64_t>(leaf, (n / 2 / leaf) * leaf); }

template <int TC>
void leaf_launch(const double* R, int64_t ldr, int64_t n, double* B, int64_t ldb, int64_t ncols, cudaStream_t s) {
  const size_t smem = sizeof(double) * ((size_t)kSolveLeaf * (kSolveLeaf + 1) + (size_t)kSolveLeaf * (TC + 1));
  // the dynamic shared-memory opt-in, once per device (setting it again is harmless)
  static std::atomic<bool> attr[kMaxDevices];
  int dev = 0;
  FTT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices || !attr[dev].load()) {
    FTT_CUDA(cudaFuncSetAttribute(trsm_leaf_kernel<kSolveLeaf, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    if (dev >= 0 && dev < kMaxDevices) attr[dev].store(true);
  }
  trsm_leaf_kernel<kSolveLeaf, TC><<<(unsigned)ceil_div(ncols, TC), TC, smem, s>>>(R, ldr, (int)n, B, ldb, ncols);
  FTT_LAUNCH();
}

// R^T X = B in place: R (n x n upper, leading dimension ldr), B (n rows x ncols,
// row stride ldb).  The update of the lower half of B is a GEMM (FP32-level when mixed).
void trsm_rt(const double* R, int64_t ldr, int64_t n, double* B, int64_t ldb, int64_t ncols, bool mixed,
             cudaStream_t s) {
  if (n <= 0 || ncols <= 0) return;
  if (n <= kSolveLeaf) {
    // 128 columns (one per thread) per block when that still fills the SMs twice over,
    // else 32: the solve is a chain of kSolveLeaf steps per column, so parallelism is in
    // the columns
    if (ncols >= 2 * 152 * kTrsmCols) leaf_launch<kTrsmCols>(R, ldr, n, B, ldb, ncols, s);
    else leaf_launch<32>(R, ldr, n, B, ldb, ncols, s);
    return;
  }
  const int64_t h = split_point(n, kSolveLeaf);
  trsm_rt(R, ldr, h, B, ldb, ncols, mixed, s);
  // B2 -= R12^T X1, R12 = R[0:h, h:n]: (R12^T)(i, k) = R[k * ldr + h + i]
  gemm(mixed, n - h, ncols, h, -1.0, R + h, 1, ldr, B, ldb, 1, 1.0, B + h * ldb, ldb, 1, s);
  trsm_rt(R + h * ldr + h, ldr, n - h, B + h * ldb, ldb, ncols, mixed, s);
}

// H (n x n, leading dimension ld, upper triangle) <- R with H = R^T R; the strict
// lower triangle of the leaf blocks is zeroed, the rest of the lower triangle is
// left as it was.  *info (device) is set on a pivot at or below tiny.
void chol_rec(double* H, int64_t ld, int64_t n, double tiny, int* info, cudaStream_t s) {
  if (n <= kLeaf) {
    chol_leaf_kernel<<<1, 256, 0, s>>>(H, ld, (int)n, tiny, info);
    FTT_LAUNCH();
    return;
  }
  const int64_t h = split_point(n);
  chol_rec(H, ld, h, tiny, info, s);
  // R12 = R11^-T H12 (in place on H[0:h, h:n])
  trsm_rt(H, ld, h, H + h, ld, n - h, false, s);
  // H22 -= R12^T R12
  gemm_f64(n - h, n - h, h, -1.0, H + h, 1, ld, H + h, ld, 1, 1.0, H + h * ld + h, ld, 1, s);
  chol_rec(H + h * ld + h, ld, n - h, tiny, info, s);
}

double max_diag(const double* H, int64_t n, int64_t ld, cudaStream_t s) {
  DBuf<unsigned long long> m(1, s);
  FTT_CUDA(cudaMemsetAsync(m.get(), 0, sizeof(unsigned long long), s));
  diag_max_kernel<<<grid_for(n), 256, 0, s>>>(H, n, ld, m.get());
  FTT_LAUNCH();
  const unsigned long long b = read_scalar(m.get(), s);
  double v;
  memcpy(&v, &b, sizeof(v));
  return v;
}

}  // namespace

void identity_f64(double* V, int64_t n, cudaStream_t s) {
  FTT_CUDA(cudaMemsetAsync(V, 0, sizeof(double) * n * n, s));
  unit_diag_kernel<<<grid_for(n), 256, 0, s>>>(V, n);
  FTT_LAUNCH();
}

bool cholesky_upper(double* H, int64_t n, double tiny_rel, cudaStream_t s) {
  if (n <= 0) return true;
  const double dmax = max_diag(H, n, n, s);
  if (!(dmax > 0.0) || !std::isfinite(dmax)) return false;
  DBuf<int> info(1, s);
  FTT_CUDA(cudaMemsetAsync(info.get(), 0, sizeof(int), s));
  chol_rec(H, n, n, tiny_rel * dmax, info.get(), s);
  zero_lower_kernel<<<grid_for(n * n), 256, 0, s>>>(H, n);
  FTT_LAUNCH();
  return read_scalar(info.get(), s) == 0;
}

void trsm_upper_t(const double* R, int64_t n, double* B, int64_t ldb, int64_t ncols, bool mixed, cudaStream_t s) {
  trsm_rt(R, n, n, B, ldb, ncols, mixed, s);
}

double identity_deviation(const double* H, int64_t n, cudaStream_t s) {
  DBuf<double> acc(1, s);
  FTT_CUDA(cudaMemsetAsync(acc.get(), 0, sizeof(double), s));
  dev_identity_kernel<<<grid_for(n * n), 256, 0, s>>>(H, n, acc.get());
  FTT_LAUNCH();
  return std::sqrt(read_scalar(acc.get(), s));
}

bool cholqr2_rows(double* Z, int64_t M, int64_t N, double* R, bool mixed, cudaStream_t s, double* dev_out) {
  if (M <= 0) return true;
  if (M > N) fail(FASTTT_EINVAL, "CholeskyQR2: more rows than columns");
  // breakdown threshold for the pivots, relative to max_i H_ii: the Gram's rounding
  // level times its order
  const double u = mixed ? 0x1p-23 : 0x1p-52;
  const double tiny_rel = 4.0 * (double)M * u;
  DBuf<double> H1((size_t)M * M, s);
  // pass 1: H1 = Z Z^T = R1^T R1, Z <- R1^-T Z
  gemm(mixed, M, M, N, 1.0, Z, N, 1, Z, 1, N, 0.0, H1.get(), M, 1, s, true);
  if (!R) {
    // Z's rows already nearly orthonormal (a re-orthonormalisation): R1 is within 0.1 of
    // I, so one pass leaves Q orthonormal to the Gram's rounding level, and R1^-T is
    // applied as one GEMM (its condition number is below 1.2)
    const double dev1 = identity_deviation(H1.get(), M, s);
    if (dev1 <= 0.1) {
      if (dev_out) *dev_out = dev1;
      if (!cholesky_upper(H1.get(), M, tiny_rel, s)) return false;
      DBuf<double> X((size_t)M * M, s), Z0((size_t)M * N, s);
      identity_f64(X.get(), M, s);
      trsm_upper_t(H1.get(), M, X.get(), M, M, false, s);   // X = R1^-T
      FTT_CUDA(cudaMemcpyAsync(Z0.get(), Z, sizeof(double) * M * N, cudaMemcpyDeviceToDevice, s));
      gemm(mixed, M, N, M, 1.0, X.get(), M, 1, Z0.get(), N, 1, 0.0, Z, N, 1, s);
      return true;
    }
  }
  if (!cholesky_upper(H1.get(), M, tiny_rel, s)) return false;
  trsm_upper_t(H1.get(), M, Z, N, N, mixed, s);
  // pass 2 on a matrix that is now well conditioned
  DBuf<double> H2((size_t)M * M, s);
  gemm(mixed, M, M, N, 1.0, Z, N, 1, Z, 1, N, 0.0, H2.get(), M, 1, s, true);
  const double dev = identity_deviation(H2.get(), M, s);
  if (dev_out) *dev_out = dev;
  if (!(dev <= 0.5)) return false;
  if (!cholesky_upper(H2.get(), M, tiny_rel, s)) return false;
  trsm_upper_t(H2.get(), M, Z, N, N, mixed, s);
  // R = R2 R1 (FP64-level product of the two triangular factors)
  if (R) gemm_f64(M, M, M, 1.0, H2.get(), M, 1, H1.get(), M, 1, 0.0, R, M, 1, s);
  return true;
}

bool orthonormalise_cols_cholqr2(double* U, int64_t rows, int64_t r, bool mixed, cudaStream_t s) {
  if (r <= 0) return true;
  if (r > rows) return false;
  DBuf<double> Ut((size_t)rows * r, s);
  transpose_f64(U, rows, r, Ut.get(), s);
  if (!cholqr2_rows(Ut.get(), r, rows, nullptr, mixed, s, nullptr)) return false;
  transpose_f64(Ut.get(), r, rows, U, s);
  return true;
}

double gram_error_probe(const double* Z, int64_t M, int64_t N, const double* G, cudaStream_t s) {
  const bool tall = (M >= N);
  const int64_t n = tall ? N : M;
  DBuf<double> X((size_t)n * kProbes, s), Y1((size_t)n * kProbes, s), Y2((size_t)n * kProbes, s),
      T((size_t)(tall ? M : N) * kProbes, s), acc(1, s);
  rademacher_kernel<<<grid_for(n * kProbes), 256, 0, s>>>(X.get(), n, 0x5eed0f9a7e11ull);
  FTT_LAUNCH();
  rows_times_probes(G, n, n, n, X.get(), Y1.get(), s);             // G~ x
  if (tall) {                                                        // Z^T (Z x)
    rows_times_probes(Z, M, N, N, X.get(), T.get(), s);
    cols_times_probes(Z, M, N, N, T.get(), Y2.get(), s);
  } else {                                                           // Z (Z^T x)
    cols_times_probes(Z, M, N, N, X.get(), T.get(), s);
    rows_times_probes(Z, M, N, N, T.get(), Y2.get(), s);
  }
  FTT_CUDA(cudaMemsetAsync(acc.get(), 0, sizeof(double), s));
  diff_sumsq_kernel<<<grid_for(n * kProbes), 256, 0, s>>>(Y1.get(), Y2.get(), n * kProbes, acc.get());
  FTT_LAUNCH();
  return std::sqrt(read_scalar(acc.get(), s) / (double)kProbes);
}

}  // namespace fasttt
