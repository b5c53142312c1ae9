// Tall-skinny SVDs of the rounding sweeps (S7-S10 direct route) by QR first:
// A (lg x n, column-major, lg >> n) = Q R by Householder TSQR, one-sided Jacobi
// on the n x n R (R V = U_R Sigma), and A V = Q (R V) written back over A.  The
// caller then reads U Sigma off A's columns and V as before, so the result is
// the one-sided Jacobi SVD of A with the long dimension handled by QR
// (backward stable: the singular values carry an absolute error of a few u ||A||,
// like LAPACK's bidiagonal route).
//
// TSQR (Demmel, Grigori, Hoemmen & Langou, SIAM J. Sci. Comput. 34, 2012): the
// rows are cut into blocks of BR rows (256 for n <= 64, 224 for n <= 128, so that
// a block fits in shared memory); each block is factored by Householder QR in
// shared memory (reflectors kept in place of the block, R written to the next
// level's input, the R factors of all blocks stacked); levels repeat until the
// stacked R factors have at most 4n rows (or one block remains), and Jacobi runs
// on that stack.  Q is applied back level by level from the top.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "dense.cuh"

namespace fasttt {

namespace {

constexpr int kQrThreads = 256;
// block rows for n columns: BR x n doubles (and BR x (n+1) for the apply) within
// the 227 KB of shared memory a block may have
constexpr int kQrRowsNarrow = 256;   // n <= 64
constexpr int kQrRowsWide = 224;     // 64 < n <= 128

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Householder QR of row block b of X (rows x n, column-major with leading
// dimension ld): block rows [b BR, ...), zero padded to BR.  The
// reflector of column j (v_j = 1 implied, v_i for i > j) replaces the block's
// column j below the diagonal; tau[b n + j]; R (n x n, zeros below the diagonal)
// goes to rows [b n, b n + n) of Rn (column-major, leading dimension ldr).
template <int BR>
__global__ void __launch_bounds__(kQrThreads) qr_blocks_kernel(double* X, int64_t rows, int64_t ld, int n,
                                                               double* tau, double* Rn, int64_t ldr) {
  extern __shared__ double sm[];   // BR x n, column-major
  __shared__ double wv[kMaxTsqrCols];
  __shared__ double red[kQrThreads / 32];
  __shared__ double coef[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = blockIdx.x, r0 = b * BR;
  const int nr = (rows - r0 < BR) ? (int)(rows - r0) : BR;
  for (int e = threadIdx.x; e < BR * n; e += kQrThreads) {
    const int i = e % BR, j = e / BR;
    sm[e] = (i < nr) ? X[(r0 + i) + (int64_t)j * ld] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    double* cj = sm + j * BR;
    double s = 0.0;
    for (int i = j + 1 + threadIdx.x; i < BR; i += kQrThreads) s = fma(cj[i], cj[i], s);
    s = warp_sum(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < kQrThreads / 32; ++w) tot += red[w];
      const double alpha = cj[j];
      double beta = alpha, tk = 0.0, scale = 0.0;
      if (tot > 0.0) {
        beta = -copysign(sqrt(fma(alpha, alpha, tot)), alpha);
        tk = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      coef[0] = tk;
      coef[1] = scale;
      cj[j] = beta;   // R_jj
      tau[b * n + j] = tk;
    }
    __syncthreads();
    const double tk = coef[0], scale = coef[1];
    for (int i = j + 1 + threadIdx.x; i < BR; i += kQrThreads) cj[i] *= scale;   // v below the diagonal
    __syncthreads();
    if (tk != 0.0) {
      // w_c = v . a_c over rows j.., one warp per column c > j
      for (int c = j + 1 + warp; c < n; c += kQrThreads / 32) {
        const double* ac = sm + c * BR;
        double acc = 0.0;
        for (int i = j + 1 + lane; i < BR; i += 32) acc = fma(cj[i], ac[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) wv[c] = tk * (ac[j] + acc);
      }
      __syncthreads();
      const int cols = n - j - 1, len = BR - j;
      for (int e = threadIdx.x; e < cols * len; e += kQrThreads) {
        const int c = j + 1 + e / len, i = j + e % len;
        const double vi = (i == j) ? 1.0 : cj[i];
        sm[c * BR + i] -= vi * wv[c];
      }
      __syncthreads();
    }
  }
  // reflectors back over the block, R to the next level
  for (int e = threadIdx.x; e < BR * n; e += kQrThreads) {
    const int i = e % BR, j = e / BR;
    if (i > j && i < nr) X[(r0 + i) + (int64_t)j * ld] = sm[e];
  }
  for (int e = threadIdx.x; e < n * n; e += kQrThreads) {
    const int i = e % n, j = e / n;
    Rn[(b * n + i) + (int64_t)j * ldr] = (i <= j) ? sm[j * BR + i] : 0.0;
  }
}

// Yout rows of block b (column-major, ldo) = Q_b [Yin rows (b n .. b n + n - 1); 0]
// with Q_b = H_0 ... H_{n-1} of block b of the level (reflectors in X as left by
// qr_blocks_kernel).  Only the block's real rows are written.
template <int BR>
__global__ void __launch_bounds__(kQrThreads) qr_apply_kernel(const double* X, int64_t rows, int64_t ld, int n,
                                                              const double* tau, const double* Yin, int64_t ldi,
                                                              double* Yout, int64_t ldo) {
  extern __shared__ double sm[];   // BR x n target, then the reflector column
  double* v = sm + BR * n;
  __shared__ double wv[kMaxTsqrCols];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = blockIdx.x, r0 = b * BR;
  const int nr = (rows - r0 < BR) ? (int)(rows - r0) : BR;
  for (int e = threadIdx.x; e < BR * n; e += kQrThreads) {
    const int i = e % BR, c = e / BR;
    sm[e] = (i < n) ? Yin[(b * n + i) + (int64_t)c * ldi] : 0.0;
  }
  for (int j = n - 1; j >= 0; --j) {
    const double tk = tau[b * n + j];
    __syncthreads();
    if (tk == 0.0) continue;
    for (int i = threadIdx.x; i < BR; i += kQrThreads)
      v[i] = (i < j) ? 0.0 : (i == j) ? 1.0 : (i < nr ? X[(r0 + i) + (int64_t)j * ld] : 0.0);
    __syncthreads();
    for (int c = warp; c < n; c += kQrThreads / 32) {
      const double* ac = sm + c * BR;
      double acc = 0.0;
      for (int i = j + lane; i < BR; i += 32) acc = fma(v[i], ac[i], acc);
      acc = warp_sum(acc);
      if (lane == 0) wv[c] = tk * acc;
    }
    __syncthreads();
    const int len = BR - j;
    for (int e = threadIdx.x; e < n * len; e += kQrThreads) {
      const int c = e / len, i = j + e % len;
      sm[c * BR + i] -= v[i] * wv[c];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < BR * n; e += kQrThreads) {
    const int i = e % BR, c = e / BR;
    if (i < nr) Yout[(r0 + i) + (int64_t)c * ldo] = sm[e];
  }
}

}  // namespace

bool tsqr_applies(int64_t lg, int n) { return n >= 2 && n <= kMaxTsqrCols && lg >= 1024; }

namespace {

template <int BR>
int64_t tsqr_jacobi_br(double* A, int64_t lg, int n, double* V, int64_t max_sweeps, cudaStream_t s) {
  const size_t smem_qr = sizeof(double) * (size_t)BR * n;
  const size_t smem_ap = sizeof(double) * (size_t)BR * (n + 1);
  // set on every call (the limit belongs to the current device's context), always to the
  // instantiation's largest need, so that concurrent callers never lower it for each other
  const int ncap = (BR == kQrRowsNarrow) ? 64 : kMaxTsqrCols;
  FTT_CUDA(cudaFuncSetAttribute(qr_blocks_kernel<BR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * (size_t)BR * ncap)));
  FTT_CUDA(cudaFuncSetAttribute(qr_apply_kernel<BR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * (size_t)BR * (ncap + 1))));
  // level l: input X_l (rows_l x n, leading dimension ld_l); level 0 is A itself.  The
  // tree stops once the stacked R factors have at most 4n rows (or one block remained).
  std::vector<double*> X{A};
  std::vector<int64_t> rows{lg}, ld{lg};
  std::vector<DBuf<double>> owned, taus;
  KClock clk;
  kclock_begin(clk, KC_TSQR, s);
  while (true) {
    const int64_t nb = ceil_div(rows.back(), BR);
    taus.emplace_back((size_t)nb * n, s);
    const int64_t next_rows = nb * n;
    owned.emplace_back((size_t)next_rows * n, s);
    qr_blocks_kernel<BR><<<(unsigned)nb, kQrThreads, smem_qr, s>>>(X.back(), rows.back(), ld.back(), n,
                                                                   taus.back().get(), owned.back().get(), next_rows);
    FTT_LAUNCH();
    X.push_back(owned.back().get());
    rows.push_back(next_rows);
    ld.push_back(next_rows);
    if (nb == 1 || next_rows <= 4 * (int64_t)n) break;
  }
  kclock_end(clk, 4.0 * (double)lg * n * n, s);
  // the stacked R factors (rows.back() x n, column-major) <- R V by one-sided Jacobi
  const int64_t sweeps = jacobi_svd_f64(X.back(), rows.back(), ld.back(), n, V, n, n, max_sweeps, s);
  // A V = Q (R V): apply the levels from the top
  KClock clk2;
  kclock_begin(clk2, KC_TSQR, s);
  for (int l = (int)taus.size() - 1; l >= 0; --l) {
    const int64_t nb = ceil_div(rows[l], BR);
    double* out = X[l];   // the block's reflectors are read before its rows are overwritten
    qr_apply_kernel<BR><<<(unsigned)nb, kQrThreads, smem_ap, s>>>(X[l], rows[l], ld[l], n, taus[l].get(), X[l + 1],
                                                                  ld[l + 1], out, ld[l]);
    FTT_LAUNCH();
  }
  kclock_end(clk2, 4.0 * (double)lg * n * n, s);
  return sweeps;
}

}  // namespace

int64_t tsqr_jacobi(double* A, int64_t lg, int n, double* V, int64_t max_sweeps, cudaStream_t s) {
  if (!tsqr_applies(lg, n)) fail(FASTTT_EINVAL, "tsqr_jacobi: shape outside the TSQR route");
  return n <= 64 ? tsqr_jacobi_br<kQrRowsNarrow>(A, lg, n, V, max_sweeps, s)
                 : tsqr_jacobi_br<kQrRowsWide>(A, lg, n, V, max_sweeps, s);
}

}  // namespace fasttt
