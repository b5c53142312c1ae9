// Dense FP64 kernels of the TT-rounding stage: a tiled DFMA GEMM with
// arbitrary element strides, a transpose, and a truncated SVD built on the
// one-sided (Hestenes) Jacobi method.
//
// The SVD of a row-major M x N matrix Z takes one of two routes:
//  * direct: one-sided Jacobi on the columns of the tall orientation of Z
//    (Z itself if M >= N, else Z^T).  Rotations are applied to Z, so singular
//    values are accurate to a few units of roundoff times sigma_1 (LAPACK-grade);
//    used while min(M, N) <= kDirectMax.
//  * Gram: G = Z^T Z (or Z Z^T) by GEMM, then one-sided Jacobi on the symmetric
//    positive semi-definite G gives its eigenpairs, sigma = sqrt(lambda), and the
//    other singular vectors by one GEMM.  Singular values below about
//    sqrt(2^-52) sigma_1 are not resolved on this route.
// Jacobi pairs columns by the round-robin (circle) schedule: n/2 disjoint pairs
// per round, n-1 rounds per sweep, one thread block per pair; sweeps repeat until
// a whole sweep rotates no pair, or the sweep bound is hit (ETIMEOUT).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>

#include "dense.cuh"

namespace fasttt {

namespace {

#define GRID_STRIDE(i, n)                                                            \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

constexpr int kTile = 64;
constexpr int kTileK = 16;
constexpr int kDirectMax = 512;

__global__ void __launch_bounds__(256)
    gemm_f64_kernel(int64_t M, int64_t N, int64_t K, double alpha, const double* __restrict__ A, int64_t sai,
                    int64_t sak, const double* __restrict__ B, int64_t sbk, int64_t sbj, double beta,
                    double* __restrict__ C, int64_t sci, int64_t scj) {
  __shared__ double As[kTileK][kTile + 1];
  __shared__ double Bs[kTileK][kTile + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * kTile, j0 = (int64_t)blockIdx.y * kTile;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  const bool a_k_fast = (sak == 1);
  const bool b_k_fast = (sbk == 1);
  for (int64_t k0 = 0; k0 < K; k0 += kTileK) {
    for (int e = threadIdx.x; e < kTile * kTileK; e += 256) {
      int kk, ii;
      if (a_k_fast) { kk = e & 15; ii = e >> 4; } else { kk = e >> 6; ii = e & 63; }
      const int64_t gi = i0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < M && gk < K) ? A[gi * sai + gk * sak] : 0.0;
      int kb, jj;
      if (b_k_fast) { kb = e & 15; jj = e >> 4; } else { kb = e >> 6; jj = e & 63; }
      const int64_t gj = j0 + jj, gkb = k0 + kb;
      Bs[kb][jj] = (gkb < K && gj < N) ? B[gkb * sbk + gj * sbj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTileK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t gi = i0 + ty + 16 * r;
    if (gi >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t gj = j0 + tx + 16 * c;
      if (gj >= N) continue;
      double* cp = C + gi * sci + gj * scj;
      *cp = (beta == 0.0) ? alpha * acc[r][c] : fma(beta, *cp, alpha * acc[r][c]);
    }
  }
}

__global__ void transpose_kernel(const double* __restrict__ src, int64_t rows, int64_t cols,
                                 double* __restrict__ dst) {
  __shared__ double t[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int64_t r = r0 + j, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[j][threadIdx.x] = src[r * cols + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int64_t c = c0 + j, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[c * rows + r] = t[threadIdx.x][j];
  }
}

__global__ void identity_kernel(double* V, int64_t n) {
  GRID_STRIDE(i, n * n) V[i] = ((i / n) == (i % n)) ? 1.0 : 0.0;
}

// Block-wide sum of three values (256 threads).
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double red[3][8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red[0][warp] = a; red[1][warp] = b; red[2][warp] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0, y = 0, z = 0;
    for (int w = 0; w < 8; ++w) { x += red[0][w]; y += red[1][w]; z += red[2][w]; }
    red[0][0] = x; red[1][0] = y; red[2][0] = z;
  }
  __syncthreads();
  a = red[0][0]; b = red[1][0]; c = red[2][0];
}

// One round of the circle schedule: block i rotates pair i.
__global__ void __launch_bounds__(256) jacobi_round_kernel(double* A, int64_t m, int64_t lda, double* V,
                                                           int64_t nv, int64_t ldv, int n, int n2, int round,
                                                           double tol, double small2, unsigned* rotations) {
  const int i = blockIdx.x;
  int p, q;
  if (i == 0) { p = round; q = n2 - 1; }
  else { p = (round + i) % (n2 - 1); q = (round - i + (n2 - 1)) % (n2 - 1); }
  if (p > q) { const int t = p; p = q; q = t; }
  if (q >= n) return;  // the dummy player of an odd n
  double* ap = A + (int64_t)p * lda;
  double* aq = A + (int64_t)q * lda;
  double alpha = 0.0, beta = 0.0, gamma = 0.0;
  for (int64_t e = threadIdx.x; e < m; e += blockDim.x) {
    const double x = ap[e], y = aq[e];
    alpha = fma(x, x, alpha);
    beta = fma(y, y, beta);
    gamma = fma(x, y, gamma);
  }
  block_sum3(alpha, beta, gamma);
  // columns at roundoff level relative to ||A||_F are treated as zero
  if (gamma == 0.0 || alpha <= small2 || beta <= small2) return;
  if (fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) return;
  const double zeta = (beta - alpha) / (2.0 * gamma);
  const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
  const double c = 1.0 / sqrt(fma(t, t, 1.0));
  const double s = c * t;
  if (threadIdx.x == 0) atomicAdd(rotations, 1u);
  for (int64_t e = threadIdx.x; e < m; e += blockDim.x) {
    const double x = ap[e], y = aq[e];
    ap[e] = c * x - s * y;
    aq[e] = s * x + c * y;
  }
  if (V) {
    double* vp = V + (int64_t)p * ldv;
    double* vq = V + (int64_t)q * ldv;
    for (int64_t e = threadIdx.x; e < nv; e += blockDim.x) {
      const double x = vp[e], y = vq[e];
      vp[e] = c * x - s * y;
      vq[e] = s * x + c * y;
    }
  }
}

__global__ void col_norms_kernel(const double* A, int64_t m, int64_t lda, int n, double* out) {
  const int j = blockIdx.x;
  if (j >= n) return;
  const double* a = A + (int64_t)j * lda;
  double s = 0.0, d1 = 0.0, d2 = 0.0;
  for (int64_t e = threadIdx.x; e < m; e += blockDim.x) s = fma(a[e], a[e], s);
  block_sum3(s, d1, d2);
  if (threadIdx.x == 0) out[j] = sqrt(s);
}

// out (rows x r, row-major): out[i, c] = src[perm[c] * ld + i] * scale[c]
__global__ void gather_cols_kernel(const double* src, int64_t ld, int64_t rows, const int32_t* perm,
                                   const double* scale, int64_t r, double* out) {
  GRID_STRIDE(e, rows * r) {
    const int64_t i = e / r, c = e % r;
    out[e] = src[(int64_t)perm[c] * ld + i] * (scale ? scale[c] : 1.0);
  }
}

// out (r x cols, row-major): out[c, j] = src[perm[c] * ld + j] * scale[c]
__global__ void gather_rows_kernel(const double* src, int64_t ld, int64_t cols, const int32_t* perm,
                                   const double* scale, int64_t r, double* out) {
  GRID_STRIDE(e, r * cols) {
    const int64_t c = e / cols, j = e % cols;
    out[e] = src[(int64_t)perm[c] * ld + j] * (scale ? scale[c] : 1.0);
  }
}

// One-sided Jacobi on the n columns (length m) of A; V (nv x n) receives the
// same rotations.  Returns the number of sweeps.
int64_t jacobi(double* A, int64_t m, int64_t lda, int n, double* V, int64_t nv, int64_t ldv,
               int64_t max_sweeps, cudaStream_t s) {
  if (n < 2) return 0;
  const int n2 = n + (n & 1);
  const double tol = sqrt((double)m) * 0x1p-52;
  double small2;
  {
    DBuf<double> norms(n, s);
    col_norms_kernel<<<n, 256, 0, s>>>(A, m, lda, n, norms.get());
    FTT_LAUNCH();
    std::vector<double> h(n);
    FTT_CUDA(cudaMemcpyAsync(h.data(), norms.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    double f2 = 0.0;
    for (double x : h) f2 += x * x;
    small2 = f2 * 0x1p-100;  // (2^-50 ||A||_F)^2
  }
  DBuf<unsigned> rot(1, s);
  const double pairs = 0.5 * (double)n * (double)(n - 1);
  for (int64_t sweep = 1; sweep <= max_sweeps; ++sweep) {
    FTT_CUDA(cudaMemsetAsync(rot.get(), 0, sizeof(unsigned), s));
    KClock clk;
    kclock_begin(clk, KC_JACOBI, s);
    for (int round = 0; round < n2 - 1; ++round) {
      jacobi_round_kernel<<<n2 / 2, 256, 0, s>>>(A, m, lda, V, nv, ldv, n, n2, round, tol, small2, rot.get());
    }
    note_launches(n2 - 2);
    FTT_LAUNCH();
    const unsigned rots = read_scalar(rot.get(), s);
    // every pair: three dot products (6m flops); every rotation: 6m + 6nv flops
    kclock_end(clk, pairs * 6.0 * (double)m + (double)rots * 6.0 * (double)(m + (V ? nv : 0)), s);
    if (rots == 0) return sweep;
  }
  fail(FASTTT_ETIMEOUT, "Jacobi SVD did not converge within the sweep bound");
}

}  // namespace

void gemm_f64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
              const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
              cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  const int64_t gx = ceil_div(M, kTile), gy = ceil_div(N, kTile);
  if (gy > 65535) fail(FASTTT_ERANK, "GEMM: N too large");
  dim3 grid((unsigned)gx, (unsigned)gy);
  KClock clk;
  kclock_begin(clk, KC_GEMM, s);
  gemm_f64_kernel<<<grid, 256, 0, s>>>(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci, scj);
  FTT_LAUNCH();
  kclock_end(clk, 2.0 * (double)M * (double)N * (double)K, s);
}

void transpose_f64(const double* src, int64_t rows, int64_t cols, double* dst, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32));
  dim3 block(32, 8);
  transpose_kernel<<<grid, block, 0, s>>>(src, rows, cols, dst);
  FTT_LAUNCH();
}

void svd_truncated(const double* Z, int64_t M, int64_t N,
                   const std::function<int64_t(const std::vector<double>&)>& choose_rank, int64_t max_sweeps,
                   SvdOut& out, cudaStream_t s) {
  const bool tall = (M >= N);
  const int64_t sm = tall ? N : M;   // number of singular values
  const int64_t lg = tall ? M : N;
  if (sm > INT32_MAX / 2) fail(FASTTT_ERANK, "SVD too large");
  const int n = (int)sm;
  const bool direct = (sm <= kDirectMax);
  DBuf<double> A;      // column-major lg x n (direct) or n x n (Gram)
  int64_t m_len, lda;
  if (direct) {
    A = DBuf<double>((size_t)lg * n, s);
    if (tall) transpose_f64(Z, M, N, A.get(), s);  // columns of Z become contiguous
    else FTT_CUDA(cudaMemcpyAsync(A.get(), Z, sizeof(double) * M * N, cudaMemcpyDeviceToDevice, s));
    m_len = lg;
    lda = lg;
  } else {
    A = DBuf<double>((size_t)n * n, s);
    if (tall)  // G = Z^T Z
      gemm_f64(N, N, M, 1.0, Z, 1, N, Z, N, 1, 0.0, A.get(), N, 1, s);
    else       // G = Z Z^T
      gemm_f64(M, M, N, 1.0, Z, N, 1, Z, 1, N, 0.0, A.get(), M, 1, s);
    m_len = n;
    lda = n;
  }
  DBuf<double> V((size_t)n * n, s);
  identity_kernel<<<grid_for((int64_t)n * n), 256, 0, s>>>(V.get(), n);
  FTT_LAUNCH();
  out.sweeps = jacobi(A.get(), m_len, lda, n, V.get(), n, n, max_sweeps, s);
  DBuf<double> norms(n, s);
  col_norms_kernel<<<n, 256, 0, s>>>(A.get(), m_len, lda, n, norms.get());
  FTT_LAUNCH();
  std::vector<double> h(n);
  FTT_CUDA(cudaMemcpyAsync(h.data(), norms.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  if (!direct)
    for (auto& x : h) x = sqrt(x);  // eigenvalues of the Gram -> singular values
  for (double x : h)
    if (!std::isfinite(x)) fail(FASTTT_ENUMERIC, "non-finite singular value");
  std::vector<int32_t> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return h[a] > h[b]; });
  out.sigma_all.resize(n);
  for (int i = 0; i < n; ++i) out.sigma_all[i] = h[perm[i]];
  int64_t r = choose_rank(out.sigma_all);
  r = std::max<int64_t>(1, std::min<int64_t>(r, n));
  out.r = r;
  std::vector<double> sig(out.sigma_all.begin(), out.sigma_all.begin() + r), inv(r);
  for (int64_t i = 0; i < r; ++i) inv[i] = sig[i] > 0.0 ? 1.0 / sig[i] : 0.0;
  DBuf<int32_t> dperm(r, s);
  DBuf<double> dinv(r, s);
  out.sigma = DBuf<double>(r, s);
  FTT_CUDA(cudaMemcpyAsync(dperm.get(), perm.data(), sizeof(int32_t) * r, cudaMemcpyHostToDevice, s));
  FTT_CUDA(cudaMemcpyAsync(dinv.get(), inv.data(), sizeof(double) * r, cudaMemcpyHostToDevice, s));
  FTT_CUDA(cudaMemcpyAsync(out.sigma.get(), sig.data(), sizeof(double) * r, cudaMemcpyHostToDevice, s));
  out.U = DBuf<double>((size_t)M * r, s);
  out.Vt = DBuf<double>((size_t)r * N, s);
  if (direct) {
    if (tall) {  // Z V = A  ->  U = A Sigma^-1, Vt = V^T
      gather_cols_kernel<<<grid_for(M * r), 256, 0, s>>>(A.get(), lda, M, dperm.get(), dinv.get(), r, out.U.get());
      FTT_LAUNCH();
      gather_rows_kernel<<<grid_for(r * N), 256, 0, s>>>(V.get(), n, N, dperm.get(), nullptr, r, out.Vt.get());
    } else {     // Z^T V = A  ->  Z = V Sigma (A Sigma^-1)^T
      gather_cols_kernel<<<grid_for(M * r), 256, 0, s>>>(V.get(), n, M, dperm.get(), nullptr, r, out.U.get());
      FTT_LAUNCH();
      gather_rows_kernel<<<grid_for(r * N), 256, 0, s>>>(A.get(), lda, N, dperm.get(), dinv.get(), r, out.Vt.get());
    }
    FTT_LAUNCH();
  } else if (tall) {  // V: right vectors; U = Z V_r Sigma^-1
    DBuf<double> Vs((size_t)N * r, s);
    gather_cols_kernel<<<grid_for(N * r), 256, 0, s>>>(V.get(), n, N, dperm.get(), dinv.get(), r, Vs.get());
    FTT_LAUNCH();
    gather_rows_kernel<<<grid_for(r * N), 256, 0, s>>>(V.get(), n, N, dperm.get(), nullptr, r, out.Vt.get());
    FTT_LAUNCH();
    gemm_f64(M, r, N, 1.0, Z, N, 1, Vs.get(), r, 1, 0.0, out.U.get(), r, 1, s);
  } else {            // V: left vectors; Vt = Sigma^-1 U_r^T Z
    gather_cols_kernel<<<grid_for(M * r), 256, 0, s>>>(V.get(), n, M, dperm.get(), nullptr, r, out.U.get());
    FTT_LAUNCH();
    DBuf<double> Us((size_t)M * r, s);
    gather_cols_kernel<<<grid_for(M * r), 256, 0, s>>>(V.get(), n, M, dperm.get(), dinv.get(), r, Us.get());
    FTT_LAUNCH();
    gemm_f64(r, N, M, 1.0, Us.get(), 1, r, Z, N, 1, 0.0, out.Vt.get(), N, 1, s);
  }
}

}  // namespace fasttt
