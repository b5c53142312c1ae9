// Dense FP64 kernels of the TT-rounding stage: a tiled DFMA GEMM with
// arbitrary element strides, a transpose, the one-sided (Hestenes) Jacobi SVD and
// the truncated SVD built on it and on the Gram eigensolvers.
//
// The SVD of a row-major M x N matrix Z takes one of two routes:
//  * direct: one-sided Jacobi on the columns of the tall orientation of Z
//    (Z itself if M >= N, else Z^T); tall-skinny shapes are first reduced to a
//    small R by Householder TSQR (tsqr.cu) or CholeskyQR2 (chol.cu) and Jacobi
//    runs on R.  Rotations are applied to the matrix, so singular values are
//    accurate to a few units of roundoff times sigma_1 (LAPACK-grade); used while
//    min(M, N) <= kDirectMax, or where a sweep is cheap.
//  * Gram: G = Z^T Z (or Z Z^T) by GEMM, its eigenpairs from gram_eig (the FP32
//    tridiagonal start refined with Ogita-Aishima steps on the slice GEMM, else the
//    FP64 tridiagonal route of tridiag.cu, else an iterative Jacobi solver),
//    sigma = sqrt(lambda), and the other singular vectors by one GEMM.  Singular
//    values below about sqrt(2^-52) sigma_1 are not resolved on this route.
// Jacobi pairs columns by the round-robin (circle) schedule: n/2 disjoint pairs
// per round, n-1 rounds per sweep, one warp (columns up to kWarpPairMax) or one
// thread block per pair; sweeps repeat until a whole sweep rotates no pair, or
// the sweep bound is hit (ETIMEOUT).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <numeric>

#include "dense.cuh"
#include "devsync.cuh"

namespace fasttt {

namespace {

#define GRID_STRIDE(i, n)                                                            \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

constexpr int kTile = 64;
constexpr int kTileK = 16;
constexpr int kDirectMax = 512;
constexpr int kOrthoLeft = 1, kOrthoRight = 2;

__global__ void __launch_bounds__(256)
    gemm_f64_kernel(int64_t M, int64_t N, int64_t K, double alpha, const double* __restrict__ A, int64_t sai,
                    int64_t sak, const double* __restrict__ B, int64_t sbk, int64_t sbj, double beta,
                    double* __restrict__ C, int64_t sci, int64_t scj, bool sym) {
  // sym: C is symmetric; tiles strictly below the diagonal are skipped (mirrored later)
  if (sym && (int64_t)blockIdx.x * kTile >= ((int64_t)blockIdx.y + 1) * kTile) return;
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
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  // row tiles stride by gridDim.y (at most 65535 of them per launch)
  for (int64_t r0 = (int64_t)blockIdx.y * 32; r0 < rows; r0 += (int64_t)gridDim.y * 32) {
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
      const int64_t r = r0 + j, c = c0 + threadIdx.x;
      if (r < rows && c < cols) t[j][threadIdx.x] = src[r * cols + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
      const int64_t c = c0 + j, r = r0 + threadIdx.x;
      if (r < rows && c < cols) dst[c * rows + r] = t[threadIdx.x][j];
    }
    __syncthreads();
  }
}

__global__ void identity_kernel(double* V, int64_t n) {
  GRID_STRIDE(i, n * n) V[i] = ((i / n) == (i % n)) ? 1.0 : 0.0;
}


template <bool kCoherent, typename T>
__device__ __forceinline__ T ld(const T* p) {
  if constexpr (kCoherent) return __ldcg(p);  // bypass L1: other blocks wrote it this launch
  else return *p;
}

// Rotate pair i of round `round` of the circle schedule (whole block).
template <bool kCoherent, typename T>
__device__ __forceinline__ void jacobi_pair(T* A, int64_t m, int64_t lda, T* V, int64_t nv, int64_t ldv, int n,
                                            int n2, int round, int i, T tol, T small2, unsigned* rotations) {
  int p, q;
  if (i == 0) { p = round; q = n2 - 1; }
  else { p = (round + i) % (n2 - 1); q = (round - i + (n2 - 1)) % (n2 - 1); }
  if (p > q) { const int t = p; p = q; q = t; }
  if (q >= n) return;  // the dummy player of an odd n
  T* ap = A + (int64_t)p * lda;
  T* aq = A + (int64_t)q * lda;
  T alpha = 0, beta = 0, gamma = 0;
  for (int64_t e = threadIdx.x; e < m; e += blockDim.x) {
    const T x = ld<kCoherent>(ap + e), y = ld<kCoherent>(aq + e);
    alpha = fma(x, x, alpha);
    beta = fma(y, y, beta);
    gamma = fma(x, y, gamma);
  }
  block_sum3<T>(alpha, beta, gamma);
  // columns at roundoff level relative to ||A||_F are treated as zero
  if (gamma == T(0) || alpha <= small2 || beta <= small2) return;
  if (fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) return;
  const T zeta = (beta - alpha) / (T(2) * gamma);
  const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, T(1))));
  const T c = T(1) / sqrt(fma(t, t, T(1)));
  const T sn = c * t;
  if (threadIdx.x == 0) atomicAdd(rotations, 1u);
  for (int64_t e = threadIdx.x; e < m; e += blockDim.x) {
    const T x = ld<kCoherent>(ap + e), y = ld<kCoherent>(aq + e);
    ap[e] = c * x - sn * y;
    aq[e] = sn * x + c * y;
  }
  if (V) {
    T* vp = V + (int64_t)p * ldv;
    T* vq = V + (int64_t)q * ldv;
    for (int64_t e = threadIdx.x; e < nv; e += blockDim.x) {
      const T x = ld<kCoherent>(vp + e), y = ld<kCoherent>(vq + e);
      vp[e] = c * x - sn * y;
      vq[e] = sn * x + c * y;
    }
  }
}

// One round of the circle schedule per launch: block i rotates pair i.
template <typename T>
__global__ void __launch_bounds__(256) jacobi_round_kernel(T* A, int64_t m, int64_t lda, T* V, int64_t nv,
                                                           int64_t ldv, int n, int n2, int round, T tol, T small2,
                                                           unsigned* rotations) {
  jacobi_pair<false, T>(A, m, lda, V, nv, ldv, n, n2, round, blockIdx.x, tol, small2, rotations);
}

constexpr int64_t kWarpPairMax = 16384;

// (a, b) <- (c a - s b, s a + c b) over n elements, U loads per lane in flight
template <typename T, int U>
__device__ __forceinline__ void rotate_cols_warp(T* a, T* b, int64_t n, T c, T sn, int lane) {
  for (int64_t e0 = 0; e0 < n; e0 += 32 * U) {
    T x[U], y[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = e0 + u * 32 + lane;
      x[u] = (e < n) ? __ldcg(a + e) : T(0);
      y[u] = (e < n) ? __ldcg(b + e) : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = e0 + u * 32 + lane;
      if (e < n) {
        a[e] = c * x[u] - sn * y[u];
        b[e] = sn * x[u] + c * y[u];
      }
    }
  }
}

// Rotate pair i of round `round` with one warp (lane-strided columns, shuffle
// reductions, all lanes hold the sums).  Loads bypass L1: the columns were
// written by other warps earlier in the same launch.
template <typename T>
__device__ __forceinline__ void jacobi_pair_warp(T* A, int64_t m, int64_t lda, T* V, int64_t nv, int64_t ldv,
                                                 int n, int n2, int round, int i, T tol, T small2,
                                                 unsigned* rotations, int lane) {
  int p, q;
  if (i == 0) { p = round; q = n2 - 1; }
  else { p = (round + i) % (n2 - 1); q = (round - i + (n2 - 1)) % (n2 - 1); }
  if (p > q) { const int t = p; p = q; q = t; }
  if (q >= n) return;
  T* ap = A + (int64_t)p * lda;
  T* aq = A + (int64_t)q * lda;
  T alpha = 0, beta = 0, gamma = 0;
  // 8 independent loads per lane in flight per step (the column lives in L2)
  constexpr int U = 8;
  for (int64_t e0 = 0; e0 < m; e0 += 32 * U) {
    T x[U], y[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = e0 + u * 32 + lane;
      x[u] = (e < m) ? __ldcg(ap + e) : T(0);
      y[u] = (e < m) ? __ldcg(aq + e) : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      alpha = fma(x[u], x[u], alpha);
      beta = fma(y[u], y[u], beta);
      gamma = fma(x[u], y[u], gamma);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    alpha += __shfl_xor_sync(0xffffffffu, alpha, o);
    beta += __shfl_xor_sync(0xffffffffu, beta, o);
    gamma += __shfl_xor_sync(0xffffffffu, gamma, o);
  }
  if (gamma == T(0) || alpha <= small2 || beta <= small2) return;
  if (fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) return;
  const T zeta = (beta - alpha) / (T(2) * gamma);
  const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, T(1))));
  const T c = T(1) / sqrt(fma(t, t, T(1)));
  const T sn = c * t;
  if (lane == 0) atomicAdd(rotations, 1u);
  rotate_cols_warp<T, U>(ap, aq, m, c, sn, lane);
  if (V) rotate_cols_warp<T, U>(V + (int64_t)p * ldv, V + (int64_t)q * ldv, nv, c, sn, lane);
}

// Block one-sided Jacobi: one sweep in one cooperative launch.  The columns are
// cut into blocks of b; blocks meet by the circle schedule; a CTA owns a block
// pair: it stages the 2b columns of A in shared memory (16-byte cp.async through
// L2), runs one local sweep over all their pairs (wpp warps per pair), keeps
// the local rotations in Q (2b x 2b), writes the columns back and multiplies
// V's 2b columns by Q (4 x 4 register tiles over double-buffered chunks of V).
// A block pair that rotated nothing skips the write-back and the V product.
// Every pair of columns meets once per sweep, so a sweep without rotations
// means convergence, as for the point schedule; rounds drop from n-1 to n/b-1.
constexpr int kBlockJacobiMaxW = 32;   // 2b at most
constexpr int kBlockJacobiMaxWpp = 4;  // warps per local pair at most

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ void dot3(const float4& x, const float4& y, float& a, float& b, float& g) {
  a = fmaf(x.x, x.x, a); a = fmaf(x.y, x.y, a); a = fmaf(x.z, x.z, a); a = fmaf(x.w, x.w, a);
  b = fmaf(y.x, y.x, b); b = fmaf(y.y, y.y, b); b = fmaf(y.z, y.z, b); b = fmaf(y.w, y.w, b);
  g = fmaf(x.x, y.x, g); g = fmaf(x.y, y.y, g); g = fmaf(x.z, y.z, g); g = fmaf(x.w, y.w, g);
}
__device__ __forceinline__ void dot3(const double2& x, const double2& y, double& a, double& b, double& g) {
  a = fma(x.x, x.x, a); a = fma(x.y, x.y, a);
  b = fma(y.x, y.x, b); b = fma(y.y, y.y, b);
  g = fma(x.x, y.x, g); g = fma(x.y, y.y, g);
}
__device__ __forceinline__ void rot2(float4& x, float4& y, float c, float s) {
  const float4 u = x, v = y;
  x = make_float4(c * u.x - s * v.x, c * u.y - s * v.y, c * u.z - s * v.z, c * u.w - s * v.w);
  y = make_float4(s * u.x + c * v.x, s * u.y + c * v.y, s * u.z + c * v.z, s * u.w + c * v.w);
}
__device__ __forceinline__ void rot2(double2& x, double2& y, double c, double s) {
  const double2 u = x, v = y;
  x = make_double2(c * u.x - s * v.x, c * u.y - s * v.y);
  y = make_double2(s * u.x + c * v.x, s * u.y + c * v.y);
}
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  const double2 t0 = reinterpret_cast<const double2*>(p)[0], t1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// dst[0, len) <- src[0, len), read through L2 (another CTA may have written src
// since this SM last read it): 16-byte cp.async when vec (both ends 16-byte
// aligned), else loads through registers.  Completion: cp_async_commit + wait.
template <typename T>
__device__ __forceinline__ void stage_async(T* __restrict__ dst, const T* __restrict__ src, int len, bool vec) {
  constexpr int W = Vec16<T>::n;
  int done = 0;
  if (vec) {
    const int nvec = len / W;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) cp_async16(dst + i * W, src + i * W);
    done = nvec * W;
  }
#pragma unroll 8
  for (int i = done + threadIdx.x; i < len; i += blockDim.x) dst[i] = __ldcg(src + i);
}

template <typename T>
__global__ void __launch_bounds__(1024, 1)
    jacobi_block_sweep_kernel(T* A, int64_t m, int64_t lda, T* V, int64_t nv, int64_t ldv, int n, int b, int nb2,
                              int wpp, int vrows, bool vec, T tol, T small2, unsigned* rotations, unsigned* bar) {
  using VT = typename Vec16<T>::type;
  constexpr int W = Vec16<T>::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int cols[kBlockJacobiMaxW];
  __shared__ T red[kBlockJacobiMaxW / 2][kBlockJacobiMaxWpp][3];
  __shared__ int any_rot;
  const int w2 = 2 * b, w2p = (w2 + 3) & ~3;
  const int mv = (int)((m + W - 1) / W);   // 16-byte vectors per staged column (zero padded)
  const int mp = mv * W;
  T* As = reinterpret_cast<T*>(smem_raw);   // column c at As + c*mp
  T* Qs = As + (size_t)w2 * mp;             // Q(k, c) at Qs[c*w2p + k]
  T* QT = Qs + (size_t)w2 * w2p;            // Q(k, c) at QT[k*w2p + c]
  T* Vb = QT + (size_t)w2 * w2p;            // two chunk buffers of V, [w2][vrows] each
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nthr = blockDim.x;
  const int pair = warp / wpp, sub = warp % wpp;
  unsigned gen = 0;
  for (int round = 0; round < nb2 - 1; ++round) {
    for (int pi = blockIdx.x; pi < nb2 / 2; pi += gridDim.x) {
      int I, J;
      if (pi == 0) { I = round; J = nb2 - 1; }
      else { I = (round + pi) % (nb2 - 1); J = (round - pi + (nb2 - 1)) % (nb2 - 1); }
      if (threadIdx.x < w2) {
        const int c = threadIdx.x;
        const int gc = ((c < b) ? I : J) * b + (c % b);
        cols[c] = (gc < n) ? gc : -1;
      }
      if (threadIdx.x == 0) any_rot = 0;
      __syncthreads();
      for (int c = 0; c < w2; ++c) {
        const int gc = cols[c];
        T* dst = As + (size_t)c * mp;
        if (gc >= 0) stage_async(dst, A + (int64_t)gc * lda, (int)m, vec);
        for (int e = (gc >= 0 ? (int)m : 0) + threadIdx.x; e < mp; e += nthr) dst[e] = T(0);
      }
      cp_async_commit();
      for (int e = threadIdx.x; e < w2 * w2p; e += nthr) Qs[e] = (e / w2p == e % w2p) ? T(1) : T(0);
      cp_async_wait<0>();
      __syncthreads();
      for (int lr = 0; lr < w2 - 1; ++lr) {
        int p = 0, q = 0;
        bool act = false;
        if (pair < b) {
          if (pair == 0) { p = lr; q = w2 - 1; }
          else { p = (lr + pair) % (w2 - 1); q = (lr - pair + (w2 - 1)) % (w2 - 1); }
          if (p > q) { const int t = p; p = q; q = t; }
          act = cols[p] >= 0 && cols[q] >= 0;
        }
        VT* ap = reinterpret_cast<VT*>(As + (size_t)p * mp);
        VT* aq = reinterpret_cast<VT*>(As + (size_t)q * mp);
        if (act) {
          T al = 0, be = 0, ga = 0;
          for (int i = sub * 32 + lane; i < mv; i += 32 * wpp) dot3(ap[i], aq[i], al, be, ga);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            ga += __shfl_xor_sync(0xffffffffu, ga, o);
          }
          if (lane == 0) { red[pair][sub][0] = al; red[pair][sub][1] = be; red[pair][sub][2] = ga; }
        }
        __syncthreads();
        if (act) {
          T al = 0, be = 0, ga = 0;
          for (int u = 0; u < wpp; ++u) { al += red[pair][u][0]; be += red[pair][u][1]; ga += red[pair][u][2]; }
          if (!(ga == T(0) || al <= small2 || be <= small2) && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
            const T zeta = (be - al) / (T(2) * ga);
            const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, T(1))));
            const T c = T(1) / sqrt(fma(t, t, T(1)));
            const T sn = c * t;
            for (int i = sub * 32 + lane; i < mv; i += 32 * wpp) {
              VT x = ap[i], y = aq[i];
              rot2(x, y, c, sn);
              ap[i] = x;
              aq[i] = y;
            }
            if (sub == 0) {
              if (lane < w2) {
                T* qp = Qs + p * w2p;
                T* qq = Qs + q * w2p;
                const T x = qp[lane], y = qq[lane];
                qp[lane] = c * x - sn * y;
                qq[lane] = sn * x + c * y;
              }
              if (lane == 0) { atomicAdd(rotations, 1u); any_rot = 1; }
            }
          }
        }
        __syncthreads();
      }
      if (any_rot) {
        for (int c = 0; c < w2; ++c) {
          const int gc = cols[c];
          if (gc < 0) continue;
          T* dst = A + (int64_t)gc * lda;
          const T* src = As + (size_t)c * mp;
          int done = 0;
          if (vec) {
            const int full = (int)(m / W);
            for (int i = threadIdx.x; i < full; i += nthr)
              reinterpret_cast<VT*>(dst)[i] = reinterpret_cast<const VT*>(src)[i];
            done = full * W;
          }
          for (int e = done + threadIdx.x; e < m; e += nthr) dst[e] = src[e];
        }
        for (int e = threadIdx.x; e < w2 * w2p; e += nthr) {
          const int k = e / w2p, c = e % w2p;
          QT[e] = (c < w2) ? Qs[c * w2p + k] : T(0);
        }
        if (V) {
          const int nch = (int)((nv + vrows - 1) / vrows);
          auto issue = [&](int ch) {
            T* buf = Vb + (size_t)(ch & 1) * w2 * vrows;
            const int64_t e0 = (int64_t)ch * vrows;
            const int rows = (nv - e0 < vrows) ? (int)(nv - e0) : vrows;
            for (int k = 0; k < w2; ++k) {
              const int gk = cols[k];
              T* dst = buf + (size_t)k * vrows;
              if (gk >= 0) stage_async(dst, V + (int64_t)gk * ldv + e0, rows, vec);
              else for (int r = threadIdx.x; r < vrows; r += nthr) dst[r] = T(0);
            }
            cp_async_commit();
          };
          issue(0);
          for (int ch = 0; ch < nch; ++ch) {
            if (ch + 1 < nch) { issue(ch + 1); cp_async_wait<1>(); }
            else cp_async_wait<0>();
            __syncthreads();
            const T* buf = Vb + (size_t)(ch & 1) * w2 * vrows;
            const int64_t e0 = (int64_t)ch * vrows;
            const int rows = (nv - e0 < vrows) ? (int)(nv - e0) : vrows;
            const int rq_n = (rows + 3) / 4, cq_n = w2p / 4;
            for (int it = threadIdx.x; it < rq_n * cq_n; it += nthr) {
              const int rq = it % rq_n, cq = it / rq_n;
              T acc[4][4];
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
              for (int k = 0; k < w2; ++k) {
                T v[4], qv[4];
                load4(buf + (size_t)k * vrows + 4 * rq, v);
                load4(QT + (size_t)k * w2p + 4 * cq, qv);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                  for (int j = 0; j < 4; ++j) acc[i][j] = fma(v[i], qv[j], acc[i][j]);
              }
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int c = 4 * cq + j;
                const int gc = (c < w2) ? cols[c] : -1;
                if (gc < 0) continue;
                T* dst = V + (int64_t)gc * ldv + e0 + 4 * rq;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                  if (4 * rq + i < rows) dst[i] = acc[i][j];
              }
            }
            __syncthreads();   // the buffer is refilled two chunks on
          }
        }
      }
      __syncthreads();
    }
    if (!grid_barrier(bar, gridDim.x, gen)) return;
  }
}

// A whole sweep in one cooperative launch, one warp per pair.
template <typename T>
__global__ void __launch_bounds__(256) jacobi_sweep_warp_kernel(T* A, int64_t m, int64_t lda, T* V, int64_t nv,
                                                                int64_t ldv, int n, int n2, T tol, T small2,
                                                                unsigned* rotations, unsigned* bar) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (blockDim.x >> 5);
  unsigned gen = 0;
  for (int round = 0; round < n2 - 1; ++round) {
    for (int i = gw; i < n2 / 2; i += nw)
      jacobi_pair_warp<T>(A, m, lda, V, nv, ldv, n, n2, round, i, tol, small2, rotations, lane);
    if (!grid_barrier(bar, gridDim.x, gen)) return;
  }
}

// A whole sweep (all n2-1 rounds) in one cooperative launch; blocks take pairs
// grid-stride and meet at a grid barrier after every round.
template <typename T>
__global__ void __launch_bounds__(256) jacobi_sweep_kernel(T* A, int64_t m, int64_t lda, T* V, int64_t nv,
                                                           int64_t ldv, int n, int n2, T tol, T small2,
                                                           unsigned* rotations, unsigned* bar) {
  unsigned gen = 0;
  for (int round = 0; round < n2 - 1; ++round) {
    for (int i = blockIdx.x; i < n2 / 2; i += gridDim.x)
      jacobi_pair<true, T>(A, m, lda, V, nv, ldv, n, n2, round, i, tol, small2, rotations);
    if (!grid_barrier(bar, gridDim.x, gen)) return;
  }
}

template <typename T>
__global__ void col_norms_kernel(const T* A, int64_t m, int64_t lda, int n, T* out) {
  const int j = blockIdx.x;
  if (j >= n) return;
  const T* a = A + (int64_t)j * lda;
  T s = 0, d1 = 0, d2 = 0;
  for (int64_t e = threadIdx.x; e < m; e += blockDim.x) s = fma(a[e], a[e], s);
  block_sum3<T>(s, d1, d2);
  if (threadIdx.x == 0) out[j] = sqrt(s);
}

__global__ void to_f32_kernel(const double* a, int64_t n, float* b) { GRID_STRIDE(i, n) b[i] = (float)a[i]; }
__global__ void to_f64_kernel(const float* a, int64_t n, double* b) { GRID_STRIDE(i, n) b[i] = (double)a[i]; }
__global__ void identity_f32_kernel(float* V, int64_t n) {
  GRID_STRIDE(i, n * n) V[i] = ((i / n) == (i % n)) ? 1.0f : 0.0f;
}
// C (n x n, row-major, leading dimension ldc): lower triangle := upper triangle
__global__ void mirror_upper_kernel(double* C, int64_t n, int64_t ldc) {
  GRID_STRIDE(e, n * n) {
    const int64_t i = e / n, j = e % n;
    if (i > j) C[i * ldc + j] = C[j * ldc + i];
  }
}
// out (M x r) = U (M x r) with column c scaled by scale[c]
__global__ void scale_cols_kernel2(const double* U, int64_t M, int64_t r, const double* scale, double* out) {
  GRID_STRIDE(e, M * r) out[e] = U[e] * scale[e % r];
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
// same rotations.  Returns the number of sweeps; -1 if the bound was hit.
template <typename T>
int64_t jacobi(T* A, int64_t m, int64_t lda, int n, T* V, int64_t nv, int64_t ldv, int64_t max_sweeps,
               cudaStream_t s, double cos_tol = 0.0) {
  if (n < 2) return 0;
  const int n2 = n + (n & 1);
  const bool f64 = sizeof(T) == 8;
  const T tol = (T)std::max(cos_tol, sqrt((double)m) * (f64 ? 0x1p-52 : 0x1p-23));
  T small2;
  {
    DBuf<T> norms(n, s);
    col_norms_kernel<T><<<n, 256, 0, s>>>(A, m, lda, n, norms.get());
    FTT_LAUNCH();
    std::vector<T> h(n);
    FTT_CUDA(cudaMemcpyAsync(h.data(), norms.get(), sizeof(T) * n, cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    double f2 = 0.0;
    for (T x : h) f2 += (double)x * (double)x;
    small2 = (T)(f2 * (f64 ? 0x1p-100 : 0x1p-42));  // (2^-50 or 2^-21 of ||A||_F)^2
  }
  DBuf<unsigned> rot(5, s);  // [0] rotations, [1..4] grid barrier (count, generation, error, poll bound)
  auto reset_rot = [&]() {
    FTT_CUDA(cudaMemsetAsync(rot.get(), 0, sizeof(unsigned), s));
    barrier_init_kernel<<<1, 1, 0, s>>>(rot.get() + 1, barrier_spins());
    FTT_LAUNCH();
  };
  // a grid barrier that gave up: with an explicit poll bound the call fails, otherwise
  // the sweep is redone one launch per round
  auto barrier_gave_up = [&]() {
    note_wait_timeout();
    if (max_spin() > 0) fail(FASTTT_ETIMEOUT, "a grid barrier of the Jacobi sweep exceeded max_spin polls");
  };
  const double pairs = 0.5 * (double)n * (double)(n - 1);
  // cooperative grid: every block resident at once (bounded by the occupancy)
  int per_sm = 0, coop = 0, dev = 0;
  FTT_CUDA(cudaGetDevice(&dev));
  FTT_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  // columns up to kWarpPairMax long: one warp per pair; longer: one block per pair
  const bool warp_pairs = (m <= kWarpPairMax && nv <= kWarpPairMax);
  void* sweep_fn = warp_pairs ? (void*)jacobi_sweep_warp_kernel<T> : (void*)jacobi_sweep_kernel<T>;
  FTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_fn, 256, 0));
  int sms = 0;
  FTT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int units_per_block = warp_pairs ? 8 : 1;
  const int coop_blocks = std::min((n2 / 2 + units_per_block - 1) / units_per_block, per_sm * sms);
  bool use_coop = coop && coop_blocks >= 1 && n2 / 2 > 1;
  // block schedule (FP32 Gram eigenproblems): b columns per block so that the block
  // pairs of a round fit on the SMs, 2b columns of A resident in shared memory
  int bj = 0, nb2 = 0, bj_grid = 0, bj_wpp = 1, bj_vrows = 0;
  bool bj_vec = false;
  size_t bj_smem = 0;
  if (!f64 && V && coop && n >= 64) {
    int smem_max = 0;
    FTT_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t budget = (size_t)std::max(0, smem_max - 4096);   // static shared memory of the kernel below
    constexpr int W = 16 / (int)sizeof(T);
    const size_t mp = (size_t)ceil_div(m, W) * W;
    auto bytes = [&](int b, int vrows) {
      const size_t w2 = 2 * b, w2p = (w2 + 3) & ~(size_t)3;
      return sizeof(T) * (w2 * mp + 2 * w2 * w2p + 2 * w2 * (size_t)vrows);
    };
    const int vr_cap = (int)std::min<int64_t>(512, (nv + 3) & ~(int64_t)3);
    int b = (int)std::min<int64_t>(kBlockJacobiMaxW / 2, std::max<int64_t>(2, ceil_div(n, 2 * sms)));
    int vrows = 0;
    for (; b >= 2; --b) {
      for (int vr = vr_cap; vr >= 4 && vrows == 0; vr = (vr > 64) ? vr / 2 : vr - 4)
        if (bytes(b, vr & ~3) <= budget) vrows = vr & ~3;
      if (vrows > 0) break;
    }
    if (b >= 2 && vrows >= 4) {
      bj_wpp = std::max(1, std::min(kBlockJacobiMaxWpp, 32 / b));
      bj_vrows = vrows;
      bj_smem = bytes(b, vrows);
      bj_vec = ((uintptr_t)A % 16 == 0) && ((uintptr_t)V % 16 == 0) && ((size_t)lda * sizeof(T)) % 16 == 0 &&
               ((size_t)ldv * sizeof(T)) % 16 == 0;
      // the whole budget (not this call's need), so that concurrent callers never lower it for each other
      FTT_CUDA(cudaFuncSetAttribute(jacobi_block_sweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)budget));
      int per = 0;
      FTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_block_sweep_kernel<T>, 32 * bj_wpp * b,
                                                             bj_smem));
      const int nb = (int)ceil_div(n, b);
      nb2 = nb + (nb & 1);
      bj_grid = std::min(nb2 / 2, per * sms);
      if (bj_grid >= 1) bj = b;
    }
  }
  for (int64_t sweep = 1; sweep <= max_sweeps; ++sweep) {
    reset_rot();
    KClock clk;
    kclock_begin(clk, f64 ? KC_JACOBI : KC_JACOBI32, s);
    bool done = false;
    if (bj > 0) {
      unsigned* rp = rot.get();
      unsigned* bp = rot.get() + 1;
      void* args[] = {(void*)&A,   (void*)&m,      (void*)&lda,      (void*)&V,      (void*)&nv,
                      (void*)&ldv, (void*)&n,      (void*)&bj,       (void*)&nb2,    (void*)&bj_wpp,
                      (void*)&bj_vrows, (void*)&bj_vec, (void*)&tol, (void*)&small2, (void*)&rp,
                      (void*)&bp};
      cudaError_t e = cudaLaunchCooperativeKernel((void*)jacobi_block_sweep_kernel<T>, dim3(bj_grid),
                                                  dim3(32 * bj_wpp * bj), args, bj_smem, s);
      note_block_sweep((int)e);
      if (e == cudaSuccess) {
        FTT_LAUNCH();
        unsigned h[4];
        FTT_CUDA(cudaMemcpyAsync(h, rot.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
        FTT_CUDA(cudaStreamSynchronize(s));
        if (h[3] == 0) done = true;
        else { barrier_gave_up(); bj = 0; }
      } else {
        cudaGetLastError();
        bj = 0;
      }
      if (!done) reset_rot();
    }
    if (!done && use_coop) {
      unsigned* rp = rot.get();
      unsigned* bp = rot.get() + 1;
      void* args[] = {(void*)&A, (void*)&m, (void*)&lda, (void*)&V, (void*)&nv, (void*)&ldv, (void*)&n,
                      (void*)&n2, (void*)&tol, (void*)&small2, (void*)&rp, (void*)&bp};
      cudaError_t e = cudaLaunchCooperativeKernel(sweep_fn, dim3(coop_blocks), dim3(256), args, 0, s);
      if (e == cudaSuccess) {
        FTT_LAUNCH();
        unsigned h[4];
        FTT_CUDA(cudaMemcpyAsync(h, rot.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
        FTT_CUDA(cudaStreamSynchronize(s));
        if (h[3] == 0) done = true;       // no barrier timed out
        else { barrier_gave_up(); use_coop = false; }   // redo this sweep round by round
      } else {
        cudaGetLastError();
        use_coop = false;
      }
      if (!done) reset_rot();
    }
    if (!done) {
      for (int round = 0; round < n2 - 1; ++round) {
        jacobi_round_kernel<T><<<n2 / 2, 256, 0, s>>>(A, m, lda, V, nv, ldv, n, n2, round, tol, small2, rot.get());
      }
      note_launches(n2 - 2);
      FTT_LAUNCH();
    }
    const unsigned rots = read_scalar(rot.get(), s);
    // every pair: three dot products (6m flops); every rotation: 6m + 6nv flops
    kclock_end(clk, pairs * 6.0 * (double)m + (double)rots * 6.0 * (double)(m + (V ? nv : 0)), s);
    if (rots == 0) return sweep;
  }
  return -1;
}

int64_t jacobi_f64(double* A, int64_t m, int64_t lda, int n, double* V, int64_t nv, int64_t ldv,
                   int64_t max_sweeps, cudaStream_t s) {
  const int64_t sw = jacobi<double>(A, m, lda, n, V, nv, ldv, max_sweeps, s);
  if (sw < 0) fail(FASTTT_ETIMEOUT, "Jacobi SVD did not converge within the sweep bound");
  return sw;
}

// Sum of squares of M (n x n, row-major) with `diag` subtracted from the
// diagonal (diag may be null); per-block partials, summed on the host in order.
__global__ void __launch_bounds__(256) sumsq_offdiag_kernel(const double* M, const double* diag, int64_t n,
                                                            double* partial) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    double x = M[e];
    if (diag && e / n == e % n) x -= diag[e / n];
    acc = fma(x, x, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// y = M v - d .* v (d may be null); one warp per row of the n x n row-major M
__global__ void matvec_kernel(const double* M, const double* d, const double* v, int64_t n, double* y) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double acc = 0.0;
  for (int64_t j = lane; j < n; j += 32) acc = fma(M[row * n + j], v[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[row] = d ? acc - d[row] * v[row] : acc;
}

// R <- I - R (R holds X^T X on entry)
__global__ void i_minus_kernel(double* R, int64_t n) {
  GRID_STRIDE(e, n * n) R[e] = ((e / n) == (e % n) ? 1.0 : 0.0) - R[e];
}

// lambda_i = s_ii / (1 - r_ii)
__global__ void oa_lambda_kernel(const double* S, const double* R, int64_t n, double* lam) {
  GRID_STRIDE(i, n) lam[i] = S[i * n + i] / (1.0 - R[i * n + i]);
}

// The correction of the refinement step: e_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)
// for |lambda_j - lambda_i| > delta, e_ij = r_ij / 2 otherwise (clusters, diagonal).
// guard > 0: the first-order correction is also withheld (e_ij = r_ij / 2) where it
// would exceed guard in magnitude, i.e. where the pair is still mixed by more than
// the first-order analysis covers (such pairs are left to the Rayleigh-Ritz step).
__global__ void oa_correction_kernel(const double* S, const double* R, const double* lam, double delta, int64_t n,
                                     double* E, double guard = 0.0) {
  GRID_STRIDE(e, n * n) {
    const int64_t i = e / n, j = e % n;
    const double d = lam[j] - lam[i];
    const double num = S[e] + lam[j] * R[e];
    const bool first_order = (i != j && fabs(d) > delta && (guard == 0.0 || fabs(num) <= guard * fabs(d)));
    E[e] = first_order ? num / d : 0.5 * R[e];
  }
}

// res[i] = sqrt(sum_{j != i} s_ij^2): the residual ||G x_i - lambda_i x_i|| of an
// orthonormal X (one warp per row)
__global__ void offdiag_row_norms_kernel(const double* S, int64_t n, double* res) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double acc = 0.0;
  for (int64_t j = lane; j < n; j += 32)
    if (j != row) acc = fma(S[row * n + j], S[row * n + j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) res[row] = sqrt(acc);
}

// v <- y / ||y|| and est = ||y|| (one block; the power method's normalisation on the device)
__global__ void __launch_bounds__(256) normalise_vec_kernel(const double* y, int64_t n, double* v, double* est) {
  __shared__ double red[8];
  __shared__ double nrm;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc = fma(y[i], y[i], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    nrm = sqrt(t);
    *est = nrm;
  }
  __syncthreads();
  const double inv = (nrm > 0.0) ? 1.0 / nrm : 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v[i] = y[i] * inv;
}

// ||M - diag(d)||_2 of a symmetric n x n matrix by 12 steps of the power method
// from a fixed start (an estimate from below; callers add a safety factor)
double norm2_sym(const double* M, const double* d, int64_t n, cudaStream_t s) {
  std::vector<double> h(n);
  for (int64_t i = 0; i < n; ++i) h[i] = 1.0 + 0.5 * sin(0.7 * (double)i + 0.3);
  double nrm = 0.0;
  for (double x : h) nrm += x * x;
  nrm = sqrt(nrm);
  for (auto& x : h) x /= nrm;
  DBuf<double> v(n, s), y(n, s), est(1, s);
  FTT_CUDA(cudaMemcpyAsync(v.get(), h.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  for (int it = 0; it < 12; ++it) {
    matvec_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, s>>>(M, d, v.get(), n, y.get());
    FTT_LAUNCH();
    normalise_vec_kernel<<<1, 256, 0, s>>>(y.get(), n, v.get(), est.get());   // ||M v|| with ||v|| = 1
    FTT_LAUNCH();
  }
  const double e = read_scalar(est.get(), s);
  return std::isfinite(e) ? e : 0.0;
}

double sumsq(const double* M, const double* diag, int64_t n, cudaStream_t s) {
  const int blocks = 2 * kNumSMs;
  DBuf<double> part(blocks, s);
  sumsq_offdiag_kernel<<<blocks, 256, 0, s>>>(M, diag, n, part.get());
  FTT_LAUNCH();
  std::vector<double> h(blocks);
  FTT_CUDA(cudaMemcpyAsync(h.data(), part.get(), sizeof(double) * blocks, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  double t = 0.0;
  for (double x : h) t += x;
  return t;
}

// Eigen-decomposition of a symmetric positive semi-definite n x n matrix G
// (FP64, row-major; left intact).  FP32 one-sided Jacobi from V = I gives
// approximate eigenvectors X (orthonormal to ~1e-7); then the iterative
// refinement for symmetric eigendecompositions of Ogita & Aishima (Japan J.
// Indust. Appl. Math. 35, 2018) in FP64, which needs only products:
//   R = I - X^T X,  S = X^T G X,  lambda_i = s_ii / (1 - r_ii),
//   delta = 2 (||S - diag(lambda)|| + ||G|| ||R||)   (Frobenius norms, >= 2-norms),
//   E_ij as in oa_correction_kernel,  X <- X + X E,
// repeated until ||R|| and ||S - diag(lambda)|| / ||G|| are at rounding level.
// V (column-major: column j = eigenvector j, i.e. row-major X^T) and the
// eigenvalues (host) are returned.  Returns the FP32 sweeps.
int64_t sym_eig_refined(const double* G, int n, double* V, std::vector<double>& lam_out, int64_t max_sweeps,
                        cudaStream_t s) {
  const int64_t nn = (int64_t)n * n;
  int64_t sweeps;
  {
    DBuf<float> G32(nn, s), V32(nn, s);
    to_f32_kernel<<<grid_for(nn), 256, 0, s>>>(G, nn, G32.get());
    FTT_LAUNCH();
    identity_f32_kernel<<<grid_for(nn), 256, 0, s>>>(V32.get(), n);
    FTT_LAUNCH();
    sweeps = jacobi<float>(G32.get(), n, n, n, V32.get(), n, n, max_sweeps, s);  // a starting point only
    to_f64_kernel<<<grid_for(nn), 256, 0, s>>>(V32.get(), nn, V);
    FTT_LAUNCH();
  }
  const double g2 = sumsq(G, nullptr, n, s);
  const double gF = sqrt(g2);
  DBuf<double> R(nn, s), W(nn, s), S(nn, s), lam(n, s);
  lam_out.assign(n, 0.0);
  double prev = INFINITY;
  for (int it = 0; it < 8; ++it) {
    // X^T is V's memory (row-major, row j = eigenvector j)
    gemm_f64(n, n, n, 1.0, V, n, 1, V, 1, n, 0.0, R.get(), n, 1, s, true);           // X^T X
    i_minus_kernel<<<grid_for(nn), 256, 0, s>>>(R.get(), n);
    FTT_LAUNCH();
    gemm_f64(n, n, n, 1.0, V, n, 1, G, n, 1, 0.0, W.get(), n, 1, s);                 // W = X^T G (row j = (G x_j)^T)
    gemm_f64(n, n, n, 1.0, V, n, 1, W.get(), 1, n, 0.0, S.get(), n, 1, s, true);     // S = X^T G X
    oa_lambda_kernel<<<grid_for(n), 256, 0, s>>>(S.get(), R.get(), n, lam.get());
    FTT_LAUNCH();
    const double offS = sqrt(sumsq(S.get(), lam.get(), n, s));
    const double rF = sqrt(sumsq(R.get(), nullptr, n, s));
    FTT_CUDA(cudaMemcpyAsync(lam_out.data(), lam.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    if (!std::isfinite(offS) || !std::isfinite(rF)) fail(FASTTT_ENUMERIC, "non-finite eigen refinement");
    // Continue while the (quadratically converging) error keeps shrinking; stop at
    // the rounding level of the n-term FP64 products or when it stalls (eigenvalue
    // clusters closer than the refinement can separate: the polish resolves them).
    const double tiny = 64.0 * (double)n * 0x1p-53;
    const double err = rF + offS / gF;
    if ((rF <= tiny && offS <= tiny * gF) || err > 0.25 * prev) break;
    prev = err;
    // delta of the refinement with 2-norms (power-method estimates with a safety
    // factor of 2; Frobenius norms would overstate them by up to sqrt(n))
    const double s2 = std::min(offS, 2.0 * norm2_sym(S.get(), lam.get(), n, s));
    const double r2 = std::min(rF, 2.0 * norm2_sym(R.get(), nullptr, n, s));
    double lmax = 0.0;
    for (double x : lam_out) lmax = std::max(lmax, fabs(x));
    const double delta = 2.0 * (s2 + lmax * r2);
    oa_correction_kernel<<<grid_for(nn), 256, 0, s>>>(S.get(), R.get(), lam.get(), delta, n, W.get());  // W <- E
    FTT_LAUNCH();
    // X <- X + X E, in X^T layout: X^T <- X^T + E^T X^T
    FTT_CUDA(cudaMemcpyAsync(S.get(), V, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    gemm_f64(n, n, n, 1.0, W.get(), 1, n, S.get(), n, 1, 1.0, V, n, 1, s);
  }
  // Orthonormalise X to FP64 rounding (Newton-Schulz: X <- 1.5 X - 0.5 X (X^T X),
  // quadratic while ||I - X^T X|| < 1), whatever the refinement left.
  for (int it = 0; it < 3; ++it) {
    gemm_f64(n, n, n, 1.0, V, n, 1, V, 1, n, 0.0, R.get(), n, 1, s, true);            // S = X^T X
    i_minus_kernel<<<grid_for(nn), 256, 0, s>>>(R.get(), n);
    FTT_LAUNCH();
    const double rF = sqrt(sumsq(R.get(), nullptr, n, s));
    if (!(rF < 0.5)) fail(FASTTT_ENUMERIC, "eigenvector basis lost orthogonality");
    if (rF <= 16.0 * (double)n * 0x1p-53) break;
    // in X^T layout: X^T <- X^T + 0.5 (I - X^T X) X^T  (equivalent to the Newton-Schulz step)
    FTT_CUDA(cudaMemcpyAsync(S.get(), V, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    gemm_f64(n, n, n, 0.5, R.get(), n, 1, S.get(), n, 1, 1.0, V, n, 1, s);
  }
  // Polish: FP64 one-sided Jacobi on A = G X with the rotations accumulated into X
  // (column-major); converged columns have norms lambda_j.  Rotates little when the
  // refinement converged; resolves eigenvalue clusters it left mixed.
  gemm_f64(n, n, n, 1.0, V, n, 1, G, n, 1, 0.0, W.get(), n, 1, s);   // row j of A^T = (G x_j)^T
  jacobi_f64(W.get(), n, n, n, V, n, n, max_sweeps, s);
  DBuf<double> norms(n, s);
  col_norms_kernel<double><<<n, 256, 0, s>>>(W.get(), n, n, n, norms.get());
  FTT_LAUNCH();
  FTT_CUDA(cudaMemcpyAsync(lam_out.data(), norms.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  return sweeps;
}

// dst row j = src row perm[j] (n x n row-major)
__global__ void permute_rows_kernel(const double* src, const int32_t* perm, int64_t n, double* dst) {
  GRID_STRIDE(e, n * n) dst[e] = src[(int64_t)perm[e / n] * n + e % n];
}

// Ogita-Aishima refinement (see sym_eig_refined) of approximate eigenvectors V
// (row j = x_j) of the symmetric G, with FP64-level products (mixed: FP32-level
// products, stopped at FP32-level residuals).  Pairs closer than the refinement's
// separation threshold delta are left mixed by it; each run of such eigenvalues
// that is wider than the rounding level gets a Rayleigh-Ritz step: FP64 one-sided
// Jacobi on G X_c with the rotations applied to X_c.  Returns false when the
// refinement does not converge (the caller takes another route).
bool refine_eig(const double* G, int n, double* V, std::vector<double>& lam_out, int64_t max_sweeps, cudaStream_t s,
                bool mixed) {
  const int64_t nn = (int64_t)n * n;
  const double g2 = sumsq(G, nullptr, n, s);
  const double gF = sqrt(g2);
  lam_out.assign(n, 0.0);
  if (g2 == 0.0) return true;   // the zero matrix: the start's V = I is exact
  if (!std::isfinite(g2)) return false;
  DBuf<double> R(nn, s), W(nn, s), S(nn, s), lam(n, s), Vbak(nn, s);
  const double u = mixed ? 0x1p-24 : 0x1p-53;
  const double tiny = (mixed ? 64.0 : 1.0) * (double)n * u;
  constexpr double kGuard = 1.0 / 16.0;   // largest first-order correction applied
  double best = INFINITY;
  int since_best = 0;
  bool have_bak = false;
  // X^T X, S = X^T G X and the Rayleigh quotients for the current V; returns err
  auto evaluate = [&](double& rF, double& offS) {
    gemm(mixed, n, n, n, 1.0, V, n, 1, V, 1, n, 0.0, R.get(), n, 1, s, true);        // X^T X
    i_minus_kernel<<<grid_for(nn), 256, 0, s>>>(R.get(), n);
    FTT_LAUNCH();
    gemm(mixed, n, n, n, 1.0, V, n, 1, G, n, 1, 0.0, W.get(), n, 1, s);              // W = X^T G
    gemm(mixed, n, n, n, 1.0, V, n, 1, W.get(), 1, n, 0.0, S.get(), n, 1, s, true);  // S = X^T G X
    oa_lambda_kernel<<<grid_for(n), 256, 0, s>>>(S.get(), R.get(), n, lam.get());
    FTT_LAUNCH();
    offS = sqrt(sumsq(S.get(), lam.get(), n, s));
    rF = sqrt(sumsq(R.get(), nullptr, n, s));
    FTT_CUDA(cudaMemcpyAsync(lam_out.data(), lam.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    return rF + offS / gF;
  };
  // Quadratic convergence is not monotone in err (a large first-order step leaves a
  // second-order loss of orthogonality that the next step removes): iterate until
  // converged or two steps without a new best, then continue from the best state.
  double rF = 0.0, offS = 0.0;
  for (int it = 0; it < 8; ++it) {
    const double err = evaluate(rF, offS);
    if (!std::isfinite(err)) return false;
    double lmax_it = 0.0;
    for (double x : lam_out) lmax_it = std::max(lmax_it, fabs(x));
    // converged: orthonormal and diagonal to the rounding level of n-term products
    // (residuals ||G x_i - lambda_i x_i|| <= ||S - D||_F against ||G||_2)
    if (rF <= tiny && offS <= tiny * lmax_it) { best = err; since_best = 0; break; }
    if (err < best) {
      best = err;
      since_best = 0;
      FTT_CUDA(cudaMemcpyAsync(Vbak.get(), V, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
      have_bak = true;
    } else if (++since_best >= 2 && it >= 4) {   // well-separated pairs converge within four steps
      break;
    }
    if (!(rF < 0.5) || it == 7) break;   // the state of the last evaluation is kept
    double lmax = 0.0;
    for (double x : lam_out) lmax = std::max(lmax, fabs(x));
    const double s2 = std::min(offS, 2.0 * norm2_sym(S.get(), lam.get(), n, s));
    const double r2 = std::min(rF, 2.0 * norm2_sym(R.get(), nullptr, n, s));
    const double delta = 2.0 * (s2 + lmax * r2);
    oa_correction_kernel<<<grid_for(nn), 256, 0, s>>>(S.get(), R.get(), lam.get(), delta, n, W.get(), kGuard);
    FTT_LAUNCH();
    // X <- X + X E, in X^T layout: X^T <- X^T + E^T X^T
    FTT_CUDA(cudaMemcpyAsync(S.get(), V, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    gemm(mixed, n, n, n, 1.0, W.get(), 1, n, S.get(), n, 1, 1.0, V, n, 1, s);
  }
  if (since_best > 0 || !(rF < 0.5)) {
    if (!have_bak) return false;
    FTT_CUDA(cudaMemcpyAsync(V, Vbak.get(), sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    evaluate(rF, offS);
    if (!(rF < 0.5)) return false;
  }
  // The refinement's separation threshold at the final state: pairs closer than it
  // were never rotated apart by the first-order correction.
  double delta_final;
  {
    double lmax = 0.0;
    for (double x : lam_out) lmax = std::max(lmax, fabs(x));
    const double s2 = std::min(offS, 2.0 * norm2_sym(S.get(), lam.get(), n, s));
    const double r2 = std::min(rF, 2.0 * norm2_sym(R.get(), nullptr, n, s));
    delta_final = 2.0 * (s2 + lmax * r2);
  }
  // Runs of close eigenvalues (ascending) that the refinement left mixed: closer
  // than its threshold, or with residuals not small against their gap (the
  // eigenvector error is bounded by residual / gap, the Rayleigh quotient's by
  // residual^2 / gap).  Each run is resolved by Rayleigh-Ritz.
  std::vector<double> res(n);
  {
    offdiag_row_norms_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, s>>>(S.get(), n, lam.get());
    FTT_LAUNCH();
    FTT_CUDA(cudaMemcpyAsync(res.data(), lam.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int32_t> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return lam_out[a] < lam_out[b]; });
  double lmax = 0.0;
  for (double x : lam_out) lmax = std::max(lmax, fabs(x));
  const double wtol = 4.0 * (double)n * u * lmax;
  const double ltol = (double)n * u * lmax;   // Rayleigh quotients err by about residual^2 / gap
  std::vector<std::pair<int, int>> runs;
  int64_t rr_work = 0;
  auto coupled = [&](int a, int b) {
    const double gap = lam_out[b] - lam_out[a], r = std::max(res[a], res[b]);
    return gap <= delta_final || gap <= 16.0 * r || r * r > ltol * gap;
  };
  for (int i = 0; i < n;) {
    int j = i + 1;
    while (j < n && coupled(perm[j - 1], perm[j])) ++j;
    // a run whose Rayleigh quotients agree to rounding is a multiple eigenvalue only if its
    // residuals are at rounding level too (a pair mixed at 45 degrees has equal quotients)
    double rmax = 0.0;
    for (int q = i; q < j; ++q) rmax = std::max(rmax, res[perm[q]]);
    if (j - i >= 2 && (lam_out[perm[j - 1]] - lam_out[perm[i]] > wtol || rmax > ltol)) {
      runs.emplace_back(i, j);
      rr_work += (int64_t)(j - i) * (j - i);
    }
    i = j;
  }
  // FP32-level refinement only needs the invariant subspaces (a run's vectors may stay
  // mixed): Rayleigh-Ritz is an FP64 step
  if (mixed) runs.clear();
  if (!runs.empty()) {
    if ((double)rr_work * (double)n > 4.0e11) return false;   // too much Jacobi work: another route
    DBuf<int32_t> dperm(n, s);
    FTT_CUDA(cudaMemcpyAsync(dperm.get(), perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    permute_rows_kernel<<<grid_for(nn), 256, 0, s>>>(V, dperm.get(), n, W.get());
    FTT_LAUNCH();
    FTT_CUDA(cudaMemcpyAsync(V, W.get(), sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    std::vector<double> sorted(n);
    for (int i = 0; i < n; ++i) sorted[i] = lam_out[perm[i]];
    lam_out = sorted;
    FTT_CUDA(cudaStreamSynchronize(s));   // perm is host memory read by the copy above
    DBuf<double> norms(n, s);
    for (const auto& rn : runs) {
      const int64_t j0 = rn.first, c = rn.second - rn.first;
      double* Vc = V + j0 * n;
      double* Wc = W.get() + j0 * n;
      gemm(mixed, c, n, n, 1.0, Vc, n, 1, G, n, 1, 0.0, Wc, n, 1, s);   // rows j0.. of X^T G: (G x_j)^T
      jacobi_f64(Wc, n, n, (int)c, Vc, n, n, max_sweeps, s);
      col_norms_kernel<double><<<(unsigned)c, 256, 0, s>>>(Wc, n, n, (int)c, norms.get());
      FTT_LAUNCH();
      std::vector<double> h(c);
      FTT_CUDA(cudaMemcpyAsync(h.data(), norms.get(), sizeof(double) * c, cudaMemcpyDeviceToHost, s));
      FTT_CUDA(cudaStreamSynchronize(s));
      // the columns of G X_c have norms |lambda|; the run's Rayleigh quotients give the sign
      const double sgn = (lam_out[j0] + lam_out[j0 + c - 1] < 0.0) ? -1.0 : 1.0;
      for (int64_t q = 0; q < c; ++q) lam_out[j0 + q] = sgn * h[q];
    }
  }
  // Orthonormalise X to the rounding level of the products (Newton-Schulz,
  // quadratic: one step takes ||I - X^T X|| from ~sqrt(n) u to the rounding floor).
  for (int it = 0; it < 4; ++it) {
    gemm(mixed, n, n, n, 1.0, V, n, 1, V, 1, n, 0.0, R.get(), n, 1, s, true);
    i_minus_kernel<<<grid_for(nn), 256, 0, s>>>(R.get(), n);
    FTT_LAUNCH();
    const double rF = sqrt(sumsq(R.get(), nullptr, n, s));
    if (!(rF < 0.5)) return false;
    if (rF <= 2.0 * (double)n * u) break;
    FTT_CUDA(cudaMemcpyAsync(S.get(), V, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    gemm(mixed, n, n, n, 0.5, R.get(), n, 1, S.get(), n, 1, 1.0, V, n, 1, s);
  }
  return true;
}

}  // namespace

int64_t jacobi_svd_f64(double* A, int64_t m, int64_t lda, int n, double* V, int64_t nv, int64_t ldv,
                       int64_t max_sweeps, cudaStream_t s) {
  return jacobi_f64(A, m, lda, n, V, nv, ldv, max_sweeps, s);
}

void gemm_f64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
              const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
              cudaStream_t s, bool sym) {
  if (gemm_engine() == 0 && K >= 64 && (double)M * (double)N * (double)K >= kTensorGemmMin &&
      gemm_ozaki(7, M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci, scj, s, sym))
    return;
  gemm_f64_dfma(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci, scj, s, sym);
}

void gemm_f64_dfma(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
                   const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
                   cudaStream_t s, bool sym) {
  if (M <= 0 || N <= 0) return;
  if (sym && (M != N || sci < N || scj != 1)) fail(FASTTT_EINVAL, "symmetric GEMM needs a square row-major C");
  const int64_t gx = ceil_div(M, kTile), gy = ceil_div(N, kTile);
  if (gy > 65535) fail(FASTTT_ERANK, "GEMM: N too large");
  dim3 grid((unsigned)gx, (unsigned)gy);
  KClock clk;
  kclock_begin(clk, KC_GEMM, s);
  gemm_f64_kernel<<<grid, 256, 0, s>>>(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci, scj, sym);
  FTT_LAUNCH();
  // algorithmic flops: the full product (a symmetric product's mirrored half is not counted twice)
  kclock_end(clk, (sym ? 1.0 : 2.0) * (double)M * (double)N * (double)K + (sym ? (double)M * K : 0.0), s);
  if (sym) {
    mirror_upper_kernel<<<grid_for(M * M), 256, 0, s>>>(C, M, sci);
    FTT_LAUNCH();
  }
}

void transpose_f64(const double* src, int64_t rows, int64_t cols, double* dst, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  if (ceil_div(cols, 32) > INT32_MAX) fail(FASTTT_ERANK, "transpose: too many columns");
  dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)std::min<int64_t>(ceil_div(rows, 32), 65535));
  dim3 block(32, 8);
  transpose_kernel<<<grid, block, 0, s>>>(src, rows, cols, dst);
  FTT_LAUNCH();
}

namespace {

// Counters of the mixed-precision Gram route (bonds kept at FP32 level, bonds
// redone with FP64-level products), read into the statistics.
std::atomic<int64_t> g_mixed_kept{0}, g_mixed_escalated{0};

// Kept eigenvalues must lie this many times above the Gram route's error floor
// for an FP32-level result to be used.
constexpr double kResolve = 64.0;

// sigma = sqrt(max(lambda, 0)) sorted descending with the permutation that sorts them.
void sigma_from_lambda(const std::vector<double>& h, std::vector<double>& sig, std::vector<int32_t>& perm) {
  const int n = (int)h.size();
  perm.resize(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::vector<double> sv(n);
  for (int i = 0; i < n; ++i) {
    sv[i] = sqrt(std::max(h[i], 0.0));
    if (!std::isfinite(sv[i])) fail(FASTTT_ENUMERIC, "non-finite singular value");
  }
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return sv[a] > sv[b]; });
  sig.resize(n);
  for (int i = 0; i < n; ++i) sig[i] = sv[perm[i]];
}

// Whether an FP32-level spectrum can decide this bond: the rank chosen does not
// change when every eigenvalue sigma_i^2 moves by +-floor, and the kept ones lie
// kResolve * floor or more above zero.  choose_rank is called on the perturbed
// spectra only; the caller calls it once more on the spectrum it keeps.
bool rank_is_resolved(const std::function<int64_t(const std::vector<double>&)>& choose_rank,
                      const std::vector<double>& sig, int64_t nkeep, double floor) {
  const int64_t n = (int64_t)sig.size();
  if (n == 0) return true;
  const int64_t r0 = std::max<int64_t>(1, std::min<int64_t>(choose_rank(sig), nkeep));
  const double sr = sig[r0 - 1];
  if (!(sr * sr >= kResolve * floor)) return false;
  std::vector<double> up(n), dn(n);
  for (int64_t i = 0; i < n; ++i) {
    up[i] = sqrt(sig[i] * sig[i] + floor);
    dn[i] = sqrt(std::max(sig[i] * sig[i] - floor, 0.0));
  }
  const int64_t ru = std::max<int64_t>(1, std::min<int64_t>(choose_rank(up), nkeep));
  const int64_t rd = std::max<int64_t>(1, std::min<int64_t>(choose_rank(dn), nkeep));
  return ru == r0 && rd == r0;
}

// The FP32 start of the Gram eigensolver, kept so that a bond redone at FP64 level
// refines the same start instead of computing it again.
struct EigStart {
  DBuf<double> V;
  std::vector<double> lam;
  bool ok = false;
  bool declined = false;   // the start did not apply: the retry goes to the FP64 routes
};

// Eigenpairs of the symmetric Gram G (n x n) into V (row j = eigenvector j) and h.
// mixed: FP32 start + FP32-level refinement, false when either declines.  FP64
// level: the stored start refined with FP64-level products if there is one, else
// the fast route, then the FP64 tridiagonal route, then the iterative one.
bool gram_eig(const double* G, int n, double* V, std::vector<double>& h, int64_t max_sweeps, cudaStream_t s,
              bool mixed, EigStart& st0, int64_t& sweeps,
              const std::function<bool(const std::vector<double>&)>& start_ok = nullptr,
              const std::function<int64_t(const std::vector<double>&)>& topk = nullptr, int64_t kmax = 0) {
  sweeps = 0;
  const int64_t nn = (int64_t)n * n;
  // few eigenvectors wanted (a rank cap): the FP64 tridiagonal route computes only those
  if (!mixed && topk) {
    if (sym_eig_tridiag(G, n, V, h, s, false, topk, kmax)) {
      note_eig(true);
      return true;
    }
  }
  if (mixed) {
    if (!sym_eig_start_f32(G, n, V, h, s)) {
      st0.declined = true;
      return false;
    }
    st0.V = DBuf<double>(nn, s);
    FTT_CUDA(cudaMemcpyAsync(st0.V.get(), V, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    st0.lam = h;
    st0.ok = true;
    // a bond that the start already shows to be unresolvable at FP32 level goes to
    // FP64 before any FP32-level refinement is spent on it
    if (start_ok && !start_ok(h)) return false;
    if (!refine_eig(G, n, V, h, max_sweeps, s, true)) return false;
    note_eig_fast();
    return true;
  }
  if (st0.ok) {
    FTT_CUDA(cudaMemcpyAsync(V, st0.V.get(), sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    h = st0.lam;
    if (refine_eig(G, n, V, h, max_sweeps, s, false)) {
      note_eig_fast();
      return true;
    }
  } else if (!st0.declined && sym_eig_fast(G, n, V, h, max_sweeps, s, false)) {
    return true;
  }
  const bool td = sym_eig_tridiag(G, n, V, h, s, false);
  note_eig(td);
  if (!td) sweeps = sym_eig_refined(G, n, V, h, max_sweeps, s);
  return true;
}

}  // namespace

int64_t mixed_bonds_kept() { return g_mixed_kept.load(); }
int64_t mixed_bonds_escalated() { return g_mixed_escalated.load(); }

namespace {

// Tall-skinny shapes (lg >= 4n, n >= 96; narrower ones are cheaper on TSQR): the tall
// orientation T (A, column-major lg x n) = Q R by FP64 CholeskyQR2, one-sided Jacobi on
// the n x n R only
// (R V = U_R Sigma), then A <- Q (R V) = T V by one FP64-level GEMM: the same result
// as Jacobi on T (backward error u ||T||) with the sweeps on n rows instead of lg.
// False, A untouched, when the shape does not apply or CholeskyQR2 breaks down (T too
// ill conditioned): the caller takes TSQR or Jacobi on T.
bool cholqr_jacobi(double* A, int64_t lg, int n, double* V, int64_t max_sweeps, cudaStream_t s, int64_t& sweeps) {
  if (n < 96 || lg < 4 * (int64_t)n) return false;
  const int64_t nn = (int64_t)n * n;
  DBuf<double> Q((size_t)lg * n, s), R(nn, s), Rc(nn, s);
  FTT_CUDA(cudaMemcpyAsync(Q.get(), A, sizeof(double) * lg * n, cudaMemcpyDeviceToDevice, s));
  // A's memory is row-major n x lg (rows = columns of T): CholeskyQR2 of its rows gives
  // A = R^T Q, i.e. T = Q^T R with Q^T's columns orthonormal
  if (!cholqr2_rows(Q.get(), n, lg, R.get(), false, s)) return false;
  transpose_f64(R.get(), n, n, Rc.get(), s);   // column-major R
  sweeps = jacobi_f64(Rc.get(), n, n, n, V, n, n, max_sweeps, s);
  // A (column-major lg x n) = Q^T (lg x n) . Rc:  A(i, j) = sum_k Q[k lg + i] Rc[j n + k]
  gemm_f64(lg, n, n, 1.0, Q.get(), 1, lg, Rc.get(), 1, n, 0.0, A, 1, lg, s);
  return true;
}

// Direct route: one-sided Jacobi (through TSQR or CholeskyQR2 for tall-skinny
// shapes) on the tall orientation of Z, FP64 whatever the precision.
void svd_direct(const double* Z, int64_t M, int64_t N,
                const std::function<int64_t(const std::vector<double>&)>& choose_rank, int64_t max_sweeps,
                SvdOut& out, cudaStream_t s) {
  const bool tall = (M >= N);
  const int64_t lg = tall ? M : N;
  const int n = (int)(tall ? N : M);
  DBuf<double> A((size_t)lg * n, s);   // column-major lg x n
  if (tall) transpose_f64(Z, M, N, A.get(), s);  // columns of Z become contiguous
  else FTT_CUDA(cudaMemcpyAsync(A.get(), Z, sizeof(double) * M * N, cudaMemcpyDeviceToDevice, s));
  DBuf<double> V((size_t)n * n, s);
  std::vector<double> h(n);
  identity_kernel<<<grid_for((int64_t)n * n), 256, 0, s>>>(V.get(), n);
  FTT_LAUNCH();
  if (cholqr_jacobi(A.get(), lg, n, V.get(), max_sweeps, s, out.sweeps)) {
    // done: Jacobi on CholeskyQR2's R
  } else if (tsqr_applies(lg, n)) {
    out.sweeps = tsqr_jacobi(A.get(), lg, n, V.get(), max_sweeps, s);
  } else {
    out.sweeps = jacobi_f64(A.get(), lg, lg, n, V.get(), n, n, max_sweeps, s);
  }
  {
    DBuf<double> norms(n, s);
    col_norms_kernel<double><<<n, 256, 0, s>>>(A.get(), lg, lg, n, norms.get());
    FTT_LAUNCH();
    FTT_CUDA(cudaMemcpyAsync(h.data(), norms.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
  }
  for (double x : h)
    if (!std::isfinite(x)) fail(FASTTT_ENUMERIC, "non-finite singular value");
  // the column norms are the singular values: sort them as they are (squares would underflow)
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
  if (tall) {  // Z V = A  ->  U = A Sigma^-1, Vt = V^T
    gather_cols_kernel<<<grid_for(M * r), 256, 0, s>>>(A.get(), lg, M, dperm.get(), dinv.get(), r, out.U.get());
    FTT_LAUNCH();
    gather_rows_kernel<<<grid_for(r * N), 256, 0, s>>>(V.get(), n, N, dperm.get(), nullptr, r, out.Vt.get());
  } else {     // Z^T V = A  ->  Z = V Sigma (A Sigma^-1)^T
    gather_cols_kernel<<<grid_for(M * r), 256, 0, s>>>(V.get(), n, M, dperm.get(), nullptr, r, out.U.get());
    FTT_LAUNCH();
    gather_rows_kernel<<<grid_for(r * N), 256, 0, s>>>(A.get(), lg, N, dperm.get(), dinv.get(), r, out.Vt.get());
  }
  FTT_LAUNCH();
  FTT_CUDA(cudaStreamSynchronize(s));   // host vectors read by the copies above
}

// Gram route at one precision level.  FP64 level (mixed = false) always completes.
// Mixed: the Gram, the refinement and the projections are FP32-level products;
// the result is kept only when (1) the probed distance of the FP32-level Gram from
// Z^T Z (or Z Z^T) plus the refinement's rounding level gives an error floor that
// the kept eigenvalues clear by kResolve and that cannot move the rank decision
// (rank_is_resolved), and (2) the factor that the projection amplifies by
// sigma_1 / sigma_r comes out of CholeskyQR2 orthonormal.  Otherwise false: the
// caller redoes the bond at FP64 level.
bool svd_gram(const double* Z, int64_t M, int64_t N,
              const std::function<int64_t(const std::vector<double>&)>& choose_rank, int64_t max_sweeps,
              SvdOut& out, cudaStream_t s, bool mixed, int ortho, EigStart& st0) {
  const bool tall = (M >= N);
  const int n = (int)(tall ? N : M);
  DBuf<double> A((size_t)n * n, s);
  if (tall)  // G = Z^T Z
    gemm(mixed, N, N, M, 1.0, Z, 1, N, Z, N, 1, 0.0, A.get(), N, 1, s, true);
  else       // G = Z Z^T
    gemm(mixed, M, M, N, 1.0, Z, N, 1, Z, 1, N, 0.0, A.get(), M, 1, s, true);
  DBuf<double> V((size_t)n * n, s);
  std::vector<double> h(n);
  int64_t sweeps = 0;
  // mixed: the error floor of the FP32-level route = the probed distance of the Gram from
  // Z^T Z (Z Z^T) plus the rounding level of the FP32-level eigen-refinement; the FP32
  // start is tested against it with its own error (FP32 tridiagonalisation) added
  const double gram_err = mixed ? 4.0 * gram_error_probe(Z, M, N, A.get(), s) : 0.0;
  auto floor_of = [&](const std::vector<double>& lam, double c) {
    double lmax = 0.0;
    for (double x : lam) lmax = std::max(lmax, fabs(x));
    return gram_err + c * sqrt((double)n) * lmax;
  };
  auto start_ok = [&](const std::vector<double>& lam) {
    std::vector<double> sg;
    std::vector<int32_t> pm;
    sigma_from_lambda(lam, sg, pm);
    return rank_is_resolved(choose_rank, sg, n, floor_of(lam, 0x1p-21));
  };
  if (!gram_eig(A.get(), n, V.get(), h, max_sweeps, s, mixed, st0, sweeps, start_ok)) return false;
  out.sweeps = sweeps;
  std::vector<int32_t> perm;
  sigma_from_lambda(h, out.sigma_all, perm);
  if (mixed && !rank_is_resolved(choose_rank, out.sigma_all, n, floor_of(h, 0x1p-23))) return false;
  A.reset();
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
  bool ok = true;
  if (tall) {  // V: right vectors; U = Z V_r Sigma^-1
    DBuf<double> Vs((size_t)N * r, s);
    gather_cols_kernel<<<grid_for(N * r), 256, 0, s>>>(V.get(), n, N, dperm.get(), dinv.get(), r, Vs.get());
    FTT_LAUNCH();
    gather_rows_kernel<<<grid_for(r * N), 256, 0, s>>>(V.get(), n, N, dperm.get(), nullptr, r, out.Vt.get());
    FTT_LAUNCH();
    gemm(mixed, M, r, N, 1.0, Z, N, 1, Vs.get(), r, 1, 0.0, out.U.get(), r, 1, s);
    if (mixed && ortho == kOrthoLeft) {
      // U = Z V Sigma^-1 carries the FP32-level product error times sigma_1 / sigma_r:
      // CholeskyQR2 makes U orthonormal, then Vt = Sigma^-1 U^T Z (U Sigma Vt = U U^T Z)
      ok = orthonormalise_cols_cholqr2(out.U.get(), M, r, true, s);
      if (ok) {
        DBuf<double> Us((size_t)M * r, s);
        scale_cols_kernel2<<<grid_for(M * r), 256, 0, s>>>(out.U.get(), M, r, dinv.get(), Us.get());
        FTT_LAUNCH();
        gemm(mixed, r, N, M, 1.0, Us.get(), 1, r, Z, N, 1, 0.0, out.Vt.get(), N, 1, s);
      }
    }
  } else {     // V: left vectors; Vt = Sigma^-1 U_r^T Z
    gather_cols_kernel<<<grid_for(M * r), 256, 0, s>>>(V.get(), n, M, dperm.get(), nullptr, r, out.U.get());
    FTT_LAUNCH();
    DBuf<double> Us((size_t)M * r, s);
    gather_cols_kernel<<<grid_for(M * r), 256, 0, s>>>(V.get(), n, M, dperm.get(), dinv.get(), r, Us.get());
    FTT_LAUNCH();
    gemm(mixed, r, N, M, 1.0, Us.get(), 1, r, Z, N, 1, 0.0, out.Vt.get(), N, 1, s);
    if (mixed && ortho == kOrthoRight) {
      // Vt = Sigma^-1 U^T Z: CholeskyQR2 on its rows, then U = Z Vt^T Sigma^-1, so that
      // U Sigma Vt = Z Vt^T Vt
      ok = cholqr2_rows(out.Vt.get(), r, N, nullptr, true, s);
      if (ok) {
        DBuf<double> ZV((size_t)M * r, s);
        gemm(mixed, M, r, N, 1.0, Z, N, 1, out.Vt.get(), 1, N, 0.0, ZV.get(), r, 1, s);
        scale_cols_kernel2<<<grid_for(M * r), 256, 0, s>>>(ZV.get(), M, r, dinv.get(), out.U.get());
        FTT_LAUNCH();
      }
    }
  }
  FTT_CUDA(cudaStreamSynchronize(s));   // host vectors read by the copies above
  return ok;
}

}  // namespace

void svd_truncated(const double* Z, int64_t M, int64_t N,
                   const std::function<int64_t(const std::vector<double>&)>& choose_rank, int64_t max_sweeps,
                   SvdOut& out, cudaStream_t s, bool mixed, int ortho) {
  const bool tall = (M >= N);
  const int64_t sm = tall ? N : M;   // number of singular values
  const int64_t lg = tall ? M : N;
  if (sm > INT32_MAX / 2) fail(FASTTT_ERANK, "SVD too large");
  // direct (accurate) route while a Jacobi sweep stays below ~4e10 flops
  const bool direct = (sm <= kDirectMax) || (9.0 * (double)lg * (double)sm * (double)sm <= 4.0e10);
  if (direct) {
    svd_direct(Z, M, N, choose_rank, max_sweeps, out, s);
    return;
  }
  EigStart st0;
  if (mixed) {
    if (svd_gram(Z, M, N, choose_rank, max_sweeps, out, s, true, ortho, st0)) {
      g_mixed_kept.fetch_add(1);
      return;
    }
    g_mixed_escalated.fetch_add(1);
    out = SvdOut();
  }
  svd_gram(Z, M, N, choose_rank, max_sweeps, out, s, false, ortho, st0);
}

bool sym_eig_fast(const double* G, int n, double* V, std::vector<double>& lam_out, int64_t max_sweeps, cudaStream_t s,
                  bool mixed) {
  if (!sym_eig_start_f32(G, n, V, lam_out, s)) return false;
  if (!refine_eig(G, n, V, lam_out, max_sweeps, s, mixed)) return false;
  note_eig_fast();
  return true;
}

void sym_eig_iterative(const double* G, int n, double* V, std::vector<double>& lam_out, int64_t max_sweeps,
                       cudaStream_t s) {
  sym_eig_refined(G, n, V, lam_out, max_sweeps, s);
}

void svd_from_gram(const double* Gram, int64_t M, int64_t N,
                   const std::function<int64_t(const std::vector<double>&)>& choose_rank, int64_t max_sweeps,
                   SvdOut& out, cudaStream_t s, bool mixed, int64_t kcap, bool partial) {
  if (M > INT32_MAX / 2) fail(FASTTT_ERANK, "SVD too large");
  const int n = (int)M;
  const int nsv = (int)std::min<int64_t>(n, N);
  // the eigenvectors the rank rule will keep, plus a margin for ties at the boundary
  auto topk = [&](const std::vector<double>& lam) -> int64_t {
    std::vector<double> sg;
    std::vector<int32_t> pm;
    sigma_from_lambda(lam, sg, pm);
    sg.resize(nsv);
    const int64_t r = std::max<int64_t>(1, std::min<int64_t>(choose_rank(sg), nsv));
    return std::min<int64_t>(n, r + 8);
  };
  const bool capped = kcap > 0 && 4 * kcap <= n;
  DBuf<double> V((size_t)n * n, s);
  std::vector<double> h(n);
  std::vector<int32_t> perm;
  EigStart st0;
  bool done = false;
  if (mixed && capped) g_mixed_escalated.fetch_add(1);   // the top-k FP64 route is cheaper than any start
  if (mixed && !capped) {
    // The Gram is an FP64 sum here: the error floor is the FP32-level refinement's
    int64_t sw = 0;
    auto start_ok = [&](const std::vector<double>& lam) {
      std::vector<double> sg;
      std::vector<int32_t> pm;
      sigma_from_lambda(lam, sg, pm);
      double lmax = 0.0;
      for (double x : lam) lmax = std::max(lmax, fabs(x));
      sg.resize(nsv);
      return rank_is_resolved(choose_rank, sg, nsv, 0x1p-21 * sqrt((double)n) * lmax);
    };
    if (gram_eig(Gram, n, V.get(), h, max_sweeps, s, true, st0, sw, start_ok)) {
      sigma_from_lambda(h, out.sigma_all, perm);
      double lmax = 0.0;
      for (double x : h) lmax = std::max(lmax, fabs(x));
      out.sigma_all.resize(nsv);
      done = rank_is_resolved(choose_rank, out.sigma_all, nsv, 0x1p-23 * sqrt((double)n) * lmax);
      out.sweeps = sw;
    }
    (done ? g_mixed_kept : g_mixed_escalated).fetch_add(1);
  }
  if (!done) {
    int64_t sw = 0;
    // the rank rule keeps at most kcap: the kcap + 16 largest eigenvalues decide it
    gram_eig(Gram, n, V.get(), h, max_sweeps, s, false, st0, sw, nullptr,
             capped ? std::function<int64_t(const std::vector<double>&)>(topk) : nullptr,
             (capped && partial) ? std::min<int64_t>(n, kcap + 16) : 0);
    out.sweeps = sw;
    sigma_from_lambda(h, out.sigma_all, perm);
    out.sigma_all.resize(nsv);
  }
  int64_t r = choose_rank(out.sigma_all);
  r = std::max<int64_t>(1, std::min<int64_t>(r, nsv));
  out.r = r;
  DBuf<int32_t> dperm(r, s);
  out.sigma = DBuf<double>(r, s);
  FTT_CUDA(cudaMemcpyAsync(dperm.get(), perm.data(), sizeof(int32_t) * r, cudaMemcpyHostToDevice, s));
  FTT_CUDA(cudaMemcpyAsync(out.sigma.get(), out.sigma_all.data(), sizeof(double) * r, cudaMemcpyHostToDevice, s));
  out.U = DBuf<double>((size_t)M * r, s);
  gather_cols_kernel<<<grid_for(M * r), 256, 0, s>>>(V.get(), n, M, dperm.get(), nullptr, r, out.U.get());
  FTT_LAUNCH();
  FTT_CUDA(cudaStreamSynchronize(s));   // perm and sigma_all are host memory read by the copies above
}


}  // namespace fasttt
