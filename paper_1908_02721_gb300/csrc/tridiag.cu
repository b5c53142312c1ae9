// Symmetric eigendecomposition of the Gram matrices of the TT-rounding SVDs
// (S7-S10) by the textbook dense route (Golub & Van Loan, Matrix Computations,
// 4th ed., Sec. 8.3 and 8.4):
//   1. Householder tridiagonalisation A = Q T Q^T, one cooperative kernel; per
//      column k every block forms the reflector of A[k, k+1:] (identical
//      fixed-order sums), the grid computes p = tau A22 v, and after a grid
//      barrier the rank-2 update A22 -= v w^T + w v^T, w = p - (tau/2)(p.v) v.
//   2. All eigenvalues of T by bisection on Sturm counts (one thread each).
//   3. Eigenvectors of T by inverse iteration (one thread each): T - lambda I
//      factored once with partial pivoting, three solves from a fixed
//      pseudo-random start; eigenvalues closer than a few ulps of ||T|| are
//      first moved apart so that their vectors differ.
//   4. Newton-Schulz re-orthonormalisation Z <- Z + Z (I - Z^T Z) / 2 in FP64.
//   5. X = Q Z with the reflectors applied back in blocked WY form
//      (I - V T V^T per block of 64, T as in LAPACK's xLARFT) on the GEMMs.
// Returns false, leaving the caller to its iterative eigensolver, when the
// inverse-iteration vectors are too far from orthonormal (tight clusters) or
// the grid barrier gave up.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dense.cuh"
#include "devsync.cuh"

namespace fasttt {

namespace {

constexpr int kWYBlock = 64;

__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

__global__ void __launch_bounds__(256)
    tridiag_kernel(double* A, int64_t n, double* d, double* e, double* tau, double* p, unsigned* bar) {
  extern __shared__ double vs[];   // the current reflector v (v_0 = 1)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + warp, W = (int64_t)gridDim.x * 8;
  unsigned gen = 0;
  for (int64_t k = 0; k + 2 < n; ++k) {
    const int64_t m = n - k - 1;
    const double* x = A + k * n + k + 1;   // A[k, k+1:] = A[k+1:, k]
    double s = 0.0, z1 = 0.0, z2 = 0.0;
    for (int64_t j = 1 + threadIdx.x; j < m; j += blockDim.x) {
      const double t = __ldcg(x + j);
      s = fma(t, t, s);
    }
    block_sum3<double>(s, z1, z2);
    const double alpha = __ldcg(x);
    double beta = alpha, tk = 0.0, scale = 0.0;
    if (s > 0.0) {
      beta = -copysign(sqrt(fma(alpha, alpha, s)), alpha);
      tk = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) vs[j] = (j == 0) ? 1.0 : __ldcg(x + j) * scale;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      d[k] = __ldcg(A + k * n + k);
      e[k] = beta;
      tau[k] = tk;
    }
    // p = tau A22 v, one warp per row
    for (int64_t i = gw; i < m; i += W) {
      const double* row = A + (k + 1 + i) * n + (k + 1);
      double acc = 0.0;
      for (int64_t j = lane; j < m; j += 32) acc = fma(__ldcg(row + j), vs[j], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) p[i] = tk * acc;
    }
    if (!grid_barrier(bar, gridDim.x, gen)) return;
    double pv = 0.0;
    z1 = z2 = 0.0;
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) pv = fma(__ldcg(p + j), vs[j], pv);
    block_sum3<double>(pv, z1, z2);
    const double K = 0.5 * tk * pv;
    if (tk != 0.0) {
      for (int64_t i = gw; i < m; i += W) {
        double* row = A + (k + 1 + i) * n + (k + 1);
        const double vi = vs[i], wi = __ldcg(p + i) - K * vi;
        for (int64_t j = lane; j < m; j += 32) {
          const double vj = vs[j], wj = __ldcg(p + j) - K * vj;
          row[j] = __ldcg(row + j) - vi * wj - wi * vj;
        }
      }
    }
    if (blockIdx.x == 0)   // keep v in row k (columns k+1:) for the back-transformation
      for (int64_t j = threadIdx.x; j < m; j += blockDim.x) A[k * n + k + 1 + j] = vs[j];
    if (!grid_barrier(bar, gridDim.x, gen)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n >= 2) {
      d[n - 2] = __ldcg(A + (n - 2) * n + n - 2);
      e[n - 2] = __ldcg(A + (n - 2) * n + n - 1);
      tau[n - 2] = 0.0;
    }
    d[n - 1] = __ldcg(A + (n - 1) * n + n - 1);
  }
}

// Number of eigenvalues of T (diagonal d, squared off-diagonal e2) below x.
__device__ int sturm_count(const double* d, const double* e2, int64_t n, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) <= pivmin) q = -pivmin;
  if (q < 0.0) ++c;
  for (int64_t i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) <= pivmin) q = -pivmin;
    if (q < 0.0) ++c;
  }
  return c;
}

// lam[j] = the j-th smallest eigenvalue (j = 0..n-1) by bisection of [gl, gu]
// down to abstol or adjacent doubles (at most 128 halvings).
__global__ void bisect_kernel(const double* d, const double* e2, int64_t n, double gl, double gu, double pivmin,
                              double abstol, double* lam) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double lo = gl, hi = gu;
    for (int it = 0; it < 128; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (!(mid > lo && mid < hi) || hi - lo <= abstol) break;
      if (sturm_count(d, e2, n, mid, pivmin) > j) hi = mid;
      else lo = mid;
    }
    lam[j] = 0.5 * (lo + hi);
  }
}

__device__ __forceinline__ double start_component(int64_t i, int64_t j) {
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + (uint64_t)j * 0xD1B54A32D192ED03ull + 0x2545F4914F6CDD1Dull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1p-52 - 1.0;   // in [-1, 1)
}

// Inverse iteration: thread t computes the eigenvector of T for shift lam[j0 + t]
// into column j0 + t of Z (n x ldz row-major).  T - lambda I = P L U with partial
// pivoting (tridiagonal LU with one fill-in diagonal); scratch arrays are laid
// out [i * nv + t] so that a warp's accesses are contiguous.
__global__ void inverse_iteration_kernel(const double* d, const double* e, int64_t n, const double* shift, int64_t j0,
                                         int64_t nv, double pert, double* sdd, double* sdu, double* sdu2, double* sdl,
                                         unsigned char* spiv, double* Z, int64_t ldz) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nv) return;
  const int64_t j = j0 + t;
  const double lam = shift[j];
#define S(a, i) a[(int64_t)(i) * nv + t]
  for (int64_t i = 0; i < n; ++i) {
    S(sdd, i) = d[i] - lam;
    if (i + 1 < n) { S(sdu, i) = e[i]; S(sdl, i) = e[i]; }
    S(sdu2, i) = 0.0;
  }
  for (int64_t i = 0; i + 1 < n; ++i) {
    const double di = S(sdd, i), li = S(sdl, i);
    if (fabs(di) >= fabs(li)) {
      const double piv = (di == 0.0) ? pert : di;
      S(sdd, i) = piv;
      const double f = li / piv;
      S(sdl, i) = f;
      S(sdd, i + 1) = S(sdd, i + 1) - f * S(sdu, i);
      S(spiv, i) = 0;
    } else {
      const double f = di / li;
      S(sdd, i) = li;
      S(sdl, i) = f;
      const double u = S(sdu, i);
      S(sdu, i) = S(sdd, i + 1);
      S(sdd, i + 1) = u - f * S(sdd, i + 1);
      if (i + 2 < n) {
        S(sdu2, i) = S(sdu, i + 1);
        S(sdu, i + 1) = -f * S(sdu, i + 1);
      }
      S(spiv, i) = 1;
    }
  }
  if (fabs(S(sdd, n - 1)) < pert) S(sdd, n - 1) = copysign(pert, S(sdd, n - 1));
  for (int64_t i = 0; i < n; ++i)
    if (fabs(S(sdd, i)) < pert) S(sdd, i) = copysign(pert, S(sdd, i));
  double* z = Z + j;
  for (int64_t i = 0; i < n; ++i) z[i * ldz] = start_component(i, j);
  for (int it = 0; it < 3; ++it) {
    for (int64_t i = 0; i + 1 < n; ++i) {   // L
      double bi = z[i * ldz], bn = z[(i + 1) * ldz];
      if (S(spiv, i)) { const double tmp = bi; bi = bn; bn = tmp; }
      z[i * ldz] = bi;
      z[(i + 1) * ldz] = bn - S(sdl, i) * bi;
    }
    for (int64_t i = n - 1; i >= 0; --i) {   // U
      double v = z[i * ldz];
      if (i + 1 < n) v -= S(sdu, i) * z[(i + 1) * ldz];
      if (i + 2 < n) v -= S(sdu2, i) * z[(i + 2) * ldz];
      z[i * ldz] = v / S(sdd, i);
    }
    double mx = 0.0;
    for (int64_t i = 0; i < n; ++i) mx = fmax(mx, fabs(z[i * ldz]));
    if (!(mx > 0.0) || !isfinite(mx)) mx = 1.0;
    double nrm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const double v = z[i * ldz] / mx;
      nrm = fma(v, v, nrm);
    }
    const double inv = 1.0 / (mx * sqrt(nrm));
    for (int64_t i = 0; i < n; ++i) z[i * ldz] *= inv;
  }
#undef S
}

// Vb (nr x kb row-major) = reflectors k0 .. k0+kb-1 on rows k0+1 .. n-1: column c
// holds v_{k0+c} from row k0+c+1 on (stored in row k0+c of A), zeros above.
__global__ void wy_vectors_kernel(const double* A, int64_t n, int64_t k0, int64_t kb, double* Vb) {
  const int64_t nr = n - k0 - 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nr * kb; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / kb, c = e % kb;
    Vb[e] = (r >= c) ? A[(k0 + c) * n + (k0 + 1 + r)] : 0.0;
  }
}

// S += V^T V for the rows of V (nr x kb row-major, kb <= 64) in this block's
// slice of rows (split over the grid; partial sums added by FP64 atomics).
__global__ void __launch_bounds__(256) wy_gram_kernel(const double* __restrict__ V, int64_t nr, int64_t kb,
                                                      double* __restrict__ S) {
  __shared__ double tile[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  const int64_t per = ceil_div_dev(nr, gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(nr, r0 + per);
  for (int64_t k0 = r0; k0 < r1; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e >> 6, c = e & 63;
      tile[kk][c] = (k0 + kk < r1 && c < kb) ? V[(k0 + kk) * kb + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = tile[kk][ty + 16 * q]; b[q] = tile[kk][tx + 16 * q]; }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[q][w] = fma(a[q], b[w], acc[q][w]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int i = ty + 16 * q, j = tx + 16 * w;
      if (i < kb && j < kb) atomicAdd(S + i * kb + j, acc[q][w]);
    }
}

// T (kb x kb, upper triangular, row-major) of H_1 ... H_kb = I - V T V^T from
// S = V^T V and the tau: T_ii = tau_i, T[0:i, i] = -tau_i T[0:i, 0:i] S[0:i, i].
__global__ void wy_t_kernel(const double* S, const double* tau, int64_t kb, double* T) {
  for (int64_t e = threadIdx.x; e < kb * kb; e += blockDim.x) T[e] = 0.0;
  __syncthreads();
  for (int64_t i = 0; i < kb; ++i) {
    const double ti = tau[i];
    if (threadIdx.x == 0) T[i * kb + i] = ti;
    for (int64_t r = threadIdx.x; r < i; r += blockDim.x) {
      double acc = 0.0;
      for (int64_t c = r; c < i; ++c) acc = fma(T[r * kb + c], S[c * kb + i], acc);
      T[r * kb + i] = -ti * acc;
    }
    __syncthreads();
  }
}

__global__ void i_minus_sym_kernel(double* R, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x)
    R[e] = ((e / n) == (e % n) ? 1.0 : 0.0) - R[e];
}

__global__ void sumsq_kernel(const double* R, int64_t n, double* part) {
  double acc = 0.0, z1 = 0.0, z2 = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    acc = fma(R[e], R[e], acc);
  block_sum3<double>(acc, z1, z2);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

double frob2(const double* R, int64_t count, cudaStream_t s) {
  const int blocks = 2 * kNumSMs;
  DBuf<double> part(blocks, s);
  sumsq_kernel<<<blocks, 256, 0, s>>>(R, count, part.get());
  FTT_LAUNCH();
  std::vector<double> h(blocks);
  FTT_CUDA(cudaMemcpyAsync(h.data(), part.get(), sizeof(double) * blocks, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  double t = 0.0;
  for (double x : h) t += x;
  return t;
}

}  // namespace

bool sym_eig_tridiag(const double* G, int n, double* V, std::vector<double>& lam_out, cudaStream_t s, bool mixed) {
  if (n < 3) return false;
  int dev = 0, coop = 0, sms = 0, smem_max = 0;
  FTT_CUDA(cudaGetDevice(&dev));
  FTT_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  FTT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  FTT_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t smem = sizeof(double) * (size_t)n;
  if (!coop || smem + 4096 > (size_t)smem_max) return false;
  const int64_t nn = (int64_t)n * n;
  DBuf<double> A(nn, s), d(n, s), e(n, s), tau(n, s), p(n, s);
  FTT_CUDA(cudaMemcpyAsync(A.get(), G, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  // 1. tridiagonalisation
  {
    FTT_CUDA(cudaFuncSetAttribute(tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per = 0;
    FTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tridiag_kernel, 256, smem));
    const int grid = std::min(2, per) * sms;
    if (grid < 1) return false;
    DBuf<unsigned> bar(4, s);
    FTT_CUDA(cudaMemsetAsync(bar.get(), 0, 4 * sizeof(unsigned), s));
    int64_t n64 = n;
    double *Ap = A.get(), *dp = d.get(), *ep = e.get(), *tp = tau.get(), *pp = p.get();
    unsigned* bp = bar.get();
    void* args[] = {(void*)&Ap, (void*)&n64, (void*)&dp, (void*)&ep, (void*)&tp, (void*)&pp, (void*)&bp};
    KClock clk;
    kclock_begin(clk, KC_TRIDIAG, s);
    const cudaError_t err = cudaLaunchCooperativeKernel((void*)tridiag_kernel, dim3(grid), dim3(256), args, smem, s);
    if (err != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    FTT_LAUNCH();
    kclock_end(clk, 2.0 * (double)n * (double)n * (double)n, s);   // symv 2m^2 + rank-2 4m^2 per column
    unsigned hb[4];
    FTT_CUDA(cudaMemcpyAsync(hb, bar.get(), sizeof(hb), cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    if (hb[2] != 0) return false;
  }
  std::vector<double> hd(n), he(n);
  FTT_CUDA(cudaMemcpyAsync(hd.data(), d.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaMemcpyAsync(he.data(), e.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  // 2. eigenvalues: Gershgorin interval, bisection
  double gl = INFINITY, gu = -INFINITY, emax2 = 0.0, tnorm = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(he[i - 1]) : 0.0) + (i + 1 < n ? fabs(he[i]) : 0.0);
    gl = std::min(gl, hd[i] - r);
    gu = std::max(gu, hd[i] + r);
    tnorm = std::max(tnorm, fabs(hd[i]) + r);
    if (i + 1 < n) emax2 = std::max(emax2, he[i] * he[i]);
  }
  if (!std::isfinite(gl) || !std::isfinite(gu)) fail(FASTTT_ENUMERIC, "non-finite tridiagonal matrix");
  const double widen = 2.0 * 0x1p-52 * std::max(tnorm, 1e-300) * n;
  gl -= widen;
  gu += widen;
  const double pivmin = 0x1p-1000 * std::max(1.0, emax2);
  std::vector<double> he2(n, 0.0);
  for (int i = 0; i + 1 < n; ++i) he2[i] = he[i] * he[i];
  DBuf<double> e2(n, s), lam(n, s), shift(n, s);
  FTT_CUDA(cudaMemcpyAsync(e2.get(), he2.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  KClock clk2;
  kclock_begin(clk2, KC_TDEIG, s);
  const double abstol = 2.0 * 0x1p-53 * std::max(tnorm, 1e-300);   // the accuracy T carries from step 1
  bisect_kernel<<<grid_for(n, 128), 128, 0, s>>>(d.get(), e2.get(), n, gl, gu, pivmin, abstol, lam.get());
  FTT_LAUNCH();
  std::vector<double> hl(n);
  FTT_CUDA(cudaMemcpyAsync(hl.data(), lam.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  // shifts for inverse iteration: eigenvalues closer than sep are moved apart
  const double sep = 16.0 * 0x1p-53 * tnorm;
  std::vector<double> hs(hl);
  for (int i = 1; i < n; ++i)
    if (hs[i] - hs[i - 1] < sep) hs[i] = hs[i - 1] + sep;
  FTT_CUDA(cudaMemcpyAsync(shift.get(), hs.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  // 3. eigenvectors of T, in batches bounding the scratch to ~2 GB
  DBuf<double> Z(nn, s);
  {
    const int64_t batch = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)(2.0e9 / (33.0 * n))));
    DBuf<double> sdd(n * batch, s), sdu(n * batch, s), sdu2(n * batch, s), sdl(n * batch, s);
    DBuf<unsigned char> spiv(n * batch, s);
    const double pert = 0x1p-53 * std::max(tnorm, 1e-300);
    for (int64_t j0 = 0; j0 < n; j0 += batch) {
      const int64_t nv = std::min<int64_t>(batch, n - j0);
      inverse_iteration_kernel<<<(unsigned)ceil_div(nv, 32), 32, 0, s>>>(
          d.get(), e.get(), n, shift.get(), j0, nv, pert, sdd.get(), sdu.get(), sdu2.get(), sdl.get(), spiv.get(),
          Z.get(), n);
      FTT_LAUNCH();
    }
  }
  kclock_end(clk2, 0.0, s);
  // 4. orthonormalise Z (rows of T's basis, columns = vectors) in FP64
  {
    DBuf<double> R(nn, s), Z0(nn, s);
    bool ok = false;
    for (int it = 0; it < 4; ++it) {
      gemm_f64(n, n, n, 1.0, Z.get(), 1, n, Z.get(), n, 1, 0.0, R.get(), n, 1, s, true);   // Z^T Z
      i_minus_sym_kernel<<<grid_for(nn), 256, 0, s>>>(R.get(), n);
      FTT_LAUNCH();
      const double rF = sqrt(frob2(R.get(), nn, s));
      if (!(rF < 0.5)) break;
      if (rF <= 16.0 * (double)n * 0x1p-53) { ok = true; break; }
      FTT_CUDA(cudaMemcpyAsync(Z0.get(), Z.get(), sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
      gemm_f64(n, n, n, 0.5, Z0.get(), n, 1, R.get(), n, 1, 1.0, Z.get(), n, 1, s);   // Z += Z R / 2
      ok = (it == 3);
    }
    if (!ok) return false;
  }
  // 5. X = Q Z, blocks of reflectors from the last to the first
  {
    const int64_t nrefl = n - 2;
    DBuf<double> Vb((size_t)(n - 1) * kWYBlock, s), S((size_t)kWYBlock * kWYBlock, s),
        T((size_t)kWYBlock * kWYBlock, s), W1((size_t)kWYBlock * n, s), W2((size_t)kWYBlock * n, s);
    for (int64_t k0 = ((nrefl - 1) / kWYBlock) * kWYBlock; k0 >= 0; k0 -= kWYBlock) {
      const int64_t kb = std::min<int64_t>(kWYBlock, nrefl - k0), nr = n - k0 - 1;
      wy_vectors_kernel<<<grid_for(nr * kb), 256, 0, s>>>(A.get(), n, k0, kb, Vb.get());
      FTT_LAUNCH();
      FTT_CUDA(cudaMemsetAsync(S.get(), 0, sizeof(double) * kb * kb, s));
      wy_gram_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nr, 64), kNumSMs)), 256, 0, s>>>(
          Vb.get(), nr, kb, S.get());
      FTT_LAUNCH();
      wy_t_kernel<<<1, 64, 0, s>>>(S.get(), tau.get() + k0, kb, T.get());
      FTT_LAUNCH();
      double* Zs = Z.get() + (k0 + 1) * n;
      gemm(mixed, kb, n, nr, 1.0, Vb.get(), 1, kb, Zs, n, 1, 0.0, W1.get(), n, 1, s);   // V^T Z
      gemm_f64(kb, n, kb, 1.0, T.get(), kb, 1, W1.get(), n, 1, 0.0, W2.get(), n, 1, s);  // T (V^T Z)
      gemm(mixed, nr, n, kb, -1.0, Vb.get(), kb, 1, W2.get(), n, 1, 1.0, Zs, n, 1, s);  // Z -= V T V^T Z
    }
  }
  transpose_f64(Z.get(), n, n, V, s);   // V: column j = eigenvector j
  lam_out = hl;
  return true;
}

}  // namespace fasttt
