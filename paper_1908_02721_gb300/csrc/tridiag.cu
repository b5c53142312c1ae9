// Symmetric eigendecomposition of the Gram matrices of the TT-rounding SVDs
// (S7-S10) by the textbook dense route (Golub & Van Loan, Matrix Computations,
// 4th ed., Sec. 8.3 and 8.4):
//   1. Householder tridiagonalisation A = Q T Q^T.  Per column k every block forms
//      the reflector of A[k, k+1:] (identical fixed-order sums), the grid computes
//      p = tau A22 v, and the rank-2 update A22 -= v w^T + w v^T,
//      w = p - (tau/2)(p.v) v, follows.  In FP64, panels of 64 columns are reduced
//      against the matrix as it was at the panel's start and the panel's updates
//      applied afterwards as one symmetric GEMM (tridiag_panel_kernel); the last
//      columns, and the FP32 start, run one cooperative kernel with the update of
//      column k-1 fused into the product of column k (tridiag_kernel).
//   2. The eigenvalues of T (all, or the largest a caller needs) by multisection on
//      Sturm counts.
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
#include <cstring>
#include <vector>

#include "dense.cuh"
#include "devsync.cuh"

namespace fasttt {

namespace {

constexpr int kWYBlock = 64;
constexpr int kClusterMax = 256;   // largest eigenvalue cluster of the FP32 start
constexpr int kPanel = 64;         // columns per panel of the blocked FP64 tridiagonalisation
constexpr int kPanelTail = 512;    // columns left to the unblocked kernel

__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Householder tridiagonalisation (one cooperative launch), one grid barrier per
// column.  Warps own rows (or row segments) of the trailing matrix; in the pass
// of column k a warp applies column k-1's rank-2 update A -= v w^T + w v^T to
// its rows and takes their dot products with reflector k in the same sweep.
// Reflector k comes from row k after column k-1's update, which every block forms
// redundantly in shared memory (no one writes it in global memory), so the only
// grid-wide dependency left is p = tau A v.  Rows are cut into up to kMaxSeg
// segments so that short rows still keep every warp busy; a segment's partial
// product goes to part[segment][row] and the partials are summed in a fixed
// order after the barrier (deterministic).  Row k keeps v_k (v_0 = 1 stored),
// written once every block has formed its copy of row k (after the barrier).
constexpr int kMaxSeg = 8;

// NW warps per block (one block per SM).  FP32: 32 warps hide the shared-memory and
// load latency of the column passes; FP64: the FP64 pipe is the limit and 8 warps keep
// it as busy as more would.
template <typename T>
struct TridiagWarps { static constexpr int value = 8; };
template <>
struct TridiagWarps<float> { static constexpr int value = 32; };

// SHARED: the row and the reflector share one buffer (v_k formed in place), so that
// three vectors of n values fit where four would not (n above ~7,000 in FP64).
template <typename T, int NW, bool SHARED>
__global__ void __launch_bounds__(NW * 32)
    tridiag_kernel(T* A, int64_t n, int64_t k0, T* d, T* e, T* tau, T* part, unsigned* bar) {
  extern __shared__ __align__(16) unsigned char vs_raw[];
  const int64_t cap = n - k0;             // longest vector: the first column's trailing size + 1
  T* vs = reinterpret_cast<T*>(vs_raw);   // v_k
  T* vp = vs + cap;                       // v_{k-1}
  T* ws = vp + cap;                       // w_{k-1} = p - (tau/2)(p.v) v
  T* rk = SHARED ? vs : ws + cap;         // row k after column k-1's update
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * NW + warp, W = (int64_t)gridDim.x * NW;
  unsigned gen = 0;
  T tprev = 0;   // tau_{k-1}
  int64_t nseg_prev = 1;
  // w of the previous column from its partials (trailing size mp)
  // partials of column k live in part[(k & 1) * kMaxSeg * n ..]: a block may write column
  // k+1's while another still reads column k's (both between the same two barriers)
  auto form_w = [&](int64_t mp, int64_t kprev) {
    const T* pp = part + (kprev & 1) * kMaxSeg * n;
    T pv = 0, z1 = 0, z2 = 0;
    for (int64_t j = threadIdx.x; j < mp; j += blockDim.x) {
      T acc = 0;
      for (int64_t sg = 0; sg < nseg_prev; ++sg) acc += __ldcg(pp + sg * n + j);
      ws[j] = acc;   // tau already applied
      pv = fma(acc, vp[j], pv);
    }
    block_sum3n<T, NW>(pv, z1, z2);   // ends with a barrier
    const T K = T(0.5) * tprev * pv;
    for (int64_t j = threadIdx.x; j < mp; j += blockDim.x) ws[j] = ws[j] - K * vp[j];
    __syncthreads();
  };
  // columns k0 .. n-3 (k0 > 0: the columns before were reduced by the blocked panels, whose
  // updates the trailing matrix has taken in full)
  for (int64_t k = k0; k + 2 < n; ++k) {
    const int64_t m = n - k - 1;
    const bool upd = (k > k0) && (tprev != T(0));   // column k-1's update is not the identity
    if (k > k0) {
      form_w(m + 1, k - 1);
      // every block has read row k-1 (before the last barrier): keep v_{k-1} there now
      if (blockIdx.x == 0)
        for (int64_t j = threadIdx.x; j < m + 1; j += blockDim.x) A[(k - 1) * n + k + j] = vp[j];
    }
    // row k after column k-1's update (index 0 of that trailing matrix)
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
      T x = __ldcg(A + k * n + k + 1 + j);
      if (upd) x = x - vp[0] * ws[1 + j] - ws[0] * vp[1 + j];
      rk[j] = x;
    }
    __syncthreads();
    // rk[0] is read before block_sum3n's barriers, so v_k below may overwrite it in place
    const T alpha = rk[0];
    T s = 0, z1 = 0, z2 = 0;
    for (int64_t j = 1 + threadIdx.x; j < m; j += blockDim.x) s = fma(rk[j], rk[j], s);
    block_sum3n<T, NW>(s, z1, z2);   // ends with a barrier
    T beta = alpha, tk = 0, scale = 0;
    if (s > T(0)) {
      beta = -copysign(sqrt(fma(alpha, alpha, s)), alpha);
      tk = (beta - alpha) / beta;
      scale = T(1) / (alpha - beta);
    }
    for (int64_t j = threadIdx.x; j < m; j += blockDim.x) vs[j] = (j == 0) ? T(1) : rk[j] * scale;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      T dk = __ldcg(A + k * n + k);
      if (upd) dk = dk - T(2) * vp[0] * ws[0];
      d[k] = dk;
      e[k] = beta;
      tau[k] = tk;
    }
    // fused pass: rows k+1+i (i < m), columns k+1+j (j < m) of the column-k trailing matrix
    const int64_t nseg = max((int64_t)1, min((int64_t)kMaxSeg, W / m));
    const int64_t seg = ((m + nseg - 1) / nseg + 31) / 32 * 32;   // segment length, a multiple of 32
    for (int64_t task = gw; task < m * nseg; task += W) {
      const int64_t i = task / nseg, sg = task % nseg;
      T* row = A + (k + 1 + i) * n + (k + 1);
      const int64_t j0 = sg * seg, j1 = min(m, j0 + seg);
      const T vi = upd ? vp[1 + i] : T(0), wi = upd ? ws[1 + i] : T(0);
      T a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = 0;
      int64_t j = j0 + lane;
      for (; j + 224 < j1; j += 256) {
        T r[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) r[u] = __ldcg(row + j + 32 * u);
        if (upd) {
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            r[u] = r[u] - vi * ws[1 + j + 32 * u] - wi * vp[1 + j + 32 * u];
            row[j + 32 * u] = r[u];
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = fma(r[u], vs[j + 32 * u], a[u]);
      }
      for (; j < j1; j += 32) {
        T r = __ldcg(row + j);
        if (upd) {
          r = r - vi * ws[1 + j] - wi * vp[1 + j];
          row[j] = r;
        }
        a[0] = fma(r, vs[j], a[0]);
      }
      T acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) part[(k & 1) * kMaxSeg * n + sg * n + i] = tk * acc;
    }
    if (!grid_barrier(bar, gridDim.x, gen)) return;
    // v_k becomes the previous reflector (SHARED: the old v_{k-1} buffer takes the next row)
    T* t = vp; vp = vs; vs = t;
    if (SHARED) rk = vs;
    tprev = tk;
    nseg_prev = nseg;
  }
  // the last 2 x 2 block after the last column's update; v of the last column into its row
  if (n >= 3 && k0 + 2 < n) {
    form_w(2, n - 3);
    if (blockIdx.x == 0)
      for (int64_t j = threadIdx.x; j < 2; j += blockDim.x) A[(n - 3) * n + n - 2 + j] = vp[j];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n >= 2) {
      const bool upd = (n >= 3) && (k0 + 2 < n) && (tprev != T(0));
      T a00 = __ldcg(A + (n - 2) * n + n - 2), a01 = __ldcg(A + (n - 2) * n + n - 1),
        a11 = __ldcg(A + (n - 1) * n + n - 1);
      if (upd) {
        a00 = a00 - T(2) * vp[0] * ws[0];
        a01 = a01 - vp[0] * ws[1] - ws[0] * vp[1];
        a11 = a11 - T(2) * vp[1] * ws[1];
      }
      d[n - 2] = a00;
      e[n - 2] = a01;
      tau[n - 2] = T(0);
      d[n - 1] = a11;
    } else {
      d[n - 1] = __ldcg(A + (n - 1) * n + n - 1);
    }
  }
}

// Blocked Householder tridiagonalisation (Dongarra, Sorensen & Hammarling, "Block
// reduction of matrices to condensed forms for eigenvalue computations", J. Comput.
// Appl. Math. 27, 1989): one cooperative launch reduces a panel of nb columns
// k0 .. k0+nb-1 without updating the trailing matrix A0.  With V = [v_0 .. v_{j-1}] and
// W = [w_0 .. w_{j-1}] the panel's reflectors and update vectors so far, the current
// matrix is A0 - V W^T - W V^T, so for column k = k0 + j
//   p = tau (A0 v - V (W^T v) - W (V^T v)),   w = p - (tau/2)(p.v) v,
// and row k+1 of the current matrix is A0's row minus the same sums.  The FP64 pipe does
// the product A0 v (read only, one pass over the trailing matrix) and sums of length
// 2j; the host then applies A0 -= V W^T + W V^T to the rows and columns after the panel
// as one symmetric product of inner dimension 2 nb on the slice GEMM.
//   X: 3 nb vectors of n values: V_t at t n, W_t at (nb + t) n, V_t again at (2 nb + t) n
//      (so that [V W] and [W V] are both nb-strided operands of the product);
//   part: kMaxSeg x (n + 2 nb) segment partials of A0 v (rows 0 .. m-1), V^T v (m ..) and
//      W^T v (m + j ..); bpart: one partial of v.(A0 v) per block;
//   rowbuf: row k+1 (columns k+2 ..) minus the panel's terms before column k, its
//      diagonal at rowbuf[n].
// Two grid barriers per column: after the products, and after w_k and row k+1's partial
// sums are written.  Row k keeps v_k (v_0 = 1 stored) for the back-transformation, as in
// tridiag_kernel.  gen0: the barrier generation at launch (the barrier words persist
// across the panels' launches).
template <int NW>
__global__ void __launch_bounds__(NW * 32)
    tridiag_panel_kernel(double* A, int64_t n, int64_t k0, int nb, double* d, double* e, double* tau, double* X,
                         double* part, double* rowbuf, double* bpart, unsigned* bar, unsigned gen0) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  double* vs = reinterpret_cast<double*>(sm_raw);   // row k, then v_k in place (n values)
  double* yz = vs + n;                              // z_t = V_t.v (t < j), y_t = W_t.v at j + t
  double* vw = yz + 2 * nb;                         // V_t[k+1] (t < nb), W_t[k+1] at nb + t
  double* red = vw + 2 * nb;                        // NW x 32 partial sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * NW + warp, W = (int64_t)gridDim.x * NW;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ps = n + 2 * (int64_t)nb;
  double* Vx = X;
  double* Wx = X + (int64_t)nb * n;
  double* V2 = X + 2 * (int64_t)nb * n;
  unsigned gen = gen0;
  for (int j = 0; j < nb; ++j) {
    const int64_t k = k0 + j, m = n - k - 1;
    // A. row k of the current matrix, then reflector k formed in place (every block)
    double dk;
    if (j == 0) {
      for (int64_t c = threadIdx.x; c < m; c += blockDim.x) vs[c] = __ldcg(A + k * n + k + 1 + c);
      dk = __ldcg(A + k * n + k);
    } else {   // column k-1's term on top of rowbuf: V_{j-1}[k] = 1, W_{j-1}[k] = w_{k-1}[0]
      const double* vq = Vx + (int64_t)(j - 1) * n;
      const double* wq = Wx + (int64_t)(j - 1) * n;
      const double a1 = __ldcg(vq + k), b1 = __ldcg(wq + k);
      for (int64_t c = threadIdx.x; c < m; c += blockDim.x)
        vs[c] = __ldcg(rowbuf + c) - a1 * __ldcg(wq + k + 1 + c) - b1 * __ldcg(vq + k + 1 + c);
      dk = __ldcg(rowbuf + n) - 2.0 * a1 * b1;
    }
    __syncthreads();
    const double alpha = vs[0];
    double sq = 0, z1 = 0, z2 = 0;
    for (int64_t c = 1 + threadIdx.x; c < m; c += blockDim.x) sq = fma(vs[c], vs[c], sq);
    block_sum3n<double, NW>(sq, z1, z2);   // ends with a barrier
    double beta = alpha, tk = 0, scale = 0;
    if (sq > 0.0) {
      beta = -copysign(sqrt(fma(alpha, alpha, sq)), alpha);
      tk = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    for (int64_t c = threadIdx.x; c < m; c += blockDim.x) vs[c] = (c == 0) ? 1.0 : vs[c] * scale;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      d[k] = dk;
      e[k] = beta;
      tau[k] = tk;
    }
    // B. A0 v over rows k+1 .., then V_t.v and W_t.v (t < j): rows of length m, cut
    //    into segments so that every warp has work; lane 0 keeps v.(A0 v) of its rows
    const int64_t rows = m + 2 * (int64_t)j;
    const int64_t nseg = max((int64_t)1, min((int64_t)kMaxSeg, W / rows));
    const int64_t seg = ((m + nseg - 1) / nseg + 31) / 32 * 32;
    double pv = 0;
    for (int64_t task = gw; task < rows * nseg; task += W) {
      const int64_t i = task / nseg, sg = task % nseg;
      const double* row = i < m ? A + (k + 1 + i) * n + k + 1
                                : (i - m < j ? Vx + (i - m) * n + k + 1 : Wx + (i - m - j) * n + k + 1);
      const int64_t j0 = sg * seg, j1 = min(m, j0 + seg);
      double a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = 0;
      int64_t c = j0 + lane;
      for (; c + 224 < j1; c += 256) {
        double r[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) r[u] = __ldcg(row + c + 32 * u);
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = fma(r[u], vs[c + 32 * u], a[u]);
      }
      for (; c < j1; c += 32) a[0] = fma(__ldcg(row + c), vs[c], a[0]);
      double acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        part[sg * ps + i] = acc;
        if (i < m) pv = fma(acc, vs[i], pv);
      }
    }
    z1 = 0;
    z2 = 0;
    block_sum3n<double, NW>(pv, z1, z2);
    if (threadIdx.x == 0) bpart[blockIdx.x] = pv;
    if (!grid_barrier(bar, gridDim.x, gen)) return;
    // C. z, y, v.(A0 v) (every block, fixed order); the panel's V_t[k+1], W_t[k+1]
    if (threadIdx.x < 2 * j) {
      double a = 0;
      for (int64_t sg = 0; sg < nseg; ++sg) a += __ldcg(part + sg * ps + m + threadIdx.x);
      yz[threadIdx.x] = a;
    }
    if (threadIdx.x < j) {
      vw[threadIdx.x] = __ldcg(Vx + (int64_t)threadIdx.x * n + k + 1);
      vw[nb + threadIdx.x] = __ldcg(Wx + (int64_t)threadIdx.x * n + k + 1);
    }
    double pvs = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) pvs += __ldcg(bpart + b);
    z1 = 0;
    z2 = 0;
    block_sum3n<double, NW>(pvs, z1, z2);   // ends with a barrier: yz, vw visible
    double yzs = 0;
    for (int t = 0; t < j; ++t) yzs = fma(yz[t], yz[j + t], yzs);
    // v.w = tau (v.A0 v - 2 y.z);  K = (tau / 2) v.w
    const double K = 0.5 * tk * tk * (pvs - 2.0 * yzs);
    // D. w_k = tau (A0 v - V y - W z) - K v into W, v_k into V, its copy and row k of A;
    //    row k+1 (columns k+2 ..) less the terms of columns before k into rowbuf.  Tasks of
    //    32 consecutive elements per block: warp q sums the terms t = q, q + NW, .. and the
    //    block adds the NW partials in warp order.
    const int64_t nw = (m + 31) / 32, nr = (j + 1 < nb) ? (m - 1 + 31) / 32 : 0;
    for (int64_t task = blockIdx.x; task < nw + nr; task += gridDim.x) {
      const bool isw = task < nw;
      const int64_t g = (isw ? task : task - nw) * 32 + lane, len = isw ? m : m - 1;
      double acc = 0;
      if (g < len) {
        if (isw) {
#pragma unroll 4
          for (int t = warp; t < j; t += NW)
            acc += __ldcg(Vx + (int64_t)t * n + k + 1 + g) * yz[j + t] + __ldcg(Wx + (int64_t)t * n + k + 1 + g) * yz[t];
        } else {
#pragma unroll 4
          for (int t = warp; t < j; t += NW)
            acc += vw[t] * __ldcg(Wx + (int64_t)t * n + k + 2 + g) + vw[nb + t] * __ldcg(Vx + (int64_t)t * n + k + 2 + g);
        }
      }
      red[warp * 32 + lane] = acc;
      __syncthreads();
      if (warp == 0 && g < len) {
        double sacc = 0;
#pragma unroll
        for (int q = 0; q < NW; ++q) sacc += red[q * 32 + lane];
        if (isw) {
          double p = 0;
          for (int64_t sg = 0; sg < nseg; ++sg) p += __ldcg(part + sg * ps + g);
          const double vi = vs[g];
          Wx[(int64_t)j * n + k + 1 + g] = tk * (p - sacc) - K * vi;
          Vx[(int64_t)j * n + k + 1 + g] = vi;
          V2[(int64_t)j * n + k + 1 + g] = vi;
          A[k * n + k + 1 + g] = vi;
        } else {
          rowbuf[g] = __ldcg(A + (k + 1) * n + k + 2 + g) - sacc;
        }
      }
      __syncthreads();
    }
    if (j + 1 < nb && gt == 0) {
      double dd = __ldcg(A + (k + 1) * n + k + 1);
      for (int t = 0; t < j; ++t) dd -= 2.0 * vw[t] * vw[nb + t];
      rowbuf[n] = dd;
    }
    if (!grid_barrier(bar, gridDim.x, gen)) return;
  }
}

// Number of eigenvalues of T (diagonal d, squared off-diagonal e2) below x.
template <typename T>
__device__ int sturm_count(const T* d, const T* e2, int64_t n, T x, T pivmin) {
  int c = 0;
  T q = d[0] - x;
  if (fabs(q) <= pivmin) q = -pivmin;
  if (q < T(0)) ++c;
  for (int64_t i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) <= pivmin) q = -pivmin;
    if (q < T(0)) ++c;
  }
  return c;
}

// The same count without a division per step (FP64 division is a sequence of several
// instructions on the narrow FP64 pipe): the leading principal minors of T - x I,
//   p_i = (d_i - x) p_{i-1} - e2_{i-1} p_{i-2},   p_{-1} = 1,   p_{-2} = 0,
// have the pivots above as ratios, q_i = p_i / p_{i-1}, so a negative pivot is a sign
// change between consecutive minors (Sturm's theorem in the form of Golub & Van Loan,
// Sec. 8.4.1).  A minor that is exactly zero stands for a negative pivot of magnitude
// 2^-600 (the guard above, far below any pivot that T's scale produces), so no minor is
// ever zero; the pair (p_i, p_{i-1}) is scaled by a power of two (exact) whenever p_i's
// exponent leaves [-256, 256].  Signs and exponents are read from the bit patterns.
__device__ int sturm_count_minors(const double* d, const double* e2, int64_t n, double x) {
  int c = 0;
  double pm = 1.0;       // p_{i-1}
  double p = d[0] - x;   // p_0
  if (p == 0.0) p = -0x1p-600;
  c += (__double_as_longlong(p) < 0);
  for (int64_t i = 1; i < n; ++i) {
    double pn = fma(d[i] - x, p, -e2[i - 1] * pm);
    if (pn == 0.0) pn = -p * 0x1p-600;
    c += ((__double_as_longlong(pn) ^ __double_as_longlong(p)) < 0);
    pm = p;
    p = pn;
    const int ex = (int)((__double_as_longlong(p) >> 52) & 0x7FF) - 1023;
    if (ex > 256 || ex < -256) {
      const double sc = __longlong_as_double((long long)(1023 - ex) << 52);   // 2^-ex, a normal double
      p *= sc;
      pm *= sc;
    }
  }
  return c;
}

// lam[j] = the j-th smallest eigenvalue (j = 0..n-1) by bisection of [gl, gu]
// down to abstol or adjacent doubles (at most 128 halvings).
template <typename T>
__global__ void bisect_kernel(const T* d, const T* e2, int64_t n, T gl, T gu, T pivmin, T abstol, T* lam) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    T lo = gl, hi = gu;
    for (int it = 0; it < 128; ++it) {
      const T mid = T(0.5) * (lo + hi);
      if (!(mid > lo && mid < hi) || hi - lo <= abstol) break;
      if (sturm_count(d, e2, n, mid, pivmin) > j) hi = mid;
      else lo = mid;
    }
    lam[j] = T(0.5) * (lo + hi);
  }
}

// Multisection: a group of G lanes (G divides 32) per eigenvalue j probes G
// points splitting [lo, hi] into G + 1 equal parts; the Sturm counts (warp ballot)
// select the part that holds the j-th smallest eigenvalue.  Same result as
// bisection (down to abstol or adjacent floating-point values) in
// log_{G+1} instead of log_2 steps.  Eigenvalues j0 .. j1-1 of T (order n).
template <typename T, int G>
__global__ void __launch_bounds__(256) multisect_kernel(const T* d, const T* e2, int64_t n, T gl, T gu, T pivmin,
                                                        T abstol, T* lam, int64_t j0, int64_t j1) {
  const int lane = threadIdx.x & 31, grp = lane / G, sub = lane % G;
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t j = j0 + warp_id * (32 / G) + grp;   // eigenvalues j0 .. j1-1 of the n
  T lo = gl, hi = gu;
  bool done = (j >= j1);
  for (int it = 0; it < 64; ++it) {
    if (!done) {
      const T mid = T(0.5) * (lo + hi);
      if (!(mid > lo && mid < hi) || hi - lo <= abstol) done = true;
    }
    if (__all_sync(0xffffffffu, done)) break;
    const T x = lo + (hi - lo) * (T)(sub + 1) / (T)(G + 1);
    int cnt = 0;
    if (!done) {
      if constexpr (sizeof(T) == 8) cnt = sturm_count_minors(d, e2, n, x);
      else cnt = sturm_count(d, e2, n, x, pivmin);
    }
    const bool above = done ? false : (cnt > j);
    const unsigned ball = __ballot_sync(0xffffffffu, above);
    if (!done) {
      const unsigned gm = (G == 32) ? ball : ((ball >> (grp * G)) & ((1u << G) - 1u));
      const int first = gm ? (__ffs(gm) - 1) : G;   // first probe above the eigenvalue
      const T nlo = (first == 0) ? lo : lo + (hi - lo) * (T)first / (T)(G + 1);
      const T nhi = (first == G) ? hi : lo + (hi - lo) * (T)(first + 1) / (T)(G + 1);
      if (!(nlo >= lo && nhi <= hi && nlo < nhi)) done = true;
      else { lo = nlo; hi = nhi; }
    }
  }
  if (j < j1 && sub == 0) lam[j] = T(0.5) * (lo + hi);
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
// out [i * nv + t] so that a warp's accesses are contiguous.  The factors stay in
// the scratch arrays (further solves: tri_solve).
#define S(a, i) a[(int64_t)(i) * nv + t]

template <typename T>
__device__ void tri_solve(int64_t n, int64_t nv, int64_t t, const T* sdd, const T* sdu, const T* sdu2, const T* sdl,
                          const unsigned char* spiv, T* z, int64_t ldz) {
  // L: the running value stays in a register; the loads do not depend on it
  T carry = z[0];
#pragma unroll 4
  for (int64_t i = 0; i + 1 < n; ++i) {
    T bn = z[(i + 1) * ldz];
    if (S(spiv, i)) { const T tmp = carry; carry = bn; bn = tmp; }
    z[i * ldz] = carry;
    carry = bn - S(sdl, i) * carry;
  }
  z[(n - 1) * ldz] = carry;
  // U (sdd holds the reciprocals of the pivots)
  T v1 = 0, v2 = 0;
#pragma unroll 4
  for (int64_t i = n - 1; i >= 0; --i) {
    T v = z[i * ldz];
    if (i + 1 < n) v -= S(sdu, i) * v1;
    if (i + 2 < n) v -= S(sdu2, i) * v2;
    v *= S(sdd, i);
    z[i * ldz] = v;
    v2 = v1;
    v1 = v;
  }
}

template <typename T>
__device__ void normalise_col(int64_t n, T* z, int64_t ldz) {
  T mx = 0;
  for (int64_t i = 0; i < n; ++i) mx = fmax(mx, fabs(z[i * ldz]));
  if (!(mx > T(0)) || !isfinite(mx)) mx = T(1);
  const T rmx = T(1) / mx;   // one division: the scaled sum of squares only guards the range
  T nrm = 0;
  for (int64_t i = 0; i < n; ++i) {
    const T v = z[i * ldz] * rmx;
    nrm = fma(v, v, nrm);
  }
  const T inv = T(1) / (mx * sqrt(nrm));
  for (int64_t i = 0; i < n; ++i) z[i * ldz] *= inv;
}

template <typename T>
__global__ void inverse_iteration_kernel(const T* d, const T* e, int64_t n, const T* shift, int64_t j0, int64_t nv,
                                         T pert, T* sdd, T* sdu, T* sdu2, T* sdl, unsigned char* spiv, T* Z,
                                         int64_t ldz, int64_t zc0) {
  constexpr int kInvIters = 3;   // fewer leave the refinement's start too rough (more Rayleigh-Ritz work)
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nv) return;
  const int64_t j = j0 + t;
  const T lam = shift[j];
  for (int64_t i = 0; i < n; ++i) {
    S(sdd, i) = d[i] - lam;
    if (i + 1 < n) { S(sdu, i) = e[i]; S(sdl, i) = e[i]; }
    S(sdu2, i) = T(0);
  }
  // one division per step: each pivot's reciprocal (pivots below pert in magnitude moved
  // out to +-pert) is stored in place of the pivot and gives the multiplier as well
  auto recip = [&](T piv) { return T(1) / ((fabs(piv) < pert) ? copysign(pert, piv) : piv); };
  for (int64_t i = 0; i + 1 < n; ++i) {
    const T di = S(sdd, i), li = S(sdl, i);
    if (fabs(di) >= fabs(li)) {
      const T rp = recip((di == T(0)) ? pert : di);
      S(sdd, i) = rp;
      const T f = li * rp;
      S(sdl, i) = f;
      S(sdd, i + 1) = S(sdd, i + 1) - f * S(sdu, i);
      S(spiv, i) = 0;
    } else {
      const T rp = recip(li);
      const T f = di * rp;
      S(sdd, i) = rp;
      S(sdl, i) = f;
      const T u = S(sdu, i);
      S(sdu, i) = S(sdd, i + 1);
      S(sdd, i + 1) = u - f * S(sdd, i + 1);
      if (i + 2 < n) {
        S(sdu2, i) = S(sdu, i + 1);
        S(sdu, i + 1) = -f * S(sdu, i + 1);
      }
      S(spiv, i) = 1;
    }
  }
  S(sdd, n - 1) = recip(S(sdd, n - 1));   // the solves multiply by the reciprocal pivots
  T* z = Z + (j - zc0);   // vector j in column j - zc0 of Z
  for (int64_t i = 0; i < n; ++i) z[i * ldz] = (T)start_component(i, j);
  for (int it = 0; it < kInvIters; ++it) {
    tri_solve<T>(n, nv, t, sdd, sdu, sdu2, sdl, spiv, z, ldz);
    normalise_col<T>(n, z, ldz);
  }
}

// Clusters of close eigenvalues (block q: columns c0[2q] .. c0[2q+1]-1 of Z):
// modified Gram-Schmidt of the cluster's columns, twice.  Inverse iteration
// returns nearly parallel vectors for eigenvalues closer than its working
// accuracy, but from independent random starts they still span the cluster's
// invariant subspace; the refinement that follows resolves the rest.
template <typename T>
__global__ void __launch_bounds__(256) cluster_orth_kernel(const int32_t* c0, int64_t n, int64_t nv, const T* sdd,
                                                           const T* sdu, const T* sdu2, const T* sdl,
                                                           const unsigned char* spiv, T* Z, int64_t ldz) {
  __shared__ T h[kClusterMax];
  __shared__ T red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t a = c0[2 * blockIdx.x], b = c0[2 * blockIdx.x + 1];
  if (a < 0 || b > n || b - a > kClusterMax) return;   // the host never sends such a cluster
  auto gram_schmidt = [&]() {
    for (int pass = 0; pass < 2; ++pass)
      for (int64_t k = a; k < b; ++k) {
        T* zk = Z + k;
        // h_j = z_j . z_k for the earlier columns of the cluster (a warp per column)
        for (int64_t jj = a + warp; jj < k; jj += 8) {
          const T* zj = Z + jj;
          T acc = 0;
          for (int64_t i = lane; i < n; i += 32) acc = fma(zj[i * ldz], zk[i * ldz], acc);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) h[jj - a] = acc;
        }
        __syncthreads();
        T nrm = 0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
          T v = zk[i * ldz];
          for (int64_t jj = a; jj < k; ++jj) v -= h[jj - a] * Z[i * ldz + jj];
          zk[i * ldz] = v;
          nrm = fma(v, v, nrm);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        if (lane == 0) red[warp] = nrm;
        __syncthreads();
        T tot = 0;
        for (int w = 0; w < 8; ++w) tot += red[w];
        const T inv = (tot > T(0)) ? T(1) / sqrt(tot) : T(0);
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) zk[i * ldz] *= inv;
        __syncthreads();
      }
  };
  gram_schmidt();
}
#undef S

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
// T lives in shared memory; four threads share each row's dot product.
__global__ void __launch_bounds__(256) wy_t_kernel(const double* S, const double* tau, int64_t kb, double* T) {
  __shared__ double sT[kWYBlock][kWYBlock + 1];
  for (int e = threadIdx.x; e < kWYBlock * (kWYBlock + 1); e += blockDim.x) (&sT[0][0])[e] = 0.0;
  __syncthreads();
  const int r = threadIdx.x >> 2, q = threadIdx.x & 3;
  for (int i = 0; i < (int)kb; ++i) {
    const double ti = __ldg(tau + i);
    double acc = 0.0;
    if (r < i)
      for (int c = r + q; c < i; c += 4) acc = fma(sT[r][c], __ldg(S + (int64_t)c * kb + i), acc);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (r < i && q == 0) sT[r][i] = -ti * acc;
    if (threadIdx.x == 0) sT[i][i] = ti;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) T[e] = sT[e / kb][e % kb];
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

// Z <- Q Z for Q = H_0 ... H_{n-3} (reflector k stored in row k of A from column
// k+1 on, v_0 = 1; tau on the device), blocks of kWYBlock reflectors from the
// last to the first in the compact WY form I - V T V^T.  mixed: the two large
// products of each block at FP32 level.
void wy_back_transform(const double* A, const double* tau, int64_t n, double* Z, bool mixed, cudaStream_t s,
                       int64_t nz = 0) {
  // Z: n rows x nz columns (row-major, leading dimension nz)
  if (nz <= 0) nz = n;
  const int64_t nrefl = n - 2;
  if (nrefl < 1) return;
  DBuf<double> Vb((size_t)(n - 1) * kWYBlock, s), S((size_t)kWYBlock * kWYBlock, s),
      T((size_t)kWYBlock * kWYBlock, s), W1((size_t)kWYBlock * nz, s), W2((size_t)kWYBlock * nz, s);
  for (int64_t k0 = ((nrefl - 1) / kWYBlock) * kWYBlock; k0 >= 0; k0 -= kWYBlock) {
    const int64_t kb = std::min<int64_t>(kWYBlock, nrefl - k0), nr = n - k0 - 1;
    wy_vectors_kernel<<<grid_for(nr * kb), 256, 0, s>>>(A, n, k0, kb, Vb.get());
    FTT_LAUNCH();
    FTT_CUDA(cudaMemsetAsync(S.get(), 0, sizeof(double) * kb * kb, s));
    wy_gram_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nr, 64), kNumSMs)), 256, 0, s>>>(
        Vb.get(), nr, kb, S.get());
    FTT_LAUNCH();
    wy_t_kernel<<<1, 256, 0, s>>>(S.get(), tau + k0, kb, T.get());
    FTT_LAUNCH();
    double* Zs = Z + (k0 + 1) * nz;
    gemm(mixed, kb, nz, nr, 1.0, Vb.get(), 1, kb, Zs, nz, 1, 0.0, W1.get(), nz, 1, s);   // V^T Z
    gemm_f64(kb, nz, kb, 1.0, T.get(), kb, 1, W1.get(), nz, 1, 0.0, W2.get(), nz, 1, s);  // T (V^T Z)
    gemm(mixed, nr, nz, kb, -1.0, Vb.get(), kb, 1, W2.get(), nz, 1, 1.0, Zs, nz, 1, s);  // Z -= V T V^T Z
  }
}

// max |x| over n doubles (sign-cleared bit patterns, atomic max; *out zeroed by the caller)
__global__ void absmax_bits_kernel(const double* x, int64_t n, unsigned long long* out) {
  unsigned long long m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)__double_as_longlong(x[i]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, (unsigned long long)__shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__global__ void scale_to_f32_kernel(const double* a, int64_t n, double sc, float* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)(a[i] * sc);
}

__global__ void f32_to_f64_kernel(const float* a, int64_t n, double* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

__global__ void identity64_kernel(double* V, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x)
    V[e] = (e / n == e % n) ? 1.0 : 0.0;
}

}  // namespace

bool sym_eig_tridiag(const double* G, int n, double* V, std::vector<double>& lam_out, cudaStream_t s, bool mixed,
                     const std::function<int64_t(const std::vector<double>&)>& need, int64_t kmax) {
  if (n < 3) return false;
  int dev = 0, coop = 0, sms = 0, smem_max = 0;
  FTT_CUDA(cudaGetDevice(&dev));
  FTT_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  FTT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  FTT_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (!coop) return false;
  const int64_t nn = (int64_t)n * n;
  DBuf<double> A(nn, s), d(n, s), e(n, s), tau(n, s);
  FTT_CUDA(cudaMemcpyAsync(A.get(), G, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  constexpr int NW = TridiagWarps<double>::value;
  // 1a. panels of kPanel columns (blocked), while the matrix after a panel keeps at least
  //     kPanelTail rows; the symmetric rank-2 kPanel update of each panel on the GEMMs
  int64_t kb = 0;
  if (n >= kPanel + kPanelTail) {
    const size_t smem_p = sizeof(double) * ((size_t)n + 4 * kPanel + 32 * NW);
    if (smem_p + 4096 > (size_t)smem_max) return false;
    FTT_CUDA(cudaFuncSetAttribute(tridiag_panel_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_max - 4096));
    int per = 0;
    FTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tridiag_panel_kernel<NW>, 32 * NW, smem_p));
    const int grid = std::min(2, per) * sms;
    if (grid < 1) return false;
    const int64_t ps = n + 2 * kPanel;
    DBuf<double> X(3 * kPanel * (int64_t)n, s), part(kMaxSeg * ps, s), rowbuf(n + 1, s), bpart(grid, s);
    DBuf<unsigned> bar(4, s);
    barrier_init_kernel<<<1, 1, 0, s>>>(bar.get(), barrier_spins());
    FTT_LAUNCH();
    unsigned gen0 = 0;
    int nbp = kPanel;
    int64_t n64 = n;
    double *Ap = A.get(), *dp = d.get(), *ep = e.get(), *tp = tau.get(), *Xp = X.get(), *pp = part.get(),
           *rp = rowbuf.get(), *bp = bpart.get();
    unsigned* brp = bar.get();
    for (; n - kb - kPanel >= kPanelTail; kb += kPanel) {
      int64_t k0 = kb;
      void* args[] = {(void*)&Ap, (void*)&n64, (void*)&k0, (void*)&nbp, (void*)&dp, (void*)&ep, (void*)&tp,
                      (void*)&Xp, (void*)&pp, (void*)&rp, (void*)&bp, (void*)&brp, (void*)&gen0};
      double work = 0.0;   // A0 v: 2 m^2; V^T v, W^T v, w and the next row: 12 j m
      for (int j = 0; j < kPanel; ++j) {
        const double m = (double)(n - kb - j - 1);
        work += 2.0 * m * m + 12.0 * j * m;
      }
      KClock clk;
      kclock_begin(clk, KC_TRIDIAG, s);
      const cudaError_t err = cudaLaunchCooperativeKernel((void*)tridiag_panel_kernel<NW>, dim3(grid),
                                                          dim3(32 * NW), args, smem_p, s);
      if (err != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      FTT_LAUNCH();
      kclock_end(clk, work, s);
      gen0 += 2 * kPanel;
      const int64_t k1 = kb + kPanel, M = n - k1;
      // A0[k1:, k1:] -= [V W] [W V]^T  (rows k1 .. of the panel's vectors)
      gemm_f64(M, M, 2 * kPanel, -1.0, Xp + k1, 1, n, Xp + kPanel * n64 + k1, n, 1, 1.0, Ap + k1 * n64 + k1, n, 1,
               s, true);
    }
    unsigned hb[4];
    FTT_CUDA(cudaMemcpyAsync(hb, bar.get(), sizeof(hb), cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    if (hb[2] != 0) {   // a grid barrier gave up: fail with an explicit bound, else the next route
      note_wait_timeout();
      if (max_spin() > 0) fail(FASTTT_ETIMEOUT, "a grid barrier of the tridiagonalisation exceeded max_spin polls");
      return false;
    }
  }
  // 1b. the remaining columns kb .. n-3 unblocked: four vectors of n - kb values in shared
  //     memory when they fit, three (row and reflector shared) otherwise
  {
    const size_t cap = (size_t)(n - kb);
    const bool shared_rk = 4 * sizeof(double) * cap + 4096 > (size_t)smem_max;
    const size_t smem = (shared_rk ? 3 : 4) * sizeof(double) * cap;
    if (smem + 4096 > (size_t)smem_max) return false;
    DBuf<double> p((size_t)2 * kMaxSeg * n, s);
    void* fn = shared_rk ? (void*)tridiag_kernel<double, NW, true> : (void*)tridiag_kernel<double, NW, false>;
    // the route's whole budget (not this call's need), so that concurrent callers never lower it
    FTT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max - 4096));
    int per = 0;
    FTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 32 * NW, smem));
    const int grid = std::min(2, per) * sms;
    if (grid < 1) return false;
    DBuf<unsigned> bar(4, s);
    barrier_init_kernel<<<1, 1, 0, s>>>(bar.get(), barrier_spins());
    FTT_LAUNCH();
    int64_t n64 = n, k0 = kb;
    double *Ap = A.get(), *dp = d.get(), *ep = e.get(), *tp = tau.get(), *pp = p.get();
    unsigned* bp = bar.get();
    void* args[] = {(void*)&Ap, (void*)&n64, (void*)&k0, (void*)&dp, (void*)&ep, (void*)&tp, (void*)&pp, (void*)&bp};
    KClock clk;
    kclock_begin(clk, KC_TRIDIAG, s);
    const cudaError_t err = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(32 * NW), args, smem, s);
    if (err != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    FTT_LAUNCH();
    const double mt = (double)(n - kb);
    kclock_end(clk, 2.0 * mt * mt * mt, s);   // symv 2m^2 + rank-2 4m^2 per column
    unsigned hb[4];
    FTT_CUDA(cudaMemcpyAsync(hb, bar.get(), sizeof(hb), cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    if (hb[2] != 0) {
      note_wait_timeout();
      if (max_spin() > 0) fail(FASTTT_ETIMEOUT, "a grid barrier of the tridiagonalisation exceeded max_spin polls");
      return false;
    }
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
  // all eigenvalues, or (kmax) the kmax largest: indices j0 .. n-1 of the ascending order
  const bool partial = need && kmax > 0 && kmax + 8 < n;
  int64_t j0 = partial ? n - kmax : 0;
  auto multisect = [&](int64_t a, int64_t b) {   // eigenvalues a .. b-1
    if (b <= a) return;
    multisect_kernel<double, 8><<<(unsigned)ceil_div(b - a, 32), 256, 0, s>>>(d.get(), e2.get(), n, gl, gu, pivmin,
                                                                            abstol, lam.get(), a, b);
    FTT_LAUNCH();
  };
  multisect(j0, n);
  std::vector<double> hl(n);
  FTT_CUDA(cudaMemcpyAsync(hl.data() + j0, lam.get() + j0, sizeof(double) * (n - j0), cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  if (j0 > 0) {   // the j0 smallest: their mean from the trace (sum of G's diagonal)
    std::vector<double> gd(n);
    FTT_CUDA(cudaMemcpy2DAsync(gd.data(), sizeof(double), G, sizeof(double) * ((size_t)n + 1), sizeof(double), n,
                               cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    double trace = 0.0, top = 0.0;
    for (int i = 0; i < n; ++i) trace += gd[i];
    for (int64_t j = j0; j < n; ++j) top += hl[j];
    const double mean = std::min((trace - top) / (double)j0, hl[j0]);
    for (int64_t j = 0; j < j0; ++j) hl[j] = mean;
  }
  // eigenvectors wanted: the kv largest (all unless the caller needs fewer)
  int64_t kv = need ? std::max<int64_t>(1, std::min<int64_t>(n, need(hl))) : n;
  if (kv > n - j0) {   // more than were computed: the rest, and the decision again
    multisect(0, j0);
    FTT_CUDA(cudaMemcpyAsync(hl.data(), lam.get(), sizeof(double) * j0, cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    j0 = 0;
    kv = std::max<int64_t>(1, std::min<int64_t>(n, need(hl)));
  }
  const int64_t v0 = n - kv;   // eigenvalues ascending: vectors v0 .. n-1
  // shifts for inverse iteration: eigenvalues closer than sep are moved apart (only the
  // computed ones: the mean that stands in for the others is no shift)
  const double sep = 16.0 * 0x1p-53 * tnorm;
  std::vector<double> hs(hl);
  for (int64_t i = std::max<int64_t>(1, j0 + 1); i < n; ++i)
    if (hs[i] - hs[i - 1] < sep) hs[i] = hs[i - 1] + sep;
  FTT_CUDA(cudaMemcpyAsync(shift.get(), hs.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  // 3. eigenvectors of T (Z: n x kv, column c = vector v0 + c), in batches bounding the scratch
  const int64_t nk = (int64_t)n * kv;
  DBuf<double> Z(nk, s);
  {
    const int64_t batch = std::max<int64_t>(1, std::min<int64_t>(kv, (int64_t)(2.0e9 / (33.0 * n))));
    DBuf<double> sdd(n * batch, s), sdu(n * batch, s), sdu2(n * batch, s), sdl(n * batch, s);
    DBuf<unsigned char> spiv(n * batch, s);
    const double pert = 0x1p-53 * std::max(tnorm, 1e-300);
    for (int64_t j0 = v0; j0 < n; j0 += batch) {
      const int64_t nv = std::min<int64_t>(batch, n - j0);
      inverse_iteration_kernel<<<(unsigned)ceil_div(nv, 32), 32, 0, s>>>(
          d.get(), e.get(), n, shift.get(), j0, nv, pert, sdd.get(), sdu.get(), sdu2.get(), sdl.get(), spiv.get(),
          Z.get(), kv, v0);
      FTT_LAUNCH();
    }
  }
  kclock_end(clk2, 0.0, s);
  // 4. orthonormalise Z's columns in FP64
  {
    const int64_t kk = kv * kv;
    DBuf<double> R(kk, s), Z0(nk, s);
    bool ok = false;
    for (int it = 0; it < 4; ++it) {
      gemm_f64(kv, kv, n, 1.0, Z.get(), 1, kv, Z.get(), kv, 1, 0.0, R.get(), kv, 1, s, true);   // Z^T Z
      i_minus_sym_kernel<<<grid_for(kk), 256, 0, s>>>(R.get(), kv);
      FTT_LAUNCH();
      const double rF = sqrt(frob2(R.get(), kk, s));
      if (!(rF < 0.5)) break;
      // 4 n u: the eigenvectors' orthogonality bound is 8 n u, and the back-transformation adds to it
      if (rF <= 4.0 * (double)n * 0x1p-53) { ok = true; break; }
      FTT_CUDA(cudaMemcpyAsync(Z0.get(), Z.get(), sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
      gemm_f64(n, kv, kv, 0.5, Z0.get(), kv, 1, R.get(), kv, 1, 1.0, Z.get(), kv, 1, s);   // Z += Z R / 2
      ok = (it == 3);
    }
    if (!ok) return false;
  }
  // 5. X = Q Z; V row j = eigenvector j (rows of the vectors not computed are zero)
  wy_back_transform(A.get(), tau.get(), n, Z.get(), mixed, s, kv);
  if (kv < n) FTT_CUDA(cudaMemsetAsync(V, 0, sizeof(double) * n * v0, s));
  transpose_f64(Z.get(), n, kv, V + v0 * n, s);
  lam_out = hl;
  return true;
}


bool sym_eig_start_f32(const double* G, int n, double* V, std::vector<double>& lam_out, cudaStream_t s) {
  if (n < 3) return false;
  int dev = 0, coop = 0, sms = 0, smem_max = 0;
  FTT_CUDA(cudaGetDevice(&dev));
  FTT_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  FTT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  FTT_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t smem = 4 * sizeof(float) * (size_t)n;
  const int64_t nn = (int64_t)n * n;
  // every vector's tridiagonal factors are kept for the cluster iterations: 17 n^2 bytes
  if (!coop || smem + 4096 > (size_t)smem_max || 17.0 * (double)nn > 6.0e9) return false;
  // 0. G scaled by a power of two to max |g_ij| in [1/2, 1) (exact), rounded to FP32
  double sc = 1.0;
  {
    DBuf<unsigned long long> mx(1, s);
    FTT_CUDA(cudaMemsetAsync(mx.get(), 0, sizeof(unsigned long long), s));
    absmax_bits_kernel<<<grid_for(nn), 256, 0, s>>>(G, nn, mx.get());
    FTT_LAUNCH();
    const unsigned long long bits = read_scalar(mx.get(), s);
    double gmax;
    std::memcpy(&gmax, &bits, sizeof(gmax));
    if (!(gmax > 0.0)) {   // the zero matrix: V = I, all eigenvalues 0
      identity64_kernel<<<grid_for(nn), 256, 0, s>>>(V, n);
      FTT_LAUNCH();
      lam_out.assign(n, 0.0);
      return true;
    }
    int eg = 0;
    std::frexp(gmax, &eg);
    sc = std::ldexp(1.0, -eg);
  }
  DBuf<float> A(nn, s), d(n, s), e(n, s), tau(n, s), p((size_t)2 * kMaxSeg * n, s);
  scale_to_f32_kernel<<<grid_for(nn), 256, 0, s>>>(G, nn, sc, A.get());
  FTT_LAUNCH();
  // 1. FP32 tridiagonalisation
  {
    // the route's whole budget (not this call's need), so that concurrent callers never lower it
    FTT_CUDA(cudaFuncSetAttribute(tridiag_kernel<float, TridiagWarps<float>::value, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_max - 4096));
    int per = 0;
    FTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tridiag_kernel<float, TridiagWarps<float>::value, false>,
                                                           32 * TridiagWarps<float>::value, smem));
    const int grid = std::min(2, per) * sms;
    if (grid < 1) return false;
    DBuf<unsigned> bar(4, s);
    barrier_init_kernel<<<1, 1, 0, s>>>(bar.get(), barrier_spins());
    FTT_LAUNCH();
    int64_t n64 = n;
    float *Ap = A.get(), *dp = d.get(), *ep = e.get(), *tp = tau.get(), *pp = p.get();
    unsigned* bp = bar.get();
    int64_t k0 = 0;
    void* args[] = {(void*)&Ap, (void*)&n64, (void*)&k0, (void*)&dp, (void*)&ep, (void*)&tp, (void*)&pp, (void*)&bp};
    KClock clk;
    kclock_begin(clk, KC_TRIDIAG32, s);
    const cudaError_t err =
        cudaLaunchCooperativeKernel((void*)tridiag_kernel<float, TridiagWarps<float>::value, false>, dim3(grid),
                                    dim3(32 * TridiagWarps<float>::value), args, smem, s);
    if (err != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    FTT_LAUNCH();
    kclock_end(clk, 2.0 * (double)n * (double)n * (double)n, s);
    unsigned hb[4];
    FTT_CUDA(cudaMemcpyAsync(hb, bar.get(), sizeof(hb), cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    if (hb[2] != 0) {   // a grid barrier gave up: fail with an explicit bound, else the next route
      note_wait_timeout();
      if (max_spin() > 0) fail(FASTTT_ETIMEOUT, "a grid barrier of the tridiagonalisation exceeded max_spin polls");
      return false;
    }
  }
  std::vector<float> hd(n), he(n);
  FTT_CUDA(cudaMemcpyAsync(hd.data(), d.get(), sizeof(float) * n, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaMemcpyAsync(he.data(), e.get(), sizeof(float) * n, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  // 2. eigenvalues of T by FP32 bisection (Gershgorin interval)
  const double u32 = 0x1p-24;
  double gl = INFINITY, gu = -INFINITY, emax2 = 0.0, tnorm = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs((double)he[i - 1]) : 0.0) + (i + 1 < n ? fabs((double)he[i]) : 0.0);
    gl = std::min(gl, (double)hd[i] - r);
    gu = std::max(gu, (double)hd[i] + r);
    tnorm = std::max(tnorm, fabs((double)hd[i]) + r);
    if (i + 1 < n) emax2 = std::max(emax2, (double)he[i] * (double)he[i]);
  }
  if (!std::isfinite(gl) || !std::isfinite(gu) || !(tnorm > 0.0)) return false;
  const double widen = 4.0 * u32 * tnorm * n;
  gl -= widen;
  gu += widen;
  std::vector<float> he2(n, 0.0f);
  for (int i = 0; i + 1 < n; ++i) he2[i] = he[i] * he[i];
  DBuf<float> e2(n, s), lam(n, s), shift(n, s);
  FTT_CUDA(cudaMemcpyAsync(e2.get(), he2.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s));
  KClock clk2;
  kclock_begin(clk2, KC_TDEIG, s);
  const float pivmin = (float)(0x1p-126 * std::max(1.0, emax2));
  multisect_kernel<float, 32><<<(unsigned)ceil_div(n, 8), 256, 0, s>>>(d.get(), e2.get(), n, (float)gl, (float)gu,
                                                                        pivmin, (float)(2.0 * u32 * tnorm), lam.get(), (int64_t)0,
                                                                        (int64_t)n);
  FTT_LAUNCH();
  std::vector<float> hl(n);
  FTT_CUDA(cudaMemcpyAsync(hl.data(), lam.get(), sizeof(float) * n, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  // shifts moved apart by sep; clusters: runs of eigenvalues closer than ctol, whose
  // inverse-iteration vectors are not independent enough to be used one by one
  const float sep = (float)(16.0 * u32 * tnorm);
  const double ctol = 128.0 * u32 * tnorm;
  std::vector<float> hs(hl);
  for (int i = 1; i < n; ++i)
    if (hs[i] - hs[i - 1] < sep) hs[i] = hs[i - 1] + sep;
  std::vector<int32_t> cb;   // cluster bounds: [cb[2q], cb[2q+1])
  for (int i = 0; i < n;) {
    int j = i + 1;
    while (j < n && (double)hl[j] - (double)hl[j - 1] <= ctol) ++j;
    if (j - i > kClusterMax) return false;   // the cluster kernel holds kClusterMax columns
    if (j - i >= 2) {
      cb.push_back(i);
      cb.push_back(j);
    }
    i = j;
  }
  FTT_CUDA(cudaMemcpyAsync(shift.get(), hs.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s));
  // 3. eigenvectors of T: inverse iteration, then subspace iteration on each cluster
  DBuf<float> Z(nn, s);
  {
    DBuf<float> sdd(nn, s), sdu(nn, s), sdu2(nn, s), sdl(nn, s);
    DBuf<unsigned char> spiv(nn, s);
    const float pert = (float)(u32 * tnorm);
    inverse_iteration_kernel<float><<<(unsigned)ceil_div(n, 32), 32, 0, s>>>(
        d.get(), e.get(), n, shift.get(), 0, n, pert, sdd.get(), sdu.get(), sdu2.get(), sdl.get(), spiv.get(),
        Z.get(), n, 0);
    FTT_LAUNCH();
    if (!cb.empty()) {
      DBuf<int32_t> dcb(cb.size(), s);
      FTT_CUDA(cudaMemcpyAsync(dcb.get(), cb.data(), sizeof(int32_t) * cb.size(), cudaMemcpyHostToDevice, s));
      cluster_orth_kernel<float><<<(unsigned)(cb.size() / 2), 256, 0, s>>>(dcb.get(), n, n, sdd.get(), sdu.get(),
                                                                         sdu2.get(), sdl.get(), spiv.get(), Z.get(), n);
      FTT_LAUNCH();
      FTT_CUDA(cudaStreamSynchronize(s));   // cb is host memory read by the copy above
    }
  }
  kclock_end(clk2, 0.0, s);
  // 4. X = Q Z in FP64 storage with FP32-level products
  DBuf<double> A64(nn, s), Z64(nn, s), tau64(n, s);
  f32_to_f64_kernel<<<grid_for(nn), 256, 0, s>>>(A.get(), nn, A64.get());
  FTT_LAUNCH();
  f32_to_f64_kernel<<<grid_for(nn), 256, 0, s>>>(Z.get(), nn, Z64.get());
  FTT_LAUNCH();
  f32_to_f64_kernel<<<grid_for(n), 256, 0, s>>>(tau.get(), n, tau64.get());
  FTT_LAUNCH();
  A.reset();
  Z.reset();
  wy_back_transform(A64.get(), tau64.get(), n, Z64.get(), true, s);
  transpose_f64(Z64.get(), n, n, V, s);   // V: row j = eigenvector j
  lam_out.resize(n);
  for (int i = 0; i < n; ++i) lam_out[i] = (double)hl[i] / sc;
  return true;
}

}  // namespace fasttt
