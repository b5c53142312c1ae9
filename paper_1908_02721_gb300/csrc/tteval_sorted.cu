// TT entry evaluation and its adjoint by index-sorted batched contractions (E3).
//
// Entry formula (Sec. 2.3): a(i) = G_1[i_1] ... G_d[i_d].  With the left partial
// products L_k(e) = G_1[i_1] ... G_k[i_k] (1 x r_k, L_0 = 1) and the right ones
// R_k(e) = G_k[i_k] ... G_d[i_d] (r_{k-1} x 1, R_{d+1} = 1), the adjoint of
// L = sum_e g_e a(i^e) is
//     dL/dG_k[:, i, :] = sum_{e : i_k(e) = i} g_e L_{k-1}(e)^T R_{k+1}(e).
// Per mode k the entries are sorted by i_k (stable radix sort), so the entries of
// one index i form a contiguous run:
//   * L_k = L_{k-1} G_k[i_k] and R_k = G_k[i_k] R_{k+1} are gathered-row GEMMs: a
//     tile of 64 sorted entries mostly shares one slice G_k[:, i, :], which is read
//     once into shared memory for the tile instead of once per entry;
//   * the gradient of slice i is a GEMM over its run (K = the entries): each chunk
//     of at most kChunk entries writes a partial r_{k-1} x r_k product, and a second
//     kernel sums a slice's chunks in a fixed order in FP64 -- no atomics, the same
//     result on every run.
// Stored partials: L_1..L_{d-1} are kept for the backward sweep.  Recompute: only
// every s-th left partial (s = ceil(sqrt(d))) is kept, and the backward sweep
// recomputes one segment of s - 1 partials from its checkpoint when it enters the
// segment, so every L_k is computed twice at most and ~2 sqrt(d) partials are held.
// Entries are processed in chunks that fit half of the free device memory; the
// gradient of a later chunk is added after the earlier one's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace fasttt {
namespace {

constexpr int kTM = 64, kTN = 64, kTK = 16;   // 64 x 64 output tiles, K in steps of 16; 256 threads, 4 x 4 each
constexpr int64_t kChunk = 4096;              // entries per gradient partial (more for large ranks)

#define TS_GRID_STRIDE(i, n)                                                       \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

// err <- 1 if any index of the (d, m) SoA array is outside [0, n_k)
__global__ void check_index_kernel(const int32_t* idx, int64_t m, int64_t ld, int d, const int32_t* dims,
                                   unsigned* err) {
  TS_GRID_STRIDE(q, (int64_t)d * m) {
    const int k = (int)(q / m);
    const int32_t i = idx[(int64_t)k * ld + q % m];
    if (i < 0 || i >= dims[k]) atomicOr(err, 1u);
  }
}

__global__ void make_keys_kernel(const int32_t* idx_k, int64_t m, uint64_t* keys, uint32_t* vals) {
  TS_GRID_STRIDE(j, m) {
    keys[j] = (uint64_t)(uint32_t)idx_k[j];
    vals[j] = (uint32_t)j;
  }
}

// sorted keys -> int32, and the [start, end) of every index's run
__global__ void runs_kernel(const uint64_t* keys, int64_t m, int32_t* key32, int64_t* start, int64_t* end) {
  TS_GRID_STRIDE(j, m) {
    const uint64_t k = keys[j];
    key32[j] = (int32_t)k;
    if (j == 0 || keys[j - 1] != k) start[k] = j;
    if (j == m - 1 || keys[j + 1] != k) end[k] = j + 1;
  }
}

// four consecutive shared-memory values (16-byte aligned) as one or two vector loads
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 q0 = *reinterpret_cast<const double2*>(p), q1 = *reinterpret_cast<const double2*>(p + 2);
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

constexpr int kGM = 128;   // sorted rows per propagation tile (8 per thread), kTN columns (4 per thread)

// Out[perm[j], c] = sum_a A[perm[j], a] Bi(a, c) for the kGM sorted rows j of this
// tile, Bi the matrix of row j's index i = key[j]: Bi(a, c) = G[i s_i + a s_k + c s_c].
// A: m x K row-major (a_ones: K = 1 and A = 1).  Out: m x N row-major.  Runs of equal
// keys inside the tile are contracted one after the other (rows outside the run
// contribute zeros).  The next K step's gathered values are loaded into registers
// while the current step is multiplied.
template <typename T>
__global__ void __launch_bounds__(256) gathered_gemm_kernel(const T* __restrict__ A, bool a_ones, int K,
                                                            const T* __restrict__ G, int64_t s_i, int64_t s_k,
                                                            int64_t s_c, int N, const uint32_t* __restrict__ perm,
                                                            const int32_t* __restrict__ key, int64_t m,
                                                            T* __restrict__ Out) {
  __shared__ __align__(16) T As[kTK][kGM + 4];
  __shared__ __align__(16) T Bs[kTK][kTN + 4];
  __shared__ uint32_t rows[kGM];
  __shared__ int32_t keys[kGM];
  const int64_t j0 = (int64_t)blockIdx.x * kGM;
  const int c0 = blockIdx.y * kTN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int nrow = (int)min((int64_t)kGM, m - j0);
  if (threadIdx.x < kGM) {
    const bool in = threadIdx.x < nrow;
    rows[threadIdx.x] = in ? perm[j0 + threadIdx.x] : 0u;
    keys[threadIdx.x] = in ? key[j0 + threadIdx.x] : -1;
  }
  __syncthreads();
  T acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const bool b_k_fast = (s_k == 1);
  // this thread's share of a K step: 8 A values (rows e / kTK, k e % kTK), 4 B values
  T ra[8], rb[4];
  for (int rs = 0; rs < nrow;) {
    const int kc = keys[rs];
    int re = rs + 1;
    while (re < nrow && keys[re] == kc) ++re;
    const T* Gi = G + (int64_t)kc * s_i;
    auto fetch = [&](int a0) {
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int e = threadIdx.x + t * 256;
        const int row = e / kTK, kk = e % kTK;
        T v = T(0);
        if (row >= rs && row < re && a0 + kk < K) v = a_ones ? T(1) : A[(int64_t)rows[row] * K + a0 + kk];
        ra[t] = v;
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int e = threadIdx.x + t * 256;
        int kk, cc;
        if (b_k_fast) { kk = e % kTK; cc = e / kTK; } else { kk = e / kTN; cc = e % kTN; }
        T v = T(0);
        if (a0 + kk < K && c0 + cc < N) v = Gi[(int64_t)(a0 + kk) * s_k + (int64_t)(c0 + cc) * s_c];
        rb[t] = v;
      }
    };
    fetch(0);
    for (int a0 = 0; a0 < K; a0 += kTK) {
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int e = threadIdx.x + t * 256;
        As[e % kTK][e / kTK] = ra[t];
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int e = threadIdx.x + t * 256;
        if (b_k_fast) Bs[e % kTK][e / kTK] = rb[t];
        else Bs[e / kTN][e % kTN] = rb[t];
      }
      __syncthreads();
      if (a0 + kTK < K) fetch(a0 + kTK);   // the next step's loads fly during the products
#pragma unroll
      for (int kk = 0; kk < kTK; ++kk) {
        T av0[4], av1[4], bv[4];
        ld4(&As[kk][ty * 8], av0);
        ld4(&As[kk][ty * 8 + 4], av1);
        ld4(&Bs[kk][tx * 4], bv);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[i][j] = fma(av0[i], bv[j], acc[i][j]);
            acc[i + 4][j] = fma(av1[i], bv[j], acc[i + 4][j]);
          }
        }
      }
      __syncthreads();
    }
    rs = re;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = ty * 8 + i;
    if (row >= nrow) continue;
    T* o = Out + (int64_t)rows[row] * N;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      if (c < N) o[c] = acc[i][j];
    }
  }
}

// partial[ch] (r0 x r1, this block's 64 x 64 tile of it) = sum over the sorted
// positions j in [lo[ch], hi[ch]) of g[perm j] L[perm j]^T R[perm j]
// (l_ones: r0 = 1, L = 1; r_ones: r1 = 1, R = 1).  The next step's gathered rows are
// loaded into registers while the current step is multiplied.
template <typename T>
__global__ void __launch_bounds__(256) grad_chunk_kernel(const T* __restrict__ L, bool l_ones, int r0,
                                                         const T* __restrict__ R, bool r_ones, int r1,
                                                         const T* __restrict__ g, const uint32_t* __restrict__ perm,
                                                         const int64_t* __restrict__ lo,
                                                         const int64_t* __restrict__ hi, T* __restrict__ partial) {
  __shared__ __align__(16) T Ls[kTK][kTM + 4];
  __shared__ __align__(16) T Rs[kTK][kTN + 4];
  const int ch = blockIdx.x;
  const int a0 = blockIdx.y * kTM, c0 = blockIdx.z * kTN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t j_lo = lo[ch], j_hi = hi[ch];
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  // this thread's share of a step: 4 L values and 4 R values (entry q / 64, column q % 64)
  T rl[4], rr[4];
  auto fetch = [&](int64_t j0) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int q = threadIdx.x + t * 256;
      const int kk = q / kTM, col = q % kTM;
      const int64_t j = j0 + kk;
      T lv = T(0), rv = T(0);
      if (j < j_hi) {
        const uint32_t e = perm[j];
        if (a0 + col < r0) lv = l_ones ? T(1) : L[(int64_t)e * r0 + a0 + col];
        if (c0 + col < r1) rv = g[e] * (r_ones ? T(1) : R[(int64_t)e * r1 + c0 + col]);
      }
      rl[t] = lv;
      rr[t] = rv;
    }
  };
  fetch(j_lo);
  for (int64_t j0 = j_lo; j0 < j_hi; j0 += kTK) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int q = threadIdx.x + t * 256;
      Ls[q / kTM][q % kTM] = rl[t];
      Rs[q / kTN][q % kTN] = rr[t];
    }
    __syncthreads();
    if (j0 + kTK < j_hi) fetch(j0 + kTK);
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      T av[4], bv[4];
      ld4(&Ls[kk][ty * 4], av);
      ld4(&Rs[kk][tx * 4], bv);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  T* P = partial + (int64_t)ch * r0 * r1;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty * 4 + i;
    if (a >= r0) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      if (c < r1) P[(int64_t)a * r1 + c] = acc[i][j];
    }
  }
}

// dG[a, i, c] += sum of the partials of index i's chunks (FP64 sum in chunk order)
template <typename T>
__global__ void grad_reduce_kernel(const T* __restrict__ partial, int r0, int r1, int n, int64_t nb,
                                   const int32_t* __restrict__ bucket, const int64_t* __restrict__ first,
                                   const int64_t* __restrict__ count, T* __restrict__ dG) {
  const int64_t per = (int64_t)r0 * r1;
  TS_GRID_STRIDE(q, nb * per) {
    const int64_t b = q / per, ac = q % per;
    const int a = (int)(ac / r1), c = (int)(ac % r1);
    double s = 0.0;
    const int64_t f = first[b], cnt = count[b];
    for (int64_t t = 0; t < cnt; ++t) s += (double)partial[(f + t) * per + ac];
    T* dst = dG + ((int64_t)a * n + bucket[b]) * r1 + c;
    *dst = (T)((double)*dst + s);
  }
}

// ---------------------------------------------------------------- host

// The entries of one chunk sorted by their mode-k index: sorted position -> entry
// (chunk-local), the index at every position, and the run of every index.
struct ModeOrder {
  DBuf<uint32_t> perm;
  DBuf<int32_t> key;
  std::vector<int64_t> start, end;
};

void sort_mode(const int32_t* idx_k, int64_t mc, int32_t n, ModeOrder& mo, uint64_t* k1, uint64_t* k2, uint32_t* v2,
               cudaStream_t s) {
  mo.perm = DBuf<uint32_t>(mc, s);
  mo.key = DBuf<int32_t>(mc, s);
  make_keys_kernel<<<grid_for(mc), 256, 0, s>>>(idx_k, mc, k1, mo.perm.get());
  FTT_LAUNCH();
  radix_sort_pairs(k1, mo.perm.get(), k2, v2, mc, bits_for((uint64_t)n), s);
  DBuf<int64_t> st(n, s), en(n, s);
  FTT_CUDA(cudaMemsetAsync(st.get(), 0, st.bytes(), s));
  FTT_CUDA(cudaMemsetAsync(en.get(), 0, en.bytes(), s));
  runs_kernel<<<grid_for(mc), 256, 0, s>>>(k1, mc, mo.key.get(), st.get(), en.get());
  FTT_LAUNCH();
  mo.start.resize(n);
  mo.end.resize(n);
  FTT_CUDA(cudaMemcpyAsync(mo.start.data(), st.get(), sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaMemcpyAsync(mo.end.data(), en.get(), sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
}

// Out (mc x N) = A (mc x K, or ones) times the slice of every entry's index
template <typename T>
void propagate(const T* A, bool a_ones, int K, const T* G, int64_t s_i, int64_t s_k, int64_t s_c, int N,
               const ModeOrder& mo, int64_t mc, T* Out, cudaStream_t s) {
  const dim3 grid((unsigned)ceil_div(mc, kGM), (unsigned)ceil_div(N, kTN));
  gathered_gemm_kernel<T><<<grid, 256, 0, s>>>(A, a_ones, K, G, s_i, s_k, s_c, N, mo.perm.get(), mo.key.get(), mc,
                                               Out);
  FTT_LAUNCH();
}

// dG[:, i, :] += sum over the entries of index i of g L^T R, by chunks of each run
template <typename T>
void gradient(const T* L, bool l_ones, int r0, const T* R, bool r_ones, int r1, const T* g, const ModeOrder& mo,
              int n, T* dG, cudaStream_t s) {
  const double per = (double)r0 * r1 * sizeof(T);
  int64_t csz = kChunk, total = 0;
  int64_t maxcnt = 0;
  for (int i = 0; i < n; ++i) maxcnt = std::max(maxcnt, mo.end[i] - mo.start[i]);
  for (;;) {   // chunks grow until the partial products fit 1 GiB (or one chunk per index)
    total = 0;
    for (int i = 0; i < n; ++i) total += ceil_div(mo.end[i] - mo.start[i], csz);
    if ((double)total * per <= 1073741824.0 || csz >= maxcnt) break;
    csz *= 2;
  }
  if (total == 0) return;
  if (total > INT32_MAX) fail(FASTTT_ERANK, "adjoint: too many gradient chunks");
  std::vector<int64_t> lo(total), hi(total), first, count;
  std::vector<int32_t> bucket;
  int64_t t = 0;
  for (int i = 0; i < n; ++i) {
    const int64_t a = mo.start[i], b = mo.end[i];
    if (b <= a) continue;
    bucket.push_back(i);
    first.push_back(t);
    count.push_back(ceil_div(b - a, csz));
    for (int64_t j = a; j < b; j += csz, ++t) {
      lo[t] = j;
      hi[t] = std::min(b, j + csz);
    }
  }
  const int64_t nb = (int64_t)bucket.size();
  DBuf<int64_t> dlo(total, s), dhi(total, s), dfirst(nb, s), dcount(nb, s);
  DBuf<int32_t> dbucket(nb, s);
  FTT_CUDA(cudaMemcpyAsync(dlo.get(), lo.data(), sizeof(int64_t) * total, cudaMemcpyHostToDevice, s));
  FTT_CUDA(cudaMemcpyAsync(dhi.get(), hi.data(), sizeof(int64_t) * total, cudaMemcpyHostToDevice, s));
  FTT_CUDA(cudaMemcpyAsync(dfirst.get(), first.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s));
  FTT_CUDA(cudaMemcpyAsync(dcount.get(), count.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s));
  FTT_CUDA(cudaMemcpyAsync(dbucket.get(), bucket.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
  DBuf<T> partial((size_t)total * r0 * r1, s);
  const dim3 grid((unsigned)total, (unsigned)ceil_div(r0, kTM), (unsigned)ceil_div(r1, kTN));
  grad_chunk_kernel<T><<<grid, 256, 0, s>>>(L, l_ones, r0, R, r_ones, r1, g, mo.perm.get(), dlo.get(), dhi.get(),
                                            partial.get());
  FTT_LAUNCH();
  grad_reduce_kernel<T><<<grid_for(nb * r0 * r1), 256, 0, s>>>(partial.get(), r0, r1, n, nb, dbucket.get(),
                                                                dfirst.get(), dcount.get(), dG);
  FTT_LAUNCH();
  // the host vectors above were staged by the copies (pageable sources) before they returned
}

void check_indices(int d, const int64_t* dims, int64_t m, const int32_t* idx, cudaStream_t s) {
  std::vector<int32_t> hd(d);
  for (int k = 0; k < d; ++k) hd[k] = (int32_t)dims[k];
  DBuf<int32_t> dd(d, s);
  DBuf<unsigned> err(1, s);
  FTT_CUDA(cudaMemcpyAsync(dd.get(), hd.data(), sizeof(int32_t) * d, cudaMemcpyHostToDevice, s));
  FTT_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(unsigned), s));
  check_index_kernel<<<grid_for((int64_t)d * m), 256, 0, s>>>(idx, m, m, d, dd.get(), err.get());
  FTT_LAUNCH();
  if (read_scalar(err.get(), s)) fail(FASTTT_EINVAL, "index out of range");
}

// entries per chunk so that the chunk's buffers take at most half of the free memory
int64_t chunk_entries(int64_t m, double bytes_per_entry) {
  size_t fr = 0, tot = 0;
  FTT_CUDA(cudaMemGetInfo(&fr, &tot));
  const double budget = 0.5 * (double)fr;
  int64_t mc = (int64_t)std::floor(budget / std::max(bytes_per_entry, 1.0));
  mc = std::min<int64_t>(mc, (int64_t)UINT32_MAX);
  if (mc < 1) fail(FASTTT_ENOMEM, "adjoint: not enough device memory for one entry's partials");
  return std::min(m, mc);
}

// forward / backward strides of core k (r0 x n x r1, row-major) for propagate
struct CoreView {
  const void* G;
  int n, r0, r1;
};

template <typename T>
void eval_sorted(int d, const std::vector<CoreView>& cv, int64_t m, const int32_t* idx, T* out, cudaStream_t s) {
  int rmax = 1;
  for (const auto& c : cv) rmax = std::max(rmax, std::max(c.r0, c.r1));
  const int64_t mc = chunk_entries(m, 2.0 * rmax * sizeof(T) + 8.0 + 24.0 + 16.0);
  DBuf<uint64_t> k1(mc, s), k2(mc, s);
  DBuf<uint32_t> v2(mc, s);
  DBuf<T> P(mc * rmax, s), Q(mc * rmax, s);
  for (int64_t e0 = 0; e0 < m; e0 += mc) {
    const int64_t mcur = std::min(mc, m - e0);
    T* cur = nullptr;
    for (int k = 0; k < d; ++k) {
      ModeOrder mo;
      sort_mode(idx + (int64_t)k * m + e0, mcur, cv[k].n, mo, k1.get(), k2.get(), v2.get(), s);
      const CoreView& c = cv[k];
      T* dst = (k == d - 1) ? out + e0 : (cur == P.get() ? Q.get() : P.get());
      propagate<T>(cur, k == 0, c.r0, (const T*)c.G, c.r1, (int64_t)c.n * c.r1, 1, c.r1, mo, mcur, dst, s);
      cur = dst;
    }
  }
}

template <typename T>
void backward_sorted(int d, const std::vector<CoreView>& cv, int64_t m, const int32_t* idx, const T* gout,
                     void* const* grads, bool recompute, cudaStream_t s) {
  // left partials kept: all of L_1..L_{d-1}, or every s-th plus one segment of s - 1
  const int seg = recompute ? std::max(1, (int)std::ceil(std::sqrt((double)d))) : 1;
  std::vector<bool> keep(d, false);
  double kept_vals = 0.0;
  int rmax = 1;
  for (int k = 0; k < d; ++k) rmax = std::max(rmax, std::max(cv[k].r0, cv[k].r1));
  for (int k = 1; k < d; ++k) {
    keep[k] = (k % seg == 0);
    if (keep[k]) kept_vals += cv[k].r0;
  }
  const double seg_vals = (seg > 1) ? (double)(seg - 1) * rmax : 0.0;
  const double bpe = sizeof(T) * (kept_vals + seg_vals + 3.0 * rmax) + 8.0 * d + 24.0 + 16.0;
  const int64_t mc = chunk_entries(m, bpe);
  DBuf<uint64_t> k1(mc, s), k2(mc, s);
  DBuf<uint32_t> v2(mc, s);
  for (int64_t e0 = 0; e0 < m; e0 += mc) {
    const int64_t mcur = std::min(mc, m - e0);
    std::vector<ModeOrder> mo(d);
    for (int k = 0; k < d; ++k)
      sort_mode(idx + (int64_t)k * m + e0, mcur, cv[k].n, mo[k], k1.get(), k2.get(), v2.get(), s);
    auto fwd = [&](int k, const T* Lk, T* Lnext) {   // L_{k+1} = L_k G_k[i_k]
      const CoreView& c = cv[k];
      propagate<T>(Lk, k == 0, c.r0, (const T*)c.G, c.r1, (int64_t)c.n * c.r1, 1, c.r1, mo[k], mcur, Lnext, s);
    };
    // forward sweep: L_k (left partial of core k, length r_k = cv[k].r0) for k = 1..d-1
    std::vector<DBuf<T>> L(d);
    {
      DBuf<T> a, b;
      const T* cur = nullptr;
      for (int k = 0; k + 1 < d; ++k) {
        DBuf<T> nxt(mcur * cv[k + 1].r0, s);
        fwd(k, cur, nxt.get());
        if (keep[k + 1]) {
          L[k + 1] = std::move(nxt);
          cur = L[k + 1].get();
        } else {
          a = std::move(nxt);
          std::swap(a, b);
          cur = b.get();
        }
      }
    }
    // backward sweep: R (right partial of core k, length r_{k+1}), gradient of core k
    DBuf<T> Rcur;
    std::vector<DBuf<T>> segL(d);
    for (int k = d - 1; k >= 0; --k) {
      const CoreView& c = cv[k];
      const T* Lk = nullptr;
      if (k > 0) {
        if (keep[k]) {
          Lk = L[k].get();
        } else {
          if (!segL[k].get()) {   // entering a segment: recompute its partials from the checkpoint
            const int c0 = (k / seg) * seg;
            const T* src = (c0 == 0) ? nullptr : L[c0].get();
            for (int j = c0; j < k; ++j) {
              DBuf<T> nxt(mcur * cv[j + 1].r0, s);
              fwd(j, src, nxt.get());
              segL[j + 1] = std::move(nxt);
              src = segL[j + 1].get();
            }
          }
          Lk = segL[k].get();
        }
      }
      gradient<T>(Lk, k == 0, c.r0, Rcur.get(), k == d - 1, c.r1, gout + e0, mo[k], c.n, (T*)grads[k], s);
      segL[k].reset();
      if (keep[k]) L[k].reset();
      if (k > 0) {   // R of core k-1 = G_k[i_k] R
        DBuf<T> Rn(mcur * c.r0, s);
        propagate<T>(Rcur.get(), k == d - 1, c.r1, (const T*)c.G, c.r1, 1, (int64_t)c.n * c.r1, c.r0, mo[k], mcur,
                     Rn.get(), s);
        Rcur = std::move(Rn);
      }
    }
  }
}

}  // namespace

// Whether the index-sorted path takes a TT: ranks from 16 to 1024 (smaller ones are
// cheapest with one thread or warp per entry, larger ones exceed its tiles' reuse)
// and mode sizes up to 2^24 (the runs of every index are kept per mode)
bool tteval_sorted_applies(int d, const int64_t* dims, const int64_t* ranks) {
  int64_t rmax = 1;
  for (int k = 0; k <= d; ++k) rmax = std::max(rmax, ranks[k]);
  for (int k = 0; k < d; ++k)
    if (dims[k] > (1 << 24)) return false;
  return rmax >= 16 && rmax <= 1024;
}

void tt_eval_sorted(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores, int dtype, int64_t m,
                    const int32_t* idx, void* out, cudaStream_t s) {
  check_indices(d, dims, m, idx, s);
  std::vector<CoreView> cv(d);
  for (int k = 0; k < d; ++k) cv[k] = {cores[k], (int)dims[k], (int)ranks[k], (int)ranks[k + 1]};
  if (dtype == FASTTT_F64) eval_sorted<double>(d, cv, m, idx, (double*)out, s);
  else eval_sorted<float>(d, cv, m, idx, (float*)out, s);
}

void tt_backward_sorted(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores, int dtype,
                        int64_t m, const int32_t* idx, const void* gout, void* const* grads, int recompute,
                        cudaStream_t s) {
  check_indices(d, dims, m, idx, s);
  std::vector<CoreView> cv(d);
  for (int k = 0; k < d; ++k) cv[k] = {cores[k], (int)dims[k], (int)ranks[k], (int)ranks[k + 1]};
  if (dtype == FASTTT_F64)
    backward_sorted<double>(d, cv, m, idx, (const double*)gout, grads, recompute != 0, s);
  else
    backward_sorted<float>(d, cv, m, idx, (const float*)gout, grads, recompute != 0, s);
}

}  // namespace fasttt
