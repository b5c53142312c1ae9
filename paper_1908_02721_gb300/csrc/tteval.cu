// TT entry evaluation and its adjoint (E3).
//
// a(i) = G_1[i_1] G_2[i_2] ... G_d[i_d]  (entry formula, Sec. 2.3): one warp per
// entry carries the row vector v (1 x r_k) in shared memory; lane j computes
// v'[b] for b = j, j+32, ... reading the slice rows G_k[a, i_k, :] coalesced.
//
// Adjoint: dG_k[:, i_k, :] += g * L_{k-1}^T R_{k+1} with L the left and R the
// right partial products.  The warp sweeps k = d..1 carrying R; L_{k-1} is either
// read from the warp's stored left partials (recompute = 0: sum_k r_k values per
// warp) or recomputed from G_1..G_{k-1} (recompute = 1: 2 r_max values per warp).
// Updates are atomic adds into the caller's gradient cores.
//
// Small TTs (d <= 8, every rank <= 8) are evaluated with one thread per entry and
// the partial product in registers.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace fasttt {

// The index-sorted batched path (tteval_sorted.cu) for ranks 16..1024.
bool tteval_sorted_applies(int d, const int64_t* dims, const int64_t* ranks);
void tt_eval_sorted(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores, int dtype, int64_t m,
                    const int32_t* idx, void* out, cudaStream_t s);
void tt_backward_sorted(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores, int dtype,
                        int64_t m, const int32_t* idx, const void* gout, void* const* grads, int recompute,
                        cudaStream_t s);

namespace {

constexpr int kMaxWarps = 8;            // warps per block at most
constexpr int64_t kSmemBudget = 200 * 1024;  // dynamic shared memory per block at most
constexpr int kMaxRank = 8192;

struct CoreArgs {
  const void* core[FASTTT_MAX_D];
  void* grad[FASTTT_MAX_D];
  int32_t n[FASTTT_MAX_D];
  int32_t r[FASTTT_MAX_D + 1];
  int64_t off[FASTTT_MAX_D + 1];  // prefix sums of r_k (stored left partials)
};

// v_out (1 x r1) = v_in (1 x r0) * G[:, i, :]
template <typename T>
__device__ __forceinline__ void vec_slice(const T* __restrict__ G, int n, int r0, int r1, int i, const T* v_in,
                                          T* v_out, int lane) {
  for (int b = lane; b < r1; b += 32) {
    T acc = 0;
    const T* col = G + (int64_t)i * r1 + b;
    const int64_t stride = (int64_t)n * r1;
    for (int a = 0; a < r0; ++a) acc = fma(v_in[a], col[a * stride], acc);
    v_out[b] = acc;
  }
  __syncwarp();
}

// u_out (r0) = G[:, i, :] * u_in (r1)
template <typename T>
__device__ __forceinline__ void slice_vec(const T* __restrict__ G, int n, int r0, int r1, int i, const T* u_in,
                                          T* u_out, int lane) {
  for (int a = lane; a < r0; a += 32) {
    const T* row = G + ((int64_t)a * n + i) * r1;
    T acc = 0;
    for (int b = 0; b < r1; ++b) acc = fma(row[b], u_in[b], acc);
    u_out[a] = acc;
  }
  __syncwarp();
}

// dynamic shared memory: per warp 2 vectors of rmax values
template <typename T>
__global__ void __launch_bounds__(kMaxWarps * 32) eval_kernel(int d, CoreArgs ca, int64_t m, const int32_t* idx,
                                                              T* out, unsigned* err, int rmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T* base = reinterpret_cast<T*>(smem_raw) + (int64_t)w * 2 * rmax;
  for (int64_t e = (int64_t)blockIdx.x * nw + w; e < m; e += (int64_t)gridDim.x * nw) {
    bool bad = false;
    for (int k = 0; k < d; ++k) {
      const int32_t i = idx[(int64_t)k * m + e];
      bad |= (i < 0 || i >= ca.n[k]);
    }
    if (bad) {
      if (lane == 0) { atomicOr(err, 1u); out[e] = 0; }
      continue;
    }
    T* v = base;
    T* v2 = base + rmax;
    if (lane == 0) v[0] = 1;
    __syncwarp();
    for (int k = 0; k < d; ++k) {
      const int32_t i = idx[(int64_t)k * m + e];
      vec_slice<T>((const T*)ca.core[k], ca.n[k], ca.r[k], ca.r[k + 1], i, v, v2, lane);
      T* t = v; v = v2; v2 = t;
    }
    if (lane == 0) out[e] = v[0];
    __syncwarp();
  }
}

// dynamic shared memory: per warp 4 vectors of rmax values
template <typename T>
__global__ void __launch_bounds__(kMaxWarps * 32) backward_kernel(int d, CoreArgs ca, int64_t m, const int32_t* idx,
                                                                  const T* gout, int recompute, T* left_store,
                                                                  int64_t left_stride, unsigned* err, int rmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T* base = reinterpret_cast<T*>(smem_raw) + (int64_t)w * 4 * rmax;
  T* Lst = left_store + ((int64_t)blockIdx.x * nw + w) * left_stride;  // per-warp scratch (global)
  for (int64_t e = (int64_t)blockIdx.x * nw + w; e < m; e += (int64_t)gridDim.x * nw) {
    bool bad = false;
    for (int k = 0; k < d; ++k) {
      const int32_t i = idx[(int64_t)k * m + e];
      bad |= (i < 0 || i >= ca.n[k]);
    }
    if (bad) {
      if (lane == 0) atomicOr(err, 1u);
      continue;
    }
    const T g = gout[e];
    T* L = base;
    T* L2 = base + rmax;
    T* R = base + 2 * rmax;
    T* R2 = base + 3 * rmax;
    if (!recompute) {
      // left partials L_0..L_{d-1} into the warp's scratch
      if (lane == 0) Lst[0] = 1;
      __syncwarp();
      for (int k = 0; k < d - 1; ++k) {
        const int32_t i = idx[(int64_t)k * m + e];
        vec_slice<T>((const T*)ca.core[k], ca.n[k], ca.r[k], ca.r[k + 1], i, Lst + ca.off[k], Lst + ca.off[k + 1],
                     lane);
      }
    }
    if (lane == 0) R[0] = 1;
    __syncwarp();
    for (int k = d - 1; k >= 0; --k) {
      const int r0 = ca.r[k], r1 = ca.r[k + 1];
      const int32_t ik = idx[(int64_t)k * m + e];
      const T* Lk;
      if (recompute) {
        if (lane == 0) L[0] = 1;
        __syncwarp();
        for (int j = 0; j < k; ++j) {
          const int32_t ij = idx[(int64_t)j * m + e];
          vec_slice<T>((const T*)ca.core[j], ca.n[j], ca.r[j], ca.r[j + 1], ij, L, L2, lane);
          T* t = L; L = L2; L2 = t;
        }
        Lk = L;
      } else {
        Lk = Lst + ca.off[k];
      }
      T* dG = (T*)ca.grad[k];
      for (int64_t q = lane; q < (int64_t)r0 * r1; q += 32) {
        const int a = (int)(q / r1), b = (int)(q % r1);
        atomicAdd(dG + ((int64_t)a * ca.n[k] + ik) * r1 + b, g * Lk[a] * R[b]);
      }
      __syncwarp();
      if (k > 0) {
        slice_vec<T>((const T*)ca.core[k], ca.n[k], r0, r1, ik, R, R2, lane);
        T* t = R; R = R2; R2 = t;
      }
      if (recompute) {  // restore buffer roles for the next k
        L = base;
        L2 = base + rmax;
      }
    }
  }
}

// ---- small TTs (d <= kSmallD, every rank <= kSmallR): entry evaluation with one
// thread per entry and the running row vector in registers.
constexpr int kSmallD = 8, kSmallR = 8;

template <typename T>
__global__ void __launch_bounds__(256) small_eval_kernel(int d, CoreArgs ca, int64_t m, const int32_t* __restrict__ idx,
                                                         T* __restrict__ out, unsigned* err) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    T v[kSmallR], w[kSmallR];
    v[0] = 1;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < kSmallD; ++k) {
      if (k < d) {
        int32_t i = __ldg(idx + (int64_t)k * m + e);
        const int r0 = ca.r[k], r1 = ca.r[k + 1], n = ca.n[k];
        if (i < 0 || i >= n) { bad = true; i = 0; }
        const T* G = (const T*)ca.core[k] + (int64_t)i * r1;
#pragma unroll
        for (int b = 0; b < kSmallR; ++b) w[b] = 0;
#pragma unroll
        for (int a = 0; a < kSmallR; ++a) {
          if (a < r0) {
            const T* row = G + (int64_t)a * n * r1;
#pragma unroll
            for (int b = 0; b < kSmallR; ++b)
              if (b < r1) w[b] = fma(v[a], __ldg(row + b), w[b]);
          }
        }
#pragma unroll
        for (int b = 0; b < kSmallR; ++b) v[b] = w[b];
      }
    }
    if (bad) { atomicOr(err, 1u); out[e] = 0; }
    else out[e] = v[0];
  }
}

bool small_shape(const CoreArgs& ca, int d) {
  if (d > kSmallD) return false;
  for (int k = 0; k <= d; ++k)
    if (ca.r[k] > kSmallR) return false;
  return true;
}

// warps per block so that `vecs` vectors of rmax values per warp fit the budget
template <typename K>
int warps_for(K kernel, int64_t rmax, int vecs, size_t esz, size_t* smem) {
  const int64_t per_warp = rmax * vecs * (int64_t)esz;
  int64_t w = std::min<int64_t>(kMaxWarps, kSmemBudget / per_warp);
  if (w < 1) fail(FASTTT_ERANK, "TT rank too large for the shared-memory vectors");
  *smem = (size_t)(w * per_warp);
  // always the budget (not this call's need), so that concurrent callers never lower it for each other
  FTT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget));
  return (int)w;
}

int max_rank_of(const CoreArgs& ca, int d) {
  int r = 1;
  for (int k = 0; k <= d; ++k) r = std::max(r, (int)ca.r[k]);
  return r;
}

void check_args(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores, int dtype, int64_t m,
                const int32_t* idx, CoreArgs& ca) {
  if (d < 1 || d > FASTTT_MAX_D) fail(FASTTT_EINVAL, "d must be in 1..64");
  if (!dims || !ranks || !cores) fail(FASTTT_EINVAL, "null argument");
  if (dtype != FASTTT_F64 && dtype != FASTTT_F32) fail(FASTTT_EINVAL, "bad dtype");
  if (m < 0 || (m > 0 && !idx)) fail(FASTTT_EINVAL, "bad index array");
  if (ranks[0] != 1 || ranks[d] != 1) fail(FASTTT_EINVAL, "r_0 and r_d must be 1");
  ca.off[0] = 0;
  for (int k = 0; k <= d; ++k) {
    if (ranks[k] < 1) fail(FASTTT_EINVAL, "ranks must be >= 1");
    if (ranks[k] > kMaxRank) fail(FASTTT_ERANK, "TT rank above 8192");
    ca.r[k] = (int32_t)ranks[k];
    if (k < d) ca.off[k + 1] = ca.off[k] + ranks[k];
  }
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1 || dims[k] > INT32_MAX) fail(FASTTT_EINVAL, "bad mode size");
    if (!cores[k]) fail(FASTTT_EINVAL, "null core pointer");
    ca.n[k] = (int32_t)dims[k];
    ca.core[k] = cores[k];
    ca.grad[k] = nullptr;
  }
}

}  // namespace

int tt_eval_at_impl(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores, int dtype, int64_t m,
                    const int32_t* idx, void* out, cudaStream_t s) {
  CoreArgs ca;
  check_args(d, dims, ranks, cores, dtype, m, idx, ca);
  if (m == 0) return FASTTT_OK;
  if (!out) fail(FASTTT_EINVAL, "null output");
  if (!small_shape(ca, d) && tteval_sorted_applies(d, dims, ranks)) {
    tt_eval_sorted(d, dims, ranks, cores, dtype, m, idx, out, s);
    return FASTTT_OK;
  }
  DBuf<unsigned> err(1, s);
  FTT_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(unsigned), s));
  const int rmax = max_rank_of(ca, d);
  size_t smem = 0;
  if (small_shape(ca, d)) {
    const int64_t blocks = std::min<int64_t>(ceil_div(m, 256), (int64_t)kNumSMs * 8);
    if (dtype == FASTTT_F64)
      small_eval_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(d, ca, m, idx, (double*)out, err.get());
    else
      small_eval_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(d, ca, m, idx, (float*)out, err.get());
  } else if (dtype == FASTTT_F64) {
    const int nw = warps_for(eval_kernel<double>, rmax, 2, 8, &smem);
    const int64_t blocks = std::min<int64_t>(ceil_div(m, nw), (int64_t)kNumSMs * 16);
    eval_kernel<double><<<(unsigned)blocks, nw * 32, smem, s>>>(d, ca, m, idx, (double*)out, err.get(), rmax);
  } else {
    const int nw = warps_for(eval_kernel<float>, rmax, 2, 4, &smem);
    const int64_t blocks = std::min<int64_t>(ceil_div(m, nw), (int64_t)kNumSMs * 16);
    eval_kernel<float><<<(unsigned)blocks, nw * 32, smem, s>>>(d, ca, m, idx, (float*)out, err.get(), rmax);
  }
  FTT_LAUNCH();
  if (read_scalar(err.get(), s)) fail(FASTTT_EINVAL, "index out of range");
  return FASTTT_OK;
}

int tt_eval_backward_impl(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores, int dtype,
                          int64_t m, const int32_t* idx, const void* gout, void* const* grads, int recompute,
                          cudaStream_t s) {
  CoreArgs ca;
  check_args(d, dims, ranks, cores, dtype, m, idx, ca);
  if (!grads) fail(FASTTT_EINVAL, "null gradient array");
  for (int k = 0; k < d; ++k) {
    if (!grads[k]) fail(FASTTT_EINVAL, "null gradient core");
    ca.grad[k] = grads[k];
  }
  if (m == 0) return FASTTT_OK;
  if (!gout) fail(FASTTT_EINVAL, "null upstream gradient");
  if (tteval_sorted_applies(d, dims, ranks)) {
    tt_backward_sorted(d, dims, ranks, cores, dtype, m, idx, gout, grads, recompute, s);
    return FASTTT_OK;
  }
  DBuf<unsigned> err(1, s);
  FTT_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(unsigned), s));
  const int rmax = max_rank_of(ca, d);
  const size_t esz = (dtype == FASTTT_F64) ? 8 : 4;
  const int64_t stride = recompute ? 0 : ca.off[d];
  size_t smem = 0;
  int nw;
  if (dtype == FASTTT_F64) nw = warps_for(backward_kernel<double>, rmax, 4, 8, &smem);
  else nw = warps_for(backward_kernel<float>, rmax, 4, 4, &smem);
  const int64_t blocks = std::min<int64_t>(ceil_div(m, nw), (int64_t)kNumSMs * 32);
  DBuf<unsigned char> left(recompute ? 0 : (size_t)blocks * nw * stride * esz, s);
  if (dtype == FASTTT_F64)
    backward_kernel<double><<<(unsigned)blocks, nw * 32, smem, s>>>(d, ca, m, idx, (const double*)gout, recompute,
                                                                    (double*)left.get(), stride, err.get(), rmax);
  else
    backward_kernel<float><<<(unsigned)blocks, nw * 32, smem, s>>>(d, ca, m, idx, (const float*)gout, recompute,
                                                                   (float*)left.get(), stride, err.get(), rmax);
  FTT_LAUNCH();
  if (read_scalar(err.get(), s)) fail(FASTTT_EINVAL, "index out of range");
  return FASTTT_OK;
}

}  // namespace fasttt

namespace fasttt {

// The adjoint with stored left partials, run in caller-provided device scratch:
// the first 256 bytes hold the error flag, the rest the per-warp left partials.
// The grid is sized so the partials fit.  Allocates no device memory.
int tt_eval_backward_prealloc(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores,
                              int dtype, int64_t m, const int32_t* idx, const void* gout, void* const* grads,
                              void* scratch, size_t scratch_bytes, cudaStream_t s) {
  CoreArgs ca;
  check_args(d, dims, ranks, cores, dtype, m, idx, ca);
  if (!grads) fail(FASTTT_EINVAL, "null gradient array");
  for (int k = 0; k < d; ++k) {
    if (!grads[k]) fail(FASTTT_EINVAL, "null gradient core");
    ca.grad[k] = grads[k];
  }
  if (m == 0) return FASTTT_OK;
  if (!gout) fail(FASTTT_EINVAL, "null upstream gradient");
  if (!scratch || scratch_bytes <= 256) fail(FASTTT_EINVAL, "no scratch");
  unsigned* err = static_cast<unsigned*>(scratch);
  const int rmax = max_rank_of(ca, d);
  const size_t esz = (dtype == FASTTT_F64) ? 8 : 4;
  const int64_t stride = ca.off[d];
  size_t smem = 0;
  int nw;
  if (dtype == FASTTT_F64) nw = warps_for(backward_kernel<double>, rmax, 4, 8, &smem);
  else nw = warps_for(backward_kernel<float>, rmax, 4, 4, &smem);
  const int64_t fit_warps = (int64_t)((scratch_bytes - 256) / ((size_t)stride * esz));
  const int64_t blocks = std::min<int64_t>(std::min<int64_t>(ceil_div(m, nw), (int64_t)kNumSMs * 32), fit_warps / nw);
  if (blocks < 1) fail(FASTTT_ERANK, "sum of TT ranks too large for the fixed scratch");
  FTT_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
  void* left = static_cast<unsigned char*>(scratch) + 256;
  if (dtype == FASTTT_F64)
    backward_kernel<double><<<(unsigned)blocks, nw * 32, smem, s>>>(d, ca, m, idx, (const double*)gout, 0,
                                                                    (double*)left, stride, err, rmax);
  else
    backward_kernel<float><<<(unsigned)blocks, nw * 32, smem, s>>>(d, ca, m, idx, (const float*)gout, 0,
                                                                   (float*)left, stride, err, rmax);
  FTT_LAUNCH();
  if (read_scalar(err, s)) fail(FASTTT_EINVAL, "index out of range");
  return FASTTT_OK;
}

}  // namespace fasttt
