// tt_fit_gd: fixed-rank fitting of a TT to given entries (the tensor-completion
// use of fixed-rank TT approximations, Sec. 3.4) by gradient descent with the
// adjoint of the entry formula (Sec. 2.3).  One step:
//   a_e = G_1[i_1^e] ... G_d[i_d^e]            (tt_eval_at kernels)
//   r_e = a_e - v_e,  L = 1/2 sum_e r_e^2      (residual_kernel, FP64 partial sums)
//   dL/dG_k = adjoint with upstream weights r_e (tt_eval_backward kernels)
//   G_k <- G_k - lr dL/dG_k, all cores from the same point (descend_kernel)
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "common.cuh"

namespace fasttt {
int tt_eval_at_impl(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores, int dtype, int64_t m,
                    const int32_t* idx, void* out, cudaStream_t s);
int tt_eval_backward_impl(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores, int dtype,
                          int64_t m, const int32_t* idx, const void* gout, void* const* grads, int recompute,
                          cudaStream_t s);
void set_last_error(const char* msg);

namespace {

constexpr int kFitThreads = 256;

__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// r_e = a_e - v_e written over a; block b's sum of r_e^2 (FP64) to partial[b]
template <typename T>
__global__ void __launch_bounds__(kFitThreads) residual_kernel(T* a, const T* v, int64_t m, double* partial) {
  __shared__ double red[kFitThreads / 32];
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)kFitThreads + threadIdx.x; e < m; e += (int64_t)gridDim.x * kFitThreads) {
    const T r = sub_rn(a[e], v[e]);
    a[e] = r;
    acc = fma((double)r, (double)r, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kFitThreads / 32; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// G <- G - lr dG (product and difference rounded separately, no fused multiply-add)
template <typename T>
__global__ void __launch_bounds__(kFitThreads) descend_kernel(T* G, const T* dG, int64_t n, T lr) {
  for (int64_t e = blockIdx.x * (int64_t)kFitThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kFitThreads)
    G[e] = sub_rn(G[e], mul_rn(lr, dG[e]));
}

template <typename T>
void fit_gd(int d, const int64_t* dims, const int64_t* ranks, void* const* cores, int dtype, int64_t m,
            const int32_t* idx, const void* vals, int64_t steps, double lr, double* losses, cudaStream_t s) {
  std::vector<const void*> ccores(cores, cores + d);
  const size_t esz = sizeof(T);
  DBuf<T> a((size_t)m, s);
  const int blocks = m > 0 ? grid_for(m, kFitThreads) : 0;
  DBuf<double> partial((size_t)blocks, s);
  std::vector<double> hp((size_t)blocks);
  auto loss_now = [&]() {   // leaves the residual in a
    tt_eval_at_impl(d, dims, ranks, ccores.data(), dtype, m, idx, a.get(), s);
    if (m == 0) return 0.0;
    residual_kernel<T><<<blocks, kFitThreads, 0, s>>>(a.get(), static_cast<const T*>(vals), m, partial.get());
    FTT_LAUNCH();
    FTT_CUDA(cudaMemcpyAsync(hp.data(), partial.get(), sizeof(double) * blocks, cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    double t = 0.0;
    for (double x : hp) t += x;
    return 0.5 * t;
  };
  losses[0] = loss_now();   // also validates the TT and the indices
  std::vector<int64_t> sizes(d);
  std::vector<DBuf<T>> g;
  std::vector<void*> gp(d);
  for (int k = 0; k < d; ++k) {
    sizes[k] = ranks[k] * dims[k] * ranks[k + 1];
    g.emplace_back((size_t)sizes[k], s);
    gp[k] = g.back().get();
  }
  for (int64_t t = 0; t < steps; ++t) {
    if (t > 0) losses[t] = loss_now();
    if (m > 0) {
      for (int k = 0; k < d; ++k) FTT_CUDA(cudaMemsetAsync(gp[k], 0, (size_t)sizes[k] * esz, s));
      tt_eval_backward_impl(d, dims, ranks, ccores.data(), dtype, m, idx, a.get(), gp.data(), 0, s);
      for (int k = 0; k < d; ++k) {
        descend_kernel<T><<<grid_for(sizes[k], kFitThreads), kFitThreads, 0, s>>>(static_cast<T*>(cores[k]),
                                                                                  g[k].get(), sizes[k], (T)lr);
        FTT_LAUNCH();
      }
    }
  }
  if (steps > 0) losses[steps] = loss_now();
  FTT_CUDA(cudaStreamSynchronize(s));
}

}  // namespace
}  // namespace fasttt

extern "C" int tt_fit_gd(int d, const int64_t* dims, const int64_t* ranks, void* const* d_cores, int dtype, int64_t m,
                         const int32_t* d_idx, const void* d_vals, int64_t steps, double lr, double* h_losses,
                         void* stream) {
  ::fasttt::set_last_error("");
  try {
    if (d < 1 || d > FASTTT_MAX_D || !dims || !ranks || !d_cores) ::fasttt::fail(FASTTT_EINVAL, "tt_fit_gd: bad TT");
    if (m < 0 || steps < 0 || !std::isfinite(lr) || !h_losses || (m > 0 && (!d_vals || !d_idx)))
      ::fasttt::fail(FASTTT_EINVAL, "tt_fit_gd: bad entries, steps, lr or loss array");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == FASTTT_F64)
      ::fasttt::fit_gd<double>(d, dims, ranks, d_cores, dtype, m, d_idx, d_vals, steps, lr, h_losses, s);
    else if (dtype == FASTTT_F32)
      ::fasttt::fit_gd<float>(d, dims, ranks, d_cores, dtype, m, d_idx, d_vals, steps, lr, h_losses, s);
    else
      ::fasttt::fail(FASTTT_EINVAL, "bad dtype");
    return FASTTT_OK;
  } catch (const ::fasttt::Error& e) {
    ::fasttt::set_last_error(e.what());
    return e.code;
  }
}
