// Block and grid synchronisation helpers shared by the dense kernels.
#pragma once

#include <cuda_runtime.h>

namespace fasttt {
namespace {

// Block-wide sum of three values (256 threads).
template <typename T>
__device__ __forceinline__ void block_sum3(T& a, T& b, T& c) {
  __shared__ T red[3][8];
  __syncthreads();  // earlier readers of red are done
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
    T x = 0, y = 0, z = 0;
    for (int w = 0; w < 8; ++w) { x += red[0][w]; y += red[1][w]; z += red[2][w]; }
    red[0][0] = x; red[1][0] = y; red[2][0] = z;
  }
  __syncthreads();
  a = red[0][0]; b = red[1][0]; c = red[2][0];
}

// Block-wide sum of three values for NW warps, summed in warp order (deterministic).
template <typename T, int NW>
__device__ __forceinline__ void block_sum3n(T& a, T& b, T& c) {
  __shared__ T red[3][NW];
  __syncthreads();  // earlier readers of red are done
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
    T x = 0, y = 0, z = 0;
    for (int w = 0; w < NW; ++w) { x += red[0][w]; y += red[1][w]; z += red[2][w]; }
    red[0][0] = x; red[1][0] = y; red[2][0] = z;
  }
  __syncthreads();
  a = red[0][0]; b = red[1][0]; c = red[2][0];
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident).  bar[0]
// counts arrivals, bar[1] is the generation, bar[2] an error flag, bar[3] the poll
// bound (0: kBarrierSpins).  The wait is bounded: after that many polls the block
// raises the error flag and every block leaves the kernel at its next barrier.
constexpr long long kBarrierSpins = 1ll << 24;

// bar[0..2] = 0, bar[3] = the poll bound (set before every cooperative launch)
__global__ void barrier_init_kernel(unsigned* bar, unsigned spins) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    bar[0] = 0u;
    bar[1] = 0u;
    bar[2] = 0u;
    bar[3] = spins;
  }
}

__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned& gen) {
  __shared__ int ok;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = bar + 1;
    volatile unsigned* verr = bar + 2;
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      const long long limit = bar[3] ? (long long)bar[3] : kBarrierSpins;
      while (*vgen == gen) {
        if (*verr) { ok = 0; break; }
        if (++it > limit) { atomicOr(bar + 2, 1u); ok = 0; break; }
        __nanosleep(64);
      }
    }
    if (*verr) ok = 0;
    __threadfence();
  }
  __syncthreads();
  ++gen;
  return ok != 0;
}

}  // namespace
}  // namespace fasttt
