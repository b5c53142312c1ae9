// Device primitives of libfasttt: a three-phase exclusive scan and a stable LSD
// radix sort of (key, value) pairs, both without inter-block waiting (every block
// only reads what earlier kernels wrote), plus dense ranking of sorted keys.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace fasttt {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048 elements per block

// Block-wide exclusive scan of kScanTile values staged in shared memory.
// Returns the block total (to every thread).
template <typename T>
__device__ T block_exclusive_scan(T* tile) {
  __shared__ T warp_tot[kScanThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  T local[kScanItems];
  T sum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    local[j] = tile[t * kScanItems + j];
    sum += local[j];
  }
  // inclusive warp scan of per-thread sums
  T incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  T warp_off = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) {
    T v = warp_tot[w];
    if (w < warp) warp_off += v;
    total += v;
  }
  T run = warp_off + incl - sum;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    tile[t * kScanItems + j] = run;
    run += local[j];
  }
  __syncthreads();
  return total;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const T* in, int64_t n, T* partial) {
  __shared__ T red[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  T s = 0;
  for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
    int64_t i = base + j;
    if (i < n) s += in[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    T tot = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) tot += red[w];
    partial[blockIdx.x] = tot;
  }
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads)
    scan_down_kernel(const T* in, T* out, int64_t n, const T* offsets, T* total_out) {
  __shared__ T tile[kScanTile];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
    int64_t i = base + j;
    tile[j] = (i < n) ? in[i] : T(0);
  }
  __syncthreads();
  T tot = block_exclusive_scan<T>(tile);
  const T off = offsets ? offsets[blockIdx.x] : T(0);
  for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
    int64_t i = base + j;
    if (i < n) out[i] = tile[j] + off;
  }
  if (total_out && threadIdx.x == 0) *total_out = off + tot;
}

template <typename T>
void exclusive_scan_rec(const T* in, T* out, int64_t n, T* total_dev, cudaStream_t s) {
  const int64_t nb = ceil_div(n, kScanTile);
  if (nb <= 1) {
    scan_down_kernel<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total_dev);
    FTT_LAUNCH();
    return;
  }
  DBuf<T> part(nb, s);
  scan_reduce_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, part.get());
  FTT_LAUNCH();
  exclusive_scan_rec<T>(part.get(), part.get(), nb, total_dev, s);
  // The last block of the recursive scan wrote the grand total; the down-sweep
  // below must not overwrite it, so it gets no total pointer.
  scan_down_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, part.get(), nullptr);
  FTT_LAUNCH();
}

// ---------------------------------------------------------------- radix sort

constexpr int kSortThreads = 256;       // == number of digit values (8-bit digits)
constexpr int kSortWarps = kSortThreads / 32;
constexpr int64_t kSortChunk = kSortThreads * 16;  // keys per block

__global__ void __launch_bounds__(kSortThreads)
    radix_hist_kernel(const uint64_t* keys, int64_t n, int shift, uint32_t* hist, int nblocks) {
  __shared__ uint32_t h[kSortWarps][256];
  const int t = threadIdx.x, warp = t >> 5;
  for (int w = 0; w < kSortWarps; ++w) h[w][t] = 0;
  __syncthreads();
  const int64_t beg = (int64_t)blockIdx.x * kSortChunk;
  const int64_t end = min(n, beg + kSortChunk);
  for (int64_t i = beg + t; i < end; i += kSortThreads) {
    uint32_t dig = (uint32_t)(keys[i] >> shift) & 255u;
    atomicAdd(&h[warp][dig], 1u);
  }
  __syncthreads();
  uint32_t c = 0;
  for (int w = 0; w < kSortWarps; ++w) c += h[w][t];
  hist[(int64_t)t * nblocks + blockIdx.x] = c;  // digit-major: scan gives global offsets
}

// Stable scatter: keys are taken in index order (tile by tile, warp by warp,
// lane by lane) and each lands after every earlier key with the same digit.
__global__ void __launch_bounds__(kSortThreads)
    radix_scatter_kernel(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                         uint32_t* vals_out, int64_t n, int shift, const uint32_t* offsets,
                         int nblocks) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[kSortWarps][256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  base[t] = offsets[(int64_t)t * nblocks + blockIdx.x];
  const int64_t beg = (int64_t)blockIdx.x * kSortChunk;
  const int64_t end = min(n, beg + kSortChunk);
  for (int64_t s0 = beg; s0 < end; s0 += kSortThreads) {
    const int64_t i = s0 + t;
    const bool valid = i < end;
    uint64_t k = 0;
    uint32_t v = 0, dig = 0;
    if (valid) {
      k = keys_in[i];
      v = vals_in[i];
      dig = (uint32_t)(k >> shift) & 255u;
    }
    for (int j = lane; j < 256; j += 32) wcnt[warp][j] = 0;
    __syncwarp();
    const unsigned active = __ballot_sync(0xffffffffu, valid);
    int rank = 0;
    if (valid) {
      const unsigned peers = __match_any_sync(active, dig);
      rank = __popc(peers & lt_mask);
      if (rank == 0) wcnt[warp][dig] = __popc(peers);
    }
    __syncthreads();
    {
      uint32_t run = base[t];
      for (int w = 0; w < kSortWarps; ++w) {
        uint32_t c = wcnt[w][t];
        wcnt[w][t] = run;
        run += c;
      }
      base[t] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = wcnt[warp][dig] + (uint32_t)rank;
      keys_out[pos] = k;
      vals_out[pos] = v;
    }
    __syncthreads();
  }
}

__global__ void heads_kernel(const uint64_t* keys, int64_t n, int64_t* heads) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    heads[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void rank_scatter_kernel(const uint64_t* keys, const uint32_t* vals, int64_t n,
                                    const int64_t* excl, int32_t* ranks, uint64_t* uniq) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool head = (i == 0 || keys[i] != keys[i - 1]);
    const int64_t r = head ? excl[i] : excl[i] - 1;
    if (ranks) ranks[vals[i]] = (int32_t)r;
    if (head && uniq) uniq[r] = keys[i];
  }
}

}  // namespace

int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  DBuf<int64_t> tot(1, s);
  exclusive_scan_rec<int64_t>(in, out, n, tot.get(), s);
  return read_scalar(tot.get(), s);
}

int64_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  DBuf<uint32_t> tot(1, s);
  exclusive_scan_rec<uint32_t>(in, out, n, tot.get(), s);
  return read_scalar(tot.get(), s);
}

void radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                      int64_t n, int bits, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return;
  if (n >= (int64_t)1 << 32) fail(FASTTT_ERANK, "radix sort: more than 2^32 - 1 keys");
  const int nblocks = (int)ceil_div(n, kSortChunk);
  DBuf<uint32_t> hist((size_t)256 * nblocks, s);
  uint64_t* kin = keys;
  uint32_t* vin = vals;
  uint64_t* kout = keys_alt;
  uint32_t* vout = vals_alt;
  const int passes = (bits + 7) / 8;
  KClock clk;
  kclock_begin(clk, KC_SORT, s);
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * 8;
    radix_hist_kernel<<<nblocks, kSortThreads, 0, s>>>(kin, n, shift, hist.get(), nblocks);
    FTT_LAUNCH();
    DBuf<uint32_t> tot(1, s);
    exclusive_scan_rec<uint32_t>(hist.get(), hist.get(), (int64_t)256 * nblocks, tot.get(), s);
    radix_scatter_kernel<<<nblocks, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, hist.get(),
                                                          nblocks);
    FTT_LAUNCH();
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  // per pass: keys read twice (histogram, scatter) + values read once + both written
  kclock_end(clk, (double)passes * (double)n * (8.0 * 2 + 4.0 + 12.0), s);
  if (kin != keys) {  // odd number of passes: result is in the alternate buffers
    FTT_CUDA(cudaMemcpyAsync(keys, kin, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    FTT_CUDA(cudaMemcpyAsync(vals, vin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
}

int64_t rank_sorted(const uint64_t* keys, const uint32_t* vals, int64_t n, int32_t* ranks,
                    uint64_t* uniq, cudaStream_t s) {
  if (n <= 0) return 0;
  DBuf<int64_t> heads(n, s);
  const int g = grid_for(n);
  heads_kernel<<<g, 256, 0, s>>>(keys, n, heads.get());
  FTT_LAUNCH();
  const int64_t total = exclusive_scan_i64(heads.get(), heads.get(), n, s);
  rank_scatter_kernel<<<g, 256, 0, s>>>(keys, vals, n, heads.get(), ranks, uniq);
  FTT_LAUNCH();
  return total;
}

}  // namespace fasttt
