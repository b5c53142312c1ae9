// Dense GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) with FP64
// operands, by exact bf16 slicing (the error-free splitting of Ozaki, Ogita,
// Oishi & Rump, Numer. Algorithms 59, 2012):
//
//   row i of A:    a_ik = 2^{e_i} sum_{s=1..S} q^A_{s,ik} 2^{-8s},  |q^A_{s,ik}| <= 256 (s = 1), <= 128 (s > 1)
//   column j of B: b_kj = 2^{f_j} sum_{t=1..S} q^B_{t,kj} 2^{-8t} + (truncation below 2^{-8S})
//
// Every slice q is an integer of at most 8 significant bits, exact in bf16, and
// every product q^A q^B is exact in FP32.  Products are grouped by level
// g = s + t (g <= S + 1; the rest is below 2^{-8S} of |a||b|):
//   (A B)_ij = 2^{e_i + f_j} sum_g 2^{-8g} sum_{s+t=g} sum_k q^A_{s,ik} q^B_{t,kj}.
// One tcgen05.mma (kind::f16, bf16 x bf16 -> FP32 in TMEM) per slice pair and
// K step of 16 accumulates a level over a K chunk of 64.  The first slice is at
// most 256 in magnitude and the others at most 128, so a product is at most 2^16
// (pair (1,1)) or 2^15, and a level's chunk sum over 64 products of at most S
// pairs stays below 2^24: every level's chunk sum is exact in FP32.  After every chunk the 4 epilogue warps read the level
// accumulators out of TMEM (tcgen05.ld) and add them into 64-bit
// integer registers: the level sums are exact integers below 2^24, so levels
// 2..5 are packed into one int64 (weights 2^{8(5-g)}) and the rest into another,
// and the whole K reduction is exact; FP64 enters only when the two packed sums
// are scaled into C.  S = 7 gives products to FP64 accuracy (levels below
// 2^{-56}); S = 3 gives FP32-level accuracy (the mixed-precision path).
//
// Tiles: 128 (M) x 64 (N) per CTA, K chunk 64 = one 128-byte bf16 row; the S
// slices of A and of B for a chunk are loaded by TMA (SWIZZLE_128B, one box per
// slice) into shared memory and consumed by K-major SW128 UMMA descriptors.
// Every mbarrier wait is bounded; a block that gives up raises the error flag,
// frees its TMEM and returns, and the caller falls back to the FP64 DFMA GEMM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "dense.cuh"

namespace fasttt {

namespace {

constexpr int kBM = 128, kBN = 64, kBK = 64;
constexpr long long kMbarSpins = 1ll << 22;
constexpr int kThreads = 256;   // 8 warps: TMEM lane quarter warp % 4, column half warp / 4

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kMbarSpins; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// K-major operand tile of rows x 64 bf16 (128-byte rows), 128-byte swizzle:
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// kind::f16 instruction descriptor: D FP32, A and B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// C tile (128 x 64) of alpha 2^{e_i + f_j} sum_g 2^{-8g} L_g + beta C.
template <int S>
__global__ void __launch_bounds__(kThreads, 1)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t M,
                      int64_t N, int64_t Kp, int64_t Mp, int64_t Np, const int* __restrict__ ea,
                      const int* __restrict__ fb, double alpha, double beta, double* __restrict__ C, int64_t sci,
                      int64_t scj, bool sym, int* err) {
  constexpr int kLevels = S;                       // g = 2 .. S + 1
  constexpr uint32_t kCols = (kLevels * kBN <= 256) ? 256 : 512;
  constexpr uint32_t kTileA = kBM * kBK * 2, kTileB = kBN * kBK * 2;
  constexpr uint32_t kStageBytes = S * (kTileA + kTileB);
  const int bm = blockIdx.x, bn = blockIdx.y;
  if (sym && (int64_t)bm * kBM >= (int64_t)(bn + 1) * kBN) return;   // strictly below the diagonal
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;                      // S tiles of 128 x 64 bf16
  unsigned char* sB = smem + S * kTileA;         // S tiles of 64 x 64 bf16
  __shared__ uint64_t full_bar, mma_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&full_bar, 1);
    mbar_init(&mma_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = idesc_bf16(kBM, kBN);
  // Exact integer accumulation of the level sums over K: levels 2..5 in hi (level
  // g weighted 2^{8(5-g)}), levels 6..S+1 in lo (weighted 2^{8(S+1-g)}); a chunk
  // adds below 2^48 to each, so 2^15 chunks fit in int64.
  constexpr int kHiLevels = (S < 4) ? S : 4;
  constexpr int kLoLevels = S - kHiLevels;
  long long hi[32], lo[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) hi[c] = lo[c] = 0;
  const int nchunks = (int)(Kp / kBK);
  const int quarter = warp & 3, half = warp >> 2;
  bool ok = true;
  int pending = 0;             // 1: a TMA phase, 2: an MMA phase left unfinished by a timeout
  uint32_t pending_parity = 0;
  if (tid == 0) {
    mbar_arrive_expect_tx(&full_bar, kStageBytes);
    for (int s = 0; s < S; ++s) {
      tma_load_2d(sA + s * kTileA, &tmA, &full_bar, 0, (int)(s * Mp + (int64_t)bm * kBM));
      tma_load_2d(sB + s * kTileB, &tmB, &full_bar, 0, (int)(s * Np + (int64_t)bn * kBN));
    }
  }
  for (int ch = 0; ch < nchunks; ++ch) {
    const uint32_t parity = (uint32_t)(ch & 1);
    if (!mbar_wait(&full_bar, parity)) abort_flag = 1;
    if (__syncthreads_or(abort_flag)) { ok = false; pending = 1; pending_parity = parity; break; }
    tc_fence_after();
    if (tid == 0) {
      // level g = s + t (g = 2 .. S + 1) accumulates in TMEM columns (g - 2) * 64 ..
      uint32_t started = 0;   // bit l: level l already has a product in this chunk
#pragma unroll 1
      for (int s = 1; s <= S; ++s) {
        const uint64_t da = sw128_desc(smem_u32(sA + (s - 1) * kTileA));
#pragma unroll 1
        for (int t = 1; t + s <= S + 1; ++t) {
          const int l = s + t - 2;
          const uint64_t db = sw128_desc(smem_u32(sB + (t - 1) * kTileB));
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {   // K steps of 16 bf16 = 32 bytes
            umma_bf16(tbase + (uint32_t)(l * kBN), da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc,
                      (started >> l) & 1u);
            started |= 1u << l;
          }
        }
      }
      umma_commit(&mma_bar);
    }
    if (!mbar_wait(&mma_bar, parity)) abort_flag = 1;
    if (__syncthreads_or(abort_flag)) { ok = false; pending = 2; pending_parity = parity; break; }
    tc_fence_after();
    // the MMAs have read the stage: load the next chunk while this one drains
    if (tid == 0 && ch + 1 < nchunks) {
      mbar_arrive_expect_tx(&full_bar, kStageBytes);
      for (int s = 0; s < S; ++s) {
        tma_load_2d(sA + s * kTileA, &tmA, &full_bar, (ch + 1) * kBK, (int)(s * Mp + (int64_t)bm * kBM));
        tma_load_2d(sB + s * kTileB, &tmB, &full_bar, (ch + 1) * kBK, (int)(s * Np + (int64_t)bn * kBN));
      }
    }
    // drain: TMEM lanes 32 * quarter .. (tile rows), columns 32 * half .. of every level
    const uint32_t lane_base = tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
#pragma unroll
    for (int l = 0; l < kLevels; ++l)
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(lane_base + (uint32_t)(l * kBN + c0), r);
        if (l < kHiLevels) {
          const int sh = 8 * (kHiLevels - 1 - l);
#pragma unroll
          for (int c = 0; c < 16; ++c) hi[c0 + c] += (long long)__float2int_rn(__uint_as_float(r[c])) << sh;
        } else {
          const int sh = 8 * (kLevels - 1 - l);
#pragma unroll
          for (int c = 0; c < 16; ++c) lo[c0 + c] += (long long)__float2int_rn(__uint_as_float(r[c])) << sh;
        }
      }
    tc_fence_before();
    __syncthreads();
  }
  if (ok) {
    const int64_t i = (int64_t)bm * kBM + quarter * 32 + lane;
    if (i < M) {
      const double si = ldexp(alpha, ea[i]);
      // value = 2^{-8(kHiLevels+1)} hi + 2^{-8(S+1)} lo
      const double whi = ldexp(1.0, -8 * (kHiLevels + 1)), wlo = ldexp(1.0, -8 * (S + 1));
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int64_t j = (int64_t)bn * kBN + half * 32 + c;
        if (j >= N) continue;
        double* cp = C + i * sci + j * scj;
        const double sum = fma((double)hi[c], whi, (kLoLevels > 0) ? (double)lo[c] * wlo : 0.0);
        const double v = ldexp(si * sum, fb[j]);
        *cp = (beta == 0.0) ? v : fma(beta, *cp, v);
      }
    }
  } else {
    // give the copies or MMAs still in flight a second bounded wait before TMEM is freed
    if (pending == 1) mbar_wait(&full_bar, pending_parity);
    if (pending == 2) mbar_wait(&mma_bar, pending_parity);
    if (tid == 0) atomicOr(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols) : "memory");
}

// Row exponents and slices of A (M x K with element strides): e_i with
// max_k |a_ik| < 2^{e_i}; q[s][i][k] (bf16, Mp x Kp per slice, zero padded).
// One warp per row (of A, or of B^T for the B operand).
template <int S>
__global__ void ozaki_split_kernel(const double* __restrict__ X, int64_t rows, int64_t cols, int64_t s_row,
                                   int64_t s_col, int64_t rows_p, int64_t cols_p, int* __restrict__ ex,
                                   __nv_bfloat16* __restrict__ q) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w; i < rows_p; i += nw) {
    double mx = 0.0;
    if (i < rows)
      for (int64_t k = lane; k < cols; k += 32) mx = fmax(mx, fabs(X[i * s_row + k * s_col]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) {
      frexp(mx, &e);   // mx = m 2^e, 0.5 <= m < 1: mx < 2^e
    }
    if (lane == 0 && i < rows) ex[i] = e;
    for (int64_t k = lane; k < cols_p; k += 32) {
      double r = (i < rows && k < cols) ? ldexp(X[i * s_row + k * s_col], -e) : 0.0;   // |r| < 1, exact
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const double t = r * 256.0;   // exact
        const double qv = rint(t);    // |qv| <= 256
        r = t - qv;                   // exact, |r| <= 1/2
        q[((int64_t)s * rows_p + i) * cols_p + k] = __float2bfloat16_rn((float)qv);
      }
    }
  }
}

__global__ void mirror_upper_oz_kernel(double* C, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (i > j) C[e] = C[j * n + i];
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols_p, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols_p, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols_p * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int S>
bool run_ozaki(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
               const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
               cudaStream_t s, bool sym) {
  const int64_t Mp = ceil_div(M, kBM) * kBM, Np = ceil_div(N, kBN) * kBN, Kp = ceil_div(K, kBK) * kBK;
  if ((S * Mp) >= INT32_MAX || (S * Np) >= INT32_MAX || Np / kBN > 65535) return false;
  if (Kp / kBK > (1 << 15)) return false;   // the int64 level accumulators hold 2^15 chunks
  const size_t smem = (size_t)S * (kBM + kBN) * kBK * 2 + 1024;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(ozaki_gemm_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr_set = true;
  }
  DBuf<__nv_bfloat16> qa((size_t)S * Mp * Kp, s), qb((size_t)S * Np * Kp, s);
  DBuf<int> ea(Mp, s), fb(Np, s), err(1, s);
  FTT_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
  // A rows: a(i, k) = A[i*sai + k*sak]; B^T rows: b(j, k) = B[k*sbk + j*sbj]
  ozaki_split_kernel<S><<<grid_for(Mp * 32), 256, 0, s>>>(A, M, K, sai, sak, Mp, Kp, ea.get(), qa.get());
  FTT_LAUNCH();
  ozaki_split_kernel<S><<<grid_for(Np * 32), 256, 0, s>>>(B, N, K, sbj, sbk, Np, Kp, fb.get(), qb.get());
  FTT_LAUNCH();
  CUtensorMap ma, mb;
  if (!make_map(&ma, qa.get(), S * Mp, Kp, kBM) || !make_map(&mb, qb.get(), S * Np, Kp, kBN)) return false;
  KClock clk;
  kclock_begin(clk, KC_GEMM_OZ, s);
  ozaki_gemm_kernel<S><<<dim3((unsigned)(Mp / kBM), (unsigned)(Np / kBN)), kThreads, smem, s>>>(
      ma, mb, M, N, Kp, Mp, Np, ea.get(), fb.get(), alpha, beta, C, sci, scj, sym, err.get());
  FTT_LAUNCH();
  kclock_end(clk, (sym ? 1.0 : 2.0) * (double)M * (double)N * (double)K, s);
  int herr = 0;
  FTT_CUDA(cudaMemcpyAsync(&herr, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  if (herr) return false;
  if (sym) {
    mirror_upper_oz_kernel<<<grid_for(M * M), 256, 0, s>>>(C, M);
    FTT_LAUNCH();
  }
  return true;
}

}  // namespace

bool gemm_ozaki(int slices, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
                const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
                cudaStream_t s, bool sym) {
  if (M <= 0 || N <= 0) return true;
  if (sym && (M != N || sci != N || scj != 1)) fail(FASTTT_EINVAL, "symmetric GEMM needs a square row-major C");
  if (K <= 0) return false;
  if (slices == 7) return run_ozaki<7>(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci, scj, s, sym);
  if (slices == 3) return run_ozaki<3>(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci, scj, s, sym);
  return false;
}

}  // namespace fasttt
