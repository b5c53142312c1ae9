// Dense GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) with FP64
// operands, by exact bf16 slicing (the error-free splitting of Ozaki, Ogita,
// Oishi & Rump, Numer. Algorithms 59, 2012), with b bits per slice:
//
//   row i of A:    a_ik = 2^{e_i} sum_{s=1..S} q^A_{s,ik} 2^{-bs},  |q_1| <= 2^b, |q_s| <= 2^{b-1} (s > 1)
//   column j of B: b_kj = 2^{f_j} sum_{t=1..S} q^B_{t,kj} 2^{-bt}   (+ rounding below 2^{-bS-1})
//
// Every slice q is an integer of at most 8 significant bits, exact in bf16, and
// every product q^A q^B is exact in FP32.  Products are grouped by level
// g = s + t (g <= S + 1; the rest is below 2^{-bS} of |a||b|):
//   (A B)_ij = 2^{e_i + f_j} sum_g 2^{-bg} sum_{s+t=g} sum_k q^A_{s,ik} q^B_{t,kj}.
// One tcgen05.mma (kind::f16, bf16 x bf16 -> FP32 in TMEM) per slice pair and K
// step of 16 accumulates a level.  A level's sum over a window of KD values of k
// is an integer below 2^24 (checked at compile time from the digit bounds), so it
// is exact in FP32; after every window the 8 warps read the level accumulators
// out of TMEM (tcgen05.ld) into 64-bit integer registers, packed four levels to an
// integer, and the whole K reduction is exact.  FP64 enters only when the packed
// sums are scaled into C.  FP64-level products: S = 8 slices of b = 7 bits
// (levels below 2^{-63} dropped), windows of 384.  FP32-level products (mixed
// precision): S = 3 slices of b = 8 bits, windows of 192.
//
// Tiles: 128 (M) x 64 (N) per CTA; K in stages of 32 (64-byte bf16 rows) through
// a two-deep shared-memory ring.  The splitting kernels write every operand as the
// shared-memory images of its tiles, already in the 64-byte swizzle, so a stage is
// S contiguous bulk copies (cp.async.bulk) per operand, consumed by K-major SW64
// UMMA descriptors; the copy of stage k+1 is issued as soon as the MMAs of stage
// k-1 have released their buffer.  Every mbarrier wait is bounded; a block that gives
// up raises a sticky device flag, waits (bounded) for its copies and MMAs in
// flight, frees its TMEM and returns; the call that launched it then fails with
// FASTTT_ETIMEOUT when the flag is read (ozaki_take_timeout, once per call).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "dense.cuh"

namespace fasttt {

namespace {

constexpr int kBM = 128, kBN = 64, kBK = 64;   // kBK: K padding of the slices
constexpr int kBKs = 32;                         // K per pipeline stage (64-byte rows)

// Set by a block that gave up on a bounded wait; read and cleared by
// ozaki_take_timeout (sticky across the calls in between, one per device).
__device__ int g_oz_timeout = 0;
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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long spins = kMbarSpins) {
  for (long long it = 0; it < spins; ++it) {
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

// Contiguous bulk copy global -> shared (size a multiple of 16 bytes, both 16-byte aligned).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// K-major operand tile of rows x 32 bf16 (64-byte rows), 64-byte swizzle: 8-row
// groups 512 bytes apart (stride byte offset), descriptor version 1, layout 4.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
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

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread), one wait.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Largest level sum per k: level g collects the pairs s + t = g of digits bounded
// by 2^BITS (the top one) and 2^{BITS-1} (the others).
template <int S, int BITS>
__host__ __device__ constexpr long long oz_level_max() {
  long long mx = 0;
  for (int g = 2; g <= S + 1; ++g) {
    long long sum = 0;
    for (int s = 1; s <= S; ++s) {
      const int t = g - s;
      if (t < 1 || t > S) continue;
      sum += ((s == 1) ? (1ll << BITS) : (1ll << (BITS - 1))) * ((t == 1) ? (1ll << BITS) : (1ll << (BITS - 1)));
    }
    mx = sum > mx ? sum : mx;
  }
  return mx;
}

// C tile (128 x 64) of alpha 2^{e_i + f_j} sum_g 2^{-BITS g} L_g + beta C.  K runs
// in stages of 32 through a two-deep shared-memory ring (bulk copies of pre-swizzled
// tile images); the
// level sums accumulate in TMEM over windows of KD and are then drained exactly
// into 64-bit integers (KD times the largest level sum per k stays below 2^24).
template <int S, int BITS, int KD, int BN, int NST>
__global__ void __launch_bounds__(kThreads, 1)
    ozaki_gemm_kernel(const __nv_bfloat16* __restrict__ qa, const __nv_bfloat16* __restrict__ qb, int64_t M,
                      int64_t N, int64_t Kp, int64_t Mp, int64_t Np, const int* __restrict__ ea,
                      const int* __restrict__ fb, double alpha, double beta, double* __restrict__ C, int64_t sci,
                      int64_t scj, bool sym, long long spins) {
  static_assert((long long)KD * oz_level_max<S, BITS>() < (1ll << 24), "level sums of a window must stay exact");
  static_assert(KD % kBKs == 0, "windows are whole stages");
  static_assert(S * BN <= 512 && BN % 64 == 0, "the level accumulators must fit TMEM");
  constexpr int kLevels = S;                       // g = 2 .. S + 1
  constexpr uint32_t kCols = (kLevels * BN <= 256) ? 256 : 512;
  constexpr uint32_t kTileA = kBM * kBKs * 2, kTileB = BN * kBKs * 2;
  constexpr uint32_t kStageBytes = S * (kTileA + kTileB);
  constexpr int kWindow = KD / kBKs;
  constexpr int kCPT = BN / 2;                     // columns per thread in the drain
  const int bm = blockIdx.x, bn = blockIdx.y;
  if (sym && (int64_t)bm * kBM >= (int64_t)(bn + 1) * BN) return;   // strictly below the diagonal
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[NST], empty_bar[NST], drain_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) {
      mbar_init(&full_bar[q], 1);
      mbar_init(&empty_bar[q], 1);
    }
    mbar_init(&drain_bar, 1);
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
  const uint32_t idesc = idesc_bf16(kBM, BN);
  const uint64_t desc0 = sw64_desc(smem_u32(smem));
  // Exact integer accumulation of the level sums over K: the first kHiLevels levels
  // in hi (level g weighted 2^{BITS(kHiLevels+1-g)}), the rest in lo (weighted
  // 2^{BITS(S+1-g)}); a window adds below 2^{24+3 BITS} to each.
  constexpr int kHiLevels = (S < 4) ? S : 4;
  constexpr int kLoLevels = S - kHiLevels;
  constexpr int kLoN = (kLoLevels > 0) ? kCPT : 1;
  long long hi[kCPT], lo[kLoN];
#pragma unroll
  for (int c = 0; c < kCPT; ++c) hi[c] = 0;
#pragma unroll
  for (int c = 0; c < kLoN; ++c) lo[c] = 0;
  const int nk = (int)(Kp / kBKs);
  const int quarter = warp & 3, half = warp >> 2;
  auto load_stage = [&](int st, int kc) {
    unsigned char* base = smem + st * kStageBytes;
    mbar_arrive_expect_tx(&full_bar[st], kStageBytes);
    // tile images: [slice][k block][64-row tile] of 4 KB (see oz_slice_kernel); the A
    // tile is two consecutive 64-row images, the B tile BN / 64
    const int64_t nkb = Kp / kBKs;
    for (int q = 0; q < S; ++q) {
      bulk_load(base + q * kTileA, qa + (((int64_t)q * nkb + kc) * (Mp / 64) + (int64_t)bm * 2) * 2048, kTileA,
                &full_bar[st]);
      bulk_load(base + S * kTileA + q * kTileB,
                qb + (((int64_t)q * nkb + kc) * (Np / 64) + (int64_t)bn * (BN / 64)) * 2048, kTileB, &full_bar[st]);
    }
  };
  // issuing thread's view of the copies in flight (for a clean exit after a timeout)
  bool tma_pending[NST];
  uint32_t tma_phase[NST], empty_phase[NST];
#pragma unroll
  for (int q = 0; q < NST; ++q) { tma_pending[q] = false; tma_phase[q] = 0; empty_phase[q] = 0; }
  if (tid == 0)
    for (int st = 0; st < NST && st < nk; ++st) { load_stage(st, st); tma_pending[st] = true; }
  bool ok = true, drain_pending = false;
  uint32_t drain_phase = 0;
  for (int w0 = 0; w0 < nk; w0 += kWindow) {
    const int w1 = (w0 + kWindow < nk) ? w0 + kWindow : nk;
    if (tid == 0 && !abort_flag) {
      for (int kc = w0; kc < w1; ++kc) {
        const int st = kc % NST;
        if (!mbar_wait(&full_bar[st], tma_phase[st], spins)) { abort_flag = 1; break; }
        tma_pending[st] = false;
        tma_phase[st] ^= 1;
        tc_fence_after();
        // descriptors: the address field is addr >> 4 in the low bits (no carry: shared
        // memory addresses stay below 2^18), so tile and K offsets are plain additions
        const uint64_t dst = desc0 + (uint64_t)((st * kStageBytes) >> 4);
        const uint32_t first = (kc == w0) ? 0u : 1u;   // the window's first stage starts every level
#pragma unroll
        for (int q = 1; q <= S; ++q) {
#pragma unroll
          for (int t = 1; t + q <= S + 1; ++t) {
            const int l = q + t - 2;
            const uint64_t da = dst + (uint64_t)(((q - 1) * kTileA) >> 4);
            const uint64_t db = dst + (uint64_t)((S * kTileA + (t - 1) * kTileB) >> 4);
            // the first product of level l in the window is (q, t) = (1, l + 1) at K step 0
            const uint32_t acc0 = (q == 1) ? first : 1u;
#pragma unroll
            for (int kk = 0; kk < kBKs / 16; ++kk)   // K steps of 16 bf16 = 32 bytes
              umma_bf16(tbase + (uint32_t)(l * BN), da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc,
                        kk == 0 ? acc0 : 1u);
          }
        }
        umma_commit(&empty_bar[st]);
        // refill the stage of step kc - 1 (its MMAs run ahead of these) with step kc - 1 + NST
        if (kc >= 1 && kc - 1 + NST < nk) {
          const int o = (kc - 1) % NST;
          if (!mbar_wait(&empty_bar[o], empty_phase[o], spins)) { abort_flag = 1; break; }
          empty_phase[o] ^= 1;
          load_stage(o, kc - 1 + NST);
          tma_pending[o] = true;
        }
      }
      if (!abort_flag) umma_commit(&drain_bar);
    }
    // the issuing thread gave up (its pipeline waits use the caller's bound): no drain
    // commit was made for this window; the abort path below waits for what is in flight
    if (__syncthreads_or(abort_flag)) { ok = false; break; }
    const bool got = mbar_wait(&drain_bar, drain_phase);
    if (__syncthreads_or(!got)) {   // the window's commit is still outstanding
      drain_pending = true;
      ok = false;
      break;
    }
    drain_phase ^= 1;
    tc_fence_after();
    // drain: TMEM lanes 32 * quarter .. (tile rows), columns kCPT * half .. of every level
    const uint32_t lane_base = tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * kCPT);
#pragma unroll
    for (int l = 0; l < kLevels; ++l) {
#pragma unroll
      for (int c0 = 0; c0 < kCPT; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(lane_base + (uint32_t)(l * BN + c0), r);
        if (l < kHiLevels) {
          const int sh = BITS * (kHiLevels - 1 - l);
#pragma unroll
          for (int c = 0; c < 32; ++c) hi[c0 + c] += (long long)__float2int_rn(__uint_as_float(r[c])) << sh;
        } else {
          const int sh = BITS * (kLevels - 1 - l);
#pragma unroll
          for (int c = 0; c < 32; ++c) lo[(c0 + c) % kLoN] += (long long)__float2int_rn(__uint_as_float(r[c])) << sh;
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (ok) {
    const int64_t i = (int64_t)bm * kBM + quarter * 32 + lane;
    if (i < M) {
      // value = 2^{e_i + f_j} alpha (2^{-BITS(kHiLevels+1)} hi + 2^{-BITS(S+1)} lo)
      const double whi = ldexp(1.0, -BITS * (kHiLevels + 1)), wlo = ldexp(1.0, -BITS * (S + 1));
      const int ei = ea[i];
#pragma unroll
      for (int c = 0; c < kCPT; ++c) {
        const int64_t j = (int64_t)bn * BN + half * kCPT + c;
        if (j >= N) continue;
        double* cp = C + i * sci + j * scj;
        const double sum = fma((double)hi[c], whi, (kLoLevels > 0) ? (double)lo[c % kLoN] * wlo : 0.0);
        const double v = ldexp(alpha * sum, ei + fb[j]);
        *cp = (beta == 0.0) ? v : fma(beta, *cp, v);
      }
    }
  } else {
    // give the copies and MMAs still in flight a bounded wait before TMEM is freed
    if (tid == 0) {
      for (int st = 0; st < NST; ++st)
        if (tma_pending[st]) mbar_wait(&full_bar[st], tma_phase[st]);
      // one commit after every MMA issued: wait for it (and for the window's own commit
      // first, if that one is still outstanding), so no arrive lands after the exit
      umma_commit(&drain_bar);
      if (drain_pending) {
        mbar_wait(&drain_bar, drain_phase);
        drain_phase ^= 1;
      }
      mbar_wait(&drain_bar, drain_phase);
      atomicOr(&g_oz_timeout, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols) : "memory");
}

// ------------------------------------------------------------------ splitting
// Row i of an operand X (rows x cols, X(i, k) = X[i*s_row + k*s_col]) is split
// as follows.  e_i is the exponent with max_k |x_ik| < 2^{e_i} (frexp's), and
//   R_ik = round(x_ik 2^{8S - e_i})          (|R| <= 2^{8S}, an exact integer)
// is written in balanced base-256 digits: the S-1 low digits d in [-128, 127]
// and the top digit q_1 = (R - low part) / 2^{8(S-1)} with |q_1| <= 256, so that
// x_ik 2^{-e_i} = sum_s q_s 2^{-8s} up to the dropped |x| 2^{-8S-1} rounding.
// Everything is integer arithmetic on the bit pattern (no FP64 instruction):
// the max of |x| is the max of the sign-cleared bits, R is the 53-bit
// significand shifted into place, and a digit becomes bf16 exactly (at most 8
// significant bits) through the FP32 pattern of a small integer.

constexpr unsigned long long kAbsMask = 0x7FFFFFFFFFFFFFFFull;

// mx[i] = max over k of the sign-cleared bits of x_ik (atomic over column chunks;
// mx zeroed by the caller).  by_row: rows are contiguous (s_row = 1), one thread
// per row; otherwise one warp per row with the lanes along k.
__global__ void oz_rowmax_kernel(const double* __restrict__ X, int64_t rows, int64_t cols, int64_t s_row,
                                 int64_t s_col, int64_t kchunk, bool by_row, unsigned long long* __restrict__ mx) {
  const int64_t k0 = (int64_t)blockIdx.y * kchunk;
  const int64_t k1 = min(cols, k0 + kchunk);
  unsigned long long m = 0;
  if (by_row) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
#pragma unroll 8
    for (int64_t k = k0; k < k1; ++k)
      m = max(m, (unsigned long long)__double_as_longlong(__ldg(X + i + k * s_col)) & kAbsMask);
    if (m) atomicMax(mx + i, m);
  } else {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= rows) return;
    const double* row = X + i * s_row;
#pragma unroll 4
    for (int64_t k = k0 + lane; k < k1; k += 32)
      m = max(m, (unsigned long long)__double_as_longlong(__ldg(row + k * s_col)) & kAbsMask);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, (unsigned long long)__shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && m) atomicMax(mx + i, m);
  }
}

// frexp's exponent of the double with sign-cleared bits a (0 for zero).
__device__ __forceinline__ int oz_exp(unsigned long long a) {
  if (a == 0) return 0;
  const int eb = (int)(a >> 52);
  if (eb) return eb - 1022;                 // a in [2^{eb-1023}, 2^{eb-1022})
  return (64 - __clzll((long long)a)) - 1074;   // subnormal: a = m 2^-1074
}

// The S balanced digits of x 2^{-e} (q[0] the top one), BITS bits per digit.
template <int S, int BITS>
__device__ __forceinline__ void oz_digits(double x, int e, int (&q)[S]) {
  const long long b = __double_as_longlong(x);
  const unsigned long long a = (unsigned long long)b & kAbsMask;
  long long R = 0;
  if (a != 0) {
    const int eb = (int)(a >> 52);
    const unsigned long long m = (a & 0xFFFFFFFFFFFFFull) | (eb ? (1ull << 52) : 0ull);
    // |x| = m 2^{E}, E = max(eb, 1) - 1075;  R = round(m 2^{sh}), sh <= 8S - 53 for normal x
    const int sh = (eb ? eb : 1) - 1075 + S * BITS - e;
    unsigned long long u;
    if (sh >= 0) u = m << sh;
    else if (sh > -64) u = (m + (1ull << (-sh - 1))) >> (-sh);
    else u = 0;
    R = (b < 0) ? -(long long)u : (long long)u;
  }
  constexpr long long kHalf = 1ll << (BITS - 1), kMask = (1ll << BITS) - 1;
#pragma unroll
  for (int t = S - 1; t >= 1; --t) {
    const long long dl = ((R + kHalf) & kMask) - kHalf;
    q[t] = (int)dl;
    R = (R - dl) >> BITS;   // exact: R - dl is a multiple of 2^BITS
  }
  q[0] = (int)R;
}

// bf16 bits of a small integer (|d| <= 2^8): exact through the FP32 pattern.
__device__ __forceinline__ uint32_t oz_bf16_bits(int d) {
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;   // 1.5 * 2^23 magic: exact for |d| < 2^22
  return __float_as_uint(f) >> 16;
}

// Slices q[s][i][k] (bf16, rows_p x cols_p per slice, zero padded) and row
// exponents ex[i], from the row maxima.  One 64 x 64 tile per block iteration:
// loaded through shared memory along X's contiguous dimension, written along k.
template <int S, int BITS>
__global__ void __launch_bounds__(256) oz_slice_kernel(const double* __restrict__ X, int64_t rows, int64_t cols,
                                                       int64_t s_row, int64_t s_col, bool by_row, int64_t rows_p,
                                                       int64_t cols_p, const unsigned long long* __restrict__ mx,
                                                       int* __restrict__ ex, __nv_bfloat16* __restrict__ q) {
  __shared__ double t[64][65];
  __shared__ int es[64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tiles_c = cols_p / 64, ntiles = (rows_p / 64) * tiles_c;
  uint32_t* q32 = reinterpret_cast<uint32_t*>(q);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = (tile / tiles_c) * 64, c0 = (tile % tiles_c) * 64;
    if (by_row) {
      for (int e = threadIdx.x; e < 64 * 64; e += 256) {
        const int cc = e >> 6, rr = e & 63;
        const int64_t i = r0 + rr, k = c0 + cc;
        t[rr][cc] = (i < rows && k < cols) ? __ldg(X + i + k * s_col) : 0.0;
      }
    } else {
      for (int e = threadIdx.x; e < 64 * 64; e += 256) {
        const int rr = e >> 6, cc = e & 63;
        const int64_t i = r0 + rr, k = c0 + cc;
        t[rr][cc] = (i < rows && k < cols) ? __ldg(X + i * s_row + k * s_col) : 0.0;
      }
    }
    if (threadIdx.x < 64) {
      const int64_t i = r0 + threadIdx.x;
      const int e = (i < rows) ? oz_exp(mx[i]) : 0;
      es[threadIdx.x] = e;
      if (c0 == 0 && i < rows) ex[i] = e;
    }
    __syncthreads();
    // Stored as the shared-memory images the GEMM's UMMA descriptors read: per slice,
    // per k block of 32 and per 64-row tile a 4 KB block of 64-byte rows (32 bf16), its
    // 16-byte chunk c of row r at position c ^ ((r >> 1) & 3) (the 64-byte swizzle).
    // Lanes 0-15 write k block c0/32 of the row, lanes 16-31 the next one.
    const int64_t nkb = cols_p / 32, nrt = rows_p / 64;
    const int kbl = lane >> 4, kk = 2 * (lane & 15), ch = kk >> 3, el = kk & 7;
#pragma unroll 1
    for (int rr = warp * 8; rr < warp * 8 + 8; ++rr) {
      const int e = es[rr];
      int d0[S], d1[S];
      oz_digits<S, BITS>(t[rr][2 * lane], e, d0);
      oz_digits<S, BITS>(t[rr][2 * lane + 1], e, d1);
      const int64_t row = r0 + rr, kb = c0 / 32 + kbl;
      const int r = (int)(row & 63);
      const int64_t within = (int64_t)r * 16 + ((ch ^ ((r >> 1) & 3)) * 4) + (el >> 1);   // in 4-byte words
#pragma unroll
      for (int sl = 0; sl < S; ++sl)
        q32[(((int64_t)sl * nkb + kb) * nrt + (row >> 6)) * 1024 + within] =
            oz_bf16_bits(d0[sl]) | (oz_bf16_bits(d1[sl]) << 16);
    }
    __syncthreads();
  }
}

// Row exponents and slices of the operand X (see above).
template <int S, int BITS>
void oz_split(const double* X, int64_t rows, int64_t cols, int64_t s_row, int64_t s_col, int64_t rows_p,
              int64_t cols_p, int* ex, __nv_bfloat16* q, cudaStream_t s) {
  DBuf<unsigned long long> mx((size_t)rows, s);
  FTT_CUDA(cudaMemsetAsync(mx.get(), 0, mx.bytes(), s));
  const bool by_row = (s_row == 1 && s_col != 1);
  // short chunks: a thread's loads form one dependent max chain, so more blocks with
  // shorter chains finish sooner (one atomic per row and chunk)
  int64_t kchunk = by_row ? 64 : 512;
  kchunk = std::max<int64_t>(kchunk, ceil_div(cols, 65535));
  const dim3 g1((unsigned)(by_row ? ceil_div(rows, 256) : ceil_div(rows, 8)), (unsigned)ceil_div(cols, kchunk));
  oz_rowmax_kernel<<<g1, 256, 0, s>>>(X, rows, cols, s_row, s_col, kchunk, by_row, mx.get());
  FTT_LAUNCH();
  const int64_t ntiles = (rows_p / 64) * (cols_p / 64);
  oz_slice_kernel<S, BITS><<<(unsigned)std::min<int64_t>(ntiles, (int64_t)kNumSMs * 8), 256, 0, s>>>(
      X, rows, cols, s_row, s_col, by_row, rows_p, cols_p, mx.get(), ex, q);
  FTT_LAUNCH();
}

__global__ void mirror_upper_oz_kernel(double* C, int64_t n, int64_t ldc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (i > j) C[i * ldc + j] = C[j * ldc + i];
  }
}

template <int S, int BITS, int KD, int BN, int NST>
bool run_ozaki(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
               const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
               cudaStream_t s, bool sym) {
  const int64_t Mp = ceil_div(M, kBM) * kBM, Np = ceil_div(N, BN) * BN, Kp = ceil_div(K, kBK) * kBK;
  if ((S * Mp) >= INT32_MAX || (S * Np) >= INT32_MAX || Np / BN > 65535 || Kp >= INT32_MAX) return false;
  // the int64 level accumulators take 2^{37 - 3 BITS} windows
  if (ceil_div(Kp, KD) > (1ll << (37 - 3 * BITS))) return false;
  const size_t smem = (size_t)NST * S * (kBM + BN) * kBKs * 2 + 1024;
  // set on every call: the limit belongs to the current device's context
  if (cudaFuncSetAttribute(ozaki_gemm_kernel<S, BITS, KD, BN, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const bool same = (A == B && M == N && sai == sbj && sak == sbk);
  DBuf<__nv_bfloat16> qa((size_t)S * Mp * Kp, s), qb(same ? 0 : (size_t)S * Np * Kp, s);
  DBuf<int> ea(Mp, s), fb(same ? 0 : Np, s);
  // A rows: a(i, k) = A[i*sai + k*sak]; B^T rows: b(j, k) = B[k*sbk + j*sbj].  When B^T is
  // A itself (a Gram product) its slices are A's, padded to Mp >= Np rows.
  oz_split<S, BITS>(A, M, K, sai, sak, Mp, Kp, ea.get(), qa.get(), s);
  if (!same) oz_split<S, BITS>(B, N, K, sbj, sbk, Np, Kp, fb.get(), qb.get(), s);

  KClock clk;
  kclock_begin(clk, KC_GEMM_OZ, s);
  ozaki_gemm_kernel<S, BITS, KD, BN, NST><<<dim3((unsigned)(Mp / kBM), (unsigned)(Np / BN)), kThreads, smem, s>>>(
      qa.get(), same ? qa.get() : qb.get(), M, N, Kp, Mp, same ? Mp : Np, ea.get(), same ? ea.get() : fb.get(), alpha,
      beta, C, sci, scj, sym, max_spin() > 0 ? (long long)max_spin() : kMbarSpins);
  FTT_LAUNCH();
  kclock_end(clk, (sym ? 1.0 : 2.0) * (double)M * (double)N * (double)K, s);
  if (sym) {
    mirror_upper_oz_kernel<<<grid_for(M * M), 256, 0, s>>>(C, M, sci);
    FTT_LAUNCH();
  }
  return true;
}

}  // namespace

void ozaki_take_timeout(cudaStream_t s) {
  int h = 0;
  const int zero = 0;
  FTT_CUDA(cudaMemcpyFromSymbolAsync(&h, g_oz_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  if (h) {
    FTT_CUDA(cudaMemcpyToSymbolAsync(g_oz_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    note_wait_timeout();
    fail(FASTTT_ETIMEOUT, "tensor-core GEMM: a bounded wait gave up");
  }
}

bool ozaki_clear_timeout(cudaStream_t s) {
  int h = 0;
  const int zero = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_oz_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (h) {
    cudaMemcpyToSymbolAsync(g_oz_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    cudaGetLastError();
  }
  return h != 0;
}

bool gemm_ozaki(int slices, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
                const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
                cudaStream_t s, bool sym) {
  if (M <= 0 || N <= 0) return true;
  if (sym && (M != N || sci < N || scj != 1)) fail(FASTTT_EINVAL, "symmetric GEMM needs a square row-major C");
  if (K <= 0) return false;
  // FP64 level: 8 slices of 7 bits (level sums exact over windows of 384: 384 x 40960 < 2^24);
  // FP32 level: 3 slices of 8 bits (windows of 192: 192 x 81920 < 2^24)
  // FP64 level: 64-column tiles (8 levels x 64 TMEM columns), two-stage ring; FP32 level:
  // 128-column tiles (3 levels x 128 columns), four-stage ring
  if (slices == 7)
    return run_ozaki<8, 7, 384, 64, 2>(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci, scj, s, sym);
  if (slices == 3)
    return run_ozaki<3, 8, 192, 128, 4>(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci, scj, s, sym);
  return false;
}

}  // namespace fasttt
