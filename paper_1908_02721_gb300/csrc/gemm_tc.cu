// Mixed-precision GEMM on the tensor cores: FP64 operands are split as
// x = hi + lo with hi = tf32(x), lo = tf32(x - hi), and C = A B is accumulated in
// FP32 from the three products lo*hi + hi*lo + hi*hi (the "3xTF32" split of
// Ootomo & Yokota, 2022), which recovers FP32-level accuracy from TF32 inputs.
//
// Tile 64 x 128 x 16 per 256-thread block, 8 warps as 2 (M) x 4 (N), each warp
// 32 x 32 from 2 x 4 mma.sync.m16n8k8 TF32 tiles.  Operands are read from FP64
// memory with arbitrary element strides (the gemm_f64 convention), split while
// being staged into shared memory (k-major, padded to avoid bank conflicts).
// Every 128 of K the FP32 MMA accumulators are added into compensated (TwoSum)
// FP32 pairs, so the rounding of the K reduction stays ~1e-7 for any K.
#include <cuda_runtime.h>

#include "dense.cuh"

namespace fasttt {
namespace {

constexpr int BM = 64, BN = 128, BK = 16, PAD = 4;
constexpr int kFlushTiles = 8;   // MMA accumulators are folded into the compensated sum every 8 x 16 = 128 of K

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// (hi, lo) += x with Knuth's TwoSum: the running sum keeps ~2 x 24 bits, so the
// FP32 rounding of the long K reduction does not grow with K.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}

// 8 warps as 2 (M) x 4 (N), each warp 32 x 32 from 2 x 4 mma.sync.m16n8k8 tiles.
__global__ void __launch_bounds__(256)
    gemm_tf32x3_kernel(int64_t M, int64_t N, int64_t K, double alpha, const double* __restrict__ A, int64_t sai,
                       int64_t sak, const double* __restrict__ B, int64_t sbk, int64_t sbj, double beta,
                       double* __restrict__ C, int64_t sci, int64_t scj, bool sym) {
  const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
  if (sym && i0 >= j0 + BN) return;   // tile strictly below the diagonal: mirrored later
  __shared__ uint32_t Ah[BK][BM + PAD], Al[BK][BM + PAD];
  __shared__ uint32_t Bh[BK][BN + PAD], Bl[BK][BN + PAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int wm = warp >> 2, wn = warp & 3;           // warp tile origin: (wm*32, wn*32)
  float acc[2][4][4], shi[2][4][4], slo[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = shi[a][b][c] = slo[a][b][c] = 0.f;
  const bool a_k_fast = (sak == 1), b_k_fast = (sbk == 1);
  int tiles = 0;
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / 256; ++r) {
      const int e = tid + r * 256;
      int kk, ii;
      if (a_k_fast) { kk = e & (BK - 1); ii = e / BK; } else { kk = e / BM; ii = e & (BM - 1); }
      const int64_t gi = i0 + ii, gk = k0 + kk;
      const float x = (gi < M && gk < K) ? (float)A[gi * sai + gk * sak] : 0.f;
      const uint32_t h = to_tf32(x);
      Ah[kk][ii] = h;
      Al[kk][ii] = to_tf32(x - __uint_as_float(h));
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / 256; ++r) {
      const int e = tid + r * 256;
      int kb, jj;
      if (b_k_fast) { kb = e & (BK - 1); jj = e / BK; } else { kb = e / BN; jj = e & (BN - 1); }
      const int64_t gj = j0 + jj, gkb = k0 + kb;
      const float y = (gkb < K && gj < N) ? (float)B[gkb * sbk + gj * sbj] : 0.f;
      const uint32_t hb = to_tf32(y);
      Bh[kb][jj] = hb;
      Bl[kb][jj] = to_tf32(y - __uint_as_float(hb));
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 8) {
      uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r0 = wm * 32 + mi * 16 + gid;
        ah[mi][0] = Ah[ks + tig][r0];     al[mi][0] = Al[ks + tig][r0];
        ah[mi][1] = Ah[ks + tig][r0 + 8]; al[mi][1] = Al[ks + tig][r0 + 8];
        ah[mi][2] = Ah[ks + tig + 4][r0];     al[mi][2] = Al[ks + tig + 4][r0];
        ah[mi][3] = Ah[ks + tig + 4][r0 + 8]; al[mi][3] = Al[ks + tig + 4][r0 + 8];
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c0 = wn * 32 + ni * 8 + gid;
        bh[ni][0] = Bh[ks + tig][c0];     bl[ni][0] = Bl[ks + tig][c0];
        bh[ni][1] = Bh[ks + tig + 4][c0]; bl[ni][1] = Bl[ks + tig + 4][c0];
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
          mma_tf32(acc[mi][ni], al[mi], bh[ni]);
          mma_tf32(acc[mi][ni], ah[mi], bl[ni]);
          mma_tf32(acc[mi][ni], ah[mi], bh[ni]);
        }
    }
    __syncthreads();
    if (++tiles == kFlushTiles || k0 + BK >= K) {
      tiles = 0;
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            two_sum_add(shi[a][b][c], slo[a][b][c], acc[a][b][c]);
            acc[a][b][c] = 0.f;
          }
    }
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t gi = i0 + wm * 32 + mi * 16 + gid + ((c & 2) ? 8 : 0);
        const int64_t gj = j0 + wn * 32 + ni * 8 + 2 * tig + (c & 1);
        if (gi < M && gj < N) {
          double* cp = C + gi * sci + gj * scj;
          const double v = alpha * ((double)shi[mi][ni][c] + (double)slo[mi][ni][c]);
          *cp = (beta == 0.0) ? v : fma(beta, *cp, v);
        }
      }
}

__global__ void mirror_upper_tc_kernel(double* C, int64_t n, int64_t ldc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (i > j) C[i * ldc + j] = C[j * ldc + i];
  }
}

}  // namespace

void gemm_tf32x3(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sai, int64_t sak,
                 const double* B, int64_t sbk, int64_t sbj, double beta, double* C, int64_t sci, int64_t scj,
                 cudaStream_t s, bool sym) {
  if (M <= 0 || N <= 0) return;
  if (sym && (M != N || sci < N || scj != 1)) fail(FASTTT_EINVAL, "symmetric GEMM needs a square row-major C");
  const int64_t gx = ceil_div(M, BM), gy = ceil_div(N, BN);
  if (gy > 65535) fail(FASTTT_ERANK, "GEMM: N too large");
  KClock clk;
  kclock_begin(clk, KC_GEMM_TC, s);
  gemm_tf32x3_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(M, N, K, alpha, A, sai, sak, B, sbk, sbj,
                                                                      beta, C, sci, scj, sym);
  FTT_LAUNCH();
  kclock_end(clk, (sym ? 1.0 : 2.0) * (double)M * (double)N * (double)K + (sym ? (double)M * K : 0.0), s);
  if (sym) {
    mirror_upper_tc_kernel<<<grid_for(M * M), 256, 0, s>>>(C, M, sci);
    FTT_LAUNCH();
  }
}

}  // namespace fasttt
