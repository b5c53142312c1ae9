// Block-sparse bond of the first SVD sweep (Alg. 6, bonds k = p+1..d-1) for
// cores too large to materialise.  Entering bond k, G_k = W_{k-1} x_1 P_k with
// P_k the right quasi-permutation core of Alg. 4: every right group alpha
// (= alpha_{k-1}) is the tuple (i_k, beta) with beta = alpha_k, so the
// k-unfolding Z = unfold_2(G_k) (rows (a, i), a < r_{k-1}, i < n_k; columns beta)
// holds column alpha of W at rows (., i_alpha) of column beta_alpha and nothing
// else.  Hence
//   Z Z^T, block (i, i') = sum over alpha, alpha' with beta_alpha = beta_alpha',
//                          i_alpha = i, i_alpha' = i' of  w_alpha w_alpha'^T,
//   (U^T Z)[:, beta]     = sum over alpha with beta_alpha = beta of U_{i_alpha}^T w_alpha,
// with U_i the r_{k-1} x r rows (., i) of U.  The self pairs alpha = alpha' of
// block (i, i) are the contiguous range of alpha with i_alpha = i (right ids are
// lexicographic ranks of (i_k, alpha_k), so sorted by i_k); the cross pairs
// come from sorting alpha by beta.  Both products run as gathered 64 x 64 x 16
// FP64 tiles (the gemm_f64 tiling), the Gram with split-K chunks added by FP64
// atomics, the projection written per alpha and summed per beta in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "dense.cuh"
#include "sparse_sweep.cuh"

namespace fasttt {

namespace {

constexpr int kT = 64;         // output tile
constexpr int kTK = 16;        // K tile
constexpr int64_t kChunk = 4096;   // pairs per Gram task (split-K)

struct GramTask {
  int32_t i, i2;      // output block (i, i2)
  int64_t q0, q1;     // pair range
};

// Gram tasks: pairs q of [q0, q1); alpha of the left factor = pa ? pa[q] : q,
// right factor = pb ? pb[q] : q.  Output rows a*nk + i, columns a'*nk + i2.
__global__ void __launch_bounds__(256)
    sparse_gram_kernel(const double* __restrict__ Wt, int64_t rp, const GramTask* __restrict__ tasks,
                       const uint32_t* __restrict__ pa, const uint32_t* __restrict__ pb, int64_t nk, int64_t M,
                       int ntile, double* __restrict__ Gram) {
  const GramTask t = tasks[blockIdx.x];
  const int ta = blockIdx.y / ntile, tb = blockIdx.y % ntile;
  const int64_t i0 = (int64_t)ta * kT, j0 = (int64_t)tb * kT;
  __shared__ double As[kTK][kT + 1];
  __shared__ double Bs[kTK][kT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int64_t k0 = t.q0; k0 < t.q1; k0 += kTK) {
    for (int e = threadIdx.x; e < kT * kTK; e += 256) {
      const int kk = e >> 6, ii = e & 63;
      const int64_t q = k0 + kk;
      double x = 0.0, y = 0.0;
      if (q < t.q1) {
        const int64_t al = pa ? (int64_t)pa[q] : q;
        const int64_t al2 = pb ? (int64_t)pb[q] : q;
        if (i0 + ii < rp) x = Wt[al * rp + i0 + ii];
        if (j0 + ii < rp) y = Wt[al2 * rp + j0 + ii];
      }
      As[kk][ii] = x;
      Bs[kk][ii] = y;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t a = i0 + ty + 16 * r;
    if (a >= rp) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t a2 = j0 + tx + 16 * c;
      if (a2 >= rp) continue;
      atomicAdd(Gram + (a * nk + t.i) * M + a2 * nk + t.i2, acc[r][c]);
    }
  }
}

// G <- (G + G^T) / 2 (the atomic sums leave rounding-level asymmetry)
__global__ void symmetrise_kernel(double* G, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (i < j) {
      const double v = 0.5 * (G[i * n + j] + G[j * n + i]);
      G[i * n + j] = v;
      G[j * n + i] = v;
    }
  }
}

// off[i] = first alpha with ridx[alpha] >= i (ridx nondecreasing), i = 0..nk
__global__ void range_starts_kernel(const int32_t* ridx, int64_t A, int64_t nk, int64_t* off) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nk; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = A;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (ridx[mid] < i) lo = mid + 1;
      else hi = mid;
    }
    off[i] = lo;
  }
}

__global__ void beta_keys_kernel(const int32_t* rchild, int64_t A, uint64_t* keys, uint32_t* vals) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A; e += (int64_t)gridDim.x * blockDim.x) {
    keys[e] = (uint64_t)rchild[e];
    vals[e] = (uint32_t)e;
  }
}

// boff[beta] = first position of beta in the sorted keys; every beta in [0, N) occurs
__global__ void beta_starts_kernel(const uint64_t* keys, int64_t A, int64_t N, int64_t* boff) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A; e += (int64_t)gridDim.x * blockDim.x)
    if (e == 0 || keys[e] != keys[e - 1]) boff[keys[e]] = e;
  if (blockIdx.x == 0 && threadIdx.x == 0) boff[N] = A;
}

// cross pairs of sorted position e: (alpha_e, alpha_f) for the other f of its beta segment
__global__ void cross_count_kernel(const uint64_t* keys, const int64_t* boff, int64_t A, int64_t* cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = (int64_t)keys[e];
    cnt[e] = boff[b + 1] - boff[b] - 1;
  }
}

__global__ void cross_emit_kernel(const uint64_t* keys, const uint32_t* vals, const int64_t* boff,
                                  const int64_t* start, int64_t A, const int32_t* ridx, int64_t nk, uint64_t* pkey,
                                  uint32_t* pidx, uint32_t* pa, uint32_t* pb) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = (int64_t)keys[e];
    int64_t w = start[e];
    const uint32_t al = vals[e];
    for (int64_t f = boff[b]; f < boff[b + 1]; ++f) {
      if (f == e) continue;
      const uint32_t al2 = vals[f];
      pkey[w] = (uint64_t)ridx[al] * (uint64_t)nk + (uint64_t)ridx[al2];
      pidx[w] = (uint32_t)w;
      pa[w] = al;
      pb[w] = al2;
      ++w;
    }
  }
}

__global__ void permute_pairs_kernel(const uint32_t* order, const uint32_t* pa, const uint32_t* pb, int64_t P,
                                     uint32_t* pa2, uint32_t* pb2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x) {
    pa2[e] = pa[order[e]];
    pb2[e] = pb[order[e]];
  }
}

__global__ void key_heads_kernel(const uint64_t* keys, int64_t P, int64_t* heads) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x)
    heads[e] = (e == 0 || keys[e] != keys[e - 1]) ? 1 : 0;
}

__global__ void key_segments_kernel(const uint64_t* keys, const int64_t* heads_scan, int64_t P, int64_t* seg_start,
                                    uint64_t* seg_key) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x)
    if (e == 0 || keys[e] != keys[e - 1]) {
      seg_start[heads_scan[e]] = e;
      seg_key[heads_scan[e]] = keys[e];
    }
}

struct ProjTask {
  int32_t i;
  int64_t j0, cnt;   // alpha in [j0, j0 + cnt), cnt <= 64
};

// Yt[alpha, c] = sum_a U[(a*nk + i)*rr + c] * Wt[alpha*rp + a] for the alpha of the task
__global__ void __launch_bounds__(256)
    sparse_project_kernel(const double* __restrict__ U, int64_t rr, const double* __restrict__ Wt, int64_t rp,
                          const ProjTask* __restrict__ tasks, int64_t nk, double* __restrict__ Yt) {
  const ProjTask t = tasks[blockIdx.x];
  const int64_t c0 = (int64_t)blockIdx.y * kT;
  __shared__ double As[kTK][kT + 1];
  __shared__ double Bs[kTK][kT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int64_t k0 = 0; k0 < rp; k0 += kTK) {
    for (int e = threadIdx.x; e < kT * kTK; e += 256) {
      {
        const int kk = e >> 6, ii = e & 63;   // A(c, a) = U[(a*nk + i)*rr + c]
        const int64_t a = k0 + kk, c = c0 + ii;
        As[kk][ii] = (a < rp && c < rr) ? U[(a * nk + t.i) * rr + c] : 0.0;
      }
      {
        const int kb = e & 15, jj = e >> 4;   // B(a, j) = Wt[(j0 + j)*rp + a]
        const int64_t a = k0 + kb;
        Bs[kb][jj] = (a < rp && jj < t.cnt) ? Wt[(t.j0 + jj) * rp + a] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t c = c0 + ty + 16 * r;
    if (c >= rr) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t j = tx + 16 * q;
      if (j >= t.cnt) continue;
      Yt[(t.j0 + j) * rr + c] = acc[r][q];
    }
  }
}

// Wt_k[beta, c] = sum of Yt[alpha, c] over the alpha of beta, in sorted order
__global__ void beta_sum_kernel(const double* Yt, const uint32_t* vals, const int64_t* boff, int64_t N, int64_t rr,
                                double* Wtk) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * rr; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / rr, c = e % rr;
    double s = 0.0;
    for (int64_t f = boff[b]; f < boff[b + 1]; ++f) s += Yt[(int64_t)vals[f] * rr + c];
    Wtk[e] = s;
  }
}

}  // namespace

SparseBond::SparseBond(const double* W, int64_t rp_, int64_t A_, const int32_t* ridx_, const int32_t* rchild_,
                       int64_t nk_, int64_t N_, cudaStream_t s)
    : rp(rp_), A(A_), nk(nk_), N(N_), ridx(ridx_), Wt((size_t)A_ * rp_, s), sorted_keys(A_, s), sorted_vals(A_, s),
      boff(N_ + 1, s), ioff(nk_ + 1, s) {
  transpose_f64(W, rp, A, Wt.get(), s);   // column alpha of W contiguous
  range_starts_kernel<<<grid_for(nk + 1), 256, 0, s>>>(ridx, A, nk, ioff.get());
  FTT_LAUNCH();
  hioff.resize(nk + 1);
  FTT_CUDA(cudaMemcpyAsync(hioff.data(), ioff.get(), sizeof(int64_t) * (nk + 1), cudaMemcpyDeviceToHost, s));
  {
    DBuf<uint64_t> kalt(A, s);
    DBuf<uint32_t> valt(A, s);
    beta_keys_kernel<<<grid_for(A), 256, 0, s>>>(rchild_, A, sorted_keys.get(), sorted_vals.get());
    FTT_LAUNCH();
    radix_sort_pairs(sorted_keys.get(), sorted_vals.get(), kalt.get(), valt.get(), A, bits_for((uint64_t)N), s);
  }
  beta_starts_kernel<<<grid_for(A), 256, 0, s>>>(sorted_keys.get(), A, N, boff.get());
  FTT_LAUNCH();
  FTT_CUDA(cudaStreamSynchronize(s));
}

void SparseBond::gram(double* Gram, cudaStream_t s) const {
  const int64_t M = rp * nk;
  FTT_CUDA(cudaMemsetAsync(Gram, 0, sizeof(double) * M * M, s));
  const int ntile = (int)ceil_div(rp, kT);
  if ((int64_t)ntile * ntile > 65535) fail(FASTTT_ERANK, "block-sparse sweep: rank too large for the Gram tiles");
  KClock clk;
  kclock_begin(clk, KC_GEMM, s);
  double flops = 0.0;
  // self pairs: block (i, i), alpha over the range of i
  std::vector<GramTask> tasks;
  for (int64_t i = 0; i < nk; ++i)
    for (int64_t q = hioff[i]; q < hioff[i + 1]; q += kChunk)
      tasks.push_back({(int32_t)i, (int32_t)i, q, std::min(q + kChunk, hioff[i + 1])});
  flops += 2.0 * (double)A * (double)rp * (double)rp;
  auto launch = [&](const std::vector<GramTask>& tk, const uint32_t* pa, const uint32_t* pb) {
    for (size_t t0 = 0; t0 < tk.size(); t0 += 65535) {
      const size_t nt = std::min<size_t>(65535, tk.size() - t0);
      DBuf<GramTask> dt(nt, s);
      FTT_CUDA(cudaMemcpyAsync(dt.get(), tk.data() + t0, sizeof(GramTask) * nt, cudaMemcpyHostToDevice, s));
      sparse_gram_kernel<<<dim3((unsigned)nt, (unsigned)(ntile * ntile)), 256, 0, s>>>(Wt.get(), rp, dt.get(), pa, pb,
                                                                                      nk, M, ntile, Gram);
      FTT_LAUNCH();
      FTT_CUDA(cudaStreamSynchronize(s));   // the host task list is released after the launch
    }
  };
  if (!tasks.empty()) launch(tasks, nullptr, nullptr);
  // cross pairs: alpha != alpha' of one beta, grouped by output block
  DBuf<int64_t> cnt(A, s), start(A, s);
  cross_count_kernel<<<grid_for(A), 256, 0, s>>>(sorted_keys.get(), boff.get(), A, cnt.get());
  FTT_LAUNCH();
  const int64_t P = exclusive_scan_i64(cnt.get(), start.get(), A, s);
  if (P > 0) {
    if (P >= ((int64_t)1 << 32) - 1) fail(FASTTT_ERANK, "block-sparse sweep: too many cross pairs");
    DBuf<uint64_t> pkey(P, s), pkey2(P, s);
    DBuf<uint32_t> pidx(P, s), pidx2(P, s), pa(P, s), pb(P, s);
    cross_emit_kernel<<<grid_for(A), 256, 0, s>>>(sorted_keys.get(), sorted_vals.get(), boff.get(), start.get(), A, ridx,
                                                  nk, pkey.get(), pidx.get(), pa.get(), pb.get());
    FTT_LAUNCH();
    radix_sort_pairs(pkey.get(), pidx.get(), pkey2.get(), pidx2.get(), P, bits_for((uint64_t)(nk * nk)), s);
    DBuf<uint32_t> spa(P, s), spb(P, s);
    permute_pairs_kernel<<<grid_for(P), 256, 0, s>>>(pidx.get(), pa.get(), pb.get(), P, spa.get(), spb.get());
    FTT_LAUNCH();
    DBuf<int64_t> heads(P, s);
    key_heads_kernel<<<grid_for(P), 256, 0, s>>>(pkey.get(), P, heads.get());
    FTT_LAUNCH();
    const int64_t nseg = exclusive_scan_i64(heads.get(), heads.get(), P, s);
    DBuf<int64_t> seg_start(nseg, s);
    DBuf<uint64_t> seg_key(nseg, s);
    key_segments_kernel<<<grid_for(P), 256, 0, s>>>(pkey.get(), heads.get(), P, seg_start.get(), seg_key.get());
    FTT_LAUNCH();
    std::vector<int64_t> hs(nseg + 1);
    std::vector<uint64_t> hk(nseg);
    FTT_CUDA(cudaMemcpyAsync(hs.data(), seg_start.get(), sizeof(int64_t) * nseg, cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaMemcpyAsync(hk.data(), seg_key.get(), sizeof(uint64_t) * nseg, cudaMemcpyDeviceToHost, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    hs[nseg] = P;
    std::vector<GramTask> ct;
    for (int64_t g = 0; g < nseg; ++g)
      for (int64_t q = hs[g]; q < hs[g + 1]; q += kChunk)
        ct.push_back({(int32_t)(hk[g] / (uint64_t)nk), (int32_t)(hk[g] % (uint64_t)nk), q, std::min(q + kChunk, hs[g + 1])});
    launch(ct, spa.get(), spb.get());
    flops += 2.0 * (double)P * (double)rp * (double)rp;
  }
  kclock_end(clk, flops, s);
  symmetrise_kernel<<<grid_for(M * M), 256, 0, s>>>(Gram, M);
  FTT_LAUNCH();
}

void SparseBond::project(const double* U, int64_t rr, DBuf<double>& W_out, cudaStream_t s) const {
  // Yt[alpha] = U_{i_alpha}^T w_alpha, tasks of up to 64 alpha within one i
  std::vector<ProjTask> tasks;
  for (int64_t i = 0; i < nk; ++i)
    for (int64_t j = hioff[i]; j < hioff[i + 1]; j += kT)
      tasks.push_back({(int32_t)i, j, std::min<int64_t>(kT, hioff[i + 1] - j)});
  DBuf<double> Yt((size_t)A * rr, s);
  KClock clk;
  kclock_begin(clk, KC_GEMM, s);
  const unsigned gy = (unsigned)ceil_div(rr, kT);
  for (size_t t0 = 0; t0 < tasks.size(); t0 += 65535) {
    const size_t nt = std::min<size_t>(65535, tasks.size() - t0);
    DBuf<ProjTask> dt(nt, s);
    FTT_CUDA(cudaMemcpyAsync(dt.get(), tasks.data() + t0, sizeof(ProjTask) * nt, cudaMemcpyHostToDevice, s));
    sparse_project_kernel<<<dim3((unsigned)nt, gy), 256, 0, s>>>(U, rr, Wt.get(), rp, dt.get(), nk, Yt.get());
    FTT_LAUNCH();
    FTT_CUDA(cudaStreamSynchronize(s));
  }
  kclock_end(clk, 2.0 * (double)A * (double)rp * (double)rr, s);
  DBuf<double> Wtk((size_t)N * rr, s);
  beta_sum_kernel<<<grid_for(N * rr), 256, 0, s>>>(Yt.get(), sorted_vals.get(), boff.get(), N, rr, Wtk.get());
  FTT_LAUNCH();
  W_out = DBuf<double>((size_t)rr * N, s);
  transpose_f64(Wtk.get(), N, rr, W_out.get(), s);   // W_k (rr x N row-major)
}

}  // namespace fasttt
