// S1-S5 of FastTT on the GPU: ingest, lexicographic prefix/suffix ranks (the
// closed form of Alg. 5 applied along Alg. 4's sweeps), Alg. 9 and the middle
// unfolding of the fiber core V (Sec. 3.1-3.2, 3.6).
//
// Every level is one stable radix sort of 64-bit keys (alpha * n + i or
// i * r~ + alpha) with the entry position as value, then head flags and a scan:
// rank = number of distinct smaller keys, i.e. the ascending-row numbering of
// Alg. 5.  All entries of a fiber share their keys, so ranking per entry equals
// ranking per fiber.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "group.cuh"

namespace fasttt {

namespace {

struct DimsArg {
  int64_t n[FASTTT_MAX_D];
};

// ---------------------------------------------------------------- S1 kernels

template <typename V>
__global__ void ingest_check_kernel(const int32_t* idx, const V* vals, int64_t nnz, int d, DimsArg dims,
                                    int64_t* keep, unsigned* err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    unsigned bad = 0;
    for (int k = 0; k < d; ++k) {
      const int32_t i = idx[(int64_t)k * nnz + e];
      if (i < 0 || (int64_t)i >= dims.n[k]) bad |= 1u;
    }
    const double v = (double)vals[e];
    if (!isfinite(v)) bad |= 2u;
    if (bad) atomicOr(err, bad);
    keep[e] = (v != 0.0) ? 1 : 0;
  }
}

template <typename V>
__global__ void ingest_compact_kernel(const int32_t* idx, const V* vals, int64_t nnz, int d,
                                      const int64_t* pos, int64_t kept, int32_t* idx_out,
                                      double* vals_out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)vals[e];
    if (v == 0.0) continue;
    const int64_t q = pos[e];
    vals_out[q] = v;
    for (int k = 0; k < d; ++k) idx_out[(int64_t)k * kept + q] = idx[(int64_t)k * nnz + e];
  }
}

// Fixed-order sum of squares: a fixed grid of per-block partials (grid-stride
// order, fixed shuffle tree), then one block sums the partials in order.
constexpr int kNormBlocks = 2 * kNumSMs;

__global__ void __launch_bounds__(256) sumsq_partial_kernel(const double* v, int64_t n, double* partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma(v[i], v[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void sum_partials_kernel(const double* partial, int n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += partial[i];
    *out = t;
  }
}

// ---------------------------------------------------------------- level keys

// key = hi * mul + lo (hi or lo may be null = 0); value = entry position
__global__ void make_key_kernel(const int32_t* hi, int64_t mul, const int32_t* lo, int64_t n,
                                uint64_t* keys, uint32_t* vals) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = hi ? (uint64_t)(uint32_t)hi[e] : 0ull;
    const uint64_t l = lo ? (uint64_t)(uint32_t)lo[e] : 0ull;
    keys[e] = h * (uint64_t)mul + l;
    vals[e] = (uint32_t)e;
  }
}

// distinct key -> (key / mul, key % mul) as int32 pairs
__global__ void decode_kernel(const uint64_t* uniq, int64_t count, int64_t mul, int32_t* hi, int32_t* lo) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = uniq[j];
    hi[j] = (int32_t)(k / (uint64_t)mul);
    lo[j] = (int32_t)(k % (uint64_t)mul);
  }
}

__global__ void dup_check_kernel(const uint64_t* keys, int64_t n, unsigned* err) {
  for (int64_t i = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (keys[i] == keys[i - 1]) atomicOr(err, 4u);
}

__global__ void combine_key_kernel(uint64_t* keys, const int32_t* col, int64_t ncols, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    keys[e] = keys[e] * (uint64_t)ncols + (uint64_t)(uint32_t)col[e];
}

__global__ void mid_gather_kernel(const uint64_t* keys, const uint32_t* pos, int64_t n, int64_t ncols,
                                  const double* vals, int64_t* row, int64_t* col, double* val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    row[i] = (int64_t)(k / (uint64_t)ncols);
    col[i] = (int64_t)(k % (uint64_t)ncols);
    val[i] = vals[pos[i]];
  }
}

// One ranking level: alpha_out[e] = dense rank of (hi[e]*mul + lo[e]);
// distinct keys decoded into (hi, lo) pairs if requested.  Returns the count.
struct Scratch {
  DBuf<uint64_t> k, k2;
  DBuf<uint32_t> v, v2;
  DBuf<uint64_t> uniq;
  Scratch(int64_t n, cudaStream_t s) : k(n, s), k2(n, s), v(n, s), v2(n, s), uniq(n, s) {}
};

int64_t rank_level(const int32_t* hi, int64_t mul, const int32_t* lo, uint64_t key_count, int64_t n,
                   int32_t* alpha_out, DBuf<int32_t>* out_hi, DBuf<int32_t>* out_lo, Scratch& sc,
                   cudaStream_t s) {
  const int g = grid_for(n);
  make_key_kernel<<<g, 256, 0, s>>>(hi, mul, lo, n, sc.k.get(), sc.v.get());
  FTT_LAUNCH();
  radix_sort_pairs(sc.k.get(), sc.v.get(), sc.k2.get(), sc.v2.get(), n, bits_for(key_count), s);
  const int64_t cnt = rank_sorted(sc.k.get(), sc.v.get(), n, alpha_out, sc.uniq.get(), s);
  if (out_hi && out_lo) {
    *out_hi = DBuf<int32_t>(cnt, s);
    *out_lo = DBuf<int32_t>(cnt, s);
    decode_kernel<<<grid_for(cnt), 256, 0, s>>>(sc.uniq.get(), cnt, mul, out_hi->get(), out_lo->get());
    FTT_LAUNCH();
  }
  return cnt;
}

typedef unsigned __int128 u128;

int64_t sat_prod(const std::vector<int64_t>& dims, int a, int b, int64_t cap) {
  // product of dims[a..b) saturated at cap
  u128 p = 1;
  for (int k = a; k < b; ++k) {
    p *= (u128)dims[k];
    if (p >= (u128)cap) return cap;
  }
  return (int64_t)p;
}

u128 f_svd(u128 m, u128 n) { return m * n * (m < n ? m : n); }   // < 2^124: m <= 2^62, n, min <= 2^31

u128 sat_add(u128 a, u128 b) { return (a + b < a) ? ~(u128)0 : a + b; }   // a sum of d terms may pass 2^128

}  // namespace

int select_p_host(const std::vector<int64_t>& dims, const std::vector<int64_t>& Rs, int64_t max_rank) {
  const int d = (int)dims.size();
  int best = 1;
  u128 best_f = 0;
  for (int p = 1; p <= d; ++p) {
    const int64_t R = Rs[p - 1];
    std::vector<int64_t> rt(d + 1, 1), r(d + 1, 1);
    for (int k = 1; k < d; ++k) {
      rt[k] = (k < p) ? sat_prod(dims, 0, k, R) : sat_prod(dims, k, d, R);   // eq. (10)
      r[k] = (max_rank > 0) ? std::min(rt[k], max_rank) : rt[k];
    }
    // eq. (13) with 1-based mode sizes n_i = dims[i-1]
    u128 f = f_svd((u128)rt[p - 1] * dims[p - 1], (u128)rt[p]);
    for (int i = p + 1; i <= d - 1; ++i) f = sat_add(f, f_svd((u128)r[i - 1] * dims[i - 1], (u128)rt[i]));
    for (int i = 2; i <= p; ++i) f = sat_add(f, f_svd((u128)rt[i - 1], (u128)dims[i - 1] * r[i]));
    if (p == 1 || f < best_f) {
      best = p;
      best_f = f;
    }
  }
  return best;
}

void ingest(int d, const int64_t* dims, int64_t nnz, const int32_t* d_idx, const void* d_vals,
            int val_dtype, Ingested& out, cudaStream_t s) {
  if (d < 2 || d > FASTTT_MAX_D) fail(FASTTT_EINVAL, "d must be in 2..64");
  if (nnz <= 0) fail(FASTTT_EINVAL, "the tensor has no nonzero entry");
  if (nnz >= ((int64_t)1 << 31)) fail(FASTTT_ERANK, "nnz must be below 2^31");
  if (!d_idx || !d_vals) fail(FASTTT_EINVAL, "null input pointer");
  if (val_dtype != FASTTT_F64 && val_dtype != FASTTT_F32) fail(FASTTT_EINVAL, "bad value dtype");
  DimsArg da{};
  out.d = d;
  out.dims.assign(dims, dims + d);
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1 || dims[k] > INT32_MAX) fail(FASTTT_EINVAL, "mode sizes must be in 1..2^31-1");
    da.n[k] = dims[k];
  }
  out.nnz_in = nnz;
  DBuf<int64_t> keep(nnz, s);
  DBuf<unsigned> err(1, s);
  FTT_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(unsigned), s));
  const int g = grid_for(nnz);
  if (val_dtype == FASTTT_F64)
    ingest_check_kernel<double><<<g, 256, 0, s>>>(d_idx, (const double*)d_vals, nnz, d, da, keep.get(), err.get());
  else
    ingest_check_kernel<float><<<g, 256, 0, s>>>(d_idx, (const float*)d_vals, nnz, d, da, keep.get(), err.get());
  FTT_LAUNCH();
  const unsigned e = read_scalar(err.get(), s);
  if (e & 1u) fail(FASTTT_EINVAL, "index out of range");
  if (e & 2u) fail(FASTTT_EINVAL, "non-finite value");
  const int64_t kept = exclusive_scan_i64(keep.get(), keep.get(), nnz, s);
  if (kept == 0) fail(FASTTT_EINVAL, "the tensor has no nonzero entry");
  out.nnz = kept;
  out.dropped = nnz - kept;
  out.idx = DBuf<int32_t>((size_t)d * kept, s);
  out.vals = DBuf<double>(kept, s);
  if (val_dtype == FASTTT_F64)
    ingest_compact_kernel<double><<<g, 256, 0, s>>>(d_idx, (const double*)d_vals, nnz, d, keep.get(), kept,
                                                    out.idx.get(), out.vals.get());
  else
    ingest_compact_kernel<float><<<g, 256, 0, s>>>(d_idx, (const float*)d_vals, nnz, d, keep.get(), kept,
                                                   out.idx.get(), out.vals.get());
  FTT_LAUNCH();
  DBuf<double> part(kNormBlocks, s), tot(1, s);
  sumsq_partial_kernel<<<kNormBlocks, 256, 0, s>>>(out.vals.get(), kept, part.get());
  FTT_LAUNCH();
  sum_partials_kernel<<<1, 32, 0, s>>>(part.get(), kNormBlocks, tot.get());
  FTT_LAUNCH();
  out.norm2 = read_scalar(tot.get(), s);
}

void group(const Ingested& in, int p_req, int64_t max_rank, Grouped& out, cudaStream_t s) {
  const int d = in.d;
  const int64_t n = in.nnz;
  const auto& dims = in.dims;
  if (p_req < 0 || p_req > d) fail(FASTTT_EINVAL, "p must be in 0..d");
  auto I = [&](int k) { return in.idx.get() + (int64_t)(k - 1) * n; };   // mode k (1-based)
  Scratch sc(n, s);
  out.rt.assign(d + 1, 1);
  // prefix ranks L_k = alpha_k of the left sweep (k = 1..d-1) and suffix ranks
  // S_k = alpha_k of the right sweep (k = d-1..1).  With p given only the levels
  // that p needs are computed (L_1..L_{p-1}, S_{d-1}..S_p).
  const bool auto_p = (p_req == 0);
  const int lmax = auto_p ? d - 1 : p_req - 1;
  const int smin = auto_p ? 1 : p_req;
  std::vector<DBuf<int32_t>> L(d), S(d + 1);
  std::vector<int64_t> lcount(d, 1), scount(d + 1, 1);
  std::vector<DBuf<int32_t>> lpar(d), lidx(d), ridx(d + 1), rchild(d + 1);
  for (int k = 1; k <= lmax; ++k) {
    L[k] = DBuf<int32_t>(n, s);
    const int32_t* prev = (k == 1) ? nullptr : L[k - 1].get();
    const uint64_t kc = (uint64_t)lcount[k - 1] * (uint64_t)dims[k - 1];
    lcount[k] = rank_level(prev, dims[k - 1], I(k), kc, n, L[k].get(), &lpar[k], &lidx[k], sc, s);
  }
  for (int k = d - 1; k >= smin; --k) {
    // alpha_k = rank of (i_{k+1}, alpha_{k+1}), alpha_d = 0
    S[k] = DBuf<int32_t>(n, s);
    const int32_t* next = (k == d - 1) ? nullptr : S[k + 1].get();
    const int64_t mul = scount[k + 1];
    const uint64_t kc = (uint64_t)dims[k] * (uint64_t)mul;
    scount[k] = rank_level(I(k + 1), mul, next, kc, n, S[k].get(), &ridx[k + 1], &rchild[k + 1], sc, s);
  }
  int p = p_req;
  if (auto_p) {
    // Alg. 9: R_p = distinct (L_{p-1}, S_p); R_1 = #S_1, R_d = #L_{d-1}
    out.Rs.assign(d, 0);
    out.Rs[0] = scount[1];
    out.Rs[d - 1] = lcount[d - 1];
    for (int q = 2; q <= d - 1; ++q) {
      const uint64_t kc = (uint64_t)lcount[q - 1] * (uint64_t)scount[q];
      out.Rs[q - 1] = rank_level(L[q - 1].get(), scount[q], S[q].get(), kc, n, nullptr, nullptr, nullptr, sc, s);
    }
    p = select_p_host(dims, out.Rs, max_rank);
    out.R = out.Rs[p - 1];
  } else {
    if (p == 1) out.R = scount[1];
    else if (p == d) out.R = lcount[d - 1];
    else {
      const uint64_t kc = (uint64_t)lcount[p - 1] * (uint64_t)scount[p];
      out.R = rank_level(L[p - 1].get(), scount[p], S[p].get(), kc, n, nullptr, nullptr, nullptr, sc, s);
    }
  }
  out.p = p;
  for (int k = 1; k < p; ++k) out.rt[k] = lcount[k];
  for (int k = p; k <= d - 1; ++k) out.rt[k] = scount[k];
  out.left_parent.clear();
  out.left_index.clear();
  for (int k = 1; k < p; ++k) {
    out.left_parent.push_back(std::move(lpar[k]));
    out.left_index.push_back(std::move(lidx[k]));
  }
  out.right_index.clear();
  out.right_child.clear();
  for (int k = p + 1; k <= d; ++k) {
    out.right_index.push_back(std::move(ridx[k]));
    out.right_child.push_back(std::move(rchild[k]));
  }
  // S5: middle unfolding X
  const int32_t* hi;
  const int32_t* lo;
  int64_t mul;
  if (p < d) {
    out.mid_rows = out.rt[p - 1] * dims[p - 1];
    out.mid_cols = out.rt[p];
    hi = (p == 1) ? nullptr : L[p - 1].get();
    mul = dims[p - 1];
    lo = I(p);
  } else {
    out.mid_rows = dims[d - 1];
    out.mid_cols = out.rt[d - 1];
    hi = nullptr;
    mul = 1;
    lo = I(d);
  }
  const u128 cells = (u128)out.mid_rows * (u128)out.mid_cols;
  if (cells >> 63) fail(FASTTT_ERANK, "middle unfolding has more than 2^63 cells");
  // row key, then the full (row, col) key = row * ncols + col
  {
    const int g = grid_for(n);
    make_key_kernel<<<g, 256, 0, s>>>(hi, mul, lo, n, sc.k.get(), sc.v.get());
    FTT_LAUNCH();
  }
  // key = row * ncols + col, built in place from the row key
  {
    const int32_t* colp = (p < d) ? S[p].get() : L[d - 1].get();
    combine_key_kernel<<<grid_for(n), 256, 0, s>>>(sc.k.get(), colp, out.mid_cols, n);
    FTT_LAUNCH();
  }
  radix_sort_pairs(sc.k.get(), sc.v.get(), sc.k2.get(), sc.v2.get(), n, bits_for((uint64_t)cells), s);
  DBuf<unsigned> err(1, s);
  FTT_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(unsigned), s));
  dup_check_kernel<<<grid_for(n), 256, 0, s>>>(sc.k.get(), n, err.get());
  FTT_LAUNCH();
  if (read_scalar(err.get(), s)) fail(FASTTT_EDUP, "duplicate coordinate in the COO input");
  out.mid_row = DBuf<int64_t>(n, s);
  out.mid_col = DBuf<int64_t>(n, s);
  out.mid_val = DBuf<double>(n, s);
  mid_gather_kernel<<<grid_for(n), 256, 0, s>>>(sc.k.get(), sc.v.get(), n, out.mid_cols, in.vals.get(),
                                               out.mid_row.get(), out.mid_col.get(), out.mid_val.get());
  FTT_LAUNCH();
}

}  // namespace fasttt
