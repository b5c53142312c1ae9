// Value Depar (S6) on the GPU: Alg. 3 with exact parallelism, restated for a
// sparse matrix whose entries are sorted by (row, col).
//
//  1. every nonzero row is divided by its first nonzero (IEEE FP64 __ddiv_rn);
//  2. each row gets a 64-bit hash of (length, columns, normalised value bits),
//     an integer sum of per-entry splitmix64 hashes (order-free and exact);
//  3. rows are stably radix-sorted by hash, so equal rows become neighbours in
//     ascending row order;
//  4. inside a run of equal hashes every row is compared entry by entry with the
//     run's earlier rows; the first equal one is its class leader (a hash
//     collision between different rows therefore never merges them);
//  5. leaders numbered in ascending row order give the class ids (first
//     occurrence), the prefactor of a row is its first nonzero, copied.
// The column pass runs the same code on the class representatives, transposed.
#include <cuda_runtime.h>

#include "depar.cuh"

namespace fasttt {

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // splitmix64 finaliser (Steele, Lea, Flood 2014)
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ull;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebull;
  z ^= z >> 31;
  return z;
}

#define GRID_STRIDE(i, n)                                                            \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

__global__ void i64_heads_kernel(const int64_t* a, int64_t n, int64_t* head) {
  GRID_STRIDE(i, n) head[i] = (i == 0 || a[i] != a[i - 1]) ? 1 : 0;
}

__global__ void u64_heads_kernel(const uint64_t* a, int64_t n, int64_t* head) {
  GRID_STRIDE(i, n) head[i] = (i == 0 || a[i] != a[i - 1]) ? 1 : 0;
}

__global__ void seg_kernel(const int64_t* major, const int64_t* excl, int64_t n, int32_t* seg,
                           int64_t* start, int64_t* ids) {
  GRID_STRIDE(i, n) {
    const bool head = (i == 0 || major[i] != major[i - 1]);
    const int64_t t = head ? excl[i] : excl[i] - 1;
    seg[i] = (int32_t)t;
    if (head) {
      start[t] = i;
      ids[t] = major[i];
    }
  }
}

__global__ void norm_hash_kernel(const int64_t* minor, const double* val, const int32_t* seg,
                                 const int64_t* start, int64_t n, double* w, unsigned long long* hash) {
  GRID_STRIDE(i, n) {
    const int32_t t = seg[i];
    const int64_t s0 = start[t];
    const double x = __ddiv_rn(val[i], val[s0]);
    w[i] = x;
    const uint64_t j = (uint64_t)(i - s0);
    const uint64_t h = mix64(mix64((uint64_t)minor[i] + 0x9E3779B97F4A7C15ull * (j + 1)) ^
                             (uint64_t)__double_as_longlong(x));
    atomicAdd(&hash[t], (unsigned long long)h);
  }
}

__device__ __forceinline__ int64_t seg_len(const int64_t* start, int64_t t, int64_t nz, int64_t n) {
  return ((t + 1 < nz) ? start[t + 1] : n) - start[t];
}

__global__ void row_key_kernel(const unsigned long long* hash, const int64_t* start, int64_t nz, int64_t n,
                               uint64_t* keys, uint32_t* vals) {
  GRID_STRIDE(t, nz) {
    keys[t] = (uint64_t)hash[t] + mix64((uint64_t)seg_len(start, t, nz, n) ^ 0x5bd1e9955bd1e995ull);
    vals[t] = (uint32_t)t;
  }
}

__device__ bool rows_equal(int64_t a, int64_t b, const int64_t* start, int64_t nz, int64_t n,
                           const int64_t* minor, const double* w) {
  const int64_t la = seg_len(start, a, nz, n), lb = seg_len(start, b, nz, n);
  if (la != lb) return false;
  const int64_t sa = start[a], sb = start[b];
  for (int64_t j = 0; j < la; ++j) {
    if (minor[sa + j] != minor[sb + j]) return false;
    if (__double_as_longlong(w[sa + j]) != __double_as_longlong(w[sb + j])) return false;
  }
  return true;
}

// q: position in hash order; excl/heads over sorted hashes give the run start.
__global__ void leader_kernel(const uint64_t* skeys, const uint32_t* srow, int64_t nz, const int64_t* excl,
                              const int64_t* run_start, const int64_t* start, int64_t n,
                              const int64_t* minor, const double* w, int32_t* leader) {
  GRID_STRIDE(q, nz) {
    const bool head = (q == 0 || skeys[q] != skeys[q - 1]);
    const int64_t run = head ? excl[q] : excl[q] - 1;
    const int64_t rs = run_start[run];
    const int64_t me = srow[q];
    int64_t lead = me;
    for (int64_t i = rs; i < q; ++i) {
      const int64_t other = srow[i];
      if (rows_equal(other, me, start, nz, n, minor, w)) {
        lead = other;
        break;
      }
    }
    leader[me] = (int32_t)lead;
  }
}

__global__ void run_start_kernel(const uint64_t* skeys, int64_t nz, const int64_t* excl, int64_t* run_start) {
  GRID_STRIDE(q, nz) {
    if (q == 0 || skeys[q] != skeys[q - 1]) run_start[excl[q]] = q;
  }
}

__global__ void is_leader_kernel(const int32_t* leader, const int64_t* start, int64_t nz, int64_t n,
                                 int64_t* isl, int64_t* replen) {
  GRID_STRIDE(t, nz) {
    const bool l = (leader[t] == t);
    isl[t] = l ? 1 : 0;
    replen[t] = l ? seg_len(start, t, nz, n) : 0;
  }
}

__global__ void class_kernel(const int32_t* leader, const int64_t* cls_excl, const int64_t* start,
                             const double* val, int64_t nz, int32_t* cls, double* pref) {
  GRID_STRIDE(t, nz) {
    cls[t] = (int32_t)cls_excl[leader[t]];
    pref[t] = val[start[t]];
  }
}

__global__ void emit_reps_kernel(const int32_t* seg, const int32_t* leader, const int64_t* start,
                                 const int64_t* rep_off, const int32_t* cls, const int64_t* minor,
                                 const double* w, int64_t n, int32_t* rep_cls, int64_t* rep_minor,
                                 double* rep_val) {
  GRID_STRIDE(i, n) {
    const int32_t t = seg[i];
    if (leader[t] != t) continue;
    const int64_t o = rep_off[t] + (i - start[t]);
    rep_cls[o] = cls[t];
    rep_minor[o] = minor[i];
    rep_val[o] = w[i];
  }
}

__global__ void class_key_kernel(const int32_t* cls, int64_t nz, uint64_t* keys, uint32_t* vals) {
  GRID_STRIDE(t, nz) {
    keys[t] = (uint64_t)(uint32_t)cls[t];
    vals[t] = (uint32_t)t;
  }
}

__global__ void class_start_kernel(const uint64_t* skeys, int64_t nz, int64_t* cstart) {
  GRID_STRIDE(q, nz) {
    if (q == 0 || skeys[q] != skeys[q - 1]) cstart[skeys[q]] = q;
  }
}

// Lambda[g] = sqrt(sum of pref^2 over class g's members, in ascending member order)
__global__ void class_norm_kernel(const int64_t* cstart, const uint32_t* members, const double* pref,
                                  int64_t beta, int64_t nz, double* lam) {
  GRID_STRIDE(g, beta) {
    const int64_t a = cstart[g], b = (g + 1 < beta) ? cstart[g + 1] : nz;
    double s = 0.0;
    for (int64_t q = a; q < b; ++q) {
      const double p = pref[members[q]];
      s = fma(p, p, s);
    }
    lam[g] = sqrt(s);
  }
}

__global__ void identity_pass_kernel(const int32_t* seg, const int64_t* minor, const double* val, int64_t n,
                                     int32_t* rep_cls, int64_t* rep_minor, double* rep_val) {
  GRID_STRIDE(i, n) {
    rep_cls[i] = seg[i];
    rep_minor[i] = minor[i];
    rep_val[i] = val[i];
  }
}

__global__ void iota_kernel(int32_t* a, int64_t n) { GRID_STRIDE(i, n) a[i] = (int32_t)i; }
__global__ void fill_kernel(double* a, int64_t n, double v) { GRID_STRIDE(i, n) a[i] = v; }

__global__ void transpose_key_kernel(const int32_t* cls, const int64_t* minor, int64_t n, int64_t beta,
                                     uint64_t* keys, uint32_t* vals) {
  GRID_STRIDE(i, n) {
    keys[i] = (uint64_t)minor[i] * (uint64_t)beta + (uint64_t)(uint32_t)cls[i];
    vals[i] = (uint32_t)i;
  }
}

__global__ void transpose_gather_kernel(const uint32_t* perm, const int32_t* cls, const int64_t* minor,
                                        const double* val, int64_t n, int64_t* tmajor, int64_t* tminor,
                                        double* tval) {
  GRID_STRIDE(q, n) {
    const uint32_t i = perm[q];
    tmajor[q] = minor[i];
    tminor[q] = (int64_t)cls[i];
    tval[q] = val[i];
  }
}

__global__ void dp_copy_kernel(const int32_t* rep_cls, const int64_t* rep_minor, int64_t n, int32_t* dp_row,
                               int32_t* dp_col) {
  GRID_STRIDE(i, n) {
    dp_col[i] = rep_cls[i];
    dp_row[i] = (int32_t)rep_minor[i];
  }
}

void run_pass(const int64_t* major, const int64_t* minor, const double* val, int64_t n, bool enabled,
              DeparPass& out, cudaStream_t s) {
  const int g = grid_for(n);
  DBuf<int64_t> head(n, s);
  i64_heads_kernel<<<g, 256, 0, s>>>(major, n, head.get());
  FTT_LAUNCH();
  const int64_t nz = exclusive_scan_i64(head.get(), head.get(), n, s);
  out.nz = nz;
  DBuf<int32_t> seg(n, s);
  DBuf<int64_t> start(nz, s);
  out.ids = DBuf<int64_t>(nz, s);
  seg_kernel<<<g, 256, 0, s>>>(major, head.get(), n, seg.get(), start.get(), out.ids.get());
  FTT_LAUNCH();
  head.reset();
  const int gz = grid_for(nz);
  out.cls = DBuf<int32_t>(nz, s);
  out.pref = DBuf<double>(nz, s);
  if (!enabled) {
    out.beta = nz;
    iota_kernel<<<gz, 256, 0, s>>>(out.cls.get(), nz);
    FTT_LAUNCH();
    fill_kernel<<<gz, 256, 0, s>>>(out.pref.get(), nz, 1.0);
    FTT_LAUNCH();
    out.lam = DBuf<double>(nz, s);
    fill_kernel<<<gz, 256, 0, s>>>(out.lam.get(), nz, 1.0);
    FTT_LAUNCH();
    out.rep_n = n;
    out.rep_cls = DBuf<int32_t>(n, s);
    out.rep_minor = DBuf<int64_t>(n, s);
    out.rep_val = DBuf<double>(n, s);
    identity_pass_kernel<<<g, 256, 0, s>>>(seg.get(), minor, val, n, out.rep_cls.get(), out.rep_minor.get(),
                                           out.rep_val.get());
    FTT_LAUNCH();
    return;
  }
  // 1-2: normalise and hash
  DBuf<double> w(n, s);
  DBuf<unsigned long long> hash(nz, s);
  FTT_CUDA(cudaMemsetAsync(hash.get(), 0, nz * sizeof(unsigned long long), s));
  norm_hash_kernel<<<g, 256, 0, s>>>(minor, val, seg.get(), start.get(), n, w.get(), hash.get());
  FTT_LAUNCH();
  // 3: stable sort of the rows by hash
  DBuf<uint64_t> k(nz, s), k2(nz, s);
  DBuf<uint32_t> v(nz, s), v2(nz, s);
  row_key_kernel<<<gz, 256, 0, s>>>(hash.get(), start.get(), nz, n, k.get(), v.get());
  FTT_LAUNCH();
  hash.reset();
  radix_sort_pairs(k.get(), v.get(), k2.get(), v2.get(), nz, 64, s);
  k2.reset();
  v2.reset();
  // 4: runs of equal hash, leaders by exact comparison
  DBuf<int64_t> hh(nz, s);
  u64_heads_kernel<<<gz, 256, 0, s>>>(k.get(), nz, hh.get());
  FTT_LAUNCH();
  const int64_t runs = exclusive_scan_i64(hh.get(), hh.get(), nz, s);
  DBuf<int64_t> run_start(runs, s);
  run_start_kernel<<<gz, 256, 0, s>>>(k.get(), nz, hh.get(), run_start.get());
  FTT_LAUNCH();
  DBuf<int32_t> leader(nz, s);
  leader_kernel<<<gz, 256, 0, s>>>(k.get(), v.get(), nz, hh.get(), run_start.get(), start.get(), n, minor,
                                   w.get(), leader.get());
  FTT_LAUNCH();
  run_start.reset();
  // 5: class ids by first occurrence, prefactors, representatives
  DBuf<int64_t> isl(nz, s), replen(nz, s);
  is_leader_kernel<<<gz, 256, 0, s>>>(leader.get(), start.get(), nz, n, isl.get(), replen.get());
  FTT_LAUNCH();
  out.beta = exclusive_scan_i64(isl.get(), isl.get(), nz, s);
  out.rep_n = exclusive_scan_i64(replen.get(), replen.get(), nz, s);
  class_kernel<<<gz, 256, 0, s>>>(leader.get(), isl.get(), start.get(), val, nz, out.cls.get(), out.pref.get());
  FTT_LAUNCH();
  out.rep_cls = DBuf<int32_t>(out.rep_n, s);
  out.rep_minor = DBuf<int64_t>(out.rep_n, s);
  out.rep_val = DBuf<double>(out.rep_n, s);
  emit_reps_kernel<<<g, 256, 0, s>>>(seg.get(), leader.get(), start.get(), replen.get(), out.cls.get(), minor,
                                     w.get(), n, out.rep_cls.get(), out.rep_minor.get(), out.rep_val.get());
  FTT_LAUNCH();
  // Lambda: members of each class in ascending order (stable sort by class)
  class_key_kernel<<<gz, 256, 0, s>>>(out.cls.get(), nz, k.get(), v.get());
  FTT_LAUNCH();
  {
    DBuf<uint64_t> ka(nz, s);
    DBuf<uint32_t> va(nz, s);
    radix_sort_pairs(k.get(), v.get(), ka.get(), va.get(), nz, bits_for((uint64_t)out.beta), s);
  }
  DBuf<int64_t> cstart(out.beta, s);
  class_start_kernel<<<gz, 256, 0, s>>>(k.get(), nz, cstart.get());
  FTT_LAUNCH();
  out.lam = DBuf<double>(out.beta, s);
  class_norm_kernel<<<grid_for(out.beta), 256, 0, s>>>(cstart.get(), v.get(), out.pref.get(), out.beta, nz,
                                                      out.lam.get());
  FTT_LAUNCH();
}

}  // namespace

void depar_pass(const int64_t* major, const int64_t* minor, const double* val, int64_t n, DeparPass& out,
                cudaStream_t s) {
  run_pass(major, minor, val, n, true, out, s);
}

void value_depar(const int64_t* row, const int64_t* col, const double* val, int64_t n, int64_t ncols,
                 bool enabled, DeparResult& out, cudaStream_t s) {
  run_pass(row, col, val, n, enabled, out.rows, s);
  // D (rows.beta x ncols) entries sorted by (class, col) -> sort by (col, class)
  const int64_t m = out.rows.rep_n;
  DBuf<uint64_t> k(m, s), k2(m, s);
  DBuf<uint32_t> v(m, s), v2(m, s);
  transpose_key_kernel<<<grid_for(m), 256, 0, s>>>(out.rows.rep_cls.get(), out.rows.rep_minor.get(), m,
                                                  out.rows.beta, k.get(), v.get());
  FTT_LAUNCH();
  radix_sort_pairs(k.get(), v.get(), k2.get(), v2.get(), m,
                   bits_for((uint64_t)ncols * (uint64_t)out.rows.beta), s);
  k2.reset();
  v2.reset();
  DBuf<int64_t> tmajor(m, s), tminor(m, s);
  DBuf<double> tval(m, s);
  transpose_gather_kernel<<<grid_for(m), 256, 0, s>>>(v.get(), out.rows.rep_cls.get(), out.rows.rep_minor.get(),
                                                     out.rows.rep_val.get(), m, tmajor.get(), tminor.get(),
                                                     tval.get());
  FTT_LAUNCH();
  run_pass(tmajor.get(), tminor.get(), tval.get(), m, enabled, out.cols, s);
  out.dp_n = out.cols.rep_n;
  out.dp_row = DBuf<int32_t>(out.dp_n, s);
  out.dp_col = DBuf<int32_t>(out.dp_n, s);
  out.dp_val = std::move(out.cols.rep_val);
  dp_copy_kernel<<<grid_for(out.dp_n), 256, 0, s>>>(out.cols.rep_cls.get(), out.cols.rep_minor.get(), out.dp_n,
                                                   out.dp_row.get(), out.dp_col.get());
  FTT_LAUNCH();
}

}  // namespace fasttt
