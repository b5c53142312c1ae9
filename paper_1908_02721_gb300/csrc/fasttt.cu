// libfasttt C ABI and the host orchestration of Alg. 7 (FastTT):
// S1 ingest -> S2-S5 grouping (Alg. 9, Alg. 4/5) -> S6 value Depar (Alg. 3)
// -> S7-S11 TT-rounding (Alg. 6 / Alg. 8) -> S12 output cores.
//
// The quasi-permutation cores of Alg. 4 are never materialised as 0/1 arrays:
// multiplying a factor into one is a gather (first SVD sweep, G_{k+1} x_1 W) or
// a scatter (second SVD sweep, G_{k-1} x_3 (V Sigma)) on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "dense.cuh"
#include "sparse_sweep.cuh"
#include "depar.cuh"
#include "group.cuh"

namespace fasttt {

// ---------------------------------------------------------------- allocation with the test hook

namespace {
std::mutex g_alloc_mu;
int64_t g_fail_after = 0;  // 0 = off
thread_local std::string g_last_error;
// Set while a handle is released: its buffers may belong to a stream the caller
// has destroyed since, so they are freed synchronously instead.
thread_local bool g_free_sync = false;
}  // namespace

namespace {
// Once per device: let the device's default memory pool (the one cudaMallocAsync
// draws from) keep up to a quarter of the device's memory cached across stream
// synchronisations instead of returning every freed block to the driver, so that
// the library's per-call work buffers are not mapped again on every call.  This is
// a setting of this process's pool (it ends with the process), not of the GPU.
constexpr int kPoolDevices = 64;
std::atomic<bool> g_pool_set[kPoolDevices];

void configure_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kPoolDevices) {
    cudaGetLastError();
    return;
  }
  if (g_pool_set[dev].exchange(true)) return;
  cudaMemPool_t pool;
  size_t fr = 0, tot = 0;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess || cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  uint64_t threshold = (uint64_t)tot / 4;
  uint64_t current = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &current) == cudaSuccess &&
      current < threshold)
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
  cudaGetLastError();
}
}  // namespace

void* dev_alloc(size_t bytes, cudaStream_t s) {
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_fail_after > 0 && --g_fail_after == 0) fail(FASTTT_ENOMEM, "injected allocation failure");
  }
  configure_pool();
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    fail(e == cudaErrorMemoryAllocation ? FASTTT_ENOMEM : FASTTT_ECUDA, buf);
  }
  return p;
}

namespace {
std::atomic<int64_t> g_launches{0};
thread_local std::vector<KClock> g_clocks;
}  // namespace

void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
std::atomic<int64_t> g_block_sweeps{0};
std::atomic<int> g_coop_err{0};
std::atomic<int64_t> g_eig_tridiag{0}, g_eig_fallback{0}, g_eig_fast{0};
}  // namespace
namespace {
thread_local int g_gemm_engine = 0;
}
void set_gemm_engine(int engine) { g_gemm_engine = engine; }
namespace {
thread_local int64_t g_max_spin = 0;
std::atomic<int64_t> g_wait_timeouts{0};
}  // namespace
void set_max_spin(int64_t spins) { g_max_spin = spins > 0 ? spins : 0; }
namespace {
// The calling thread's poll bound for the duration of one call, back to the
// defaults afterwards (so that later calls without the option are not bounded).
struct MaxSpinScope {
  explicit MaxSpinScope(int64_t spins) { set_max_spin(spins); }
  ~MaxSpinScope() { set_max_spin(0); }
};
}  // namespace
int64_t max_spin() { return g_max_spin; }
void note_wait_timeout() { g_wait_timeouts.fetch_add(1, std::memory_order_relaxed); }
int64_t wait_timeouts() { return g_wait_timeouts.load(); }
int gemm_engine() { return g_gemm_engine; }
void note_eig(bool tridiag) { (tridiag ? g_eig_tridiag : g_eig_fallback).fetch_add(1, std::memory_order_relaxed); }
void note_eig_fast() { g_eig_fast.fetch_add(1, std::memory_order_relaxed); }
void note_block_sweep(int err) {
  if (err) g_coop_err.store(err);
  else g_block_sweeps.fetch_add(1, std::memory_order_relaxed);
}
int64_t block_sweep_count() { return g_block_sweeps.load(); }
int last_coop_error() { return g_coop_err.load(); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

void kclock_begin(KClock& c, int cls, cudaStream_t s) {
  c.cls = cls;
  cudaEventCreate(&c.a);
  cudaEventCreate(&c.b);
  cudaEventRecord(c.a, s);
}

void kclock_end(KClock& c, double work, cudaStream_t s) {
  c.work = work;
  cudaEventRecord(c.b, s);
  g_clocks.push_back(c);
  c.a = c.b = nullptr;
}

void kclock_reset() {
  for (auto& c : g_clocks) {
    if (c.a) cudaEventDestroy(c.a);
    if (c.b) cudaEventDestroy(c.b);
  }
  g_clocks.clear();
}

void kclock_collect(double ms[KC_COUNT], double work[KC_COUNT]) {
  for (int i = 0; i < KC_COUNT; ++i) ms[i] = work[i] = 0.0;
  for (auto& c : g_clocks) {
    float t = 0.f;
    if (cudaEventSynchronize(c.b) == cudaSuccess && cudaEventElapsedTime(&t, c.a, c.b) == cudaSuccess) {
      ms[c.cls] += t;
      work[c.cls] += c.work;
    }
  }
}

void dev_free(void* p, cudaStream_t s) {
  if (!p) return;
  if (g_free_sync) cudaFree(p);
  else cudaFreeAsync(p, s);
}

namespace {

#define GRID_STRIDE(i, n)                                                            \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

// first-sweep bonds: the implicit (block-sparse) core when the dense one would
// exceed kDenseCoreBytes and its Gram side r_{k-1} n_k stays within kSparseGramMax
constexpr double kDenseCoreBytes = 2.0 * 1024 * 1024 * 1024;
constexpr int64_t kSparseGramMax = 16384;

// ---------------------------------------------------------------- factor kernels

// C (beta_r x beta_c row-major) = Lambda_S D' Lambda_T, entry (lam_s * d') * lam_t
__global__ void build_C_kernel(const int32_t* dp_row, const int32_t* dp_col, const double* dp_val, int64_t n,
                               const double* lam_s, const double* lam_t, int64_t ldc, double* C) {
  GRID_STRIDE(e, n) {
    const int32_t g = dp_row[e], h = dp_col[e];
    C[(int64_t)g * ldc + h] = (lam_s[g] * dp_val[e]) * lam_t[h];
  }
}

// out (ld-wide rows): row ids[t] = (pref[t] / lam[cls[t]]) * src[cls[t], :r]   (Q_S U_C)
__global__ void expand_rows_kernel(const int64_t* ids, const int32_t* cls, const double* pref,
                                   const double* lam, int64_t nz, const double* src, int64_t r,
                                   double* out) {
  GRID_STRIDE(e, nz * r) {
    const int64_t t = e / r, a = e % r;
    const int32_t g = cls[t];
    out[ids[t] * r + a] = (pref[t] / lam[g]) * src[(int64_t)g * r + a];
  }
}

// out (r x ncols row-major): column ids[u] = sigma * Vt[:, cls[u]] * (pref[u]/lam[cls[u]])   (Sigma V^T Q_T)
__global__ void expand_cols_kernel(const int64_t* ids, const int32_t* cls, const double* pref,
                                   const double* lam, int64_t nz, const double* Vt, int64_t ldv,
                                   const double* sigma, int64_t r, int64_t ncols, double* out) {
  GRID_STRIDE(e, nz * r) {
    const int64_t u = e / r, a = e % r;
    const int32_t h = cls[u];
    out[a * ncols + ids[u]] = sigma[a] * Vt[a * ldv + h] * (pref[u] / lam[h]);
  }
}

// G_k (r x n x rnext) from a right quasi-permutation core: column (ridx[al], rchild[al]) of
// unfold_1(G_k) = W[:, al]  (the first-sweep merge G_k x_1 W)
__global__ void merge_right_kernel(const double* W, int64_t r, int64_t rt_prev, const int32_t* ridx,
                                   const int32_t* rchild, int64_t n, int64_t rnext, double* G) {
  GRID_STRIDE(e, r * rt_prev) {
    const int64_t a = e / rt_prev, al = e % rt_prev;
    G[(a * n + ridx[al]) * rnext + rchild[al]] = W[a * rt_prev + al];
  }
}

// G_k (rprev x n x r) from a left quasi-permutation core: row (lpar[al], lidx[al]) of
// unfold_2(G_k) = VS[al, :]  (the second-sweep merge G_k x_3 (V Sigma))
__global__ void merge_left_kernel(const double* VS, int64_t rt_k, int64_t r, const int32_t* lpar,
                                  const int32_t* lidx, int64_t n, double* G) {
  GRID_STRIDE(e, rt_k * r) {
    const int64_t al = e / r, a = e % r;
    G[((int64_t)lpar[al] * n + lidx[al]) * r + a] = VS[al * r + a];
  }
}

// out (M x r) = U (M x r) scaled column-wise by sigma
__global__ void scale_cols_kernel(const double* U, int64_t M, int64_t r, const double* sigma, double* out) {
  GRID_STRIDE(e, M * r) out[e] = U[e] * sigma[e % r];
}

// out (r x N) = sigma (row-wise) * Vt
__global__ void scale_rows_kernel(const double* Vt, int64_t r, int64_t N, const double* sigma, double* out) {
  GRID_STRIDE(e, r * N) out[e] = Vt[e] * sigma[e / N];
}

// Block construction of the TT sum (Lemma 2, eq. (6)): src (r0 x n x r1, row-major)
// times scale goes to rows [o0, o0 + r0) and columns [o1, o1 + r1) of every slice
// of dst (R0 x n x R1, row-major, zeroed by the caller); add = true accumulates
// (the d = 1 sum, where both blocks cover the whole core).
__global__ void place_block_kernel(const double* src, int64_t r0, int64_t n, int64_t r1, double scale, double* dst,
                                   int64_t R1, int64_t o0, int64_t o1, bool add) {
  GRID_STRIDE(e, r0 * n * r1) {
    const int64_t c = e % r1, j = (e / r1) % n, i = e / (r1 * n);
    double* t = dst + ((o0 + i) * n + j) * R1 + (o1 + c);
    const double v = __dmul_rn(scale, src[e]);   // no FMA contraction: A + beta B rounded twice, as written
    *t = add ? __dadd_rn(*t, v) : v;
  }
}

}  // namespace

// ---------------------------------------------------------------- handle

struct Handle {
  int d = 0;
  int64_t wait0 = wait_timeouts();   // device waits given up before this call
  std::vector<int64_t> dims, ranks;
  std::vector<DBuf<double>> cores;
  fasttt_stats st{};
  bool kept = false;
  Grouped grp;
  DeparResult dep;
  std::vector<std::vector<double>> sigmas;  // per bond (index k), host copies
};

}  // namespace fasttt

struct fasttt_tt {
  fasttt::Handle h;
};

namespace fasttt {
int tt_eval_at_impl(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores, int dtype, int64_t m,
                    const int32_t* idx, void* out, cudaStream_t s);
int tt_eval_backward_impl(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores, int dtype,
                          int64_t m, const int32_t* idx, const void* gout, void* const* grads, int recompute,
                          cudaStream_t s);
}  // namespace fasttt

namespace fasttt {
namespace {

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  double lap() {  // ms since construction / last lap
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    std::swap(a, b);
    return ms;
  }
};

// rank rule S11: smallest r >= 1 with sqrt(sum_{i>r} s_i^2) <= delta (tails summed
// from the smallest value up); eps = 0: s_i > max(M,N) 2^-52 s_1 for the full
// k-unfolding of A; capped by max_rank.
int64_t rank_rule(const std::vector<double>& s, double delta, bool eps_zero, const std::vector<int64_t>& dims,
                  int bond, int64_t max_rank) {
  const int64_t n = (int64_t)s.size();
  int64_t r = n;
  if (!eps_zero) {
    std::vector<double> tail(n + 1, 0.0);
    double acc = 0.0;
    for (int64_t i = n - 1; i >= 0; --i) {
      acc += s[i] * s[i];
      tail[i] = acc;
    }
    const double d2 = delta * delta;
    for (int64_t c = 1; c <= n; ++c)
      if (tail[c] <= d2) { r = c; break; }
  } else {
    // max(prod(n_1..n_k), prod(n_{k+1}..n_d)) as a double (exact integers up to 2^53)
    double a = 1.0, b = 1.0;
    for (int k = 0; k < bond; ++k) a *= (double)dims[k];
    for (int k = bond; k < (int)dims.size(); ++k) b *= (double)dims[k];
    const double tol = std::max(a, b) * 0x1p-52 * (n ? s[0] : 0.0);
    int64_t c = 0;
    for (double x : s) c += (x > tol) ? 1 : 0;
    r = std::max<int64_t>(1, c);
  }
  if (max_rank > 0) r = std::min(r, max_rank);
  return r;
}

void finish_stats(fasttt_stats& st, int64_t launches0) {
  double ms[KC_COUNT], work[KC_COUNT];
  kclock_collect(ms, work);
  st.ms_gemm = ms[KC_GEMM];
  st.flop_gemm = work[KC_GEMM];
  st.ms_jacobi = ms[KC_JACOBI];
  st.flop_jacobi = work[KC_JACOBI];
  st.ms_sort = ms[KC_SORT];
  st.bytes_sort = work[KC_SORT];
  st.ms_jacobi32 = ms[KC_JACOBI32];
  st.flop_jacobi32 = work[KC_JACOBI32];
  st.ms_gemm_tc = ms[KC_GEMM_TC];
  st.flop_gemm_tc = work[KC_GEMM_TC];
  st.ms_tridiag = ms[KC_TRIDIAG];
  st.flop_tridiag = work[KC_TRIDIAG];
  st.ms_tdeig = ms[KC_TDEIG];
  st.ms_gemm_oz = ms[KC_GEMM_OZ];
  st.flop_gemm_oz = work[KC_GEMM_OZ];
  st.ms_tridiag32 = ms[KC_TRIDIAG32];
  st.flop_tridiag32 = work[KC_TRIDIAG32];
  st.ms_tsqr = ms[KC_TSQR];
  st.flop_tsqr = work[KC_TSQR];
  kclock_reset();
  st.launches = launch_count() - launches0;
}

struct CounterSnap {
  int64_t block_sweeps, eig_tridiag, eig_fallback, eig_fast, mixed_kept, mixed_esc;
};
CounterSnap counter_snap() {
  return {block_sweep_count(), g_eig_tridiag.load(), g_eig_fallback.load(), g_eig_fast.load(),
          mixed_bonds_kept(), mixed_bonds_escalated()};
}
void finish_block_stats(fasttt_stats& st, const CounterSnap& c0) {
  st.jacobi_block_sweeps = block_sweep_count() - c0.block_sweeps;
  st.coop_launch_error = last_coop_error();
  st.eig_tridiag = g_eig_tridiag.load() - c0.eig_tridiag;
  st.eig_fallbacks = g_eig_fallback.load() - c0.eig_fallback;
  st.eig_fast = g_eig_fast.load() - c0.eig_fast;
  st.mixed_fp32_bonds = mixed_bonds_kept() - c0.mixed_kept;
  st.mixed_fp64_bonds = mixed_bonds_escalated() - c0.mixed_esc;
}

double tail2(const std::vector<double>& s, int64_t r) {
  double acc = 0.0;
  for (int64_t i = (int64_t)s.size() - 1; i >= r; --i) acc += s[i] * s[i];
  return acc;
}

// QR step of Alg. 6's right-to-left sweep for Z = unfold_1(G_k) (M x N, N = n_k r_k):
// Z = R^T Q with Q's rows orthonormal.  M <= N: CholeskyQR2 of Z's rows (G_k <- Q,
// US <- R^T, q = M); false, G_k untouched, when it breaks down (the caller takes
// an untruncated SVD).  M > N: Q = I (G_k <- the N x N identity, US <- Z, q = N),
// which is exact.
bool qr_factor(DBuf<double>& Gk, int64_t M, int64_t N, bool mixed, DBuf<double>& US, int64_t& q, cudaStream_t s) {
  if (M > N) {
    US = std::move(Gk);
    Gk = DBuf<double>((size_t)N * N, s);
    identity_f64(Gk.get(), N, s);
    q = N;
    return true;
  }
  DBuf<double> Z((size_t)M * N, s), R((size_t)M * M, s);
  FTT_CUDA(cudaMemcpyAsync(Z.get(), Gk.get(), Z.bytes(), cudaMemcpyDeviceToDevice, s));
  if (!cholqr2_rows(Z.get(), M, N, R.get(), mixed, s)) return false;
  Gk = std::move(Z);
  US = DBuf<double>((size_t)M * M, s);
  transpose_f64(R.get(), M, M, US.get(), s);
  q = M;
  return true;
}

void run(int d, const int64_t* dims, int64_t nnz, const int32_t* d_idx, const void* d_vals, int val_dtype,
         double eps, const fasttt_opts& o, cudaStream_t s, Handle& H) {
  if (!(eps >= 0.0) || !std::isfinite(eps)) fail(FASTTT_EINVAL, "eps must be finite and >= 0");
  if (o.rounding != FASTTT_STATIC && o.rounding != FASTTT_DYNAMIC) fail(FASTTT_EINVAL, "bad rounding mode");
  if (o.precision != FASTTT_PREC_FP64 && o.precision != FASTTT_PREC_MIXED) fail(FASTTT_EINVAL, "unsupported precision");
  const bool mixed = (o.precision == FASTTT_PREC_MIXED);
  if (o.stage != FASTTT_STAGE_FULL && o.stage != FASTTT_STAGE_EXACT && o.stage != FASTTT_STAGE_DEPAR)
    fail(FASTTT_EINVAL, "bad stage");
  if (o.sparse_sweep < FASTTT_SWEEP_AUTO || o.sparse_sweep > FASTTT_SWEEP_DENSE)
    fail(FASTTT_EINVAL, "bad sparse_sweep mode");
  if (o.gemm_engine != FASTTT_GEMM_TENSOR && o.gemm_engine != FASTTT_GEMM_DFMA)
    fail(FASTTT_EINVAL, "bad gemm_engine");
  set_gemm_engine(o.gemm_engine);
  MaxSpinScope spin_scope(o.max_spin);
  const int64_t max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : 40;
  fasttt_stats& st = H.st;
  st.d = d;
  kclock_reset();
  const int64_t launches0 = launch_count();
  const CounterSnap snap0 = counter_snap();
  Timer total(s), lap(s);
  // S1
  Ingested in;
  ingest(d, dims, nnz, d_idx, d_vals, val_dtype, in, s);
  st.nnz_in = in.nnz_in;
  st.nnz = in.nnz;
  st.dropped = in.dropped;
  st.norm2 = in.norm2;
  st.ms_ingest = lap.lap();
  H.d = d;
  H.dims = in.dims;
  // S2-S5
  Grouped& g = H.grp;
  group(in, o.p, o.max_rank, g, s);
  const int p = g.p;
  st.p = p;
  st.R = g.R;
  for (size_t q = 0; q < g.Rs.size(); ++q) st.Rs[q] = g.Rs[q];
  for (int k = 0; k <= d; ++k) st.rt[k] = g.rt[k];
  st.ms_group = lap.lap();
  in.idx.reset();
  in.vals.reset();
  if (o.stage == FASTTT_STAGE_EXACT) {
    H.kept = true;
    for (int k = 0; k <= d; ++k) st.ranks[k] = g.rt[k];
    H.ranks.assign(g.rt.begin(), g.rt.end());
    st.ms_total = total.lap();
    finish_stats(st, launches0);
    return;
  }
  // S6
  DeparResult& dp = H.dep;
  value_depar(g.mid_row.get(), g.mid_col.get(), g.mid_val.get(), in.nnz, g.mid_cols, o.depar_values != 0, dp, s);
  st.beta_r = dp.rows.beta;
  st.beta_c = dp.cols.beta;
  st.ms_depar = lap.lap();
  if (o.stage == FASTTT_STAGE_DEPAR) {
    H.kept = true;
    for (int k = 0; k <= d; ++k) st.ranks[k] = g.rt[k];
    H.ranks.assign(g.rt.begin(), g.rt.end());
    st.ms_total = total.lap();
    finish_stats(st, launches0);
    return;
  }

  // S7-S11
  const std::vector<int64_t>& n = H.dims;
  const double normA = std::sqrt(in.norm2);
  const bool eps0 = (eps == 0.0);
  const double c = std::sqrt((double)(p - 1)) + std::sqrt((double)(d - p));
  double d_right = std::sqrt((double)(d - p)) / c * eps * normA;   // Alg. 8 budgets
  double d_left = std::sqrt((double)(p - 1)) / c * eps * normA;
  auto delta_for = [&](int bond, bool right_side) {
    if (o.rounding == FASTTT_STATIC) return eps * normA / c;                      // eq. (11)
    return right_side ? d_right / std::sqrt((double)(d - bond)) : d_left / std::sqrt((double)bond);
  };
  H.sigmas.assign(d + 1, {});
  std::vector<int64_t> r(d + 1, 1);
  for (int k = 0; k <= d; ++k) r[k] = g.rt[k];
  std::vector<DBuf<double>> G(d + 1);  // 1-based dense cores
  DBuf<double> UC;                      // G_p = Q_S UC while G[p] is empty (p < d)
  // first-sweep core G_k (k > p) held implicitly: G_k = Wk x_1 P_k while G[k] is empty
  DBuf<double> Wk;
  auto keep_sparse = [&](int k, int64_t rp) {
    if (k >= d) return false;   // the last core (r~_d = 1) is always small
    if ((double)rp * (double)n[k - 1] > (double)kSparseGramMax) return false;
    if (o.sparse_sweep == FASTTT_SWEEP_SPARSE) return true;
    if (o.sparse_sweep == FASTTT_SWEEP_DENSE) return false;
    return (double)rp * (double)n[k - 1] * (double)g.rt[k] * 8.0 > kDenseCoreBytes;
  };
  auto expand_Q_S = [&](const double* U, int64_t rr) {
    DBuf<double> X((size_t)g.mid_rows * rr, s);
    FTT_CUDA(cudaMemsetAsync(X.get(), 0, X.bytes(), s));
    expand_rows_kernel<<<grid_for(dp.rows.nz * rr), 256, 0, s>>>(
        dp.rows.ids.get(), dp.rows.cls.get(), dp.rows.pref.get(), dp.rows.lam.get(), dp.rows.nz, U, rr, X.get());
    FTT_LAUNCH();
    return X;
  };
  double err2 = 0.0;
  std::vector<double> kappa(d + 1, 0.0);   // sigma_1 / sigma_r of the kept values per bond
  auto record = [&](int bond, const SvdOut& sv, double dl) {
    const double e2 = tail2(sv.sigma_all, sv.r);
    if (sv.r > 0 && sv.r <= (int64_t)sv.sigma_all.size() && sv.sigma_all[sv.r - 1] > 0.0)
      kappa[bond] = sv.sigma_all[0] / sv.sigma_all[sv.r - 1];
    err2 += e2;
    st.deltas[bond] = dl;
    st.jacobi_sweeps += sv.sweeps;
    if (o.keep_intermediates) H.sigmas[bond] = sv.sigma_all;
    return e2;
  };
  // --- the first SVD, on C = Lambda_S D' Lambda_T
  {
    const int64_t br = dp.rows.beta, bc = dp.cols.beta;
    if ((double)br * (double)bc > 4.0e9) fail(FASTTT_ERANK, "value-Depar factor C too large for the dense SVD");
    DBuf<double> C((size_t)br * bc, s);
    FTT_CUDA(cudaMemsetAsync(C.get(), 0, C.bytes(), s));
    build_C_kernel<<<grid_for(dp.dp_n), 256, 0, s>>>(dp.dp_row.get(), dp.dp_col.get(), dp.dp_val.get(), dp.dp_n,
                                                     dp.rows.lam.get(), dp.cols.lam.get(), bc, C.get());
    FTT_LAUNCH();
    const int bond = (p < d) ? p : d - 1;
    const double dl = delta_for(bond, p < d);
    SvdOut sv;
    svd_truncated(C.get(), br, bc, [&](const std::vector<double>& sg) {
      return rank_rule(sg, dl, eps0, n, bond, o.max_rank);
    }, max_sweeps, sv, s, mixed, 1);  // U_C becomes G_p (p < d) or G_d^T (p = d)
    C.reset();
    const double e2 = record(bond, sv, dl);
    const int64_t rr = sv.r;
    // U_X = Q_S U_C (mid_rows x rr), V-side: Sigma V_C^T Q_T (rr x mid_cols).  For p < d
    // G_p stays factored as Q_S U_C until the QR sweep multiplies R^T into it.
    DBuf<double> UX;
    if (p < d) {
      UC = std::move(sv.U);
    } else {
      UX = expand_Q_S(sv.U.get(), rr);
    }
    DBuf<double> SW((size_t)rr * g.mid_cols, s);
    FTT_CUDA(cudaMemsetAsync(SW.get(), 0, SW.bytes(), s));
    expand_cols_kernel<<<grid_for(dp.cols.nz * rr), 256, 0, s>>>(
        dp.cols.ids.get(), dp.cols.cls.get(), dp.cols.pref.get(), dp.cols.lam.get(), dp.cols.nz, sv.Vt.get(), bc,
        sv.sigma.get(), rr, g.mid_cols, SW.get());
    FTT_LAUNCH();
    if (p < d) {
      // G_p := U_X (held as U_C) ; G_{p+1} := G_{p+1} x_1 (Sigma V^T)  (right quasi-permutation core)
      r[p] = rr;
      const int k1 = p + 1;
      if (keep_sparse(k1, rr)) {
        Wk = std::move(SW);
      } else {
        DBuf<double> Gn((size_t)rr * n[k1 - 1] * r[k1], s);
        FTT_CUDA(cudaMemsetAsync(Gn.get(), 0, Gn.bytes(), s));
        merge_right_kernel<<<grid_for(rr * g.rt[p]), 256, 0, s>>>(SW.get(), rr, g.rt[p], g.right_index[0].get(),
                                                                   g.right_child[0].get(), n[k1 - 1], r[k1], Gn.get());
        FTT_LAUNCH();
        G[k1] = std::move(Gn);
      }
      if (o.rounding == FASTTT_DYNAMIC) d_right = std::sqrt(std::max(d_right * d_right - e2, 0.0));
    } else {
      // p = d: G_d := U_X^T (r x n_d x 1); G_{d-1} := G_{d-1} x_3 (V Sigma) (left quasi-permutation core)
      DBuf<double> Gd((size_t)rr * n[d - 1], s);
      transpose_f64(UX.get(), g.mid_rows, rr, Gd.get(), s);
      G[d] = std::move(Gd);
      r[d - 1] = rr;
      DBuf<double> VS((size_t)g.mid_cols * rr, s);
      transpose_f64(SW.get(), rr, g.mid_cols, VS.get(), s);
      const int k0 = d - 1;
      DBuf<double> Gp((size_t)r[k0 - 1] * n[k0 - 1] * rr, s);
      FTT_CUDA(cudaMemsetAsync(Gp.get(), 0, Gp.bytes(), s));
      merge_left_kernel<<<grid_for(g.rt[k0] * rr), 256, 0, s>>>(VS.get(), g.rt[k0], rr, g.left_parent[k0 - 1].get(),
                                                                 g.left_index[k0 - 1].get(), n[k0 - 1], Gp.get());
      FTT_LAUNCH();
      G[k0] = std::move(Gp);
      if (o.rounding == FASTTT_DYNAMIC) d_left = std::sqrt(std::max(d_left * d_left - e2, 0.0));
    }
  }
  int start;
  if (p < d) {
    // --- first SVD sweep k = p+1..d-1 (Alg. 6)
    for (int k = p + 1; k <= d - 1; ++k) {
      const int64_t M = r[k - 1] * n[k - 1], N = r[k];
      const double dl = delta_for(k, true);
      auto choose = [&](const std::vector<double>& sg) { return rank_rule(sg, dl, eps0, n, k, o.max_rank); };
      SvdOut sv;
      DBuf<double> W;
      if (!G[k].get()) {
        // block-sparse bond: Gram and projection from W_{k-1} and the maps of P_k
        SparseBond sb(Wk.get(), r[k - 1], g.rt[k - 1], g.right_index[k - p - 1].get(), g.right_child[k - p - 1].get(),
                      n[k - 1], N, s);
        Wk.reset();
        {
          DBuf<double> Gram((size_t)M * M, s);
          sb.gram(Gram.get(), s);
          svd_from_gram(Gram.get(), M, N, choose, max_sweeps, sv, s, mixed, o.max_rank, !o.keep_intermediates);
        }
        sb.project(sv.U.get(), sv.r, W, s);   // W_k = U^T Z = Sigma V^T
        ++st.sparse_bonds;
      } else {
        svd_truncated(G[k].get(), M, N, choose, max_sweeps, sv, s, mixed, 1);
        W = DBuf<double>((size_t)sv.r * N, s);
        scale_rows_kernel<<<grid_for(sv.r * N), 256, 0, s>>>(sv.Vt.get(), sv.r, N, sv.sigma.get(), W.get());
        FTT_LAUNCH();
      }
      const double e2 = record(k, sv, dl);
      const int64_t rr = sv.r;
      G[k] = std::move(sv.U);
      r[k] = rr;
      const int k1 = k + 1;
      if (keep_sparse(k1, rr)) {
        Wk = std::move(W);
      } else {
        DBuf<double> Gn((size_t)rr * n[k1 - 1] * r[k1], s);
        FTT_CUDA(cudaMemsetAsync(Gn.get(), 0, Gn.bytes(), s));
        merge_right_kernel<<<grid_for(rr * g.rt[k]), 256, 0, s>>>(W.get(), rr, g.rt[k], g.right_index[k - p].get(),
                                                                   g.right_child[k - p].get(), n[k1 - 1], r[k1],
                                                                   Gn.get());
        FTT_LAUNCH();
        G[k1] = std::move(Gn);
      }
      if (o.rounding == FASTTT_DYNAMIC) d_right = std::sqrt(std::max(d_right * d_right - e2, 0.0));
    }
    // --- QR sweep k = d..p+1: unfold_1^T(G_k) = Q R by an untruncated SVD of
    // unfold_1(G_k) = U S V^T (Q = V, R = S U^T); G_{k-1} := G_{k-1} x_3 R^T
    for (int k = d; k >= p + 1; --k) {
      const int64_t M = r[k - 1], N = n[k - 1] * r[k];
      int64_t q = 0;
      DBuf<double> US;
      // FP32-level CholeskyQR2 only where bond k-1's kept singular values (those of
      // unfold_1(G_k) while everything right of it is orthonormal) span less than
      // 2^-6 of the FP32 level's u^{-1/2}; FP64-level otherwise
      const double kap = kappa[k - 1];
      const bool qr_mixed = mixed && kap > 0.0 && std::isfinite(kap) && kap * kap * 0x1p-23 < 0x1p-6;
      if (qr_factor(G[k], M, N, qr_mixed, US, q, s)) {
        ++st.qr_cholqr2;
      } else {
        SvdOut sv;
        svd_truncated(G[k].get(), M, N, [&](const std::vector<double>& sg) { return (int64_t)sg.size(); },
                      max_sweeps, sv, s, mixed, 2);
        st.jacobi_sweeps += sv.sweeps;
        q = sv.r;
        G[k] = std::move(sv.Vt);
        US = DBuf<double>((size_t)M * q, s);
        scale_cols_kernel<<<grid_for(M * q), 256, 0, s>>>(sv.U.get(), M, q, sv.sigma.get(), US.get());
        FTT_LAUNCH();
        ++st.qr_svd;
      }
      if (k - 1 == p && UC.get()) {
        // G_p = Q_S UC:  G_p R^T = Q_S (UC R^T), a beta_r-row GEMM, then one expansion
        const int64_t br = dp.rows.beta;
        DBuf<double> UC2((size_t)br * q, s);
        gemm(mixed, br, q, M, 1.0, UC.get(), M, 1, US.get(), q, 1, 0.0, UC2.get(), q, 1, s);
        UC.reset();
        G[p] = expand_Q_S(UC2.get(), q);
      } else {
        const int64_t Mp = r[k - 2] * n[k - 2];
        DBuf<double> Gp((size_t)Mp * q, s);
        gemm(mixed, Mp, q, M, 1.0, G[k - 1].get(), M, 1, US.get(), q, 1, 0.0, Gp.get(), q, 1, s);
        G[k - 1] = std::move(Gp);
      }
      r[k - 1] = q;
    }
    start = p;
  } else {
    start = d - 1;
  }
  // --- second SVD sweep k = start..2: SVD of unfold_1^T(G_k) via unfold_1(G_k) = U S V^T:
  // G_k := V^T rows, G_{k-1} := G_{k-1} x_3 (U S)  (left quasi-permutation core)
  for (int k = start; k >= 2; --k) {
    const int64_t M = r[k - 1], N = n[k - 1] * r[k];
    const double dl = delta_for(k - 1, false);
    SvdOut sv;
    svd_truncated(G[k].get(), M, N, [&](const std::vector<double>& sg) {
      return rank_rule(sg, dl, eps0, n, k - 1, o.max_rank);
    }, max_sweeps, sv, s, mixed, 2);
    const double e2 = record(k - 1, sv, dl);
    const int64_t rr = sv.r;
    G[k] = std::move(sv.Vt);
    DBuf<double> US((size_t)M * rr, s);
    scale_cols_kernel<<<grid_for(M * rr), 256, 0, s>>>(sv.U.get(), M, rr, sv.sigma.get(), US.get());
    FTT_LAUNCH();
    const int k0 = k - 1;
    DBuf<double> Gp((size_t)r[k0 - 1] * n[k0 - 1] * rr, s);
    FTT_CUDA(cudaMemsetAsync(Gp.get(), 0, Gp.bytes(), s));
    merge_left_kernel<<<grid_for(g.rt[k0] * rr), 256, 0, s>>>(US.get(), g.rt[k0], rr, g.left_parent[k0 - 1].get(),
                                                               g.left_index[k0 - 1].get(), n[k0 - 1], Gp.get());
    FTT_LAUNCH();
    G[k0] = std::move(Gp);
    r[k0] = rr;
    if (o.rounding == FASTTT_DYNAMIC) d_left = std::sqrt(std::max(d_left * d_left - e2, 0.0));
  }
  // S12
  st.err2 = err2;
  H.cores.clear();
  for (int k = 1; k <= d; ++k) H.cores.push_back(std::move(G[k]));
  H.ranks.assign(d + 1, 1);
  for (int k = 1; k < d; ++k) H.ranks[k] = r[k];
  for (int k = 0; k <= d; ++k) st.ranks[k] = H.ranks[k];
  H.kept = o.keep_intermediates != 0;
  if (!H.kept) {
    H.grp = Grouped();
    H.dep = DeparResult();
  }
  st.ms_round = lap.lap();
  st.ms_total = total.lap();
  ozaki_take_timeout(s);
  finish_stats(st, launches0);
  finish_block_stats(st, snap0);
}

// Checks a TT given by device cores: 1 <= d <= FASTTT_MAX_D, n_k >= 1, r_0 = r_d = 1,
// r_k >= 1, no null core; returns the ranks and mode sizes as vectors.
void check_tt(int d, const int64_t* dims, const int64_t* ranks, const double* const* cores, const char* what) {
  const std::string w(what);
  if (d < 1 || d > FASTTT_MAX_D) fail(FASTTT_EINVAL, w + ": d must be in 1..FASTTT_MAX_D");
  if (!dims || !ranks || !cores) fail(FASTTT_EINVAL, w + ": null argument");
  if (ranks[0] != 1 || ranks[d] != 1) fail(FASTTT_EINVAL, w + ": r_0 and r_d must be 1");
  for (int k = 1; k <= d; ++k) {
    if (dims[k - 1] < 1 || ranks[k] < 1) fail(FASTTT_EINVAL, w + ": mode sizes and ranks must be >= 1");
    if (!cores[k - 1]) fail(FASTTT_EINVAL, w + ": null core");
    if ((double)ranks[k - 1] * (double)dims[k - 1] * (double)ranks[k] > 0x1p40)
      fail(FASTTT_ERANK, w + ": core too large");
  }
}

// Alg. 2 (TT-rounding of a TT given by its cores), Section 2.4:
//  1. right-to-left orthogonalisation, k = d..2: unfold_1(G_k) = (U S) V^T, untruncated
//     (min(M,N) singular triplets, the size of the QR factorisation it stands for);
//     G_k := V^T (orthonormal rows) and G_{k-1} := G_{k-1} x_3 (U S).  Nothing is
//     dropped: in a Lemma 2 difference of close TTs the difference lives in the cores'
//     small singular directions.  A direction whose singular value is exactly zero gets
//     a zero row in V^T and a zero column in U S, which leaves the tensor and the
//     singular values of the next sweep unchanged.
//  2. ||A||_F = ||G_1||_F (the sum of the first bond's sigma^2), delta = eps ||A|| / sqrt(d-1).
//  3. left-to-right compression, k = 1..d-1: delta-truncated SVD of unfold_2(G_k);
//     G_k := U, G_{k+1} := (S V^T) x_1 G_{k+1}.
// The rank rule, the eps = 0 reading and the max_rank cap are those of the
// decomposition (S11).
void round_tt(int d, const int64_t* dims, const int64_t* ranks, const double* const* cores, double eps,
              const fasttt_opts& o, cudaStream_t s, Handle& H) {
  check_tt(d, dims, ranks, cores, "tt_round");
  if (!(eps >= 0.0) || !std::isfinite(eps)) fail(FASTTT_EINVAL, "eps must be finite and >= 0");
  if (o.rounding != FASTTT_STATIC) fail(FASTTT_EINVAL, "tt_round: Alg. 2 fixes delta (static rounding only)");
  if (o.precision != FASTTT_PREC_FP64 && o.precision != FASTTT_PREC_MIXED) fail(FASTTT_EINVAL, "unsupported precision");
  if (o.gemm_engine != FASTTT_GEMM_TENSOR && o.gemm_engine != FASTTT_GEMM_DFMA) fail(FASTTT_EINVAL, "bad gemm_engine");
  if (o.max_rank < 0) fail(FASTTT_EINVAL, "max_rank must be >= 0");
  set_gemm_engine(o.gemm_engine);
  MaxSpinScope spin_scope(o.max_spin);
  const bool mixed = (o.precision == FASTTT_PREC_MIXED);
  const bool eps0 = (eps == 0.0);
  const int64_t max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : 40;
  fasttt_stats& st = H.st;
  st.d = d;
  kclock_reset();
  const int64_t launches0 = launch_count();
  const CounterSnap snap0 = counter_snap();
  Timer total(s);
  std::vector<int64_t> n(dims, dims + d), r(ranks, ranks + d + 1);
  std::vector<DBuf<double>> G(d + 1);   // 1-based
  for (int k = 1; k <= d; ++k) {
    G[k] = DBuf<double>((size_t)(r[k - 1] * n[k - 1] * r[k]), s);
    FTT_CUDA(cudaMemcpyAsync(G[k].get(), cores[k - 1], G[k].bytes(), cudaMemcpyDeviceToDevice, s));
  }
  // 1. right-to-left orthogonalisation
  for (int k = d; k >= 2; --k) {
    const int64_t M = r[k - 1], N = n[k - 1] * r[k];
    SvdOut sv;
    svd_truncated(G[k].get(), M, N, [](const std::vector<double>& sg) { return (int64_t)sg.size(); }, max_sweeps,
                  sv, s, mixed, 2);
    st.jacobi_sweeps += sv.sweeps;
    const int64_t q = sv.r;
    G[k] = std::move(sv.Vt);
    DBuf<double> US((size_t)(M * q), s);
    scale_cols_kernel<<<grid_for(M * q), 256, 0, s>>>(sv.U.get(), M, q, sv.sigma.get(), US.get());
    FTT_LAUNCH();
    const int64_t Mp = r[k - 2] * n[k - 2];
    DBuf<double> Gp((size_t)(Mp * q), s);
    gemm(mixed, Mp, q, M, 1.0, G[k - 1].get(), M, 1, US.get(), q, 1, 0.0, Gp.get(), q, 1, s);
    G[k - 1] = std::move(Gp);
    r[k - 1] = q;
  }
  // 2.-3. norm from the first bond's singular values, then left-to-right compression
  double normA = 0.0, delta = 0.0, err2 = 0.0;
  if (d == 1) {
    SvdOut sv;   // ||A|| of a one-mode TT: the single singular value of the 1 x n_1 core
    svd_truncated(G[1].get(), 1, n[0], [](const std::vector<double>&) { return (int64_t)1; }, max_sweeps, sv, s,
                  mixed, 0);
    normA = sv.sigma_all.empty() ? 0.0 : sv.sigma_all[0];
  }
  for (int k = 1; k <= d - 1; ++k) {
    const int64_t M = r[k - 1] * n[k - 1], N = r[k];
    SvdOut sv;
    svd_truncated(G[k].get(), M, N, [&](const std::vector<double>& sg) {
      if (k == 1) {
        double acc = 0.0;
        for (size_t i = sg.size(); i-- > 0;) acc += sg[i] * sg[i];
        normA = std::sqrt(acc);
        delta = eps * normA / std::sqrt((double)(d - 1));
      }
      return rank_rule(sg, delta, eps0, n, k, o.max_rank);
    }, max_sweeps, sv, s, mixed, 1);
    st.jacobi_sweeps += sv.sweeps;
    err2 += tail2(sv.sigma_all, sv.r);
    st.deltas[k] = delta;
    if (o.keep_intermediates) {
      if (H.sigmas.empty()) H.sigmas.assign(d + 1, {});
      H.sigmas[k] = sv.sigma_all;
    }
    const int64_t rr = sv.r;
    G[k] = std::move(sv.U);
    DBuf<double> W((size_t)(rr * N), s);
    scale_rows_kernel<<<grid_for(rr * N), 256, 0, s>>>(sv.Vt.get(), rr, N, sv.sigma.get(), W.get());
    FTT_LAUNCH();
    const int64_t N1 = n[k] * r[k + 1];
    DBuf<double> Gn((size_t)(rr * N1), s);
    gemm(mixed, rr, N1, N, 1.0, W.get(), N, 1, G[k + 1].get(), N1, 1, 0.0, Gn.get(), N1, 1, s);
    G[k + 1] = std::move(Gn);
    r[k] = rr;
  }
  st.norm2 = normA * normA;
  st.err2 = err2;
  H.d = d;
  H.dims = n;
  H.ranks = r;
  H.cores.clear();
  for (int k = 1; k <= d; ++k) H.cores.push_back(std::move(G[k]));
  for (int k = 0; k <= d; ++k) st.ranks[k] = r[k];
  H.kept = o.keep_intermediates != 0;
  st.ms_round = total.lap();
  st.ms_total = st.ms_round;
  ozaki_take_timeout(s);
  finish_stats(st, launches0);
  finish_block_stats(st, snap0);
}

// Lemma 2 (eq. (6)): the cores of A + beta B.  Core 1 is [A_1, beta B_1] (columns),
// core d is [A_d; B_d] (rows), the cores in between are block diagonal; for d = 1
// the single core is A_1 + beta B_1.  Ranks r_k^A + r_k^B for 0 < k < d.
void add_tt(int d, const int64_t* dims, const int64_t* ranks_a, const double* const* cores_a, const int64_t* ranks_b,
            const double* const* cores_b, double beta, cudaStream_t s, Handle& H) {
  check_tt(d, dims, ranks_a, cores_a, "tt_add (A)");
  check_tt(d, dims, ranks_b, cores_b, "tt_add (B)");
  if (!std::isfinite(beta)) fail(FASTTT_EINVAL, "tt_add: beta must be finite");
  const int64_t launches0 = launch_count();
  Timer total(s);
  std::vector<int64_t> n(dims, dims + d), r(d + 1, 1);
  for (int k = 1; k < d; ++k) r[k] = ranks_a[k] + ranks_b[k];
  H.cores.clear();
  for (int k = 1; k <= d; ++k) {
    const int64_t ra0 = ranks_a[k - 1], ra1 = ranks_a[k], rb0 = ranks_b[k - 1], rb1 = ranks_b[k], nk = n[k - 1];
    DBuf<double> C((size_t)(r[k - 1] * nk * r[k]), s);
    FTT_CUDA(cudaMemsetAsync(C.get(), 0, C.bytes(), s));
    const bool one = (d == 1);
    const int64_t ob0 = (k == 1) ? 0 : ra0, ob1 = (k == d) ? 0 : ra1;   // offsets of B's block
    place_block_kernel<<<grid_for(ra0 * nk * ra1), 256, 0, s>>>(cores_a[k - 1], ra0, nk, ra1, 1.0, C.get(), r[k], 0, 0,
                                                                false);
    FTT_LAUNCH();
    place_block_kernel<<<grid_for(rb0 * nk * rb1), 256, 0, s>>>(cores_b[k - 1], rb0, nk, rb1, k == 1 ? beta : 1.0,
                                                                C.get(), r[k], one ? 0 : ob0, one ? 0 : ob1, one);
    FTT_LAUNCH();
    H.cores.push_back(std::move(C));
  }
  fasttt_stats& st = H.st;
  st.d = d;
  H.d = d;
  H.dims = n;
  H.ranks = r;
  for (int k = 0; k <= d; ++k) st.ranks[k] = r[k];
  st.ms_total = total.lap();
  st.launches = launch_count() - launches0;
}

int handle_error(const Error& e) {
  g_last_error = e.what();
  return e.code;
}

// A call that failed after a tensor-core GEMM gave up on a bounded wait computed on
// that GEMM's unfinished output: report the give-up (ETIMEOUT) as the cause, and
// clear the sticky flag so that it does not fail the next call.
int timeout_as_cause(int rc, cudaStream_t s) {
  if (rc == FASTTT_ETIMEOUT) {
    ozaki_clear_timeout(s);
    return rc;
  }
  if (ozaki_clear_timeout(s)) {
    g_last_error = "tensor-core GEMM: a bounded wait gave up (then: " + g_last_error + ")";
    note_wait_timeout();
    return FASTTT_ETIMEOUT;
  }
  return rc;
}

}  // namespace

void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

}  // namespace fasttt

using namespace fasttt;

namespace {
// Runs body (which fills a fresh handle) under the ABI's error conventions.
template <class F>
int make_handle(void* stream, fasttt_tt** out, fasttt_stats* stats, F&& body) {
  g_last_error.clear();
  if (!out) {
    g_last_error = "null argument";
    return FASTTT_EINVAL;
  }
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::unique_ptr<fasttt_tt> tt(new fasttt_tt());
  int rc = FASTTT_OK;
  try {
    body(s, tt->h);
  } catch (const Error& e) {
    rc = handle_error(e);
  } catch (const std::exception& e) {
    g_last_error = e.what();
    rc = FASTTT_ECUDA;
  }
  if (rc != FASTTT_OK) {
    cudaStreamSynchronize(s);
    rc = timeout_as_cause(rc, s);
  }
  tt->h.st.wait_timeouts = wait_timeouts() - tt->h.wait0;
  if (stats) *stats = tt->h.st;
  if (rc != FASTTT_OK) return rc;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    g_last_error = std::string("CUDA error: ") + cudaGetErrorString(e);
    return FASTTT_ECUDA;
  }
  *out = tt.release();
  return FASTTT_OK;
}
}  // namespace

extern "C" {

void fasttt_default_opts(fasttt_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->p = 0;
  o->precision = FASTTT_PREC_FP64;
  o->rounding = FASTTT_STATIC;
  o->depar_values = 1;
  o->stage = FASTTT_STAGE_FULL;
  o->keep_intermediates = 0;
  o->max_rank = 0;
  o->max_sweeps = 0;
}

int fasttt_decompose(int d, const int64_t* dims, int64_t nnz, const int32_t* d_idx, const void* d_vals,
                     int val_dtype, double eps, const fasttt_opts* opts, void* stream, fasttt_tt** out,
                     fasttt_stats* stats) {
  g_last_error.clear();
  if (!out || !dims) {
    g_last_error = "null argument";
    return FASTTT_EINVAL;
  }
  *out = nullptr;
  fasttt_opts o;
  if (opts) o = *opts;
  else fasttt_default_opts(&o);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::unique_ptr<fasttt_tt> tt(new fasttt_tt());
  int rc = FASTTT_OK;
  try {
    run(d, dims, nnz, d_idx, d_vals, val_dtype, eps, o, s, tt->h);
  } catch (const Error& e) {
    rc = handle_error(e);
  } catch (const std::exception& e) {
    g_last_error = e.what();
    rc = FASTTT_ECUDA;
  }
  if (rc != FASTTT_OK) {
    cudaStreamSynchronize(s);
    rc = timeout_as_cause(rc, s);
  }
  tt->h.st.wait_timeouts = wait_timeouts() - tt->h.wait0;
  if (stats) *stats = tt->h.st;
  if (rc != FASTTT_OK) return rc;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    g_last_error = std::string("CUDA error: ") + cudaGetErrorString(e);
    return FASTTT_ECUDA;
  }
  *out = tt.release();
  return FASTTT_OK;
}

int fasttt_tt_round(int d, const int64_t* dims, const int64_t* ranks, const double* const* d_cores, double eps,
                    const fasttt_opts* opts, void* stream, fasttt_tt** out, fasttt_stats* stats) {
  fasttt_opts o;
  if (opts) o = *opts;
  else fasttt_default_opts(&o);
  return make_handle(stream, out, stats, [&](cudaStream_t s, Handle& H) {
    round_tt(d, dims, ranks, d_cores, eps, o, s, H);
  });
}

int fasttt_tt_add(int d, const int64_t* dims, const int64_t* ranks_a, const double* const* d_cores_a,
                  const int64_t* ranks_b, const double* const* d_cores_b, double beta, void* stream,
                  fasttt_tt** out) {
  return make_handle(stream, out, nullptr, [&](cudaStream_t s, Handle& H) {
    add_tt(d, dims, ranks_a, d_cores_a, ranks_b, d_cores_b, beta, s, H);
  });
}

void fasttt_tt_free(fasttt_tt* tt) {
  if (!tt) return;
  cudaDeviceSynchronize();
  g_free_sync = true;
  delete tt;
  g_free_sync = false;
}

int fasttt_tt_stats(const fasttt_tt* tt, fasttt_stats* st) {
  if (!tt || !st) return FASTTT_EINVAL;
  *st = tt->h.st;
  return FASTTT_OK;
}

int fasttt_tt_ranks(const fasttt_tt* tt, int64_t* ranks) {
  if (!tt || !ranks) return FASTTT_EINVAL;
  for (int k = 0; k <= tt->h.d; ++k) ranks[k] = tt->h.ranks[k];
  return FASTTT_OK;
}

int fasttt_tt_core(const fasttt_tt* tt, int k, const double** d_core) {
  if (!tt || !d_core || k < 1 || k > tt->h.d || tt->h.cores.empty()) return FASTTT_EINVAL;
  *d_core = tt->h.cores[k - 1].get();
  return FASTTT_OK;
}

namespace {
struct ArrRef {
  const void* p = nullptr;
  int64_t n = -1;
  size_t elem = 0;
};

ArrRef lookup(const fasttt_tt* tt, int what, int k) {
  ArrRef a;
  if (!tt) return a;
  const Handle& H = tt->h;
  const int p = H.st.p, d = H.d;
  auto set = [&](const void* ptr, int64_t n, size_t e) { a.p = ptr; a.n = n; a.elem = e; };
  switch (what) {
    case FASTTT_ARR_CORE:
      if (k >= 1 && k <= d && !H.cores.empty())
        set(H.cores[k - 1].get(), H.ranks[k - 1] * H.dims[k - 1] * H.ranks[k], 8);
      break;
    case FASTTT_ARR_LEFT_PARENT:
    case FASTTT_ARR_LEFT_INDEX:
      if (H.kept && k >= 1 && k < p) {
        const auto& b = (what == FASTTT_ARR_LEFT_PARENT) ? H.grp.left_parent[k - 1] : H.grp.left_index[k - 1];
        set(b.get(), H.st.rt[k], 4);
      }
      break;
    case FASTTT_ARR_RIGHT_INDEX:
    case FASTTT_ARR_RIGHT_CHILD:
      if (H.kept && k > p && k <= d) {
        const auto& b = (what == FASTTT_ARR_RIGHT_INDEX) ? H.grp.right_index[k - p - 1] : H.grp.right_child[k - p - 1];
        set(b.get(), H.st.rt[k - 1], 4);
      }
      break;
    case FASTTT_ARR_MID_ROW: if (H.kept) set(H.grp.mid_row.get(), H.st.nnz, 8); break;
    case FASTTT_ARR_MID_COL: if (H.kept) set(H.grp.mid_col.get(), H.st.nnz, 8); break;
    case FASTTT_ARR_MID_VAL: if (H.kept) set(H.grp.mid_val.get(), H.st.nnz, 8); break;
    case FASTTT_ARR_ROW_ID: if (H.kept && H.dep.rows.nz) set(H.dep.rows.ids.get(), H.dep.rows.nz, 8); break;
    case FASTTT_ARR_ROW_CLASS: if (H.kept && H.dep.rows.nz) set(H.dep.rows.cls.get(), H.dep.rows.nz, 4); break;
    case FASTTT_ARR_ROW_PREF: if (H.kept && H.dep.rows.nz) set(H.dep.rows.pref.get(), H.dep.rows.nz, 8); break;
    case FASTTT_ARR_COL_ID: if (H.kept && H.dep.cols.nz) set(H.dep.cols.ids.get(), H.dep.cols.nz, 8); break;
    case FASTTT_ARR_COL_CLASS: if (H.kept && H.dep.cols.nz) set(H.dep.cols.cls.get(), H.dep.cols.nz, 4); break;
    case FASTTT_ARR_COL_PREF: if (H.kept && H.dep.cols.nz) set(H.dep.cols.pref.get(), H.dep.cols.nz, 8); break;
    case FASTTT_ARR_DP_ROW: if (H.kept && H.dep.dp_n) set(H.dep.dp_row.get(), H.dep.dp_n, 4); break;
    case FASTTT_ARR_DP_COL: if (H.kept && H.dep.dp_n) set(H.dep.dp_col.get(), H.dep.dp_n, 4); break;
    case FASTTT_ARR_DP_VAL: if (H.kept && H.dep.dp_n) set(H.dep.dp_val.get(), H.dep.dp_n, 8); break;
    case FASTTT_ARR_LAM_S: if (H.kept && H.dep.rows.beta) set(H.dep.rows.lam.get(), H.dep.rows.beta, 8); break;
    case FASTTT_ARR_LAM_T: if (H.kept && H.dep.cols.beta) set(H.dep.cols.lam.get(), H.dep.cols.beta, 8); break;
    case FASTTT_ARR_SIGMA:
      if (H.kept && k >= 1 && k < d && k < (int)H.sigmas.size() && !H.sigmas[k].empty())
        set(H.sigmas[k].data(), (int64_t)H.sigmas[k].size(), 8);
      break;
    default: break;
  }
  return a;
}
}  // namespace

int64_t fasttt_tt_count(const fasttt_tt* tt, int what, int k) {
  ArrRef a = lookup(tt, what, k);
  if (a.n < 0) {
    g_last_error = "array not available";
    return FASTTT_EINVAL;
  }
  return a.n;
}

int fasttt_tt_copy(const fasttt_tt* tt, int what, int k, void* dst, int64_t count) {
  ArrRef a = lookup(tt, what, k);
  if (a.n < 0 || count != a.n || (!dst && count)) {
    g_last_error = "array not available or count mismatch";
    return FASTTT_EINVAL;
  }
  if (count == 0) return FASTTT_OK;
  cudaError_t e = cudaMemcpy(dst, a.p, (size_t)count * a.elem, cudaMemcpyDefault);
  if (e != cudaSuccess) {
    g_last_error = std::string("copy failed: ") + cudaGetErrorString(e);
    return FASTTT_ECUDA;
  }
  return FASTTT_OK;
}

int tt_eval_at(int d, const int64_t* dims, const int64_t* ranks, const void* const* d_cores, int dtype, int64_t m,
               const int32_t* d_idx, void* d_out, void* stream) {
  g_last_error.clear();
  try {
    return tt_eval_at_impl(d, dims, ranks, d_cores, dtype, m, d_idx, d_out, static_cast<cudaStream_t>(stream));
  } catch (const Error& e) {
    return handle_error(e);
  }
}

int tt_eval_backward(int d, const int64_t* dims, const int64_t* ranks, const void* const* d_cores, int dtype,
                     int64_t m, const int32_t* d_idx, const void* d_grad_out, void* const* d_grad_cores,
                     int recompute, void* stream) {
  g_last_error.clear();
  try {
    return tt_eval_backward_impl(d, dims, ranks, d_cores, dtype, m, d_idx, d_grad_out, d_grad_cores, recompute,
                                 static_cast<cudaStream_t>(stream));
  } catch (const Error& e) {
    return handle_error(e);
  }
}

const char* fasttt_last_error(void) { return g_last_error.c_str(); }

const char* fasttt_version(void) { return "fasttt-gb300 0.1 (sm_103a)"; }

void fasttt_debug_fail_alloc_after(int64_t n) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_fail_after = n > 0 ? n : 0;
}

int fasttt_debug_select_p(int d, const int64_t* dims, const int64_t* Rs, int64_t max_rank) {
  g_last_error.clear();
  try {
    if (d < 2 || d > FASTTT_MAX_D || !dims || !Rs || max_rank < 0) fail(FASTTT_EINVAL, "select_p: bad arguments");
    for (int k = 0; k < d; ++k) {
      if (dims[k] < 1 || dims[k] > INT32_MAX) fail(FASTTT_EINVAL, "select_p: mode sizes must be in 1..2^31-1");
      if (Rs[k] < 1 || Rs[k] > INT32_MAX) fail(FASTTT_EINVAL, "select_p: R must be in 1..2^31-1");
    }
    return select_p_host(std::vector<int64_t>(dims, dims + d), std::vector<int64_t>(Rs, Rs + d), max_rank);
  } catch (const Error& e) {
    return handle_error(e);
  }
}

int64_t fasttt_debug_rank_rule(const double* h_sigma, int64_t n, double delta, int eps_zero, int d,
                               const int64_t* dims, int bond, int64_t max_rank) {
  g_last_error.clear();
  try {
    if (!h_sigma || n < 1 || d < 2 || d > FASTTT_MAX_D || !dims || bond < 1 || bond >= d || max_rank < 0 ||
        !(delta >= 0.0))
      fail(FASTTT_EINVAL, "rank_rule: bad arguments");
    return rank_rule(std::vector<double>(h_sigma, h_sigma + n), delta, eps_zero != 0,
                     std::vector<int64_t>(dims, dims + d), bond, max_rank);
  } catch (const Error& e) {
    return handle_error(e);
  }
}

int fasttt_debug_gemm(int64_t M, int64_t N, int64_t K, const double* d_A, const double* d_B, double* d_C, int engine,
                      void* stream) {
  try {
    if (M < 1 || N < 1 || K < 1 || !d_A || !d_B || !d_C || engine < 0 || engine > 3)
      fail(FASTTT_EINVAL, "fasttt_debug_gemm: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (engine == 0) gemm_f64_dfma(M, N, K, 1.0, d_A, K, 1, d_B, N, 1, 0.0, d_C, N, 1, s);
    else if (engine == 3) gemm_tf32x3(M, N, K, 1.0, d_A, K, 1, d_B, N, 1, 0.0, d_C, N, 1, s);
    else if (!gemm_ozaki(engine == 1 ? 7 : 3, M, N, K, 1.0, d_A, K, 1, d_B, N, 1, 0.0, d_C, N, 1, s))
      fail(FASTTT_ENUMERIC, "tensor-core GEMM declined or gave up");
    FTT_CUDA(cudaStreamSynchronize(s));
    ozaki_take_timeout(s);
    return FASTTT_OK;
  } catch (const Error& e) {
    return handle_error(e);
  }
}

int fasttt_debug_svd(int64_t M, int64_t N, const double* d_Z, double* h_sigma, double* d_U, double* d_Vt,
                     int precision, void* stream) {
  try {
    if (M < 1 || N < 1 || !d_Z || !h_sigma || !d_U || !d_Vt ||
        (precision != FASTTT_PREC_FP64 && precision != FASTTT_PREC_MIXED))
      fail(FASTTT_EINVAL, "fasttt_debug_svd: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    set_gemm_engine(FASTTT_GEMM_TENSOR);
    SvdOut sv;
    svd_truncated(d_Z, M, N, [](const std::vector<double>& sg) { return (int64_t)sg.size(); }, 200, sv, s,
                  precision == FASTTT_PREC_MIXED, 0);
    const int64_t r = sv.r;
    FTT_CUDA(cudaMemcpyAsync(d_U, sv.U.get(), sizeof(double) * M * r, cudaMemcpyDeviceToDevice, s));
    FTT_CUDA(cudaMemcpyAsync(d_Vt, sv.Vt.get(), sizeof(double) * r * N, cudaMemcpyDeviceToDevice, s));
    FTT_CUDA(cudaStreamSynchronize(s));
    ozaki_take_timeout(s);
    std::copy(sv.sigma_all.begin(), sv.sigma_all.begin() + r, h_sigma);
    return FASTTT_OK;
  } catch (const Error& e) {
    return handle_error(e);
  }
}

int fasttt_debug_cholqr(int64_t M, int64_t N, double* d_Z, double* d_R, int precision, void* stream) {
  try {
    if (M < 1 || N < M || !d_Z || !d_R || (precision != FASTTT_PREC_FP64 && precision != FASTTT_PREC_MIXED))
      fail(FASTTT_EINVAL, "fasttt_debug_cholqr: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    set_gemm_engine(FASTTT_GEMM_TENSOR);
    const bool ok = cholqr2_rows(d_Z, M, N, d_R, precision == FASTTT_PREC_MIXED, s);
    FTT_CUDA(cudaStreamSynchronize(s));
    ozaki_take_timeout(s);
    if (!ok) fail(FASTTT_ENUMERIC, "CholeskyQR2 broke down (matrix too ill conditioned for the Gram's precision)");
    return FASTTT_OK;
  } catch (const Error& e) {
    return handle_error(e);
  }
}

int fasttt_debug_gram(int64_t M, int64_t K, const double* d_A, double* d_C, int engine, void* stream) {
  try {
    if (M < 1 || K < 1 || !d_A || !d_C || engine < 0 || engine > 3)
      fail(FASTTT_EINVAL, "fasttt_debug_gram: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // A(i, k) = A[i K + k], B(k, j) = A[j K + k]
    if (engine == 0) gemm_f64_dfma(M, M, K, 1.0, d_A, K, 1, d_A, 1, K, 0.0, d_C, M, 1, s, true);
    else if (engine == 3) gemm_tf32x3(M, M, K, 1.0, d_A, K, 1, d_A, 1, K, 0.0, d_C, M, 1, s, true);
    else if (!gemm_ozaki(engine == 1 ? 7 : 3, M, M, K, 1.0, d_A, K, 1, d_A, 1, K, 0.0, d_C, M, 1, s, true))
      fail(FASTTT_ENUMERIC, "tensor-core GEMM declined or gave up");
    FTT_CUDA(cudaStreamSynchronize(s));
    ozaki_take_timeout(s);
    return FASTTT_OK;
  } catch (const Error& e) {
    return handle_error(e);
  }
}

int fasttt_debug_sym_eig(const double* d_G, int64_t n, double* d_V, double* h_lam, int method, void* stream) {
  try {
    if (!d_G || !d_V || !h_lam || n < 1 || n > INT32_MAX / 2 || method < 0 || method > 3)
      fail(FASTTT_EINVAL, "fasttt_debug_sym_eig: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<double> lam;
    bool ok = false;
    if (method == 2 || method == 3) ok = sym_eig_fast(d_G, (int)n, d_V, lam, 40, s, false);
    if (!ok && method == 3) fail(FASTTT_ENUMERIC, "fast route declined");
    if (!ok && method != 1) ok = sym_eig_tridiag(d_G, (int)n, d_V, lam, s, false);
    if (!ok && method == 0) fail(FASTTT_ENUMERIC, "tridiagonal route declined");
    if (!ok) sym_eig_iterative(d_G, (int)n, d_V, lam, 40, s);
    FTT_CUDA(cudaStreamSynchronize(s));
    ozaki_take_timeout(s);
    std::copy(lam.begin(), lam.end(), h_lam);
    return FASTTT_OK;
  } catch (const Error& e) {
    return handle_error(e);
  }
}

}  // extern "C"
