// Shared host/device helpers of libfasttt: error handling, stream-ordered device
// buffers (with the allocation-failure test hook) and launch sizing for GB300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <string>
#include <utility>

#include "../../include/fasttt.h"

namespace fasttt {

// GB300: 152 SMs on two dies.
constexpr int kNumSMs = 152;

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] inline void fail(int code, const std::string& msg) { throw Error(code, msg); }

inline void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
  if (e != cudaSuccess) {
    int code = (e == cudaErrorMemoryAllocation) ? FASTTT_ENOMEM : FASTTT_ECUDA;
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
    fail(code, buf);
  }
}
// Kernel launches of this process (every launch site reports itself).
void note_launches(int64_t n);
int64_t launch_count();
// Jacobi sweeps run on the block (shared-memory) schedule, and the last CUDA error
// a cooperative launch returned (0 if none), for the statistics.
void note_block_sweep(int err);
int64_t block_sweep_count();
int last_coop_error();
void note_eig(bool tridiag);
void note_eig_fast();
// GEMM engine for the FP64 GEMMs of the calling thread: 0 = tensor cores (exact bf16
// slices) for large products, 1 = FP64 DFMA only.
void set_gemm_engine(int engine);
// Poll bound of the device spin-waits for the calling thread's next calls (the
// max_spin option): 0 = each wait's default bound, with the cooperative kernels
// falling back to one launch per round when a grid barrier gives up; > 0 = that
// bound, and a wait that gives up fails the call with FASTTT_ETIMEOUT.
void set_max_spin(int64_t spins);
int64_t max_spin();
// Device waits that gave up since the library was loaded (statistics).
void note_wait_timeout();
int64_t wait_timeouts();
// The grid-barrier poll bound to store in bar[3] (0 = the kernel's default).
inline unsigned barrier_spins() {
  const int64_t v = max_spin();
  return v <= 0 ? 0u : (v > 0xFFFFFFFFll ? 0xFFFFFFFFu : (unsigned)v);
}
int gemm_engine();   // Gram eigensolver: tridiagonal route taken, or the iterative fallback

#define FTT_CUDA(call) ::fasttt::cuda_check((call), #call, __FILE__, __LINE__)
#define FTT_LAUNCH()                                                             \
  do {                                                                           \
    ::fasttt::note_launches(1);                                                  \
    ::fasttt::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__); \
  } while (0)

// Per-call device timing of the heavy kernel classes, by CUDA events on the
// launching stream (read once at the end of a call).
enum KernelClass {
  KC_GEMM = 0,
  KC_JACOBI = 1,
  KC_SORT = 2,
  KC_JACOBI32 = 3,
  KC_GEMM_TC = 4,
  KC_TRIDIAG = 5,   // Householder tridiagonalisation
  KC_TDEIG = 6,     // bisection + inverse iteration on the tridiagonal matrix
  KC_GEMM_OZ = 7,   // tcgen05 GEMMs on exact bf16 slices of FP64 operands
  KC_TRIDIAG32 = 8, // FP32 tridiagonalisation (fast eigensolver start)
  KC_TSQR = 9,      // Householder TSQR and its Q application
  KC_COUNT = 10
};
struct KClock {
  cudaEvent_t a = nullptr, b = nullptr;
  int cls = 0;
  double work = 0.0;  // algorithmic flops (GEMM, Jacobi) or bytes (sort)
};
void kclock_begin(KClock& c, int cls, cudaStream_t s);
void kclock_end(KClock& c, double work, cudaStream_t s);
void kclock_reset();
// Sums (ms, work) per class over the clocks recorded since the last reset.
void kclock_collect(double ms[KC_COUNT], double work[KC_COUNT]);

void* dev_alloc(size_t bytes, cudaStream_t s);   // stream-ordered, honours the failure hook
void dev_free(void* p, cudaStream_t s);

// Owning, stream-ordered device array.
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(size_t count, cudaStream_t st) : n(count), s(st) {
    p = count ? static_cast<T*>(dev_alloc(count * sizeof(T), st)) : nullptr;
  }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { reset(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { reset(); }
  void reset() { if (p) dev_free(p, s); p = nullptr; n = 0; }
  T* get() const { return p; }
  size_t bytes() const { return n * sizeof(T); }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Grid for grid-stride element-wise kernels: a multiple of the SM count,
// never more blocks than there is work for.
inline int grid_for(int64_t n, int block = 256, int per_sm = 8) {
  int64_t need = ceil_div(n > 0 ? n : 1, block);
  int64_t cap = (int64_t)kNumSMs * per_sm;
  return (int)(need < cap ? need : cap);
}

template <typename T>
inline T read_scalar(const T* d, cudaStream_t s) {
  T h;
  FTT_CUDA(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, s));
  FTT_CUDA(cudaStreamSynchronize(s));
  return h;
}

// ---------------------------------------------------------------- primitives (prims.cu)

// Exclusive prefix sum of n values (int64 accumulate); out may alias in.  Returns total.
int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
int64_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the keys.
// keys/vals are sorted in place (alt buffers are scratch of the same size).
void radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                      int64_t n, int bits, cudaStream_t s);

// After a sort: ranks[vals[i]] = (dense rank of keys[i]); distinct keys written to
// uniq (capacity n).  Returns the number of distinct keys.
int64_t rank_sorted(const uint64_t* keys, const uint32_t* vals, int64_t n, int32_t* ranks,
                    uint64_t* uniq, cudaStream_t s);

inline int bits_for(uint64_t count) {  // bits needed for values 0..count-1
  int b = 0;
  while (b < 64 && (count - 1) >> b) ++b;
  return b;
}

}  // namespace fasttt
