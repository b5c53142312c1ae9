// tt_eval_backward_noalloc: the entry-evaluation adjoint for callers that cannot
// allocate device memory.  Its scratch (an error flag and the per-warp left
// partial products) lives in the file-scope device array below, which every GPU
// that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include "common.cuh"

namespace fasttt {
int tt_eval_backward_prealloc(int d, const int64_t* dims, const int64_t* ranks, const void* const* cores,
                              int dtype, int64_t m, const int32_t* idx, const void* gout, void* const* grads,
                              void* scratch, size_t scratch_bytes, cudaStream_t s);
void set_last_error(const char* msg);
}  // namespace fasttt

namespace {

constexpr size_t kScratchBytes = FASTTT_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host code cannot use g_noalloc_scratch's name as a device address: it is a
// host-side stand-in.  The device address is looked up on every call, with the
// caller's device current (the lookup allocates nothing), so it always names the
// array of the context the call runs in, also after a device reset.
void* scratch_for_current_device() {
  void* ptr = nullptr;
  FTT_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
  return ptr;
}

}  // namespace

extern "C" int tt_eval_backward_noalloc(int d, const int64_t* dims, const int64_t* ranks,
                                        const void* const* d_cores, int dtype, int64_t m,
                                        const int32_t* d_idx, const void* d_grad_out,
                                        void* const* d_grad_cores, void* stream) {
  ::fasttt::set_last_error("");
  try {
    void* scratch = scratch_for_current_device();
    return ::fasttt::tt_eval_backward_prealloc(d, dims, ranks, d_cores, dtype, m, d_idx, d_grad_out, d_grad_cores,
                                               scratch, kScratchBytes, static_cast<cudaStream_t>(stream));
  } catch (const ::fasttt::Error& e) {
    ::fasttt::set_last_error(e.what());
    return e.code;
  }
}
