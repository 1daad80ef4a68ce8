// vct_trace_backward_noalloc: the adjoint for callers that cannot allocate
// device memory.  Its scratch (the float32 gradient pyramid and work-queue
// header that vct_trace_backward takes as `workspace`) lives in a file-scope
// device array of fixed size, so the caller passes only inputs and outputs.
//
// Some callers cannot call cudaMalloc: host applications that hand a plugin
// only pre-sized buffers and no allocator, code that runs where the device
// heap is partitioned up front, or callers that must not perturb a memory
// pool they do not own.  This entry point needs no allocation at any point.
#include <mutex>

#include "vct_internal.cuh"

namespace {

// 5 MiB: the float32 gradient pyramid (plus header) of any grid up to 64^3.
constexpr size_t kNoAllocScratchBytes = (size_t)5 << 20;
constexpr int kMaxDevices = 64;

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_bwd_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_bwd_scratch on the current device (looked up once per
// device: in host code the array's name is only a host-side stand-in).
cudaError_t scratch_for_current_device(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_bwd_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" vct_status vct_trace_backward_noalloc(const vct_pyramid *pyr, const vct_view *views,
                                                 const vct_view_grad *grads, int32_t n_views,
                                                 const vct_trace_params *params,
                                                 const vct_launch_config *cfg,
                                                 float *grad_level0_dense, vct_stream_t stream) {
  const size_t need = vct_trace_backward_workspace_bytes(pyr);
  if (need == 0)  // invalid pyramid: let the regular entry point report it
    return vct_trace_backward(pyr, views, grads, n_views, params, cfg, grad_level0_dense,
                              nullptr, 0, stream);
  if (need > kNoAllocScratchBytes)
    return vct::set_last_error(
        VCT_ERR_WORKSPACE,
        "vct_trace_backward_noalloc: this pyramid needs %zu bytes of scratch; the fixed "
        "scratch array holds %zu bytes (grids up to 64^3)",
        need, kNoAllocScratchBytes);
  void *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess)
    return vct::set_last_error(VCT_ERR_CUDA,
                               "vct_trace_backward_noalloc: cudaGetSymbolAddress: %s",
                               cudaGetErrorString(e));
  return vct_trace_backward(pyr, views, grads, n_views, params, cfg, grad_level0_dense, scratch,
                            kNoAllocScratchBytes, stream);
}
