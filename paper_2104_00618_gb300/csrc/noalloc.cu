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

// 5 MiB: the float32 gradient pyramid (plus header) of a dense or bricked
// grid up to 64^3 (4.79 MB), or of an anisotropic one up to 32^3 (0.97 MB;
// its coarse levels hold six volumes each, 7.79 MB at 64^3).
constexpr size_t kNoAllocScratchBytes = (size_t)5 << 20;

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_bwd_scratch[kNoAllocScratchBytes];

// The array's device address belongs to a CUDA context: the primary context
// of a device, or a context the caller created and made current.  In host
// code the array's name is only a host-side stand-in, so the address is
// looked up (cudaGetSymbolAddress) in the current context on every call made
// outside a stream capture, and kept per context ID (unique for the life of
// the process: a context that is destroyed and re-created, e.g. by
// cudaDeviceReset, gets a new ID).  A call made while its stream is being
// captured takes the address kept for the current context and fails if there
// is none.
constexpr int kCachedContexts = 64;
struct CachedAddress {
  unsigned long long ctx_id;
  void *ptr;
};
std::mutex g_mu;
CachedAddress g_cache[kCachedContexts] = {};
int g_next = 0;

typedef CUresult (*PFN_ctx_get_current)(CUcontext *);
typedef CUresult (*PFN_ctx_get_id)(CUcontext, unsigned long long *);

template <typename F>
F driver_fn(const char *name) {
  void *p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<F>(p);
}

// ID of the context current on this thread.
cudaError_t current_context_id(unsigned long long *id) {
  static PFN_ctx_get_current get_current = nullptr;
  static PFN_ctx_get_id get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    get_current = driver_fn<PFN_ctx_get_current>("cuCtxGetCurrent");
    get_id = driver_fn<PFN_ctx_get_id>("cuCtxGetId");
  });
  if (!get_current || !get_id) return cudaErrorNotSupported;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return cudaErrorDeviceUninitialized;
  if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

// Device address of g_bwd_scratch in the current context.
vct_status scratch_for_current_context(cudaStream_t stream, void **out) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &cs);
  if (e != cudaSuccess)
    return vct::set_last_error(VCT_ERR_CUDA, "vct_trace_backward_noalloc: %s",
                               cudaGetErrorString(e));
  // Outside a capture the lookup comes first: it binds the device's primary
  // context to this thread if no context is current yet.
  void *p = nullptr;
  if (cs == cudaStreamCaptureStatusNone) {
    e = cudaGetSymbolAddress(&p, g_bwd_scratch);
    if (e != cudaSuccess)
      return vct::set_last_error(VCT_ERR_CUDA,
                                 "vct_trace_backward_noalloc: cudaGetSymbolAddress: %s",
                                 cudaGetErrorString(e));
  }
  unsigned long long id = 0;
  e = current_context_id(&id);
  if (e != cudaSuccess)
    return vct::set_last_error(VCT_ERR_CUDA,
                               "vct_trace_backward_noalloc: current context: %s",
                               cudaGetErrorString(e));
  std::lock_guard<std::mutex> g(g_mu);
  int slot = -1;
  for (int i = 0; i < kCachedContexts; ++i)
    if (g_cache[i].ptr != nullptr && g_cache[i].ctx_id == id) slot = i;
  if (cs != cudaStreamCaptureStatusNone) {
    if (slot < 0)
      return vct::set_last_error(
          VCT_ERR_CUDA,
          "vct_trace_backward_noalloc: called during a stream capture in a context where "
          "it has not been called before (make one call in this context first)");
    *out = g_cache[slot].ptr;
    return VCT_OK;
  }
  if (slot < 0) {
    slot = g_next;
    g_next = (g_next + 1) % kCachedContexts;
  }
  g_cache[slot].ctx_id = id;
  g_cache[slot].ptr = p;
  *out = p;
  return VCT_OK;
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
  if (need > kNoAllocScratchBytes) {
    const bool aniso = pyr->layout == VCT_LAYOUT_ANISO;
    return vct::set_last_error(
        VCT_ERR_WORKSPACE,
        "vct_trace_backward_noalloc: this %s pyramid (n = %d, %d levels) needs %zu bytes of "
        "scratch; the fixed scratch array holds %zu bytes (%s)",
        aniso ? "anisotropic" : (pyr->layout == VCT_LAYOUT_BRICKS ? "bricked" : "dense"),
        pyr->n, pyr->levels, need, kNoAllocScratchBytes,
        aniso ? "anisotropic grids up to 32^3" : "dense and bricked grids up to 64^3");
  }
  void *scratch = nullptr;
  const vct_status st = scratch_for_current_context((cudaStream_t)stream, &scratch);
  if (st != VCT_OK) return st;
  return vct_trace_backward(pyr, views, grads, n_views, params, cfg, grad_level0_dense, scratch,
                            kNoAllocScratchBytes, stream);
}
