// Host-buffer frame pipeline: two device slots and three streams (copies in,
// kernels, copies out) ordered by events, so that the copies of one frame
// overlap the mip build and trace of its neighbours.
#include <cmath>
#include <cstring>
#include <new>

#include "vct_internal.cuh"

struct vct_pipeline {
  vct_pipeline_desc desc;
  vct_trace_params params;
  cudaStream_t h2d, comp, d2h;
  cudaEvent_t start;          // recorded on the caller's stream at each submit
  cudaEvent_t in_free[2];     // slot inputs consumed (trace done)
  cudaEvent_t in_ready[2];    // slot inputs copied
  cudaEvent_t out_ready[2];   // slot outputs computed
  cudaEvent_t out_free[2];    // slot outputs copied back
  struct Slot {
    float *level0, *pos, *nrm, *rough, *D, *S, *V;
    uint8_t *mask, *pyr, *ws;
    uint64_t pyr_bytes;
  } slot[2];
  uint64_t frames;
  int device;
};

namespace {

size_t px_count(const vct_pipeline_desc &d) { return (size_t)d.width * d.height; }

void release(vct_pipeline *p) {
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  if (p->h2d) cudaStreamSynchronize(p->h2d);
  if (p->comp) cudaStreamSynchronize(p->comp);
  if (p->d2h) cudaStreamSynchronize(p->d2h);
  for (auto &s : p->slot) {
    void *bufs[] = {s.level0, s.pos, s.nrm, s.rough, s.D, s.S, s.V, s.mask, s.pyr, s.ws};
    for (void *b : bufs)
      if (b) cudaFree(b);
  }
  cudaEvent_t evs[] = {p->start,        p->in_free[0],   p->in_free[1], p->in_ready[0],
                       p->in_ready[1], p->out_ready[0], p->out_ready[1], p->out_free[0],
                       p->out_free[1]};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (p->h2d) cudaStreamDestroy(p->h2d);
  if (p->comp) cudaStreamDestroy(p->comp);
  if (p->d2h) cudaStreamDestroy(p->d2h);
  cudaSetDevice(cur);
  delete p;
}

vct_pyramid slot_pyramid(const vct_pipeline *p, int s) {
  vct_pyramid y{};
  y.n = p->desc.n;
  y.levels = p->desc.levels;
  y.dtype = p->desc.dtype;
  y.layout = VCT_LAYOUT_DENSE;
  for (int a = 0; a < 3; ++a) y.origin[a] = p->desc.origin[a];
  y.size = p->desc.size;
  y.data = p->slot[s].pyr;
  y.bytes = p->slot[s].pyr_bytes;
  return y;
}

}  // namespace

extern "C" {

vct_status vct_pipeline_create(const vct_pipeline_desc *desc, const vct_trace_params *params,
                               vct_pipeline **out) {
  if (!desc || !params || !out)
    return vct::set_last_error(VCT_ERR_INVALID_ARG, "vct_pipeline_create: NULL argument");
  *out = nullptr;
  const vct_pipeline_desc &d = *desc;
  const size_t pyr_bytes = vct_pyramid_bytes(d.n, d.levels, d.dtype);
  if (pyr_bytes == 0)
    return vct::set_last_error(VCT_ERR_INVALID_ARG, "vct_pipeline_create: bad pyramid shape");
  if (d.width < 1 || d.height < 1 || d.width > 65535 || d.height > 65535 ||
      (int64_t)d.width * d.height > ((int64_t)1 << 29))
    return vct::set_last_error(VCT_ERR_INVALID_ARG, "vct_pipeline_create: bad view size");
  if ((d.outputs & 7) == 0 || (d.outputs & ~7) != 0)
    return vct::set_last_error(VCT_ERR_INVALID_ARG, "vct_pipeline_create: outputs must be 1..7");
  if ((d.has_roughness != 0 && d.has_roughness != 1) || (d.has_mask != 0 && d.has_mask != 1))
    return vct::set_last_error(VCT_ERR_INVALID_ARG,
                               "vct_pipeline_create: has_roughness/has_mask must be 0 or 1");
  if (!(d.size > 0.0f) || !std::isfinite(d.size))
    return vct::set_last_error(VCT_ERR_INVALID_ARG, "vct_pipeline_create: bad size");
  if (params->flags & VCT_FLAG_SHADE)
    return vct::set_last_error(VCT_ERR_UNSUPPORTED,
                               "vct_pipeline_create: no radiance output in the pipeline");
  vct_pipeline *p = new (std::nothrow) vct_pipeline();
  if (!p) return vct::set_last_error(VCT_ERR_CUDA, "vct_pipeline_create: out of host memory");
  p->desc = d;
  p->params = *params;
  cudaGetDevice(&p->device);
  const size_t npx = px_count(d);
  const size_t n3 = (size_t)d.n * d.n * d.n;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](auto **ptr, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMalloc(reinterpret_cast<void **>(ptr), bytes);
  };
  for (auto &s : p->slot) {
    s.pyr_bytes = pyr_bytes;
    alloc(&s.level0, n3 * 16);
    alloc(&s.pyr, pyr_bytes);
    alloc(&s.pos, npx * 12);
    alloc(&s.nrm, npx * 12);
    if (d.has_roughness) alloc(&s.rough, npx * 4);
    if (d.has_mask) alloc(&s.mask, npx);
    if (d.outputs & 1) alloc(&s.D, npx * 16);
    if (d.outputs & 2) alloc(&s.S, npx * 16);
    if (d.outputs & 4) alloc(&s.V, npx * 4);
    alloc(&s.ws, 256);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking);
  cudaEvent_t *evs[] = {&p->start,        &p->in_free[0],   &p->in_free[1], &p->in_ready[0],
                        &p->in_ready[1], &p->out_ready[0], &p->out_ready[1], &p->out_free[0],
                        &p->out_free[1]};
  for (cudaEvent_t *ev : evs)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    release(p);
    return vct::set_last_error(VCT_ERR_CUDA, "vct_pipeline_create: %s", cudaGetErrorString(e));
  }
  *out = p;
  return VCT_OK;
}

vct_status vct_pipeline_submit(vct_pipeline *p, const vct_host_frame *f, vct_stream_t after) {
  if (!p || !f) return vct::set_last_error(VCT_ERR_INVALID_ARG, "vct_pipeline_submit: NULL");
  const vct_pipeline_desc &d = p->desc;
  if (!f->level0 || !f->position || !f->normal || (d.has_roughness && !f->roughness) ||
      (d.has_mask && !f->mask) || ((d.outputs & 1) && !f->out_diffuse) ||
      ((d.outputs & 2) && !f->out_specular) || ((d.outputs & 4) && !f->out_visibility))
    return vct::set_last_error(VCT_ERR_INVALID_ARG, "vct_pipeline_submit: missing buffer");
  const int s = (int)(p->frames & 1u);
  auto &sl = p->slot[s];
  const size_t npx = px_count(d);
  const size_t n3 = (size_t)d.n * d.n * d.n;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  // inputs: after the caller's work and once the slot's previous trace is done
  chk(cudaEventRecord(p->start, (cudaStream_t)after));
  chk(cudaStreamWaitEvent(p->h2d, p->start, 0));
  chk(cudaStreamWaitEvent(p->h2d, p->in_free[s], 0));
  chk(cudaMemcpyAsync(sl.level0, f->level0, n3 * 16, cudaMemcpyHostToDevice, p->h2d));
  chk(cudaMemcpyAsync(sl.pos, f->position, npx * 12, cudaMemcpyHostToDevice, p->h2d));
  chk(cudaMemcpyAsync(sl.nrm, f->normal, npx * 12, cudaMemcpyHostToDevice, p->h2d));
  if (d.has_roughness)
    chk(cudaMemcpyAsync(sl.rough, f->roughness, npx * 4, cudaMemcpyHostToDevice, p->h2d));
  if (d.has_mask) chk(cudaMemcpyAsync(sl.mask, f->mask, npx, cudaMemcpyHostToDevice, p->h2d));
  chk(cudaEventRecord(p->in_ready[s], p->h2d));
  if (e != cudaSuccess)
    return vct::set_last_error(VCT_ERR_CUDA, "vct_pipeline_submit copy-in: %s",
                               cudaGetErrorString(e));
  // kernels: once the inputs are in and the slot's previous outputs are out
  chk(cudaStreamWaitEvent(p->comp, p->in_ready[s], 0));
  chk(cudaStreamWaitEvent(p->comp, p->out_free[s], 0));
  if (e != cudaSuccess)
    return vct::set_last_error(VCT_ERR_CUDA, "vct_pipeline_submit: %s", cudaGetErrorString(e));
  const vct_pyramid pyr = slot_pyramid(p, s);
  vct_status st = vct_build_mips(sl.level0, &pyr, p->comp);
  if (st != VCT_OK) return st;
  vct_view v{};
  v.width = d.width;
  v.height = d.height;
  v.position = sl.pos;
  v.normal = sl.nrm;
  v.roughness = d.has_roughness ? sl.rough : nullptr;
  v.mask = d.has_mask ? sl.mask : nullptr;
  for (int a = 0; a < 3; ++a) v.camera[a] = f->camera[a];
  v.out_diffuse = sl.D;
  v.out_specular = sl.S;
  v.out_visibility = sl.V;
  st = vct_trace(&pyr, 1, &v, 1, &p->params, nullptr, sl.ws, 256, p->comp);
  if (st != VCT_OK) return st;
  chk(cudaEventRecord(p->in_free[s], p->comp));
  chk(cudaEventRecord(p->out_ready[s], p->comp));
  // outputs back
  chk(cudaStreamWaitEvent(p->d2h, p->out_ready[s], 0));
  if (d.outputs & 1)
    chk(cudaMemcpyAsync(f->out_diffuse, sl.D, npx * 16, cudaMemcpyDeviceToHost, p->d2h));
  if (d.outputs & 2)
    chk(cudaMemcpyAsync(f->out_specular, sl.S, npx * 16, cudaMemcpyDeviceToHost, p->d2h));
  if (d.outputs & 4)
    chk(cudaMemcpyAsync(f->out_visibility, sl.V, npx * 4, cudaMemcpyDeviceToHost, p->d2h));
  chk(cudaEventRecord(p->out_free[s], p->d2h));
  if (e != cudaSuccess)
    return vct::set_last_error(VCT_ERR_CUDA, "vct_pipeline_submit copy-out: %s",
                               cudaGetErrorString(e));
  ++p->frames;
  return VCT_OK;
}

vct_status vct_pipeline_join(vct_pipeline *p, vct_stream_t stream) {
  if (!p) return vct::set_last_error(VCT_ERR_INVALID_ARG, "vct_pipeline_join: NULL");
  for (int s = 0; s < 2; ++s) {
    cudaError_t e = cudaStreamWaitEvent((cudaStream_t)stream, p->out_free[s], 0);
    if (e != cudaSuccess)
      return vct::set_last_error(VCT_ERR_CUDA, "vct_pipeline_join: %s", cudaGetErrorString(e));
  }
  return VCT_OK;
}

vct_status vct_pipeline_stats(vct_pipeline *p, int32_t slot, vct_trace_stats *out) {
  if (!p || !out || slot < 0 || slot > 1)
    return vct::set_last_error(VCT_ERR_INVALID_ARG, "vct_pipeline_stats: bad argument");
  cudaError_t e = cudaEventSynchronize(p->out_ready[slot]);
  if (e == cudaSuccess)
    e = cudaMemcpy(out, p->slot[slot].ws, sizeof(vct_trace_stats), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess)
    return vct::set_last_error(VCT_ERR_CUDA, "vct_pipeline_stats: %s", cudaGetErrorString(e));
  return VCT_OK;
}

void vct_pipeline_destroy(vct_pipeline *p) {
  if (p) release(p);
}

}  // extern "C"
