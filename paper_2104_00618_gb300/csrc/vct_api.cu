// C ABI of libvct: argument validation, pyramid layout, launch assembly and
// the launch-shape tuner.  Every entry point returns a vct_status and records
// a thread-local message on failure; nothing aborts or throws across the ABI.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gbuffer.cuh"
#include "voxelize.cuh"

using namespace vct;

namespace {

thread_local std::string g_last_error;

vct_status fail(vct_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

vct_status cuda_fail(cudaError_t e, const char *what) {
  return fail(VCT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
bool finite(float v) { return std::isfinite(v); }
bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool shape_ok(int n, int levels, int dtype) {
  return is_pow2(n) && n >= 2 && n <= 1024 && levels >= 1 && levels <= ilog2(n) + 1 &&
         (dtype == VCT_F32 || dtype == VCT_F16);
}

vct_status check_pyramid(const vct_pyramid *p, const char *what) {
  if (!p) return fail(VCT_ERR_INVALID_ARG, "%s: NULL pyramid", what);
  if (!shape_ok(p->n, p->levels, p->dtype) ||
      (p->layout != VCT_LAYOUT_DENSE && p->layout != VCT_LAYOUT_BRICKS &&
       p->layout != VCT_LAYOUT_ANISO))
    return fail(VCT_ERR_INVALID_ARG, "%s: bad pyramid shape n=%d levels=%d dtype=%d", what, p->n,
                p->levels, p->dtype);
  if (p->layout == VCT_LAYOUT_ANISO && p->dtype != VCT_F32)
    return fail(VCT_ERR_UNSUPPORTED, "%s: anisotropic pyramids are VCT_F32 only", what);
  if (!(p->size > 0.0f) || !finite(p->size) || !finite(p->origin[0]) || !finite(p->origin[1]) ||
      !finite(p->origin[2]))
    return fail(VCT_ERR_INVALID_ARG, "%s: bad pyramid origin/size", what);
  if (!p->data || !aligned(p->data, 256))
    return fail(VCT_ERR_INVALID_ARG, "%s: pyramid data NULL or not 256-byte aligned", what);
  const Layout L = make_layout(p->n, p->levels, p->dtype, p->layout);
  if (p->bytes < L.total)
    return fail(VCT_ERR_INVALID_ARG, "%s: pyramid bytes %llu < required %llu", what,
                (unsigned long long)p->bytes, (unsigned long long)L.total);
  return VCT_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Layout of the float32 gradient pyramid of the adjoint: dense for dense and
// brick pyramids, anisotropic (six volumes per level >= 1) for anisotropic ones.
int grad_layout(const vct_pyramid &p) {
  return p.layout == VCT_LAYOUT_ANISO ? VCT_LAYOUT_ANISO : VCT_LAYOUT_DENSE;
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// ---------------------------------------------------------------------------
// trace parameters
// ---------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846;

bool aperture_ok(float g) { return finite(g) && g > 0.0f && g < (float)kPi; }

constexpr int kFlagsAll = VCT_FLAG_OCC_SMOOTH | VCT_FLAG_SPEC_GRACE | VCT_FLAG_DIFFUSE_FIRST_HIT |
                          VCT_FLAG_SHADE | VCT_FLAG_SHADE_IMPL | VCT_FLAG_PREMULTIPLIED;

// `backward`: checked for the adjoint, which covers every cone variant; the
// shading flags only add the radiance output, which the adjoint leaves out.
vct_status check_params(const vct_trace_params *P, bool backward) {
  (void)backward;
  if (!P) return fail(VCT_ERR_INVALID_ARG, "params: NULL");
  if (P->n_diffuse < 0 || P->n_diffuse > VCT_MAX_DIFFUSE)
    return fail(VCT_ERR_INVALID_ARG, "params: n_diffuse %d out of [0, %d]", P->n_diffuse,
                VCT_MAX_DIFFUSE);
  if ((P->spec_enable != 0 && P->spec_enable != 1) || (P->occ_enable != 0 && P->occ_enable != 1))
    return fail(VCT_ERR_INVALID_ARG, "params: spec_enable/occ_enable must be 0 or 1");
  if (P->flags & ~kFlagsAll) return fail(VCT_ERR_INVALID_ARG, "params: unknown flags 0x%x", P->flags);
  if ((P->flags & VCT_FLAG_SHADE_IMPL) && !(P->flags & VCT_FLAG_SHADE))
    return fail(VCT_ERR_INVALID_ARG, "params: VCT_FLAG_SHADE_IMPL needs VCT_FLAG_SHADE");
  if ((P->flags & VCT_FLAG_OCC_SMOOTH) &&
      (!finite(P->shadow_str) || !(P->occ_max_dist > 0.0f) || !finite(P->occ_max_dist)))
    return fail(VCT_ERR_INVALID_ARG, "params: shadow_str must be finite and occ_max_dist > 0");
  if ((P->flags & (VCT_FLAG_SPEC_GRACE | VCT_FLAG_SHADE)) &&
      (!finite(P->shininess) || P->shininess < 0.0f))
    return fail(VCT_ERR_INVALID_ARG, "params: shininess must be finite and >= 0");
  if ((P->flags & VCT_FLAG_SPEC_GRACE) &&
      (!finite(P->shininess_falloff) || P->shininess_falloff < 0.0f))
    return fail(VCT_ERR_INVALID_ARG, "params: shininess_falloff must be finite and >= 0");
  if ((P->flags & VCT_FLAG_SHADE) &&
      (!finite(P->diffuse_str) || !finite(P->specular_str) || !finite(P->light_color[0]) ||
       !finite(P->light_color[1]) || !finite(P->light_color[2])))
    return fail(VCT_ERR_INVALID_ARG, "params: shading strengths and light_color must be finite");
  if (P->flags & (VCT_FLAG_SPEC_GRACE | VCT_FLAG_SHADE)) {
    const float l2 = P->light_dir[0] * P->light_dir[0] + P->light_dir[1] * P->light_dir[1] +
                     P->light_dir[2] * P->light_dir[2];
    if (!finite(l2) || !(l2 > 0.0f))
      return fail(VCT_ERR_INVALID_ARG, "params: light_dir must be finite and non-zero");
  }
  if (P->n_diffuse > 0 && !aperture_ok(P->diffuse_aperture))
    return fail(VCT_ERR_INVALID_ARG, "params: diffuse_aperture must be in (0, pi)");
  for (int k = 0; k < P->n_diffuse; ++k)
    if (!finite(P->diffuse_dir[k][0]) || !finite(P->diffuse_dir[k][1]) ||
        !finite(P->diffuse_dir[k][2]) || !finite(P->diffuse_weight[k]))
      return fail(VCT_ERR_INVALID_ARG, "params: diffuse cone %d not finite", k);
  if (P->spec_enable) {
    if (!aperture_ok(P->spec_aperture_min) || !aperture_ok(P->spec_aperture_max))
      return fail(VCT_ERR_INVALID_ARG, "params: specular apertures must be in (0, pi)");
    if (!finite(P->roughness_min) || P->roughness_min >= 1.0f)
      return fail(VCT_ERR_INVALID_ARG, "params: roughness_min must be < 1");
  }
  if (P->occ_enable) {
    if (!aperture_ok(P->occ_aperture))
      return fail(VCT_ERR_INVALID_ARG, "params: occ_aperture must be in (0, pi)");
    if (!finite(P->light_dir[0]) || !finite(P->light_dir[1]) || !finite(P->light_dir[2]))
      return fail(VCT_ERR_INVALID_ARG, "params: light_dir not finite");
  }
  if (!(P->beta > 0.0f) || !finite(P->beta) || !(P->t0_voxels > 0.0f) || !finite(P->t0_voxels) ||
      !(P->t_max > 0.0f) || !finite(P->t_max) || !finite(P->normal_offset_voxels))
    return fail(VCT_ERR_INVALID_ARG, "params: beta, t0_voxels, t_max must be > 0 and finite");
  // with t_max <= 2^20 voxels (checked per pyramid), sample positions stay
  // within 2^21 voxels of the apex's voxel
  if (!(fabsf(P->normal_offset_voxels) <= 524288.0f))
    return fail(VCT_ERR_INVALID_ARG, "params: |normal_offset_voxels| must be <= 2^19");
  return VCT_OK;
}

vct_status fill_pyr(const vct_pyramid &p, const vct_trace_params &P, DevPyr &d) {
  const Layout L = make_layout(p.n, p.levels, p.dtype, p.layout);
  memset(&d, 0, sizeof(d));
  for (int l = 0; l < p.levels; ++l)
    d.lvl[l] = static_cast<const uint8_t *>(p.data) + L.level_off[l];
  d.pool = static_cast<const uint8_t *>(p.data) + L.pool_off;
  d.bricked = L.bricked;
  if (L.bricked && p.bytes > L.pool_off)
    d.pool_slots = (uint32_t)std::min<uint64_t>(
        (p.bytes - L.pool_off) / ((uint64_t)texel_bytes(p.dtype) << kBrickShift), 0xffffffffull);
  for (int a = 0; a < 3; ++a) d.origin_f[a] = p.origin[a];
  const double scale = (double)p.n / (double)p.size;  // scene units -> level-0 voxels
  d.scale_hi = (float)scale;
  d.scale_lo = (float)(scale - (double)d.scale_hi);
  const double tmax_vox = (double)P.t_max * scale;
  // sample coordinates relative to the apex stay below 2^21 voxels
  if (tmax_vox > 1048576.0)
    return fail(VCT_ERR_INVALID_ARG, "params: t_max spans more than 2^20 voxels");
  d.log2_tmax_t0 = (float)log2(tmax_vox / (double)P.t0_voxels);
  d.n = p.n;
  d.levels = p.levels;
  d.dtype = p.dtype;
  d.h0 = (float)((double)p.size / (double)p.n);
  const double beta = P.beta, t0 = P.t0_voxels;
  auto mk = [&](float g, ConeConst &c, const char *name) -> vct_status {
    c = cone_const((double)g, beta, t0, tmax_vox);
    if (c.kmax > kMaxSteps)
      return fail(VCT_ERR_INVALID_ARG, "params: %s cone needs more than %d steps", name,
                  kMaxSteps);
    return VCT_OK;
  };
  vct_status st = VCT_OK;
  if (P.n_diffuse > 0 && (st = mk(P.diffuse_aperture, d.diffuse, "diffuse")) != VCT_OK) return st;
  if (P.occ_enable && (st = mk(P.occ_aperture, d.occ, "occlusion")) != VCT_OK) return st;
  if (P.spec_enable) {
    if ((st = mk(P.spec_aperture_min, d.spec_fixed, "specular")) != VCT_OK) return st;
    ConeConst tmp;
    if ((st = mk(P.spec_aperture_max, tmp, "specular")) != VCT_OK) return st;
  }
  return VCT_OK;
}

template <typename LaunchT>
void fill_common(const vct_trace_params &P, LaunchT &L) {
  L.n_diffuse = P.n_diffuse;
  L.spec_enable = P.spec_enable;
  L.occ_enable = P.occ_enable;
  for (int k = 0; k < VCT_MAX_DIFFUSE; ++k) {
    for (int a = 0; a < 3; ++a) L.diffuse_dir[k][a] = k < P.n_diffuse ? P.diffuse_dir[k][a] : 0.f;
    L.diffuse_weight[k] = k < P.n_diffuse ? P.diffuse_weight[k] : 0.f;
  }
  for (int a = 0; a < 3; ++a) L.light[a] = P.light_dir[a];
  L.normal_offset = P.normal_offset_voxels;
  L.spec.gmin = P.spec_aperture_min;
  L.spec.gdelta = P.spec_aperture_max - P.spec_aperture_min;
  L.spec.rough_min = P.roughness_min;
  L.spec.inv_rough_span = (float)(1.0 / (1.0 - (double)P.roughness_min));
  L.spec.two_beta = 2.0f * P.beta;
  L.spec.t0_vox = P.t0_voxels;
}

void fill_variants(const vct_trace_params &P, Variants &v) {
  v.flags = P.flags;
  v.shadow_str = P.shadow_str;
  v.occ_max_dist = P.occ_max_dist;
  v.grace = (float)(0.008 * kPi * (double)P.shininess);
  v.falloff = P.shininess_falloff;
  v.shininess = P.shininess;
  v.kd = P.diffuse_str;
  v.ks = P.specular_str;
  for (int a = 0; a < 3; ++a) {
    v.light_color[a] = P.light_color[a];
    v.light_dir[a] = P.light_dir[a];
  }
}

// `flags`: the VCT_FLAG_* bits of the call (forward), or -1 for the adjoint
// (which reads no albedo and writes no radiance).
vct_status check_view(const vct_view &v, int i, int n_pyr, int flags) {
  const bool need_outputs = flags >= 0;
  if (v.width < 1 || v.height < 1 || v.width > 65535 || v.height > 65535 ||
      (int64_t)v.width * v.height > (int64_t)1 << 29)
    return fail(VCT_ERR_INVALID_ARG, "view %d: bad size %dx%d", i, v.width, v.height);
  if (v.pyramid < 0 || v.pyramid >= n_pyr || v.reserved != 0)
    return fail(VCT_ERR_INVALID_ARG, "view %d: pyramid index %d out of range", i, v.pyramid);
  if (!v.position || !v.normal || !aligned(v.position, 4) || !aligned(v.normal, 4))
    return fail(VCT_ERR_INVALID_ARG, "view %d: position/normal NULL or misaligned", i);
  if (v.roughness && !aligned(v.roughness, 4))
    return fail(VCT_ERR_INVALID_ARG, "view %d: roughness misaligned", i);
  if ((v.out_diffuse && !aligned(v.out_diffuse, 16)) ||
      (v.out_specular && !aligned(v.out_specular, 16)) ||
      (v.out_visibility && !aligned(v.out_visibility, 4)))
    return fail(VCT_ERR_INVALID_ARG, "view %d: outputs must be 16-byte aligned", i);
  if ((v.albedo && !aligned(v.albedo, 4)) || (v.out_radiance && !aligned(v.out_radiance, 16)) ||
      (v.cone_state && !aligned(v.cone_state, 8)))
    return fail(VCT_ERR_INVALID_ARG, "view %d: albedo/out_radiance/cone_state misaligned", i);
  if (need_outputs && v.out_radiance && !(flags & VCT_FLAG_SHADE))
    return fail(VCT_ERR_INVALID_ARG, "view %d: out_radiance needs VCT_FLAG_SHADE", i);
  if (need_outputs && !v.out_diffuse && !v.out_specular && !v.out_visibility && !v.out_radiance)
    return fail(VCT_ERR_INVALID_ARG, "view %d: no output buffer", i);
  if (!finite(v.camera[0]) || !finite(v.camera[1]) || !finite(v.camera[2]))
    return fail(VCT_ERR_INVALID_ARG, "view %d: camera not finite", i);
  return VCT_OK;
}

void fill_view(const vct_view &v, int tile_w, int tile_h, int &tile_cursor, DevView &d) {
  d.pos = v.position;
  d.nrm = v.normal;
  d.rough = v.roughness;
  d.mask = v.mask;
  d.outD = v.out_diffuse;
  d.outS = v.out_specular;
  d.outV = v.out_visibility;
  d.albedo = v.albedo;
  d.outL = v.out_radiance;
  d.state = static_cast<uint2 *>(v.cone_state);
  for (int a = 0; a < 3; ++a) d.cam[a] = v.camera[a];
  d.W = (uint16_t)v.width;
  d.H = (uint16_t)v.height;
  d.pyr = (uint16_t)v.pyramid;
  d.tiles_x = (uint16_t)((v.width + tile_w - 1) / tile_w);
  d.tile_begin = tile_cursor;
  tile_cursor += d.tiles_x * ((v.height + tile_h - 1) / tile_h);
  d.y_split = (uint16_t)v.height;
  d.small_tiles_x = (uint16_t)((v.width + kSmallTileW - 1) / kSmallTileW);
  d.small_begin = 0;
}

// Splits the work of a launch into big tiles followed by small tail tiles:
// the bottom big-tile rows of the last views, about `tail_px` pixels, are
// re-tiled with kSmallTileW x kSmallTileH tiles.  Returns the item count;
// big items come first (view by view), then the small ones.
int assign_tail_tiles(DevView *v, int nv, int tile_w, int tile_h, int64_t tail_px, int &n_big) {
  for (int i = nv - 1; i >= 0 && tail_px > 0; --i) {
    const int rows = (v[i].H + tile_h - 1) / tile_h;
    const int64_t row_px = (int64_t)tile_h * v[i].W;
    int take = (int)std::min<int64_t>(rows, (tail_px + row_px - 1) / row_px);
    v[i].y_split = (uint16_t)((rows - take) * tile_h);
    tail_px -= (int64_t)take * row_px;
  }
  int cursor = 0;
  for (int i = 0; i < nv; ++i) {
    v[i].tile_begin = cursor;
    // a view outside the tail keeps all its big-tile rows, the last one
    // partial when tile_h does not divide its height
    const int big_rows = v[i].y_split >= v[i].H ? (v[i].H + tile_h - 1) / tile_h
                                                 : v[i].y_split / tile_h;
    cursor += v[i].tiles_x * big_rows;
  }
  n_big = cursor;
  for (int i = 0; i < nv; ++i) {
    v[i].small_begin = cursor;
    if (v[i].y_split < v[i].H)
      cursor += v[i].small_tiles_x * ((v[i].H - v[i].y_split + kSmallTileH - 1) / kSmallTileH);
  }
  return cursor;
}

bool cfg_ok(const vct_launch_config &c) {
  const int lpp = c.lanes_per_pixel;
  return c.tile_w >= 1 && c.tile_h >= 1 && c.tile_w * c.tile_h <= kMaxSortPixels &&
         (lpp == 1 || lpp == 2 || lpp == 4 || lpp == 8) && c.ctas_per_sm >= 0 &&
         c.ctas_per_sm <= 32;
}

// Launch-shape cache filled by vct_autotune_trace.
using TuneKey = std::tuple<int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, vct_launch_config> g_tuned;

TuneKey tune_key(const vct_pyramid *pyrs, const vct_view *views, const vct_trace_params *P) {
  int dev = 0;
  cudaGetDevice(&dev);
  return TuneKey(dev, pyrs[0].dtype, pyrs[0].n, P->spec_enable, P->occ_enable,
                 views[0].roughness != nullptr, P->flags);
}

vct_launch_config default_cfg() { return vct_launch_config{16, 16, 1, 0}; }

vct_launch_config pick_cfg(const vct_launch_config *cfg, const vct_pyramid *pyrs,
                           const vct_view *views, const vct_trace_params *P) {
  if (cfg) return *cfg;
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tuned.find(tune_key(pyrs, views, P));
  return it == g_tuned.end() ? default_cfg() : it->second;
}

struct TraceStatsLayout {
  static constexpr size_t queue_off = offsetof(vct_trace_stats, queue);
};

}  // namespace

namespace vct {
vct_status set_last_error(vct_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}
}  // namespace vct

namespace vct {
namespace {
// Writes index i to buf[i] for i < declared + extra through the bounds check
// against `declared`: the last `extra` writes are caught and skipped (the
// caller's buffer holds declared + extra words, so even an unchecked write
// would stay inside it).
__global__ void bounds_probe_kernel(uint32_t *buf, uint32_t declared, uint32_t extra) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < declared + extra;
       i += gridDim.x * blockDim.x)
    if (in_bounds(i, declared, kOobProbe)) buf[i] = i;
}
}  // namespace

cudaError_t launch_bounds_probe(uint32_t *buf, uint32_t declared, uint32_t extra,
                                cudaStream_t s) {
  const uint32_t total = declared + extra;
  const int grid = (int)std::min<uint32_t>((total + 255) / 256, 1024u);
  bounds_probe_kernel<<<grid, 256, 0, s>>>(buf, declared, extra);
  return cudaGetLastError();
}

VCT_OOB_ACCESSOR(oob_flags_api)
}  // namespace vct

extern "C" {

const char *vct_status_string(vct_status s) {
  switch (s) {
    case VCT_OK: return "VCT_OK";
    case VCT_ERR_INVALID_ARG: return "VCT_ERR_INVALID_ARG";
    case VCT_ERR_CUDA: return "VCT_ERR_CUDA";
    case VCT_ERR_WORKSPACE: return "VCT_ERR_WORKSPACE";
    case VCT_ERR_UNSUPPORTED: return "VCT_ERR_UNSUPPORTED";
    case VCT_ERR_TIMEOUT: return "VCT_ERR_TIMEOUT";
  }
  return "VCT_ERR_UNKNOWN";
}

const char *vct_last_error(void) { return g_last_error.c_str(); }

int32_t vct_version(void) { return 1; }

size_t vct_pyramid_bytes(int32_t n, int32_t levels, int32_t dtype) {
  if (!shape_ok(n, levels, dtype)) return 0;
  return (size_t)make_layout(n, levels, dtype).total;
}

size_t vct_pyramid_bytes_aniso(int32_t n, int32_t levels, int32_t dtype) {
  if (!shape_ok(n, levels, dtype) || dtype != VCT_F32) return 0;
  return (size_t)make_layout(n, levels, dtype, VCT_LAYOUT_ANISO).total;
}

uint64_t vct_pyramid_level_offset(int32_t n, int32_t levels, int32_t dtype, int32_t level) {
  if (!shape_ok(n, levels, dtype) || level < 0 || level >= levels) return 0;
  return make_layout(n, levels, dtype).level_off[level];
}

vct_status vct_build_mips(const float *level0_dense, const vct_pyramid *pyr, vct_stream_t stream) {
  vct_status st = check_pyramid(pyr, "vct_build_mips");
  if (st != VCT_OK) return st;
  if (!level0_dense || !aligned(level0_dense, 16))
    return fail(VCT_ERR_INVALID_ARG, "vct_build_mips: level0 NULL or not 16-byte aligned");
  if (pyr->layout == VCT_LAYOUT_ANISO) {
    cudaError_t e = launch_build_aniso(level0_dense, *pyr, sm_count(), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "vct_build_mips (anisotropic) launch");
    return VCT_OK;
  }
  if (streamed_build(level0_dense, *pyr)) {  // no tensor map to encode
    cudaError_t e = launch_pack_mips(level0_dense, *pyr, nullptr, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "vct_build_mips launch");
    return VCT_OK;
  }
  auto enc = encode_fn();
  if (!enc) return fail(VCT_ERR_CUDA, "vct_build_mips: cuTensorMapEncodeTiled unavailable");
  const int n = pyr->n, B = pack_block(n);
  alignas(64) CUtensorMap map;
  cuuint64_t dims[4] = {4, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[3] = {16, 16ull * n, 16ull * n * n};
  cuuint32_t box[4] = {4, (cuuint32_t)B, (cuuint32_t)B, (cuuint32_t)B};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(level0_dense),
                   dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(VCT_ERR_CUDA, "vct_build_mips: tensor map encode failed (%d)", (int)r);
  cudaError_t e = launch_pack_mips(level0_dense, *pyr, &map, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "vct_build_mips launch");
  return VCT_OK;
}

vct_status vct_pyramid_read_level(const vct_pyramid *pyr, int32_t level, float *dense_out,
                                  vct_stream_t stream) {
  vct_status st = check_pyramid(pyr, "vct_pyramid_read_level");
  if (st != VCT_OK) return st;
  if (level < 0 || level >= pyr->levels)
    return fail(VCT_ERR_INVALID_ARG, "vct_pyramid_read_level: level %d out of range", level);
  if (!dense_out || !aligned(dense_out, 16))
    return fail(VCT_ERR_INVALID_ARG, "vct_pyramid_read_level: output NULL or misaligned");
  cudaError_t e = launch_read_level(*pyr, level, dense_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "vct_pyramid_read_level launch");
  return VCT_OK;
}

vct_status vct_pyramid_read_volume(const vct_pyramid *pyr, int32_t level, int32_t direction,
                                   float *dense_out, vct_stream_t stream) {
  vct_status st = check_pyramid(pyr, "vct_pyramid_read_volume");
  if (st != VCT_OK) return st;
  if (level < 0 || level >= pyr->levels)
    return fail(VCT_ERR_INVALID_ARG, "vct_pyramid_read_volume: level %d out of range", level);
  const int dirs = (pyr->layout == VCT_LAYOUT_ANISO && level >= 1) ? 6 : 1;
  if (direction < 0 || direction >= dirs)
    return fail(VCT_ERR_INVALID_ARG, "vct_pyramid_read_volume: direction %d out of range",
                direction);
  if (!dense_out || !aligned(dense_out, 16))
    return fail(VCT_ERR_INVALID_ARG, "vct_pyramid_read_volume: output NULL or misaligned");
  cudaError_t e = launch_read_level(*pyr, level, dense_out, (cudaStream_t)stream, direction);
  if (e != cudaSuccess) return cuda_fail(e, "vct_pyramid_read_volume launch");
  return VCT_OK;
}

vct_status vct_pyramid_status(const vct_pyramid *pyr, vct_stream_t stream) {
  vct_status st = check_pyramid(pyr, "vct_pyramid_status");
  if (st != VCT_OK) return st;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "vct_pyramid_status sync");
  uint32_t word = 0, zero = 0;
  e = cudaMemcpy(&word, pyr->data, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(pyr->data, &zero, 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "vct_pyramid_status copy");
  if (word == (uint32_t)VCT_ERR_TIMEOUT)
    return fail(VCT_ERR_TIMEOUT, "a kernel gave up a bounded wait while building this pyramid");
  if (word == (uint32_t)VCT_ERR_WORKSPACE)
    return fail(VCT_ERR_WORKSPACE,
                "the brick pool of this pyramid was too small for its occupied bricks");
  return VCT_OK;
}

size_t vct_pyramid_bytes_bricks(int32_t n, int32_t levels, int32_t dtype, uint64_t occupied) {
  if (!shape_ok(n, levels, dtype)) return 0;
  const Layout L = make_layout(n, levels, dtype, VCT_LAYOUT_BRICKS);
  return (size_t)(L.total + occupied * ((uint64_t)texel_bytes(dtype) << kBrickShift));
}

size_t vct_pyramid_plan_scratch_bytes(int32_t n, int32_t levels, int32_t dtype) {
  if (!shape_ok(n, levels, dtype)) return 0;
  return (size_t)make_layout(n, levels, dtype, VCT_LAYOUT_BRICKS).pool_off;
}

vct_status vct_pyramid_plan_bricks(const float *level0_dense, int32_t n, int32_t levels,
                                   int32_t dtype, void *scratch, size_t scratch_bytes,
                                   uint64_t *occupied_out, uint64_t *bytes_out,
                                   vct_stream_t stream) {
  if (!shape_ok(n, levels, dtype))
    return fail(VCT_ERR_INVALID_ARG, "vct_pyramid_plan_bricks: bad shape n=%d levels=%d", n,
                levels);
  if (!level0_dense || !aligned(level0_dense, 16))
    return fail(VCT_ERR_INVALID_ARG, "vct_pyramid_plan_bricks: level0 NULL or misaligned");
  const Layout L = make_layout(n, levels, dtype, VCT_LAYOUT_BRICKS);
  if (!scratch || scratch_bytes < L.pool_off || !aligned(scratch, 256))
    return fail(VCT_ERR_WORKSPACE, "vct_pyramid_plan_bricks: scratch needs %llu bytes",
                (unsigned long long)L.pool_off);
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t *base = static_cast<uint8_t *>(scratch);
  cudaError_t e = launch_brick_tables(level0_dense, n, levels, L, base, ~0ull, s);
  if (e != cudaSuccess) return cuda_fail(e, "vct_pyramid_plan_bricks launch");
  uint64_t count = 0;
  if ((e = cudaMemcpyAsync(&count, base + kHeaderCountOff, 8, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "vct_pyramid_plan_bricks copy");
  if (occupied_out) *occupied_out = count;
  if (bytes_out) *bytes_out = vct_pyramid_bytes_bricks(n, levels, dtype, count);
  return VCT_OK;
}

size_t vct_trace_workspace_bytes(void) { return 256; }

static vct_status trace_impl(const vct_pyramid *pyrs, int32_t n_pyr, const vct_view *views,
                             int32_t n_views, const vct_trace_params *params,
                             const vct_launch_config &cfg, void *workspace,
                             size_t workspace_bytes, cudaStream_t stream, bool zero_stats) {
  auto L = std::make_unique<TraceLaunch>();
  memset(L.get(), 0, sizeof(TraceLaunch));
  fill_common(*params, *L);
  fill_variants(*params, L->var);
  for (int i = 0; i < n_pyr; ++i) {
    vct_status st = fill_pyr(pyrs[i], *params, L->pyr[i]);
    if (st != VCT_OK) return st;
  }
  L->n_pyr = n_pyr;
  L->tile_w = cfg.tile_w;
  L->tile_h = cfg.tile_h;
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  L->stats = reinterpret_cast<unsigned long long *>(ws);
  L->queue = reinterpret_cast<unsigned *>(ws + TraceStatsLayout::queue_off);
  cudaError_t e;
  if (zero_stats && (e = cudaMemsetAsync(ws, 0, sizeof(vct_trace_stats), stream)) != cudaSuccess)
    return cuda_fail(e, "vct_trace workspace clear");
  int per_sm = cfg.ctas_per_sm;
  if (per_sm == 0)
    per_sm = std::max(1, trace_occupancy(cfg.lanes_per_pixel, pyrs[0].dtype, params->flags != 0));
  const int sms = sm_count();
  for (int v0 = 0; v0 < n_views; v0 += kMaxViewsPerLaunch) {
    const int nv = std::min(kMaxViewsPerLaunch, n_views - v0);
    int cursor = 0;
    bool mixed = false, bricks = false;
    const bool aniso = pyrs[views[v0].pyramid].layout == VCT_LAYOUT_ANISO;
    for (int i = 0; i < nv; ++i) {
      fill_view(views[v0 + i], cfg.tile_w, cfg.tile_h, cursor, L->views[i]);
      mixed |= pyrs[views[v0 + i].pyramid].dtype != pyrs[views[v0].pyramid].dtype;
      mixed |= (pyrs[views[v0 + i].pyramid].layout == VCT_LAYOUT_ANISO) != aniso;
      bricks |= pyrs[views[v0 + i].pyramid].layout == VCT_LAYOUT_BRICKS;
    }
    if (mixed)
      return fail(VCT_ERR_UNSUPPORTED,
                  "vct_trace: views of one call must use pyramids of one dtype, and all or "
                  "none anisotropic");
    L->n_views = nv;
    const int grid = std::max(1, std::min(cursor, per_sm * sms));
    // about two waves of the launch's warps, in small tiles, at the end
    const int64_t tail_px = (int64_t)2 * grid * (kFwdThreads / 32) * kSmallTileW * kSmallTileH;
    L->total_tiles = assign_tail_tiles(L->views, nv, cfg.tile_w, cfg.tile_h, tail_px, L->n_big);
    if (v0 > 0 && (e = cudaMemsetAsync(L->queue, 0, 4, stream)) != cudaSuccess)
      return cuda_fail(e, "vct_trace queue clear");
    e = launch_trace(*L, cfg.lanes_per_pixel, pyrs[views[v0].pyramid].dtype, bricks, grid,
                     stream, aniso);
    if (e != cudaSuccess) return cuda_fail(e, "vct_trace launch");
  }
  return VCT_OK;
}

static vct_status trace_checks(const vct_pyramid *pyrs, int32_t n_pyr, const vct_view *views,
                               int32_t n_views, const vct_trace_params *params,
                               void *workspace, size_t workspace_bytes) {
  if (!pyrs || n_pyr < 1 || n_pyr > VCT_MAX_PYRAMIDS)
    return fail(VCT_ERR_INVALID_ARG, "vct_trace: need 1..%d pyramids", VCT_MAX_PYRAMIDS);
  for (int i = 0; i < n_pyr; ++i) {
    vct_status st = check_pyramid(pyrs + i, "vct_trace");
    if (st != VCT_OK) return st;
  }
  if (!views || n_views < 1) return fail(VCT_ERR_INVALID_ARG, "vct_trace: no views");
  vct_status st = check_params(params, false);
  if (st != VCT_OK) return st;
  for (int i = 0; i < n_views; ++i)
    if ((st = check_view(views[i], i, n_pyr, params->flags)) != VCT_OK) return st;
  if (!workspace || workspace_bytes < vct_trace_workspace_bytes() || !aligned(workspace, 8))
    return fail(VCT_ERR_WORKSPACE, "vct_trace: workspace needs %zu bytes, 8-byte aligned",
                vct_trace_workspace_bytes());
  return VCT_OK;
}

vct_status vct_trace(const vct_pyramid *pyrs, int32_t n_pyr, const vct_view *views,
                     int32_t n_views, const vct_trace_params *params,
                     const vct_launch_config *cfg, void *workspace, size_t workspace_bytes,
                     vct_stream_t stream) {
  vct_status st = trace_checks(pyrs, n_pyr, views, n_views, params, workspace, workspace_bytes);
  if (st != VCT_OK) return st;
  const vct_launch_config c = pick_cfg(cfg, pyrs, views, params);
  if (!cfg_ok(c)) return fail(VCT_ERR_INVALID_ARG, "vct_trace: bad launch config");
  return trace_impl(pyrs, n_pyr, views, n_views, params, c, workspace, workspace_bytes,
                    (cudaStream_t)stream, true);
}

vct_status vct_autotune_trace(const vct_pyramid *pyrs, int32_t n_pyr, const vct_view *views,
                              int32_t n_views, const vct_trace_params *params, void *workspace,
                              size_t workspace_bytes, vct_stream_t stream,
                              vct_launch_config *best) {
  vct_status st = trace_checks(pyrs, n_pyr, views, n_views, params, workspace, workspace_bytes);
  if (st != VCT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(VCT_ERR_CUDA, "vct_autotune_trace: event create failed");
  const int tiles[4][2] = {{4, 8}, {8, 8}, {8, 16}, {16, 16}};
  const int lpps[4] = {1, 2, 4, 8};
  float best_ms = 1e30f;
  vct_launch_config bc = default_cfg();
  for (auto &t : tiles)
    for (int lpp : lpps) {
      vct_launch_config c{t[0], t[1], lpp, 0};
      float ms_sum = 0.f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, s);
        st = trace_impl(pyrs, n_pyr, views, n_views, params, c, workspace, workspace_bytes, s, true);
        cudaEventRecord(e1, s);
        if (st != VCT_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          st = fail(VCT_ERR_CUDA, "vct_autotune_trace: kernel failed");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) ms_sum += ms;  // first run warms caches
      }
      if (st != VCT_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
      }
      if (ms_sum < best_ms) {
        best_ms = ms_sum;
        bc = c;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tuned[tune_key(pyrs, views, params)] = bc;
  }
  if (best) *best = bc;
  return VCT_OK;
}

size_t vct_trace_backward_workspace_bytes(const vct_pyramid *pyr) {
  if (!pyr || !shape_ok(pyr->n, pyr->levels, pyr->dtype)) return 0;
  return (size_t)make_layout(pyr->n, pyr->levels, VCT_F32, grad_layout(*pyr)).total;
}

}  // extern "C"

namespace {

// Texels of gradient level l: six volumes per anisotropic level >= 1.
uint64_t grad_texels(int n, int l, bool aniso) {
  return vct::level_texels(n, l) * ((aniso && l >= 1) ? 6 : 1);
}

// Fixed-point levels of the deterministic adjoint: 4 x uint64 per texel,
// each level 256-byte aligned, after the float32 gradient pyramid.
uint64_t fix_level_off(const vct::Layout &gl, int n, int l, bool aniso) {
  uint64_t off = vct::align256(gl.total);
  for (int k = 0; k < l; ++k) off += vct::align256(grad_texels(n, k, aniso) * 32);
  return off;
}

vct_status trace_backward_impl(const vct_pyramid *pyr, const vct_view *views,
                               const vct_view_grad *grads, int32_t n_views,
                               const vct_trace_params *params, const vct_launch_config *cfg,
                               float *grad_level0_dense, void *workspace, size_t workspace_bytes,
                               vct_stream_t stream, bool deterministic) {
  using namespace vct;
  vct_status st = check_pyramid(pyr, "vct_trace_backward");
  if (st != VCT_OK) return st;
  const bool aniso = pyr->layout == VCT_LAYOUT_ANISO;
  if (!views || !grads || n_views < 1)
    return fail(VCT_ERR_INVALID_ARG, "vct_trace_backward: no views");
  if ((st = check_params(params, true)) != VCT_OK) return st;
  for (int i = 0; i < n_views; ++i) {
    if ((st = check_view(views[i], i, 1, -1)) != VCT_OK) return st;
    const vct_view_grad &g = grads[i];
    if ((g.grad_diffuse && !aligned(g.grad_diffuse, 16)) ||
        (g.grad_specular && !aligned(g.grad_specular, 16)) ||
        (g.grad_visibility && !aligned(g.grad_visibility, 4)) ||
        (g.grad_radiance && !aligned(g.grad_radiance, 16)))
      return fail(VCT_ERR_INVALID_ARG, "view %d: gradients must be 16-byte aligned", i);
    if (g.grad_radiance && !(params->flags & VCT_FLAG_SHADE))
      return fail(VCT_ERR_INVALID_ARG, "view %d: grad_radiance needs VCT_FLAG_SHADE", i);
    // L_impl = Vis (D + direct) + S: its adjoint reads the forward's D and Vis
    if (g.grad_radiance && (params->flags & VCT_FLAG_SHADE_IMPL) &&
        (!views[i].out_diffuse || (params->occ_enable && !views[i].out_visibility)))
      return fail(VCT_ERR_INVALID_ARG,
                  "view %d: grad_radiance of L_impl needs the forward's out_diffuse and "
                  "out_visibility", i);
  }
  if (!grad_level0_dense || !aligned(grad_level0_dense, 16))
    return fail(VCT_ERR_INVALID_ARG, "vct_trace_backward: grad_level0 NULL or misaligned");
  const Layout gl = make_layout(pyr->n, pyr->levels, VCT_F32, grad_layout(*pyr));
  const uint64_t need = deterministic ? fix_level_off(gl, pyr->n, pyr->levels, aniso) : gl.total;
  if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
    return fail(VCT_ERR_WORKSPACE, "vct_trace_backward: workspace needs %llu bytes, 256-byte aligned",
                (unsigned long long)need);
  vct_launch_config c = cfg ? *cfg : vct_launch_config{8, 8, 1, 0};
  if (!cfg_ok(c)) return fail(VCT_ERR_INVALID_ARG, "vct_trace_backward: bad launch config");

  auto L = std::make_unique<BwdLaunch>();
  memset(L.get(), 0, sizeof(BwdLaunch));
  fill_common(*params, *L);
  fill_variants(*params, L->var);
  if ((st = fill_pyr(*pyr, *params, L->pyr)) != VCT_OK) return st;
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  for (int l = 0; l < pyr->levels; ++l) {
    L->gpyr_lvl[l] = reinterpret_cast<float *>(ws + gl.level_off[l]);
    if (deterministic)
      L->gfix_lvl[l] =
          reinterpret_cast<unsigned long long *>(ws + fix_level_off(gl, pyr->n, l, aniso));
  }
  L->deterministic = deterministic ? 1 : 0;
  L->aniso = aniso ? 1 : 0;
  L->queue = reinterpret_cast<unsigned *>(ws);
  L->tile_w = c.tile_w;
  L->tile_h = c.tile_h;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(ws, 0, need, s);
  if (e != cudaSuccess) return cuda_fail(e, "vct_trace_backward workspace clear");
  int per_sm = c.ctas_per_sm ? c.ctas_per_sm
                             : std::max(1, trace_bwd_occupancy(c.lanes_per_pixel, pyr->dtype,
                                                               L->pyr.bricked != 0));
  const int sms = sm_count();
  for (int v0 = 0; v0 < n_views; v0 += kMaxBwdViewsPerLaunch) {
    const int nv = std::min(kMaxBwdViewsPerLaunch, n_views - v0);
    int cursor = 0;
    for (int i = 0; i < nv; ++i) {
      fill_view(views[v0 + i], c.tile_w, c.tile_h, cursor, L->views[i].v);
      L->views[i].v.pyr = 0;
      L->views[i].gD = grads[v0 + i].grad_diffuse;
      L->views[i].gS = grads[v0 + i].grad_specular;
      L->views[i].gV = grads[v0 + i].grad_visibility;
      L->views[i].gL = grads[v0 + i].grad_radiance;
    }
    L->n_views = nv;
    L->total_tiles = cursor;
    if (v0 > 0 && (e = cudaMemsetAsync(L->queue, 0, 4, s)) != cudaSuccess)
      return cuda_fail(e, "vct_trace_backward queue clear");
    const int grid = std::max(1, std::min(cursor, per_sm * sms));
    e = launch_trace_bwd(*L, c.lanes_per_pixel, grid, s);
    if (e != cudaSuccess) return cuda_fail(e, "vct_trace_backward launch");
  }
  if (deterministic)
    for (int l = 0; l < pyr->levels; ++l) {
      e = launch_fix_to_float(L->gfix_lvl[l], L->gpyr_lvl[l], grad_texels(pyr->n, l, aniso) * 4,
                              s);
      if (e != cudaSuccess) return cuda_fail(e, "vct_trace_backward fixed-point conversion");
    }
  e = aniso ? launch_mip_adjoint_aniso(*pyr, reinterpret_cast<const float *>(ws),
                                       grad_level0_dense, sms, s)
            : launch_mip_adjoint(reinterpret_cast<const float *>(ws), gl, pyr->n, pyr->levels,
                                 grad_level0_dense, s);
  if (e != cudaSuccess) return cuda_fail(e, "vct_trace_backward mip adjoint launch");
  return VCT_OK;
}

}  // namespace

extern "C" {

vct_status vct_trace_backward(const vct_pyramid *pyr, const vct_view *views,
                              const vct_view_grad *grads, int32_t n_views,
                              const vct_trace_params *params, const vct_launch_config *cfg,
                              float *grad_level0_dense, void *workspace, size_t workspace_bytes,
                              vct_stream_t stream) {
  return trace_backward_impl(pyr, views, grads, n_views, params, cfg, grad_level0_dense,
                             workspace, workspace_bytes, stream, false);
}

size_t vct_trace_backward_deterministic_workspace_bytes(const vct_pyramid *pyr) {
  if (!pyr || !shape_ok(pyr->n, pyr->levels, pyr->dtype)) return 0;
  return (size_t)fix_level_off(make_layout(pyr->n, pyr->levels, VCT_F32, grad_layout(*pyr)),
                               pyr->n, pyr->levels, pyr->layout == VCT_LAYOUT_ANISO);
}

vct_status vct_trace_backward_deterministic(const vct_pyramid *pyr, const vct_view *views,
                                            const vct_view_grad *grads, int32_t n_views,
                                            const vct_trace_params *params,
                                            const vct_launch_config *cfg,
                                            float *grad_level0_dense, void *workspace,
                                            size_t workspace_bytes, vct_stream_t stream) {
  return trace_backward_impl(pyr, views, grads, n_views, params, cfg, grad_level0_dense,
                             workspace, workspace_bytes, stream, true);
}

size_t vct_voxelize_workspace_bytes(int32_t n, int32_t n_triangles) {
  if (!is_pow2(n) || n < 2 || n > 1024 || n_triangles < 0 || n_triangles > (1 << 30)) return 0;
  return voxelize_workspace_bytes(n, n_triangles);
}

vct_status vct_voxelize(const vct_mesh *mesh, int32_t n, const float origin[3], float size,
                        const vct_voxel_light *light, float *level0_dense, void *workspace,
                        size_t workspace_bytes, vct_stream_t stream) {
  if (!mesh || !light || !origin) return fail(VCT_ERR_INVALID_ARG, "vct_voxelize: NULL argument");
  if (!is_pow2(n) || n < 2 || n > 1024)
    return fail(VCT_ERR_INVALID_ARG, "vct_voxelize: n=%d must be a power of two in [2, 1024]", n);
  if (!(size > 0.0f) || !finite(size) || !finite(origin[0]) || !finite(origin[1]) ||
      !finite(origin[2]))
    return fail(VCT_ERR_INVALID_ARG, "vct_voxelize: bad origin/size");
  if (mesh->n_vertices < 0 || mesh->n_triangles < 0 || mesh->n_triangles > (1 << 30))
    return fail(VCT_ERR_INVALID_ARG, "vct_voxelize: bad mesh counts (%d vertices, %d triangles)",
                mesh->n_vertices, mesh->n_triangles);
  if (mesh->n_triangles > 0 &&
      (!mesh->indices || !mesh->colors || !aligned(mesh->indices, 4) || !aligned(mesh->colors, 4)))
    return fail(VCT_ERR_INVALID_ARG, "vct_voxelize: indices/colors NULL or misaligned");
  if (mesh->n_vertices > 0 && (!mesh->vertices || !aligned(mesh->vertices, 4)))
    return fail(VCT_ERR_INVALID_ARG, "vct_voxelize: vertices NULL or misaligned");
  for (int a = 0; a < 3; ++a)
    if (!finite(light->light_dir[a]) || !finite(light->light_color[a]))
      return fail(VCT_ERR_INVALID_ARG, "vct_voxelize: light not finite");
  if (!finite(light->ambient) || !finite(light->diffuse_str))
    return fail(VCT_ERR_INVALID_ARG, "vct_voxelize: light strengths not finite");
  if (!level0_dense || !aligned(level0_dense, 16))
    return fail(VCT_ERR_INVALID_ARG, "vct_voxelize: output NULL or not 16-byte aligned");
  const size_t need = voxelize_workspace_bytes(n, mesh->n_triangles);
  if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
    return fail(VCT_ERR_WORKSPACE, "vct_voxelize: workspace needs %zu bytes, 256-byte aligned",
                need);
  cudaError_t e = launch_voxelize(*mesh, n, origin, size, *light, level0_dense, workspace,
                                  sm_count(), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "vct_voxelize launch");
  return VCT_OK;
}

size_t vct_gbuffer_workspace_bytes(int32_t width, int32_t height, int32_t n_triangles,
                                   uint64_t pair_capacity) {
  if (width < 1 || width > 16384 || height < 1 || height > 16384 || n_triangles < 0 ||
      n_triangles > (1 << 30) || pair_capacity > (1ull << 31))
    return 0;
  return gbuffer_fixed_bytes(width, height, n_triangles) + (size_t)align256(pair_capacity * 4);
}

vct_status vct_gbuffer(const vct_mesh *mesh, const vct_camera *camera, float *position,
                       float *normal, float *albedo, uint8_t *mask, int32_t *triangle,
                       void *workspace, size_t workspace_bytes, vct_stream_t stream) {
  if (!mesh || !camera) return fail(VCT_ERR_INVALID_ARG, "vct_gbuffer: NULL argument");
  const vct_camera &c = *camera;
  if (c.width < 1 || c.width > 16384 || c.height < 1 || c.height > 16384)
    return fail(VCT_ERR_INVALID_ARG, "vct_gbuffer: image %dx%d outside 1..16384", c.width,
                c.height);
  if (mesh->n_vertices < 0 || mesh->n_triangles < 0 || mesh->n_triangles > (1 << 30))
    return fail(VCT_ERR_INVALID_ARG, "vct_gbuffer: bad mesh counts (%d vertices, %d triangles)",
                mesh->n_vertices, mesh->n_triangles);
  if (mesh->n_triangles > 0 &&
      (!mesh->indices || !mesh->colors || !aligned(mesh->indices, 4) || !aligned(mesh->colors, 4)))
    return fail(VCT_ERR_INVALID_ARG, "vct_gbuffer: indices/colors NULL or misaligned");
  if (mesh->n_vertices > 0 && (!mesh->vertices || !aligned(mesh->vertices, 4)))
    return fail(VCT_ERR_INVALID_ARG, "vct_gbuffer: vertices NULL or misaligned");
  if (!(c.frame_size > 0.0f) || !finite(c.frame_size) || !(c.tan_half_fov > 0.0f) ||
      !finite(c.tan_half_fov))
    return fail(VCT_ERR_INVALID_ARG, "vct_gbuffer: frame_size and tan_half_fov must be > 0");
  const double lim = 1.0 + 1.0 / 1024.0;
  for (int a = 0; a < 3; ++a) {
    if (!finite(c.eye[a]) || !finite(c.frame_origin[a]))
      return fail(VCT_ERR_INVALID_ARG, "vct_gbuffer: eye/frame_origin not finite");
    if (!(fabs(c.forward[a]) <= lim) || !(fabs(c.right[a]) <= lim) || !(fabs(c.up[a]) <= lim))
      return fail(VCT_ERR_INVALID_ARG,
                  "vct_gbuffer: basis components must have magnitude <= 1 + 2^-10");
  }
  const double det =
      (double)c.right[0] * ((double)c.up[1] * c.forward[2] - (double)c.up[2] * c.forward[1]) -
      (double)c.up[0] * ((double)c.right[1] * c.forward[2] - (double)c.right[2] * c.forward[1]) +
      (double)c.forward[0] * ((double)c.right[1] * c.up[2] - (double)c.right[2] * c.up[1]);
  if (!(fabs(det) >= 0.25))
    return fail(VCT_ERR_INVALID_ARG, "vct_gbuffer: |det(right, up, forward)| = %g < 0.25", det);
  const float tx = (float)((double)c.tan_half_fov * (double)c.width / (double)c.height);
  if (!((double)tx + (double)c.tan_half_fov <= 2.99))
    return fail(VCT_ERR_INVALID_ARG,
                "vct_gbuffer: field of view too wide (tx + tan_half_fov = %g > 2.99)",
                (double)tx + c.tan_half_fov);
  const float s = (float)((double)kFrameUnits / (double)c.frame_size);
  for (int a = 0; a < 3; ++a) {
    long long X;
    if (!frame_snap(c.eye[a], c.frame_origin[a], s, &X))
      return fail(VCT_ERR_INVALID_ARG, "vct_gbuffer: eye outside the fixed-point frame");
  }
  if (!position || !normal || !aligned(position, 4) || !aligned(normal, 4) ||
      (albedo && !aligned(albedo, 4)) || (triangle && !aligned(triangle, 4)))
    return fail(VCT_ERR_INVALID_ARG, "vct_gbuffer: outputs NULL or misaligned");
  const size_t need = gbuffer_fixed_bytes(c.width, c.height, mesh->n_triangles);
  if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
    return fail(VCT_ERR_WORKSPACE, "vct_gbuffer: workspace needs at least %zu bytes, 256-byte "
                "aligned", need);
  cudaError_t e = launch_gbuffer(*mesh, c, position, normal, albedo, mask, triangle, workspace,
                                 workspace_bytes, sm_count(), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "vct_gbuffer launch");
  return VCT_OK;
}

vct_status vct_debug_bounds_flags(uint32_t *flags_out, int32_t reset) {
  if (!flags_out) return fail(VCT_ERR_INVALID_ARG, "vct_debug_bounds_flags: NULL argument");
#ifdef VCT_DEBUG_BOUNDS
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "vct_debug_bounds_flags");
  const bool r = reset != 0;
  *flags_out = oob_flags_api(r) | oob_flags_mips(r) | oob_flags_trace(r) |
               oob_flags_trace_bwd(r) | oob_flags_voxelize(r) | oob_flags_gbuffer(r);
  return VCT_OK;
#else
  (void)reset;
  *flags_out = 0;
  return fail(VCT_ERR_UNSUPPORTED, "vct_debug_bounds_flags: not a debug-bounds build");
#endif
}

vct_status vct_debug_bounds_probe(uint32_t *buf_dev, uint32_t declared, uint32_t extra,
                                  vct_stream_t stream) {
  if (!buf_dev || !aligned(buf_dev, 4) || declared == 0 || extra == 0 || extra > 1024u ||
      declared > (1u << 30))
    return fail(VCT_ERR_INVALID_ARG, "vct_debug_bounds_probe: bad arguments");
#ifdef VCT_DEBUG_BOUNDS
  cudaError_t e = launch_bounds_probe(buf_dev, declared, extra, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "vct_debug_bounds_probe launch");
  return VCT_OK;
#else
  (void)stream;
  return fail(VCT_ERR_UNSUPPORTED, "vct_debug_bounds_probe: not a debug-bounds build");
#endif
}

vct_status vct_debug_wait_probe(uint32_t *flag_dev, uint64_t max_ns, vct_stream_t stream) {
  if (!flag_dev || !aligned(flag_dev, 4))
    return fail(VCT_ERR_INVALID_ARG, "vct_debug_wait_probe: flag NULL or misaligned");
  if (max_ns == 0 || max_ns > 10000000000ull)
    return fail(VCT_ERR_INVALID_ARG, "vct_debug_wait_probe: max_ns must be in (0, 1e10]");
  cudaError_t e = launch_wait_probe(flag_dev, max_ns, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "vct_debug_wait_probe launch");
  return VCT_OK;
}

}  // extern "C"
