// Internal definitions shared by the libvct translation units.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "vct.h"

namespace vct {

constexpr int kHeaderBytes = 256;
constexpr int kTraceThreads = 256;      // CTA shape of the adjoint trace kernel
// Forward trace CTAs: warps work independently, so the CTA size only sets the
// register budget, 65536 / (kFwdThreads * kTraceMinBlocks) per thread.
#ifndef VCT_FWD_THREADS
#define VCT_FWD_THREADS 256
#endif
#ifndef VCT_TRACE_MIN_BLOCKS
#define VCT_TRACE_MIN_BLOCKS 2
#endif
constexpr int kFwdThreads = VCT_FWD_THREADS;
constexpr int kTraceMinBlocks = VCT_TRACE_MIN_BLOCKS;
constexpr int kMaxViewsPerLaunch = 256;  // keeps the forward launch under 32 KB
constexpr int kMaxSortPixels = 256;      // largest pixel tile of one work item
constexpr int kMaxBwdViewsPerLaunch = 128;
constexpr int kMaxSteps = 1 << 16;       // per-cone step cap (parameter check)

// ---------------------------------------------------------------------------
// pyramid layout (host and device)
// ---------------------------------------------------------------------------
__host__ __device__ inline uint64_t align256(uint64_t x) { return (x + 255ull) & ~255ull; }
__host__ __device__ inline int texel_bytes(int dtype) { return dtype == VCT_F16 ? 8 : 16; }
__host__ __device__ inline uint64_t level_texels(int n, int l) {
  uint64_t m = (uint64_t)(n >> l);
  return m * m * m;
}
__host__ __device__ inline int ilog2(int n) {
  int k = 0;
  while ((1 << (k + 1)) <= n) ++k;
  return k;
}
// Edge of the block one CTA of the fused pack/mip kernel handles.
__host__ __device__ inline int pack_block(int n) { return n < 16 ? n : 16; }

// Brick storage (VCT_LAYOUT_BRICKS): levels with at least kBrickMinEdge
// texels per axis are cut into 8^3 bricks (brick id = Morton code >> 9) and
// keep one uint32 pool slot per brick; slot 0 is the shared all-zero brick.
constexpr int kBrickShift = 9;  // 512 texels per brick
constexpr int kBrickMinEdge = 16;
constexpr uint64_t kHeaderCountOff = 8;  // uint64 occupied-brick count in the header

__host__ __device__ inline bool level_bricked(int n, int l, int layout) {
  return layout == VCT_LAYOUT_BRICKS && (n >> l) >= kBrickMinEdge;
}
__host__ __device__ inline uint64_t level_bricks(int n, int l) {
  return level_texels(n, l) >> kBrickShift;
}

struct Layout {
  uint64_t level_off[VCT_MAX_LEVELS];  // bytes from data (slot table of a bricked level)
  uint64_t staging_off[2];             // FP32 staging (VCT_F16, or any brick layout)
  uint64_t pool_off;                   // brick pool (brick layout), else total
  uint64_t total;                      // dense: whole pyramid; bricks: with the zero brick only
  uint32_t bricked;                    // bit l: level l is bricked
};

__host__ __device__ inline Layout make_layout(int n, int levels, int dtype,
                                              int layout = VCT_LAYOUT_DENSE) {
  Layout L{};
  uint64_t off = kHeaderBytes;
  int tb = texel_bytes(dtype);
  for (int l = 0; l < levels; ++l) {
    L.level_off[l] = off;
    if (level_bricked(n, l, layout)) {
      L.bricked |= 1u << l;
      off += align256(level_bricks(n, l) * 4);
    } else if (layout == VCT_LAYOUT_ANISO && l >= 1) {
      off += align256(6 * level_texels(n, l) * tb);  // six directional volumes
    } else {
      off += align256(level_texels(n, l) * tb);
    }
  }
  if (dtype == VCT_F16 || layout == VCT_LAYOUT_BRICKS) {
    int m0 = ilog2(pack_block(n));
    L.staging_off[0] = off;
    off += align256(level_texels(n, m0) * 16);
    L.staging_off[1] = off;
    off += align256(level_texels(n, m0 < ilog2(n) ? m0 + 1 : m0) * 16);
  }
  L.pool_off = off;
  if (layout == VCT_LAYOUT_BRICKS) off += (uint64_t)tb << kBrickShift;  // the zero brick
  L.total = off;
  return L;
}

// ---------------------------------------------------------------------------
// Morton helpers: x in bits 0,3,6..., y in 1,4,7..., z in 2,5,8...
// ---------------------------------------------------------------------------
constexpr uint32_t kMortonX = 0x09249249u;  // bits 0,3,...,27 (10 coordinate bits)

__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint32_t v) {
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030C30C3u;
  v = (v | (v >> 4)) & 0x0300F00Fu;
  v = (v | (v >> 8)) & 0x030000FFu;
  v = (v | (v >> 16)) & 0x000003FFu;
  return v;
}
__host__ __device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// ---------------------------------------------------------------------------
// bounds-checked builds (-DVCT_DEBUG_BOUNDS)
// ---------------------------------------------------------------------------
// A debug-bounds build compares every computed texel, brick-slot, table and
// list index with the length of its array before the access.  A bad index
// sets a bit of its translation unit's flag word (vct_debug_bounds_flags
// reads and clears them) and the access is skipped (a load reads zero); no
// kernel traps.  Release builds compile the checks away.
enum : uint32_t {
  kOobTexel = 1u,    // trace: texel of a dense level
  kOobBrick = 2u,    // trace, mips: slot table or brick pool
  kOobGrad = 4u,     // adjoint: gradient texel
  kOobMip = 8u,      // mips: stored texel
  kOobVoxel = 16u,   // voxelizer: owner word or colour table
  kOobGbuffer = 32u, // G-buffer: tile counters, lists, records
  kOobProbe = 64u,   // vct_debug_bounds_probe
};
#ifdef VCT_DEBUG_BOUNDS
static __device__ uint32_t g_vct_oob;  // one flag word per translation unit
__device__ __forceinline__ bool in_bounds(uint64_t i, uint64_t n, uint32_t what) {
  if (i < n) return true;
  atomicOr(&g_vct_oob, what);
  return false;
}
// Defines the host accessor of this translation unit's flag word.
#define VCT_OOB_ACCESSOR(name)                                              \
  uint32_t name(bool reset) {                                               \
    uint32_t v = 0;                                                         \
    if (cudaMemcpyFromSymbol(&v, g_vct_oob, sizeof(v)) != cudaSuccess) return 0xffffffffu; \
    if (reset) {                                                            \
      const uint32_t z = 0;                                                 \
      cudaMemcpyToSymbol(g_vct_oob, &z, sizeof(z));                         \
    }                                                                       \
    return v;                                                               \
  }
#else
__device__ __forceinline__ bool in_bounds(uint64_t, uint64_t, uint32_t) { return true; }
#define VCT_OOB_ACCESSOR(name) \
  uint32_t name(bool) { return 0u; }
#endif
// Per-translation-unit accessors (debug-bounds builds; 0 otherwise).
uint32_t oob_flags_api(bool reset);
uint32_t oob_flags_mips(bool reset);
uint32_t oob_flags_trace(bool reset);
uint32_t oob_flags_trace_bwd(bool reset);
uint32_t oob_flags_voxelize(bool reset);
uint32_t oob_flags_gbuffer(bool reset);

// ---------------------------------------------------------------------------
// texel load/store
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 ld_texel(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ float4 ld_texel(const uint2 *p) {
  uint2 u = __ldg(p);
  __half2 a = *reinterpret_cast<__half2 *>(&u.x);
  __half2 b = *reinterpret_cast<__half2 *>(&u.y);
  float2 fa = __half22float2(a), fb = __half22float2(b);
  return make_float4(fa.x, fa.y, fb.x, fb.y);
}
__device__ __forceinline__ uint2 pack_half4(float4 v) {
  __half2 a = __floats2half2_rn(v.x, v.y);
  __half2 b = __floats2half2_rn(v.z, v.w);
  uint2 u;
  u.x = *reinterpret_cast<uint32_t *>(&a);
  u.y = *reinterpret_cast<uint32_t *>(&b);
  return u;
}

// ---------------------------------------------------------------------------
// bounded waits (every device-side wait gives up after a time budget)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of `bar` to complete; gives up after max_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t max_ns) {
  uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > max_ns) return false;
  }
  return true;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_4d(void *smem_dst, const CUtensorMap *map,
                                            uint64_t *bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_u32(bar))
      : "memory");
}

constexpr uint64_t kWaitBudgetNs = 2000000000ull;  // 2 s

// ---------------------------------------------------------------------------
// trace launch description (kernel parameter, < 32 KB)
// ---------------------------------------------------------------------------
// Per-cone-kind march constants.  T (t in level-0 voxel units) at step k is
// T0 * 2^(k * l2r) with l2r = log2(1 + 2 beta tan(gamma/2)) (the thesis's
// t += beta * 2 t tan(gamma/2) in closed form), and the level at step k is
// lam0 + k * l2r with lam0 = log2(2 T0 tan(gamma/2)).  hi/lo pairs carry the
// FP64 values to ~2^-48.
struct ConeConst {
  float l2r_hi, l2r_lo, lam0_hi, lam0_lo;
  int kmax;  // number of steps with t <= t_max
  int pad;
};

struct DevPyr {
  const uint8_t *lvl[VCT_MAX_LEVELS];  // level base pointers (slot table if bricked)
  const uint8_t *pool;                 // brick pool (brick layout)
  uint32_t bricked;                    // bit l: level l is bricked
  uint32_t pool_slots;                 // bricks the pool holds (bounds checks)
  float log2_tmax_t0;                  // log2(t_max / t0), both in level-0 voxels
  int n, levels, dtype;
  float h0;  // level-0 voxel edge in scene units
  float origin_f[3];         // origin (float32, as given)
  float scale_hi, scale_lo;  // n / size (scene units -> level-0 voxels) as a float pair
  ConeConst diffuse, occ, spec_fixed;
};

// One view of a launch.  Sizes are 16-bit (width, height <= 65535) so that
// 256 views fit the 32 KB kernel-parameter space.
struct DevView {
  const float *pos, *nrm, *rough;
  const uint8_t *mask;
  float *outD, *outS, *outV;
  const float *albedo;
  float *outL;
  uint2 *state;  // per-cone (K, transmittance before the last sample), or null
  float cam[3];
  int tile_begin, small_begin;  // first big / small tile item of the view
  uint16_t W, H, pyr, tiles_x;  // big tiles cover rows [0, y_split)
  uint16_t y_split, small_tiles_x;  // small tiles cover rows [y_split, H)
};

// Variant switches and shading constants of a forward launch (Ch. 5.4.4,
// Ch. 3.3, Ch. 4.2.2).
struct Variants {
  int flags;            // VCT_FLAG_* bits
  float shadow_str;     // occlusion fade: smoothstep(0, occ_max_dist, sqrt(t) shadow_str)
  float occ_max_dist;
  float grace;          // angular grace 0.008 pi shininess (radians)
  float falloff;        // exponent of the angular-grace BRDF
  float shininess;      // Phong exponent of the direct light
  float kd, ks;         // material ratios
  float light_color[3];
  float light_dir[3];   // as given (not normalised), like the occlusion cone axis
};

// Launch constants of the specular cone set-up and of the march (float32:
// the device path has no double-precision arithmetic).
struct SpecSetup {
  float gmin, gdelta;      // specular aperture at roughness_min, and its span
  float rough_min, inv_rough_span;  // roughness_min, 1 / (1 - roughness_min)
  float two_beta;          // 2 beta
  float t0_vox;            // start distance in level-0 voxels
};

// Tail tiles: the last pixels of a launch are handed out in small tiles so
// that warps finish together (forward trace only).
constexpr int kSmallTileW = 8, kSmallTileH = 4;

struct TraceLaunch {
  int n_views, total_tiles, tile_w, tile_h;
  int n_big;  // items [0, n_big) are big tiles, the rest small tiles
  int n_pyr;  // pyramids in pyr[]
  int n_diffuse, spec_enable, occ_enable, pad0;
  Variants var;
  float diffuse_dir[VCT_MAX_DIFFUSE][3];
  float diffuse_weight[VCT_MAX_DIFFUSE];
  float light[3];
  float normal_offset;  // voxels
  SpecSetup spec;
  unsigned *queue;
  unsigned long long *stats;  // vct_trace_stats::samples / cones
  DevPyr pyr[VCT_MAX_PYRAMIDS];
  DevView views[kMaxViewsPerLaunch];
};

struct BwdView {
  DevView v;
  const float *gD, *gS, *gV;
  const float *gL;  // dL/d(shaded radiance), or null
};

struct BwdLaunch {
  int n_views, total_tiles, tile_w, tile_h;
  int n_diffuse, spec_enable, occ_enable;
  int deterministic;  // 1: accumulate in 64-bit fixed point (gfix_lvl), not float
  int aniso;          // 1: anisotropic pyramid (gradient levels >= 1 hold six volumes)
  float diffuse_dir[VCT_MAX_DIFFUSE][3];
  float diffuse_weight[VCT_MAX_DIFFUSE];
  float light[3];
  float normal_offset;
  SpecSetup spec;
  Variants var;  // the modified cones (Ch. 5.4.4) and compositing variant
  unsigned *queue;
  float *gpyr_lvl[VCT_MAX_LEVELS];  // float32 gradient pyramid levels
  unsigned long long *gfix_lvl[VCT_MAX_LEVELS];  // fixed-point levels (deterministic mode)
  DevPyr pyr;
  BwdView views[kMaxBwdViewsPerLaunch];
};

// Flags that change the adjoint's march or walk (the shading flags only add
// an output the adjoint does not differentiate).
inline bool bwd_has_variants(int flags) {
  return (flags & (VCT_FLAG_OCC_SMOOTH | VCT_FLAG_SPEC_GRACE | VCT_FLAG_DIFFUSE_FIRST_HIT |
                   VCT_FLAG_PREMULTIPLIED)) != 0;
}

// March constants of a cone of full aperture `gamma` (host, FP64).
inline ConeConst cone_const(double gamma, double beta, double t0_vox,
                                                double tmax_vox) {
  ConeConst c{};
  double th = tan(0.5 * gamma);
  double x = 2.0 * beta * th;
  double l2r = log1p(x) / 0.69314718055994530942;
  double lam0 = log2(2.0 * t0_vox * th);
  int kmax = 0;
  if (t0_vox <= tmax_vox) {
    double e = log2(tmax_vox / t0_vox) / l2r;
    double kf = floor(e) + 1.0;
    kmax = kf > (double)kMaxSteps ? kMaxSteps + 1 : (int)kf;
  }
  c.l2r_hi = (float)l2r;
  c.l2r_lo = (float)(l2r - (double)c.l2r_hi);
  c.lam0_hi = (float)lam0;
  c.lam0_lo = (float)(lam0 - (double)c.lam0_hi);
  c.kmax = kmax;
  return c;
}

// Records the thread-local message returned by vct_last_error(); returns st.
vct_status set_last_error(vct_status st, const char *fmt, ...);

// Host entry points implemented in the .cu files (internal linkage across TUs).
// True when launch_pack_mips streams the grid (dense layout, float32 with
// n >= 32 or binary16 with 32 <= n <= 256, a 32-byte aligned level 0) and
// needs no tensor map.
bool streamed_build(const float *level0, const vct_pyramid &pyr);
// `map`: the level-0 tensor map of the TMA path; unused (may be null) when
// streamed_build() holds.
cudaError_t launch_pack_mips(const float *level0, const vct_pyramid &pyr,
                             const CUtensorMap *map, cudaStream_t s);
cudaError_t launch_read_level(const vct_pyramid &pyr, int level, float *out, cudaStream_t s,
                              int direction = 0);
cudaError_t launch_build_aniso(const float *level0, const vct_pyramid &pyr, int sms,
                               cudaStream_t s);
// Brick occupancy of a level-0 grid and the slot tables of every bricked
// level, written at layout L's table offsets from `base`; the occupied count
// goes to base + kHeaderCountOff.  More than `capacity` bricks (zero brick
// included) leaves every slot 0 and writes VCT_ERR_WORKSPACE to the status word.
cudaError_t launch_brick_tables(const float *level0, int n, int levels, const Layout &L,
                                uint8_t *base, uint64_t capacity, cudaStream_t s);
cudaError_t launch_mip_adjoint(const float *gpyr_base, const Layout &gl, int n, int levels,
                               float *grad0, cudaStream_t s);
// Adjoint of launch_build_aniso at the anisotropic pyramid `pyr`: the
// gradient pyramid at gpyr_base (same layout) is pushed down coarse to fine
// (in place), then its level 0 is added into the dense grad0.
cudaError_t launch_mip_adjoint_aniso(const vct_pyramid &pyr, const float *gpyr_base,
                                     float *grad0, int sms, cudaStream_t s);
cudaError_t launch_wait_probe(uint32_t *flag, uint64_t max_ns, cudaStream_t s);
cudaError_t launch_bounds_probe(uint32_t *buf, uint32_t declared, uint32_t extra,
                                cudaStream_t s);
cudaError_t launch_trace(const TraceLaunch &L, int lpp, int dtype, bool bricks, int grid,
                         cudaStream_t s, bool aniso = false);
int trace_occupancy(int lpp, int dtype, bool variants);
cudaError_t launch_trace_bwd(const BwdLaunch &L, int lpp, int grid, cudaStream_t s);
// Fixed-point gradient (units of 2^-32) -> float32, `count` values.
cudaError_t launch_fix_to_float(const unsigned long long *fix, float *out, uint64_t count,
                                cudaStream_t s);
// Deterministic adjoint: contributions are rounded to multiples of 2^-32 and
// summed as 64-bit integers, so the order of the atomics does not matter.
constexpr float kFixScale = 4294967296.0f;  // 2^32
int trace_bwd_occupancy(int lpp, int dtype, bool bricks);

}  // namespace vct
