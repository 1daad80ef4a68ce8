// Mip pyramid kernels: fused Morton packing + 2x2x2 box filter (Ch. 4.3.3),
// level readback, the adjoint of the box filter, and the bounded-wait probe.
#include <algorithm>

#include "vct_internal.cuh"

namespace vct {

namespace {

// Bulk (non-tensor) copies from shared to global memory: 16-byte aligned
// addresses, sizes a multiple of 16 bytes.
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(
                   reinterpret_cast<uint64_t>(gdst)),
               "r"(smem_u32(ssrc)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until the committed bulk copies have read their shared-memory sources.
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Waits until the committed bulk copies are complete.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Texel type stored for a pyramid dtype.
template <int DT> struct Tex;
template <> struct Tex<VCT_F32> { using T = float4; };
template <> struct Tex<VCT_F16> { using T = uint2; };

__device__ __forceinline__ void st_texel(float4 *p, float4 v) { *p = v; }
__device__ __forceinline__ void st_texel(uint2 *p, float4 v) { *p = pack_half4(v); }

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 mul4(float4 a, float s) {
  return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
// Mean of 8 children in child order 0..7 (x fastest, then y, then z).
__device__ __forceinline__ float4 mean8(const float4 *c) {
  float4 s = c[0];
#pragma unroll
  for (int i = 1; i < 8; ++i) s = add4(s, c[i]);
  return mul4(s, 0.125f);
}

struct PackArgs {
  uint8_t *lvl[VCT_MAX_LEVELS];  // level texels, or the slot table of a bricked level
  uint8_t *pool;                 // brick pool (brick layout)
  uint32_t bricked;              // bit l: level l is bricked
  uint32_t pool_slots;           // bricks the pool holds (bounds checks)
  float4 *staging;  // FP32 copy of level m_top (VCT_F16 or bricks), else null
  uint32_t *status;
  int n, B, m_top;  // block edge, last level produced inside a block
  uint32_t nblocks;  // (n / B)^3
  int lv_texels;     // texels of levels 1..m_top of one block
};

// Stores the texel with Morton code `code` of level l: in place for a dense
// level; for a bricked level in its brick's pool slot (nothing for an empty
// brick, whose slot is the shared zero brick).
template <int DT, bool BR>
__device__ __forceinline__ void put(uint8_t *const *lvl, const uint8_t *pool, uint32_t bricked,
                                    uint32_t pool_slots, int n, int l, uint32_t code, float4 v) {
  using T = typename Tex<DT>::T;
  if (!in_bounds(code, level_texels(n, l), kOobMip)) return;
  if (BR && ((bricked >> l) & 1u)) {
    const uint32_t slot = reinterpret_cast<const uint32_t *>(lvl[l])[code >> kBrickShift];
    if (slot != 0u && in_bounds(slot, pool_slots, kOobBrick))
      st_texel(reinterpret_cast<T *>(const_cast<uint8_t *>(pool)) +
                   (((size_t)slot << kBrickShift) | (code & 511u)),
               v);
  } else {
    st_texel(reinterpret_cast<T *>(lvl[l]) + code, v);
  }
}

// Level 0 (Morton order, into `mort`) and level 1 (into lvf, float32) of
// one B^3 block from its dense copy in shared memory.  For B = 16 the lanes
// of a warp take cells and child order such that the eight lanes of each
// shared-memory phase touch eight different 16-byte bank groups, reading
// the dense copy and writing `mort`: lane l owns x cell (l >> 1) & 3 (+4
// with bit 3) and starts at child l, so lanes that share a cell column read
// opposite x parities.
template <int DT>
__device__ __forceinline__ void block_level01(const PackArgs &a, const float4 *dense,
                                              typename Tex<DT>::T *mort, float4 *lvf) {
  const int B = a.B;
  const int B3 = B * B * B;
  const int cells = B3 / 8;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = threadIdx.x; c < cells; c += blockDim.x) {
    int cx, cy, cz, rot;
    if (B == 16) {
      const int it = c >> 8;  // bit 8 of the cell's thread-pass index
      cx = ((lane >> 1) & 3) | (((lane >> 3) & 1) << 2);
      cy = (lane & 1) | (((lane >> 4) & 1) << 1) | ((w & 1) << 2);
      cz = ((w >> 1) & 3) | (it << 2);
      rot = lane;
    } else {
      cx = compact3(c);
      cy = compact3(c >> 1);
      cz = compact3(c >> 2);
      rot = 0;
    }
    const uint32_t code = morton3(cx, cy, cz);
    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = (i + rot) & 7;
      const int x = 2 * cx + (j & 1), y = 2 * cy + ((j >> 1) & 1), z = 2 * cz + (j >> 2);
      const float4 v = dense[(z * B + y) * B + x];
      sum = add4(sum, v);
      st_texel(mort + 8 * code + j, v);
    }
    if (a.m_top >= 1) lvf[code] = mul4(sum, 0.125f);
  }
}

// Copies `cnt` texels of level l with Morton codes code .. code+cnt-1 from
// shared memory to the pyramid (bulk copies; a bricked level gets one copy
// per occupied brick the range touches, none for empty bricks).
template <int DT, bool BR>
__device__ __forceinline__ void store_range(const PackArgs &a, int l, uint32_t code, uint32_t cnt,
                                            const typename Tex<DT>::T *src) {
  using T = typename Tex<DT>::T;
  if (!in_bounds((uint64_t)code + cnt, level_texels(a.n, l) + 1, kOobMip)) return;
  if (BR && ((a.bricked >> l) & 1u)) {
    const uint32_t *tbl = reinterpret_cast<const uint32_t *>(a.lvl[l]);
    T *pool = reinterpret_cast<T *>(a.pool);
    for (uint32_t c = code; c < code + cnt;) {
      const uint32_t end = min(code + cnt, ((c >> kBrickShift) + 1u) << kBrickShift);
      uint32_t slot = tbl[c >> kBrickShift];
      if (!in_bounds(slot, a.pool_slots, kOobBrick)) slot = 0u;
      T *dst = pool + (((size_t)slot << kBrickShift) | (c & 511u));
      if (slot != 0u && ((end - c) * sizeof(T)) % 16u != 0u) {
        for (uint32_t k = c; k < end; ++k) dst[k - c] = src[k - code];
      } else if (slot != 0u) {
        bulk_store(dst, src + (c - code), (end - c) * (uint32_t)sizeof(T));
      }
      c = end;
    }
  } else if ((cnt * sizeof(T)) % 16u != 0u) {
    // a single binary16 texel: too small for a bulk copy
    for (uint32_t k = 0; k < cnt; ++k) reinterpret_cast<T *>(a.lvl[l])[code + k] = src[k];
  } else {
    bulk_store(reinterpret_cast<T *>(a.lvl[l]) + code, src, cnt * (uint32_t)sizeof(T));
  }
}

// Persistent CTAs, each taking blocks blockIdx.x, blockIdx.x + gridDim.x,
// ... (Morton indices of the B^3 blocks of level 0).  Each block arrives by
// one TMA tensor copy into one of two shared-memory buffers (the copy of
// the next block is in flight while this one is reduced); the CTA assembles
// the block's level-0 texels in Morton order and its levels 1..m_top (each
// child group contiguous) in shared memory, and bulk copies write them out
// whole, so the pyramid is written in full lines.
template <int DT, bool BR>
__global__ void __launch_bounds__(256) pack_mips_kernel(const __grid_constant__ CUtensorMap map,
                                                        const PackArgs a) {
  using T = typename Tex<DT>::T;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  // TMA destinations must be 128-byte aligned.
  float4 *buf0 = reinterpret_cast<float4 *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int B = a.B;
  const int B3 = B * B * B;
  float4 *const buf1 = buf0 + B3;
  T *mort = reinterpret_cast<T *>(buf0 + 2 * B3);           // level 0, Morton order
  float4 *lvf = reinterpret_cast<float4 *>(mort + B3);      // levels 1..m_top, float32
  const int lv_texels = a.lv_texels;                        // texels of levels 1..m_top
  T *lvo = DT == VCT_F32 ? reinterpret_cast<T *>(lvf)       // levels 1..m_top as stored
                         : reinterpret_cast<T *>(lvf + lv_texels);
  __shared__ __align__(8) uint64_t bar[2];

  auto issue = [&](uint32_t b, int s) {
    const int bx = compact3(b), by = compact3(b >> 1), bz = compact3(b >> 2);
    uint64_t *br = s ? &bar[1] : &bar[0];
    mbar_expect_tx(br, (uint32_t)B3 * 16u);
    tma_load_4d(s ? buf1 : buf0, &map, br, 0, bx * B, by * B, bz * B);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  uint32_t blk = blockIdx.x;
  if (threadIdx.x == 0 && blk < a.nblocks) issue(blk, 0);
  uint32_t ph0 = 0u, ph1 = 0u;  // phase of each buffer's barrier
  int s = 0;
  for (; blk < a.nblocks; blk += gridDim.x, s ^= 1) {
    const uint32_t nxt = blk + gridDim.x;
    if (threadIdx.x == 0 && nxt < a.nblocks) {
      // buf[s ^ 1] was last read before the barriers that ended the previous block
      fence_proxy_async_smem();
      issue(nxt, s ^ 1);
    }
    uint64_t *br = s ? &bar[1] : &bar[0];
    const uint32_t ph = s ? ph1 : ph0;
    const bool got = mbar_wait_bounded(br, ph, kWaitBudgetNs);
    // the previous block's bulk stores have read `mort` and the levels
    if (threadIdx.x == 0) bulk_wait_read();
    if (!__syncthreads_and(got)) {
      // Give up: flag it, then wait once more (bounded) for the copies in
      // flight so that none is left writing this CTA's shared memory.
      if (threadIdx.x == 0) atomicExch(a.status, (uint32_t)VCT_ERR_TIMEOUT);
      mbar_wait_bounded(br, ph, kWaitBudgetNs);
      if (nxt < a.nblocks)
        mbar_wait_bounded(s ? &bar[0] : &bar[1], s ? ph0 : ph1, kWaitBudgetNs);
      if (threadIdx.x == 0) bulk_wait_all();
      return;
    }
    if (s)
      ph1 ^= 1u;
    else
      ph0 ^= 1u;
    block_level01<DT>(a, s ? buf1 : buf0, mort, lvf);
    // Levels 2..m_top inside the block.
    float4 *src = lvf;
    int cnt = B3 / 8;
    for (int l = 2; l <= a.m_top; ++l) {
      __syncthreads();
      float4 *dst = src + cnt;
      const int nc = cnt / 8;
      for (int j = threadIdx.x; j < nc; j += blockDim.x) dst[j] = mean8(src + 8 * j);
      src = dst;
      cnt = nc;
    }
    __syncthreads();
    if (DT != VCT_F32) {
      for (int j = threadIdx.x; j < lv_texels; j += blockDim.x) st_texel(lvo + j, lvf[j]);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      // FP32 copy of the block's top level (one texel, index blk of level
      // m_top) for the tail kernel; only set when the tail runs.
      if (a.staging != nullptr) a.staging[blk] = src[0];
      fence_proxy_async_smem();  // the generic writes above feed the bulk copies
      store_range<DT, BR>(a, 0, blk * (uint32_t)B3, (uint32_t)B3, mort);
      const T *lsrc = lvo;
      for (int l = 1, c = B3 / 8; l <= a.m_top; ++l, c /= 8) {
        store_range<DT, BR>(a, l, blk * (uint32_t)c, (uint32_t)c, lsrc);
        lsrc += c;
      }
      bulk_commit();
    }
    // (the next iteration's barriers order the reuse of the buffers)
  }
  if (threadIdx.x == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// dense float32 pyramids, n >= 32: levels 0 and 1 by streaming the grid in
// rows, then levels 2.. by CTA-sized groups of the (L2-resident) level 1
// ---------------------------------------------------------------------------
// 32-byte loads of the dense grid (read once: not kept in L1, first out of
// L2) and 32-byte stores (one whole sector each).
__device__ __forceinline__ void ld_stream_32(const float4 *p, float4 &a, float4 &b) {
  asm volatile(
      "ld.global.nc.L1::no_allocate.L2::evict_first.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, "
      "[%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}
__device__ __forceinline__ void st_stream_32(float4 *p, float4 a, float4 b) {
  asm volatile("st.global.L2::evict_first.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p),
               "f"(a.x), "f"(a.y), "f"(a.z), "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
               : "memory");
}
__device__ __forceinline__ void ld_32(const float4 *p, float4 &a, float4 &b) {
  asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z),
                 "=f"(b.w)
               : "l"(p));
}

// Programmatic dependent launch: a kernel launched after this one with the
// programmatic-serialization attribute may be scheduled before this one
// ends; it waits (griddepcontrol.wait) until this grid has completed and its
// memory is visible before it reads what this grid wrote.
__device__ __forceinline__ void allow_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void wait_for_previous_grid() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Levels 0 .. top (top <= 4) of one patch of X x 16 x 16 level-0 voxels per
// CTA (X = min(n, 256); the patch's origin a multiple of its extent), so
// that the levels above 1 are reduced on chip instead of re-reading level 1.
// The patch is taken in 16 phases, one per level-2 row (qy, qz) of it, each
// phase the four level-1 rows (2 qy + iy, 2 qz + iz), in units of 8 x 4
// level-1 cells: lane = cx' | row << 3 (row = iy | iz << 1), so a unit holds
// four whole level-2 cells and a warp reduces them with shuffles, with no
// barrier between phases.  Warp w takes units w and w + 8 of each phase.  A
// lane's cell: its 8 children as four 32-byte x pairs (rows of a unit are
// 256-byte pieces), written to level 0 at Morton codes 8 code .. 8 code + 7
// (child jx | jy << 1 | jz << 2, the x pairs contiguous), and their mean to
// level 1.  The loads of the next phase are issued as soon as the stores have
// taken the registers.  After the 16 phases the patch's level-3 and level-4
// texels come from its level-2 values, kept in shared memory.  Level-1 means
// add the children in the order the TMA pack kernel does for the same cell
// (starting at child (cy & 1) | (cx & 3) << 1); coarser levels add them in
// child order (mean8), as the group and pack kernels do, so every path gives
// the same bits.
constexpr int kStreamTop = 4;    // levels made by the streaming kernel: 0 .. 4
constexpr int kPatchX = 256;     // longest x extent of a patch
constexpr int kPatchYZ = 16;     // y and z extent of a patch (2^kStreamTop)
struct StreamArgs {
  const float4 *dense;
  void *lvl[kStreamTop + 1];        // texels as stored (float4 or binary16 x 4)
  uint64_t texels[kStreamTop + 1];
  float4 *staging;                  // float32 copy of level 4 (binary16 pyramids), or null
  int n, X, top;
};
// 32 bytes of four binary16 texels (one whole sector), first out of L2
__device__ __forceinline__ void st_stream_32(uint2 *p, uint2 a, uint2 b, uint2 c, uint2 d) {
  asm volatile("st.global.L2::evict_first.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p),
               "r"(a.x), "r"(a.y), "r"(b.x), "r"(b.y), "r"(c.x), "r"(c.y), "r"(d.x), "r"(d.y)
               : "memory");
}
// Stored texels of one level (DT: float32 or binary16).
template <int DT>
__device__ __forceinline__ typename Tex<DT>::T *level_ptr(const StreamArgs &a, int l) {
  return reinterpret_cast<typename Tex<DT>::T *>(a.lvl[l]);
}
template <int DT>
__global__ void __launch_bounds__(256, 2) stream_levels_kernel(const __grid_constant__ StreamArgs a) {
  __shared__ float4 s2[16 * (kPatchX / 4)];  // the patch's level 2, row qz * 4 + qy
  __shared__ float4 s3[4 * (kPatchX / 8)];   // level 3, row rz * 2 + ry
  allow_dependents();
  const uint32_t n = (uint32_t)a.n, X = (uint32_t)a.X, hx = X >> 1;
  const uint32_t pxn = n / X, pyn = n / kPatchYZ;
  const uint64_t patches = (uint64_t)pxn * pyn * pyn;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t units = hx / 8;  // units per phase (2 .. 16)
  const uint32_t row = lane >> 3;
  float4 r[2][8];
  // level-1 cell (gx, gy, gz) of this lane in unit slot k of phase p of patch P
  auto cell = [&](uint64_t P, int p, int k, uint32_t &gx, uint32_t &gy, uint32_t &gz) {
    const uint32_t u = warp + 8u * (uint32_t)k;
    const uint32_t px = (uint32_t)(P % pxn), py = (uint32_t)((P / pxn) % pyn),
                   pz = (uint32_t)(P / ((uint64_t)pxn * pyn));
    gx = px * hx + 8u * u + (lane & 7u);
    gy = py * (kPatchYZ / 2) + 2u * (uint32_t)(p & 3) + (row & 1u);
    gz = pz * (kPatchYZ / 2) + 2u * (uint32_t)(p >> 2) + (row >> 1);
    return u < units;
  };
  auto load = [&](uint64_t P, int p) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      uint32_t gx, gy, gz;
      if (!cell(P, p, k, gx, gy, gz)) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {  // q = jy | jz << 1
        const uint64_t y = 2 * gy + (q & 1), z = 2 * gz + (q >> 1);
        ld_stream_32(a.dense + (z * n + y) * n + 2 * gx, r[k][2 * q], r[k][2 * q + 1]);
      }
    }
  };
  if (blockIdx.x < patches) load(blockIdx.x, 0);
  for (uint64_t P = blockIdx.x; P < patches; P += gridDim.x) {
    const uint32_t px = (uint32_t)(P % pxn), py = (uint32_t)((P / pxn) % pyn),
                   pz = (uint32_t)(P / ((uint64_t)pxn * pyn));
    for (int p = 0; p < 16; ++p) {
      float4 m[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        uint32_t gx, gy, gz;
        m[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!cell(P, p, k, gx, gy, gz)) continue;
        const uint32_t code = morton3(gx, gy, gz);
        if (in_bounds(8 * (uint64_t)code + 7, a.texels[0], kOobMip)) {
          if constexpr (DT == VCT_F32) {
            float4 *dst = level_ptr<DT>(a, 0) + 8 * (uint64_t)code;
#pragma unroll
            for (int q = 0; q < 4; ++q) st_stream_32(dst + 2 * q, r[k][2 * q], r[k][2 * q + 1]);
          } else {
            uint2 *dst = level_ptr<DT>(a, 0) + 8 * (uint64_t)code;
#pragma unroll
            for (int h = 0; h < 2; ++h)
              st_stream_32(dst + 4 * h, pack_half4(r[k][4 * h]), pack_half4(r[k][4 * h + 1]),
                           pack_half4(r[k][4 * h + 2]), pack_half4(r[k][4 * h + 3]));
          }
        }
        if (a.top < 1) continue;
        // rotate so that u[i] = r[(i + rot) & 7], then add in order
        const int rot = (int)((gy & 1u) | ((gx & 3u) << 1));
        float4 u[8], w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) u[i] = (rot & 1) ? r[k][(i + 1) & 7] : r[k][i];
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = (rot & 2) ? u[(i + 2) & 7] : u[i];
#pragma unroll
        for (int i = 0; i < 8; ++i) u[i] = (rot & 4) ? w[(i + 4) & 7] : w[i];
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 8; ++i) sum = add4(sum, u[i]);
        m[k] = mul4(sum, 0.125f);
        if (in_bounds(code, a.texels[1], kOobMip)) st_texel(level_ptr<DT>(a, 1) + code, m[k]);
      }
      // the next phase's loads (the stores above have taken r)
      if (p + 1 < 16)
        load(P, p + 1);
      else if (P + gridDim.x < patches)
        load(P + gridDim.x, 0);
      if (a.top < 2) continue;
      // level-2 cells of each unit: lanes 0..3 take cell c = lane, children
      // i at lane 2c + (i & 1) + (i >> 1) * 8 (child order, as mean8)
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const uint32_t u = warp + 8u * (uint32_t)k;
        if (u >= units) continue;  // warp-uniform
        const uint32_t c = lane & 3u;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int src = (int)(2u * c) + (i & 1) + (i >> 1) * 8;
          float4 ch;
          ch.x = __shfl_sync(0xffffffffu, m[k].x, src);
          ch.y = __shfl_sync(0xffffffffu, m[k].y, src);
          ch.z = __shfl_sync(0xffffffffu, m[k].z, src);
          ch.w = __shfl_sync(0xffffffffu, m[k].w, src);
          v = i == 0 ? ch : add4(v, ch);
        }
        v = mul4(v, 0.125f);
        if (lane < 4u) {
          const uint32_t qx = 4u * u + c;
          const uint32_t code = morton3(px * (X / 4) + qx, py * (kPatchYZ / 4) + (p & 3),
                                        pz * (kPatchYZ / 4) + (p >> 2));
          if (in_bounds(code, a.texels[2], kOobMip)) st_texel(level_ptr<DT>(a, 2) + code, v);
          s2[p * (X / 4) + qx] = v;
        }
      }
    }
    __syncthreads();
    const uint32_t t = threadIdx.x;
    const uint32_t w3 = X / 8;  // level-3 texels per row of the patch
    if (a.top >= 3 && t < 4 * w3) {
      const uint32_t rx = t % w3, ry = (t / w3) & 1u, rz = t / (2 * w3);
      float4 c[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        c[i] = s2[((2 * rz + (i >> 2)) * 4 + 2 * ry + ((i >> 1) & 1)) * (X / 4) + 2 * rx + (i & 1)];
      const float4 v = mean8(c);
      const uint32_t code = morton3(px * w3 + rx, py * 2 + ry, pz * 2 + rz);
      if (in_bounds(code, a.texels[3], kOobMip)) st_texel(level_ptr<DT>(a, 3) + code, v);
      s3[(rz * 2 + ry) * w3 + rx] = v;
    }
    __syncthreads();
    if (a.top >= 4 && t < X / 16) {
      float4 c[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) c[i] = s3[(i >> 1) * w3 + 2 * t + (i & 1)];
      const float4 v = mean8(c);
      const uint32_t code = morton3(px * (X / 16) + t, py, pz);
      if (in_bounds(code, a.texels[4], kOobMip)) {
        st_texel(level_ptr<DT>(a, 4) + code, v);
        if (a.staging != nullptr) a.staging[code] = v;  // the tail's float32 source
      }
    }
    // the next patch's level-2 writes to s2 must not overtake the reads above
    __syncthreads();
  }
}

// Levels s+1 .. s+k of a dense float32 pyramid from level s, one CTA per
// group of 8^k consecutive level-s texels (Morton order: a 2^k cube); the
// children of texel j are 8j .. 8j+7.  Levels above the first are reduced in
// shared memory.
constexpr int kGroupLevels = 4;  // 4096 source texels per CTA
// The one-CTA tail starts from a level of at most this many texels.
constexpr uint64_t kTailSourceTexels = 4096;
struct GroupArgs {
  const float4 *src;
  float4 *dst[kGroupLevels];
  uint64_t dst_texels[kGroupLevels];
  uint64_t src_texels;  // texels of one volume of level s (the volume stride)
  int k;
};
// The plain box filter: the mean of the 8 children (volume unused).
struct MeanOf8 {
  __device__ __forceinline__ float4 operator()(const float4 *c, int) const { return mean8(c); }
};
// Reduce(children, volume): the texel from its 8 children; blockIdx.y is the
// volume (the direction of an anisotropic level, 0 for a dense pyramid).
template <class Reduce>
__global__ void __launch_bounds__(256) mip_group_kernel(const __grid_constant__ GroupArgs a) {
  __shared__ float4 sm[512 + 64 + 8 + 1];
  wait_for_previous_grid();  // level s comes from the previous kernel
  allow_dependents();
  const Reduce red;
  const int vol = (int)blockIdx.y;
  const float4 *src = a.src + (uint64_t)vol * a.src_texels;
  const int first = 1 << (3 * (a.k - 1));  // texels of level s+1 per group
  const uint64_t g = blockIdx.x;
  float4 *cur = sm;
  // two level-(s+1) texels per thread (blockDim.x = 256, first <= 512), the
  // loads of both issued before either reduction
  const int j0 = threadIdx.x, j1 = threadIdx.x + blockDim.x;
  float4 ch0[8], ch1[8];
  if (j0 < first) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      ld_32(src + 8 * (g * first + j0) + 2 * q, ch0[2 * q], ch0[2 * q + 1]);
  }
  if (j1 < first) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      ld_32(src + 8 * (g * first + j1) + 2 * q, ch1[2 * q], ch1[2 * q + 1]);
  }
  if (j0 < first) {
    const uint64_t o = g * first + j0;
    const float4 v = red(ch0, vol);
    if (in_bounds(o, a.dst_texels[0], kOobMip)) a.dst[0][(uint64_t)vol * a.dst_texels[0] + o] = v;
    cur[j0] = v;
  }
  if (j1 < first) {
    const uint64_t o = g * first + j1;
    const float4 v = red(ch1, vol);
    if (in_bounds(o, a.dst_texels[0], kOobMip)) a.dst[0][(uint64_t)vol * a.dst_texels[0] + o] = v;
    cur[j1] = v;
  }
  int cnt = first;
  for (int l = 1; l < a.k; ++l) {
    __syncthreads();
    float4 *nxt = cur + cnt;
    const int nc = cnt / 8;
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
      const float4 v = red(cur + 8 * j, vol);
      nxt[j] = v;
      const uint64_t o = g * nc + j;
      if (in_bounds(o, a.dst_texels[l], kOobMip)) a.dst[l][(uint64_t)vol * a.dst_texels[l] + o] = v;
    }
    cur = nxt;
    cnt = nc;
  }
}

struct TailArgs {
  uint8_t *lvl[VCT_MAX_LEVELS];
  uint8_t *pool;
  uint32_t bricked;
  uint32_t pool_slots;
  const float4 *src0;  // FP32 values of level m_top
  float4 *ping[2];     // FP32 scratch for levels above m_top (VCT_F16 or bricks), or null
  int n, levels, m_top;
};

// One CTA: levels m_top+1 .. levels-1 from the FP32 values of level m_top.
template <int DT, bool BR, bool kAfterPdl = false>
__global__ void __launch_bounds__(1024) mip_tail_kernel(const TailArgs a) {
  if constexpr (kAfterPdl) wait_for_previous_grid();
  // A dense FP32 level doubles as the FP32 source of the next one.
  constexpr bool kInPlace = DT == VCT_F32 && !BR;
  const float4 *src = a.src0;
  for (int l = a.m_top + 1; l < a.levels; ++l) {
    const int cnt = (int)level_texels(a.n, l);
    float4 *f32dst = kInPlace ? reinterpret_cast<float4 *>(a.lvl[l])
                              : a.ping[(l - a.m_top - 1) & 1];
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      float4 ch[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) ch[i] = src[8 * j + i];
      float4 m = mean8(ch);
      put<DT, BR>(a.lvl, a.pool, a.bricked, a.pool_slots, a.n, l, (uint32_t)j, m);
      if (!kInPlace) f32dst[j] = m;
    }
    __syncthreads();
    src = f32dst;
  }
}

// Level to dense; `tbl` (bricked level) maps bricks to pool slots, else null.
template <int DT>
__global__ void read_level_kernel(const uint8_t *lvl, const uint32_t *tbl, const uint8_t *pool,
                                  int m, float4 *out) {
  using T = typename Tex<DT>::T;
  const uint64_t total = (uint64_t)m * m * m;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = (uint32_t)(i % m), y = (uint32_t)((i / m) % m), z = (uint32_t)(i / ((uint64_t)m * m));
    const uint32_t code = morton3(x, y, z);
    const T *p = tbl ? reinterpret_cast<const T *>(pool) +
                           (((size_t)tbl[code >> kBrickShift] << kBrickShift) | (code & 511u))
                     : reinterpret_cast<const T *>(lvl) + code;
    out[i] = in_bounds(code, total, kOobMip) ? ld_texel(p) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// ---------------------------------------------------------------------------
// anisotropic mips (VCT_LAYOUT_ANISO, float32)
// ---------------------------------------------------------------------------
// Level 0 in Morton order from the dense grid: one thread per texel, reading
// along the dense rows (coalesced) and writing scattered 16-byte texels.
__global__ void aniso_level0_kernel(const float4 *__restrict__ dense, float4 *__restrict__ lvl0,
                                    int n) {
  const uint64_t total = (uint64_t)n * n * n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = (uint32_t)(i % n), y = (uint32_t)((i / n) % n),
                   z = (uint32_t)(i / ((uint64_t)n * n));
    const uint32_t code = morton3(x, y, z);
    if (in_bounds(code, total, kOobMip)) lvl0[code] = __ldcs(dense + i);
  }
}

// The pair (front, back) seen along the direction of travel: front-to-back
// opacity and the straight colour of the premultiplied composite.
__device__ __forceinline__ float4 pair_composite(float4 f, float4 b) {
  const float t = 1.0f - f.w;
  const float a = fmaf(t, b.w, f.w);
  const float tb = t * b.w;
  if (!(a > 0.0f)) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float inv = __frcp_rn(a);  // one reciprocal for the three channels
  return make_float4(fmaf(f.w, f.x, tb * b.x) * inv, fmaf(f.w, f.y, tb * b.y) * inv,
                     fmaf(f.w, f.z, tb * b.z) * inv, a);
}

// Texel of direction d (axis d >> 1, negative travel if d & 1) from its 8
// children, child c = dx | dy << 1 | dz << 2: the mean over the four pairs
// (c, c | 1 << axis) along the axis, each composited in the order of travel.
__device__ __forceinline__ float4 aniso_texel(const float4 ch[8], int d) {
  const int axis = d >> 1, neg = d & 1;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if ((c >> axis) & 1) continue;
    const float4 lo = ch[c], hi = ch[c | (1 << axis)];
    const float4 p = neg ? pair_composite(hi, lo) : pair_composite(lo, hi);
    acc.x += p.x;
    acc.y += p.y;
    acc.z += p.z;
    acc.w += p.w;
  }
  return make_float4(acc.x * 0.25f, acc.y * 0.25f, acc.z * 0.25f, acc.w * 0.25f);
}

// The texels of both directions of one axis (travel towards +axis into
// `pos`, towards -axis into `neg`) from the same 8 children: a pair's
// opacity 1 - (1 - a_f)(1 - a_b) is the same for either order of travel, so
// each pair's opacity and its reciprocal serve both directions.
__device__ __forceinline__ void aniso_axis(const float4 ch[8], int axis, float4 &pos,
                                           float4 &neg) {
  pos = make_float4(0.f, 0.f, 0.f, 0.f);
  neg = pos;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if ((c >> axis) & 1) continue;
    const float4 lo = ch[c], hi = ch[c | (1 << axis)];
    const float a = fmaf(1.0f - lo.w, hi.w, lo.w);
    if (!(a > 0.0f)) continue;
    const float inv = __fdividef(1.0f, a);  // a in (0, 1]: within 2 ulp of 1 / a
    const float tl = (1.0f - lo.w) * hi.w, th = (1.0f - hi.w) * lo.w;
    pos.x += fmaf(lo.w, lo.x, tl * hi.x) * inv;
    pos.y += fmaf(lo.w, lo.y, tl * hi.y) * inv;
    pos.z += fmaf(lo.w, lo.z, tl * hi.z) * inv;
    neg.x += fmaf(hi.w, hi.x, th * lo.x) * inv;
    neg.y += fmaf(hi.w, hi.y, th * lo.y) * inv;
    neg.z += fmaf(hi.w, hi.z, th * lo.z) * inv;
    pos.w += a;
    neg.w += a;
  }
  pos = make_float4(pos.x * 0.25f, pos.y * 0.25f, pos.z * 0.25f, pos.w * 0.25f);
  neg = make_float4(neg.x * 0.25f, neg.y * 0.25f, neg.z * 0.25f, neg.w * 0.25f);
}

// Levels 0 and 1 in one pass: one thread per level-1 texel j reads its 2x2x2
// block of the dense grid once, stores it as level-0 texels 8j .. 8j+7 (128
// contiguous bytes) and writes texel j of all six level-1 volumes.
__global__ void aniso_level01_kernel(const float4 *__restrict__ dense, float4 *__restrict__ lvl0,
                                     float4 *__restrict__ lvl1, int n) {
  const uint32_t m = (uint32_t)n >> 1;
  const uint64_t texels1 = (uint64_t)m * m * m, texels0 = 8 * texels1;
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < texels1;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x1 = compact3((uint32_t)j), y1 = compact3((uint32_t)(j >> 1)),
                   z1 = compact3((uint32_t)(j >> 2));
    float4 ch[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const uint64_t x = 2 * x1 + (c & 1), y = 2 * y1 + ((c >> 1) & 1), z = 2 * z1 + (c >> 2);
      ch[c] = __ldcs(dense + (z * (uint64_t)n + y) * (uint64_t)n + x);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (in_bounds(8 * j + c, texels0, kOobMip)) lvl0[8 * j + c] = ch[c];
#pragma unroll
    for (int d = 0; d < 6; ++d)
      if (in_bounds(j, texels1, kOobMip)) lvl1[(uint64_t)d * texels1 + j] = aniso_texel(ch, d);
  }
}

// The anisotropic reduction for the level-group kernel (volume = direction;
// the switch keeps the children's indices compile-time constants, so they
// stay in registers).
struct AnisoOf8 {
  __device__ __forceinline__ float4 operator()(const float4 *c, int d) const {
    switch (d) {
      case 0: return aniso_texel(c, 0);
      case 1: return aniso_texel(c, 1);
      case 2: return aniso_texel(c, 2);
      case 3: return aniso_texel(c, 3);
      case 4: return aniso_texel(c, 4);
      default: return aniso_texel(c, 5);
    }
  }
};

// Levels 0, 1 and 2 of an anisotropic pyramid from a 32-byte aligned dense
// grid (n >= 16), in units of 8 x 4 level-1 cells: the four level-1 rows
// (2 uy + iy, 2 uz + iz) under level-2 row (uy, uz), x cells 8 ux .. 8 ux +
// 7, lane = cx' | row << 3 (row = iy | iz << 1), ux fastest, so a warp reads
// 256-byte pieces of 16 rows of the grid.  A lane's cell: its 8 children as
// four 32-byte x pairs, written to level 0 at Morton codes 8 code .. 8 code
// + 7, and texel `code` of the six level-1 volumes; a unit holds four whole
// level-2 cells, whose six directional texels lanes 0..3 form from the
// level-1 texels of their children, gathered by shuffles.  The next unit's
// loads are issued before the level-2 work of this one.
__global__ void __launch_bounds__(256) aniso_stream012_kernel(const float4 *__restrict__ dense,
                                                              float4 *__restrict__ lvl0,
                                                              float4 *__restrict__ lvl1,
                                                              float4 *__restrict__ lvl2, int n,
                                                              int top) {
  allow_dependents();
  const uint32_t un = (uint32_t)n;
  const uint32_t uxn = un / 16, uyn = un / 4;
  const uint64_t units = (uint64_t)uxn * uyn * uyn;
  const uint64_t texels1 = (uint64_t)(un / 2) * (un / 2) * (un / 2), texels0 = 8 * texels1;
  const uint64_t texels2 = texels1 / 8;
  const uint32_t lane = threadIdx.x & 31u, row = lane >> 3, c = lane & 3u;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  // cell of this lane in unit u
  auto cell = [&](uint64_t u, uint32_t &cx, uint32_t &cy, uint32_t &cz) {
    const uint32_t ux = (uint32_t)(u % uxn), uy = (uint32_t)((u / uxn) % uyn),
                   uz = (uint32_t)(u / ((uint64_t)uxn * uyn));
    cx = 8u * ux + (lane & 7u);
    cy = 2u * uy + (row & 1u);
    cz = 2u * uz + (row >> 1);
  };
  auto load = [&](uint64_t u, float4 ch[8]) {
    uint32_t cx, cy, cz;
    cell(u, cx, cy, cz);
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // q = jy | jz << 1
      const uint64_t y = 2 * cy + (q & 1), z = 2 * cz + (q >> 1);
      ld_stream_32(dense + (z * un + y) * un + 2 * cx, ch[2 * q], ch[2 * q + 1]);
    }
  };
  const uint64_t u0 = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  float4 ch[8];
  if (u0 < units) load(u0, ch);
  for (uint64_t u = u0; u < units; u += warps) {
    uint32_t cx, cy, cz;
    cell(u, cx, cy, cz);
    const uint32_t code = morton3(cx, cy, cz);
    if (in_bounds(8 * (uint64_t)code + 7, texels0, kOobMip)) {
      float4 *dst = lvl0 + 8 * (uint64_t)code;
#pragma unroll
      for (int q = 0; q < 4; ++q) st_stream_32(dst + 2 * q, ch[2 * q], ch[2 * q + 1]);
    }
    if (top < 1) {
      if (u + warps < units) load(u + warps, ch);
      continue;
    }
    float4 t[6];
#pragma unroll
    for (int axis = 0; axis < 3; ++axis) aniso_axis(ch, axis, t[2 * axis], t[2 * axis + 1]);
#pragma unroll
    for (int d = 0; d < 6; ++d)
      if (in_bounds(code, texels1, kOobMip)) lvl1[(uint64_t)d * texels1 + code] = t[d];
    // the next unit's loads (ch is no longer needed) overlap the level-2 work
    if (u + warps < units) load(u + warps, ch);
    if (top < 2) continue;
    // lane c < 4 holds cell (8 ux + c, 2 uy, 2 uz): its level-2 cell is 4 ux + c
    const uint32_t code2 = morton3((cx + c) / 2u, cy / 2u, cz / 2u);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      // children i of lane c's level-2 cell at lanes 2c + (i & 1) + (i >> 1) * 8
      float4 k[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int src = (int)(2u * c) + (i & 1) + (i >> 1) * 8;
        k[i].x = __shfl_sync(0xffffffffu, t[d].x, src);
        k[i].y = __shfl_sync(0xffffffffu, t[d].y, src);
        k[i].z = __shfl_sync(0xffffffffu, t[d].z, src);
        k[i].w = __shfl_sync(0xffffffffu, t[d].w, src);
      }
      if (lane < 4u) {
        const float4 v = aniso_texel(k, d);
        if (in_bounds(code2, texels2, kOobMip)) lvl2[(uint64_t)d * texels2 + code2] = v;
      }
    }
  }
}

// Level l >= 2 of all six directions: one thread per (direction, texel); the
// 8 children of texel j are j*8 .. j*8+7 of the same direction's volume of
// level l - 1.
__global__ void aniso_level_kernel(const float4 *__restrict__ src_level, uint64_t src_texels,
                                   float4 *__restrict__ dst_level, uint64_t dst_texels) {
  const uint64_t total = 6 * dst_texels;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const int d = (int)(i / dst_texels);
    const uint64_t j = i - (uint64_t)d * dst_texels;
    const float4 *src = src_level + (uint64_t)d * src_texels + 8 * j;
    float4 ch[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) ch[c] = __ldg(src + c);
    if (in_bounds(j, dst_texels, kOobMip)) dst_level[(uint64_t)d * dst_texels + j] = aniso_texel(ch, d);
  }
}

// Adjoint of pair_composite for one child of the pair (f, b): G is the
// gradient of the pair's (C, alpha) (the texel's gradient times 1/4).  With
// the front and back weights w_f = a_f / alpha, w_b = (1 - a_f) a_b / alpha
// (C = w_f c_f + w_b c_b, w_f + w_b = 1) and D = c_b - c_f:
//   dalpha/da_f = 1 - a_b,  dalpha/da_b = 1 - a_f,
//   dC/dc_f = w_f,  dC/dc_b = w_b,
//   dC/da_f = -D (w_b + a_b w_f) / alpha,  dC/da_b = (1 - a_f) w_f D / alpha,
// the same partials as (c_f - a_b c_b - C (1 - a_b)) / alpha and
// (1 - a_f) (c_b - C) / alpha written without their cancellation when the
// two colours are close.  Where alpha = 0 the colour is 0 by definition and
// passes no gradient.
__device__ __forceinline__ float4 pair_adjoint(float4 f, float4 b, float4 G, bool own_front) {
  const float af = f.w, ab = b.w;
  const float a = fmaf(1.0f - af, ab, af);
  float4 r = make_float4(0.f, 0.f, 0.f, G.w * (own_front ? 1.0f - ab : 1.0f - af));
  if (!(a > 0.0f)) return r;
  const float wf = __fdiv_rn(af, a), wb = __fdiv_rn((1.0f - af) * ab, a);
  const float fc[3] = {f.x, f.y, f.z}, bc[3] = {b.x, b.y, b.z}, gc[3] = {G.x, G.y, G.z};
  // dC/da of this child per unit colour difference D
  const float k = own_front ? -__fdiv_rn(fmaf(ab, wf, wb), a) : __fdiv_rn((1.0f - af) * wf, a);
  const float wo = own_front ? wf : wb;
  float o[3], ga = 0.0f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o[c] = gc[c] * wo;
    ga = fmaf(gc[c], bc[c] - fc[c], ga);
  }
  r.x = o[0];
  r.y = o[1];
  r.z = o[2];
  r.w = fmaf(k, ga, r.w);
  return r;
}

// Transpose of aniso_level_kernel for level l >= 2: one thread per (direction
// d, child k of level l - 1): the child k gets, from its parent k >> 3 in
// volume d, the pair adjoint of its pair along axis(d) (partner k ^ 1 << axis;
// the front child is the one whose axis bit equals the travel sign bit).
__global__ void aniso_adjoint_level_kernel(const float4 *__restrict__ fwd_child,
                                           float4 *__restrict__ g_child,
                                           const float4 *__restrict__ g_parent,
                                           uint64_t child_texels) {
  const uint64_t total = 6 * child_texels, parent_texels = child_texels >> 3;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const int d = (int)(i / child_texels);
    const uint64_t k = i - (uint64_t)d * child_texels;
    const int axis = d >> 1, neg = d & 1;
    const bool own_front = (int)((k >> axis) & 1u) == neg;
    const float4 *vol = fwd_child + (uint64_t)d * child_texels;
    const float4 own = __ldg(vol + k), oth = __ldg(vol + (k ^ (1ull << axis)));
    const float4 G = mul4(__ldg(g_parent + (uint64_t)d * parent_texels + (k >> 3)), 0.25f);
    const float4 r = own_front ? pair_adjoint(own, oth, G, true) : pair_adjoint(oth, own, G, false);
    const uint64_t o = (uint64_t)d * child_texels + k;
    if (in_bounds(o, total, kOobMip)) g_child[o] = add4(g_child[o], r);
  }
}

// Level 1 -> level 0: one thread per level-0 texel k, summing the pair
// adjoints of its six parents (one per direction).
__global__ void aniso_adjoint_level0_kernel(const float4 *__restrict__ lvl0,
                                            float4 *__restrict__ g0,
                                            const float4 *__restrict__ g1, uint64_t texels0) {
  const uint64_t texels1 = texels0 >> 3;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < texels0;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const float4 own = __ldg(lvl0 + k);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const int axis = d >> 1, neg = d & 1;
      const bool own_front = (int)((k >> axis) & 1u) == neg;
      const float4 oth = __ldg(lvl0 + (k ^ (1ull << axis)));
      const float4 G = mul4(__ldg(g1 + (uint64_t)d * texels1 + (k >> 3)), 0.25f);
      acc = add4(acc, own_front ? pair_adjoint(own, oth, G, true) : pair_adjoint(oth, own, G, false));
    }
    if (in_bounds(k, texels0, kOobMip)) g0[k] = add4(g0[k], acc);
  }
}

struct AdjArgs {
  const float4 *g[VCT_MAX_LEVELS];
  int n, levels;
};

// grad0[z][y][x] += sum over levels of the level-l gradient of the ancestor,
// pushed down coarse to fine with 1/8 per level (transpose of the box filter).
__global__ void mip_adjoint_kernel(const AdjArgs a, float4 *grad0) {
  const uint64_t n = (uint64_t)a.n;
  const uint64_t total = n * n * n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = (uint32_t)(i % n), y = (uint32_t)((i / n) % n), z = (uint32_t)(i / (n * n));
    const uint32_t m = morton3(x, y, z);
    float4 acc = a.g[a.levels - 1][m >> (3 * (a.levels - 1))];
    for (int l = a.levels - 2; l >= 0; --l) {
      float4 g = a.g[l][m >> (3 * l)];
      acc = add4(g, mul4(acc, 0.125f));
    }
    float4 o = grad0[i];
    grad0[i] = add4(o, acc);
  }
}

__global__ void wait_probe_kernel(uint32_t *flag, uint64_t max_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  // Nothing ever arrives: the bounded wait must give up.
  if (!mbar_wait_bounded(&bar, 0, max_ns)) {
    if (threadIdx.x == 0) atomicExch(flag, (uint32_t)VCT_ERR_TIMEOUT);
  }
}

int grid_for(uint64_t work, int threads) {
  uint64_t g = (work + threads - 1) / threads;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t cap = (uint64_t)sms * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

template <int DT, bool BR>
cudaError_t pack_t(const CUtensorMap &map, const PackArgs &a, int blocks, size_t smem,
                   cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(pack_mips_kernel<DT, BR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pack_mips_kernel<DT, BR>, 256, smem);
  const int grid = std::max(1, std::min(blocks, sms * std::max(per_sm, 1)));
  pack_mips_kernel<DT, BR><<<grid, 256, smem, s>>>(map, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_build_aniso(const float *level0, const vct_pyramid &pyr, int sms,
                               cudaStream_t s) {
  const Layout L = make_layout(pyr.n, pyr.levels, pyr.dtype, pyr.layout);
  uint8_t *base = static_cast<uint8_t *>(pyr.data);
  const int n = pyr.n;
  auto grid_of = [&](uint64_t work) {
    return (int)std::max<uint64_t>(1, std::min<uint64_t>((work + 255) / 256, (uint64_t)sms * 16));
  };
  if (pyr.levels == 1) {
    aniso_level0_kernel<<<grid_of(level_texels(n, 0)), 256, 0, s>>>(
        reinterpret_cast<const float4 *>(level0), reinterpret_cast<float4 *>(base + L.level_off[0]),
        n);
    return cudaGetLastError();
  }
  auto lvl = [&](int l) { return reinterpret_cast<float4 *>(base + L.level_off[l]); };
  if (n >= 16 && reinterpret_cast<uintptr_t>(level0) % 32 == 0) {
    // levels 0..2 streamed, then level groups (programmatic dependents)
    const int top = std::min(2, pyr.levels - 1);
    aniso_stream012_kernel<<<sms * 8, 256, 0, s>>>(reinterpret_cast<const float4 *>(level0),
                                                    lvl(0), lvl(1), top >= 2 ? lvl(2) : nullptr,
                                                    n, top);
    cudaError_t e = cudaGetLastError();
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc{};
    lc.stream = s;
    lc.attrs = pdl;
    lc.numAttrs = 1;
    lc.blockDim = dim3(256);  // 256 threads: see the kernel
    for (int m = top; m < pyr.levels - 1 && e == cudaSuccess;) {
      // levels m+1 .. m+k of all six volumes from level m (8^k divides its texels)
      const int k = std::min(kGroupLevels, pyr.levels - 1 - m);
      GroupArgs g{};
      g.src = lvl(m);
      g.src_texels = level_texels(n, m);
      g.k = k;
      for (int i = 0; i < k; ++i) {
        g.dst[i] = lvl(m + 1 + i);
        g.dst_texels[i] = level_texels(n, m + 1 + i);
      }
      lc.gridDim = dim3((unsigned)(level_texels(n, m) >> (3 * k)), 6);
      e = cudaLaunchKernelEx(&lc, mip_group_kernel<AnisoOf8>, g);
      m += k;
    }
    return e;
  }
  aniso_level01_kernel<<<grid_of(level_texels(n, 1)), 256, 0, s>>>(
      reinterpret_cast<const float4 *>(level0), lvl(0), lvl(1), n);
  cudaError_t e = cudaGetLastError();
  for (int l = 2; l < pyr.levels && e == cudaSuccess; ++l) {
    aniso_level_kernel<<<grid_of(6 * level_texels(n, l)), 256, 0, s>>>(
        reinterpret_cast<const float4 *>(base + L.level_off[l - 1]), level_texels(n, l - 1),
        reinterpret_cast<float4 *>(base + L.level_off[l]), level_texels(n, l));
    e = cudaGetLastError();
  }
  return e;
}

// Dense pyramids from a 32-byte aligned grid, n >= 32 (binary16: n <= 256):
// stream_levels_kernel (levels 0 .. 4), then, for float32, groups of
// kGroupLevels levels while the level below holds more than one tail CTA's
// worth of texels, then the one-CTA tail (binary16: from the float32 copy of
// level 4 in the staging area, as the TMA path hands it over).
static cudaError_t build_dense_streamed(const float *level0, const vct_pyramid &pyr,
                                        cudaStream_t s) {
  const Layout L = make_layout(pyr.n, pyr.levels, pyr.dtype, pyr.layout);
  uint8_t *base = static_cast<uint8_t *>(pyr.data);
  auto lvl = [&](int l) { return reinterpret_cast<float4 *>(base + L.level_off[l]); };
  const bool f16 = pyr.dtype == VCT_F16;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  StreamArgs sa{};
  sa.dense = reinterpret_cast<const float4 *>(level0);
  sa.n = pyr.n;
  sa.X = std::min(pyr.n, kPatchX);
  sa.top = std::min(kStreamTop, pyr.levels - 1);
  for (int l = 0; l <= sa.top; ++l) {
    sa.lvl[l] = base + L.level_off[l];
    sa.texels[l] = level_texels(pyr.n, l);
  }
  const bool tail = sa.top < pyr.levels - 1;
  sa.staging = (f16 && tail) ? reinterpret_cast<float4 *>(base + L.staging_off[0]) : nullptr;
  const uint64_t patches = (uint64_t)(pyr.n / sa.X) * (pyr.n / kPatchYZ) * (pyr.n / kPatchYZ);
  const int grid1 = (int)std::min<uint64_t>(patches, (uint64_t)sms * 2);
  if (f16)
    stream_levels_kernel<VCT_F16><<<grid1, 256, 0, s>>>(sa);
  else
    stream_levels_kernel<VCT_F32><<<grid1, 256, 0, s>>>(sa);
  cudaError_t e = cudaGetLastError();
  int m = sa.top;  // the last level made so far
  if (e != cudaSuccess || !tail) return e;
  cudaLaunchAttribute pdl[1];
  pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t lc{};
  lc.stream = s;
  lc.attrs = pdl;
  lc.numAttrs = 1;
  // levels m+1 .. m+k from level m (8^k divides its texels: k <= log2(n) - m)
  while (!f16 && m < pyr.levels - 1 && level_texels(pyr.n, m) > kTailSourceTexels) {
    const int k = std::min(kGroupLevels, pyr.levels - 1 - m);
    GroupArgs g{};
    g.src = lvl(m);
    g.k = k;
    for (int i = 0; i < k; ++i) {
      g.dst[i] = lvl(m + 1 + i);
      g.dst_texels[i] = level_texels(pyr.n, m + 1 + i);
    }
    lc.gridDim = dim3((unsigned)(level_texels(pyr.n, m) >> (3 * k)));
    lc.blockDim = dim3(256);  // 256 threads: see the kernel
    g.src_texels = level_texels(pyr.n, m);
    if ((e = cudaLaunchKernelEx(&lc, mip_group_kernel<MeanOf8>, g)) != cudaSuccess) return e;
    m += k;
  }
  if (m >= pyr.levels - 1) return cudaSuccess;
  TailArgs t{};
  for (int l = 0; l < pyr.levels; ++l) t.lvl[l] = base + L.level_off[l];
  t.pool = base + L.pool_off;
  t.n = pyr.n;
  t.levels = pyr.levels;
  t.m_top = m;
  lc.gridDim = dim3(1);
  lc.blockDim = dim3(1024);
  if (!f16) {
    t.src0 = lvl(m);
    return cudaLaunchKernelEx(&lc, mip_tail_kernel<VCT_F32, false, true>, t);
  }
  t.src0 = reinterpret_cast<const float4 *>(base + L.staging_off[0]);
  t.ping[0] = reinterpret_cast<float4 *>(base + L.staging_off[1]);
  // levels above m+1 are at most 1/8 of staging_off[1] and land at the start
  // of staging_off[0], whose values were consumed
  t.ping[1] = reinterpret_cast<float4 *>(base + L.staging_off[0]);
  return cudaLaunchKernelEx(&lc, mip_tail_kernel<VCT_F16, false, true>, t);
}

bool streamed_build(const float *level0, const vct_pyramid &pyr) {
  // (its 32-byte loads need a 32-byte aligned grid; the TMA path needs 16)
  return pyr.layout == VCT_LAYOUT_DENSE && pyr.n >= 32 &&
         (pyr.dtype == VCT_F32 || (pyr.dtype == VCT_F16 && pyr.n <= 256)) &&
         reinterpret_cast<uintptr_t>(level0) % 32 == 0;
}

cudaError_t launch_pack_mips(const float *level0, const vct_pyramid &pyr,
                             const CUtensorMap *map, cudaStream_t s) {
  const bool br = pyr.layout == VCT_LAYOUT_BRICKS;
  if (streamed_build(level0, pyr)) return build_dense_streamed(level0, pyr, s);
  if (map == nullptr) return cudaErrorInvalidValue;
  const Layout L = make_layout(pyr.n, pyr.levels, pyr.dtype, pyr.layout);
  uint8_t *base = static_cast<uint8_t *>(pyr.data);
  const int B = pack_block(pyr.n);
  const int mB = ilog2(B);
  const int m_top = mB < pyr.levels - 1 ? mB : pyr.levels - 1;
  cudaError_t e;
  if (br) {
    // slot tables, then the zero brick
    const uint64_t tb = (uint64_t)texel_bytes(pyr.dtype);
    const uint64_t capacity = (pyr.bytes - L.pool_off) / (tb << kBrickShift);
    e = launch_brick_tables(level0, pyr.n, pyr.levels, L, base, capacity, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(base + L.pool_off, 0, tb << kBrickShift, s);
    if (e != cudaSuccess) return e;
  }
  PackArgs a{};
  for (int l = 0; l < pyr.levels; ++l) a.lvl[l] = base + L.level_off[l];
  a.pool = base + L.pool_off;
  a.bricked = L.bricked;
  a.pool_slots = br ? (uint32_t)std::min<uint64_t>((pyr.bytes - L.pool_off) /
                                                       ((uint64_t)texel_bytes(pyr.dtype) << kBrickShift),
                                                   0xffffffffull)
                    : 0u;
  a.status = reinterpret_cast<uint32_t *>(base);
  a.n = pyr.n;
  a.B = B;
  a.m_top = m_top;
  const bool tail = m_top < pyr.levels - 1;
  a.staging = ((pyr.dtype == VCT_F16 || br) && tail)
                  ? reinterpret_cast<float4 *>(base + L.staging_off[0]) : nullptr;
  const int B3 = B * B * B;
  const size_t tb = (size_t)texel_bytes(pyr.dtype);
  int lv_texels = 0;
  for (int l = 1, c = B3 / 8; l <= m_top; ++l, c /= 8) lv_texels += c;
  a.lv_texels = lv_texels;
  // two dense input buffers, level 0 in Morton order, levels 1..m_top in
  // float32 (and as stored, for VCT_F16)
  size_t smem = 128 + (size_t)B3 * 32 + (size_t)B3 * tb + (size_t)lv_texels * 16 +
                (pyr.dtype == VCT_F32 ? 0 : (size_t)lv_texels * tb);
  const int blocks = (int)level_texels(pyr.n, mB);  // (n/B)^3
  a.nblocks = (uint32_t)blocks;
  if (pyr.dtype == VCT_F32)
    e = br ? pack_t<VCT_F32, true>(*map, a, blocks, smem, s)
           : pack_t<VCT_F32, false>(*map, a, blocks, smem, s);
  else
    e = br ? pack_t<VCT_F16, true>(*map, a, blocks, smem, s)
           : pack_t<VCT_F16, false>(*map, a, blocks, smem, s);
  if (e != cudaSuccess || !tail) return e;

  TailArgs t{};
  for (int l = 0; l < pyr.levels; ++l) t.lvl[l] = base + L.level_off[l];
  t.pool = base + L.pool_off;
  t.bricked = L.bricked;
  t.pool_slots = a.pool_slots;
  t.n = pyr.n;
  t.levels = pyr.levels;
  t.m_top = m_top;
  if (pyr.dtype == VCT_F32 && !br) {
    t.src0 = reinterpret_cast<const float4 *>(base + L.level_off[m_top]);
    mip_tail_kernel<VCT_F32, false><<<1, 1024, 0, s>>>(t);
  } else {
    t.src0 = reinterpret_cast<const float4 *>(base + L.staging_off[0]);
    t.ping[0] = reinterpret_cast<float4 *>(base + L.staging_off[1]);
    // Levels above m_top+1 are at most 1/8 of the staging_off[1] region and
    // land at the start of staging_off[0], whose values were consumed.
    t.ping[1] = reinterpret_cast<float4 *>(base + L.staging_off[0]);
    if (pyr.dtype == VCT_F32)
      mip_tail_kernel<VCT_F32, true><<<1, 1024, 0, s>>>(t);
    else if (br)
      mip_tail_kernel<VCT_F16, true><<<1, 1024, 0, s>>>(t);
    else
      mip_tail_kernel<VCT_F16, false><<<1, 1024, 0, s>>>(t);
  }
  return cudaGetLastError();
}

cudaError_t launch_read_level(const vct_pyramid &pyr, int level, float *out, cudaStream_t s,
                              int direction) {
  const Layout L = make_layout(pyr.n, pyr.levels, pyr.dtype, pyr.layout);
  const uint8_t *base = static_cast<const uint8_t *>(pyr.data);
  const uint8_t *lvl = base + L.level_off[level] +
                       (uint64_t)direction * level_texels(pyr.n, level) * texel_bytes(pyr.dtype);
  const uint32_t *tbl =
      ((L.bricked >> level) & 1u) ? reinterpret_cast<const uint32_t *>(lvl) : nullptr;
  const uint8_t *pool = base + L.pool_off;
  const int m = pyr.n >> level;
  const int grid = grid_for(level_texels(pyr.n, level), 256);
  if (pyr.dtype == VCT_F32)
    read_level_kernel<VCT_F32><<<grid, 256, 0, s>>>(lvl, tbl, pool, m,
                                                    reinterpret_cast<float4 *>(out));
  else
    read_level_kernel<VCT_F16><<<grid, 256, 0, s>>>(lvl, tbl, pool, m,
                                                    reinterpret_cast<float4 *>(out));
  return cudaGetLastError();
}

cudaError_t launch_mip_adjoint(const float *gpyr_base, const Layout &gl, int n, int levels,
                               float *grad0, cudaStream_t s) {
  AdjArgs a{};
  for (int l = 0; l < levels; ++l)
    a.g[l] = reinterpret_cast<const float4 *>(reinterpret_cast<const uint8_t *>(gpyr_base) +
                                              gl.level_off[l]);
  a.n = n;
  a.levels = levels;
  const int grid = grid_for(level_texels(n, 0), 256);
  mip_adjoint_kernel<<<grid, 256, 0, s>>>(a, reinterpret_cast<float4 *>(grad0));
  return cudaGetLastError();
}

cudaError_t launch_mip_adjoint_aniso(const vct_pyramid &pyr, const float *gpyr_base,
                                     float *grad0, int sms, cudaStream_t s) {
  const Layout L = make_layout(pyr.n, pyr.levels, VCT_F32, VCT_LAYOUT_ANISO);
  const uint8_t *fwd = static_cast<const uint8_t *>(pyr.data);
  uint8_t *g = reinterpret_cast<uint8_t *>(const_cast<float *>(gpyr_base));
  const int n = pyr.n;
  auto grid_of = [&](uint64_t work) {
    return (int)std::max<uint64_t>(1, std::min<uint64_t>((work + 255) / 256, (uint64_t)sms * 16));
  };
  cudaError_t e = cudaSuccess;
  for (int l = pyr.levels - 1; l >= 2 && e == cudaSuccess; --l) {
    aniso_adjoint_level_kernel<<<grid_of(6 * level_texels(n, l - 1)), 256, 0, s>>>(
        reinterpret_cast<const float4 *>(fwd + L.level_off[l - 1]),
        reinterpret_cast<float4 *>(g + L.level_off[l - 1]),
        reinterpret_cast<const float4 *>(g + L.level_off[l]), level_texels(n, l - 1));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && pyr.levels >= 2) {
    aniso_adjoint_level0_kernel<<<grid_of(level_texels(n, 0)), 256, 0, s>>>(
        reinterpret_cast<const float4 *>(fwd + L.level_off[0]),
        reinterpret_cast<float4 *>(g + L.level_off[0]),
        reinterpret_cast<const float4 *>(g + L.level_off[1]), level_texels(n, 0));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  return launch_mip_adjoint(gpyr_base, L, n, 1, grad0, s);  // unpack level 0
}

cudaError_t launch_wait_probe(uint32_t *flag, uint64_t max_ns, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(flag, max_ns);
  return cudaGetLastError();
}

VCT_OOB_ACCESSOR(oob_flags_mips)

}  // namespace vct
