// Mip pyramid kernels: fused Morton packing + 2x2x2 box filter (Ch. 4.3.3),
// level readback, the adjoint of the box filter, and the bounded-wait probe.
#include "vct_internal.cuh"

namespace vct {

namespace {

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
  float4 *staging;  // FP32 copy of level m_top (VCT_F16 or bricks), else null
  uint32_t *status;
  int n, B, m_top;  // block edge, last level produced inside a block
};

// Stores the texel with Morton code `code` of level l: in place for a dense
// level; for a bricked level in its brick's pool slot (nothing for an empty
// brick, whose slot is the shared zero brick).
template <int DT, bool BR>
__device__ __forceinline__ void put(uint8_t *const *lvl, const uint8_t *pool, uint32_t bricked,
                                    int l, uint32_t code, float4 v) {
  using T = typename Tex<DT>::T;
  if (BR && ((bricked >> l) & 1u)) {
    const uint32_t slot = reinterpret_cast<const uint32_t *>(lvl[l])[code >> kBrickShift];
    if (slot != 0u)
      st_texel(reinterpret_cast<T *>(const_cast<uint8_t *>(pool)) +
                   (((size_t)slot << kBrickShift) | (code & 511u)),
               v);
  } else {
    st_texel(reinterpret_cast<T *>(lvl[l]) + code, v);
  }
}

// One CTA per B^3 block of level 0 (blockIdx.x = Morton index of the block).
// The dense block arrives by one TMA tensor copy into shared memory; the CTA
// writes the block's level-0 texels in Morton order and reduces it level by
// level in shared memory (levels 1..m_top), each child group contiguous.
template <int DT, bool BR>
__global__ void __launch_bounds__(256) pack_mips_kernel(const __grid_constant__ CUtensorMap map,
                                                        const PackArgs a) {
  using T = typename Tex<DT>::T;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  // TMA destinations must be 128-byte aligned.
  float4 *dense = reinterpret_cast<float4 *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int B = a.B;
  const int B3 = B * B * B;
  float4 *lv = dense + B3;  // reduced levels, Morton order, back to back
  __shared__ __align__(8) uint64_t bar;

  const uint32_t blk = blockIdx.x;
  const int bx = compact3(blk), by = compact3(blk >> 1), bz = compact3(blk >> 2);

  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, (uint32_t)B3 * 16u);
    tma_load_4d(dense, &map, &bar, 0, bx * B, by * B, bz * B);
  }
  if (!mbar_wait_bounded(&bar, 0, kWaitBudgetNs)) {
    // Give up: flag it, then wait once more (bounded) for the copy so that no
    // write into this CTA's shared memory is left in flight.
    if (threadIdx.x == 0) atomicExch(a.status, (uint32_t)VCT_ERR_TIMEOUT);
    mbar_wait_bounded(&bar, 0, kWaitBudgetNs);
    return;
  }

  // Level 0 (Morton) and level 1.
  const uint32_t code0 = blk * (uint32_t)B3;
  const int cells = B3 / 8;
  for (int c = threadIdx.x; c < cells; c += blockDim.x) {
    const int cx = compact3(c), cy = compact3(c >> 1), cz = compact3(c >> 2);
    float4 ch[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int x = 2 * cx + (i & 1), y = 2 * cy + ((i >> 1) & 1), z = 2 * cz + (i >> 2);
      ch[i] = dense[(z * B + y) * B + x];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) put<DT, BR>(a.lvl, a.pool, a.bricked, 0, code0 + 8 * c + i, ch[i]);
    if (a.m_top >= 1) {
      float4 m = mean8(ch);
      lv[c] = m;
      put<DT, BR>(a.lvl, a.pool, a.bricked, 1, blk * (uint32_t)cells + c, m);
    }
  }
  // Levels 2..m_top inside the block.
  float4 *src = lv;
  int cnt = cells;
  for (int l = 2; l <= a.m_top; ++l) {
    __syncthreads();
    float4 *dst = src + cnt;
    const int nc = cnt / 8;
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
      float4 m = mean8(src + 8 * j);
      dst[j] = m;
      put<DT, BR>(a.lvl, a.pool, a.bricked, l, blk * (uint32_t)nc + j, m);
    }
    src = dst;
    cnt = nc;
  }
  // FP32 copy of the block's top level (one texel, index blk of level m_top)
  // for the tail kernel; only set when the tail runs (m_top = log2 B >= 1).
  __syncthreads();
  if (a.staging != nullptr && threadIdx.x == 0) a.staging[blk] = src[0];
}

struct TailArgs {
  uint8_t *lvl[VCT_MAX_LEVELS];
  uint8_t *pool;
  uint32_t bricked;
  const float4 *src0;  // FP32 values of level m_top
  float4 *ping[2];     // FP32 scratch for levels above m_top (VCT_F16 or bricks), or null
  int n, levels, m_top;
};

// One CTA: levels m_top+1 .. levels-1 from the FP32 values of level m_top.
template <int DT, bool BR>
__global__ void __launch_bounds__(1024) mip_tail_kernel(const TailArgs a) {
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
      put<DT, BR>(a.lvl, a.pool, a.bricked, l, (uint32_t)j, m);
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
    out[i] = ld_texel(p);
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
  pack_mips_kernel<DT, BR><<<blocks, 256, smem, s>>>(map, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pack_mips(const float *level0, const vct_pyramid &pyr,
                             const CUtensorMap &map, cudaStream_t s) {
  const bool br = pyr.layout == VCT_LAYOUT_BRICKS;
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
  a.status = reinterpret_cast<uint32_t *>(base);
  a.n = pyr.n;
  a.B = B;
  a.m_top = m_top;
  const bool tail = m_top < pyr.levels - 1;
  a.staging = ((pyr.dtype == VCT_F16 || br) && tail)
                  ? reinterpret_cast<float4 *>(base + L.staging_off[0]) : nullptr;
  const int B3 = B * B * B;
  size_t smem = (size_t)B3 * 16 + 128;
  int c = B3 / 8;
  for (int l = 1; l <= m_top; ++l, c /= 8) smem += (size_t)c * 16;
  const int blocks = (int)level_texels(pyr.n, mB);  // (n/B)^3
  if (pyr.dtype == VCT_F32)
    e = br ? pack_t<VCT_F32, true>(map, a, blocks, smem, s)
           : pack_t<VCT_F32, false>(map, a, blocks, smem, s);
  else
    e = br ? pack_t<VCT_F16, true>(map, a, blocks, smem, s)
           : pack_t<VCT_F16, false>(map, a, blocks, smem, s);
  if (e != cudaSuccess || !tail) return e;

  TailArgs t{};
  for (int l = 0; l < pyr.levels; ++l) t.lvl[l] = base + L.level_off[l];
  t.pool = base + L.pool_off;
  t.bricked = L.bricked;
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

cudaError_t launch_read_level(const vct_pyramid &pyr, int level, float *out, cudaStream_t s) {
  const Layout L = make_layout(pyr.n, pyr.levels, pyr.dtype, pyr.layout);
  const uint8_t *base = static_cast<const uint8_t *>(pyr.data);
  const uint8_t *lvl = base + L.level_off[level];
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

cudaError_t launch_wait_probe(uint32_t *flag, uint64_t max_ns, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(flag, max_ns);
  return cudaGetLastError();
}

}  // namespace vct
