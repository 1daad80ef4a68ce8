// Brick occupancy and slot tables of a VCT_LAYOUT_BRICKS pyramid (Ch. 5.1:
// sparse storage in place of a full 3D texture): which 8^3 bricks of every bricked level hold a non-zero texel, and where
// in the pool each occupied brick goes.
#include <algorithm>

#include "vct_internal.cuh"

namespace vct {

namespace {

struct TableArgs {
  uint32_t *tbl[VCT_MAX_LEVELS];  // slot table of each bricked level
  uint64_t nb[VCT_MAX_LEVELS];    // bricks of each bricked level
  int nbricked;                   // bricked levels are 0 .. nbricked-1
  uint32_t *status;
  unsigned long long *count;
  uint64_t capacity;              // pool bricks, the zero brick included
};

// One warp per level-0 brick: 1 if any channel of its 512 texels is non-zero.
// level0 is dense [z][y][x][4]; the brick's rows of 8 texels are 128 bytes.
__global__ void __launch_bounds__(256) occupancy_kernel(const float4 *level0, int n,
                                                        uint32_t *flags, uint64_t bricks) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t b = warp; b < bricks; b += nwarps) {
    const uint32_t id = (uint32_t)b;  // Morton id of the brick
    const int bx = compact3(id), by = compact3(id >> 1), bz = compact3(id >> 2);
    bool any = false;
    // lane k reads texels k, k + 32, ...: each pass covers 4 rows of 8 texels
    for (int k = lane; k < 512; k += 32) {
      const int x = k & 7, y = (k >> 3) & 7, z = k >> 6;
      const float4 v = __ldcs(level0 + ((size_t)(8 * bz + z) * n + (8 * by + y)) * n + 8 * bx + x);
      any |= (v.x != 0.0f) | (v.y != 0.0f) | (v.z != 0.0f) | (v.w != 0.0f);
    }
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) flags[id] = any ? 1u : 0u;
  }
}

// One CTA: occupancy of the coarser bricked levels (a brick is occupied if
// any of its 8 child bricks, ids 8p .. 8p+7 one level down, is), then slots
// by an exclusive scan over all bricked levels in level order.
__global__ void __launch_bounds__(1024) tables_kernel(const TableArgs a) {
  __shared__ unsigned long long s_warp[32];
  __shared__ unsigned long long s_carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int l = 1; l < a.nbricked; ++l) {
    for (uint64_t p = threadIdx.x; p < a.nb[l]; p += blockDim.x) {
      const uint4 *c = reinterpret_cast<const uint4 *>(a.tbl[l - 1] + 8 * p);
      const uint4 u = c[0], v = c[1];
      a.tbl[l][p] = (u.x | u.y | u.z | u.w | v.x | v.y | v.z | v.w) ? 1u : 0u;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int l = 0; l < a.nbricked; ++l) {
    for (uint64_t base = 0; base < a.nb[l]; base += blockDim.x) {
      const uint64_t e = base + threadIdx.x;
      const unsigned long long f = e < a.nb[l] ? a.tbl[l][e] : 0u;
      unsigned long long x = f;
#pragma unroll
      for (int m = 1; m < 32; m <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, m);
        if (lane >= m) x += y;
      }
      if (lane == 31) s_warp[wid] = x;
      __syncthreads();
      if (wid == 0) {
        unsigned long long w = s_warp[lane];
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) {
          const unsigned long long y = __shfl_up_sync(0xffffffffu, w, m);
          if (lane >= m) w += y;
        }
        s_warp[lane] = w;
      }
      __syncthreads();
      const unsigned long long before = (wid ? s_warp[wid - 1] : 0ull) + s_carry;
      // slot 1 + (occupied bricks before this one); 0 for an empty brick
      if (e < a.nb[l]) a.tbl[l][e] = f ? (uint32_t)(1ull + before + x - f) : 0u;
      __syncthreads();
      if (threadIdx.x == blockDim.x - 1) s_carry = before + x;
      __syncthreads();
    }
  }
  const unsigned long long total = s_carry;
  if (threadIdx.x == 0) *a.count = total;
  if (1ull + total > a.capacity) {
    // The pool is too small: leave every brick empty and report it.
    for (int l = 0; l < a.nbricked; ++l)
      for (uint64_t e = threadIdx.x; e < a.nb[l]; e += blockDim.x) a.tbl[l][e] = 0u;
    if (threadIdx.x == 0) atomicExch(a.status, (uint32_t)VCT_ERR_WORKSPACE);
  }
}

}  // namespace

cudaError_t launch_brick_tables(const float *level0, int n, int levels, const Layout &L,
                                uint8_t *base, uint64_t capacity, cudaStream_t s) {
  TableArgs a{};
  a.nbricked = 0;
  for (int l = 0; l < levels; ++l)
    if ((L.bricked >> l) & 1u) {
      a.tbl[l] = reinterpret_cast<uint32_t *>(base + L.level_off[l]);
      a.nb[l] = level_bricks(n, l);
      a.nbricked = l + 1;
    }
  a.status = reinterpret_cast<uint32_t *>(base);
  a.count = reinterpret_cast<unsigned long long *>(base + kHeaderCountOff);
  a.capacity = capacity;
  if (a.nbricked == 0) {
    cudaError_t e = cudaMemsetAsync(base + kHeaderCountOff, 0, 8, s);
    return e;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t warps = a.nb[0];
  const int grid = (int)std::min<uint64_t>((warps + 7) / 8, (uint64_t)sms * 16);
  occupancy_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float4 *>(level0), n, a.tbl[0],
                                        a.nb[0]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tables_kernel<<<1, 1024, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace vct
