// Mesh voxelization (Ch. 4.4): every triangle is rasterised once along its
// dominant axis into the level-0 grid (Ch. 4.4, Ch. 5.4.4 voxelize()).
//
// Coverage, depth and the winner of each voxel are exact integer decisions
// on vertices snapped to 1/256 voxel, so the result does not depend on the
// order in which threads run: every fragment raises the voxel's owner word
// to (triangle index + 1) with atomicMax, and a final pass writes the
// owner's colour (the highest triangle index wins, as in serial draw order).
//
// Kernels: clear (memset) -> setup_kernel (one thread per triangle:
// snap, dominant axis, colour; rasterises small triangles itself and lists
// the others) -> scan_kernel (one CTA: work items of the listed triangles)
// -> raster_large_kernel (warps take 1024-pixel items) -> resolve_kernel
// (owner grid -> dense RGBA grid).
#include <algorithm>

#include "voxelize.cuh"

namespace vct {

namespace {

constexpr int kSub = 256;                 // sub-voxel steps per voxel
constexpr float kCoordLimit = 524288.0f;  // 2^19 sub-voxel steps
constexpr int kSmallArea = 64;            // bounding boxes up to this: one thread
constexpr int kItemPixels = 1024;         // pixels per warp item of a large triangle
constexpr int kItemBatch = 4;             // consecutive items a warp claims at once
constexpr int kVoxThreads = 256;

struct LargeEntry {
  uint32_t tri, items;
};

struct VoxArgs {
  const float *vert;
  const int32_t *idx;
  const float *col;
  int nv, nt, n, pad;
  float org[3], s;
  float l[3], lc[3], amb, kd;
  vct_voxelize_stats *st;
  uint32_t *owner;
  float4 *colour;        // [nt]
  LargeEntry *large;     // [nt]
  uint64_t *first;       // [nt] first item of each listed triangle
  float4 *out;
};

// Snapped, projected triangle (components picked by the dominant axis, so
// that nothing is indexed at run time).
struct Tri {
  long long pu[3], pv[3];  // projection (u, v), counter-clockwise
  long long Nu, Nv, Nd;    // normal components along u, v and the dominant axis
  long long Vu, Vv, Vd;    // first vertex along u, v and the dominant axis
  int dom;
  int i0, i1, j0, j1;      // pixel bounding box clamped to the viewport (may be empty)
};

__device__ __forceinline__ long long floor_div(long long a, long long b) {
  if (b < 0) {
    a = -a;
    b = -b;
  }
  long long q = a / b;
  if (a % b != 0 && a < 0) --q;
  return q;
}

__device__ __forceinline__ long long iabs64(long long a) { return a < 0 ? -a : a; }

// floor(a / b), b != 0: a float32 estimate of the quotient, corrected to the
// exact value with one multiply (64-bit division only if the estimate is off
// by more than one, which the 2^-21 relative error of the estimate rules out
// for the quotients met here, |a / b| < 2^21).
__device__ __forceinline__ long long floor_div_fast(long long a, long long b) {
  if (b < 0) {
    a = -a;
    b = -b;
  }
  long long q = __float2ll_rd(__fdividef(__ll2float_rn(a), __ll2float_rn(b)));
  long long r = a - q * b;
  if (r < 0) {
    --q;
    r += b;
  } else if (r >= b) {
    ++q;
    r -= b;
  }
  if (r < 0 || r >= b) q = floor_div(a, b);
  return q;
}

// Component `a` of (x, y, z), a in {0, 1, 2}, without run-time indexing.
__device__ __forceinline__ long long pick(long long x, long long y, long long z, int a) {
  return a == 0 ? x : (a == 1 ? y : z);
}

// 0: usable, 1: bad index or vertex out of range, 2: zero snapped area.
__device__ int setup_tri(const VoxArgs &A, int t, Tri &T, int ix[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ix[k] = __ldg(A.idx + 3 * t + k);
    if (ix[k] < 0 || ix[k] >= A.nv) return 1;
  }
  long long X[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // float32 arithmetic without contraction, then round half to even
      const float b = __fmul_rn(__fsub_rn(__ldg(A.vert + 3 * ix[k] + a), A.org[a]), A.s);
      if (!(fabsf(b) < kCoordLimit)) return 1;
      X[k][a] = __float2ll_rn(b);
    }
  long long e1[3], e2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    e1[a] = X[1][a] - X[0][a];
    e2[a] = X[2][a] - X[0][a];
  }
  const long long N0 = e1[1] * e2[2] - e1[2] * e2[1];
  const long long N1 = e1[2] * e2[0] - e1[0] * e2[2];
  const long long N2 = e1[0] * e2[1] - e1[1] * e2[0];
  if (N0 == 0 && N1 == 0 && N2 == 0) return 2;
  const long long ax = iabs64(N0), ay = iabs64(N1), az = iabs64(N2);
  // dominant axis, first on ties; raster axes as in Ch. 4.4.2's swizzle:
  // x-dominant (u, v) = (z, y), y-dominant (x, z), z-dominant (x, y)
  int au, av;
  if (ax >= ay && ax >= az) {
    T.dom = 0; au = 2; av = 1;
  } else if (ay >= az) {
    T.dom = 1; au = 0; av = 2;
  } else {
    T.dom = 2; au = 0; av = 1;
  }
  T.Nu = pick(N0, N1, N2, au);
  T.Nv = pick(N0, N1, N2, av);
  T.Nd = pick(N0, N1, N2, T.dom);
  T.Vu = pick(X[0][0], X[0][1], X[0][2], au);
  T.Vv = pick(X[0][0], X[0][1], X[0][2], av);
  T.Vd = pick(X[0][0], X[0][1], X[0][2], T.dom);
  long long P[3][2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    P[k][0] = pick(X[k][0], X[k][1], X[k][2], au);
    P[k][1] = pick(X[k][0], X[k][1], X[k][2], av);
  }
  const long long area2 =
      (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[1][1] - P[0][1]) * (P[2][0] - P[0][0]);
  const bool flip = area2 < 0;
  T.pu[0] = P[0][0];
  T.pv[0] = P[0][1];
  T.pu[1] = flip ? P[2][0] : P[1][0];
  T.pv[1] = flip ? P[2][1] : P[1][1];
  T.pu[2] = flip ? P[1][0] : P[2][0];
  T.pv[2] = flip ? P[1][1] : P[2][1];
  const long long umin = min(P[0][0], min(P[1][0], P[2][0]));
  const long long umax = max(P[0][0], max(P[1][0], P[2][0]));
  const long long vmin = min(P[0][1], min(P[1][1], P[2][1]));
  const long long vmax = max(P[0][1], max(P[1][1], P[2][1]));
  // pixel centres 256 i + 128 inside [umin, umax]
  const long long hi = A.n - 1;
  T.i0 = (int)max(0ll, floor_div(umin - kSub / 2 + kSub - 1, kSub));
  T.i1 = (int)min(hi, floor_div(umax - kSub / 2, kSub));
  T.j0 = (int)max(0ll, floor_div(vmin - kSub / 2 + kSub - 1, kSub));
  T.j1 = (int)min(hi, floor_div(vmax - kSub / 2, kSub));
  return 0;
}

// Edge a -> b of a counter-clockwise triangle: is the centre (pu, pv)
// inside, with centres on the edge counted for top and left edges only?
__device__ __forceinline__ bool edge_in(long long au, long long av, long long bu, long long bv,
                                        long long pu, long long pv) {
  const long long eu = bu - au, ev = bv - av;
  const long long e = eu * (pv - av) - ev * (pu - au);
  return e > 0 || (e == 0 && (ev < 0 || (ev == 0 && eu < 0)));
}

// Linear voxel index of the fragment at pixel (i, j), or -1.
__device__ __forceinline__ long long fragment(const Tri &T, int n, int i, int j) {
  const long long pu = (long long)kSub * i + kSub / 2, pv = (long long)kSub * j + kSub / 2;
  if (!edge_in(T.pu[0], T.pv[0], T.pu[1], T.pv[1], pu, pv) ||
      !edge_in(T.pu[1], T.pv[1], T.pu[2], T.pv[2], pu, pv) ||
      !edge_in(T.pu[2], T.pv[2], T.pu[0], T.pv[0], pu, pv))
    return -1;
  // plane N . (X - V0) = 0 solved for the dominant coordinate, floored
  const long long off = -(T.Nu * (pu - T.Vu) + T.Nv * (pv - T.Vv));
  const long long depth = T.Vd + floor_div_fast(off, T.Nd);
  const long long k = floor_div(depth, kSub);
  if (k < 0 || k >= n) return -1;
  const long long nn = n;
  if (T.dom == 0) return ((long long)i * nn + j) * nn + k;  // x = k, y = j, z = i
  if (T.dom == 1) return ((long long)j * nn + k) * nn + i;  // x = i, y = k, z = j
  return (k * nn + j) * nn + i;                             // x = i, y = j, z = k
}

__device__ __forceinline__ void warp_add_u64(unsigned long long *dst, unsigned long long v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}
__device__ __forceinline__ void warp_add_u32(unsigned *dst, unsigned v) {
  v = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

__global__ void __launch_bounds__(kVoxThreads) setup_kernel(const __grid_constant__ VoxArgs A) {
  unsigned long long frags = 0;
  unsigned skipped = 0, degenerate = 0;
  const int stride = gridDim.x * blockDim.x;
  // whole warps iterate together so that the warp reductions below see every lane
  const int nt_pad = (A.nt + 31) & ~31;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt_pad; t += stride) {
    if (t >= A.nt) continue;
    Tri T;
    int ix[3];
    const int r = setup_tri(A, t, T, ix);
    if (r == 1) {
      ++skipped;
      continue;
    }
    if (r == 2) {
      ++degenerate;
      continue;
    }
    // direct diffuse light (Phong without the glossy term) of the unsnapped triangle
    float a3[3], b3[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float v0 = __ldg(A.vert + 3 * ix[0] + a);
      a3[a] = __ldg(A.vert + 3 * ix[1] + a) - v0;
      b3[a] = __ldg(A.vert + 3 * ix[2] + a) - v0;
    }
    const float nx = a3[1] * b3[2] - a3[2] * b3[1];
    const float ny = a3[2] * b3[0] - a3[0] * b3[2];
    const float nz = a3[0] * b3[1] - a3[1] * b3[0];
    const float len = sqrtf(nx * nx + ny * ny + nz * nz);
    const float lam =
        len > 0.0f ? fmaxf((nx * A.l[0] + ny * A.l[1] + nz * A.l[2]) / len, 0.0f) : 0.0f;
    const float f = A.amb + A.kd * lam;
    A.colour[t] = make_float4(__ldg(A.col + 3 * t) * A.lc[0] * f,
                              __ldg(A.col + 3 * t + 1) * A.lc[1] * f,
                              __ldg(A.col + 3 * t + 2) * A.lc[2] * f, 1.0f);
    if (T.i0 > T.i1 || T.j0 > T.j1) continue;
    const int w = T.i1 - T.i0 + 1, h = T.j1 - T.j0 + 1;
    const long long area = (long long)w * h;
    if (area <= kSmallArea) {
      for (int j = T.j0; j <= T.j1; ++j)
        for (int i = T.i0; i <= T.i1; ++i) {
          const long long v = fragment(T, A.n, i, j);
          if (v >= 0 && in_bounds((uint64_t)v, (uint64_t)A.n * A.n * A.n, kOobVoxel)) {
            atomicMax(A.owner + v, (unsigned)(t + 1));
            ++frags;
          }
        }
    } else {
      const unsigned slot = atomicAdd(&A.st->large_triangles, 1u);
      A.large[slot] = LargeEntry{(uint32_t)t, (uint32_t)((area + kItemPixels - 1) / kItemPixels)};
    }
  }
  warp_add_u64(reinterpret_cast<unsigned long long *>(&A.st->fragments), frags);
  warp_add_u32(&A.st->skipped, skipped);
  warp_add_u32(&A.st->degenerate, degenerate);
}

// One CTA: exclusive scan of the listed triangles' item counts.
__global__ void __launch_bounds__(1024) scan_kernel(const __grid_constant__ VoxArgs A) {
  __shared__ unsigned long long s_warp[32];
  __shared__ unsigned long long s_carry;
  const unsigned count = A.st->large_triangles;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (unsigned base = 0; base < count; base += 1024) {
    const unsigned e = base + threadIdx.x;
    unsigned long long x = e < count ? A.large[e].items : 0;
    // inclusive warp scan
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
      s_warp[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const unsigned long long before = (wid ? s_warp[wid - 1] : 0ull) + s_carry;
    const unsigned long long mine = e < count ? A.large[e].items : 0;
    if (e < count) A.first[e] = before + x - mine;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) A.st->large_items = s_carry;
}

__global__ void __launch_bounds__(kVoxThreads)
    raster_large_kernel(const __grid_constant__ VoxArgs A) {
  const unsigned count = A.st->large_triangles;
  const unsigned long long total = A.st->large_items;
  const int lane = threadIdx.x & 31;
  unsigned long long frags = 0;
  for (;;) {
    unsigned long long item0 = 0;
    if (lane == 0)
      item0 = atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->item_cursor),
                        (unsigned long long)kItemBatch);
    item0 = __shfl_sync(0xffffffffu, item0, 0);
    if (item0 >= total) break;
    // the listed triangle whose item range holds item0 (binary search), then
    // forwards through the batch
    unsigned lo = 0, hi = count - 1;
    while (lo < hi) {
      const unsigned mid = (lo + hi + 1) >> 1;
      if (A.first[mid] <= item0)
        lo = mid;
      else
        hi = mid - 1;
    }
    int cur = -1;
    Tri T;
    int ix[3];
    const unsigned long long item_end = min(item0 + (unsigned long long)kItemBatch, total);
    for (unsigned long long item = item0; item < item_end; ++item) {
      while (lo + 1 < count && A.first[lo + 1] <= item) ++lo;
      const int t = (int)A.large[lo].tri;
      if (t != cur) {
        setup_tri(A, t, T, ix);  // usable: it was listed by setup_kernel
        cur = t;
      }
      const int w = T.i1 - T.i0 + 1;
      const long long area = (long long)w * (T.j1 - T.j0 + 1);
      const long long p0 = (long long)(item - A.first[lo]) * kItemPixels;
      const long long p1 = min(p0 + kItemPixels, area);
      for (long long p = p0 + lane; p < p1; p += 32) {
        const int i = T.i0 + (int)(p % w), j = T.j0 + (int)(p / w);
        const long long v = fragment(T, A.n, i, j);
        if (v >= 0 && in_bounds((uint64_t)v, (uint64_t)A.n * A.n * A.n, kOobVoxel)) {
          atomicMax(A.owner + v, (unsigned)(t + 1));
          ++frags;
        }
      }
    }
  }
  warp_add_u64(reinterpret_cast<unsigned long long *>(&A.st->fragments), frags);
}

// Owner grid -> dense RGBA grid.  Each warp covers 128 consecutive voxels
// per pass, lane-contiguous, so owner loads and RGBA stores coalesce.
__global__ void __launch_bounds__(kVoxThreads) resolve_kernel(const __grid_constant__ VoxArgs A,
                                                             long long nvox) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * 128; base < nvox; base += nwarps * 128) {
    uint32_t o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long v = base + 32 * k + lane;
      o[k] = v < nvox ? __ldcs(A.owner + v) : 0u;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long v = base + 32 * k + lane;
      if (v < nvox)
        __stcs(A.out + v, o[k] && in_bounds(o[k] - 1, (uint64_t)A.nt, kOobVoxel)
                              ? __ldg(A.colour + (o[k] - 1)) : make_float4(0.f, 0.f, 0.f, 0.f));
    }
  }
}

}  // namespace

size_t voxelize_workspace_bytes(int n, int nt) {
  const uint64_t nv = (uint64_t)n * n * n;
  return (size_t)(kHeaderBytes + align256(nv * 4) + align256((uint64_t)nt * 16) +
                  align256((uint64_t)nt * 8) + align256((uint64_t)nt * 8));
}

cudaError_t launch_voxelize(const vct_mesh &m, int n, const float origin[3], float size,
                            const vct_voxel_light &light, float *out, void *ws, int sms,
                            cudaStream_t s) {
  VoxArgs A{};
  A.vert = m.vertices;
  A.idx = m.indices;
  A.col = m.colors;
  A.nv = m.n_vertices;
  A.nt = m.n_triangles;
  A.n = n;
  for (int a = 0; a < 3; ++a) {
    A.org[a] = origin[a];
    A.l[a] = light.light_dir[a];
    A.lc[a] = light.light_color[a];
  }
  A.s = (float)(256.0 * (double)n / (double)size);
  A.amb = light.ambient;
  A.kd = light.diffuse_str;
  uint8_t *w = static_cast<uint8_t *>(ws);
  const uint64_t nvox = (uint64_t)n * n * n;
  A.st = reinterpret_cast<vct_voxelize_stats *>(w);
  uint64_t off = kHeaderBytes;
  A.owner = reinterpret_cast<uint32_t *>(w + off);
  off += align256(nvox * 4);
  A.colour = reinterpret_cast<float4 *>(w + off);
  off += align256((uint64_t)A.nt * 16);
  A.large = reinterpret_cast<LargeEntry *>(w + off);
  off += align256((uint64_t)A.nt * 8);
  A.first = reinterpret_cast<uint64_t *>(w + off);
  A.out = reinterpret_cast<float4 *>(out);
  cudaError_t e = cudaMemsetAsync(ws, 0, kHeaderBytes + nvox * 4, s);
  if (e != cudaSuccess) return e;
  if (A.nt > 0) {
    const long long need = ((long long)A.nt + kVoxThreads - 1) / kVoxThreads;
    const int grid = (int)std::min<long long>(need, (long long)sms * 16);
    setup_kernel<<<grid, kVoxThreads, 0, s>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    scan_kernel<<<1, 1024, 0, s>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    raster_large_kernel<<<sms * 8, kVoxThreads, 0, s>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const long long chunks = (long long)((nvox + 127) / 128);  // one warp pass each
  const int rgrid = (int)std::min<long long>((chunks + kVoxThreads / 32 - 1) / (kVoxThreads / 32),
                                             (long long)sms * 8);
  resolve_kernel<<<rgrid, kVoxThreads, 0, s>>>(A, (long long)nvox);
  return cudaGetLastError();
}

VCT_OOB_ACCESSOR(oob_flags_voxelize)

}  // namespace vct
