// Camera G-buffer: the geometry pass that fills the per-pixel position,
// normal and material buffers the cone tracer reads (Ch. 5.4: the scene is
// drawn into these buffers before the cone-tracing pass).
//
// Every coverage and depth decision is exact integer arithmetic on vertices,
// eye and pixel directions snapped to a fixed-point frame, so the result does
// not depend on the order in which triangles are met:
//   - |vertex - eye| <= 2^19 and |direction| <= 2^20 per component keep the
//     edge volumes D.(B x C) (|.| <= 3 * 2^59), their sum n.D and det(A, B, C)
//     (<= 3 * 2^58) inside int64;
//   - the nearest hit compares det / (n.D) fractions by 128-bit products.
// Triangles reach pixels through 16x16 tile lists built from a conservative
// screen box: the triangle clipped to a guard-band frustum two pixels wider
// than the image, projected, widened by one pixel (float rounding there only
// moves the box by far less than a pixel).
//
// Kernels: memset (stats, tile counters) -> gb_setup_kernel (one thread per
// triangle: snap, edge-volume coefficients, screen box, tile counts) ->
// gb_scan_kernel (one CTA: tile offsets) -> gb_fill_kernel (tile lists) ->
// gb_raster_kernel (one CTA per tile, one pixel per thread, warps of 8x4 pixels).
#include <algorithm>
#include <cmath>

#include "gbuffer.cuh"

namespace vct {

namespace {

constexpr int kSetupThreads = 256;
constexpr int kRasterThreads = kGbTile * kGbTile;  // one pixel per thread
constexpr int kChunk = kRasterThreads;             // records staged per pass
constexpr float kDirScale = 262144.0f;             // 2^18
constexpr int kWarpTiles = 16;  // tile boxes larger than this: the warp enumerates them

// Per-triangle record: the edge volumes of a pixel direction D are c[0..2].D,
// c[3..5].D, c[6..8].D; the box bounds the pixels the triangle can cover.
struct __align__(16) TriRec {
  long long c[9];         // B x C, C x A, A x B (snapped, relative to the eye)
  long long det;          // det(A, B, C); 0 never hits
  unsigned short box[4];  // pixel box x0, x1, y0, y1 inclusive; x0 > x1 = none
  long long pad;
};
static_assert(sizeof(TriRec) == 96, "TriRec is six 16-byte words");

struct GbArgs {
  const float *vert;
  const int32_t *idx;
  const float *col;
  int nv, nt, W, H;
  int tiles_x, tiles_y;
  float org[3], s, tx, ty;
  float f[3], r[3], u[3];  // camera basis as given (pixel directions)
  float inv[3][3];         // rows: coordinates along right, up, forward
  float gx, gy;            // guard-band half extents, tan units
  float kx, ky;            // pixels per tan unit: W / (2 tx), H / (2 ty)
  long long O[3];          // snapped eye
  vct_gbuffer_stats *st;
  uint32_t *off;     // [T + 1] tile counts, then exclusive offsets
  uint32_t *cursor;  // [T]
  TriRec *rec;       // [nt]
  uint32_t *pairs;   // [cap]
  uint32_t cap;
  float *pos, *nrm, *alb;
  uint8_t *mask;
  int32_t *tri;
};

__device__ __forceinline__ void warp_add(unsigned *dst, unsigned v) {
  v = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// Keeps the part of the polygon (x, y, z)[0..n) with a x + b y + c z >= 0.
__device__ int clip(const float *x, const float *y, const float *z, int n, float a, float b,
                    float c, float *ox, float *oy, float *oz) {
  int m = 0;
  for (int k = 0; k < n; ++k) {
    const int k2 = k + 1 == n ? 0 : k + 1;
    const float d1 = a * x[k] + b * y[k] + c * z[k];
    const float d2 = a * x[k2] + b * y[k2] + c * z[k2];
    if (d1 >= 0.0f) {
      ox[m] = x[k];
      oy[m] = y[k];
      oz[m] = z[k];
      ++m;
    }
    if ((d1 >= 0.0f) != (d2 >= 0.0f)) {
      const float w = d1 / (d1 - d2);
      ox[m] = x[k] + w * (x[k2] - x[k]);
      oy[m] = y[k] + w * (y[k2] - y[k]);
      oz[m] = z[k] + w * (z[k2] - z[k]);
      ++m;
    }
  }
  return m;
}

// 0 visible (box set), 1 skipped, 2 degenerate, 3 culled; *wide if the box
// had to be the whole image.
__device__ int setup_tri(const GbArgs &A, int t, TriRec &R, bool *wide) {
  *wide = false;
  int ix[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ix[k] = __ldg(A.idx + 3 * t + k);
    if (ix[k] < 0 || ix[k] >= A.nv) return 1;
  }
  long long V[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      long long X;
      if (!frame_snap(__ldg(A.vert + 3 * ix[k] + a), A.org[a], A.s, &X)) return 1;
      V[k][a] = X - A.O[a];
    }
  long long e1[3], e2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    e1[a] = V[1][a] - V[0][a];
    e2[a] = V[2][a] - V[0][a];
  }
  if (e1[1] * e2[2] - e1[2] * e2[1] == 0 && e1[2] * e2[0] - e1[0] * e2[2] == 0 &&
      e1[0] * e2[1] - e1[1] * e2[0] == 0)
    return 2;
  // c[3k..3k+2] = P_k x Q_k with (P, Q) = (B, C), (C, A), (A, B)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const long long *P = V[(k + 1) % 3], *Q = V[(k + 2) % 3];
    R.c[3 * k + 0] = P[1] * Q[2] - P[2] * Q[1];
    R.c[3 * k + 1] = P[2] * Q[0] - P[0] * Q[2];
    R.c[3 * k + 2] = P[0] * Q[1] - P[1] * Q[0];
  }
  R.det = R.c[0] * V[0][0] + R.c[1] * V[0][1] + R.c[2] * V[0][2];
  if (R.det == 0) return 3;  // the eye lies in the triangle's plane
  // camera coordinates (along right, up, forward): a pixel direction is
  // (sx, sy, 1) there up to rounding
  float x[8], y[8], z[8], x2[8], y2[8], z2[8];
  float M = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float p0 = (float)V[k][0], p1 = (float)V[k][1], p2 = (float)V[k][2];
    x[k] = A.inv[0][0] * p0 + A.inv[0][1] * p1 + A.inv[0][2] * p2;
    y[k] = A.inv[1][0] * p0 + A.inv[1][1] * p1 + A.inv[1][2] * p2;
    z[k] = A.inv[2][0] * p0 + A.inv[2][1] * p1 + A.inv[2][2] * p2;
    M = fmaxf(M, fabsf(x[k]) + fabsf(y[k]) + fabsf(z[k]));
  }
  int n = clip(x, y, z, 3, 1.0f, 0.0f, A.gx, x2, y2, z2);
  n = clip(x2, y2, z2, n, -1.0f, 0.0f, A.gx, x, y, z);
  n = clip(x, y, z, n, 0.0f, 1.0f, A.gy, x2, y2, z2);
  n = clip(x2, y2, z2, n, 0.0f, -1.0f, A.gy, x, y, z);
  if (n == 0) return 3;
  float lo_x = 3.0e38f, hi_x = -3.0e38f, lo_y = 3.0e38f, hi_y = -3.0e38f;
  // below this depth the float32 projection could move a vertex by a sizeable
  // fraction of a pixel: such triangles are binned to every tile
  const float zmin = M * (1.0f / 64.0f);
  for (int k = 0; k < n; ++k) {
    if (!(z[k] >= zmin)) {
      *wide = true;
      break;
    }
    const float px = x[k] / z[k] * A.kx, py = -y[k] / z[k] * A.ky;
    lo_x = fminf(lo_x, px);
    hi_x = fmaxf(hi_x, px);
    lo_y = fminf(lo_y, py);
    hi_y = fmaxf(hi_y, py);
  }
  int x0 = 0, x1 = A.W - 1, y0 = 0, y1 = A.H - 1;
  if (!*wide) {
    // pixel i has its centre at tan-coordinate offset i + 1/2 - W/2
    const float cx = 0.5f * A.W - 0.5f, cy = 0.5f * A.H - 0.5f;
    const float fx0 = fmaxf(floorf(lo_x + cx) - 1.0f, 0.0f);
    const float fx1 = fminf(ceilf(hi_x + cx) + 1.0f, (float)(A.W - 1));
    const float fy0 = fmaxf(floorf(lo_y + cy) - 1.0f, 0.0f);
    const float fy1 = fminf(ceilf(hi_y + cy) + 1.0f, (float)(A.H - 1));
    if (fx0 > fx1 || fy0 > fy1) return 3;
    x0 = (int)fx0;
    x1 = (int)fx1;
    y0 = (int)fy0;
    y1 = (int)fy1;
  }
  R.box[0] = (unsigned short)x0;
  R.box[1] = (unsigned short)x1;
  R.box[2] = (unsigned short)y0;
  R.box[3] = (unsigned short)y1;
  return 0;
}

// Calls f(t, tile) for every tile of every lane's box; boxes of more than
// kWarpTiles tiles are enumerated by the whole warp.  All lanes must call.
template <class F>
__device__ __forceinline__ void for_tiles(const GbArgs &A, int t, bool active, const TriRec &R,
                                          F f) {
  const int lane = threadIdx.x & 31;
  int tx0 = 0, ty0 = 0, w = 0, cnt = 0;
  if (active) {
    tx0 = R.box[0] / kGbTile;
    ty0 = R.box[2] / kGbTile;
    w = R.box[1] / kGbTile - tx0 + 1;
    cnt = w * (R.box[3] / kGbTile - ty0 + 1);
  }
  const bool big = cnt > kWarpTiles;
  if (!big)
    for (int k = 0; k < cnt; ++k) f(t, (ty0 + k / w) * A.tiles_x + tx0 + k % w);
  unsigned m = __ballot_sync(0xffffffffu, big);
  while (m) {
    const int src = __ffs(m) - 1;
    m &= m - 1;
    const int st = __shfl_sync(0xffffffffu, t, src);
    const int sx0 = __shfl_sync(0xffffffffu, tx0, src);
    const int sy0 = __shfl_sync(0xffffffffu, ty0, src);
    const int sw = __shfl_sync(0xffffffffu, w, src);
    const int sc = __shfl_sync(0xffffffffu, cnt, src);
    for (int k = lane; k < sc; k += 32) f(st, (sy0 + k / sw) * A.tiles_x + sx0 + k % sw);
  }
}

__global__ void __launch_bounds__(kSetupThreads) gb_setup_kernel(const __grid_constant__ GbArgs A) {
  unsigned skipped = 0, degenerate = 0, culled = 0, wide = 0;
  const int stride = gridDim.x * blockDim.x;
  // whole warps iterate together (warp-wide tile enumeration and reductions)
  const int nt_pad = (A.nt + 31) & ~31;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt_pad; t += stride) {
    TriRec R;
    int r = 3;
    bool w = false;
    if (t < A.nt) {
      r = setup_tri(A, t, R, &w);
      skipped += r == 1;
      degenerate += r == 2;
      culled += r == 3;
      wide += r == 0 && w;
      if (r != 0) {
        R.box[0] = 1;
        R.box[1] = 0;
        R.box[2] = 1;
        R.box[3] = 0;
      }
      A.rec[t] = R;
    }
    for_tiles(A, t, r == 0, R, [&](int, int tile) {
      if (in_bounds(tile, (uint64_t)A.tiles_x * A.tiles_y, kOobGbuffer)) atomicAdd(A.off + tile, 1u);
    });
  }
  warp_add(&A.st->skipped, skipped);
  warp_add(&A.st->degenerate, degenerate);
  warp_add(&A.st->culled, culled);
  warp_add(&A.st->wide, wide);
}

// One CTA: tile counts -> exclusive offsets (off[T] = total), overflow flag.
__global__ void __launch_bounds__(1024) gb_scan_kernel(const __grid_constant__ GbArgs A) {
  __shared__ unsigned long long s_warp[32];
  const int T = A.tiles_x * A.tiles_y;
  const int chunk = (T + 1023) / 1024;
  const int lo = min(T, (int)threadIdx.x * chunk), hi = min(T, lo + chunk);
  unsigned long long sum = 0;
  for (int k = lo; k < hi; ++k) sum += A.off[k];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long x = sum;
#pragma unroll
  for (int m = 1; m < 32; m <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, m);
    if (lane >= m) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned long long v = s_warp[lane];
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, v, m);
      if (lane >= m) v += y;
    }
    s_warp[lane] = v;
  }
  __syncthreads();
  unsigned long long run = (wid ? s_warp[wid - 1] : 0ull) + x - sum;
  for (int k = lo; k < hi; ++k) {
    const unsigned c = A.off[k];
    A.off[k] = (uint32_t)min(run, 0xffffffffull);
    run += c;
  }
  if (threadIdx.x == 1023) {
    const unsigned long long total = s_warp[31];
    A.off[T] = (uint32_t)min(total, 0xffffffffull);
    A.st->pairs = total;
    A.st->pair_capacity = A.cap;
    A.st->overflow = total > A.cap ? 1u : 0u;
  }
}

__global__ void __launch_bounds__(kSetupThreads) gb_fill_kernel(const __grid_constant__ GbArgs A) {
  if (A.st->overflow) return;
  const int stride = gridDim.x * blockDim.x;
  const int nt_pad = (A.nt + 31) & ~31;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt_pad; t += stride) {
    TriRec R;
    bool active = false;
    if (t < A.nt) {
      const uint2 b = *reinterpret_cast<const uint2 *>(&A.rec[t].box[0]);
      *reinterpret_cast<uint2 *>(&R.box[0]) = b;
      active = R.box[0] <= R.box[1];
    }
    for_tiles(A, t, active, R, [&](int tt, int tile) {
      if (!in_bounds(tile, (uint64_t)A.tiles_x * A.tiles_y, kOobGbuffer)) return;
      const uint32_t k = A.off[tile] + atomicAdd(A.cursor + tile, 1u);
      if (in_bounds(k, A.cap, kOobGbuffer)) A.pairs[k] = (uint32_t)tt;  // k < total <= cap
    });
  }
}

// a * b - c * d with one rounding error at most per product pair
// (Kahan's difference of products via a fused multiply-add)
__device__ __forceinline__ float diff_prod(float a, float b, float c, float d) {
  const float w = c * d;
  const float e = fmaf(-c, d, w);
  const float f = fmaf(a, b, -w);
  return f + e;
}

__global__ void __launch_bounds__(kRasterThreads) gb_raster_kernel(const __grid_constant__ GbArgs A) {
  __shared__ uint4 s_rec[kChunk * 6];
  __shared__ int s_tri[kChunk];
  const int tile = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx = (tile % A.tiles_x) * kGbTile + (warp & 1) * 8;
  const int by = (tile / A.tiles_x) * kGbTile + (warp >> 1) * 4;
  const int px = bx + (lane & 7), py = by + (lane >> 3);
  // snapped direction of the pixel centre (float32 steps, no contraction)
  const int ic = min(px, A.W - 1), jc = min(py, A.H - 1);
  const float sx =
      __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * ic + 1), (float)A.W), 1.0f), A.tx);
  const float sy =
      __fmul_rn(__fsub_rn(1.0f, __fdiv_rn((float)(2 * jc + 1), (float)A.H)), A.ty);
  long long D[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float d = __fadd_rn(__fadd_rn(A.f[a], __fmul_rn(sx, A.r[a])), __fmul_rn(sy, A.u[a]));
    D[a] = __float2ll_rn(__fmul_rn(d, kDirScale));
  }
  uint32_t begin = A.off[tile], end = A.off[tile + 1];
  if (A.st->overflow) end = begin;
  unsigned long long bnum = 0, bden = 1;
  int best = -1;
  bool bflip = false;
  for (uint32_t base = begin; base < end; base += kChunk) {
    const int n = (int)min((uint32_t)kChunk, end - base);
    __syncthreads();
    if ((int)threadIdx.x < n) {
      int t = (int)A.pairs[base + threadIdx.x];
      if (!in_bounds((uint32_t)t, (uint64_t)A.nt, kOobGbuffer)) t = 0;  // nt >= 1 here
      s_tri[threadIdx.x] = t;
      const uint4 *src = reinterpret_cast<const uint4 *>(A.rec + t);
#pragma unroll
      for (int k = 0; k < 6; ++k) s_rec[threadIdx.x * 6 + k] = __ldg(src + k);
    }
    __syncthreads();
    for (int q = 0; q < n; ++q) {
      const uint4 w5 = s_rec[q * 6 + 5];
      const int x0 = (int)(w5.x & 0xffffu), x1 = (int)(w5.x >> 16);
      const int y0 = (int)(w5.y & 0xffffu), y1 = (int)(w5.y >> 16);
      if (x0 > bx + 7 || x1 < bx || y0 > by + 3 || y1 < by) continue;  // warp-uniform
      if (px < x0 || px > x1 || py < y0 || py > y1) continue;
      const long long *c = reinterpret_cast<const long long *>(&s_rec[q * 6]);
      const long long det = c[9];
      // each edge volume must be zero or of det's sign
      const long long v0 = c[0] * D[0] + c[1] * D[1] + c[2] * D[2];
      if (v0 != 0 && (v0 ^ det) < 0) continue;
      const long long v1 = c[3] * D[0] + c[4] * D[1] + c[5] * D[2];
      if (v1 != 0 && (v1 ^ det) < 0) continue;
      const long long v2 = c[6] * D[0] + c[7] * D[1] + c[8] * D[2];
      if (v2 != 0 && (v2 ^ det) < 0) continue;
      if ((v0 | v1 | v2) == 0) continue;
      const long long den = v0 + v1 + v2;  // n . D, of det's sign
      const unsigned long long num = (unsigned long long)(det < 0 ? -det : det);
      const unsigned long long dena = (unsigned long long)(den < 0 ? -den : den);
      const int t = s_tri[q];
      bool take = best < 0;
      if (!take) {
        // num / dena < bnum / bden, exactly: both products below 2^122
        const unsigned long long h1 = __umul64hi(num, bden), l1 = num * bden;
        const unsigned long long h2 = __umul64hi(bnum, dena), l2 = bnum * dena;
        take = h1 < h2 || (h1 == h2 && (l1 < l2 || (l1 == l2 && t < best)));
      }
      if (take) {
        best = t;
        bnum = num;
        bden = dena;
        bflip = den > 0;  // the snapped normal faces away from the eye
      }
    }
  }
  if (px >= A.W || py >= A.H) return;
  const size_t p = (size_t)py * A.W + px;
  if (A.mask) A.mask[p] = best >= 0 ? 1 : 0;
  if (A.tri) A.tri[p] = best;
  float P[3] = {0.0f, 0.0f, 0.0f}, N[3] = {0.0f, 0.0f, 0.0f}, C[3] = {0.0f, 0.0f, 0.0f};
  if (best >= 0) {
    const float t = __fdiv_rn(__ull2float_rn(bnum), __ull2float_rn(bden));
#pragma unroll
    for (int a = 0; a < 3; ++a)
      P[a] = __fadd_rn(A.org[a], __fdiv_rn(fmaf(t, (float)D[a], (float)A.O[a]), A.s));
    const int i0 = __ldg(A.idx + 3 * best), i1 = __ldg(A.idx + 3 * best + 1),
              i2 = __ldg(A.idx + 3 * best + 2);
    float e[3], g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float v0 = __ldg(A.vert + 3 * i0 + a);
      e[a] = __ldg(A.vert + 3 * i1 + a) - v0;
      g[a] = __ldg(A.vert + 3 * i2 + a) - v0;
    }
    const float n0 = diff_prod(e[1], g[2], e[2], g[1]);
    const float n1 = diff_prod(e[2], g[0], e[0], g[2]);
    const float n2 = diff_prod(e[0], g[1], e[1], g[0]);
    const float len = sqrtf(n0 * n0 + n1 * n1 + n2 * n2);
    if (len > 0.0f) {
      const float sc = (bflip ? -1.0f : 1.0f) / len;
      N[0] = n0 * sc;
      N[1] = n1 * sc;
      N[2] = n2 * sc;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) C[a] = __ldg(A.col + 3 * best + a);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    A.pos[3 * p + a] = P[a];
    A.nrm[3 * p + a] = N[a];
    if (A.alb) A.alb[3 * p + a] = C[a];
  }
}

int tiles_x_of(int W) { return (W + kGbTile - 1) / kGbTile; }
int tiles_y_of(int H) { return (H + kGbTile - 1) / kGbTile; }

}  // namespace

size_t gbuffer_fixed_bytes(int W, int H, int nt) {
  const uint64_t T = (uint64_t)tiles_x_of(W) * tiles_y_of(H);
  return (size_t)(kHeaderBytes + align256((T + 1) * 4) + align256(T * 4) +
                  align256((uint64_t)nt * sizeof(TriRec)));
}

cudaError_t launch_gbuffer(const vct_mesh &m, const vct_camera &cam, float *position,
                           float *normal, float *albedo, uint8_t *mask, int32_t *triangle,
                           void *ws, size_t ws_bytes, int sms, cudaStream_t s) {
  GbArgs A{};
  A.vert = m.vertices;
  A.idx = m.indices;
  A.col = m.colors;
  A.nv = m.n_vertices;
  A.nt = m.n_triangles;
  A.W = cam.width;
  A.H = cam.height;
  A.tiles_x = tiles_x_of(A.W);
  A.tiles_y = tiles_y_of(A.H);
  A.s = (float)((double)kFrameUnits / (double)cam.frame_size);
  A.tx = (float)((double)cam.tan_half_fov * (double)A.W / (double)A.H);
  A.ty = cam.tan_half_fov;
  A.gx = (float)((double)A.tx * (1.0 + 4.0 / A.W));
  A.gy = (float)((double)A.ty * (1.0 + 4.0 / A.H));
  A.kx = (float)(0.5 * A.W / (double)A.tx);
  A.ky = (float)(0.5 * A.H / (double)A.ty);
  for (int a = 0; a < 3; ++a) {
    A.org[a] = cam.frame_origin[a];
    A.f[a] = cam.forward[a];
    A.r[a] = cam.right[a];
    A.u[a] = cam.up[a];
    frame_snap(cam.eye[a], A.org[a], A.s, &A.O[a]);  // checked by the caller
  }
  // inverse of the basis matrix [right up forward] (columns), by cofactors
  const double M[3][3] = {{cam.right[0], cam.up[0], cam.forward[0]},
                          {cam.right[1], cam.up[1], cam.forward[1]},
                          {cam.right[2], cam.up[2], cam.forward[2]}};
  const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                     M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                     M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const int j1 = (j + 1) % 3, j2 = (j + 2) % 3, i1 = (i + 1) % 3, i2 = (i + 2) % 3;
      // inverse[i][j] = cofactor[j][i] / det
      A.inv[i][j] = (float)((M[j1][i1] * M[j2][i2] - M[j1][i2] * M[j2][i1]) / det);
    }
  const uint64_t T = (uint64_t)A.tiles_x * A.tiles_y;
  uint8_t *w = static_cast<uint8_t *>(ws);
  uint64_t o = kHeaderBytes;
  A.st = reinterpret_cast<vct_gbuffer_stats *>(w);
  A.off = reinterpret_cast<uint32_t *>(w + o);
  o += align256((T + 1) * 4);
  A.cursor = reinterpret_cast<uint32_t *>(w + o);
  o += align256(T * 4);
  A.rec = reinterpret_cast<TriRec *>(w + o);
  o += align256((uint64_t)A.nt * sizeof(TriRec));
  A.pairs = reinterpret_cast<uint32_t *>(w + o);
  A.cap = (uint32_t)std::min<uint64_t>((ws_bytes - o) / 4, 1ull << 31);
  A.pos = position;
  A.nrm = normal;
  A.alb = albedo;
  A.mask = mask;
  A.tri = triangle;
  cudaError_t e = cudaMemsetAsync(ws, 0, (size_t)(kHeaderBytes + align256((T + 1) * 4) + T * 4), s);
  if (e != cudaSuccess) return e;
  const long long need = ((long long)A.nt + kSetupThreads - 1) / kSetupThreads;
  const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)sms * 8));
  if (A.nt > 0) {
    gb_setup_kernel<<<grid, kSetupThreads, 0, s>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  gb_scan_kernel<<<1, 1024, 0, s>>>(A);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (A.nt > 0) {
    gb_fill_kernel<<<grid, kSetupThreads, 0, s>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  gb_raster_kernel<<<(unsigned)T, kRasterThreads, 0, s>>>(A);
  return cudaGetLastError();
}

VCT_OOB_ACCESSOR(oob_flags_gbuffer)

}  // namespace vct
