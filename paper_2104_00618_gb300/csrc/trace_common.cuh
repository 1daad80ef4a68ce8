// Device code shared by the forward and adjoint cone-trace kernels.
#pragma once

#include "vct_internal.cuh"

namespace vct {

template <int DT> struct TexOf;
template <> struct TexOf<VCT_F32> { using T = float4; };
template <> struct TexOf<VCT_F16> { using T = uint2; };

enum ConeKind { kDiffuse = 0, kSpecular = 1, kOcclusion = 2 };

// Apex of a pixel's cones split into an integer voxel and a small float
// remainder, so that sample coordinates keep full float32 precision relative
// to the apex (level-0 voxel units).
struct Apex {
  int Xi[3];
  float Of[3];
};

// Per-pixel set-up (Ch. 4.2: cone apex on the surface, offset along the
// normal; Ch. 6.2: an offset of a voxel avoids self-collision).
__device__ __forceinline__ void make_apex(const DevPyr &P, const float x[3], const float n[3],
                                          float normal_offset, Apex &A) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double X = ((double)x[a] - P.origin[a]) * P.scale;
    const double fl = floor(X);
    A.Xi[a] = (int)fl;
    A.Of[a] = (float)((X - fl) + (double)normal_offset * (double)n[a]);
  }
}

// Tangent frame: T = normalize(a x n), B = n x T, a = x-axis unless n is
// close to it.
__device__ __forceinline__ void tangent_frame(const float n[3], float T[3], float B[3]) {
  const float ax = fabsf(n[0]) < 0.9f ? 1.0f : 0.0f;
  const float ay = 1.0f - ax;
  float t0 = ay * n[2];
  float t1 = -ax * n[2];
  float t2 = ax * n[1] - ay * n[0];
  const float inv = 1.0f / sqrtf(t0 * t0 + t1 * t1 + t2 * t2);
  T[0] = t0 * inv;
  T[1] = t1 * inv;
  T[2] = t2 * inv;
  B[0] = n[1] * T[2] - n[2] * T[1];
  B[1] = n[2] * T[0] - n[0] * T[2];
  B[2] = n[0] * T[1] - n[1] * T[0];
}

// Reflection of the view ray about the normal, in FP64 (narrow cones are
// sensitive to their axis).
__device__ __forceinline__ void reflect_dir(const float x[3], const float cam[3],
                                            const float n[3], float R[3]) {
  double v[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) v[a] = (double)x[a] - (double)cam[a];
  const double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) v[a] /= len;
  const double vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) R[a] = (float)(v[a] - 2.0 * vn * (double)n[a]);
}

// Step k of a cone: T = t / h0 = T0 * 2^(k l2r) and the mip level
// lam = log2(d / h0) = lam0 + k l2r (Ch. 4.3.2 step rule in closed form).
__device__ __forceinline__ void step_at(const ConeConst &cc, float T0, int k, float &T,
                                        float &lam) {
  const float kf = (float)k;
  const float p = kf * cc.l2r_hi;
  float q = fmaf(kf, cc.l2r_hi, -p);
  q = fmaf(kf, cc.l2r_lo, q);
  const float e = floorf(p);
  const float phi = (p - e) + q;
  T = T0 * exp2f(phi) * __int_as_float(((int)e + 127) << 23);
  lam = (cc.lam0_hi + p) + (q + cc.lam0_lo);
}

// One level of the quadrilinear lookup: the 2x2x2 stencil around the sample.
struct LevelStencil {
  uint32_t sx[2], sy[2], sz[2];  // spread Morton bits of the two corners per axis
  float wx[2], wyz[4];           // x weights (times the level weight), y*z weights
  uint32_t valid;  // bit c set if corner c = dx | dy<<1 | dz<<2 is inside the level
};

__device__ __forceinline__ void level_stencil(int l, int Nl, float lw, const Apex &A,
                                              const float F[3], LevelStencil &s) {
  const float sc = __int_as_float((127 - l) << 23);  // 2^-l
  const int mask = (1 << l) - 1;
  int b[3];
  float fr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ri = A.Xi[a] & mask;
    const int qi = A.Xi[a] >> l;
    // u = (Xi + F) / 2^l - 1/2, formed from small numbers only
    const float v = fmaf(F[a], sc, fmaf((float)ri, sc, -0.5f));
    const float fl = floorf(v);
    fr[a] = v - fl;
    b[a] = qi + (int)fl;
  }
  s.wx[0] = lw * (1.0f - fr[0]);
  s.wx[1] = lw * fr[0];
  const float wy0 = 1.0f - fr[1], wz0 = 1.0f - fr[2];
  s.wyz[0] = wy0 * wz0;
  s.wyz[1] = fr[1] * wz0;
  s.wyz[2] = wy0 * fr[2];
  s.wyz[3] = fr[1] * fr[2];
  const uint32_t x0 = spread3((uint32_t)b[0]);
  const uint32_t y0 = spread3((uint32_t)b[1]);
  const uint32_t z0 = spread3((uint32_t)b[2]);
  s.sx[0] = x0;
  s.sx[1] = spread3_inc(x0);
  s.sy[0] = y0 << 1;
  s.sy[1] = spread3_inc(y0) << 1;
  s.sz[0] = z0 << 2;
  s.sz[1] = spread3_inc(z0) << 2;
  // Interior stencils (the common case) need no per-corner test.
  const uint32_t lim = (uint32_t)Nl - 1u;
  if ((uint32_t)b[0] < lim && (uint32_t)b[1] < lim && (uint32_t)b[2] < lim) {
    s.valid = 0xffu;
    return;
  }
  const uint32_t vx = ((uint32_t)b[0] < (uint32_t)Nl ? 1u : 0u) |
                      ((uint32_t)(b[0] + 1) < (uint32_t)Nl ? 2u : 0u);
  const uint32_t vy = ((uint32_t)b[1] < (uint32_t)Nl ? 1u : 0u) |
                      ((uint32_t)(b[1] + 1) < (uint32_t)Nl ? 2u : 0u);
  const uint32_t vz = ((uint32_t)b[2] < (uint32_t)Nl ? 1u : 0u) |
                      ((uint32_t)(b[2] + 1) < (uint32_t)Nl ? 2u : 0u);
  uint32_t valid = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const bool ok = ((vx >> (c & 1)) & 1u) && ((vy >> ((c >> 1) & 1)) & 1u) &&
                    ((vz >> (c >> 2)) & 1u);
    valid |= ok ? (1u << c) : 0u;
  }
  s.valid = valid;
}

__device__ __forceinline__ uint32_t corner_index(const LevelStencil &s, int c) {
  return s.sx[c & 1] | s.sy[(c >> 1) & 1] | s.sz[c >> 2];
}
// Weight of corner c (level weight included).
__device__ __forceinline__ float corner_weight(const LevelStencil &s, int c) {
  return s.wx[c & 1] * s.wyz[c >> 1];
}

// Adds one level's weighted corners to acc = (r, g, b, a) and to `om`, the
// interpolated transparency sum_c w_c (1 - a_c), formed corner by corner
// (one rounding each) so that it is exactly 0 inside opaque regions and keeps
// its relative precision when the sample is nearly opaque.  Corners outside
// the grid are empty: they add w_c to `om` and nothing to acc.
template <int DT>
__device__ __forceinline__ void accumulate_level(const uint8_t *lvl, const LevelStencil &s,
                                                 float4 &acc, float &om) {
  using T = typename TexOf<DT>::T;
  const T *base = reinterpret_cast<const T *>(lvl);
  float4 v[8];
  if (s.valid == 0xffu) {
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = ld_texel(base + corner_index(s, c));
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      v[c] = make_float4(0.f, 0.f, 0.f, 0.f);
      if ((s.valid >> c) & 1u) v[c] = ld_texel(base + corner_index(s, c));
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float w = corner_weight(s, c);
    acc.x = fmaf(w, v[c].x, acc.x);
    acc.y = fmaf(w, v[c].y, acc.y);
    acc.z = fmaf(w, v[c].z, acc.z);
    acc.w = fmaf(w, v[c].w, acc.w);
    om += fmaf(-w, v[c].w, w);
  }
}

// Level choice of Ch. 4.5 with the quadrilinear blend of Ch. 4.3.3.
struct LodPick {
  int l0, l1;
  float f;  // weight of l1
};
__device__ __forceinline__ LodPick pick_levels(float lam, int levels) {
  LodPick r;
  const float lc = fminf(fmaxf(lam, 0.0f), (float)(levels - 1));
  r.l0 = (int)lc;
  r.f = lc - (float)r.l0;
  r.l1 = min(r.l0 + 1, levels - 1);
  return r;
}

// 1 - a_s: directly from a_s while the sample is at most half opaque (exact 1
// for empty space), from the per-corner transparency sum otherwise (exact 0
// for opaque space, full relative precision when nearly opaque).
__device__ __forceinline__ float select_transparency(float a, float om_sum) {
  return a <= 0.5f ? 1.0f - a : om_sum;
}

// The full sample S(p, lambda) at apex-relative voxel coordinates F;
// `om` receives the sample's transparency 1 - a_s.
template <int DT>
__device__ __forceinline__ float4 sample(const DevPyr &P, const Apex &A, const float F[3],
                                         float lam, float &om) {
  const LodPick lp = pick_levels(lam, P.levels);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  om = 0.f;
  LevelStencil s;
  level_stencil(lp.l0, P.n >> lp.l0, 1.0f - lp.f, A, F, s);
  accumulate_level<DT>(P.lvl[lp.l0], s, acc, om);
  if (lp.f > 0.0f) {
    level_stencil(lp.l1, P.n >> lp.l1, lp.f, A, F, s);
    accumulate_level<DT>(P.lvl[lp.l1], s, acc, om);
  }
  om = select_transparency(acc.w, om);
  return acc;
}

// Per-warp work queue: lane 0 takes the next item, the warp shares it.
__device__ __forceinline__ int next_item(unsigned *queue) {
  int item = 0;
  if ((threadIdx.x & 31) == 0) item = (int)atomicAdd(queue, 1u);
  return __shfl_sync(0xffffffffu, item, 0);
}

// The i-th cone of a pixel in the order [specular?, occlusion?, diffuse...].
struct ConeSel {
  int kind, diffuse_index;
};
__device__ __forceinline__ ConeSel select_cone(int c, int spec, int occ) {
  ConeSel s;
  if (spec && c == 0) {
    s.kind = kSpecular;
    s.diffuse_index = -1;
  } else if (occ && c == spec) {
    s.kind = kOcclusion;
    s.diffuse_index = -1;
  } else {
    s.kind = kDiffuse;
    s.diffuse_index = c - spec - occ;
  }
  return s;
}

// Specular aperture from roughness, and its march constants (FP64).
__device__ __forceinline__ ConeConst spec_const(const DevPyr &P, double gmin, double gmax,
                                                double rmin, double beta, double t0_vox,
                                                const float *rough, int p) {
  if (rough == nullptr) return P.spec_fixed;
  double f = ((double)rough[p] - rmin) / (1.0 - rmin);
  f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
  const double g = gmin + f * (gmax - gmin);
  return cone_const(g, beta, t0_vox, P.tmax_vox);
}

}  // namespace vct
