// Device code shared by the forward and adjoint cone-trace kernels.
//
// The adjoint recomputes the forward's samples, and with the forward's
// per-cone state (sample count, transmittance before the last sample) it
// relies on recomputing them bit for bit in another kernel.  Every value a
// sample depends on is therefore written with explicit roundings (fmaf,
// __fmul_rn, __fadd_rn, ...), never as a multiply followed by an add that
// the compiler may or may not contract into an fma depending on the code
// around it.
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
// normal; Ch. 6.2: an offset of a voxel avoids self-collision).  The grid
// coordinate X = (x - origin) * scale is split into floor(X) and a float
// remainder without double precision: x - origin exactly as s + e (TwoSum),
// s * scale_hi exactly as p + pe (one fma), and the small terms s * scale_lo
// and e * scale_hi added to the remainder p - floor(p), which is exact.
__device__ __forceinline__ void make_apex(const DevPyr &P, const float x[3], const float n[3],
                                          float normal_offset, Apex &A) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float o = P.origin_f[a];
    const float sd = x[a] - o;
    const float bb = sd - x[a];
    const float e = (x[a] - (sd - bb)) - (o + bb);  // x - o = sd + e exactly
    const float p = __fmul_rn(sd, P.scale_hi);      // rounded product, never contracted
    const float pe = fmaf(sd, P.scale_hi, -p);      // sd * scale_hi = p + pe exactly
    const float fl = floorf(p);
    A.Xi[a] = (int)fl;
    A.Of[a] = __fadd_rn(__fadd_rn(__fsub_rn(p, fl),
                                  __fadd_rn(pe, fmaf(sd, P.scale_lo, __fmul_rn(e, P.scale_hi)))),
                        __fmul_rn(normal_offset, n[a]));
  }
}

// Tangent frame: T = normalize(a x n), B = n x T, a = x-axis unless n is
// close to it.
__device__ __forceinline__ void tangent_frame(const float n[3], float T[3], float B[3]) {
  // a x n is (0, -n_z, n_y) for a = x and (n_z, 0, -n_x) for a = y
  const bool ax = fabsf(n[0]) < 0.9f;
  const float t0 = ax ? 0.0f : n[2];
  const float t1 = ax ? -n[2] : 0.0f;
  const float t2 = ax ? n[1] : -n[0];
  const float inv = 1.0f / sqrtf(fmaf(t0, t0, fmaf(t1, t1, __fmul_rn(t2, t2))));
  T[0] = __fmul_rn(t0, inv);
  T[1] = __fmul_rn(t1, inv);
  T[2] = __fmul_rn(t2, inv);
  B[0] = __fsub_rn(__fmul_rn(n[1], T[2]), __fmul_rn(n[2], T[1]));
  B[1] = __fsub_rn(__fmul_rn(n[2], T[0]), __fmul_rn(n[0], T[2]));
  B[2] = __fsub_rn(__fmul_rn(n[0], T[1]), __fmul_rn(n[1], T[0]));
}

// Reflection of the view ray about the normal.
__device__ __forceinline__ void reflect_dir(const float x[3], const float cam[3],
                                            const float n[3], float R[3]) {
  float v[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) v[a] = x[a] - cam[a];
  const float len = sqrtf(fmaf(v[0], v[0], fmaf(v[1], v[1], __fmul_rn(v[2], v[2]))));
#pragma unroll
  for (int a = 0; a < 3; ++a) v[a] = v[a] / len;
  const float vn = fmaf(v[0], n[0], fmaf(v[1], n[1], __fmul_rn(v[2], n[2])));
#pragma unroll
  for (int a = 0; a < 3; ++a) R[a] = fmaf(-2.0f * vn, n[a], v[a]);
}

// floor(v) of |v| < 2^22 as (float, int): v + 1.5 * 2^23 rounded down keeps
// floor(v) in the low mantissa bits (no float-to-int conversion needed).
constexpr float kFloorMagic = 12582912.0f;  // 1.5 * 2^23, bits 0x4B400000
__device__ __forceinline__ float floor_split(float v, int &iv) {
  const float t = __fadd_rd(v, kFloorMagic);
  iv = __float_as_int(t) - 0x4B400000;
  return t - kFloorMagic;
}

// Step k of a cone: T = t / h0 = T0 * 2^(k l2r) and the mip level
// lam = log2(d / h0) = lam0 + k l2r (Ch. 4.3.2 step rule in closed form).
__device__ __forceinline__ void step_at(const ConeConst &cc, float T0, int k, float &T,
                                        float &lam) {
  const float kf = (float)k;
  const float p = __fmul_rn(kf, cc.l2r_hi);
  float q = fmaf(kf, cc.l2r_hi, -p);
  q = fmaf(kf, cc.l2r_lo, q);
  int ie;
  const float e = floor_split(p, ie);
  const float phi = __fadd_rn(__fsub_rn(p, e), q);
  T = __fmul_rn(__fmul_rn(T0, exp2f(phi)), __int_as_float((ie + 127) << 23));
  lam = __fadd_rn(__fadd_rn(cc.lam0_hi, p), __fadd_rn(q, cc.lam0_lo));
}

// ---------------------------------------------------------------------------
// packed float32 pairs (Blackwell f32x2 arithmetic): RGBA is carried as the
// two pairs (r, g) and (b, a), halving the instruction count of the lerps.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 f2_pack(float a, float b) {
  f32x2 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ float2 f2_unpack(f32x2 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// a + b rounded towards minus infinity, both lanes
__device__ __forceinline__ f32x2 f2_add_rm(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// a + t (b - a), both lanes
__device__ __forceinline__ f32x2 f2_lerp(f32x2 a, f32x2 b, f32x2 t) {
  return f2_fma(t, f2_sub(b, a), a);
}

__device__ __forceinline__ void ld_texel2(const float4 *p, f32x2 &rg, f32x2 &ba) {
  asm("ld.global.nc.v2.u64 {%0, %1}, [%2];" : "=l"(rg), "=l"(ba) : "l"(p));
}
__device__ __forceinline__ void ld_texel2(const uint2 *p, f32x2 &rg, f32x2 &ba) {
  const uint2 u = __ldg(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
  rg = f2_pack(a.x, a.y);
  ba = f2_pack(b.x, b.y);
}

// ---------------------------------------------------------------------------
// one level of the quadrilinear lookup: the 2x2x2 cell around the sample
// ---------------------------------------------------------------------------
struct LevelStencil {
  uint32_t sx[2], sy[2], sz[2];  // spread Morton bits of the two corners per axis
  float fr[3];                   // position inside the cell, per axis
  uint32_t valid;  // bit c set if corner c = dx | dy<<1 | dz<<2 is inside the level
};

// lut: three tables of 1024 entries (shared memory, fill_spread_lut): the
// Morton bits of x, y and z (spread3(i), << 1, << 2), each with those of i + 1.
// kPacked: x and y as float32 pairs (the same operations per element, so
// the same bits): the isotropic sampler of both passes; the anisotropic
// sampler (measured slower packed) uses the scalar form.
template <bool kPacked = true>
__device__ __forceinline__ void level_stencil(int l, int Nl, const Apex &A, const float F[3],
                                              const uint2 *lut, LevelStencil &s) {
  const float sc = __int_as_float((127 - l) << 23);  // 2^-l
  const int mask = (1 << l) - 1;
  int b[3];
  // u = (Xi + F) / 2^l - 1/2, formed from small numbers only; floor(u) by
  // the magic-number add of floor_split.
  if constexpr (kPacked) {
    const f32x2 sc2 = f2_pack(sc, sc);
    const f32x2 c = f2_fma(f2_pack((float)(A.Xi[0] & mask), (float)(A.Xi[1] & mask)), sc2,
                           f2_pack(-0.5f, -0.5f));
    const f32x2 v = f2_fma(f2_pack(F[0], F[1]), sc2, c);
    const f32x2 magic = f2_pack(kFloorMagic, kFloorMagic);
    const f32x2 t = f2_add_rm(v, magic);
    const float2 fr = f2_unpack(f2_sub(v, f2_sub(t, magic)));
    const float2 tt = f2_unpack(t);
    s.fr[0] = fr.x;
    s.fr[1] = fr.y;
    b[0] = (A.Xi[0] >> l) + (__float_as_int(tt.x) - 0x4B400000);
    b[1] = (A.Xi[1] >> l) + (__float_as_int(tt.y) - 0x4B400000);
  }
#pragma unroll
  for (int a = kPacked ? 2 : 0; a < 3; ++a) {
    const float v = fmaf(F[a], sc, fmaf((float)(A.Xi[a] & mask), sc, -0.5f));
    int iv;
    const float fl = floor_split(v, iv);
    s.fr[a] = v - fl;
    b[a] = (A.Xi[a] >> l) + iv;
  }
  const uint2 xe = lut[(uint32_t)b[0] & 1023u];
  const uint2 ye = lut[1024u + ((uint32_t)b[1] & 1023u)];
  const uint2 ze = lut[2048u + ((uint32_t)b[2] & 1023u)];
  s.sx[0] = xe.x;
  s.sx[1] = xe.y;
  s.sy[0] = ye.x;
  s.sy[1] = ye.y;
  s.sz[0] = ze.x;
  s.sz[1] = ze.y;
  // Interior cells (the common case) need no per-corner test.
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

// Address of the texel with Morton code `code` in a bricked level: its
// brick's pool slot (slot 0, the zero brick, for an empty brick).
template <typename T>
__device__ __forceinline__ const T *brick_texel(const uint32_t *tbl, const T *pool,
                                                uint32_t code) {
  const uint32_t slot = __ldg(tbl + (code >> kBrickShift));
  return pool + (((size_t)slot << kBrickShift) | (code & 511u));
}

// Bounds checks of the lookups (debug-bounds builds; always true otherwise):
// a valid corner's Morton code lies inside its level, a bricked level's
// slot inside the pool.
__device__ __forceinline__ bool texel_ok(const DevPyr &P, int l, uint32_t code) {
  return in_bounds(code, level_texels(P.n, l), kOobTexel);
}
__device__ __forceinline__ bool slot_ok(const DevPyr &P, const uint32_t *tbl, uint32_t code) {
#ifdef VCT_DEBUG_BOUNDS
  return in_bounds(__ldg(tbl + (code >> kBrickShift)), P.pool_slots, kOobBrick);
#else
  return true;
#endif
}

// Trilinear lookup of level l as seven packed lerps (x, then y, then z);
// corners outside the grid read as zero.  BR: the pyramid may have bricked
// levels (VCT_LAYOUT_BRICKS).
template <int DT, bool BR = false>
__device__ __forceinline__ void trilerp(const DevPyr &P, int l, const LevelStencil &s,
                                        f32x2 &rg, f32x2 &ba) {
  using T = typename TexOf<DT>::T;
  const T *base = reinterpret_cast<const T *>(P.lvl[l]);
  f32x2 c_rg[8], c_ba[8];
  if (BR && ((P.bricked >> l) & 1u)) {
    const uint32_t *tbl = reinterpret_cast<const uint32_t *>(P.lvl[l]);
    const T *pool = reinterpret_cast<const T *>(P.pool);
    // Two corners per axis share a brick unless the cell straddles a brick
    // face; when all eight do (7 cells in 8 per axis), one slot serves all.
    const uint32_t cross = (s.sx[0] ^ s.sx[1]) | (s.sy[0] ^ s.sy[1]) | (s.sz[0] ^ s.sz[1]);
    if (s.valid == 0xffu && (cross >> kBrickShift) == 0u) {
      const uint32_t c0 = corner_index(s, 0);
      const bool ok = texel_ok(P, l, c0) && slot_ok(P, tbl, c0);
      const T *brick = pool + ((size_t)(ok ? __ldg(tbl + (c0 >> kBrickShift)) : 0u) << kBrickShift);
#pragma unroll
      for (int c = 0; c < 8; ++c) ld_texel2(brick + (corner_index(s, c) & 511u), c_rg[c], c_ba[c]);
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        c_rg[c] = 0ull;
        c_ba[c] = 0ull;
        const uint32_t code = corner_index(s, c);
        if (((s.valid >> c) & 1u) && texel_ok(P, l, code) && slot_ok(P, tbl, code))
          ld_texel2(brick_texel(tbl, pool, code), c_rg[c], c_ba[c]);
      }
    }
  } else if (s.valid == 0xffu) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const uint32_t code = corner_index(s, c);
#ifdef VCT_DEBUG_BOUNDS
      c_rg[c] = 0ull;
      c_ba[c] = 0ull;
      if (texel_ok(P, l, code))
#endif
        ld_texel2(base + code, c_rg[c], c_ba[c]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      c_rg[c] = 0ull;
      c_ba[c] = 0ull;
      const uint32_t code = corner_index(s, c);
      if (((s.valid >> c) & 1u) && texel_ok(P, l, code)) ld_texel2(base + code, c_rg[c], c_ba[c]);
    }
  }
  const f32x2 tx = f2_pack(s.fr[0], s.fr[0]);
  const f32x2 ty = f2_pack(s.fr[1], s.fr[1]);
  const f32x2 tz = f2_pack(s.fr[2], s.fr[2]);
  f32x2 e_rg[4], e_ba[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    e_rg[i] = f2_lerp(c_rg[2 * i], c_rg[2 * i + 1], tx);
    e_ba[i] = f2_lerp(c_ba[2 * i], c_ba[2 * i + 1], tx);
  }
  const f32x2 g0_rg = f2_lerp(e_rg[0], e_rg[1], ty), g1_rg = f2_lerp(e_rg[2], e_rg[3], ty);
  const f32x2 g0_ba = f2_lerp(e_ba[0], e_ba[1], ty), g1_ba = f2_lerp(e_ba[2], e_ba[3], ty);
  rg = f2_lerp(g0_rg, g1_rg, tz);
  ba = f2_lerp(g0_ba, g1_ba, tz);
}

// Level choice of Ch. 4.5 with the quadrilinear blend of Ch. 4.3.3.
struct LodPick {
  int l0, l1;
  float f;  // weight of l1
};
__device__ __forceinline__ LodPick pick_levels(float lam, int levels) {
  LodPick r;
  const float lc = fminf(fmaxf(lam, 0.0f), (float)(levels - 1));
  r.f = lc - floor_split(lc, r.l0);
  r.l1 = min(r.l0 + 1, levels - 1);
  return r;
}

// 1 - a_s, clamped at zero: with texel opacities in [0, 1] the exact value is
// >= 0, and rounding can put an all-opaque sample a hair above one.
__device__ __forceinline__ float transparency(float a) { return fmaxf(1.0f - a, 0.0f); }

// The full sample S(p, lambda) at apex-relative voxel coordinates F (levels
// floor(lambda) and floor(lambda)+1 blended linearly); `om` receives 1 - a_s.
// When `st` is non-null the two stencils are kept for the adjoint.
template <int DT, bool BR = false, bool kPacked = true>
__device__ __forceinline__ float4 sample_at(const DevPyr &P, const Apex &A, const float F[3],
                                            const LodPick &lp, const uint2 *lut, float &om,
                                            LevelStencil *st = nullptr) {
  LevelStencil s;
  f32x2 rg, ba;
  level_stencil<kPacked>(lp.l0, P.n >> lp.l0, A, F, lut, s);
  trilerp<DT, BR>(P, lp.l0, s, rg, ba);
  if (st) st[0] = s;
  if (lp.f > 0.0f) {
    level_stencil<kPacked>(lp.l1, P.n >> lp.l1, A, F, lut, s);
    f32x2 rg1, ba1;
    trilerp<DT, BR>(P, lp.l1, s, rg1, ba1);
    const f32x2 tf = f2_pack(lp.f, lp.f);
    rg = f2_lerp(rg, rg1, tf);
    ba = f2_lerp(ba, ba1, tf);
    if (st) st[1] = s;
  }
  const float2 v0 = f2_unpack(rg), v1 = f2_unpack(ba);
  om = transparency(v1.y);
  return make_float4(v0.x, v0.y, v1.x, v1.y);
}
template <int DT, bool BR = false, bool kPacked = true>
__device__ __forceinline__ float4 sample(const DevPyr &P, const Apex &A, const float F[3],
                                         float lam, const uint2 *lut, float &om,
                                         LodPick &lp, LevelStencil *st = nullptr) {
  lp = pick_levels(lam, P.levels);
  return sample_at<DT, BR, kPacked>(P, A, F, lp, lut, om, st);
}

// Cone march variants (Ch. 5.4.4): the plain march, the occlusion cone that
// fades its samples near the apex, and the diffuse cone that stops at the
// first sample with opacity above 1/100.
enum MarchMode { kPlain = 0, kOccSmooth = 1, kFirstHit = 2 };

// GLSL smoothstep(0, e1, x).
__device__ __forceinline__ float smoothstep0(float e1, float x) {
  const float u = fminf(fmaxf(x / e1, 0.0f), 1.0f);
  return __fmul_rn(__fmul_rn(u, u), fmaf(-2.0f, u, 3.0f));
}

// Angular-grace specular BRDF (Ch. 5.4.4): (1 - max(0, g - p) / pi)^q with g
// the angle between the cone axis w and the light direction, taken as
// atan2(|w x l|, w . l) (well conditioned at every angle).
__device__ __forceinline__ float spec_grace(const Variants &v, const float w[3]) {
  const float *l = v.light_dir;
  const float cx = fmaf(w[1], l[2], -__fmul_rn(w[2], l[1]));
  const float cy = fmaf(w[2], l[0], -__fmul_rn(w[0], l[2]));
  const float cz = fmaf(w[0], l[1], -__fmul_rn(w[1], l[0]));
  const float d = fmaf(w[0], l[0], fmaf(w[1], l[1], __fmul_rn(w[2], l[2])));
  const float g = atan2f(sqrtf(fmaf(cx, cx, fmaf(cy, cy, __fmul_rn(cz, cz)))), d);
  const float e = fmaxf(g - v.grace, 0.0f);
  return powf(1.0f - e * 0.318309886f, v.falloff);
}

// Direct light of pixel p for the shading epilogue: Phong with one
// directional light (Ch. 3.3), direct = light_color * albedo * lobe with
// lobe = kd max(n.l, 0) + ks max(v.R, 0)^shininess; alb receives the albedo.
__device__ __forceinline__ void shade_direct(const Variants &v, const DevView &V, int p,
                                             float direct[3], float alb[3]) {
  float x[3], n[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    x[a] = V.pos[3 * p + a];
    n[a] = V.nrm[3 * p + a];
    alb[a] = V.albedo ? V.albedo[3 * p + a] : 1.0f;
  }
  const float *l = v.light_dir;
  const float nl = n[0] * l[0] + n[1] * l[1] + n[2] * l[2];
  float R[3], e[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R[a] = fmaf(2.0f * nl, n[a], -l[a]);
    e[a] = V.cam[a] - x[a];
  }
  const float inv = rsqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
  const float wr = (e[0] * R[0] + e[1] * R[1] + e[2] * R[2]) * inv;
  const float lobe = v.kd * fmaxf(nl, 0.0f) + v.ks * powf(fmaxf(wr, 0.0f), v.shininess);
#pragma unroll
  for (int a = 0; a < 3; ++a) direct[a] = v.light_color[a] * alb[a] * lobe;
}

// ---------------------------------------------------------------------------
// anisotropic pyramids (VCT_LAYOUT_ANISO, float32)
// ---------------------------------------------------------------------------
// A level l >= 1 is read as sum_a wt[a] * (volume vol[a] of level l), wt[a]
// = w_a^2 / |w|^2 and vol[a] = 2 a + (w_a < 0) for a cone of axis w.  A
// volume whose weight is below 2^-24 (its share of the unit weight sum is
// below float32 resolution) is not read: axis-aligned cones, whose other
// components are float roundings of cos(90 deg) ~ 1e-17, read one volume.
constexpr float kAnisoSkip = 5.9604645e-08f;  // 2^-24
struct AnisoW {
  float wt[3];
  int vol[3];
};
__device__ __forceinline__ AnisoW aniso_weights(const float w[3]) {
  AnisoW r;
  const float inv = 1.0f / fmaf(w[0], w[0], fmaf(w[1], w[1], __fmul_rn(w[2], w[2])));
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r.wt[a] = __fmul_rn(__fmul_rn(w[a], w[a]), inv);
    r.vol[a] = 2 * a + (w[a] < 0.0f ? 1 : 0);
  }
  return r;
}

// Trilinear lookup (seven packed lerps) in volume `vol` of level l of an
// anisotropic pyramid; corners outside the grid read as zero.
__device__ __forceinline__ void trilerp_vol(const DevPyr &P, int l, int vol, const LevelStencil &s,
                                            f32x2 &rg, f32x2 &ba) {
  const uint64_t texels = level_texels(P.n, l);
  const float4 *base = reinterpret_cast<const float4 *>(P.lvl[l]) + (uint64_t)vol * texels;
  f32x2 c_rg[8], c_ba[8];
  if (s.valid == 0xffu) {  // interior cell: no per-corner test
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const uint32_t code = corner_index(s, c);
#ifdef VCT_DEBUG_BOUNDS
      c_rg[c] = 0ull;
      c_ba[c] = 0ull;
      if (in_bounds(code, texels, kOobTexel))
#endif
        ld_texel2(base + code, c_rg[c], c_ba[c]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      c_rg[c] = 0ull;
      c_ba[c] = 0ull;
      const uint32_t code = corner_index(s, c);
      if (((s.valid >> c) & 1u) && in_bounds(code, texels, kOobTexel))
        ld_texel2(base + code, c_rg[c], c_ba[c]);
    }
  }
  const f32x2 tx = f2_pack(s.fr[0], s.fr[0]);
  const f32x2 ty = f2_pack(s.fr[1], s.fr[1]);
  const f32x2 tz = f2_pack(s.fr[2], s.fr[2]);
  f32x2 e_rg[4], e_ba[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    e_rg[i] = f2_lerp(c_rg[2 * i], c_rg[2 * i + 1], tx);
    e_ba[i] = f2_lerp(c_ba[2 * i], c_ba[2 * i + 1], tx);
  }
  const f32x2 g0_rg = f2_lerp(e_rg[0], e_rg[1], ty), g1_rg = f2_lerp(e_rg[2], e_rg[3], ty);
  const f32x2 g0_ba = f2_lerp(e_ba[0], e_ba[1], ty), g1_ba = f2_lerp(e_ba[2], e_ba[3], ty);
  rg = f2_lerp(g0_rg, g1_rg, tz);
  ba = f2_lerp(g0_ba, g1_ba, tz);
}

// One level of an anisotropic pyramid: level 0 is isotropic, a coarser
// level the direction-weighted sum of three volumes.
__device__ __forceinline__ void aniso_level(const DevPyr &P, int l, const LevelStencil &s,
                                            const AnisoW &aw, f32x2 &rg, f32x2 &ba) {
  if (l == 0) {
    trilerp_vol(P, 0, 0, s, rg, ba);
    return;
  }
  rg = 0ull;
  ba = 0ull;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (aw.wt[a] < kAnisoSkip) continue;
    f32x2 r, b;
    trilerp_vol(P, l, aw.vol[a], s, r, b);
    const f32x2 wt = f2_pack(aw.wt[a], aw.wt[a]);
    rg = f2_fma(wt, r, rg);
    ba = f2_fma(wt, b, ba);
  }
}

// S(p, lambda) of an anisotropic pyramid for travel along the cone axis.
__device__ __forceinline__ float4 sample_aniso_at(const DevPyr &P, const Apex &A,
                                                  const float F[3], const LodPick &lp,
                                                  const uint2 *lut, const AnisoW &aw,
                                                  float &om, LevelStencil *st = nullptr) {
  LevelStencil s;
  f32x2 rg, ba;
  level_stencil<false>(lp.l0, P.n >> lp.l0, A, F, lut, s);
  aniso_level(P, lp.l0, s, aw, rg, ba);
  if (st) st[0] = s;
  if (lp.f > 0.0f) {
    level_stencil<false>(lp.l1, P.n >> lp.l1, A, F, lut, s);
    f32x2 rg1, ba1;
    aniso_level(P, lp.l1, s, aw, rg1, ba1);
    const f32x2 tf = f2_pack(lp.f, lp.f);
    rg = f2_lerp(rg, rg1, tf);
    ba = f2_lerp(ba, ba1, tf);
    if (st) st[1] = s;
  }
  const float2 v0 = f2_unpack(rg), v1 = f2_unpack(ba);
  om = transparency(v1.y);
  return make_float4(v0.x, v0.y, v1.x, v1.y);
}
__device__ __forceinline__ float4 sample_aniso(const DevPyr &P, const Apex &A, const float F[3],
                                               float lam, const uint2 *lut, const AnisoW &aw,
                                               float &om, LodPick &lp,
                                               LevelStencil *st = nullptr) {
  lp = pick_levels(lam, P.levels);
  return sample_aniso_at(P, A, F, lp, lut, aw, om, st);
}

// Step table of the cones whose aperture is a launch constant (diffuse and
// occlusion): per pyramid and kind, entry k = (T, f, l0, l1) of step k as
// step_at and pick_levels give them, for the first kStepTab steps.
constexpr int kStepTab = 64;
__device__ __forceinline__ const float4 *step_table(const float4 *tab, int pyr, int kind_occ) {
  return tab + (size_t)(2 * pyr + kind_occ) * kStepTab;
}
__device__ __forceinline__ void fill_step_table(float4 *tab, const DevPyr *pyrs, int n_pyr,
                                                float T0) {
  for (int i = threadIdx.x; i < n_pyr * 2 * kStepTab; i += blockDim.x) {
    const int k = i % kStepTab;
    const int kind = (i / kStepTab) & 1;
    const DevPyr &P = pyrs[i / (2 * kStepTab)];
    float T, lam;
    step_at(kind ? P.occ : P.diffuse, T0, k, T, lam);
    const LodPick lp = pick_levels(lam, P.levels);
    tab[i] = make_float4(T, lp.f, __int_as_float(lp.l0), __int_as_float(lp.l1));
  }
}

// Fills the Morton spread tables (shared memory, kSpreadLut entries) of a
// CTA: for axis a = i >> 10 and coordinate c = i & 1023 the spread bits of c
// and of c + 1 (10-bit wrap), in place for the axis (shifted left by a).
constexpr int kSpreadLut = 3 * 1024;
__device__ __forceinline__ void fill_spread_lut(uint2 *lut) {
  for (int i = threadIdx.x; i < kSpreadLut; i += blockDim.x) {
    const uint32_t c = (uint32_t)i & 1023u;
    lut[i] = make_uint2(spread3(c) << (i >> 10), spread3((c + 1u) & 1023u) << (i >> 10));
  }
  __syncthreads();
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
// The aperture interpolates linearly in roughness; the step ratio and the
// first level follow from it as in cone_const, in float32 (log1pf, tanf and
// log2f are within two units in the last place, which moves the positions
// of a cone's last steps by less than 1e-6 of their distance).
__device__ __forceinline__ ConeConst spec_const(const DevPyr &P, const SpecSetup &S,
                                                const float *rough, int p) {
  if (rough == nullptr) return P.spec_fixed;
  const float f = fminf(fmaxf((rough[p] - S.rough_min) * S.inv_rough_span, 0.0f), 1.0f);
  const float g = fmaf(f, S.gdelta, S.gmin);
  const float th = tanf(0.5f * g);
  ConeConst c{};
  c.l2r_hi = log1pf(S.two_beta * th) * 1.44269504088896341f;  // / ln 2
  c.lam0_hi = log2f(2.0f * S.t0_vox * th);
  const float e = P.log2_tmax_t0 / c.l2r_hi;
  c.kmax = e >= 0.0f ? (int)fminf(floorf(e) + 1.0f, (float)(kMaxSteps + 1)) : 0;
  return c;
}

}  // namespace vct
