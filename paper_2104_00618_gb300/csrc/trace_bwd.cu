// Adjoint of the cone trace (no counterpart in the thesis: the transpose of
// the Ch. 4.3.2 accumulation and the Ch. 4.5 sampler).  No per-sample state
// is stored: each cone is marched forwards once (same stopping rule as the
// forward kernel: alpha = 1 - T < 1 in float32) to find its length K and its transmittance
// before the last sample, then walked backwards k = K-1 .. 0, recomputing
// every sample.  For samples (c_k, a_k) and T_k = prod_{j<k} (1 - a_j):
//   C = sum_k T_k a_k c_k,  A = 1 - prod_k (1 - a_k)
//   dC/dc_k = T_k a_k,  dC/da_k = T_k (c_k - R_{k+1}),  dA/da_k = T_k Q_{k+1}
// with R_k = a_k c_k + (1 - a_k) R_{k+1}, Q_k = (1 - a_k) Q_{k+1} built during
// the backward walk and T_k = T_{k+1} / (1 - a_k) recovered from the
// product-form T_{K-1} of the forward pass (every a_k with k < K-1 is below
// one, otherwise the march would have stopped at k).  Both passes go
// through the same inlined sample code, so they see bit-identical samples.
// The derivatives are scattered through the quadrilinear weights into a
// float32 gradient pyramid with vector atomics (for an anisotropic pyramid,
// into the directional volumes a sample read, times their weights).
#include <algorithm>

#include "trace_common.cuh"

namespace vct {

namespace {

// Gradient texel of level l (float32 gradient pyramid in global memory).
// Every level is accumulated there with float atomics: measured on the
// learnable 128^3 workload, per-CTA shared-memory copies of the coarse
// levels were slower (their flush and the shared-memory atomics cost more
// than the contention they avoided, the warp reduce-scatter below already
// merging the lanes that share a cell).
__device__ __forceinline__ float *grad_texel(const BwdLaunch &L, int l, uint32_t idx) {
  return reinterpret_cast<float *>(L.gpyr_lvl[l]) + 4 * (size_t)idx;
}

// One contribution in the fixed-point mode: v rounded to a multiple of
// 2^-32, two's complement (integer addition of these is associative).
__device__ __forceinline__ unsigned long long to_fix(float v) {
  return (unsigned long long)__float2ll_rn(v * kFixScale);
}
__device__ __forceinline__ unsigned long long *fix_texel(const BwdLaunch &L, int l, uint32_t idx) {
  return L.gfix_lvl[l] + 4 * (size_t)idx;
}

// The 8 trilinear corner weights of a stencil (fractions fr) times the level
// weight lw, corner c = cx | cy << 1 | cz << 2: products of the per-axis weights.
__device__ __forceinline__ void corner_weights(const float fr[3], float lw, float w[8]) {
  const float wx[2] = {1.0f - fr[0], fr[0]};
  const float wy[2] = {1.0f - fr[1], fr[1]};
  const float wz[2] = {lw * (1.0f - fr[2]), lw * fr[2]};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float wyz = wy[k & 1] * wz[k >> 1];
    w[2 * k] = wx[0] * wyz;
    w[2 * k + 1] = wx[1] * wyz;
  }
}

// Per-lane scatter of one level's 8 corners (lanes in different cells) into
// the gradient texels vbase + code (vbase: the volume's first texel in an
// anisotropic level, else 0; lim: the texels of the gradient level).
__device__ __forceinline__ void scatter_lane(const BwdLaunch &L, int l, uint32_t vbase,
                                             uint32_t lim, const LevelStencil &s, float lw,
                                             const float g[4]) {
  float w[8];
  corner_weights(s.fr, lw, w);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (!((s.valid >> c) & 1u)) continue;
    const uint32_t idx = vbase + corner_index(s, c);
    if (!in_bounds(idx, lim, kOobGrad)) continue;
    if (L.deterministic) {
      if (w[c] == 0.0f) continue;
      unsigned long long *q = fix_texel(L, l, idx);
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) atomicAdd(q + ch, to_fix(w[c] * g[ch]));
    } else {
      atomicAdd(reinterpret_cast<float4 *>(grad_texel(L, l, idx)),
                make_float4(w[c] * g[0], w[c] * g[1], w[c] * g[2], w[c] * g[3]));
    }
  }
}

// Scatter of one level for the whole warp (warp-uniform call).  Lanes are
// grouped by (level, 2x2x2 cell).  A lane whose group has fewer than
// kReduceMin lanes scatters its own corners.  For each larger group the 32 values
// (8 corners x 4 channels) are summed over the group by recursive halving,
// so that lane j ends with the group total of value j, and each lane issues
// one atomic on a distinct address: contending atomics (the same texel from
// many lanes) are what makes a naive scatter slow at the coarse levels.
// Measured on the learnable 128^3 workload (fwd + adjoint): 59.3 / 57.8 /
// 55.4 / 53.7 / 57.1 / 91.2 ms for thresholds 2 / 4 / 8 / 16 / 20 / 32, and
// 544 ms without the reduction.
constexpr int kReduceMin = 16;
// The reproducible mode pays four 64-bit atomics per corner and channel
// group, so there every cell shared by two or more lanes is summed first
// (fwd + adjoint on the same workload: 108.6 ms with 16, 64.7 ms with 2).
constexpr int kReduceMinFix = 2;

// Slot of the key-offset table holding the total (after the per-level offsets).
constexpr int kKeyTotal = VCT_MAX_LEVELS;

template <bool AN>
__device__ __forceinline__ void scatter_warp(const BwdLaunch &L, const uint32_t *code_off,
                                             bool act, int l, uint32_t vbase, uint32_t lim,
                                             const LevelStencil &s, float lw, const float g[4]) {
  const unsigned full = 0xffffffffu;
  act = act && s.valid != 0u;  // a cell wholly outside the level has nothing to scatter
  if (__ballot_sync(full, act) == 0u) return;
  const int lane = threadIdx.x & 31;
  // (level, volume, cell) as one 32-bit key: the cell's Morton code offset by
  // its volume's first texel and by the texels of all finer levels (< 2^31
  // for n <= 1024, anisotropic levels included); lanes with one key share the
  // cell's corners and their validity.  The Morton code names the cell only
  // while its lower corner (corner 0) lies inside the level; a cell with a
  // valid corner but its lower corner outside starts at -1 on some axes (its
  // spread code there is that of 1023, the 10-bit wrap of -1).  Such a cell
  // is keyed by bit 31, the mask of those axes (bits 28-30) and the offset
  // code of the cell moved to 0 on them, which is unique, and below the
  // per-lane keys 0xffffff00 + lane and the inactive key, while every key
  // offset stays below 0x0fffff00 (code_off[kKeyTotal]; n <= 512); above that
  // the lane takes a key of its own and scatters alone.
  uint32_t key = 0xffffffffu;
  if (act) {
    if (s.valid & 1u) {
      key = code_off[l] + vbase + (s.sx[0] | s.sy[0] | s.sz[0]);
    } else if (code_off[kKeyTotal] < 0x0fffff00u) {
      const uint32_t mx = s.sx[0] == kMortonX ? 1u : 0u;
      const uint32_t my = s.sy[0] == (kMortonX << 1) ? 2u : 0u;
      const uint32_t mz = s.sz[0] == (kMortonX << 2) ? 4u : 0u;
      const uint32_t cell = (mx ? s.sx[1] : s.sx[0]) | (my ? s.sy[1] : s.sy[0]) |
                            (mz ? s.sz[1] : s.sz[0]);
      key = 0x80000000u | ((mx | my | mz) << 28) | (code_off[l] + vbase + cell);
    } else {
      key = 0xffffff00u + (uint32_t)lane;
    }
  }
  const unsigned grp = __match_any_sync(full, key);
  const bool big = act && __popc(grp) >= (L.deterministic ? kReduceMinFix : kReduceMin);
  if (act && !big) scatter_lane(L, l, vbase, lim, s, lw, g);
  unsigned pending = __ballot_sync(full, big);
  if (pending == 0u) return;
  // A lane without a sample here holds unset fractions and derivatives: its
  // operands are replaced by zeros once, so that every product below is of
  // finite values and a lane outside a group adds exact zeros (level weight
  // 0).  The weight is selected inside the loop, which also keeps the 32
  // products from being hoisted out of it and held in registers.
  const float fr[3] = {act ? s.fr[0] : 0.0f, act ? s.fr[1] : 0.0f, act ? s.fr[2] : 0.0f};
  const float ga[4] = {act ? g[0] : 0.0f, act ? g[1] : 0.0f, act ? g[2] : 0.0f,
                       act ? g[3] : 0.0f};
  const float lwa = act ? lw : 0.0f;
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const unsigned lgrp = __shfl_sync(full, grp, leader);
    const bool in = (lgrp >> lane) & 1u;
    float v[32];
    {
      float w[8];
      corner_weights(fr, in ? lwa : 0.0f, w);
#pragma unroll
      for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) v[4 * c + ch] = w[c] * ga[ch];
    }
#pragma unroll
    for (int half = 16; half >= 1; half >>= 1) {
      const bool upper = (lane & half) != 0;
#pragma unroll
      for (int i = 0; i < half; ++i) {
        const float send = upper ? v[i] : v[i + half];
        const float keep = upper ? v[i + half] : v[i];
        v[i] = keep + __shfl_xor_sync(full, send, half);
      }
    }
    // Lane j holds the group total of corner j / 4, channel j % 4.  The cell
    // is the leader's: take its spread coordinates (a shuffle returns the
    // source lane's value, so per-corner choices are made afterwards).
    const int c = lane >> 2, ch = lane & 3;
    const int ll = __shfl_sync(full, l, leader);  // this lane's own level may differ
    uint32_t lvbase = 0u, llim;
    if constexpr (AN) {
      lvbase = __shfl_sync(full, vbase, leader);
      llim = __shfl_sync(full, lim, leader);
    } else {
      llim = (uint32_t)level_texels(L.pyr.n, ll);
    }
    const uint32_t lvalid = __shfl_sync(full, s.valid, leader);
    const uint32_t sx0 = __shfl_sync(full, s.sx[0], leader), sx1 = __shfl_sync(full, s.sx[1], leader);
    const uint32_t sy0 = __shfl_sync(full, s.sy[0], leader), sy1 = __shfl_sync(full, s.sy[1], leader);
    const uint32_t sz0 = __shfl_sync(full, s.sz[0], leader), sz1 = __shfl_sync(full, s.sz[1], leader);
    const uint32_t idx =
        lvbase + (((c & 1) ? sx1 : sx0) | (((c >> 1) & 1) ? sy1 : sy0) | ((c >> 2) ? sz1 : sz0));
    if (((lvalid >> c) & 1u) && v[0] != 0.0f && in_bounds(idx, llim, kOobGrad)) {
      if (L.deterministic)
        atomicAdd(fix_texel(L, ll, idx) + ch, to_fix(v[0]));
      else
        atomicAdd(grad_texel(L, ll, idx) + ch, v[0]);
    }
    pending &= ~lgrp;
  }
}

// Scatter of one level of the quadrilinear stencil (level weight lw).  In an
// anisotropic pyramid a level >= 1 was read from up to three volumes weighted
// by w_a^2: each receives the derivatives times its weight, the volumes the
// forward skipped none (warp-uniform trip count).
template <bool AN>
__device__ __forceinline__ void scatter_level(const BwdLaunch &L, const uint32_t *code_off,
                                              bool act, int l, const LevelStencil &s, float lw,
                                              const float g[4], const AnisoW &aw) {
  const uint32_t tex = (uint32_t)level_texels(L.pyr.n, l);
  if constexpr (!AN) {
    scatter_warp<false>(L, code_off, act, l, 0u, tex, s, lw, g);
  } else {
    const bool dir = l >= 1;
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
      const bool on = act && (dir ? aw.wt[a] >= kAnisoSkip : a == 0);
      if (__any_sync(0xffffffffu, on))
        scatter_warp<true>(L, code_off, on, l, dir ? (uint32_t)aw.vol[a] * tex : 0u,
                     dir ? 6u * tex : tex, s, dir ? lw * aw.wt[a] : lw, g);
    }
  }
}

// Adjoint of one cone for every lane of the warp (warp-uniform call; lanes
// with active == false take no samples).  With `state` (warp-uniform: null
// or not for all lanes) the cone's length and transmittance before its last
// sample come from the forward trace and the forward pass is skipped.
// `mode` (per lane) is the cone's march variant (Ch. 5.4.4), recomputed
// exactly as the forward marched it: the occlusion fade scales the sampled
// opacity by a factor of t alone (the texel opacity receives dL/da times
// it); a first-hit diffuse cone returns its hit sample's colour, so only that
// sample's colour channels receive gradient.  With premultiplied colour
// (C = sum T_k c_k): dC/dc_k = T_k, dC/da_k = -T_k R'_{k+1}, R'_k = c_k +
// (1 - a_k) R'_{k+1}.
template <int DT, bool BR, bool kVar, bool AN = false>
__device__ __forceinline__ void cone_adjoint(const BwdLaunch &L, const uint32_t *code_off,
                                             const uint2 *lut, bool active,
                                             const Apex &A, const float w[3],
                                             const ConeConst &cc, float T0, float gc0, float gc1,
                                             float gc2, float ga, const uint2 *state, int mode) {
  const unsigned full = 0xffffffffu;
  const DevPyr &P = L.pyr;
  // kVar: a launch with a cone variant; the plain instances keep none of it
  const bool premul = kVar && (L.var.flags & VCT_FLAG_PREMULTIPLIED) != 0;
  if constexpr (!kVar) mode = kPlain;
  AnisoW aw{};
  if constexpr (AN) aw = aniso_weights(w);
  float prod = 1.f, prod_last = 1.f;
  float tr_next = 0.f, R0 = 0.f, R1 = 0.f, R2 = 0.f, Q = 1.f;
  int k = 0;                    // this lane's forward step
  int K = active ? -1 : 0;      // this lane's sample count once known
  bool rev = false;             // warp-uniform
  int kr = 0;                   // warp-uniform backward step
  if (state != nullptr) {
    if (active) {
      const uint2 e = *state;
      K = (int)e.x;
      prod_last = __uint_as_float(e.y);
    }
    rev = true;
    kr = (int)__reduce_max_sync(full, (unsigned)K);  // decremented before the first step
  }
  for (;;) {
    if (!rev) {
      if (K < 0 && !(k < cc.kmax && (1.0f - prod) < 1.0f)) K = k;
      if (__all_sync(full, K >= 0)) {
        rev = true;
        kr = (int)__reduce_max_sync(full, (unsigned)K) - 1;
      }
    } else {
      --kr;
    }
    // a first-hit cone needs its last step only; the walk ends when every
    // lane has passed its lowest step (lanes without samples have K = 0)
    bool act;
    if constexpr (kVar) {
      if (rev && __all_sync(full, kr < 0 || (mode == kFirstHit && kr < K - 1))) break;
      act = rev ? (kr >= 0 && kr < K && (mode != kFirstHit || kr == K - 1)) : (K < 0);
    } else {
      if (rev && kr < 0) break;
      act = rev ? (kr < K) : (K < 0);
    }
    const int ks = rev ? kr : k;
    LevelStencil st[2];
    st[0].valid = 0u;
    st[1].valid = 0u;
    LodPick lp;
    lp.l0 = lp.l1 = 0;
    lp.f = 0.f;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    float om = 1.f, fade = 1.f;
    if (act) {
      float T, lam;
      step_at(cc, T0, ks, T, lam);
      const float F[3] = {fmaf(T, w[0], A.Of[0]), fmaf(T, w[1], A.Of[1]), fmaf(T, w[2], A.Of[2])};
      if constexpr (AN)
        v = sample_aniso(P, A, F, lam, lut, aw, om, lp, st);
      else
        v = sample<DT, BR>(P, A, F, lam, lut, om, lp, st);
      if (kVar && mode == kOccSmooth) {  // as the forward march
        fade = smoothstep0(L.var.occ_max_dist, sqrtf(T * P.h0) * L.var.shadow_str);
        v.w *= fade;
        om = transparency(v.w);
      }
    }
    if (!rev) {
      if (act) {
        if (kVar && mode == kFirstHit) {
          if (v.w > 0.01f) K = k + 1;  // the hit ends the cone
        } else {
          prod_last = prod;
          prod *= om;
        }
        ++k;
      }
      continue;
    }
    float g[4] = {0.f, 0.f, 0.f, 0.f};
    if (kVar && act && mode == kFirstHit) {
      if (v.w > 0.01f) {  // a hit (not the end of the cone without one)
        g[0] = gc0;
        g[1] = gc1;
        g[2] = gc2;
      }
    } else if (act) {
      // (om > 0 before the last sample, else the forward would have ended
      // there; the guard keeps a mismatch from spreading NaN)
      const float tr = (kr == K - 1) ? prod_last : (om > 0.0f ? tr_next / om : 0.0f);
      if (premul) {
        g[0] = gc0 * tr;
        g[1] = gc1 * tr;
        g[2] = gc2 * tr;
        g[3] = tr * (ga * Q - (gc0 * R0 + gc1 * R1 + gc2 * R2));
        R0 = fmaf(om, R0, v.x);
        R1 = fmaf(om, R1, v.y);
        R2 = fmaf(om, R2, v.z);
      } else {
        const float ta = tr * v.w;  // same T_k as the forward's colour weight
        g[0] = gc0 * ta;
        g[1] = gc1 * ta;
        g[2] = gc2 * ta;
        g[3] = tr * (gc0 * (v.x - R0) + gc1 * (v.y - R1) + gc2 * (v.z - R2) + ga * Q);
        R0 = fmaf(v.w, v.x, om * R0);
        R1 = fmaf(v.w, v.y, om * R1);
        R2 = fmaf(v.w, v.z, om * R2);
      }
      if constexpr (kVar) g[3] *= fade;
      Q *= om;
      tr_next = tr;
    }
    scatter_level<AN>(L, code_off, act, lp.l0, st[0], 1.0f - lp.f, g, aw);
    const bool two = act && lp.f > 0.0f;
    if (__any_sync(full, two)) scatter_level<AN>(L, code_off, two, lp.l1, st[1], lp.f, g, aw);
  }
}

template <int LPP, int DT, bool BR, bool kVar, bool AN = false>
__global__ void __launch_bounds__(kTraceThreads, 2) trace_bwd_kernel(const __grid_constant__ BwdLaunch L) {
  constexpr int kPixPerRound = 32 / LPP;
  const int lane = threadIdx.x & 31;
  const int slot = lane % LPP;
  const int pr = lane / LPP;
  const int n_cones = L.n_diffuse + L.spec_enable + L.occ_enable;
  const float T0 = L.spec.t0_vox;
  const DevPyr &P = L.pyr;

  // per level: texels of all finer levels (offsets of the scatter's cell
  // keys; six volumes per anisotropic level >= 1); slot kKeyTotal: all of them
  __shared__ uint32_t s_code_off[kKeyTotal + 1];
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int l = 0; l < VCT_MAX_LEVELS; ++l) {
      s_code_off[l] = acc;
      if (l < P.levels) acc += (uint32_t)level_texels(P.n, l) * ((AN && l >= 1) ? 6u : 1u);
    }
    s_code_off[kKeyTotal] = acc;
  }
  __shared__ uint2 s_lut[kSpreadLut];
  fill_spread_lut(s_lut);  // (its barrier also covers s_code_off)

  for (;;) {
    const int item = next_item(L.queue);
    if (item >= L.total_tiles) break;
    int lo = 0, hi = L.n_views - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (L.views[mid].v.tile_begin <= item)
        lo = mid;
      else
        hi = mid - 1;
    }
    const BwdView &BV = L.views[lo];
    const DevView &V = BV.v;
    const int t = item - V.tile_begin;
    const int tx0 = (t % V.tiles_x) * L.tile_w;
    const int ty0 = (t / V.tiles_x) * L.tile_h;
    const int tile_pix = L.tile_w * L.tile_h;

    for (int base = 0; base < tile_pix; base += kPixPerRound) {
      const int pi = base + pr;
      const int px = tx0 + pi % L.tile_w;
      const int py = ty0 + pi / L.tile_w;
      const bool inimg = pi < tile_pix && px < V.W && py < V.H;
      const int p = inimg ? py * V.W + px : 0;
      const bool pix_on = inimg && (V.mask == nullptr || V.mask[p] != 0);
      float x[3] = {0.f, 0.f, 0.f}, n[3] = {0.f, 0.f, 1.f};
      float4 gD = make_float4(0.f, 0.f, 0.f, 0.f), gS = gD;
      float gV = 0.f;
      if (pix_on) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          x[a] = V.pos[3 * p + a];
          n[a] = V.nrm[3 * p + a];
        }
        if (BV.gD) gD = reinterpret_cast<const float4 *>(BV.gD)[p];
        if (BV.gS) gS = reinterpret_cast<const float4 *>(BV.gS)[p];
        if (BV.gV) gV = BV.gV[p];
        if (BV.gL && (L.var.flags & VCT_FLAG_SHADE)) {
          // chain rule through the shading epilogue: L_ch depends on D_ch,
          // S_ch and Vis (L_vxct = alb (kd D + ks S) + Vis direct; L_impl =
          // Vis (D + direct) + S, which needs the forward's D and Vis)
          const float4 gL = reinterpret_cast<const float4 *>(BV.gL)[p];
          float direct[3], alb[3];
          shade_direct(L.var, V, p, direct, alb);
          const float gl[3] = {gL.x, gL.y, gL.z};
          float dD[3], dS[3], dV = 0.f;
          if (L.var.flags & VCT_FLAG_SHADE_IMPL) {
            const float4 Df = reinterpret_cast<const float4 *>(V.outD)[p];
            const float vis = (L.occ_enable && V.outV) ? V.outV[p] : 1.0f;
            const float Dc[3] = {Df.x, Df.y, Df.z};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              dD[a] = gl[a] * vis;
              dS[a] = gl[a];
              dV = fmaf(gl[a], Dc[a] + direct[a], dV);
            }
          } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              dD[a] = gl[a] * alb[a] * L.var.kd;
              dS[a] = gl[a] * alb[a] * L.var.ks;
              dV = fmaf(gl[a], direct[a], dV);
            }
          }
          gD.x += dD[0];
          gD.y += dD[1];
          gD.z += dD[2];
          gS.x += dS[0];
          gS.y += dS[1];
          gS.z += dS[2];
          gV += dV;
        }
      }
      Apex A;
      make_apex(P, x, n, L.normal_offset, A);
      float Tf[3], Bf[3];
      tangent_frame(n, Tf, Bf);
      // The warp runs its lanes' cones together (the trip count is the same
      // for every lane: warp-collective operations inside need it).
      for (int c0 = 0; c0 < n_cones; c0 += LPP) {
        const int c = c0 + slot;
        const bool has_cone = c < n_cones;
        const ConeSel cs = select_cone(has_cone ? c : 0, L.spec_enable, L.occ_enable);
        float w[3] = {0.f, 0.f, 1.f};
        ConeConst cc = P.diffuse;
        float g0, g1, g2, ga;
        int mode = kPlain;
        if (cs.kind == kSpecular) {
          if (pix_on) reflect_dir(x, V.cam, n, w);
          cc = pix_on ? spec_const(P, L.spec, V.rough, p) : P.spec_fixed;
          // the angular-grace factor scales the specular colour only
          const float f =
              (kVar && (L.var.flags & VCT_FLAG_SPEC_GRACE)) ? spec_grace(L.var, w) : 1.0f;
          g0 = f * gS.x;
          g1 = f * gS.y;
          g2 = f * gS.z;
          ga = gS.w;
        } else if (cs.kind == kOcclusion) {
          w[0] = L.light[0];
          w[1] = L.light[1];
          w[2] = L.light[2];
          cc = P.occ;
          g0 = g1 = g2 = 0.f;
          ga = -gV;  // Vis = 1 - alpha
          if (L.var.flags & VCT_FLAG_OCC_SMOOTH) mode = kOccSmooth;
        } else {
          const float *d = L.diffuse_dir[cs.diffuse_index];
#pragma unroll
          for (int a = 0; a < 3; ++a) w[a] = fmaf(Tf[a], d[0], fmaf(Bf[a], d[1], n[a] * d[2]));
          const float wt = L.diffuse_weight[cs.diffuse_index];
          g0 = wt * gD.x;
          g1 = wt * gD.y;
          g2 = wt * gD.z;
          ga = wt * gD.w;
          if (L.var.flags & VCT_FLAG_DIFFUSE_FIRST_HIT) mode = kFirstHit;
        }
        const bool on = pix_on && has_cone && (g0 != 0.f || g1 != 0.f || g2 != 0.f || ga != 0.f);
        const uint2 *st = V.state == nullptr ? nullptr
                          : V.state + (on ? (size_t)c * V.W * V.H + p : 0);
        if (__any_sync(0xffffffffu, on))
          cone_adjoint<DT, BR, kVar, AN>(L, s_code_off, s_lut, on, A, w, cc, T0, g0, g1, g2, ga,
                                         st, mode);
      }
    }
  }
}

__global__ void fix_to_float_kernel(const unsigned long long *fix, float *out, uint64_t count) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = __ll2float_rn((long long)fix[i]) * (1.0f / kFixScale);
}

template <int LPP, int DT, bool BR, bool kVar, bool AN = false>
cudaError_t launch_b(const BwdLaunch &L, int grid, cudaStream_t s) {
  trace_bwd_kernel<LPP, DT, BR, kVar, AN><<<grid, kTraceThreads, 0, s>>>(L);
  return cudaGetLastError();
}

template <int LPP, int DT, bool BR, bool kVar>
int occ_b() {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_bwd_kernel<LPP, DT, BR, kVar>,
                                                kTraceThreads, 0);
  return b;
}

template <int DT, bool BR, bool kVar, bool AN = false>
cudaError_t launch_lpp(const BwdLaunch &L, int lpp, int grid, cudaStream_t s) {
  switch (lpp) {
    case 1: return launch_b<1, DT, BR, kVar, AN>(L, grid, s);
    case 2: return launch_b<2, DT, BR, kVar, AN>(L, grid, s);
    case 4: return launch_b<4, DT, BR, kVar, AN>(L, grid, s);
    case 8: return launch_b<8, DT, BR, kVar, AN>(L, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int DT, bool BR, bool AN = false>
cudaError_t launch_var(const BwdLaunch &L, int lpp, int grid, cudaStream_t s) {
  return bwd_has_variants(L.var.flags) ? launch_lpp<DT, BR, true, AN>(L, lpp, grid, s)
                                       : launch_lpp<DT, BR, false, AN>(L, lpp, grid, s);
}

template <int DT, bool BR>
int occ_lpp(int lpp) {
  switch (lpp) {
    case 1: return occ_b<1, DT, BR, false>();
    case 2: return occ_b<2, DT, BR, false>();
    case 4: return occ_b<4, DT, BR, false>();
    case 8: return occ_b<8, DT, BR, false>();
    default: return 0;
  }
}

}  // namespace

static_assert(sizeof(BwdLaunch) <= 32000, "adjoint launch parameters exceed the 32 KB limit");

cudaError_t launch_trace_bwd(const BwdLaunch &L, int lpp, int grid, cudaStream_t s) {
  if (L.aniso) return launch_var<VCT_F32, false, true>(L, lpp, grid, s);  // FP32, dense only
  const bool br = L.pyr.bricked != 0;
  if (L.pyr.dtype == VCT_F16)
    return br ? launch_var<VCT_F16, true>(L, lpp, grid, s) : launch_var<VCT_F16, false>(L, lpp, grid, s);
  return br ? launch_var<VCT_F32, true>(L, lpp, grid, s) : launch_var<VCT_F32, false>(L, lpp, grid, s);
}

cudaError_t launch_fix_to_float(const unsigned long long *fix, float *out, uint64_t count,
                                cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const int grid = (int)std::min<uint64_t>((count + 255) / 256, 4096);
  fix_to_float_kernel<<<grid, 256, 0, s>>>(fix, out, count);
  return cudaGetLastError();
}

int trace_bwd_occupancy(int lpp, int dtype, bool bricks) {
  if (dtype == VCT_F16) return bricks ? occ_lpp<VCT_F16, true>(lpp) : occ_lpp<VCT_F16, false>(lpp);
  return bricks ? occ_lpp<VCT_F32, true>(lpp) : occ_lpp<VCT_F32, false>(lpp);
}

VCT_OOB_ACCESSOR(oob_flags_trace_bwd)

}  // namespace vct
