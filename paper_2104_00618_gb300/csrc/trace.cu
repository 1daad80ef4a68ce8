// Forward cone trace: persistent CTAs pull pixel tiles from a queue; every
// pixel marches its diffuse, specular and occlusion cones through the
// Morton-ordered pyramid (Ch. 4.2 cone set, Ch. 4.3.2 march, Ch. 4.5 sampler).
#include "trace_common.cuh"

namespace vct {

namespace {

// Finds the view whose big-tile (small = false) or small-tile range holds
// `item` (both ranges increase with the view index).
__device__ __forceinline__ int find_view(const TraceLaunch &L, int item, bool small) {
  int lo = 0, hi = L.n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int begin = small ? L.views[mid].small_begin : L.views[mid].tile_begin;
    if (begin <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// One cone: returns (rgb, alpha) and, in `trans`, the transmittance
// T = prod_k (1 - a_k).  The thesis's accumulation (Ch. 4.3.2) is evaluated as
//   c += T_k a_k c_k,  alpha += T_k a_k,  T_{k+1} = T_k (1 - a_k)
// (alpha_k = 1 - T_k: the same recurrence), which keeps alpha precise when it
// is small and T precise when alpha is close to one; the loop runs while
// alpha = 1 - T < 1 in float32 and t <= t_max.  kVar instances also take the
// Ch. 5.4.4 variants selected by `mode`.
//
// The step position and level pair of step k (T, lambda -> l0, l1, f) depend
// on the cone's aperture and the pyramid only.  For the diffuse and
// occlusion cones, whose aperture is a launch constant, they are read from
// the CTA's step table (`tab`, shared memory, the first kStepTab steps; the
// same step_at / pick_levels arithmetic, done once per CTA); other cones
// compute them per step.
template <int DT, bool kVar, bool BR, bool AN = false>
__device__ __forceinline__ float4 march(const DevPyr &P, const Apex &A, const float w[3],
                                        const ConeConst &cc, float T0, const uint2 *lut,
                                        const float4 *tab, uint32_t &nsamp, float &trans,
                                        uint2 &state, int mode = kPlain,
                                        const Variants *var = nullptr) {
  float cr = 0.f, cg = 0.f, cb = 0.f, al = 0.f, tr = 1.f, tp = 1.f;
  int k = 0;
  AnisoW aw;
  if constexpr (AN) aw = aniso_weights(w);
  for (; k < cc.kmax; ++k) {
    if (!((1.0f - tr) < 1.0f)) break;
    float T, om;
    LodPick lp;
    if (tab != nullptr && k < kStepTab) {
      const float4 e = tab[k];
      T = e.x;
      lp.f = e.y;
      lp.l0 = __float_as_int(e.z);
      lp.l1 = __float_as_int(e.w);
    } else {
      float lam;
      step_at(cc, T0, k, T, lam);
      lp = pick_levels(lam, P.levels);
    }
    const float F[3] = {fmaf(T, w[0], A.Of[0]), fmaf(T, w[1], A.Of[1]), fmaf(T, w[2], A.Of[2])};
    float4 s;
    if constexpr (AN)
      s = sample_aniso_at(P, A, F, lp, lut, aw, om);
    else
      s = sample_at<DT, BR>(P, A, F, lp, lut, om);
    if constexpr (kVar) {
      if (mode == kFirstHit) {
        if (s.w > 0.01f) {
          nsamp += (uint32_t)(k + 1);
          trans = 0.0f;
          state = make_uint2((uint32_t)(k + 1), __float_as_uint(tr));
          return make_float4(s.x, s.y, s.z, 1.0f);
        }
        continue;
      }
      if (mode == kOccSmooth) {
        // t = T h0 in scene units
        s.w *= smoothstep0(var->occ_max_dist, sqrtf(T * P.h0) * var->shadow_str);
        om = transparency(s.w);
      }
    }
    const float wg = tr * s.w;  // front-to-back weight T_k a_s
    float wc = wg;              // colour weight: T_k a_s, or T_k for premultiplied colour
    if constexpr (kVar) {
      if (var->flags & VCT_FLAG_PREMULTIPLIED) wc = tr;
    }
    cr = fmaf(wc, s.x, cr);
    cg = fmaf(wc, s.y, cg);
    cb = fmaf(wc, s.z, cb);
    al += wg;
    tp = tr;
    tr *= om;
  }
  nsamp += (uint32_t)k;
  trans = tr;
  state = make_uint2((uint32_t)k, __float_as_uint(tp));
  return make_float4(cr, cg, cb, al);
}

// Shading epilogue, split in the part without the specular cone (`first`)
// and its specular term (`spec`), so that a deferred specular cone adds its
// term later.  Direct light: Phong with one directional light (Ch. 3.3)
//   direct = light_color * albedo * (kd max(n.l, 0) + ks max(v.R, 0)^shininess)
// L_vxct (Ch. 4.2.2): L = albedo (kd D + ks S) + Vis direct
// L_impl (Ch. 5.4.4): L = Vis D + S + Vis direct.
__device__ __forceinline__ float4 shade_first(const Variants &v, const DevView &V, int p,
                                              const float4 &D, float vis) {
  float direct[3], alb[3];
  shade_direct(v, V, p, direct, alb);
  const bool impl = (v.flags & VCT_FLAG_SHADE_IMPL) != 0;
  const float Dc[3] = {D.x, D.y, D.z};
  float o[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    o[a] = impl ? vis * (Dc[a] + direct[a]) : fmaf(alb[a] * v.kd, Dc[a], vis * direct[a]);
  return make_float4(o[0], o[1], o[2], 1.0f);
}

__device__ __forceinline__ float4 shade_spec(const Variants &v, const DevView &V, int p,
                                             const float4 &S, float4 L) {
  if (v.flags & VCT_FLAG_SHADE_IMPL) {
    L.x += S.x;
    L.y += S.y;
    L.z += S.z;
  } else {
    const float a0 = V.albedo ? V.albedo[3 * p] : 1.0f;
    const float a1 = V.albedo ? V.albedo[3 * p + 1] : 1.0f;
    const float a2 = V.albedo ? V.albedo[3 * p + 2] : 1.0f;
    L.x = fmaf(a0 * v.ks, S.x, L.x);
    L.y = fmaf(a1 * v.ks, S.y, L.y);
    L.z = fmaf(a2 * v.ks, S.z, L.z);
  }
  return L;
}

// Estimated step count of the specular cone (sort key only; float32).
__device__ __forceinline__ uint32_t spec_steps_estimate(const TraceLaunch &L, const DevPyr &P,
                                                        const float *rough, int p) {
  float g = L.spec.gmin;
  if (rough != nullptr) {
    const float f = fminf(fmaxf((rough[p] - L.spec.rough_min) * L.spec.inv_rough_span, 0.0f), 1.0f);
    g = fmaf(f, L.spec.gdelta, g);
  }
  const float l2r = log1pf(L.spec.two_beta * tanf(0.5f * g)) * 1.44269504f;
  const float e = P.log2_tmax_t0 / l2r;
  return (uint32_t)fminf(fmaxf(e + 1.0f, 1.0f), 65535.0f);
}

// Bitonic sort (descending) of n = 2^k keys in shared memory by one warp.
__device__ __forceinline__ void warp_sort_desc(uint32_t *keys, int n) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < n; i += 32) {
        const int q = i ^ j;
        if (q > i) {
          const uint32_t a = keys[i], b = keys[q];
          const bool desc = (i & k) == 0;
          if (desc ? (a < b) : (a > b)) {
            keys[i] = b;
            keys[q] = a;
          }
        }
      }
      __syncwarp();
    }
  }
}

// Each warp works independently: it takes a tile of pixels from the queue
// and covers it in rounds of 32 / LPP pixels (LPP lanes share one pixel's
// cones).  No block-wide barrier in the work loop.  With one lane per pixel
// the specular cones of the tile are marched last, longest first: the
// tile's estimated specular step counts are sorted so that the lanes of a
// warp march cones of similar length together (the aperture, hence the
// length, varies from pixel to pixel with the roughness).
// kVar instances add the Ch. 5.4.4 cone variants and the shading epilogue
// (any VCT_FLAG_* set); the plain instances carry none of that code.  BR
// instances read brick pyramids (VCT_LAYOUT_BRICKS).
template <int LPP, int DT, bool kVar, bool BR, bool AN>
__global__ void __launch_bounds__(kFwdThreads, kTraceMinBlocks) trace_kernel(const __grid_constant__ TraceLaunch L) {
  constexpr int kPixPerRound = 32 / LPP;
  constexpr bool kSortSpec = (LPP == 1);
  uint32_t n_samp[3] = {0u, 0u, 0u}, n_cone[3] = {0u, 0u, 0u};
  const int lane = threadIdx.x & 31;
  const int slot = lane % LPP;
  const int pr = lane / LPP;
  const bool defer_spec = kSortSpec && L.spec_enable;
  const int n_cones = L.n_diffuse + L.spec_enable + L.occ_enable;
  const int first_cone = defer_spec ? 1 : 0;  // the specular cone is cone 0
  const float T0 = L.spec.t0_vox;
  __shared__ uint2 s_lut[kSpreadLut];
  __shared__ uint32_t s_keys[kFwdThreads / 32][kMaxSortPixels];
  extern __shared__ __align__(16) float4 s_tab[];  // n_pyr * 2 * kStepTab entries
  uint32_t *keys = s_keys[threadIdx.x >> 5];
  fill_step_table(s_tab, L.pyr, L.n_pyr, T0);
  fill_spread_lut(s_lut);  // (its barrier also covers s_tab)

  for (;;) {
    const int item = next_item(L.queue);
    if (item >= L.total_tiles) break;
    const bool small = item >= L.n_big;
    const int vi = find_view(L, item, small);
    const DevView &V = L.views[vi];
    const DevPyr &P = L.pyr[V.pyr];
    int tile_w, tx0, ty0, tile_pix;
    if (!small) {
      const int t = item - V.tile_begin;
      tile_w = L.tile_w;
      tx0 = (t % V.tiles_x) * L.tile_w;
      ty0 = (t / V.tiles_x) * L.tile_h;
      tile_pix = L.tile_w * L.tile_h;
    } else {
      const int t = item - V.small_begin;
      tile_w = kSmallTileW;
      tx0 = (t % V.small_tiles_x) * kSmallTileW;
      ty0 = V.y_split + (t / V.small_tiles_x) * kSmallTileH;
      tile_pix = kSmallTileW * kSmallTileH;
    }

    for (int base = 0; base < tile_pix; base += kPixPerRound) {
      const int pi = base + pr;
      const int px = tx0 + pi % tile_w;
      const int py = ty0 + pi / tile_w;
      const bool inimg = pi < tile_pix && px < V.W && py < V.H;
      const int p = py * V.W + px;
      bool active = inimg && (V.mask == nullptr || V.mask[p] != 0);

      float4 D = make_float4(0.f, 0.f, 0.f, 0.f), S = D;
      float vis = 0.f;  // transmittance of the occlusion cone, summed over the pixel's lanes
      int has_occ = 0;
      if (active) {
        float x[3], n[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          x[a] = V.pos[3 * p + a];
          n[a] = V.nrm[3 * p + a];
        }
        Apex A;
        make_apex(P, x, n, L.normal_offset, A);
        float Tf[3], Bf[3];
        tangent_frame(n, Tf, Bf);
        for (int c = first_cone + slot; c < n_cones; c += LPP) {
          const ConeSel cs = select_cone(c, L.spec_enable, L.occ_enable);
          float w[3];
          ConeConst cc;
          const float4 *tab = nullptr;
          if (cs.kind == kSpecular) {
            reflect_dir(x, V.cam, n, w);
            cc = spec_const(P, L.spec, V.rough, p);
          } else if (cs.kind == kOcclusion) {
            w[0] = L.light[0];
            w[1] = L.light[1];
            w[2] = L.light[2];
            cc = P.occ;
            tab = step_table(s_tab, V.pyr, 1);
          } else {
            const float *d = L.diffuse_dir[cs.diffuse_index];
#pragma unroll
            for (int a = 0; a < 3; ++a) w[a] = fmaf(Tf[a], d[0], fmaf(Bf[a], d[1], n[a] * d[2]));
            cc = P.diffuse;
            tab = step_table(s_tab, V.pyr, 0);
          }
          float trans;
          int mode = kPlain;
          if constexpr (kVar) {
            if (cs.kind == kOcclusion && (L.var.flags & VCT_FLAG_OCC_SMOOTH)) mode = kOccSmooth;
            if (cs.kind == kDiffuse && (L.var.flags & VCT_FLAG_DIFFUSE_FIRST_HIT)) mode = kFirstHit;
          }
          uint2 cst;
          float4 r = march<DT, kVar, BR, AN>(P, A, w, cc, T0, s_lut, tab, n_samp[cs.kind], trans,
                                             cst, mode, &L.var);
          n_cone[cs.kind] += 1u;
          if (V.state) V.state[(size_t)c * V.W * V.H + p] = cst;
          if constexpr (kVar) {
            if (cs.kind == kSpecular && (L.var.flags & VCT_FLAG_SPEC_GRACE)) {
              const float f = spec_grace(L.var, w);
              r.x *= f;
              r.y *= f;
              r.z *= f;
            }
          }
          if (cs.kind == kDiffuse) {
            const float wt = L.diffuse_weight[cs.diffuse_index];
            D.x = fmaf(wt, r.x, D.x);
            D.y = fmaf(wt, r.y, D.y);
            D.z = fmaf(wt, r.z, D.z);
            D.w = fmaf(wt, r.w, D.w);
          } else if (cs.kind == kSpecular) {
            S = r;
          } else {
            vis = trans;
            has_occ = 1;
          }
        }
      }
      // Combine the lanes that share a pixel.
#pragma unroll
      for (int m = 1; m < LPP; m <<= 1) {
        D.x += __shfl_xor_sync(0xffffffffu, D.x, m);
        D.y += __shfl_xor_sync(0xffffffffu, D.y, m);
        D.z += __shfl_xor_sync(0xffffffffu, D.z, m);
        D.w += __shfl_xor_sync(0xffffffffu, D.w, m);
        S.x += __shfl_xor_sync(0xffffffffu, S.x, m);
        S.y += __shfl_xor_sync(0xffffffffu, S.y, m);
        S.z += __shfl_xor_sync(0xffffffffu, S.z, m);
        S.w += __shfl_xor_sync(0xffffffffu, S.w, m);
        vis += __shfl_xor_sync(0xffffffffu, vis, m);
        has_occ |= __shfl_xor_sync(0xffffffffu, has_occ, m);
      }
      if (inimg && slot == 0) {
        if (V.outD) reinterpret_cast<float4 *>(V.outD)[p] = D;
        if (V.outS && !(defer_spec && active)) reinterpret_cast<float4 *>(V.outS)[p] = S;
        if (V.outV) V.outV[p] = has_occ ? vis : 1.0f;
        if constexpr (kVar) {
          if (V.outL) {
            float4 Lp = make_float4(0.f, 0.f, 0.f, 0.f);
            if (active) {
              Lp = shade_first(L.var, V, p, D, has_occ ? vis : 1.0f);
              if (!defer_spec) Lp = shade_spec(L.var, V, p, S, Lp);
            }
            reinterpret_cast<float4 *>(V.outL)[p] = Lp;
          }
        }
      }
      if (defer_spec) {
        // key: valid bit, estimated steps, pixel within the tile
        keys[pi] = active ? (0x80000000u | (spec_steps_estimate(L, P, V.rough, p) << 8) |
                             (uint32_t)pi)
                          : 0u;
      }
    }
    if (!defer_spec) continue;

    // Specular cones of the tile, longest first.
    int nsort = 32;
    while (nsort < tile_pix) nsort <<= 1;
    for (int i = tile_pix + lane; i < nsort; i += 32) keys[i] = 0u;
    __syncwarp();
    warp_sort_desc(keys, nsort);
    for (int base = 0; base < tile_pix; base += 32) {
      const uint32_t key = keys[base + lane];
      if (!(key & 0x80000000u)) continue;
      const int pi = (int)(key & 0xffu);
      const int px = tx0 + pi % tile_w;
      const int py = ty0 + pi / tile_w;
      const int p = py * V.W + px;
      float x[3], n[3], w[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        x[a] = V.pos[3 * p + a];
        n[a] = V.nrm[3 * p + a];
      }
      Apex A;
      make_apex(P, x, n, L.normal_offset, A);
      reflect_dir(x, V.cam, n, w);
      const ConeConst cc = spec_const(P, L.spec, V.rough, p);
      float trans;
      uint2 cst;
      float4 r = march<DT, kVar, BR, AN>(P, A, w, cc, T0, s_lut, nullptr, n_samp[kSpecular],
                                         trans, cst, kPlain, &L.var);
      n_cone[kSpecular] += 1u;
      if (V.state) V.state[p] = cst;  // the specular cone is cone 0
      if constexpr (kVar) {
        if (L.var.flags & VCT_FLAG_SPEC_GRACE) {
          const float f = spec_grace(L.var, w);
          r.x *= f;
          r.y *= f;
          r.z *= f;
        }
        // The first part of the pixel's radiance was written by another lane
        // of this warp before the __syncwarp that precedes the sort.
        if (V.outL) {
          float4 *q = reinterpret_cast<float4 *>(V.outL) + p;
          *q = shade_spec(L.var, V, p, r, *q);
        }
      }
      if (V.outS) reinterpret_cast<float4 *>(V.outS)[p] = r;
    }
    __syncwarp();
  }
  // Per-kind sample and cone counters: one atomic per warp.
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint32_t s = __reduce_add_sync(0xffffffffu, n_samp[k]);
    const uint32_t c = __reduce_add_sync(0xffffffffu, n_cone[k]);
    if ((threadIdx.x & 31) == 0) {
      if (s) atomicAdd(L.stats + k, (unsigned long long)s);
      if (c) atomicAdd(L.stats + 3 + k, (unsigned long long)c);
    }
  }
}

// Dynamic shared memory of a launch: the step tables of its pyramids.
inline size_t step_table_bytes(int n_pyr) { return (size_t)n_pyr * 2 * kStepTab * sizeof(float4); }

template <int LPP, int DT, bool BR, bool AN = false>
cudaError_t launch_t(const TraceLaunch &L, int grid, cudaStream_t s) {
  const size_t dyn = step_table_bytes(L.n_pyr);
  if (L.var.flags)
    trace_kernel<LPP, DT, true, BR, AN><<<grid, kFwdThreads, dyn, s>>>(L);
  else
    trace_kernel<LPP, DT, false, BR, AN><<<grid, kFwdThreads, dyn, s>>>(L);
  return cudaGetLastError();
}

// Anisotropic pyramids are float32 and dense (no brick instance).
template <int LPP, int DT>
cudaError_t launch_l(const TraceLaunch &L, bool br, int grid, cudaStream_t s, bool an) {
  if constexpr (DT == VCT_F32) {
    if (an) return launch_t<LPP, DT, false, true>(L, grid, s);
  }
  if (an) return cudaErrorInvalidValue;
  return br ? launch_t<LPP, DT, true>(L, grid, s) : launch_t<LPP, DT, false>(L, grid, s);
}

template <int LPP, int DT>
int occ_t(bool var) {
  int b = 0;
  if (var)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_kernel<LPP, DT, true, false, false>,
                                                  kFwdThreads, step_table_bytes(VCT_MAX_PYRAMIDS));
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_kernel<LPP, DT, false, false, false>,
                                                  kFwdThreads, step_table_bytes(VCT_MAX_PYRAMIDS));
  return b;
}

}  // namespace

static_assert(sizeof(TraceLaunch) <= 32000, "trace launch parameters exceed the 32 KB limit");

cudaError_t launch_trace(const TraceLaunch &L, int lpp, int dtype, bool bricks, int grid,
                         cudaStream_t s, bool aniso) {
  const bool h = dtype == VCT_F16;
  const bool b = bricks;
  const bool a = aniso;
  switch (lpp) {
    case 1: return h ? launch_l<1, VCT_F16>(L, b, grid, s, a) : launch_l<1, VCT_F32>(L, b, grid, s, a);
    case 2: return h ? launch_l<2, VCT_F16>(L, b, grid, s, a) : launch_l<2, VCT_F32>(L, b, grid, s, a);
    case 4: return h ? launch_l<4, VCT_F16>(L, b, grid, s, a) : launch_l<4, VCT_F32>(L, b, grid, s, a);
    case 8: return h ? launch_l<8, VCT_F16>(L, b, grid, s, a) : launch_l<8, VCT_F32>(L, b, grid, s, a);
    default: return cudaErrorInvalidValue;
  }
}

int trace_occupancy(int lpp, int dtype, bool var) {
  const bool h = dtype == VCT_F16;
  switch (lpp) {
    case 1: return h ? occ_t<1, VCT_F16>(var) : occ_t<1, VCT_F32>(var);
    case 2: return h ? occ_t<2, VCT_F16>(var) : occ_t<2, VCT_F32>(var);
    case 4: return h ? occ_t<4, VCT_F16>(var) : occ_t<4, VCT_F32>(var);
    case 8: return h ? occ_t<8, VCT_F16>(var) : occ_t<8, VCT_F32>(var);
    default: return 0;
  }
}

VCT_OOB_ACCESSOR(oob_flags_trace)

}  // namespace vct
