// Adjoint of the cone trace (row a7).  No per-sample state is stored: each
// cone is marched forwards once (same stopping rule as the forward kernel:
// alpha = 1 - T < 1 in float32) to find its length K and its transmittance
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
// float32 gradient pyramid with vector atomics.
#include "trace_common.cuh"

namespace vct {

namespace {

// Levels with at most 16^3 texels are accumulated per CTA in shared memory
// (every sample of a coarse level lands on a handful of texels, so global
// atomics there would serialize) and added to global memory once per CTA.
struct SmemGrad {
  float *base;      // shared float[4 * texels of levels >= first]
  int first;        // first level kept in shared memory
  int off[VCT_MAX_LEVELS];  // texel offset of each such level
};

__device__ __forceinline__ float *grad_texel(const BwdLaunch &L, const SmemGrad &sg, int l,
                                             uint32_t idx) {
  return l >= sg.first ? sg.base + 4 * (sg.off[l] + idx)
                       : reinterpret_cast<float *>(L.gpyr_lvl[l]) + 4 * (size_t)idx;
}

// Per-lane scatter of one level's 8 corners (lanes in different cells).
__device__ __forceinline__ void scatter_lane(const BwdLaunch &L, const SmemGrad &sg, int l,
                                             const LevelStencil &s, float lw, const float g[4]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (!((s.valid >> c) & 1u)) continue;
    const float w = corner_weight(s, lw, c);
    if (w == 0.0f) continue;
    float *t = grad_texel(L, sg, l, corner_index(s, c));
    if (l >= sg.first) {
      atomicAdd(t + 0, w * g[0]);
      atomicAdd(t + 1, w * g[1]);
      atomicAdd(t + 2, w * g[2]);
      atomicAdd(t + 3, w * g[3]);
    } else {
      atomicAdd(reinterpret_cast<float4 *>(t), make_float4(w * g[0], w * g[1], w * g[2], w * g[3]));
    }
  }
}

// Scatter of one level for the whole warp (warp-uniform call).  Lanes are
// grouped by (level, 2x2x2 cell).  A lane whose group has fewer than four
// lanes scatters its own corners.  For each larger group the 32 values
// (8 corners x 4 channels) are summed over the group by recursive halving,
// so that lane j ends with the group total of value j, and each lane issues
// one atomic on a distinct address: contending atomics (the same texel from
// many lanes) are what makes a naive scatter slow at the coarse levels.
__device__ __forceinline__ void scatter_warp(const BwdLaunch &L, const SmemGrad &sg, bool act,
                                             int l, const LevelStencil &s, float lw,
                                             const float g[4]) {
  const unsigned full = 0xffffffffu;
  if (__ballot_sync(full, act) == 0u) return;
  const int lane = threadIdx.x & 31;
  const unsigned long long key =
      act ? ((unsigned long long)(uint32_t)l << 40) | ((unsigned long long)s.valid << 32) |
                (s.sx[0] | s.sy[0] | s.sz[0])
          : ~0ull;
  const unsigned grp = __match_any_sync(full, key);
  const bool big = act && __popc(grp) >= 4;
  if (act && !big) scatter_lane(L, sg, l, s, lw, g);
  unsigned pending = __ballot_sync(full, big);
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const unsigned lgrp = __shfl_sync(full, grp, leader);
    const bool in = (lgrp >> lane) & 1u;
    float v[32];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float w = in ? corner_weight(s, lw, c) : 0.0f;
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) v[4 * c + ch] = w * g[ch];
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
    const int ll = __shfl_sync(full, l, leader);
    const uint32_t lvalid = __shfl_sync(full, s.valid, leader);
    const uint32_t sx0 = __shfl_sync(full, s.sx[0], leader), sx1 = __shfl_sync(full, s.sx[1], leader);
    const uint32_t sy0 = __shfl_sync(full, s.sy[0], leader), sy1 = __shfl_sync(full, s.sy[1], leader);
    const uint32_t sz0 = __shfl_sync(full, s.sz[0], leader), sz1 = __shfl_sync(full, s.sz[1], leader);
    const uint32_t idx = ((c & 1) ? sx1 : sx0) | (((c >> 1) & 1) ? sy1 : sy0) | ((c >> 2) ? sz1 : sz0);
    if (((lvalid >> c) & 1u) && v[0] != 0.0f) atomicAdd(grad_texel(L, sg, ll, idx) + ch, v[0]);
    pending &= ~lgrp;
  }
}

// Adjoint of one cone for every lane of the warp (warp-uniform call; lanes
// with active == false take no samples).
__device__ __forceinline__ void cone_adjoint(const BwdLaunch &L, const SmemGrad &sg,
                                             const uint32_t *lut, bool active,
                                             const Apex &A, const float w[3],
                                             const ConeConst &cc, float T0, float gc0, float gc1,
                                             float gc2, float ga) {
  const unsigned full = 0xffffffffu;
  const DevPyr &P = L.pyr;
  float prod = 1.f, prod_last = 1.f;
  float tr_next = 0.f, R0 = 0.f, R1 = 0.f, R2 = 0.f, Q = 1.f;
  int k = 0;                    // this lane's forward step
  int K = active ? -1 : 0;      // this lane's sample count once known
  bool rev = false;             // warp-uniform
  int kr = 0;                   // warp-uniform backward step
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
    if (rev && kr < 0) break;
    const bool act = rev ? (kr < K) : (K < 0);
    const int ks = rev ? kr : k;
    LevelStencil st[2];
    st[0].valid = 0u;
    st[1].valid = 0u;
    LodPick lp;
    lp.l0 = lp.l1 = 0;
    lp.f = 0.f;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    float om = 1.f;
    if (act) {
      float T, lam;
      step_at(cc, T0, ks, T, lam);
      const float F[3] = {fmaf(T, w[0], A.Of[0]), fmaf(T, w[1], A.Of[1]), fmaf(T, w[2], A.Of[2])};
      v = sample<VCT_F32>(P, A, F, lam, lut, om, lp, st);
    }
    if (!rev) {
      if (act) {
        prod_last = prod;
        prod *= om;
        ++k;
      }
      continue;
    }
    float g[4] = {0.f, 0.f, 0.f, 0.f};
    if (act) {
      const float tr = (kr == K - 1) ? prod_last : tr_next / om;
      const float ta = tr * v.w;  // same T_k as the forward's colour weight
      g[0] = gc0 * ta;
      g[1] = gc1 * ta;
      g[2] = gc2 * ta;
      g[3] = tr * (gc0 * (v.x - R0) + gc1 * (v.y - R1) + gc2 * (v.z - R2) + ga * Q);
      R0 = fmaf(v.w, v.x, om * R0);
      R1 = fmaf(v.w, v.y, om * R1);
      R2 = fmaf(v.w, v.z, om * R2);
      Q *= om;
      tr_next = tr;
    }
    scatter_warp(L, sg, act, lp.l0, st[0], 1.0f - lp.f, g);
    const bool two = act && lp.f > 0.0f;
    if (__any_sync(full, two)) scatter_warp(L, sg, two, lp.l1, st[1], lp.f, g);
  }
}

template <int LPP>
__global__ void __launch_bounds__(kTraceThreads, 3) trace_bwd_kernel(const __grid_constant__ BwdLaunch L) {
  constexpr int kPixPerRound = 32 / LPP;
  const int lane = threadIdx.x & 31;
  const int slot = lane % LPP;
  const int pr = lane / LPP;
  const int n_cones = L.n_diffuse + L.spec_enable + L.occ_enable;
  const float T0 = (float)L.t0_vox;
  const DevPyr &P = L.pyr;

  extern __shared__ __align__(16) float s_grad[];
  SmemGrad sg;
  sg.base = s_grad;
  sg.first = L.smem_first_level;
  int smem_texels = 0;
  for (int l = 0; l < VCT_MAX_LEVELS; ++l) {
    sg.off[l] = smem_texels;
    if (l >= sg.first && l < P.levels) smem_texels += (int)level_texels(P.n, l);
  }
  for (int i = threadIdx.x; i < 4 * smem_texels; i += blockDim.x) s_grad[i] = 0.f;
  __shared__ uint32_t s_lut[1024];
  fill_spread_lut(s_lut);  // (its barrier also covers the zeroing above)

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
        if (cs.kind == kSpecular) {
          if (pix_on) reflect_dir(x, V.cam, n, w);
          cc = pix_on ? spec_const(P, L.spec_gmin, L.spec_gmax, L.rough_min, L.beta, L.t0_vox,
                                   V.rough, p)
                      : P.spec_fixed;
          g0 = gS.x;
          g1 = gS.y;
          g2 = gS.z;
          ga = gS.w;
        } else if (cs.kind == kOcclusion) {
          w[0] = L.light[0];
          w[1] = L.light[1];
          w[2] = L.light[2];
          cc = P.occ;
          g0 = g1 = g2 = 0.f;
          ga = -gV;  // Vis = 1 - alpha
        } else {
          const float *d = L.diffuse_dir[cs.diffuse_index];
#pragma unroll
          for (int a = 0; a < 3; ++a) w[a] = fmaf(Tf[a], d[0], fmaf(Bf[a], d[1], n[a] * d[2]));
          const float wt = L.diffuse_weight[cs.diffuse_index];
          g0 = wt * gD.x;
          g1 = wt * gD.y;
          g2 = wt * gD.z;
          ga = wt * gD.w;
        }
        const bool on = pix_on && has_cone && (g0 != 0.f || g1 != 0.f || g2 != 0.f || ga != 0.f);
        if (__any_sync(0xffffffffu, on))
          cone_adjoint(L, sg, s_lut, on, A, w, cc, T0, g0, g1, g2, ga);
      }
    }
  }
  // Add this CTA's coarse-level gradients to global memory.
  __syncthreads();
  for (int l = sg.first; l < P.levels; ++l) {
    const int cnt = (int)level_texels(P.n, l);
    float4 *g = reinterpret_cast<float4 *>(L.gpyr_lvl[l]);
    const float4 *src = reinterpret_cast<const float4 *>(s_grad) + sg.off[l];
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const float4 v = src[i];
      if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) atomicAdd(g + i, v);
    }
  }
}

template <int LPP>
cudaError_t launch_b(const BwdLaunch &L, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(trace_bwd_kernel<LPP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  trace_bwd_kernel<LPP><<<grid, kTraceThreads, smem, s>>>(L);
  return cudaGetLastError();
}

template <int LPP>
int occ_b(size_t smem) {
  int b = 0;
  cudaFuncSetAttribute(trace_bwd_kernel<LPP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_bwd_kernel<LPP>, kTraceThreads, smem);
  return b;
}

}  // namespace

static_assert(sizeof(BwdLaunch) <= 32000, "adjoint launch parameters exceed the 32 KB limit");

size_t bwd_smem_bytes(int n, int levels, int first) {
  size_t t = 0;
  for (int l = first; l < levels; ++l) t += level_texels(n, l);
  return t * 16;
}

cudaError_t launch_trace_bwd(const BwdLaunch &L, int lpp, int grid, cudaStream_t s) {
  const size_t smem = bwd_smem_bytes(L.pyr.n, L.pyr.levels, L.smem_first_level);
  switch (lpp) {
    case 1: return launch_b<1>(L, grid, smem, s);
    case 2: return launch_b<2>(L, grid, smem, s);
    case 4: return launch_b<4>(L, grid, smem, s);
    case 8: return launch_b<8>(L, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

int trace_bwd_occupancy(int lpp, size_t smem) {
  switch (lpp) {
    case 1: return occ_b<1>(smem);
    case 2: return occ_b<2>(smem);
    case 4: return occ_b<4>(smem);
    case 8: return occ_b<8>(smem);
    default: return 0;
  }
}

}  // namespace vct
