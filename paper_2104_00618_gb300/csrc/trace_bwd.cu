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

__device__ __forceinline__ void scatter_level(float *glvl, const LevelStencil &s, float dc0,
                                              float dc1, float dc2, float da) {
  float4 *g = reinterpret_cast<float4 *>(glvl);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (!((s.valid >> c) & 1u)) continue;
    const float w = corner_weight(s, c);
    if (w == 0.0f) continue;
    atomicAdd(g + corner_index(s, c), make_float4(w * dc0, w * dc1, w * dc2, w * da));
  }
}

__device__ __forceinline__ void cone_adjoint(const BwdLaunch &L, const Apex &A, const float w[3],
                                             const ConeConst &cc, float T0, float gc0, float gc1,
                                             float gc2, float ga) {
  const DevPyr &P = L.pyr;
  float prod = 1.f, prod_last = 1.f;
  float tr_next = 0.f, R0 = 0.f, R1 = 0.f, R2 = 0.f, Q = 1.f;
  int k = 0, K = 0;
  bool rev = false;
  for (;;) {
    if (!rev) {
      if (k >= cc.kmax || !((1.0f - prod) < 1.0f)) {
        K = k;
        rev = true;
        k = K - 1;
        if (k < 0) break;
      }
    } else if (k < 0) {
      break;
    }
    float T, lam;
    step_at(cc, T0, k, T, lam);
    const float F[3] = {fmaf(T, w[0], A.Of[0]), fmaf(T, w[1], A.Of[1]), fmaf(T, w[2], A.Of[2])};
    const LodPick lp = pick_levels(lam, P.levels);
    LevelStencil s0, s1;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    level_stencil(lp.l0, P.n >> lp.l0, 1.0f - lp.f, A, F, s0);
    accumulate_level<VCT_F32>(P.lvl[lp.l0], s0, v);
    if (lp.f > 0.0f) {
      level_stencil(lp.l1, P.n >> lp.l1, lp.f, A, F, s1);
      accumulate_level<VCT_F32>(P.lvl[lp.l1], s1, v);
    }
    const float om = 1.0f - v.w;
    if (!rev) {
      prod_last = prod;
      prod *= om;
      ++k;
    } else {
      const float tr = (k == K - 1) ? prod_last : tr_next / om;
      const float ta = tr * v.w;  // same T_k as the forward's colour weight
      const float dc0 = gc0 * ta, dc1 = gc1 * ta, dc2 = gc2 * ta;
      const float da = tr * (gc0 * (v.x - R0) + gc1 * (v.y - R1) + gc2 * (v.z - R2) + ga * Q);
      R0 = fmaf(v.w, v.x, om * R0);
      R1 = fmaf(v.w, v.y, om * R1);
      R2 = fmaf(v.w, v.z, om * R2);
      Q *= om;
      scatter_level(L.gpyr_lvl[lp.l0], s0, dc0, dc1, dc2, da);
      if (lp.f > 0.0f) scatter_level(L.gpyr_lvl[lp.l1], s1, dc0, dc1, dc2, da);
      tr_next = tr;
      --k;
    }
  }
}

template <int LPP>
__global__ void __launch_bounds__(kTraceThreads, 2) trace_bwd_kernel(const __grid_constant__ BwdLaunch L) {
  constexpr int kPixPerRound = 32 / LPP;
  const int lane = threadIdx.x & 31;
  const int slot = lane % LPP;
  const int pr = lane / LPP;
  const int n_cones = L.n_diffuse + L.spec_enable + L.occ_enable;
  const float T0 = (float)L.t0_vox;
  const DevPyr &P = L.pyr;

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
      const int p = py * V.W + px;
      if (!inimg || (V.mask != nullptr && V.mask[p] == 0)) continue;
      float x[3], n[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        x[a] = V.pos[3 * p + a];
        n[a] = V.nrm[3 * p + a];
      }
      float4 gD = make_float4(0.f, 0.f, 0.f, 0.f), gS = gD;
      float gV = 0.f;
      if (BV.gD) gD = reinterpret_cast<const float4 *>(BV.gD)[p];
      if (BV.gS) gS = reinterpret_cast<const float4 *>(BV.gS)[p];
      if (BV.gV) gV = BV.gV[p];
      Apex A;
      make_apex(P, x, n, L.normal_offset, A);
      float Tf[3], Bf[3];
      tangent_frame(n, Tf, Bf);
      for (int c = slot; c < n_cones; c += LPP) {
        const ConeSel cs = select_cone(c, L.spec_enable, L.occ_enable);
        float w[3];
        ConeConst cc;
        float g0, g1, g2, ga;
        if (cs.kind == kSpecular) {
          reflect_dir(x, V.cam, n, w);
          cc = spec_const(P, L.spec_gmin, L.spec_gmax, L.rough_min, L.beta, L.t0_vox, V.rough, p);
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
          cc = P.diffuse;
          const float wt = L.diffuse_weight[cs.diffuse_index];
          g0 = wt * gD.x;
          g1 = wt * gD.y;
          g2 = wt * gD.z;
          ga = wt * gD.w;
        }
        if (g0 == 0.f && g1 == 0.f && g2 == 0.f && ga == 0.f) continue;
        cone_adjoint(L, A, w, cc, T0, g0, g1, g2, ga);
      }
    }
  }
}

template <int LPP>
cudaError_t launch_b(const BwdLaunch &L, int grid, cudaStream_t s) {
  trace_bwd_kernel<LPP><<<grid, kTraceThreads, 0, s>>>(L);
  return cudaGetLastError();
}

template <int LPP>
int occ_b() {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_bwd_kernel<LPP>, kTraceThreads, 0);
  return b;
}

}  // namespace

static_assert(sizeof(BwdLaunch) <= 32000, "adjoint launch parameters exceed the 32 KB limit");

cudaError_t launch_trace_bwd(const BwdLaunch &L, int lpp, int grid, cudaStream_t s) {
  switch (lpp) {
    case 1: return launch_b<1>(L, grid, s);
    case 2: return launch_b<2>(L, grid, s);
    case 4: return launch_b<4>(L, grid, s);
    case 8: return launch_b<8>(L, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int trace_bwd_occupancy(int lpp) {
  switch (lpp) {
    case 1: return occ_b<1>();
    case 2: return occ_b<2>();
    case 4: return occ_b<4>();
    case 8: return occ_b<8>();
    default: return 0;
  }
}

}  // namespace vct
