"""The largest grid the library accepts, n = 1024 (11 levels, 17 GB of
level 0), checked through properties that hold at any size, since an FP64
oracle pyramid of that size does not fit a test's host memory:

- an empty grid gives no indirect light: D = S = 0 and Vis = 1 exactly;
- a homogeneous medium (every voxel (c0, a)) has every mip level equal to
  (c0, a), and a cone whose samples all lie inside the grid composites
  alpha = 1 - (1 - a)^K, colour = c0 alpha (K = the number of steps with
  t <= t_max, the Ch. 4.3.2 step rule in closed form);
- the adjoint summed over all level-0 voxels equals the derivative of the
  loss under a uniform shift of every voxel, d/da sum_px alpha = sum_px
  K (1 - a)^(K - 1) for the opacity and d/dc sum_px c = sum_px alpha for a
  colour channel.

The values 1/16 and multiples of 1/4 make every mip mean exact in float32.
"""
import math

import numpy as np
import pytest
import torch

import paper_2104_00618_gb300 as vct
import vct_synth as vs

pytestmark = pytest.mark.gpu

N = 1024
A = 0.0625
C0 = (0.25, 0.5, 0.75)
T_MAX = 0.15  # every sample of every cone stays well inside the grid from the centre


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vct.lib()
    yield
    torch.cuda.empty_cache()


def _params():
    dirs, w = vs.cone_table_ring6()
    return vs.trace_params(dirs, w, math.radians(60), spec_enable=True,
                           spec_aperture_min=math.radians(10), occ_enable=True,
                           occ_aperture=0.55, light=(0.3, 0.8, 0.52), t_max=T_MAX)


def _view(count=512, seed=3):
    """Pixels near the grid's centre with random unit normals, one camera."""
    rng = np.random.default_rng(seed)
    pos = (0.5 + 0.01 * (2 * rng.random((count, 3)) - 1)).astype(np.float32)
    nrm = rng.normal(size=(count, 3))
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    return vs.view_dict(pos.reshape(-1), nrm.reshape(-1), np.ones(count, np.uint8), count, 1,
                        np.array([0.5, 0.9, 0.2], np.float32))


def _steps(aperture, prm):
    """K = #{k >= 0 : t0 r^k <= t_max} in level-0 voxels, FP64 from the
    float32 parameters, with its distance to a tie."""
    beta = float(np.float32(prm["beta"]))
    t0 = float(np.float32(prm["t0_voxels"]))
    tmax = float(np.float32(prm["t_max"])) * N
    l2r = math.log2(1.0 + 2.0 * beta * math.tan(0.5 * float(np.float32(aperture))))
    e = math.log2(tmax / t0) / l2r
    return math.floor(e) + 1, abs(e - round(e)) * l2r


def test_max_size_empty_grid():
    g = torch.zeros((N, N, N, 4), dtype=torch.float32, device="cuda")
    P = vct.build_mips(g)
    assert P.levels == 11
    del g
    v = vct.View.from_host(_view())
    vct.trace([P], [v], _params())
    torch.cuda.synchronize()
    assert torch.all(v.out_diffuse == 0) and torch.all(v.out_specular == 0)
    assert torch.all(v.out_visibility == 1)
    del P, v
    torch.cuda.empty_cache()


def test_max_size_homogeneous_medium_forward_and_adjoint_sums():
    prm = _params()
    g = torch.empty((N, N, N, 4), dtype=torch.float32, device="cuda")
    g[..., 0], g[..., 1], g[..., 2], g[..., 3] = C0[0], C0[1], C0[2], A
    P = vct.build_mips(g)
    # every level of a constant grid is that constant (read levels 2..10)
    want = torch.tensor([*C0, A], device="cuda")
    for l in range(2, P.levels):
        lv = vct.read_level(P, l)
        assert torch.equal(lv, want.expand_as(lv)), l
        del lv

    hv = _view()
    npx = hv["width"]
    v = vct.View.from_host(hv)
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    vct.trace([P], [v], prm, workspace=ws)
    torch.cuda.synchronize()
    kd, md = _steps(prm["diffuse_aperture"], prm)
    ks, ms = _steps(prm["spec_aperture_min"], prm)
    ko, mo = _steps(prm["occ_aperture"], prm)
    assert min(md, ms, mo) > 1e-5, (md, ms, mo)  # no cone ends near t_max
    ad, as_, ao = (1.0 - (1.0 - A) ** k for k in (kd, ks, ko))
    wsum = float(np.sum(np.asarray(prm["diffuse_weight"], np.float64)[:prm["n_diffuse"]]))
    D = v.out_diffuse.double().cpu().numpy()
    S = v.out_specular.double().cpu().numpy()
    Vis = v.out_visibility.double().cpu().numpy()
    wantD = wsum * np.array([C0[0] * ad, C0[1] * ad, C0[2] * ad, ad])
    wantS = np.array([C0[0] * as_, C0[1] * as_, C0[2] * as_, as_])
    assert np.allclose(D, wantD, rtol=1e-5, atol=0), np.abs(D / wantD - 1).max()
    assert np.allclose(S, wantS, rtol=1e-5, atol=0), np.abs(S / wantS - 1).max()
    assert np.allclose(Vis, (1.0 - A) ** ko, rtol=1e-5, atol=0)
    st = vct.read_stats(ws)
    assert st["samples"] == [npx * prm["n_diffuse"] * kd, npx * ks, npx * ko], (st, kd, ks, ko)

    # adjoint: L = sum_px (D.r + D.a + S.g + S.a + Vis)
    gD = torch.zeros((npx, 4), device="cuda")
    gD[:, 0] = 1.0
    gD[:, 3] = 1.0
    gS = torch.zeros((npx, 4), device="cuda")
    gS[:, 1] = 1.0
    gS[:, 3] = 1.0
    gV = torch.ones(npx, device="cuda")
    grad = torch.zeros_like(g)
    del g
    torch.cuda.empty_cache()
    vct.trace_backward(P, [v], [(gD, gS, gV)], prm, grad_level0=grad)
    sums = grad.sum(dim=(0, 1, 2), dtype=torch.float64).cpu().numpy()
    del grad, P, v
    torch.cuda.empty_cache()
    # d alpha / d a under a uniform shift, per cone kind: K (1 - a)^(K - 1)
    dd, ds, do = (k * (1.0 - A) ** (k - 1) for k in (kd, ks, ko))
    # opacity channel: D.r = wsum c0r alpha_d and D.a = wsum alpha_d depend on
    # a; S.g = c0g alpha_s and S.a = alpha_s; Vis = 1 - alpha_o
    want_a = npx * (wsum * (C0[0] + 1.0) * dd + (C0[1] + 1.0) * ds - do)
    want_r = npx * wsum * ad          # d/dc0r of D.r
    want_g = npx * as_                # d/dc0g of S.g
    assert abs(sums[3] - want_a) <= 1e-4 * abs(want_a), (sums[3], want_a)
    assert abs(sums[0] - want_r) <= 1e-4 * abs(want_r), (sums[0], want_r)
    assert abs(sums[1] - want_g) <= 1e-4 * abs(want_g), (sums[1], want_g)
    assert abs(sums[2]) <= 1e-6 * abs(want_r)
