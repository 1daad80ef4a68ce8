"""Anisotropic mips (VCT_LAYOUT_ANISO, Villegas' anisotropic filtering,
Ch. 5.1) on the CUDA path against the oracle: every directional volume of
every level, the direction-weighted trace, and the adjoint through both."""
import numpy as np
import pytest
import torch

import oracle
import paper_2104_00618_gb300 as vct
import vct_synth as vs
from gpu_cases import FP32_BOUND, room_case
from metrics import report

pytestmark = pytest.mark.gpu

OCC, GRACE, FIRST, SHADE = (vct.FLAG_OCC_SMOOTH, vct.FLAG_SPEC_GRACE,
                            vct.FLAG_DIFFUSE_FIRST_HIT, vct.FLAG_SHADE)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vct.lib()


def aniso_gpu(grid, offset16=False):
    """Anisotropic pyramid of a grid; offset16: level 0 placed 16 bytes past a
    32-byte boundary (the build then takes its one-launch-per-level path
    instead of the streaming kernel, which wants 32-byte alignment)."""
    g = torch.from_numpy(np.ascontiguousarray(grid, np.float32)).cuda()
    if offset16:
        buf = torch.empty(g.numel() + 8, dtype=torch.float32, device="cuda")
        assert buf.data_ptr() % 32 == 0
        g2 = buf[4:4 + g.numel()].view(g.shape)
        g2.copy_(g)
        g = g2
    return vct.build_mips(g, layout="aniso")


@pytest.mark.parametrize("n,offset16", [(2, False), (8, False), (32, False), (64, False),
                                        (128, False), (64, True)])
def test_aniso_levels_match_oracle(n, offset16):
    rng = np.random.default_rng(n)
    g = rng.random((n, n, n, 4)).astype(np.float32)
    g[rng.random((n, n, n)) < 0.4] = 0.0  # empty voxels: alpha-0 pairs
    P = aniso_gpu(g, offset16)
    O = oracle.build_mips_aniso(g)
    assert np.array_equal(vct.read_level(P, 0).cpu().numpy(), g)
    for l in range(1, P.levels):
        for d in range(6):
            got = vct.read_volume(P, l, d).cpu().numpy().astype(np.float64)
            want = O.level(l, d)
            assert np.allclose(got, want, rtol=2e-6, atol=1e-7), (n, offset16, l, d,
                                                                  np.abs(got - want).max())
    dense = vct.build_mips(torch.from_numpy(g).cuda())
    print("aniso / dense bytes:", P.storage.numel() / dense.storage.numel())


@pytest.mark.parametrize("flags", [0, OCC | GRACE | FIRST | SHADE])
@pytest.mark.parametrize("shape", [(16, 16, 1), (8, 8, 2), (4, 8, 4), (8, 4, 8)])
def test_aniso_trace_matches_oracle(flags, shape):
    """Room scene, ragged 131x77 view, roughness, 10 % masked: D, S, Vis
    within the FP32 bound of the oracle on the same anisotropic pyramid."""
    scene, view, prm0 = room_case(n=64, width=131, height=77)
    prm = vs.variant_params(prm0, flags) if flags else prm0
    if flags & SHADE:
        view = dict(view, albedo=vs.albedo(131, 77, 3))
    P = aniso_gpu(scene["grid"])
    v = vct.View.from_host(view, outputs=False)
    v.alloc_outputs(radiance=bool(flags & SHADE))
    vct.trace([P], [v], prm, cfg=vct.launch_config(*shape))
    torch.cuda.synchronize()
    ref = oracle.trace(oracle.build_mips_aniso(scene["grid"]), view, prm)
    outs = {"D": v.out_diffuse, "S": v.out_specular, "Vis": v.out_visibility}
    if flags & SHADE:
        outs["L"] = v.out_radiance
    m = view["mask"] != 0
    for k, t in outs.items():
        g = t.cpu().numpy()
        sel = m
        if k == "Vis":
            # a cone whose transmittance falls below 2^-24 stops in float32
            # (1 - T rounds to 1) while the FP64 march goes on: both values are
            # then below 6e-8 and count as the same opaque result
            sel = m & ~((g < 6e-8) & (ref["Vis"] < 6e-8))
        e = report(g[sel], ref[k][sel])[0].max()
        # a first-hit decision on the threshold may go either way
        if flags & FIRST and e > FP32_BOUND:
            assert ref["hit_margin"] < 1e-5, (k, e)
            continue
        assert e <= FP32_BOUND, (k, e)


def test_aniso_room_1080p_sampled():
    """The 256^3 room at 1920x1080 with an anisotropic pyramid: 20000 seeded
    pixels against the oracle; the anisotropic trace is slower than the
    isotropic one (three volumes per coarse sample) and differs from it."""
    c = vs.config_room_1080p()
    scene, view, prm = c["scenes"][0], c["views"][0], c["params"]
    P = aniso_gpu(scene["grid"])
    v = vct.View.from_host(view)
    vct.trace([P], [v], prm)
    torch.cuda.synchronize()
    rng = np.random.default_rng(321)
    idx = np.sort(rng.choice(view["width"] * view["height"], 20000, replace=False))
    ref = oracle.trace(oracle.build_mips_aniso(scene["grid"]), view, prm, idx=idx)
    for k, t in (("D", v.out_diffuse), ("S", v.out_specular), ("Vis", v.out_visibility)):
        g = t.cpu().numpy()[idx]
        sel = ~((g < 6e-8) & (ref[k] < 6e-8)) if k == "Vis" else slice(None)
        e = report(g[sel], ref[k][sel])[0].max()
        print("aniso 1080p", k, e)
        assert e <= FP32_BOUND, (k, e)
    iso = vct.View.from_host(view)
    vct.trace([vct.build_mips(torch.from_numpy(scene["grid"]).cuda())], [iso], prm)
    assert not torch.equal(iso.out_diffuse, v.out_diffuse)


def test_aniso_refusals():
    scene, view, prm = room_case(n=32, width=20, height=16)
    P = aniso_gpu(scene["grid"])
    D = vct.build_mips(torch.from_numpy(scene["grid"]).cuda())
    w = vct.View.from_host(dict(view, pyramid=1))
    with pytest.raises(vct.VctError) as e:
        vct.trace([P, D], [vct.View.from_host(view), w], prm)
    assert e.value.status == vct._abi.VCT_ERR_UNSUPPORTED
    with pytest.raises(vct.VctError):
        vct.Pyramid(32, dtype="f16", layout="aniso")


# ---------------------------------------------------------------------------
# the adjoint through an anisotropic pyramid
# ---------------------------------------------------------------------------
def _aniso_diff_case(n=32, W=48, H=40, seed=81):
    """Two views of a box room; a learnable grid of random colours and
    opacities in [0.05, 0.3] (every pair composite smooth, no cone saturates)."""
    import math
    gt = vs.box_scene(n, 6, seed, room=True)
    rng = np.random.default_rng(seed + 1)
    views = [vs.interior_view(gt, W, H, rng, with_roughness=True) for _ in range(2)]
    dirs, w = vs.cone_table_ring6()
    prm = vs.trace_params(dirs, w, math.radians(60), spec_enable=True,
                          spec_aperture_min=math.radians(10),
                          spec_aperture_max=math.radians(40), occ_enable=True, occ_aperture=0.55,
                          light=gt["light"])
    learn = np.empty((n, n, n, 4), np.float32)
    learn[..., :3] = rng.uniform(0.0, 1.0, (n, n, n, 3))
    learn[..., 3] = rng.uniform(0.05, 0.3, (n, n, n))
    return gt, views, prm, learn


def _aniso_ref(gt, views, prm, learn):
    O_gt = oracle.build_mips_aniso(gt["grid"])
    O = oracle.build_mips_aniso(learn)
    grad_ref = np.zeros(learn.shape)
    gpu_grads = []
    for v in views:
        t, r = oracle.trace(O_gt, v, prm), oracle.trace(O, v, prm)
        gD, gS, gV = r["D"] - t["D"], r["S"] - t["S"], r["Vis"] - t["Vis"]
        grad_ref += oracle.trace_backward(O, v, prm, gD, gS, gV)
        gpu_grads.append(tuple(torch.from_numpy(a.astype(np.float32)).cuda()
                               for a in (gD, gS, gV)))
    return grad_ref, gpu_grads


def _check_grad(grad, grad_ref, what):
    scale = np.abs(grad_ref).max()
    err = np.abs(grad - grad_ref)
    print(what, "max abs err / max |grad| =", err.max() / scale)
    assert err.max() <= 1e-4 * scale
    assert np.linalg.norm(grad - grad_ref) <= 1e-5 * np.linalg.norm(grad_ref)


@pytest.mark.parametrize("flags", [0, vct.FLAG_OCC_SMOOTH | vct.FLAG_SPEC_GRACE
                                   | vct.FLAG_PREMULTIPLIED])
@pytest.mark.parametrize("lpp", [1, 4])
def test_aniso_backward_matches_oracle(flags, lpp):
    """dL/d(level 0) through the anisotropic build and the direction-weighted
    trace against the FP64 adjoint (oracle), plain and with modified cones."""
    gt, views, prm, learn = _aniso_diff_case()
    if flags:
        prm = dict(vs.variant_params(prm, flags), occ_max_dist=1.0)
    grad_ref, gpu_grads = _aniso_ref(gt, views, prm, learn)
    P = aniso_gpu(learn)
    gviews = [vct.View.from_host(v) for v in views]
    grad = vct.trace_backward(P, gviews, gpu_grads, prm, cfg=vct.launch_config(8, 8, lpp))
    _check_grad(grad.cpu().numpy().astype(np.float64), grad_ref, f"aniso flags {flags} lpp {lpp}")
    iso = vct.trace_backward(vct.build_mips(torch.from_numpy(learn).cuda()), gviews, gpu_grads,
                             prm)
    assert not torch.allclose(iso, grad, rtol=1e-3, atol=1e-6)


def test_aniso_backward_deterministic():
    """The reproducible adjoint of an anisotropic pyramid: identical bits on
    every run, within the fixed-point rounding of the float adjoint."""
    gt, views, prm, learn = _aniso_diff_case()
    grad_ref, gpu_grads = _aniso_ref(gt, views, prm, learn)
    P = aniso_gpu(learn)
    gviews = [vct.View.from_host(v) for v in views]
    runs = [vct.trace_backward(P, gviews, gpu_grads, prm, deterministic=True) for _ in range(3)]
    assert all(torch.equal(runs[0], r) for r in runs[1:])
    flt = vct.trace_backward(P, gviews, gpu_grads, prm).cpu().numpy()
    det = runs[0].cpu().numpy().astype(np.float64)
    assert np.abs(det - flt).max() <= 1e-5 * np.abs(grad_ref).max()
    _check_grad(det, grad_ref, "aniso deterministic")


def test_aniso_render_autograd():
    """torch.autograd through render(layout="aniso"): the forward records the
    per-cone state, the adjoint starts its reverse walk from it; the gradient
    of an L2 loss equals the oracle's."""
    gt, views, prm, learn = _aniso_diff_case(seed=83)
    view = views[0]
    O_gt = oracle.build_mips_aniso(gt["grid"])
    t = oracle.trace(O_gt, view, prm)
    grid = torch.from_numpy(learn).cuda().requires_grad_()
    D, S, V = vct.render(grid, vct.View.from_host(view, outputs=False), prm, layout="aniso")
    tD, tS, tV = (torch.from_numpy(t[k].astype(np.float32)).cuda() for k in ("D", "S", "Vis"))
    loss = 0.5 * (((D - tD) ** 2).sum() + ((S - tS) ** 2).sum() + ((V - tV) ** 2).sum())
    loss.backward()
    O = oracle.build_mips_aniso(learn)
    r = oracle.trace(O, view, prm)
    grad_ref = oracle.trace_backward(O, view, prm, r["D"] - t["D"], r["S"] - t["S"],
                                     r["Vis"] - t["Vis"])
    _check_grad(grid.grad.cpu().numpy().astype(np.float64), grad_ref, "aniso render")
