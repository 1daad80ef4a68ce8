"""The thesis's modified cones (Ch. 5.4.4) and the shading epilogue (Ch. 3.3,
Ch. 4.2.2, Ch. 5.4.4) on the CUDA path against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2104_00618_gb300 as vct
import vct_synth as vs
from gpu_cases import FP32_BOUND, MIN_STEP_MARGIN, gpu_pyramid, room_case
from metrics import report

pytestmark = pytest.mark.gpu

OCC, GRACE, FIRST, SHADE, IMPL, PREMUL = (vct.FLAG_OCC_SMOOTH, vct.FLAG_SPEC_GRACE,
                                          vct.FLAG_DIFFUSE_FIRST_HIT, vct.FLAG_SHADE,
                                          vct.FLAG_SHADE_IMPL, vct.FLAG_PREMULTIPLIED)
TIE = 1e-5  # |a_s - 1/100| below this: either first-hit decision is correct


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vct.lib()


def variant_params(prm, flags):
    return vs.variant_params(prm, flags)


def with_albedo(view, seed):
    return dict(view, albedo=vs.albedo(view["width"], view["height"], seed))


def run_gpu(pyr, view_host, prm, cfg=None):
    v = vct.View.from_host(view_host, outputs=False)
    v.alloc_outputs(radiance=bool(prm.get("flags", 0) & SHADE))
    ws = vct.trace([pyr], [v], prm, cfg=cfg)
    torch.cuda.synchronize()
    out = {"D": v.out_diffuse.cpu().numpy(), "S": v.out_specular.cpu().numpy(),
           "Vis": v.out_visibility.cpu().numpy()}
    if v.out_radiance is not None:
        out["L"] = v.out_radiance.cpu().numpy()
    return out, vct.read_stats(ws)


def pixel_errors(gpu, ref):
    """Per-pixel floored relative error (max over channels), tau per channel
    = 1e-3 * max |oracle| of that channel."""
    g = np.asarray(gpu, dtype=np.float64)
    o = np.asarray(ref, dtype=np.float64)
    if o.ndim == 1:
        g, o = g[:, None], o[:, None]
    tau = np.maximum(1e-3 * np.abs(o).max(axis=0), 1e-30)
    return (np.abs(g - o) / np.maximum(np.abs(o), tau)).max(axis=1)


def check_against_oracle(out, ref, prm, O, view, idx=None):
    """Every output within the FP32 bound except pixels that the oracle itself
    shows to be near-ties: a first-hit decision with |a_s - 1/100| < TIE, or
    a cone whose last step lies within MIN_STEP_MARGIN (relative) of t_max,
    where the float32 step schedule may take one sample more or less."""
    keys = ["D"] + (["S"] if prm["spec_enable"] else []) + \
        (["Vis"] if prm["occ_enable"] else []) + (["L"] if "L" in ref else [])
    sel = slice(None) if idx is None else idx
    bad = np.zeros(len(ref["D"]), dtype=bool)
    for k in keys:
        bad |= pixel_errors(out[k][sel], ref[k]) > FP32_BOUND
    bad_px = np.flatnonzero(bad) if idx is None else np.asarray(idx)[bad]
    ties = 0
    for p in bad_px:
        r = oracle.trace(O, view, prm, idx=[p])
        hit_tie = bool(prm["flags"] & FIRST) and r["hit_margin"] < TIE
        assert hit_tie or r["margin"] < MIN_STEP_MARGIN, (
            "pixel", int(p), {k: float(pixel_errors(out[k][[p]], r[k])[0]) for k in keys})
        ties += 1
    assert ties <= 0.002 * len(ref["D"]), ties
    good = ~bad
    res = {k: report(out[k][sel][good], ref[k][good])[0] for k in keys}
    return res, ties


_CASE = {}


def _case():
    if "c" not in _CASE:
        scene, view, prm = room_case()
        view = with_albedo(view, 5)
        _CASE["c"] = (scene, view, prm, oracle.build_mips(scene["grid"]))
    return _CASE["c"]


FLAG_SETS = [OCC, GRACE, FIRST, SHADE, SHADE | IMPL, PREMUL, OCC | GRACE | FIRST | SHADE,
             OCC | GRACE | FIRST | SHADE | IMPL, PREMUL | OCC | GRACE | SHADE]


@pytest.mark.parametrize("flags", FLAG_SETS)
@pytest.mark.parametrize("shape", [(16, 16, 1), (8, 8, 2), (4, 8, 4), (8, 4, 8)])
def test_variants_room_ragged(flags, shape):
    """Room scene, ragged 203x117 view, roughness, 10% masked, albedo: each
    variant (and all together) under launch shapes with 1, 2, 4, 8 lanes per
    pixel (one lane per pixel defers and sorts the specular cones)."""
    scene, view, prm0, O = _case()
    prm = variant_params(prm0, flags)
    key = ("ref", flags)
    if key not in _CASE:
        _CASE[key] = oracle.trace(O, view, prm)
    ref = _CASE[key]
    P = gpu_pyramid(scene["grid"])
    out, stats = run_gpu(P, view, prm, cfg=vct.launch_config(*shape))
    res, ties = check_against_oracle(out, ref, prm, O, view)
    print(flags, shape, "ties", ties, {k: float(v.max()) for k, v in res.items()})
    m = view["mask"] == 0
    if flags & SHADE:
        assert np.all(out["L"][m] == 0)
        assert np.all(out["L"][~m][:, 3] == 1)
    assert stats["cones"] == [int(ref["cones"][k]) for k in range(3)]


def test_variants_change_the_result():
    """Each variant changes its own output (guards against a flag that is
    silently ignored) and leaves the others as they were."""
    scene, view, prm0, O = _case()
    P = gpu_pyramid(scene["grid"])
    base, _ = run_gpu(P, view, variant_params(prm0, 0))
    m = view["mask"] != 0
    for flags, changed in [(OCC, "Vis"), (GRACE, "S"), (FIRST, "D")]:  # (PREMUL changes D and S)
        out, _ = run_gpu(P, view, variant_params(prm0, flags))
        for k in ("D", "S", "Vis"):
            err = pixel_errors(out[k][m], base[k][m]).max()
            if k == changed:
                assert err > 1e-2, (flags, k, err)
            else:  # another kernel instance: same arithmetic up to contraction
                assert err < 1e-6, (flags, k, err)


def test_shading_without_albedo_and_with_unit_ratios():
    """L_vxct with albedo 1, kd = ks = 1 reduces to D + S + Vis * direct;
    L_impl to Vis D + S + Vis direct (checked on the GPU's own D, S, Vis
    against its L, and against the oracle)."""
    scene, view, prm0 = room_case(n=32, width=61, height=35, seed=3)
    P = gpu_pyramid(scene["grid"])
    O = oracle.build_mips(scene["grid"])
    for flags in (SHADE, SHADE | IMPL):
        prm = dict(prm0, flags=flags, shininess=16.0, diffuse_str=1.0, specular_str=1.0,
                   light_color=(1.0, 1.0, 1.0))
        out, _ = run_gpu(P, view, prm)
        ref = oracle.trace(O, view, prm)
        res, ties = check_against_oracle(out, ref, prm, O, view)
        assert ties == 0
        m = view["mask"] != 0
        # L - (combination of the indirect terms) = Vis * direct >= 0
        D, S, V, L = out["D"][m], out["S"][m], out["Vis"][m], out["L"][m]
        ind = (V[:, None] * D[:, :3] + S[:, :3]) if flags & IMPL else (D[:, :3] + S[:, :3])
        assert np.all(L[:, :3] - ind >= -1e-5)


def test_variants_room_1080p_sampled():
    """The 256^3 room at 1920x1080 with every variant and L_vxct shading, in
    the default launch shape; 20000 seeded pixels against the oracle."""
    c = vs.config_room_1080p()
    prm0, scene = c["params"], c["scenes"][0]
    view = with_albedo(c["views"][0], 11)
    prm = variant_params(prm0, OCC | GRACE | FIRST | SHADE)
    P = gpu_pyramid(scene["grid"])
    out, stats = run_gpu(P, view, prm)
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(view["width"] * view["height"], 20000, replace=False))
    O = oracle.build_mips(scene["grid"])
    ref = oracle.trace(O, view, prm, idx=idx)
    res, ties = check_against_oracle(out, ref, prm, O, view, idx=idx)
    print("1080p variants:", "ties", ties, {k: float(v.max()) for k, v in res.items()})
    for k, v in res.items():
        assert v.max() <= FP32_BOUND, (k, v)


def test_variants_fp16_storage_report():
    """FP16 storage with every variant: error reported against the oracle on
    the FP32 grid (the storage rounding dominates)."""
    scene, view, prm0, O = _case()
    prm = variant_params(prm0, OCC | GRACE | SHADE)
    P = gpu_pyramid(scene["grid"], dtype="f16")
    out, _ = run_gpu(P, view, prm)
    ref = oracle.trace(O, view, prm)
    errs = {k: float(report(out[k], ref[k])[0].max()) for k in ("D", "S", "Vis", "L")}
    print("fp16 variants:", errs)
    assert max(errs.values()) < 5e-3, errs


@pytest.mark.parametrize("flags", [OCC, GRACE, FIRST, PREMUL, OCC | GRACE | FIRST | PREMUL])
@pytest.mark.parametrize("lpp", [1, 4])
def test_variant_adjoint_matches_oracle(flags, lpp):
    """Adjoint of the modified cones and of premultiplied compositing on the
    box room (roughness, 10 % masked) against the FP64 adjoint, for seeded
    upstream gradients; with 4 lanes per pixel one warp mixes cone kinds.
    The forward's per-cone state gives the same gradient as the re-march.
    Pixels whose first-hit decision the oracle shows to be a near-tie get a
    zero upstream gradient (either decision is correct there)."""
    seed = 3
    scene, view, prm0 = room_case(n=32, width=30, height=20, seed=seed)
    prm = dict(variant_params(prm0, flags), occ_max_dist=0.5)
    O = oracle.build_mips(scene["grid"])
    rng = np.random.default_rng(seed + 50)
    npx = view["width"] * view["height"]
    gD, gS, gV = rng.normal(size=(npx, 4)), rng.normal(size=(npx, 4)), rng.normal(size=npx)
    if flags & FIRST:
        ties = [p for p in range(npx) if oracle.trace(O, view, prm, idx=[p])["hit_margin"] < TIE]
        gD[ties], gS[ties], gV[ties] = 0.0, 0.0, 0.0
        assert len(ties) < 0.05 * npx, len(ties)
    ref = oracle.trace_backward(O, view, prm, gD, gS, gV)
    P = gpu_pyramid(scene["grid"])
    cuda = [torch.from_numpy(a.astype(np.float32)).cuda() for a in (gD, gS, gV)]
    cfg = vct.launch_config(8, 8, lpp)
    grads = []
    for with_state in (False, True):
        v = vct.View.from_host(view)
        if with_state:
            v.alloc_cone_state(prm)
            vct.trace([P], [v], prm, cfg=cfg)
        grads.append(vct.trace_backward(P, [v], [tuple(cuda)], prm, cfg=cfg).cpu().numpy())
    g = grads[0].astype(np.float64)
    scale = np.abs(ref).max()
    err = np.abs(g - ref)
    print(f"flags {flags} lpp {lpp}: max abs err / max |grad| = {err.max() / scale:.3g}")
    assert scale > 0
    assert err.max() <= 1e-4 * scale
    assert np.linalg.norm(g - ref) <= 1e-5 * np.linalg.norm(ref)
    assert np.abs(grads[1] - grads[0]).max() <= 1e-6 * scale
    if flags & FIRST:  # the first-hit cones add nothing to the opacity channel
        only_d = oracle.trace_backward(O, view, prm, gD, np.zeros_like(gS), np.zeros(npx))
        assert not np.any(only_d[..., 3])


@pytest.mark.parametrize("flags", [SHADE, SHADE | IMPL, SHADE | IMPL | OCC | GRACE | PREMUL])
def test_shading_adjoint_matches_oracle(flags):
    """dL/d(shaded radiance) passed down through the shading epilogue (L_vxct
    and L_impl) together with dL/dD, against the FP64 adjoint; L_impl reads
    the forward's D and Vis from the view's outputs."""
    scene, view, prm0 = room_case(n=32, width=30, height=20, seed=4)
    view = with_albedo(view, 9)
    prm = dict(variant_params(prm0, flags), occ_max_dist=0.5)
    O = oracle.build_mips(scene["grid"])
    rng = np.random.default_rng(77)
    npx = view["width"] * view["height"]
    gD, gL = rng.normal(size=(npx, 4)), rng.normal(size=(npx, 4))
    gL[:, 3] = 0.0
    z4, z1 = np.zeros((npx, 4)), np.zeros(npx)
    ref = oracle.trace_backward(O, view, prm, gD, z4, z1, gL=gL)
    P = gpu_pyramid(scene["grid"])
    v = vct.View.from_host(view, outputs=False)
    v.alloc_outputs(radiance=True)
    vct.trace([P], [v], prm)
    cuda = [torch.from_numpy(a.astype(np.float32)).cuda() for a in (gD, gL)]
    g = vct.trace_backward(P, [v], [(cuda[0], None, None, cuda[1])], prm).cpu().numpy()
    scale = np.abs(ref).max()
    err = np.abs(g.astype(np.float64) - ref)
    print(f"shading flags {flags}: max abs err / max |grad| = {err.max() / scale:.3g}")
    assert scale > 0 and err.max() <= 1e-4 * scale
    assert np.linalg.norm(g - ref) <= 1e-5 * np.linalg.norm(ref)
    # without the shading flag the radiance gradient is refused
    with pytest.raises(vct.VctError):
        vct.trace_backward(P, [v], [(cuda[0], None, None, cuda[1])], prm0)
