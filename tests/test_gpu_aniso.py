"""Anisotropic mips (VCT_LAYOUT_ANISO, Villegas' anisotropic filtering,
Ch. 5.1) on the CUDA path against the oracle: every directional volume of
every level, and the direction-weighted trace."""
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


def aniso_gpu(grid):
    return vct.build_mips(torch.from_numpy(np.ascontiguousarray(grid, np.float32)).cuda(),
                          layout="aniso")


@pytest.mark.parametrize("n", [2, 8, 32])
def test_aniso_levels_match_oracle(n):
    rng = np.random.default_rng(n)
    g = rng.random((n, n, n, 4)).astype(np.float32)
    g[rng.random((n, n, n)) < 0.4] = 0.0  # empty voxels: alpha-0 pairs
    P = aniso_gpu(g)
    O = oracle.build_mips_aniso(g)
    assert np.array_equal(vct.read_level(P, 0).cpu().numpy(), g)
    for l in range(1, P.levels):
        for d in range(6):
            got = vct.read_volume(P, l, d).cpu().numpy().astype(np.float64)
            want = O.level(l, d)
            assert np.allclose(got, want, rtol=2e-6, atol=1e-7), (n, l, d,
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
    v = vct.View.from_host(view)
    vct.trace([P], [v], prm)
    with pytest.raises(vct.VctError) as e:
        vct.trace_backward(P, [v], [(v.out_diffuse, None, None)], prm)
    assert e.value.status == vct._abi.VCT_ERR_UNSUPPORTED
    w = vct.View.from_host(dict(view, pyramid=1))
    with pytest.raises(vct.VctError) as e:
        vct.trace([P, D], [vct.View.from_host(view), w], prm)
    assert e.value.status == vct._abi.VCT_ERR_UNSUPPORTED
    with pytest.raises(vct.VctError):
        vct.Pyramid(32, dtype="f16", layout="aniso")
