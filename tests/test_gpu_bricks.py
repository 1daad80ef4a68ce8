"""Brick storage (VCT_LAYOUT_BRICKS): the same texel values as the dense
pyramid with the empty 8^3 bricks left out, hence the same trace outputs."""
import numpy as np
import pytest
import torch

import oracle
import paper_2104_00618_gb300 as vct
import vct_synth as vs
from gpu_cases import FP32_BOUND, room_case
from metrics import report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vct.lib()


def sparse_grid(n, seed, boxes=6):
    """Mostly empty grid: a few boxes of random values, one negative-valued
    texel (occupied although its brick's mean may vanish one level up)."""
    rng = np.random.default_rng(seed)
    g = np.zeros((n, n, n, 4), np.float32)
    for _ in range(boxes):
        s = rng.integers(1, max(2, n // 6), size=3)
        lo = rng.integers(0, n - s + 1)
        g[lo[2]:lo[2] + s[2], lo[1]:lo[1] + s[1], lo[0]:lo[0] + s[0]] = rng.random(4)
    g[n - 1, 0, n // 2] = (-0.5, 0.25, 0.0, 0.0)
    return g


def numpy_occupied(g, levels):
    """Occupied bricks per bricked level from the definition: a level-0
    brick holds a non-zero channel; a coarser brick has an occupied child."""
    n = g.shape[0]
    if n < 16:
        return []
    b = n // 8
    occ = [np.abs(g).reshape(b, 8, b, 8, b, 8, 4).max(axis=(1, 3, 5, 6)) > 0]
    for l in range(1, levels):
        if (n >> l) < 16:
            break
        o = occ[-1]
        m = o.shape[0] // 2
        occ.append(o.reshape(m, 2, m, 2, m, 2).any(axis=(1, 3, 5)))
    return [int(o.sum()) for o in occ]


@pytest.mark.parametrize("n", [16, 64, 256])
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_brick_levels_equal_dense(n, dtype):
    g = sparse_grid(n, n)
    level0 = torch.from_numpy(g).cuda()
    dense = vct.build_mips(level0, dtype=dtype)
    occ, nbytes = vct.plan_bricks(level0, dtype=dtype)
    bricks = vct.build_mips(level0, dtype=dtype, layout="bricks")
    vct.pyramid_status(bricks)
    assert occ == sum(numpy_occupied(g, dense.levels)) == bricks.occupied_bricks()
    assert bricks.storage.numel() == nbytes < dense.storage.numel()
    for l in range(dense.levels):
        a = vct.read_level(dense, l).cpu().numpy()
        b = vct.read_level(bricks, l).cpu().numpy()
        assert np.array_equal(a, b), (n, dtype, l)


def test_brick_trace_equals_dense_all_shapes_and_variants():
    scene, view, prm = room_case(n=64, width=131, height=77)
    level0 = torch.from_numpy(scene["grid"]).cuda()
    dense = vct.build_mips(level0)
    bricks = vct.build_mips(level0, layout="bricks")
    ref = oracle.trace(oracle.build_mips(scene["grid"]), view, prm)
    for flags in (0, vct.FLAG_OCC_SMOOTH | vct.FLAG_DIFFUSE_FIRST_HIT | vct.FLAG_SPEC_GRACE):
        p = vs.variant_params(prm, flags) if flags else prm
        for shape in [(16, 16, 1), (8, 8, 2), (4, 8, 4), (8, 4, 8)]:
            outs = []
            for P in (dense, bricks):
                v = vct.View.from_host(view)
                vct.trace([P], [v], p, cfg=vct.launch_config(*shape))
                outs.append([t.cpu().numpy() for t in (v.out_diffuse, v.out_specular,
                                                       v.out_visibility)])
            for a, b in zip(*outs):
                assert np.array_equal(a, b), (flags, shape)
        if not flags:
            for k, o in zip(("D", "S", "Vis"), outs[1]):
                assert report(o, ref[k])[0].max() <= FP32_BOUND, k


def test_mixed_layouts_in_one_call():
    scene_a, view_a, prm = room_case(n=64, width=64, height=48, seed=3)
    scene_b, view_b, _ = room_case(n=32, width=50, height=30, seed=4)
    view_b = dict(view_b, pyramid=1)
    Pa = vct.build_mips(torch.from_numpy(scene_a["grid"]).cuda(), layout="bricks")
    Pb = vct.build_mips(torch.from_numpy(scene_b["grid"]).cuda())
    vs_ = [vct.View.from_host(view_a), vct.View.from_host(view_b)]
    vct.trace([Pa, Pb], vs_, prm)
    for P, hv, v in ((Pa, view_a, vs_[0]), (Pb, dict(view_b, pyramid=0), vs_[1])):
        w = vct.View.from_host(hv)
        vct.trace([P], [w], prm)
        assert torch.equal(v.out_diffuse, w.out_diffuse)
        assert torch.equal(v.out_visibility, w.out_visibility)


def test_pool_too_small_is_reported():
    g = sparse_grid(64, 9)
    level0 = torch.from_numpy(g).cuda()
    occ, _ = vct.plan_bricks(level0)
    small = vct.Pyramid(64, layout="bricks", occupied=occ - 1)
    vct.build_mips(level0, out=small)
    with pytest.raises(vct.VctError) as e:
        vct.pyramid_status(small)
    assert e.value.status == vct._abi.VCT_ERR_WORKSPACE
    # every brick was left empty: level 0 reads as zeros
    assert not vct.read_level(small, 0).any()
    ok = vct.Pyramid(64, layout="bricks", occupied=occ)
    vct.build_mips(level0, out=ok)
    vct.pyramid_status(ok)


def test_backward_bricks_equals_dense():
    """The adjoint reads a brick pyramid's texels as the forward did: the
    gradient equals the dense pyramid's (up to the order of the float
    atomics), also with the forward's per-cone state."""
    g = sparse_grid(64, 21)
    scene, view, prm = room_case(n=64, width=40, height=28)
    level0 = torch.from_numpy(g).cuda()
    grads = {}
    for layout in ("dense", "bricks"):
        P = vct.build_mips(level0, layout=layout)
        v = vct.View.from_host(view).alloc_cone_state(prm)
        vct.trace([P], [v], prm)
        gr = [(v.out_diffuse * 0.5, v.out_specular, v.out_visibility - 0.25)]
        grads[layout] = vct.trace_backward(P, [v], gr, prm).cpu().numpy()
        grads[layout + "_det"] = vct.trace_backward(P, [v], gr, prm,
                                                    deterministic=True).cpu().numpy()
    a, b = grads["dense"], grads["bricks"]
    assert np.abs(a).max() > 0
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()
    assert np.array_equal(grads["dense_det"], grads["bricks_det"])


def test_voxelized_512_room_in_bricks():
    """The 512^3 room voxelized from its mesh (surface shells only): the brick
    pyramid takes a fraction of the dense one and traces the same frame."""
    scene = vs.box_scene(512, 32, 2, room=True)
    mesh = vct.Mesh.from_host(vs.scene_mesh(scene, tess=8, n_spheres=4, seed=102))
    level0 = vct.voxelize(mesh, 512, light={"light_dir": scene["light"]})
    dense = vct.build_mips(level0)
    bricks = vct.build_mips(level0, layout="bricks")
    vct.pyramid_status(bricks)
    ratio = bricks.storage.numel() / dense.storage.numel()
    print("512^3 bricks / dense bytes:", ratio, bricks.occupied_bricks())
    assert ratio < 0.5
    rng = np.random.default_rng(8)
    view = vs.interior_view(scene, 480, 270, rng)
    prm = vs.params_room9(scene["light"])
    outs = []
    for P in (dense, bricks):
        v = vct.View.from_host(view)
        vct.trace([P], [v], prm)
        outs.append((v.out_diffuse.cpu(), v.out_specular.cpu(), v.out_visibility.cpu()))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
