"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2104_00618_gb300 as vct
import vct_synth as vs
from gpu_cases import (FP32_BOUND, MIN_STEP_MARGIN, compare, gpu_pyramid, gpu_trace,
                       oracle_with_spec_ties, room_case,
                       worst)
from metrics import U16, check_fp16_outputs, report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vct.lib()


# ---------------------------------------------------------------------------
# a1 + a2: packing and mip build
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64, 128])
def test_mips_fp32_match_oracle(n):
    rng = np.random.default_rng(n)
    g = rng.random((n, n, n, 4)).astype(np.float32)
    P = gpu_pyramid(g)
    O = oracle.build_mips(g)
    vct.pyramid_status(P)
    for l in range(P.levels):
        got = vct.read_level(P, l).cpu().numpy().astype(np.float64)
        want = O.level(l)
        if l == 0:
            assert np.array_equal(got, want), "level 0 must round-trip exactly"
        else:
            assert np.max(np.abs(got - want) / np.abs(want).clip(1e-30)) < 2e-6, (n, l)


@pytest.mark.parametrize("n,levels", [(64, 3), (64, 5), (32, 1), (256, 9)])
def test_mips_partial_levels_and_large(n, levels):
    rng = np.random.default_rng(100 + n)
    g = (rng.random((n, n, n, 4)) * (rng.random((n, n, n, 1)) < 0.2)).astype(np.float32)
    P = gpu_pyramid(g, levels=levels)
    O = oracle.build_mips(g, levels=levels)
    for l in range(levels):
        got = vct.read_level(P, l).cpu().numpy().astype(np.float64)
        want = O.level(l)
        assert np.allclose(got, want, rtol=2e-6, atol=1e-12), (n, levels, l)


@pytest.mark.parametrize("n", [8, 64, 256])
def test_mips_fp16_within_rounding(n):
    rng = np.random.default_rng(200 + n)
    g = rng.random((n, n, n, 4)).astype(np.float32)
    P = gpu_pyramid(g, dtype="f16")
    O = oracle.build_mips(g)
    for l in range(P.levels):
        got = vct.read_level(P, l).cpu().numpy().astype(np.float64)
        want = O.level(l)
        # one rounding to binary16 of a float32 value computed from float32 values
        assert np.all(np.abs(got - want) <= 2.0 ** -11 * np.abs(want) + 1e-6 * np.abs(want)
                      + 2.0 ** -24), (n, l)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_mips_unaligned_grid_same_bits(dtype):
    """A level 0 that starts 16 bytes past a 32-byte boundary takes the TMA
    pack kernel instead of the streaming one (whose loads want 32-byte
    alignment): every level must come out bit for bit the same."""
    n = 64
    rng = np.random.default_rng(640)
    g = torch.from_numpy(rng.random((n, n, n, 4)).astype(np.float32)).cuda()
    buf = torch.empty(g.numel() + 8, dtype=torch.float32, device="cuda")
    assert buf.data_ptr() % 32 == 0
    g16 = buf[4:4 + g.numel()].view(g.shape)
    g16.copy_(g)
    a = vct.build_mips(g, dtype=dtype)
    b = vct.build_mips(g16, dtype=dtype)
    for l in range(a.levels):
        assert torch.equal(vct.read_level(a, l), vct.read_level(b, l)), (dtype, l)


def test_mips_mean_preserved_on_gpu():
    c = vs.config_small_fp32()
    g = c["scenes"][0]["grid"]
    P = gpu_pyramid(g)
    m0 = g.reshape(-1, 4).astype(np.float64).mean(0)
    for l in range(P.levels):
        lv = vct.read_level(P, l).cpu().numpy().astype(np.float64)
        assert np.allclose(lv.reshape(-1, 4).mean(0), m0, rtol=1e-6), l


# ---------------------------------------------------------------------------
# a3 - a6: the trace
# ---------------------------------------------------------------------------
def test_empty_grid_gives_no_indirect_light():
    scene, view, prm = room_case(n=32, width=40, height=24)
    P = gpu_pyramid(np.zeros((32, 32, 32, 4), np.float32))
    (D, S, V), _ = gpu_trace([P], [view], prm)[0][0], None
    assert np.all(D == 0) and np.all(S == 0) and np.all(V == 1.0)


def test_small_config_full_frame():
    """64^3, 12 boxes, 128x128 surface samples, 6x60deg + 10deg cones."""
    c = vs.config_small_fp32()
    prm = c["params"]
    view = c["views"][0]
    P = gpu_pyramid(c["scenes"][0]["grid"])
    O = oracle.build_mips(c["scenes"][0]["grid"])
    (out,), stats = gpu_trace([P], [view], prm)
    ref = oracle.trace(O, view, prm)
    res = compare(out, ref, prm=prm)
    print("small config errors (max, mean):", {k: (v[0].max(), v[1].max()) for k, v in res.items()})
    assert ref["margin"] > MIN_STEP_MARGIN, ref["margin"]
    assert worst(res) <= FP32_BOUND, res
    # Sample counts: float32 alpha rounds to exactly 1 (ending the march)
    # while the float64 alpha is still 1 - 1e-8 or so, so the GPU may take
    # fewer samples on saturated cones; the dropped terms are below 6e-8.
    for k in range(2):
        assert 0 <= ref["steps"][k] - stats["samples"][k] <= 0.01 * ref["steps"][k]
        assert stats["cones"][k] == ref["cones"][k]
    # the launch shape the library's tuner picks for this frame (the one the
    # benchmark times): the same outputs within the bound
    best = vct.autotune([P], [vct.View.from_host(view)], prm)
    (out2,), stats2 = gpu_trace([P], [view], prm, cfg=best)
    res2 = compare(out2, ref, prm=prm)
    assert worst(res2) <= FP32_BOUND, (best.tile_w, best.tile_h, best.lanes_per_pixel, res2)
    assert stats2["samples"] == stats["samples"] and stats2["cones"] == stats["cones"]


@pytest.mark.parametrize("tile", [(4, 8), (8, 8), (8, 16), (16, 16)])
@pytest.mark.parametrize("lpp", [1, 2, 4, 8])
def test_room_ragged_all_launch_shapes(tile, lpp):
    """Room scene, ragged 203x117 view, roughness, 10% masked, 9 diffuse +
    specular + occlusion cones, under every candidate launch shape."""
    scene, view, prm = _room_fixture()
    O = _room_oracle()
    P = gpu_pyramid(scene["grid"])
    (out,), stats = gpu_trace([P], [view], prm, cfg=vct.launch_config(*tile, lpp))
    res = compare(out, O, prm=prm)
    assert O["margin"] > MIN_STEP_MARGIN, O["margin"]
    assert worst(res) <= FP32_BOUND, (tile, lpp, res)
    m = view["mask"] == 0
    assert np.all(out[0][m] == 0) and np.all(out[1][m] == 0) and np.all(out[2][m] == 1)


_ROOM = {}


def _room_fixture():
    if "case" not in _ROOM:
        _ROOM["case"] = room_case()
    return _ROOM["case"]


def _room_oracle():
    if "ref" not in _ROOM:
        scene, view, prm = _room_fixture()
        _ROOM["ref"] = oracle.trace(oracle.build_mips(scene["grid"]), view, prm)
    return _ROOM["ref"]


def test_room_1080p_full_size_sampled():
    """The 256^3 room at 1920x1080 in the default launch shape; 20000 seeded
    pixels checked against the oracle one by one."""
    c = vs.config_room_1080p()
    prm, view, scene = c["params"], c["views"][0], c["scenes"][0]
    P = gpu_pyramid(scene["grid"])
    (out,), stats = gpu_trace([P], [view], prm)
    rng = np.random.default_rng(99)
    idx = np.sort(rng.choice(view["width"] * view["height"], 20000, replace=False))
    O = oracle.build_mips(scene["grid"])
    ref = oracle.trace(O, view, prm, idx=idx)
    res = compare(out, ref, idx=idx, prm=prm)
    print("1080p sampled errors:", {k: (v[0].max(), v[1].max()) for k, v in res.items()})
    assert ref["margin"] > MIN_STEP_MARGIN, ref["margin"]
    assert worst(res) <= FP32_BOUND, res
    total = sum(stats["samples"])
    assert total > 1e8
    assert stats["cones"] == [9 * view["mask"].sum(), view["mask"].sum(), view["mask"].sum()]


def test_fp16_storage_error_report():
    """Same scene as the small config with the pyramid stored in binary16;
    compositing stays float32.  Every output channel of every pixel lies
    within the binary16-storage bound (tests/metrics.py: one rounding of
    2^-11 per texel carried through the convex lerps and the compositing,
    plus the float32 path's own 1e-4), and the mean floored relative error
    stays below 2^-11."""
    c = vs.config_small_fp32()
    prm = dict(c["params"], occ_enable=1)
    view = c["views"][0]
    grid = c["scenes"][0]["grid"]
    P = gpu_pyramid(grid, dtype="f16")
    O = oracle.build_mips(grid)
    (out,), _ = gpu_trace([P], [view], prm)
    ref = oracle.trace(O, view, prm)
    c_max = grid[..., :3].reshape(-1, 3).max(axis=0)
    ratio, res = check_fp16_outputs(out, ref, c_max, k_max=150)
    print("fp16 storage errors (max, mean):", {k: (v[0].tolist(), v[1].tolist()) for k, v in res.items()},
          "worst |err| / bound:", ratio)
    assert max(float(v[1].max()) for v in res.values()) <= U16


def test_batched_views_over_several_pyramids():
    scenes = [vs.box_scene(n, 6, 300 + n, room=True) for n in (16, 64, 32)]
    rng = np.random.default_rng(5)
    views = []
    for i, (sc, (w, h)) in enumerate(zip(scenes * 2, [(37, 21), (64, 48), (17, 33),
                                                       (80, 9), (5, 5), (41, 40)])):
        v = vs.interior_view(sc, w, h, rng)
        v["pyramid"] = i % 3
        views.append(v)
    prm = vs.params_room9(scenes[0]["light"])
    pyrs = [gpu_pyramid(sc["grid"]) for sc in scenes]
    outs, stats = gpu_trace(pyrs, views, prm)
    for v, out in zip(views, outs):
        O = oracle.build_mips(scenes[v["pyramid"]]["grid"])
        ref = oracle.trace(O, v, prm)
        res = compare(out, ref, prm=prm)
        assert worst(res) <= FP32_BOUND, res


@pytest.mark.parametrize("tile", [(8, 16), (16, 16), (4, 8)])
def test_multi_view_partial_tile_rows(tile):
    """Views whose height the tile height does not divide, large enough that
    the first ones lie outside the launch's small-tile tail: every pixel is
    traced (one specular cone each) and matches the oracle, including the
    last, partial row of tiles of each view."""
    scene = vs.box_scene(32, 6, 12, room=True)
    rng = np.random.default_rng(13)
    hv = [vs.interior_view(scene, 500, h, rng) for h in (333, 301, 250, 77)]
    prm = vs.params_room9(scene["light"])
    P = gpu_pyramid(scene["grid"])
    outs, stats = gpu_trace([P], hv, prm, cfg=vct.launch_config(*tile, 1))
    assert stats["cones"][1] == sum(v["width"] * v["height"] for v in hv)
    O = oracle.build_mips(scene["grid"])
    for v, out in zip(hv, outs):
        W, H = v["width"], v["height"]
        last_rows = np.arange((H - H % tile[1] if H % tile[1] else H - tile[1]) * W, H * W)
        idx = np.unique(np.concatenate([rng.choice(W * H, 500, replace=False),
                                        last_rows[::7]]))
        ref, _ = oracle_with_spec_ties(O, v, prm, idx, lambda ii: out[1][ii])
        assert worst(compare(out, ref, idx=idx, prm=prm)) <= FP32_BOUND


def test_null_outputs_and_no_specular():
    scene, view, prm = room_case(n=32, width=30, height=20)
    prm = dict(prm, spec_enable=0)
    P = gpu_pyramid(scene["grid"])
    v = vct.View.from_host(view, outputs=False)
    v.alloc_outputs(diffuse=True, specular=False, visibility=False)
    vct.trace([P], [v], prm)
    ref = oracle.trace(oracle.build_mips(scene["grid"]), view, prm)
    D = v.out_diffuse.cpu().numpy()
    assert report(D, ref["D"])[0].max() <= FP32_BOUND


# ---------------------------------------------------------------------------
# a7 + a8: the adjoint
# ---------------------------------------------------------------------------
def _diff_case(n=32, W=48, H=40, seed=61):
    gt = vs.box_scene(n, 6, seed, room=True)
    rng = np.random.default_rng(seed + 1)
    views = [vs.interior_view(gt, W, H, rng, with_roughness=False) for _ in range(2)]
    dirs, w = vs.cone_table_ring6()
    prm = vs.trace_params(dirs, w, math.radians(60), spec_enable=True,
                          spec_aperture_min=math.radians(10), occ_enable=True, occ_aperture=0.55,
                          light=gt["light"])
    learn = np.full((n, n, n, 4), 0.1, np.float32)
    return gt, views, prm, learn


@pytest.mark.parametrize("lpp,occ", [(1, 1), (2, 0), (4, 1), (8, 0)])
def test_backward_matches_oracle_gradient(lpp, occ):
    gt, views, prm, learn = _diff_case()
    prm = dict(prm, occ_enable=occ)
    O_gt = oracle.build_mips(gt["grid"])
    targets = [oracle.trace(O_gt, v, prm) for v in views]
    O = oracle.build_mips(learn)
    grad_ref = np.zeros(learn.shape)
    gpu_grads = []
    for v, t in zip(views, targets):
        r = oracle.trace(O, v, prm)
        gD, gS, gV = r["D"] - t["D"], r["S"] - t["S"], r["Vis"] - t["Vis"]
        grad_ref += oracle.trace_backward(O, v, prm, gD, gS, gV)
        gpu_grads.append(tuple(torch.from_numpy(a.astype(np.float32)).cuda()
                               for a in (gD, gS, gV)))
    P = gpu_pyramid(learn)
    gviews = [vct.View.from_host(v) for v in views]
    grad = vct.trace_backward(P, gviews, gpu_grads, prm, cfg=vct.launch_config(8, 8, lpp))
    grad = grad.cpu().numpy().astype(np.float64)
    scale = np.abs(grad_ref).max()
    err = np.abs(grad - grad_ref)
    print("gradient: max abs err / max |grad| =", err.max() / scale)
    assert err.max() <= 1e-4 * scale
    assert np.linalg.norm(grad - grad_ref) <= 1e-5 * np.linalg.norm(grad_ref)


def test_backward_central_differences():
    """dL/dV on 64 seeded voxels x 4 channels: central differences
    (eps = 1e-3) of the FP64 loss against the CUDA adjoint."""
    gt, views, prm, learn = _diff_case(n=16, W=24, H=20, seed=71)
    views = views[:1]
    O_gt = oracle.build_mips(gt["grid"])
    t = oracle.trace(O_gt, views[0], prm)

    def loss(g):
        r = oracle.trace(oracle.build_mips(g), views[0], prm)
        return 0.5 * (np.sum((r["D"] - t["D"]) ** 2) + np.sum((r["S"] - t["S"]) ** 2)
                      + np.sum((r["Vis"] - t["Vis"]) ** 2)), r

    L0, r = loss(learn.astype(np.float64))
    grads = [tuple(torch.from_numpy(a.astype(np.float32)).cuda()
                   for a in (r["D"] - t["D"], r["S"] - t["S"], r["Vis"] - t["Vis"]))]
    P = gpu_pyramid(learn)
    grad = vct.trace_backward(P, [vct.View.from_host(views[0])], grads, prm).cpu().numpy()
    rng = np.random.default_rng(3)
    vox = rng.integers(0, 16, size=(64, 3))
    eps = 1e-3
    scale = np.abs(grad).max()
    for (x, y, z) in vox:
        for ch in range(4):
            gp = learn.astype(np.float64).copy()
            gm = gp.copy()
            gp[z, y, x, ch] += eps
            gm[z, y, x, ch] -= eps
            fd = (loss(gp)[0] - loss(gm)[0]) / (2 * eps)
            an = float(grad[z, y, x, ch])
            assert abs(fd - an) <= 2e-3 * max(abs(fd), 0.05 * scale), (x, y, z, ch, fd, an)


def test_autograd_render():
    gt, views, prm, learn = _diff_case(n=16, W=20, H=12, seed=81)
    v = vct.View.from_host(views[0])
    g = torch.from_numpy(learn).cuda().requires_grad_(True)
    D, S, V = vct.render(g, v, prm)
    loss = D.square().sum() + S.square().sum() + V.square().sum()
    loss.backward()
    P = gpu_pyramid(learn)
    ref = vct.trace_backward(P, [v], [(2 * D.detach(), 2 * S.detach(), 2 * V.detach())], prm)
    assert torch.allclose(g.grad, ref, rtol=1e-5, atol=1e-7 * ref.abs().max().item())


@pytest.mark.parametrize("dtype,layout,det", [("f32", "dense", True), ("f16", "bricks", False)])
def test_autograd_render_shaded_variants(dtype, layout, det):
    """render() with the shading epilogue and the modified cones, FP16 /
    brick storage and the reproducible adjoint: the autograd gradient of a
    loss on L and D equals the explicit adjoint call with dL/dL and dL/dD."""
    gt, views, prm, learn = _diff_case(n=32, W=20, H=12, seed=82)
    prm = dict(vs.variant_params(prm, vct.FLAG_SHADE | vct.FLAG_OCC_SMOOTH |
                                 vct.FLAG_SPEC_GRACE), occ_max_dist=0.5)
    v = vct.View.from_host(views[0])
    grid = np.asarray(gt["grid"], np.float32)
    g = torch.from_numpy(grid).cuda().requires_grad_(True)
    D, S, V, L = vct.render(g, v, prm, dtype=dtype, layout=layout, deterministic=det)
    loss = L[:, :3].square().sum() + D.square().sum()
    loss.backward()
    P = vct.build_mips(torch.from_numpy(grid).cuda(), dtype=dtype, layout=layout)
    w = vct.View.from_host(views[0], outputs=False)
    w.alloc_outputs(radiance=True)
    vct.trace([P], [w], prm)
    gL = 2 * L.detach()
    gL[:, 3] = 0
    ref = vct.trace_backward(P, [w], [(2 * D.detach(), None, None, gL)], prm, deterministic=det)
    assert ref.abs().max() > 0
    assert torch.allclose(g.grad, ref, rtol=1e-5, atol=1e-6 * ref.abs().max().item())


# ---------------------------------------------------------------------------
# failure paths
# ---------------------------------------------------------------------------
def test_bounded_wait_gives_up_with_status():
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    import ctypes
    st = vct.lib().vct_debug_wait_probe(ctypes.c_void_p(flag.data_ptr()), 5_000_000,
                                        torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    assert int(flag.item()) == 5  # VCT_ERR_TIMEOUT
    # the context is still usable
    assert float(torch.ones(4, device="cuda").sum().item()) == 4.0


def test_invalid_arguments_rejected():
    P = gpu_pyramid(np.zeros((8, 8, 8, 4), np.float32))
    scene, view, prm = room_case(n=8, width=4, height=4, n_boxes=1)
    bad = dict(prm, beta=-1.0)
    with pytest.raises(vct.VctError):
        vct.trace([P], [vct.View.from_host(view)], bad)
    bad = dict(prm, spec_aperture_min=1e-7)
    with pytest.raises(vct.VctError):
        vct.trace([P], [vct.View.from_host(view)], bad)
    # a gradient grid of the wrong shape
    with pytest.raises(ValueError):
        vct.trace_backward(P, [vct.View.from_host(view)], [(None, None, None)], prm,
                           grad_level0=torch.zeros((4, 4, 4, 4), device="cuda"))


# ---------------------------------------------------------------------------
# batching: autotuned shape, CUDA-graph replay, FP16 pyramids
# ---------------------------------------------------------------------------
def _batch(dtype="f32"):
    scenes = [vs.box_scene(n, 6, 400 + n, room=True) for n in (32, 64)]
    rng = np.random.default_rng(9)
    hv = []
    for i, (w, h) in enumerate([(70, 33), (41, 64), (16, 16), (97, 11)]):
        v = vs.interior_view(scenes[i % 2], w, h, rng)
        v["pyramid"] = i % 2
        hv.append(v)
    prm = vs.params_room9(scenes[0]["light"])
    pyrs = [gpu_pyramid(sc["grid"], dtype=dtype) for sc in scenes]
    return scenes, hv, prm, pyrs


def test_autotune_then_graph_replay_matches_direct_call():
    scenes, hv, prm, pyrs = _batch()
    views = [vct.View.from_host(v) for v in hv]
    best = vct.autotune(pyrs, views, prm)
    assert best.lanes_per_pixel in (1, 2, 4, 8) and best.tile_w * best.tile_h >= 32
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    vct.trace(pyrs, views, prm, workspace=ws)
    torch.cuda.synchronize()
    direct = [(v.out_diffuse.clone(), v.out_specular.clone(), v.out_visibility.clone())
              for v in views]
    for v in views:
        v.out_diffuse.fill_(-1)
        v.out_specular.fill_(-1)
        v.out_visibility.fill_(-1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        vct.trace(pyrs, views, prm, workspace=ws)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for v, d in zip(views, direct):
        assert torch.equal(v.out_diffuse, d[0]) and torch.equal(v.out_specular, d[1])
        assert torch.equal(v.out_visibility, d[2])
    # the replayed stats count one call (the workspace is cleared inside the graph)
    st = vct.read_stats(ws)
    assert st["cones"][1] == sum(int(v["mask"].sum()) for v in hv)


def test_batched_fp16_pyramids_against_oracle():
    scenes, hv, prm, pyrs = _batch("f16")
    outs, _ = gpu_trace(pyrs, hv, prm)
    worst_fp16, worst_ratio = 0.0, 0.0
    for v, out in zip(hv, outs):
        grid = scenes[v["pyramid"]]["grid"]
        ref = oracle.trace(oracle.build_mips(grid), v, prm)
        ratio, res = check_fp16_outputs(out, ref, grid[..., :3].reshape(-1, 3).max(axis=0),
                                        k_max=150)
        worst_ratio = max(worst_ratio, ratio)
        worst_fp16 = max(worst_fp16, worst(res))
    print("batched fp16 worst floored rel error:", worst_fp16, "worst |err| / bound:", worst_ratio)


def test_backward_with_cone_state_matches_recomputed_march():
    """The adjoint given the forward's per-cone state (sample count and
    transmittance before the last sample) equals the adjoint that re-marches
    every cone, and the state's sample counts add up to the trace's."""
    gt, views_host, prm, learn = _diff_case()
    P = gpu_pyramid(learn)
    outs = {}
    for with_state in (False, True):
        views = [vct.View.from_host(v) for v in views_host]
        if with_state:
            for v in views:
                v.alloc_cone_state(prm)
        ws = vct.trace([P], views, prm)
        torch.cuda.synchronize()
        if with_state:
            st = vct.read_stats(ws)
            total = sum(int(v.cone_state[..., 0].long()[:, torch.from_numpy(
                views_host[i]["mask"] != 0).cuda()].sum()) for i, v in enumerate(views))
            assert total == sum(st["samples"])
        grads = [(v.out_diffuse * 0.5, v.out_specular, v.out_visibility - 0.25) for v in views]
        outs[with_state] = vct.trace_backward(P, views, grads, prm).cpu().numpy()
    a, b = outs[False], outs[True]
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max(), np.abs(a - b).max()


@pytest.mark.parametrize("lpp", [1, 4])
def test_deterministic_backward_reproducible_and_close(lpp):
    """vct_trace_backward_deterministic: the same gradient bit for bit on
    every run (fixed-point sums do not depend on the order of the atomics),
    within the fixed-point rounding of the float adjoint, and as close to the
    FP64 adjoint as the float adjoint is."""
    gt, views, prm, learn = _diff_case()
    O_gt = oracle.build_mips(gt["grid"])
    O = oracle.build_mips(learn)
    grad_ref = np.zeros(learn.shape)
    gpu_grads = []
    for v in views:
        t, r = oracle.trace(O_gt, v, prm), oracle.trace(O, v, prm)
        gD, gS, gV = r["D"] - t["D"], r["S"] - t["S"], r["Vis"] - t["Vis"]
        grad_ref += oracle.trace_backward(O, v, prm, gD, gS, gV)
        gpu_grads.append(tuple(torch.from_numpy(a.astype(np.float32)).cuda()
                               for a in (gD, gS, gV)))
    P = gpu_pyramid(learn)
    gviews = [vct.View.from_host(v) for v in views]
    cfg = vct.launch_config(8, 8, lpp)
    runs = [vct.trace_backward(P, gviews, gpu_grads, prm, cfg=cfg, deterministic=True)
            for _ in range(3)]
    assert all(torch.equal(runs[0], r) for r in runs[1:])
    flt = vct.trace_backward(P, gviews, gpu_grads, prm, cfg=cfg).cpu().numpy()
    det = runs[0].cpu().numpy().astype(np.float64)
    scale = np.abs(grad_ref).max()
    assert np.abs(det - flt).max() <= 1e-5 * scale
    err = np.abs(det - grad_ref)
    print("deterministic gradient: max abs err / max |grad| =", err.max() / scale)
    assert err.max() <= 1e-4 * scale
    assert np.linalg.norm(det - grad_ref) <= 1e-5 * np.linalg.norm(grad_ref)


def test_backward_fp16_pyramid():
    """FP16 storage in the adjoint: on the constant learnable grid (0.1 at
    every level) the FP16 pyramid holds exactly binary16(0.1) everywhere, so
    its gradient equals the FP32 adjoint's, and the FP64 adjoint's, on that
    grid; on a box scene it stays within FP16 storage error of the FP32
    gradient."""
    gt, views, prm, learn = _diff_case()
    h = np.float32(np.float16(0.1))
    learn_h = np.full_like(learn, h)
    O_gt = oracle.build_mips(gt["grid"])
    O = oracle.build_mips(learn_h)
    grad_ref = np.zeros(learn.shape)
    gpu_grads = []
    for v in views:
        t, r = oracle.trace(O_gt, v, prm), oracle.trace(O, v, prm)
        gD, gS, gV = r["D"] - t["D"], r["S"] - t["S"], r["Vis"] - t["Vis"]
        grad_ref += oracle.trace_backward(O, v, prm, gD, gS, gV)
        gpu_grads.append(tuple(torch.from_numpy(a.astype(np.float32)).cuda()
                               for a in (gD, gS, gV)))
    gviews = [vct.View.from_host(v) for v in views]
    P16 = gpu_pyramid(learn, dtype="f16")
    P32 = gpu_pyramid(learn_h)
    g16 = vct.trace_backward(P16, gviews, gpu_grads, prm).cpu().numpy().astype(np.float64)
    g32 = vct.trace_backward(P32, gviews, gpu_grads, prm).cpu().numpy().astype(np.float64)
    scale = np.abs(grad_ref).max()
    assert np.abs(g16 - g32).max() <= 1e-6 * scale
    assert np.abs(g16 - grad_ref).max() <= 1e-4 * scale
    # a box scene: FP16 texels differ from FP32 by half an ulp of binary16
    scene, view, prm2 = room_case(n=32, width=30, height=20, seed=8)
    outs = {}
    for dt in ("f32", "f16"):
        P = gpu_pyramid(scene["grid"], dtype=dt)
        v = vct.View.from_host(view)
        vct.trace([P], [v], prm2)
        gr = [(torch.ones_like(v.out_diffuse), torch.ones_like(v.out_specular),
               torch.ones_like(v.out_visibility))]
        outs[dt] = vct.trace_backward(P, [v], gr, prm2).cpu().numpy()
    rel = np.abs(outs["f16"] - outs["f32"]).max() / np.abs(outs["f32"]).max()
    print("fp16 adjoint vs fp32, box scene:", rel)
    assert rel < 5e-3
