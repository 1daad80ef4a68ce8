"""Helpers shared by the GPU tests: run the CUDA path and the oracle on the
same seeded inputs and compare."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2104_00618_gb300 as vct
from metrics import report

FP32_BOUND = 1e-4  # max floored relative error per channel, FP32 path
# The float32 step schedule places a cone's samples within 1e-6 of their
# distance; inputs whose oracle has a cone ending closer than this to t_max
# (relative) could count one sample more or less on either side.
MIN_STEP_MARGIN = 2e-6


def gpu_pyramid(grid: np.ndarray, dtype="f32", levels=None):
    g = torch.from_numpy(np.ascontiguousarray(grid, dtype=np.float32)).cuda()
    return vct.build_mips(g, levels=levels, dtype=dtype)


def gpu_trace(pyrs, views_host, prm, cfg=None):
    views = [vct.View.from_host(v) for v in views_host]
    ws = vct.trace(pyrs, views, prm, cfg=cfg)
    torch.cuda.synchronize()
    outs = [(v.out_diffuse.cpu().numpy(), v.out_specular.cpu().numpy(),
             v.out_visibility.cpu().numpy()) for v in views]
    return outs, vct.read_stats(ws)


def compare(gpu_out, ref, idx=None, prm=None):
    """Per-output (max, mean) floored relative errors, restricted to idx."""
    D, S, V = gpu_out
    if idx is not None:
        D, S, V = D[idx], S[idx], V[idx]
    res = {}
    res["D"] = report(D, ref["D"])
    if prm is None or prm["spec_enable"]:
        res["S"] = report(S, ref["S"])
    if prm is None or prm["occ_enable"]:
        res["Vis"] = report(V, ref["Vis"])
    return res


def worst(res):
    return max(float(np.max(v[0])) for v in res.values())


def room_case(n=64, n_boxes=8, width=203, height=117, seed=7, roughness=True, mask_frac=0.1):
    import vct_synth as vs
    rng = np.random.default_rng(seed)
    scene = vs.box_scene(n, n_boxes, seed, room=True)
    view = vs.interior_view(scene, width, height, rng, with_roughness=roughness)
    if mask_frac:
        view["mask"] = (rng.random(width * height) >= mask_frac).astype(np.uint8)
    prm = vs.params_room9(scene["light"])
    return scene, view, prm
