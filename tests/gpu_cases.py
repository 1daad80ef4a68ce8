"""Helpers shared by the GPU tests: run the CUDA path and the oracle on the
same seeded inputs and compare."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2104_00618_gb300 as vct
from metrics import report

FP32_BOUND = 1e-4  # max floored relative error per channel, FP32 path
# The float32 march stops once 1 - T rounds to one (T < 2^-25; the FP64
# oracle goes on until its alpha rounds to one): the samples it leaves out
# carry at most T of opacity, and T times the largest texel colour (<= 1 in
# these scenes) of colour.  Where a view's channel is tiny everywhere (a
# view in shadow: Vis ~ 1e-10), the floored relative error of that absolute
# difference is not small; comparisons at the configured sizes allow it
# explicitly.
R12_ABS = 2.0 ** -24
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


def spec_near_ties(view, prm, n, idx, tol=1e-5):
    """Split the listed pixels into (plain, ties): ties are pixels whose
    specular cone has a step within `tol` (relative) of t_max, where the
    float32 march (per-pixel schedule in float32) and the FP64 oracle may
    legitimately disagree on whether that last step is taken.  The cone's
    steps are t_k = t0 r^k with r = 1 + 2 beta tan(gamma/2) and the
    aperture gamma from the pixel's roughness; step k lands on t_max when
    k = e = log2(t_max / t0) / log2(r)."""
    idx = np.asarray(idx)
    if not prm["spec_enable"] or view.get("roughness") is None:
        return idx, idx[:0]
    rho = np.asarray(view["roughness"], dtype=np.float64)[idx]
    rmin = float(prm["roughness_min"])
    f = np.clip((rho - rmin) / (1.0 - rmin), 0.0, 1.0)
    g = prm["spec_aperture_min"] + f * (prm["spec_aperture_max"] - prm["spec_aperture_min"])
    l2r = np.log2(1.0 + 2.0 * prm["beta"] * np.tan(0.5 * g))
    e = np.log2(prm["t_max"] * n / prm["t0_voxels"]) / l2r
    dist = np.abs(e - np.round(e)) * l2r * np.log(2.0)
    tie = dist < tol
    return idx[~tie], idx[tie]


def oracle_with_spec_ties(O, view, prm, idx, gpu_S, tol=1e-5):
    """The oracle's outputs for the listed pixels, with the specular near-ties
    of spec_near_ties resolved: for such a pixel S is taken from the oracle
    run with t_max moved by -2 tol or +2 tol (the near step left out, or
    taken), whichever is closer to the GPU's S (gpu_S(idx) -> [k, 4]); D and
    Vis do not depend on it.  The oracle's own step margin over the other
    pixels must exceed MIN_STEP_MARGIN.  Returns (ref, number of ties)."""
    plain, ties = spec_near_ties(view, prm, O.n, idx, tol)
    ref = oracle.trace(O, view, prm, idx=idx)
    if len(plain):
        r0 = oracle.trace(O, view, prm, idx=plain)
        assert r0["margin"] > MIN_STEP_MARGIN, r0["margin"]
    if len(ties):
        pos = np.searchsorted(idx, ties)
        assert np.array_equal(np.asarray(idx)[pos], ties)
        lo = oracle.trace(O, view, dict(prm, t_max=prm["t_max"] * (1 - 2 * tol)), idx=ties)
        hi = oracle.trace(O, view, dict(prm, t_max=prm["t_max"] * (1 + 2 * tol)), idx=ties)
        g = np.asarray(gpu_S(ties), dtype=np.float64).reshape(-1, 4)
        use_hi = np.abs(g - hi["S"]).max(axis=1) < np.abs(g - lo["S"]).max(axis=1)
        ref["S"][pos] = np.where(use_hi[:, None], hi["S"], lo["S"])
    return ref, len(ties)


def fp32_ratio(gpu, ref, floor_frac=1e-3):
    """max over pixels and channels of |gpu - oracle| / (FP32_BOUND *
    max(|oracle|, tau) + R12_ABS): <= 1 passes (tau = floor_frac * the
    channel's largest |oracle| over the given pixels)."""
    g = np.asarray(gpu, dtype=np.float64)
    o = np.asarray(ref, dtype=np.float64)
    if o.ndim == 1:
        o, g = o[:, None], g[:, None]
    g = g.reshape(o.shape)
    tau = np.maximum(floor_frac * np.abs(o).max(axis=0, keepdims=True), 1e-30)
    return float((np.abs(g - o) / (FP32_BOUND * np.maximum(np.abs(o), tau) + R12_ABS)).max())
