"""Error metrics for GPU-vs-oracle comparisons.

Floating-point outputs are compared per channel with a floored relative
error: err = max_px |gpu - oracle| / max(|oracle|, tau), tau = floor_frac *
max_px |oracle| of that channel.  The FP32 path's bound is 1e-4.
"""
import numpy as np


def floored_rel(gpu, ref, floor_frac=1e-3):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        ref, gpu = ref[:, None], gpu[:, None]
    out = []
    for c in range(ref.shape[1]):
        o, g = ref[:, c], gpu[:, c]
        scale = np.max(np.abs(o)) if o.size else 0.0
        tau = max(floor_frac * scale, 1e-30)
        out.append(float(np.max(np.abs(g - o) / np.maximum(np.abs(o), tau))) if o.size else 0.0)
    return np.array(out)


def report(gpu, ref, floor_frac=1e-3):
    """(max floored-rel per channel, mean floored-rel per channel)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        ref, gpu = ref[:, None], gpu[:, None]
    mx, mean = [], []
    for c in range(ref.shape[1]):
        o, g = ref[:, c], gpu[:, c]
        tau = max(floor_frac * np.max(np.abs(o)), 1e-30)
        e = np.abs(g - o) / np.maximum(np.abs(o), tau)
        mx.append(float(e.max()))
        mean.append(float(e.mean()))
    return np.array(mx), np.array(mean)


# binary16 storage: unit roundoff of a normal half, and the largest rounding
# error of a subnormal one (half its spacing 2^-24).
U16 = 2.0 ** -11
SUB16 = 2.0 ** -25


def fp16_storage_bound(ref, size, alpha, c_max, k_max, fp32_bound=1e-4, floor_frac=1e-3):
    """Per-pixel, per-channel bound on |gpu - oracle| for a pyramid stored in
    binary16 and composited in float32, against the FP64 oracle on the
    unrounded pyramid.

    Every stored texel value v >= 0 becomes h with |h - v| <= U16 v + SUB16
    (levels >= 1 are rounded once from their float32 means).  A sample is a
    convex combination of texels, so its colour c' and opacity a' obey the
    same bound relative to the exact sample.  For front-to-back compositing
    C = sum_k w_k c_k with w_k = T_k a_k and A = 1 - T_K:
      sum_k |w'_k - w_k| is at most twice the probability that two coupled
      termination processes with opacities a and a' part, which is at most
      sum_k T_k |a'_k - a_k| <= U16 A + SUB16 K, so
      |dA| <= U16 A + SUB16 K and
      |dC| <= sum_k w'_k |dc_k| + c_max sum_k |dw_k|
           <= 1.001 U16 C + SUB16 + 2 c_max (U16 A + SUB16 K).
    A diffuse sum with non-negative weights inherits the bound.  Added: a
    float32 march that stops when alpha rounds to one (dropped terms below
    6e-8 (1 + c_max)) and the float32 path's own tolerance
    fp32_bound * max(|o|, tau).

    ref: [P, C] oracle outputs (for the floored float32 term); size: [P, C]
    the quantity the storage term scales with (the colour C of a colour
    channel, the opacity A of an opacity channel, 1 - Vis for Vis); alpha:
    [P] the output's opacity; c_max: [C] the largest texel value of each
    colour channel (0 for opacity channels).  Returns the [P, C] bound."""
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        ref = ref[:, None]
    size = np.asarray(size, dtype=np.float64).reshape(ref.shape)
    a = np.asarray(alpha, dtype=np.float64).reshape(-1, 1)
    c_max = np.asarray(c_max, dtype=np.float64).reshape(1, -1)
    tau = np.maximum(floor_frac * np.abs(ref).max(axis=0, keepdims=True), 1e-30)
    storage = 1.01 * U16 * (np.abs(size) + 2.0 * c_max * a)
    absolute = SUB16 * (1.0 + (2.0 * c_max + 1.0) * k_max) + 6e-8 * (1.0 + c_max)
    return storage + absolute + fp32_bound * np.maximum(np.abs(ref), tau)


def check_fp16_outputs(gpu, ref, c_max_rgb, k_max, spec=True, occ=True):
    """Asserts the binary16-storage bound on D, S and Vis (gpu: (D, S, Vis)
    arrays for the oracle's pixels; ref: the oracle's dict); returns the worst
    ratio |gpu - oracle| / bound and the per-output (max, mean) floored
    relative errors."""
    D, S, V = gpu
    cm = np.concatenate([np.asarray(c_max_rgb, dtype=np.float64).reshape(3), [0.0]])
    worst_ratio = 0.0
    errs = {}
    outs = [("D", D, ref["D"], ref["D"], ref["D"][:, 3], cm)]
    if spec:
        outs.append(("S", S, ref["S"], ref["S"], ref["S"][:, 3], cm))
    if occ:
        outs.append(("Vis", V, ref["Vis"], 1.0 - ref["Vis"], 1.0 - ref["Vis"], np.zeros(1)))
    for name, g, o, size, a, c in outs:
        o = np.asarray(o, dtype=np.float64)
        g = np.asarray(g, dtype=np.float64).reshape(o.shape)
        b = fp16_storage_bound(o, size, a, c, k_max)
        diff = np.abs(g - o).reshape(b.shape)
        ratio = float((diff / b).max()) if diff.size else 0.0
        assert ratio <= 1.0, (name, ratio)
        worst_ratio = max(worst_ratio, ratio)
        errs[name] = report(g, o)
    return worst_ratio, errs
