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
