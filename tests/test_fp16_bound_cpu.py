"""The binary16-storage error bound used by the FP16 GPU tests, checked on the
CPU: the FP64 oracle traced through a pyramid whose every texel is rounded
to binary16 differs from the oracle on the unrounded pyramid by less than
the bound (with no float32 term), and the bound is not vacuous (the worst
ratio is a sizeable fraction of it)."""
import numpy as np
import pytest

import oracle
import vct_synth as vs
from metrics import fp16_storage_bound


def _rounded(O):
    return oracle.Pyramid(O.data.astype(np.float16).astype(np.float64), O.n, O.levels,
                          O.origin, O.size)


def _ratios(ref, got, c_max, k_max):
    out = {}
    cm = np.concatenate([c_max, [0.0]])
    for name, size, a, c in (("D", ref["D"], ref["D"][:, 3], cm),
                             ("S", ref["S"], ref["S"][:, 3], cm),
                             ("Vis", 1.0 - ref["Vis"], 1.0 - ref["Vis"], np.zeros(1))):
        o = ref[name]
        b = fp16_storage_bound(o, size, a, c, k_max, fp32_bound=0.0)
        d = np.abs(np.asarray(got[name]) - o).reshape(b.shape)
        out[name] = float((d / b).max())
    return out


@pytest.mark.parametrize("seed", [3, 4])
def test_fp16_rounded_pyramid_within_bound(seed):
    scene = vs.box_scene(32, 8, seed, room=True)
    rng = np.random.default_rng(seed)
    view = vs.interior_view(scene, 40, 30, rng)
    prm = vs.params_room9(scene["light"])
    O = oracle.build_mips(scene["grid"])
    ref = oracle.trace(O, view, prm)
    got = oracle.trace(_rounded(O), view, prm)
    c_max = scene["grid"][..., :3].reshape(-1, 3).max(axis=0).astype(np.float64)
    r = _ratios(ref, got, c_max, k_max=150)
    assert max(r.values()) <= 1.0, r
    # the bound is a bound on a real effect: rounding moves the outputs by a
    # visible fraction of it
    assert max(r.values()) >= 0.01, r


def test_fp16_bound_catches_coarser_storage():
    """The same comparison with texels rounded to 8 mantissa bits instead of
    11 (a storage format 8x coarser) exceeds the bound."""
    scene = vs.box_scene(32, 8, 5, room=True)
    rng = np.random.default_rng(5)
    view = vs.interior_view(scene, 40, 30, rng)
    prm = vs.params_room9(scene["light"])
    O = oracle.build_mips(scene["grid"])
    ref = oracle.trace(O, view, prm)
    m, e = np.frexp(O.data)
    coarse = oracle.Pyramid(np.ldexp(np.round(m * 2.0 ** 8) / 2.0 ** 8, e), O.n, O.levels,
                            O.origin, O.size)
    got = oracle.trace(coarse, view, prm)
    c_max = scene["grid"][..., :3].reshape(-1, 3).max(axis=0).astype(np.float64)
    r = _ratios(ref, got, c_max, k_max=150)
    assert max(r.values()) > 1.0, r
