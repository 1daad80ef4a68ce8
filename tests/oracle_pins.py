"""Checks that pin the FP64 oracle to things other than itself.

Each ``check_*`` raises AssertionError when the oracle disagrees with a brute
force, closed form, invariant or thesis-fixed value.  They are collected by
``test_oracle_pins.py`` for the committed oracle and re-run by
``test_oracle_mutants.py`` against oracle builds with planted mistakes (each
mistake must trip at least one check).

Brute-force and closed-form helpers here are written independently of the
oracle's C code: the sampler is a tent-weight sum over every texel of every
level (no floor/fraction stencil), mips are numpy block means, the step
schedule is the closed form t0 * r^k, and compositing uses the product form
sum_k T_k a_k c_k.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

# --------------------------------------------------------------------------
# brute-force helpers
# --------------------------------------------------------------------------


def bf_levels(level0: np.ndarray, levels: int):
    """Level l texel = mean of level 0 over its 2^l cube (numpy block means)."""
    n = level0.shape[0]
    out = []
    for l in range(levels):
        b = 1 << l
        m = n // b
        out.append(level0.astype(np.float64).reshape(m, b, m, b, m, b, 4)
                   .mean(axis=(1, 3, 5)))
    return out


def bf_tri(V: np.ndarray, q) -> np.ndarray:
    """Tent-weighted sum over all texels of one level (centres at (i+1/2)/N);
    texels that do not exist simply do not contribute."""
    m = V.shape[0]
    idx = np.arange(m)
    w = [np.maximum(0.0, 1.0 - np.abs(q[a] * m - 0.5 - idx)) for a in range(3)]
    return np.einsum("z,y,x,zyxc->c", w[2], w[1], w[0], V)


def bf_sample(levels_list, q, lam) -> np.ndarray:
    L = len(levels_list)
    lc = min(max(lam, 0.0), L - 1.0)
    out = np.zeros(4)
    for l, V in enumerate(levels_list):
        wl = max(0.0, 1.0 - abs(lc - l))
        if wl > 0.0:
            out += wl * bf_tri(V, q)
    return out


def closed_form_steps(t0, t_max, aperture, beta):
    """Number of k >= 0 with t0 r^k <= t_max, r = 1 + 2 beta tan(aperture/2)."""
    r = 1.0 + 2.0 * beta * math.tan(aperture / 2.0)
    k = 0
    while t0 * r ** k <= t_max:
        k += 1
    return k


def bf_ray(levels_list, apex, w, aperture, t0, t_max, beta, h0):
    """Product-form march: C = sum_k T_k a_k c_k, A = 1 - prod_k (1 - a_k)."""
    r = 1.0 + 2.0 * beta * math.tan(aperture / 2.0)
    C, T, k = np.zeros(3), 1.0, 0
    while True:
        t = t0 * r ** k
        if t > t_max or T <= 0.0:
            break
        d = 2.0 * t * math.tan(aperture / 2.0)
        v = bf_sample(levels_list, np.asarray(apex) + t * np.asarray(w),
                      math.log2(d / h0))
        C += T * v[3] * v[:3]
        T *= 1.0 - v[3]
        k += 1
    return np.concatenate([C, [1.0 - T]]), k


def base_params(**kw):
    prm = {
        "n_diffuse": 0, "diffuse_dir": np.zeros((0, 3)), "diffuse_weight": np.zeros(0),
        "diffuse_aperture": 0.5, "spec_enable": 0, "spec_aperture_min": 0.2,
        "spec_aperture_max": 0.2, "roughness_min": 0.05, "occ_enable": 0,
        "occ_aperture": 0.55, "light_dir": np.array([0.0, 1.0, 0.0]), "beta": 0.5,
        "t0_voxels": 1.0, "normal_offset_voxels": 1.0, "t_max": 1.0}
    prm.update(kw)
    return prm


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


# --------------------------------------------------------------------------
# mip pyramid
# --------------------------------------------------------------------------


def check_mip_block_means():
    rng = np.random.default_rng(10)
    for n in (2, 8, 16):
        g = rng.random((n, n, n, 4))
        L = oracle.num_levels(n)
        P = oracle.build_mips(g)
        for l, V in enumerate(bf_levels(g, L)):
            assert np.allclose(P.level(l), V, rtol=1e-13, atol=0), (n, l)


def check_mip_mean_preserved():
    rng = np.random.default_rng(11)
    g = rng.random((16, 16, 16, 4))
    P = oracle.build_mips(g)
    m0 = g.reshape(-1, 4).mean(0)
    for l in range(P.levels):
        assert rel(P.level(l).reshape(-1, 4).mean(0), m0) < 1e-13, l
    assert rel(P.level(P.levels - 1).reshape(4), m0) < 1e-13


def check_mip_constant():
    g = np.empty((8, 8, 8, 4))
    g[...] = (0.25, 0.5, 0.125, 0.75)
    P = oracle.build_mips(g)
    for l in range(P.levels):
        assert np.all(P.level(l) == g[0, 0, 0]), l


def check_mip_adjoint_identity():
    """<M x, y> = <x, M^T y> for the whole-pyramid operator M."""
    rng = np.random.default_rng(12)
    n = 8
    x = rng.standard_normal((n, n, n, 4))
    P = oracle.build_mips(x)
    y = rng.standard_normal(P.data.shape)
    lhs = float(P.data @ y)
    rhs = float(x.reshape(-1) @ oracle.mip_adjoint(y, n, P.levels).reshape(-1))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs)), (lhs, rhs)


# --------------------------------------------------------------------------
# sampling
# --------------------------------------------------------------------------


def check_sample_tent_bruteforce():
    rng = np.random.default_rng(13)
    n = 8
    g = rng.random((n, n, n, 4))
    P = oracle.build_mips(g)
    lv = bf_levels(g, P.levels)
    for _ in range(300):
        q = rng.uniform(-0.15, 1.15, size=3)
        lam = rng.uniform(-1.0, P.levels + 0.5)
        got = oracle.sample_lod(P, q, lam)
        want = bf_sample(lv, q, lam)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-14), (q, lam, got, want)
    # integer levels and exact texel centres
    for lam in range(P.levels):
        m = n >> lam
        x1 = min(1, m - 1)
        q = (np.array([x1, 0, m - 1]) + 0.5) / m
        got = oracle.sample_lod(P, q, float(lam))
        assert np.allclose(got, P.level(lam)[m - 1, 0, x1], rtol=1e-14), lam


def check_sample_affine():
    """An affine field is kept by the box filter (mean of an affine function
    over a cube = value at its centre) and reproduced exactly by linear
    interpolation, so every interior lookup returns a.q + b."""
    n = 16
    idx = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    A = np.array([[0.3, -0.2, 0.7], [0.1, 0.4, -0.5], [-0.6, 0.2, 0.3], [0.2, 0.2, 0.2]])
    b = np.array([0.1, 0.2, 0.3, 0.4])
    g = np.stack([A[c, 0] * X + A[c, 1] * Y + A[c, 2] * Z + b[c] for c in range(4)], -1)
    P = oracle.build_mips(g)
    rng = np.random.default_rng(14)
    for _ in range(200):
        lam = rng.uniform(-0.5, 2.0)  # levels 0..3, N_l >= 2
        q = rng.uniform(0.25, 0.75, size=3)
        got = oracle.sample_lod(P, q, lam)
        want = A @ q + b
        assert np.allclose(got, want, rtol=0, atol=1e-13), (q, lam, got, want)


def check_sample_diameter_levels():
    """sample(p, d) with d = h0 * 2^l reads level l (scene units, offset grid)."""
    rng = np.random.default_rng(15)
    n = 8
    g = rng.random((n, n, n, 4))
    origin, size = np.array([-1.0, 2.0, 0.5]), 2.0
    P = oracle.build_mips(g, origin=origin, size=size)
    lv = bf_levels(g, P.levels)
    h0 = size / n
    for _ in range(60):
        q = rng.uniform(0.0, 1.0, size=3)
        l = int(rng.integers(0, P.levels))
        frac = rng.uniform(0.0, 1.0) if l < P.levels - 1 else 0.0
        got = oracle.sample(P, origin + size * q, h0 * 2.0 ** (l + frac))
        want = bf_sample(lv, q, l + frac)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# cone march
# --------------------------------------------------------------------------


def check_empty_grid():
    import vct_synth as vs
    c = vs.config_small_fp32(n=16, n_boxes=3, width=6, height=5)
    P = oracle.build_mips(np.zeros((16, 16, 16, 4)))
    prm = dict(c["params"], occ_enable=1)
    r = oracle.trace(P, c["views"][0], prm)
    assert np.all(r["D"] == 0.0) and np.all(r["S"] == 0.0) and np.all(r["Vis"] == 1.0)


def check_homogeneous_medium():
    """Constant (c0, a) with every footprint inside the grid: after K steps
    alpha = 1 - (1-a)^K and c = c0 (1 - (1-a)^K), K from the closed form."""
    n = 64
    c0 = np.array([0.3, 0.6, 0.9])
    for a, aperture, beta, t_max in ((0.05, math.radians(30), 0.5, 0.25),
                                     (0.5, math.radians(20), 0.5, 0.2),
                                     (0.6, math.radians(30), 0.3, 0.25)):
        g = np.empty((n, n, n, 4))
        g[..., :3], g[..., 3] = c0, a
        P = oracle.build_mips(g)
        prm = base_params(beta=beta, t_max=t_max)
        w = np.array([2.0, -1.0, 2.0]) / 3.0
        out, k = oracle.trace_cone(P, [0.5, 0.5, 0.5], w, aperture, prm)
        K = closed_form_steps(1.0 / n, t_max, aperture, beta)
        assert k == K, (k, K)
        tr = (1.0 - a) ** K
        assert rel(out[3], 1.0 - tr) < 1e-12
        assert rel(out[:3], c0 * (1.0 - tr)) < 1e-12


def check_opaque_first_sample_stops():
    n = 16
    g = np.empty((n, n, n, 4))
    g[..., :3], g[..., 3] = (0.2, 0.4, 0.8), 1.0
    P = oracle.build_mips(g)
    out, k = oracle.trace_cone(P, [0.5, 0.5, 0.5], [1.0, 0.0, 0.0], 0.3, base_params())
    assert k == 1 and np.allclose(out, [0.2, 0.4, 0.8, 1.0], rtol=1e-14)


def check_small_aperture_ray():
    """Footprint below one voxel at every step: the cone reduces to a ray
    march over level-0 trilinear samples (brute-force product form)."""
    rng = np.random.default_rng(16)
    n = 8
    g = rng.random((n, n, n, 4))
    g[..., 3] *= 0.5
    P = oracle.build_mips(g)
    lv = bf_levels(g, P.levels)
    h0 = 1.0 / n
    for _ in range(20):
        apex = rng.uniform(0.2, 0.8, size=3)
        w = rng.standard_normal(3)
        w /= np.linalg.norm(w)
        t_max = rng.uniform(0.3, 0.9)
        aperture = 2.0 * math.atan(0.9 * h0 / (2.0 * t_max))  # d(t_max) < h0
        prm = base_params(t_max=t_max, beta=0.5)
        got, k = oracle.trace_cone(P, apex, w, aperture, prm)
        want, kb = bf_ray(lv, apex, w, aperture, h0, t_max, 0.5, h0)
        assert k == kb, (k, kb)
        assert np.allclose(got, want, rtol=1e-11, atol=1e-14), (got, want)


def check_general_cone_bruteforce():
    """Wide cones on a tiny grid: whole march against the brute-force sampler
    and product-form compositing (levels > 0, partial blends, borders)."""
    rng = np.random.default_rng(17)
    n = 8
    g = rng.random((n, n, n, 4))
    g[..., 3] *= 0.3
    P = oracle.build_mips(g)
    lv = bf_levels(g, P.levels)
    h0 = 1.0 / n
    for _ in range(20):
        apex = rng.uniform(0.1, 0.9, size=3)
        w = rng.standard_normal(3)
        w /= np.linalg.norm(w)
        aperture = rng.uniform(0.2, 1.5)
        beta = rng.uniform(0.3, 1.0)
        t0v = rng.uniform(0.5, 2.0)
        prm = base_params(t_max=1.0, beta=beta, t0_voxels=t0v)
        got, k = oracle.trace_cone(P, apex, w, aperture, prm)
        want, kb = bf_ray(lv, apex, w, aperture, t0v * h0, 1.0, beta, h0)
        assert k == kb and np.allclose(got, want, rtol=1e-11, atol=1e-14)


def check_single_step_lod():
    """t_max = t0: one sample at t0 with level log2(2 t0 tan(g/2) / h0)."""
    rng = np.random.default_rng(18)
    n = 16
    g = rng.random((n, n, n, 4))
    P = oracle.build_mips(g)
    lv = bf_levels(g, P.levels)
    h0 = 1.0 / n
    for lam in (1.5, 0.25, 2.75, -0.5):
        aperture = 2.0 * math.atan(2.0 ** lam / 2.0)  # t0 = h0
        apex = rng.uniform(0.3, 0.7, size=3)
        w = rng.standard_normal(3)
        w /= np.linalg.norm(w)
        prm = base_params(t_max=h0, t0_voxels=1.0)
        got, k = oracle.trace_cone(P, apex, w, aperture, prm)
        v = bf_sample(lv, apex + h0 * w, lam)
        assert k == 1
        assert np.allclose(got, [*(v[3] * v[:3]), v[3]], rtol=1e-12, atol=1e-15)


def check_rgb_linearity():
    import vct_synth as vs
    c = vs.config_small_fp32(n=16, n_boxes=4, width=8, height=8)
    g = c["scenes"][0]["grid"].astype(np.float64)
    prm = dict(c["params"], occ_enable=1)
    r1 = oracle.trace(oracle.build_mips(g), c["views"][0], prm)
    g2 = g.copy()
    g2[..., :3] *= 3.0
    r2 = oracle.trace(oracle.build_mips(g2), c["views"][0], prm)
    assert np.allclose(r2["D"][:, :3], 3.0 * r1["D"][:, :3], rtol=1e-13, atol=0)
    assert np.allclose(r2["S"][:, :3], 3.0 * r1["S"][:, :3], rtol=1e-13, atol=0)
    assert np.array_equal(r2["D"][:, 3], r1["D"][:, 3])
    assert np.array_equal(r2["Vis"], r1["Vis"])


def check_mask_and_vis():
    import vct_synth as vs
    c = vs.config_small_fp32(n=16, n_boxes=4, width=8, height=8)
    v = dict(c["views"][0])
    v["mask"] = (np.arange(64) % 3 != 0).astype(np.uint8)
    P = oracle.build_mips(c["scenes"][0]["grid"])
    prm = dict(c["params"], occ_enable=1)
    r = oracle.trace(P, v, prm)
    off = v["mask"] == 0
    assert np.all(r["D"][off] == 0) and np.all(r["S"][off] == 0)
    assert np.all(r["Vis"][off] == 1.0)
    # Vis = 1 - alpha of one cone along the light from the apex
    for px in np.nonzero(~off)[0][:6]:
        cs = oracle.cone_set(v, px, prm, 16)
        assert cs["kind"][-1] == 2
        out, _ = oracle.trace_cone(P, cs["apex"], cs["dir"][-1], cs["aperture"][-1], prm)
        assert r["Vis"][px] == 1.0 - out[3]


# --------------------------------------------------------------------------
# per-pixel set-up
# --------------------------------------------------------------------------


def check_tangent_frame():
    rng = np.random.default_rng(19)
    normals = [np.array(v, dtype=np.float64) for v in
               ((0, 0, 1), (0, 0, -1), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0))]
    normals += [v / np.linalg.norm(v) for v in rng.standard_normal((30, 3))]
    for nrm in normals:
        T, B = oracle.tangent_frame(nrm)
        assert abs(T @ nrm) < 1e-14 and abs(B @ nrm) < 1e-14 and abs(T @ B) < 1e-14
        assert abs(np.linalg.norm(T) - 1) < 1e-14 and abs(np.linalg.norm(B) - 1) < 1e-14
        assert np.allclose(np.cross(T, B), nrm, atol=1e-14)  # right-handed


def _one_pixel_view(x, nrm, cam, roughness=None):
    return {"width": 1, "height": 1, "position": np.asarray(x, np.float32),
            "normal": np.asarray(nrm, np.float32), "mask": None,
            "roughness": None if roughness is None else np.asarray([roughness], np.float32),
            "camera": np.asarray(cam, np.float32)}


def check_cone_set():
    import vct_synth as vs
    dirs, w = vs.cone_table_thesis9()
    prm = vs.trace_params(dirs, w, 0.55, spec_enable=True, spec_aperture_min=0.1,
                          spec_aperture_max=1.0, roughness_min=0.05, occ_enable=True,
                          occ_aperture=0.55, light=(0.0, 0.6, 0.8))
    n = 16
    # floor: normal +y, camera up and to the side -> mirror flips the y component
    x, nrm, cam = (0.5, 0.25, 0.5), (0.0, 1.0, 0.0), (0.25, 0.75, 0.5)
    for rough, ap in ((0.05, 0.1), (1.0, 1.0), (0.525, 0.55)):
        cs = oracle.cone_set(_one_pixel_view(x, nrm, cam, rough), 0, prm, n)
        assert list(cs["kind"]) == [0] * 9 + [1, 2]
        assert np.allclose(cs["apex"], np.array(x) + np.array(nrm) / n, atol=1e-15)
        v = np.array(x) - np.array(cam)
        v /= np.linalg.norm(v)
        assert np.allclose(cs["dir"][9], [v[0], -v[1], v[2]], atol=1e-7)
        assert abs(cs["aperture"][9] - ap) < 1e-6, (rough, cs["aperture"][9])
        assert np.allclose(cs["dir"][10], prm["light_dir"], atol=0)
        # the front cone runs along the normal; the table's angles survive
        assert np.allclose(cs["dir"][0], nrm, atol=1e-15)
        D = cs["dir"][:9]
        want = np.asarray(prm["diffuse_dir"], np.float64)
        assert np.allclose(D @ D.T, want @ want.T, atol=1e-12)
        assert np.allclose(D @ np.array(nrm), want[:, 2], atol=1e-12)
    # no roughness buffer -> minimum aperture
    cs = oracle.cone_set(_one_pixel_view(x, nrm, cam), 0, prm, n)
    assert abs(cs["aperture"][9] - np.float32(0.1)) < 1e-12


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------


def _small_diff_problem(seed=20, n=8):
    import vct_synth as vs
    rng = np.random.default_rng(seed)
    g = rng.uniform(0.0, 0.3, size=(n, n, n, 4))
    W = H = 3
    pos = rng.uniform(0.3, 0.7, size=(W * H, 3)).astype(np.float32)
    nrm = np.zeros((W * H, 3), np.float32)
    nrm[np.arange(W * H), rng.integers(0, 3, W * H)] = rng.choice([-1.0, 1.0], W * H)
    view = {"width": W, "height": H, "position": pos.reshape(-1),
            "normal": nrm.reshape(-1), "mask": None,
            "roughness": rng.uniform(0.05, 1.0, W * H).astype(np.float32),
            "camera": np.array([0.1, 0.9, 0.2], np.float32)}
    dirs, w = vs.cone_table_ring6()
    prm = vs.trace_params(dirs, w, math.radians(60), spec_enable=True,
                          spec_aperture_min=math.radians(10),
                          spec_aperture_max=math.radians(40), occ_enable=True,
                          occ_aperture=0.55, light=(0.3, 0.8, 0.52), t_max=0.6)
    tD = rng.random((W * H, 4))
    tS = rng.random((W * H, 4))
    tV = rng.random(W * H)
    return g, view, prm, (tD, tS, tV)


def _loss(g, view, prm, targets):
    r = oracle.trace(oracle.build_mips(g), view, prm)
    tD, tS, tV = targets
    L = 0.5 * (np.sum((r["D"] - tD) ** 2) + np.sum((r["S"] - tS) ** 2)
               + np.sum((r["Vis"] - tV) ** 2))
    return L, r


def check_gradient_fd():
    """Central differences of the FP64 loss against the adjoint.  With every
    opacity small the march never saturates, the loss is a polynomial in the
    voxel values, and the central difference is exact up to O(eps^2)."""
    g, view, prm, targets = _small_diff_problem()
    L, r = _loss(g, view, prm, targets)
    tD, tS, tV = targets
    P = oracle.build_mips(g)
    grad = oracle.trace_backward(P, view, prm, r["D"] - tD, r["S"] - tS, r["Vis"] - tV)
    rng = np.random.default_rng(21)
    eps = 1e-4
    big = np.argsort(-np.abs(grad).reshape(-1))[:12]
    picks = list(big) + list(rng.integers(0, g.size, 12))
    for flat in picks:
        gp, gm = g.copy(), g.copy()
        gp.reshape(-1)[flat] += eps
        gm.reshape(-1)[flat] -= eps
        fd = (_loss(gp, view, prm, targets)[0] - _loss(gm, view, prm, targets)[0]) / (2 * eps)
        an = grad.reshape(-1)[flat]
        assert abs(fd - an) <= 1e-7 * max(1e-3, abs(an)), (flat, fd, an)
    assert np.abs(grad).max() > 1e-3


# --------------------------------------------------------------------------
# the thesis's modified cones (Ch. 5.4.4) and the shading epilogue
# --------------------------------------------------------------------------


def glsl_smoothstep(e0, e1, x):
    t = min(max((x - e0) / (e1 - e0), 0.0), 1.0)
    return t * t * (3.0 - 2.0 * t)


def check_first_hit_diffuse():
    """The modified diffuse cone returns the colour of the first sample whose
    opacity exceeds 1/100 (brute-force sampler on a slab), alpha 1."""
    n = 16
    g = np.zeros((n, n, n, 4))
    g[:, :, 11:, :3] = (0.2, 0.5, 0.7)
    g[:, :, 11:, 3] = 1.0
    P = oracle.build_mips(g)
    lv = bf_levels(g, P.levels)
    h0 = 1.0 / n
    prm = base_params(flags=oracle.DIFF_FIRST, beta=0.5, t_max=1.0)
    apex, w, ap = np.array([0.25, 0.52, 0.47]), np.array([1.0, 0.0, 0.0]), 0.4
    got, k = oracle.trace_cone(P, apex, w, ap, prm, kind=0)
    r = 1.0 + 2.0 * 0.5 * math.tan(ap / 2)
    for kk in range(200):
        t = h0 * r ** kk
        v = bf_sample(lv, apex + t * w, math.log2(2 * t * math.tan(ap / 2) / h0))
        if v[3] > 0.01:
            break
    assert k == kk + 1, (k, kk)
    assert np.allclose(got, [*v[:3], 1.0], rtol=1e-12, atol=1e-15), (got, v)
    # below the threshold everywhere: nothing is returned
    g2 = np.full((n, n, n, 4), 0.005)
    out, _ = oracle.trace_cone(oracle.build_mips(g2), apex, w, ap, prm, kind=0)
    assert np.all(out == 0.0)


def check_smoothstep_occlusion():
    """Homogeneous medium: alpha = 1 - prod_k (1 - a s(t_k)) with
    s(t) = smoothstep(0, max_dist, sqrt(t) shadow_str) and t_k = t0 r^k."""
    n = 64
    a, ap, beta, t_max, md, st = 0.3, math.radians(25), 0.5, 0.25, 0.8, 1.7
    g = np.empty((n, n, n, 4))
    g[..., :3], g[..., 3] = 0.5, a
    P = oracle.build_mips(g)
    prm = base_params(flags=oracle.OCC_SMOOTH, beta=beta, t_max=t_max, occ_max_dist=md,
                      shadow_str=st)
    out, k = oracle.trace_cone(P, [0.5, 0.5, 0.5], [0.0, 0.6, 0.8], ap, prm, kind=2)
    r = 1.0 + 2.0 * beta * math.tan(ap / 2)
    T, kk = 1.0, 0
    while (1.0 / n) * r ** kk <= t_max:
        T *= 1.0 - a * glsl_smoothstep(0.0, md, math.sqrt((1.0 / n) * r ** kk) * st)
        kk += 1
    assert k == kk
    assert rel(out[3], 1.0 - T) < 1e-12
    # the variant is off for the other kinds
    plain, _ = oracle.trace_cone(P, [0.5, 0.5, 0.5], [0.0, 0.6, 0.8], ap, prm, kind=0)
    assert rel(plain[3], 1.0 - (1.0 - a) ** kk) < 1e-12


def check_spec_grace():
    """f = (1 - max(0, acos(w.l) - 0.008 pi shininess) / pi)^q."""
    for theta_deg, shin, q in ((40.0, 10.0, 5.0), (3.0, 20.0, 8.0), (170.0, 0.0, 2.0)):
        th = math.radians(theta_deg)
        w = np.array([math.sin(th), math.cos(th), 0.0])
        prm = base_params(light_dir=np.array([0.0, 1.0, 0.0]), shininess=shin,
                          shininess_falloff=q)
        want = (1.0 - max(0.0, th - 0.008 * math.pi * shin) / math.pi) ** q
        assert abs(oracle.spec_grace(w, prm) - want) < 1e-13


def _shade_view(x, nrm, cam, albedo):
    return {"width": 1, "height": 1, "position": np.asarray(x, np.float32),
            "normal": np.asarray(nrm, np.float32), "mask": None, "roughness": None,
            "albedo": np.asarray(albedo, np.float32), "camera": np.asarray(cam, np.float32)}


def check_shading_epilogue():
    """L_vxct and L_impl at one pixel against the Phong terms written out
    (light (0.6, 0.8, 0): n.l = 0.8, mirror direction (-0.6, 0.8, 0))."""
    import vct_synth as vs
    n = 16
    g = np.zeros((n, n, n, 4))
    g[:, 12:, :, :3], g[:, 12:, :, 3] = (0.9, 0.4, 0.1), 1.0
    P = oracle.build_mips(g)
    dirs, w = vs.cone_table_ring6()
    x, nrm = np.array([0.5, 0.25, 0.5]), np.array([0.0, 1.0, 0.0])
    cam = x + 0.3 * np.array([-0.6, 0.8, 0.0]) + np.array([0.0, 0.0, 0.05])
    alb = np.array([0.3, 0.6, 0.9])
    light = np.array([0.6, 0.8, 0.0])
    base = vs.trace_params(dirs, w, math.radians(60), spec_enable=True,
                           spec_aperture_min=math.radians(15), occ_enable=True, light=light)
    base.update(diffuse_str=0.7, specular_str=0.4, shininess=12.0,
                light_color=np.array([1.0, 0.9, 0.8]))
    view = _shade_view(x, nrm, cam.astype(np.float32), alb)
    x32 = np.asarray(view["position"], np.float64)
    c64 = np.asarray(view["camera"], np.float64)
    l64 = np.asarray(base["light_dir"], np.float64)
    alb = np.asarray(view["albedo"], np.float64)
    wv = (c64 - x32) / np.linalg.norm(c64 - x32)
    R = -l64 + 2.0 * (l64 @ nrm) * nrm
    gloss = max(wv @ R, 0.0) ** 12.0
    for flags in (oracle.SHADE, oracle.SHADE | oracle.SHADE_IMPL):
        prm = dict(base, flags=flags)
        r = oracle.trace(P, view, prm)
        D, S, V = r["D"][0], r["S"][0], r["Vis"][0]
        assert 0.0 < V < 1.0 and S[:3].max() > 0.0
        direct = np.array([1.0, 0.9, 0.8]) * alb * (0.7 * max(l64 @ nrm, 0.0) + 0.4 * gloss)
        if flags & oracle.SHADE_IMPL:
            want = V * D[:3] + S[:3] + V * direct
        else:
            want = alb * (0.7 * D[:3] + 0.4 * S[:3]) + V * direct
        assert np.allclose(r["L"][0, :3], want, rtol=1e-12, atol=1e-15), (flags, r["L"][0], want)
