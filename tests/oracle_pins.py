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


def _fd_check(g, view, prm, targets, picks, eps, tol):
    L, r = _loss(g, view, prm, targets)
    tD, tS, tV = targets
    grad = oracle.trace_backward(oracle.build_mips(g), view, prm, r["D"] - tD, r["S"] - tS,
                                 r["Vis"] - tV)
    for flat in picks:
        gp, gm = g.copy(), g.copy()
        gp.reshape(-1)[flat] += eps
        gm.reshape(-1)[flat] -= eps
        fd = (_loss(gp, view, prm, targets)[0] - _loss(gm, view, prm, targets)[0]) / (2 * eps)
        an = grad.reshape(-1)[flat]
        assert abs(fd - an) <= tol * max(1e-3, abs(an)), (prm["flags"], flat, fd, an)
    return grad, r


def check_gradient_fd_modified_cones():
    """Central differences against the adjoint with each of the thesis's
    modified cones (Ch. 5.4.4) and with premultiplied compositing: the
    occlusion fade (a factor of t alone on the sample opacity), the angular
    grace (a factor of the cone axis alone on the specular colour), the
    first-hit diffuse cone (the hit sample's colour; no first-hit decision
    within reach of the perturbation) and c += T_k c_s."""
    import vct_synth as vs
    for flags in (1, 2, 4, 32, 1 | 2 | 32):
        # first hit: opacities around the 1/100 threshold, so that some cones
        # hit after their first sample, and a perturbation below the margin
        eps = 1e-5 if flags & 4 else 1e-4
        for seed in range(20, 40):
            g, view, prm, targets = _small_diff_problem(seed=seed)
            if flags & 4:
                g[..., 3] *= 0.1
            # a fade that is still below one at the samples of this small grid
            prm = dict(vs.variant_params(prm, flags), occ_max_dist=1.0)
            r = oracle.trace(oracle.build_mips(g), view, prm)
            if not (flags & 4) or (r["hit_margin"] > 4 * eps and r["steps"][0] > r["cones"][0]):
                break
        else:
            raise AssertionError("no seed keeps the first-hit decisions away from the threshold")
        L, r = _loss(g, view, prm, targets)
        tD, tS, tV = targets
        grad = oracle.trace_backward(oracle.build_mips(g), view, prm, r["D"] - tD,
                                     r["S"] - tS, r["Vis"] - tV)
        rng = np.random.default_rng(seed + 100)
        big = np.argsort(-np.abs(grad).reshape(-1))[:10]
        picks = list(big) + list(rng.integers(0, g.size, 8))
        if flags & 4:  # the hit samples' colours, and an alpha (zero gradient)
            picks += list(np.flatnonzero(np.abs(grad[..., 3]).reshape(-1) == 0)[:2] * 4 + 3)
        _fd_check(g, view, prm, targets, picks, eps, 1e-6)
        assert np.abs(grad).max() > 1e-3, flags
        if flags & 4:  # the first-hit diffuse cones pass no gradient to alpha
            only_d = oracle.trace_backward(oracle.build_mips(g), view, prm, r["D"] - tD,
                                           np.zeros_like(tS), np.zeros(len(tV)))
            assert not np.any(only_d[..., 3]) and np.abs(only_d[..., :3]).max() > 0


def check_gradient_fd_shading():
    """Central differences of a loss on the shaded radiance (L_vxct and
    L_impl, Ch. 4.2.2 / Ch. 5.4.4) against the adjoint given dL/dL: the
    chain rule through the shading epilogue (linear in D and S, bilinear in
    Vis and D for L_impl) into the cones."""
    import vct_synth as vs
    eps = 1e-4
    for flags in (8, 8 | 16, 8 | 1 | 2):
        g, view, prm, _ = _small_diff_problem(seed=33)
        view = dict(view, albedo=np.random.default_rng(3).uniform(0.2, 1.0, (9, 3)))
        prm = dict(vs.variant_params(prm, flags), occ_max_dist=1.0)
        tL = np.random.default_rng(4).random((9, 4))

        def loss(grid):
            r = oracle.trace(oracle.build_mips(grid), view, prm)
            return 0.5 * np.sum((r["L"][:, :3] - tL[:, :3]) ** 2), r

        L0, r = loss(g)
        gL = np.zeros((9, 4))
        gL[:, :3] = r["L"][:, :3] - tL[:, :3]
        z4, z1 = np.zeros((9, 4)), np.zeros(9)
        grad = oracle.trace_backward(oracle.build_mips(g), view, prm, z4, z4, z1, gL=gL)
        rng = np.random.default_rng(flags)
        big = np.argsort(-np.abs(grad).reshape(-1))[:10]
        for flat in list(big) + list(rng.integers(0, g.size, 8)):
            gp, gm = g.copy(), g.copy()
            gp.reshape(-1)[flat] += eps
            gm.reshape(-1)[flat] -= eps
            fd = (loss(gp)[0] - loss(gm)[0]) / (2 * eps)
            an = grad.reshape(-1)[flat]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)), (flags, flat, fd, an)
        assert np.abs(grad).max() > 1e-3, flags


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


# --------------------------------------------------------------------------
# voxelization (Ch. 4.4): brute force with exact rationals
# --------------------------------------------------------------------------
from fractions import Fraction  # noqa: E402

_SWIZZLE = {0: (2, 1), 1: (0, 2), 2: (0, 1)}  # raster axes (u, v) per dominant axis


def bf_snap(verts, origin, size, n):
    """Fixed-point vertex coordinates (1/256 voxel) by float32 arithmetic."""
    s = np.float32(256.0 * n / np.float64(np.float32(size)))
    a = np.asarray(verts, np.float32) - np.asarray(origin, np.float32)
    return np.rint(a * s).astype(np.int64)


def bf_voxelize(mesh, n, origin=(0.0, 0.0, 0.0), size=1.0, light=None):
    """Serial voxelization from the definition: every pixel centre of the
    dominant-axis projection, tested by exact barycentric coordinates (a
    centre on an edge counts for top and left edges of the counter-clockwise
    projection), depth = barycentric blend of the vertex depths, floor."""
    light = light or {}
    l = np.asarray(light.get("light_dir", (0.0, 1.0, 0.0)), np.float64)
    lc = np.asarray(light.get("light_color", (1.0, 1.0, 1.0)), np.float64)
    amb, kd = float(light.get("ambient", 0.0)), float(light.get("diffuse_str", 1.0))
    verts = np.asarray(mesh["vertices"], np.float32).reshape(-1, 3)
    X = bf_snap(verts, origin, size, n)
    owner = np.zeros((n, n, n), np.int32)
    grid = np.zeros((n, n, n, 4))
    frags = 0
    for t, tri in enumerate(np.asarray(mesh["indices"]).reshape(-1, 3)):
        V = [tuple(int(c) for c in X[k]) for k in tri]
        nrm = np.cross(np.subtract(V[1], V[0]), np.subtract(V[2], V[0]))
        if not nrm.any():
            continue
        dom = int(np.argmax(np.abs(nrm)))  # first maximum on ties
        u, v = _SWIZZLE[dom]
        P = [(Fraction(p[u]), Fraction(p[v])) for p in V]
        A = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[1][1] - P[0][1]) * (P[2][0] - P[0][0])
        if A < 0:
            P = [P[0], P[2], P[1]]
            V = [V[0], V[2], V[1]]
            A = -A
        f = np.asarray(verts[tri], np.float64)
        g = np.cross(f[1] - f[0], f[2] - f[0])
        lam = max(float(g @ l) / np.linalg.norm(g), 0.0) if np.linalg.norm(g) > 0 else 0.0
        rgb = np.asarray(mesh["colors"], np.float64).reshape(-1, 3)[t] * lc * (amb + kd * lam)
        for j in range(n):
            for i in range(n):
                c = (Fraction(256 * i + 128), Fraction(256 * j + 128))
                bary, ok = [], True
                for k in range(3):  # weight of vertex k: area opposite to it
                    a, b = P[(k + 1) % 3], P[(k + 2) % 3]
                    w = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
                    if w == 0:  # on the edge a -> b: top (horizontal, heading -u) or left (heading -v)
                        ok = (b[1] - a[1] < 0) or (b[1] == a[1] and b[0] - a[0] < 0)
                    elif w < 0:
                        ok = False
                    if not ok:
                        break
                    bary.append(w / A)
                if not ok:
                    continue
                depth = sum(bary[k] * V[k][dom] for k in range(3))
                kk = math.floor(depth / 256)
                if not 0 <= kk < n:
                    continue
                cell = [0, 0, 0]
                cell[u], cell[v], cell[dom] = i, j, kk
                frags += 1
                owner[cell[2], cell[1], cell[0]] = t + 1
                grid[cell[2], cell[1], cell[0]] = (*rgb, 1.0)
    return grid, owner, frags


def _random_mesh(rng, n, count, snap_half=True):
    """Small random triangles; with snap_half, coordinates on the half-voxel
    lattice so that edges run through pixel centres (tie cases)."""
    verts, idx = [], []
    for t in range(count):
        c = rng.uniform(0.5, n - 0.5, size=3)
        tri = c + rng.uniform(-3.0, 3.0, size=(3, 3))
        if snap_half and t % 2 == 0:
            tri = np.round(tri * 2.0) / 2.0
        if t % 5 == 1:
            tri[:, t % 3] = np.round(tri[0, t % 3]) + 0.5  # axis-aligned plane through voxel centres
        verts.extend(tri / n)
        idx.append([3 * t, 3 * t + 1, 3 * t + 2])
    cols = rng.uniform(0.1, 1.0, size=(count, 3))
    return {"vertices": np.asarray(verts, np.float32), "indices": np.asarray(idx, np.int32),
            "colors": np.asarray(cols, np.float32)}


def check_voxelize_bruteforce():
    rng = np.random.default_rng(2104)
    n = 10
    mesh = _random_mesh(rng, n, 40)
    light = {"light_dir": (0.3, 0.8, 0.52), "light_color": (1.0, 0.8, 0.6), "ambient": 0.1,
             "diffuse_str": 0.9}
    g, o, st = oracle.voxelize(mesh, n, light=light)
    bg, bo, bf = bf_voxelize(mesh, n, light=light)
    assert st["fragments"] == bf, (st, bf)
    assert np.array_equal(o, bo), int((o != bo).sum())
    assert np.allclose(g, bg, rtol=1e-12, atol=1e-15)
    # the same scene in a grid of edge 2.5 at another origin
    origin, size = np.array([-0.75, 0.5, 0.125]), 2.5
    moved = dict(mesh, vertices=(origin + size * mesh["vertices"].astype(np.float64))
                 .astype(np.float32))
    g, o, st = oracle.voxelize(moved, n, origin=origin, size=size, light=light)
    bg, bo, bf = bf_voxelize(moved, n, origin=origin, size=size, light=light)
    assert st["fragments"] == bf and np.array_equal(o, bo), (st, bf)
    assert np.allclose(g, bg, rtol=1e-12, atol=1e-15)
    assert bf > 50


def check_voxelize_shared_edges_cover_once():
    """A planar grid of triangles whose vertices sit on pixel centres: every
    centre inside the region is covered by exactly one triangle."""
    n = 16
    verts, idx = [], []
    xs = [2.5, 4.5, 7.5, 8.5, 12.5]
    ys = [1.5, 3.5, 6.5, 11.5]
    z = 5.5
    vid = {}
    for a, x in enumerate(xs):
        for b, y in enumerate(ys):
            vid[a, b] = len(verts)
            verts.append((x / n, y / n, z / n))
    for a in range(len(xs) - 1):
        for b in range(len(ys) - 1):
            q = (vid[a, b], vid[a + 1, b], vid[a + 1, b + 1], vid[a, b + 1])
            if (a + b) % 2:
                idx += [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
            else:
                idx += [[q[0], q[1], q[3]], [q[3], q[1], q[2]]]
    mesh = {"vertices": np.asarray(verts, np.float32), "indices": np.asarray(idx, np.int32),
            "colors": np.ones((len(idx), 3), np.float32)}
    g, o, st = oracle.voxelize(mesh, n)
    # centres (i + 1/2) with 2.5 <= i + 1/2 <= 12.5 and 1.5 <= j + 1/2 <= 11.5, on the
    # region's boundary only its left and top sides count: i in [2, 12), j in (1, 11]
    want = (12 - 2) * (11 - 1)
    assert st["fragments"] == want and int((o > 0).sum()) == want, (st, int((o > 0).sum()))
    assert np.all(o[5][o[5] > 0] > 0) and int((o[:5] > 0).sum() + (o[6:] > 0).sum()) == 0


def check_voxelize_box_shell():
    """A box whose faces run through voxel centres, in-plane inset by 1/4
    voxel: its voxelization is exactly the box's one-voxel shell, each face
    with its Lambert colour."""
    n = 16
    lo, hi = np.array([3, 5, 2]), np.array([11, 9, 14])  # voxels lo .. hi-1
    a, b = lo + 0.5, hi - 0.5
    e = 0.25
    verts, idx, cols = [], [], []
    light = {"light_dir": (0.48, 0.6, 0.64), "light_color": (1.0, 1.0, 1.0), "ambient": 0.05}
    normals = []
    for axis in range(3):
        for side, pos in ((-1, a[axis]), (+1, b[axis])):
            u, v = [x for x in range(3) if x != axis]
            corners = []
            for cu, cv in ((a[u] - e, a[v] - e), (b[u] + e, a[v] - e), (b[u] + e, b[v] + e),
                           (a[u] - e, b[v] + e)):
                p = np.zeros(3)
                p[axis], p[u], p[v] = pos, cu, cv
                corners.append(p / n)
            base = len(verts)
            verts += corners
            nrm = np.zeros(3)
            nrm[axis] = side
            tri = [[0, 1, 2], [0, 2, 3]]
            g = np.cross(corners[1] - corners[0], corners[2] - corners[0])
            if g @ nrm < 0:
                tri = [[0, 2, 1], [0, 3, 2]]
            for t in tri:
                idx.append([base + t[0], base + t[1], base + t[2]])
                cols.append((0.8, 0.5, 0.3))
                normals.append(nrm)
    mesh = {"vertices": np.asarray(verts, np.float32), "indices": np.asarray(idx, np.int32),
            "colors": np.asarray(cols, np.float32)}
    g, o, st = oracle.voxelize(mesh, n, light=light)
    zz, yy, xx = np.meshgrid(range(n), range(n), range(n), indexing="ij")
    inside = ((xx >= lo[0]) & (xx < hi[0]) & (yy >= lo[1]) & (yy < hi[1]) &
              (zz >= lo[2]) & (zz < hi[2]))
    core = ((xx > lo[0]) & (xx < hi[0] - 1) & (yy > lo[1]) & (yy < hi[1] - 1) &
            (zz > lo[2]) & (zz < hi[2] - 1))
    shell = inside & ~core
    assert np.array_equal(o > 0, shell)
    assert np.array_equal(g[..., 3], shell.astype(np.float64))
    ldir = np.asarray(light["light_dir"])
    for t in np.unique(o[o > 0]):
        lam = max(float(normals[t - 1] @ ldir), 0.0)
        want = np.array([0.8, 0.5, 0.3], np.float32).astype(np.float64) * (0.05 + lam)
        assert np.allclose(g[o == t][:, :3], want, rtol=1e-6), (t, g[o == t][0], want)


def check_voxelize_draw_order_and_skips():
    n = 8
    tri = np.array([[0.1, 0.1, 0.55], [0.9, 0.1, 0.55], [0.1, 0.9, 0.55]], np.float32)
    bad = np.array([[0.1, 0.1, 0.3], [1e7, 0.5, 0.3], [0.5, 0.9, 0.3]], np.float32)
    line = np.array([[0.1, 0.1, 0.2], [0.5, 0.5, 0.2], [0.9, 0.9, 0.2]], np.float32)
    verts = np.concatenate([tri, tri, bad, line])
    mesh = {"vertices": verts,
            "indices": np.array([[0, 1, 2], [3, 4, 5], [6, 7, 8], [9, 10, 11], [0, 1, 99]],
                                np.int32),
            "colors": np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [1, 1, 1]],
                               np.float32)}
    light = {"light_dir": (0.0, 0.0, 1.0)}
    g, o, st = oracle.voxelize(mesh, n, light=light)
    assert st["skipped"] == 2 and st["degenerate"] == 1, st
    assert np.all(o[o > 0] == 2) and np.all(g[o > 0][:, :3] == (0.0, 1.0, 0.0))
    assert st["fragments"] == 2 * int((o > 0).sum())
    mesh["indices"], mesh["colors"] = mesh["indices"][[1, 0]], mesh["colors"][[1, 0]]
    g, o, st = oracle.voxelize(mesh, n, light=light)
    assert np.all(g[o > 0][:, :3] == (1.0, 0.0, 0.0))


def check_voxelize_area_and_clip():
    """Fragment count of a large triangle is its projected area up to the
    boundary pixels; a triangle reaching outside the grid keeps only the
    fragments inside."""
    n = 64
    p = np.array([[0.05, 0.1, 0.4], [0.93, 0.2, 0.45], [0.3, 0.97, 0.5]], np.float32)
    mesh = {"vertices": p, "indices": np.array([[0, 1, 2]], np.int32),
            "colors": np.ones((1, 3), np.float32)}
    _, o, st = oracle.voxelize(mesh, n)
    q = p.astype(np.float64) * n
    area = 0.5 * abs(np.cross(q[1] - q[0], q[2] - q[0])[2])
    perim = sum(np.linalg.norm((q[(k + 1) % 3] - q[k])[:2]) for k in range(3))
    assert abs(st["fragments"] - area) <= perim + 1, (st, area, perim)
    big = np.array([[-0.5, -0.5, 0.5], [1.5, -0.5, 0.5], [-0.5, 1.5, 0.5]], np.float32)
    mesh["vertices"] = big
    _, o, st = oracle.voxelize(mesh, n)
    i, j = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    want = int(((i + j) < n).sum())  # the hypotenuse u + v = n passes no centre
    assert st["fragments"] == want and int((o > 0).sum()) == want


def check_premultiplied_compositing():
    """Premultiplied sample colour (c += (1 - alpha) c_s) in a homogeneous
    medium (c0, a): c = c0 * sum_{k<K} (1-a)^k = c0 (1 - (1-a)^K) / a, alpha
    as in the straight form; the flag changes every cone kind alike."""
    n = 64
    c0 = np.array([0.3, 0.6, 0.9])
    a, aperture, beta, t_max = 0.2, math.radians(30), 0.5, 0.25
    g = np.empty((n, n, n, 4))
    g[..., :3], g[..., 3] = c0, a
    P = oracle.build_mips(g)
    prm = dict(base_params(beta=beta, t_max=t_max), flags=oracle.PREMUL)
    w = np.array([2.0, -1.0, 2.0]) / 3.0
    K = closed_form_steps(1.0 / n, t_max, aperture, beta)
    for kind in (-1, 0, 1, 2):
        out, k = oracle.trace_cone(P, [0.5, 0.5, 0.5], w, aperture, prm, kind=kind)
        tr = (1.0 - a) ** K
        assert k == K and rel(out[3], 1.0 - tr) < 1e-12
        assert rel(out[:3], c0 * (1.0 - tr) / a) < 1e-12, (kind, out)


# --------------------------------------------------------------------------
# camera G-buffer (Ch. 5.4 geometry pass): closed forms, an independent
# slab raycaster, exact ties
# --------------------------------------------------------------------------
TAN30 = math.tan(math.radians(30.0))


def _gb_camera(eye, f, r, u, W, H, origin=(0.0, 0.0, 0.0), size=1.0):
    v = lambda a: np.asarray(a, np.float32).reshape(3)  # noqa: E731
    return {"eye": v(eye), "forward": v(f), "right": v(r), "up": v(u),
            "tan_half": float(np.float32(TAN30)), "width": W, "height": H,
            "frame_origin": v(origin), "frame_size": float(size)}


def _gb_mesh(quads, colours):
    """Quads (c0, c1, c2, c3) -> triangles (c0, c1, c2), (c0, c2, c3)."""
    V, I, C = [], [], []
    for q, col in zip(quads, colours):
        b = len(V)
        V.extend(q)
        I += [[b, b + 1, b + 2], [b, b + 2, b + 3]]
        C += [col, col]
    return {"vertices": np.asarray(V, np.float32), "indices": np.asarray(I, np.int32),
            "colors": np.asarray(C, np.float32)}


def _plane_quad(z, lo=-0.9, hi=1.9, flip=False):
    q = [(lo, lo, z), (hi, lo, z), (hi, hi, z), (lo, hi, z)]
    return [q[0], q[3], q[2], q[1]] if flip else q  # same diagonal c0 - c2


def _pixel_dirs(W, H):
    """Directions (-sx, sy, 1) of the camera looking along +z with right =
    -x, up = +y, float64 (the pixel-centre model of a pinhole camera)."""
    i, j = np.meshgrid(np.arange(W), np.arange(H), indexing="xy")
    sx = ((2 * i.ravel() + 1) / W - 1.0) * TAN30 * W / H
    sy = (1.0 - (2 * j.ravel() + 1) / H) * TAN30
    return np.stack([-sx, sy, np.ones_like(sx)], 1)


def check_gbuffer_plane_closed_form():
    """A plane z = 0.7 facing a camera at z = 0.1: every hit at eye + 0.6 d,
    normal -z for either winding, the triangle by the side of the diagonal
    y = x; the same with another fixed-point frame; a pixel subset equals the
    full image."""
    W, H, eye = 24, 16, np.array([0.5, 0.5, 0.1])
    d = _pixel_dirs(W, H)
    want = eye + 0.6 * d
    side = want[:, 1] - want[:, 0]
    for flip, origin, size in ((False, (0, 0, 0), 1.0), (True, (0, 0, 0), 1.0),
                               (False, (-0.5, 0.25, -1.0), 4.0)):
        mesh = _gb_mesh([_plane_quad(0.7, flip=flip)], [(0.2, 0.4, 0.6)])
        mesh["colors"][1] = (0.9, 0.1, 0.3)
        cam = _gb_camera(eye, (0, 0, 1), (-1, 0, 0), (0, 1, 0), W, H, origin, size)
        g = oracle.gbuffer(mesh, cam)
        tol = 2e-5 * size
        assert g["mask"].all() and np.abs(g["position"] - want).max() < tol, (flip, origin)
        assert np.array_equal(g["normal"], np.tile([0.0, 0.0, -1.0], (W * H, 1))), flip
        far = np.abs(side) > 1e-4
        upper = side > 0  # (c0, c2, c3) of the unflipped quad
        tri = np.where(upper, 1, 0) if not flip else np.where(upper, 0, 1)
        assert np.array_equal(g["tri"][far], tri[far]), flip
        assert np.array_equal(g["albedo"], mesh["colors"][g["tri"]].astype(np.float64))
        sel = np.array([0, 5, 77, W * H - 1, 200])
        s = oracle.gbuffer(mesh, cam, pixels=sel)
        for k in ("tri", "position", "normal", "albedo", "mask"):
            assert np.array_equal(s[k], g[k][sel]), k


def check_gbuffer_depth_order_and_ties():
    """Nearest plane wins in either index order; coincident triangles and a
    ray through a shared edge go to the lower index; a plane behind the
    camera is never hit."""
    W, H, eye = 25, 15, (0.5, 0.5, 0.1)
    cam = _gb_camera(eye, (0, 0, 1), (-1, 0, 0), (0, 1, 0), W, H)
    A, B = (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)
    near, far, behind = _plane_quad(0.5), _plane_quad(0.8), _plane_quad(-0.3)
    for quads, cols, win in (([far, near], [A, B], B), ([near, far], [A, B], A),
                             ([near, near], [A, B], A), ([behind, far], [A, B], B)):
        g = oracle.gbuffer(_gb_mesh(quads, cols), cam)
        assert g["mask"].all() and np.all(g["albedo"] == win), (cols, win)
    g = oracle.gbuffer(_gb_mesh([behind], [A]), cam)
    assert not g["mask"].any() and np.all(g["tri"] == -1)
    # a diamond split along x = 0.5: the centre column (sx = 0) looks along
    # the shared edge's plane exactly; both triangles are hit at equal depth
    top, right, bot, left = (0.5, 0.9, 0.7), (0.8, 0.5, 0.7), (0.5, 0.1, 0.7), (0.2, 0.5, 0.7)
    for order in ((0, 1), (1, 0)):
        tris = [[top, right, bot], [top, bot, left]]
        tris = [tris[k] for k in order]
        mesh = {"vertices": np.asarray(tris, np.float32).reshape(-1, 3),
                "indices": np.arange(6, dtype=np.int32).reshape(2, 3),
                "colors": np.asarray([A, B], np.float32)}
        g = oracle.gbuffer(mesh, cam)
        centre = np.arange(H) * W + W // 2
        assert g["mask"][centre].all() and np.all(g["tri"][centre] == 0), order
        # off the edge: the right half of the image (-x side) is the left triangle
        i = np.arange(W * H) % W
        wing = [k for k in order].index(1)  # index of [top, bot, left] (x < 0.5)
        hit = g["mask"].astype(bool)
        assert np.all(g["tri"][hit & (i > W // 2)] == wing), order
        assert np.all(g["tri"][hit & (i < W // 2)] == 1 - wing), order


def check_gbuffer_against_slab_raycaster():
    """Boxes and the room as triangles seen from an interior camera: the
    same mask, face normals and positions as the slab-test raycaster of the
    input generator (double precision, analytic boxes), up to the pixels
    whose rays pass within rounding of a box edge."""
    import vct_synth as vs
    scene = vs.box_scene(32, 6, 5, room=True)
    rng = np.random.default_rng(11)
    W, H = 48, 32
    mesh = vs.box_mesh(scene, tess=2)
    for _ in range(2):
        eye = vs.interior_camera(rng, scene["boxes"], 32)
        target = vs.interior_camera(rng, scene["boxes"], 32)
        pos, nrm, mask = vs.raycast_gbuffer(scene, W, H, eye, target)
        g = oracle.gbuffer(mesh, vs.camera(eye, target, W, H))
        assert np.array_equal(g["mask"], mask)
        same = np.all(g["normal"] == nrm.reshape(-1, 3), axis=1)
        assert same.mean() > 0.99, same.mean()
        err = np.abs(g["position"] - pos.reshape(-1, 3))[same].max()
        assert err < 2e-5, err


def check_gbuffer_skips_and_frame():
    """Bad indices and vertices beyond two frame sizes are skipped, zero-area
    triangles are degenerate; a camera outside the frame is refused."""
    W, H = 8, 6
    cam = _gb_camera((0.5, 0.5, 0.1), (0, 0, 1), (-1, 0, 0), (0, 1, 0), W, H)
    verts = np.array([[-1.9, -1.9, 0.7], [1.9, -1.9, 0.7], [0.5, 1.9, 0.7],   # usable
                      [-1.0, -1.0, 0.6], [2.5, -1.0, 0.6], [0.5, 2.1, 0.6],   # y > 2
                      [0.1, 0.1, 0.5], [0.5, 0.5, 0.5], [0.9, 0.9, 0.5]],     # collinear
                     np.float32)
    mesh = {"vertices": verts,
            "indices": np.array([[0, 1, 2], [3, 4, 5], [6, 7, 8], [0, 1, 9]], np.int32),
            "colors": np.ones((4, 3), np.float32)}
    g = oracle.gbuffer(mesh, cam)
    assert (g["skipped"], g["degenerate"]) == (2, 1), g
    assert g["mask"].all() and np.all(g["tri"] == 0)
    bad = dict(cam, eye=np.array([0.5, 0.5, 2.5], np.float32))
    try:
        oracle.gbuffer(mesh, bad)
    except ValueError:
        pass
    else:
        raise AssertionError("camera outside the frame accepted")


# --------------------------------------------------------------------------
# anisotropic mips (Villegas' anisotropic filtering, Ch. 5.1): brute force
# of the definition, closed forms, the direction-weighted sampler
# --------------------------------------------------------------------------
def bf_aniso_levels(level0, levels):
    """Directional volumes by numpy: for direction d (axis, sign) the mean
    over the 4 child pairs along the axis of the pair composited in the
    order of travel (front first), colour stored straight."""
    out = {0: {d: level0 for d in range(6)}}
    for l in range(1, levels):
        out[l] = {}
        for d in range(6):
            axis, neg = d // 2, d % 2
            src = out[l - 1][d]  # [z, y, x, 4]
            ax = 2 - axis        # array axis of this coordinate
            lo = np.take(src, np.arange(0, src.shape[ax], 2), axis=ax)
            hi = np.take(src, np.arange(1, src.shape[ax], 2), axis=ax)
            f, b = (hi, lo) if neg else (lo, hi)
            a = f[..., 3:] + (1 - f[..., 3:]) * b[..., 3:]
            pre = f[..., 3:] * f[..., :3] + (1 - f[..., 3:]) * b[..., 3:] * b[..., :3]
            c = np.where(a > 0, pre / np.where(a > 0, a, 1), 0.0)
            comp = np.concatenate([c, a], axis=-1)
            m = comp.shape
            # mean over the two remaining axes' pairs
            sh = list(m)
            for other in range(3):
                if other == ax:
                    continue
                sh[other] //= 2
            r = comp
            for other in range(3):
                if other == ax:
                    continue
                r = 0.5 * (np.take(r, np.arange(0, r.shape[other], 2), axis=other) +
                           np.take(r, np.arange(1, r.shape[other], 2), axis=other))
            out[l][d] = r
    return out


def check_aniso_mips_bruteforce():
    rng = np.random.default_rng(41)
    for n in (2, 8):
        g = rng.random((n, n, n, 4))
        g[rng.random((n, n, n)) < 0.4] = 0.0  # empty voxels, alpha-0 pairs
        P = oracle.build_mips_aniso(g)
        bf = bf_aniso_levels(g, P.levels)
        for l in range(1, P.levels):
            for d in range(6):
                assert np.allclose(P.level(l, d), bf[l][d], rtol=1e-12, atol=1e-14), (n, l, d)


def check_aniso_constant_closed_form():
    """A homogeneous medium (c, a): every directional texel of level l has
    the colour c and the opacity of 2^l voxels in a row, 1 - (1 - a)^(2^l)."""
    n, a = 16, 0.3
    c0 = np.array([0.2, 0.5, 0.8])
    g = np.empty((n, n, n, 4))
    g[..., :3], g[..., 3] = c0, a
    P = oracle.build_mips_aniso(g)
    for l in range(1, P.levels):
        for d in range(6):
            v = P.level(l, d)
            assert np.allclose(v[..., :3], c0, rtol=1e-12), (l, d)
            assert np.allclose(v[..., 3], 1 - (1 - a) ** (2 ** l), rtol=1e-12), (l, d)


def check_aniso_direction_weights():
    """The sampler reads level >= 1 from the three volumes facing the travel
    direction, weighted w_a^2 / |w|^2: an axis direction reads one volume
    (its sign picks +/-), a general one the weighted sum; level 0 is the
    isotropic grid."""
    rng = np.random.default_rng(43)
    n = 8
    g = rng.random((n, n, n, 4))
    P = oracle.build_mips_aniso(g)
    bf = bf_aniso_levels(g, P.levels)
    iso = oracle.build_mips(g)
    for _ in range(40):
        q = rng.uniform(-0.1, 1.1, 3)
        lam = float(rng.choice([1.0, 2.0, 1.6, 2.3]))
        l0 = int(np.floor(lam))
        f = lam - l0
        l1 = min(l0 + 1, P.levels - 1)
        w = rng.normal(size=3)
        got = oracle.sample_lod_aniso(P, q, lam, w)
        want = np.zeros(4)
        for lk, lw in ((l0, 1 - f), (l1, f)):
            for ax in range(3):
                d = 2 * ax + (1 if w[ax] < 0 else 0)
                one = oracle.Pyramid(_dense_pyr(bf, d, P.levels), n, P.levels)
                want += lw * w[ax] ** 2 / (w @ w) * bf_sample(_levels_of(one), q, lk)
        assert np.allclose(got, want, rtol=1e-10, atol=1e-12), (q, lam, got, want)
        e = np.zeros(3)
        e[rng.integers(3)] = rng.choice([-1.0, 1.0])
        ax = int(np.flatnonzero(e)[0])
        d = 2 * ax + (1 if e[ax] < 0 else 0)
        one = oracle.Pyramid(_dense_pyr(bf, d, P.levels), n, P.levels)
        assert np.allclose(oracle.sample_lod_aniso(P, q, 2.0, e),
                           bf_sample(_levels_of(one), q, 2.0), rtol=1e-10, atol=1e-12)
        assert np.allclose(oracle.sample_lod_aniso(P, q, 0.0, w), oracle.sample_lod(iso, q, 0.0))


def _dense_pyr(bf, d, levels):
    return np.concatenate([bf[l][d].reshape(-1) for l in range(levels)])


def _levels_of(pyr):
    return [pyr.level(l) for l in range(pyr.levels)]


def check_aniso_homogeneous_march():
    """A cone through a homogeneous medium of an anisotropic pyramid: each
    sample's opacity is the level blend of 1 - (1 - a)^(2^l) (the colour
    stays c), composited front to back: alpha = 1 - prod (1 - a_k)."""
    n, a = 64, 0.05
    c0 = np.array([0.3, 0.6, 0.9])
    g = np.empty((n, n, n, 4))
    g[..., :3], g[..., 3] = c0, a
    P = oracle.build_mips_aniso(g)
    aperture, beta, t_max = math.radians(30), 0.5, 0.25
    prm = base_params(beta=beta, t_max=t_max)
    h0 = 1.0 / n
    w = np.array([2.0, -1.0, 2.0]) / 3.0
    out, k = oracle.trace_cone(P, [0.5, 0.5, 0.5], w, aperture, prm)
    t, trans, alpha, K = h0, 1.0, 0.0, 0
    while alpha < 1 and t <= t_max:
        d = 2 * t * math.tan(aperture / 2)
        lam = min(max(math.log2(d / h0), 0.0), P.levels - 1)
        l0 = math.floor(lam)
        f = lam - l0
        l1 = min(l0 + 1, P.levels - 1)
        a_s = (1 - f) * (1 - (1 - a) ** (2 ** l0)) + f * (1 - (1 - a) ** (2 ** l1))
        alpha += trans * a_s
        trans *= 1 - a_s
        t += beta * d
        K += 1
    assert k == K and abs(out[3] - (1 - trans)) < 1e-12, (k, K, out[3], 1 - trans)
    assert np.allclose(out[:3], c0 * (1 - trans), rtol=1e-12)


def check_aniso_mip_adjoint_vjp():
    """The adjoint of the anisotropic build against central differences of
    the build itself: <(B(g + eps v) - B(g - eps v)) / 2 eps, y> =
    <v, B^T y> for random directions v and texel weights y, on grids whose
    opacities are all in [0.05, 0.9] (the pair composite is smooth there)."""
    for n, seed in ((2, 61), (4, 62), (8, 63)):
        rng = np.random.default_rng(seed)
        g = rng.uniform(0.05, 0.9, (n, n, n, 4))
        P = oracle.build_mips_aniso(g)
        for _ in range(3):
            y = rng.standard_normal(P.data.size)
            v = rng.standard_normal(g.shape)
            eps = 1e-6
            fd = (oracle.build_mips_aniso(g + eps * v).data
                  - oracle.build_mips_aniso(g - eps * v).data) @ y / (2 * eps)
            an = float(np.sum(oracle.mip_adjoint_aniso(P, y) * v))
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (n, fd, an)


def check_aniso_mip_adjoint_empty():
    """All-empty children (alpha = 0 everywhere): each texel of direction d
    has alpha = (1/4) sum over its pairs of a_f + (1 - a_f) a_b, so every
    child opacity receives 1/4 of its parent's alpha gradient from each of
    the six directions, and no colour gradient (the colour is 0 by
    definition where alpha = 0)."""
    n = 2
    g = np.zeros((n, n, n, 4))
    g[..., :3] = np.random.default_rng(64).random((n, n, n, 3))
    P = oracle.build_mips_aniso(g)
    rng = np.random.default_rng(65)
    y = np.zeros(P.data.size)
    y[n ** 3 * 4:] = rng.standard_normal(P.data.size - n ** 3 * 4)
    gr = oracle.mip_adjoint_aniso(P, y)
    top = y[n ** 3 * 4:].reshape(6, 4)  # level 1: one texel per direction
    assert np.all(gr[..., :3] == 0.0)
    assert np.allclose(gr[..., 3], top[:, 3].sum() / 4.0, rtol=0, atol=1e-15)


def check_gradient_fd_aniso():
    """Central differences of the FP64 loss through an anisotropic pyramid
    against the adjoint (trace scatter into the directional volumes weighted
    by w_a^2, then the transpose of the pair-composite build), with opacities
    in [0.05, 0.3]: no cone saturates and every pair composite is smooth;
    plain, and with the occlusion fade, the angular grace and premultiplied
    colour together."""
    import vct_synth as vs
    g, view, prm, targets = _small_diff_problem(seed=66)
    _fd_aniso(g, view, prm, targets)
    _fd_aniso(g, view, dict(vs.variant_params(prm, 1 | 2 | 32), occ_max_dist=1.0), targets)


def _fd_aniso(g, view, prm, targets):
    g[..., 3] = np.random.default_rng(67).uniform(0.05, 0.3, g.shape[:3])
    tD, tS, tV = targets

    def loss(grid):
        r = oracle.trace(oracle.build_mips_aniso(grid), view, prm)
        return 0.5 * (np.sum((r["D"] - tD) ** 2) + np.sum((r["S"] - tS) ** 2)
                      + np.sum((r["Vis"] - tV) ** 2)), r

    L, r = loss(g)
    grad = oracle.trace_backward(oracle.build_mips_aniso(g), view, prm, r["D"] - tD,
                                 r["S"] - tS, r["Vis"] - tV)
    iso = oracle.trace_backward(oracle.build_mips(g), view, prm, r["D"] - tD, r["S"] - tS,
                                r["Vis"] - tV)
    assert not np.allclose(grad, iso)
    rng = np.random.default_rng(68)
    big = np.argsort(-np.abs(grad).reshape(-1))[:12]
    picks = list(big) + list(rng.integers(0, g.size, 12))
    eps = 1e-5
    for flat in picks:
        gp, gm = g.copy(), g.copy()
        gp.reshape(-1)[flat] += eps
        gm.reshape(-1)[flat] -= eps
        fd = (loss(gp)[0] - loss(gm)[0]) / (2 * eps)
        an = grad.reshape(-1)[flat]
        assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)), (flat, fd, an)
    assert np.abs(grad).max() > 1e-3
