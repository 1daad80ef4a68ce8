"""FP64 CPU oracle for the voxel-cone-tracing hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference arm of ``bench.py``.  The product package
never imports it.  The arithmetic lives in ``vct_oracle.c`` (plain C, double
precision, OpenMP over pixels); this module only compiles it and marshals
numpy arrays.  See the header of ``vct_oracle.c`` for the thesis passages
each function follows and for the readings of open or garbled passages.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LOCK = threading.Lock()
_LIB = None
MAX_DIFFUSE = 32


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("n_diffuse", ctypes.c_int32),
        ("spec_enable", ctypes.c_int32),
        ("occ_enable", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("diffuse_dir", (ctypes.c_double * 3) * MAX_DIFFUSE),
        ("diffuse_weight", ctypes.c_double * MAX_DIFFUSE),
        ("diffuse_aperture", ctypes.c_double),
        ("spec_aperture_min", ctypes.c_double),
        ("spec_aperture_max", ctypes.c_double),
        ("roughness_min", ctypes.c_double),
        ("occ_aperture", ctypes.c_double),
        ("light_dir", ctypes.c_double * 3),
        ("beta", ctypes.c_double),
        ("t0_voxels", ctypes.c_double),
        ("normal_offset_voxels", ctypes.c_double),
        ("t_max", ctypes.c_double),
        ("shadow_str", ctypes.c_double),
        ("occ_max_dist", ctypes.c_double),
        ("shininess", ctypes.c_double),
        ("shininess_falloff", ctypes.c_double),
        ("diffuse_str", ctypes.c_double),
        ("specular_str", ctypes.c_double),
        ("light_color", ctypes.c_double * 3),
    ]


# variant flags (same bit values as the library's, an input convention)
OCC_SMOOTH, SPEC_GRACE, DIFF_FIRST, SHADE, SHADE_IMPL, PREMUL = 1, 2, 4, 8, 16, 32
ANISO = 64  # internal: the pyramid is anisotropic (set from Pyramid.aniso)


class OrcView(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("position", ctypes.c_void_p),
        ("normal", ctypes.c_void_p),
        ("roughness", ctypes.c_void_p),
        ("mask", ctypes.c_void_p),
        ("albedo", ctypes.c_void_p),
        ("camera", ctypes.c_double * 3),
    ]


def _source_files():
    return [os.path.join(_HERE, f) for f in ("vct_oracle.c", "vct_voxelize.c", "vct_gbuffer.c")]


def compile_source(sources, out_dir=None, tag=None) -> str:
    """Compile oracle C sources into a shared library; returns its path."""
    h = hashlib.sha1()
    for s in sources:
        with open(s, "rb") as f:
            h.update(f.read())
    out_dir = out_dir or os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, f"libvct_oracle_{tag or h.hexdigest()[:12]}.so")
    if not os.path.exists(so):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=c11",
               "-shared", "-fPIC", *sources, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return so


def library_path() -> str:
    """Compile (once per source revision) and return the shared library path."""
    return compile_source(_source_files())


def build() -> None:
    _lib()


def load_library(path: str):
    """Load an oracle shared library (the committed one or a test variant)."""
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.orc_level_offset.argtypes = [i32, i32]
    lib.orc_level_offset.restype = ctypes.c_size_t
    lib.orc_num_threads.restype = i32
    lib.orc_build_mips.argtypes = [vp, i32, i32, vp]
    lib.orc_mip_adjoint.argtypes = [vp, i32, i32, vp]
    lib.orc_sample.argtypes = [vp, i32, i32, vp, dbl, vp, dbl, vp]
    lib.orc_sample_lod.argtypes = [vp, i32, i32, vp, dbl, vp]
    lib.orc_sample_lod_aniso.argtypes = [vp, i32, i32, vp, dbl, vp, vp]
    lib.orc_sample_lod_aniso.restype = None
    lib.orc_aniso_offset.argtypes = [i32, i32, i32]
    lib.orc_aniso_offset.restype = ctypes.c_size_t
    lib.orc_build_mips_aniso.argtypes = [vp, i32, i32, vp]
    lib.orc_build_mips_aniso.restype = None
    lib.orc_mip_adjoint_aniso.argtypes = [vp, vp, i32, i32, vp]
    lib.orc_mip_adjoint_aniso.restype = None
    lib.orc_trace_cone.argtypes = [vp, i32, i32, vp, dbl, vp, vp, dbl, vp, i32, vp, vp]
    lib.orc_spec_grace.argtypes = [vp, vp]
    lib.orc_spec_grace.restype = dbl
    lib.orc_tangent_frame.argtypes = [vp, vp, vp]
    lib.orc_cone_set.argtypes = [vp, dbl, i32, vp, i64, vp, vp, vp, vp, vp, vp]
    lib.orc_cone_set.restype = i32
    lib.orc_trace.argtypes = [vp, i32, i32, vp, dbl, vp, vp, vp, i64, vp, vp,
                              vp, vp, vp, vp, vp, vp]
    lib.orc_trace_backward.argtypes = [vp, i32, i32, vp, dbl, vp, vp, vp, i64,
                                       vp, vp, vp, vp, vp, vp]
    lib.orc_voxelize.argtypes = [vp, i64, vp, i64, vp, i32, vp, ctypes.c_float, vp, vp, dbl,
                                 dbl, vp, vp, vp]
    lib.orc_voxelize.restype = None
    lib.orc_gbuffer.argtypes = [vp, i64, vp, i64, vp, vp, ctypes.c_float, vp, vp, vp, vp,
                                ctypes.c_float, i32, i32, vp, i64, vp, vp, vp, vp, vp, vp]
    lib.orc_gbuffer.restype = i32
    for f in ("orc_build_mips", "orc_mip_adjoint", "orc_sample", "orc_sample_lod",
              "orc_trace_cone", "orc_tangent_frame", "orc_trace",
              "orc_trace_backward"):
        getattr(lib, f).restype = None
    return lib


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = load_library(library_path())
        return _LIB


class _Using:
    """Context manager that points this module at another oracle library
    (used by the planted-mistake tests); restores the default on exit."""

    def __init__(self, lib):
        self.lib = lib

    def __enter__(self):
        global _LIB
        _lib()
        with _LOCK:
            self.saved, _LIB = _LIB, self.lib
        return self

    def __exit__(self, *exc):
        global _LIB
        with _LOCK:
            _LIB = self.saved
        return False


def using(lib):
    return _Using(lib)


def num_threads() -> int:
    return int(_lib().orc_num_threads())


def _p(a: np.ndarray):
    return a.ctypes.data if a is not None else None


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def level_offset(n: int, level: int) -> int:
    return int(_lib().orc_level_offset(n, level))


def num_levels(n: int) -> int:
    return int(round(np.log2(n))) + 1


class Pyramid:
    """Dense FP64 pyramid: ``data`` holds all levels back to back (with
    ``aniso``, six directional volumes per level >= 1, see
    orc_build_mips_aniso)."""

    def __init__(self, data: np.ndarray, n: int, levels: int,
                 origin=(0.0, 0.0, 0.0), size: float = 1.0, aniso: bool = False):
        self.data, self.n, self.levels = data, n, levels
        self.origin = _f64(origin)
        self.size = float(size)
        self.aniso = aniso

    def level(self, l: int, direction: int = 0) -> np.ndarray:
        """Level l ([z,y,x,4]); of an anisotropic pyramid the volume for
        travel direction 0..5 = +x, -x, +y, -y, +z, -z (level 0 has one)."""
        m = self.n >> l
        off = (_lib().orc_aniso_offset(self.n, l, direction) if self.aniso
               else level_offset(self.n, l))
        return self.data[off:off + m * m * m * 4].reshape(m, m, m, 4)


def build_mips(level0: np.ndarray, levels: int | None = None,
               origin=(0.0, 0.0, 0.0), size: float = 1.0) -> Pyramid:
    level0 = _f64(level0)
    n = level0.shape[0]
    assert level0.shape == (n, n, n, 4)
    levels = num_levels(n) if levels is None else levels
    out = np.empty(level_offset(n, levels), dtype=np.float64)
    _lib().orc_build_mips(_p(level0), n, levels, _p(out))
    return Pyramid(out, n, levels, origin, size)


def build_mips_aniso(level0: np.ndarray, levels: int | None = None,
                     origin=(0.0, 0.0, 0.0), size: float = 1.0) -> Pyramid:
    """Anisotropic pyramid: level 0 isotropic, six directional volumes per
    coarser level (orc_build_mips_aniso)."""
    level0 = _f64(level0)
    n = level0.shape[0]
    assert level0.shape == (n, n, n, 4)
    levels = num_levels(n) if levels is None else levels
    out = np.empty(_lib().orc_aniso_offset(n, levels, 0), dtype=np.float64)
    _lib().orc_build_mips_aniso(_p(level0), n, levels, _p(out))
    return Pyramid(out, n, levels, origin, size, aniso=True)


def sample_lod_aniso(pyr: Pyramid, q, lam: float, w) -> np.ndarray:
    """Lookup of an anisotropic pyramid at level lam for travel along w."""
    out = np.zeros(4)
    q, w = _f64(q), _f64(w)
    _lib().orc_sample_lod_aniso(_p(pyr.data), pyr.n, pyr.levels, _p(q), float(lam), _p(w),
                                _p(out))
    return out


def mip_adjoint(gpyr: np.ndarray, n: int, levels: int) -> np.ndarray:
    """Adjoint of build_mips: per-level gradients -> level-0 gradient."""
    g = _f64(gpyr).copy()
    out = np.zeros(n * n * n * 4, dtype=np.float64)
    _lib().orc_mip_adjoint(_p(g), n, levels, _p(out))
    return out.reshape(n, n, n, 4)


def mip_adjoint_aniso(pyr: Pyramid, gpyr: np.ndarray) -> np.ndarray:
    """Adjoint of build_mips_aniso at the pyramid pyr: gradients of every
    texel (pyr's layout) -> level-0 gradient (orc_mip_adjoint_aniso)."""
    assert pyr.aniso
    g = _f64(gpyr).copy()
    assert g.size == pyr.data.size
    out = np.zeros(pyr.n ** 3 * 4, dtype=np.float64)
    _lib().orc_mip_adjoint_aniso(_p(pyr.data), _p(g), pyr.n, pyr.levels, _p(out))
    return out.reshape(pyr.n, pyr.n, pyr.n, 4)


def sample(pyr: Pyramid, p, diameter: float) -> np.ndarray:
    out = np.zeros(4)
    p = _f64(p)
    _lib().orc_sample(_p(pyr.data), pyr.n, pyr.levels, _p(pyr.origin), pyr.size,
                      _p(p), float(diameter), _p(out))
    return out


def sample_lod(pyr: Pyramid, q, lam: float) -> np.ndarray:
    out = np.zeros(4)
    q = _f64(q)
    _lib().orc_sample_lod(_p(pyr.data), pyr.n, pyr.levels, _p(q), float(lam), _p(out))
    return out


def params_struct(prm: dict) -> OrcParams:
    P = OrcParams()
    P.n_diffuse = int(prm["n_diffuse"])
    assert 0 <= P.n_diffuse <= MAX_DIFFUSE
    dirs = np.asarray(prm["diffuse_dir"], dtype=np.float64).reshape(-1, 3)
    wts = np.asarray(prm["diffuse_weight"], dtype=np.float64).reshape(-1)
    for k in range(P.n_diffuse):
        for a in range(3):
            P.diffuse_dir[k][a] = float(dirs[k, a])
        P.diffuse_weight[k] = float(wts[k])
    P.diffuse_aperture = float(prm["diffuse_aperture"])
    P.spec_enable = int(prm["spec_enable"])
    P.spec_aperture_min = float(prm["spec_aperture_min"])
    P.spec_aperture_max = float(prm["spec_aperture_max"])
    P.roughness_min = float(prm["roughness_min"])
    P.occ_enable = int(prm["occ_enable"])
    P.occ_aperture = float(prm["occ_aperture"])
    for a in range(3):
        P.light_dir[a] = float(np.asarray(prm["light_dir"], dtype=np.float64)[a])
    P.beta = float(prm["beta"])
    P.t0_voxels = float(prm["t0_voxels"])
    P.normal_offset_voxels = float(prm["normal_offset_voxels"])
    P.t_max = float(prm["t_max"])
    P.flags = int(prm.get("flags", 0)) & ~ANISO
    P.shadow_str = float(prm.get("shadow_str", 1.0))
    P.occ_max_dist = float(prm.get("occ_max_dist", 1.0))
    P.shininess = float(prm.get("shininess", 32.0))
    P.shininess_falloff = float(prm.get("shininess_falloff", 1.0))
    P.diffuse_str = float(prm.get("diffuse_str", 1.0))
    P.specular_str = float(prm.get("specular_str", 1.0))
    lc = np.asarray(prm.get("light_color", (1.0, 1.0, 1.0)), dtype=np.float64).reshape(3)
    for a in range(3):
        P.light_color[a] = float(lc[a])
    return P


def trace_cone(pyr: Pyramid, apex, direction, aperture: float, prm: dict, kind: int = -1):
    """One cone; returns (rgba, number of samples).  kind (0 diffuse, 1
    specular, 2 occlusion) selects the variant enabled by prm["flags"]."""
    P = params_struct(prm)
    if pyr.aniso:
        P.flags |= ANISO
    out = np.zeros(4)
    steps = np.zeros(1, dtype=np.int64)
    apex, direction = _f64(apex), _f64(direction)
    _lib().orc_trace_cone(_p(pyr.data), pyr.n, pyr.levels, _p(pyr.origin), pyr.size,
                          _p(apex), _p(direction), float(aperture),
                          ctypes.byref(P), int(kind), _p(out), _p(steps))
    return out, int(steps[0])


def spec_grace(direction, prm: dict) -> float:
    P = params_struct(prm)
    d = _f64(direction)
    return float(_lib().orc_spec_grace(_p(d), ctypes.byref(P)))


def tangent_frame(nrm):
    T, B = np.zeros(3), np.zeros(3)
    nrm = _f64(nrm)
    _lib().orc_tangent_frame(_p(nrm), _p(T), _p(B))
    return T, B


def cone_set(view: dict, px: int, prm: dict, n: int, origin=(0.0, 0.0, 0.0),
             size: float = 1.0):
    """Per-pixel cone set: dict(apex, kind[c], weight[c], aperture[c], dir[c,3])."""
    keep: list = []
    V = _view_struct(view, keep)
    P = params_struct(prm)
    apex = np.zeros(3)
    cap = MAX_DIFFUSE + 2
    kind = np.zeros(cap, dtype=np.int32)
    w, ap = np.zeros(cap), np.zeros(cap)
    d = np.zeros((cap, 3))
    origin = _f64(origin)
    cnt = _lib().orc_cone_set(_p(origin), float(size), int(n), ctypes.byref(V),
                              int(px), ctypes.byref(P), _p(apex), _p(kind), _p(w),
                              _p(ap), _p(d))
    return {"apex": apex, "kind": kind[:cnt], "weight": w[:cnt],
            "aperture": ap[:cnt], "dir": d[:cnt]}


def _view_struct(view: dict, keep: list) -> OrcView:
    V = OrcView()
    V.width, V.height = int(view["width"]), int(view["height"])
    arrs = {}
    for key in ("position", "normal"):
        arrs[key] = np.ascontiguousarray(view[key], dtype=np.float32)
    arrs["roughness"] = (None if view.get("roughness") is None else
                         np.ascontiguousarray(view["roughness"], dtype=np.float32))
    arrs["mask"] = (None if view.get("mask") is None else
                    np.ascontiguousarray(view["mask"], dtype=np.uint8))
    arrs["albedo"] = (None if view.get("albedo") is None else
                      np.ascontiguousarray(view["albedo"], dtype=np.float32))
    keep.extend(a for a in arrs.values() if a is not None)
    V.position, V.normal = _p(arrs["position"]), _p(arrs["normal"])
    V.roughness, V.mask = _p(arrs["roughness"]), _p(arrs["mask"])
    V.albedo = _p(arrs["albedo"])
    for a in range(3):
        V.camera[a] = float(np.asarray(view["camera"], dtype=np.float64)[a])
    return V


def trace(pyr: Pyramid, view: dict, prm: dict, idx=None):
    """Per-pixel outputs for the listed pixels (all if idx is None).

    Returns dict(D [k,4], S [k,4], Vis [k], steps[3], cones[3], margin) where
    steps/cones are per cone kind (diffuse, specular, occlusion)."""
    keep: list = []
    V = _view_struct(view, keep)
    P = params_struct(prm)
    if pyr.aniso:
        P.flags |= ANISO
    if idx is None:
        count, idx_arr = V.width * V.height, None
    else:
        idx_arr = np.ascontiguousarray(idx, dtype=np.int64)
        count = len(idx_arr)
    D = np.zeros((count, 4))
    S = np.zeros((count, 4))
    Vis = np.zeros(count)
    L = np.zeros((count, 4))
    steps = np.zeros(3, dtype=np.int64)
    cones = np.zeros(3, dtype=np.int64)
    margin = np.array([np.inf])
    hit_margin = np.array([np.inf])
    _lib().orc_trace(_p(pyr.data), pyr.n, pyr.levels, _p(pyr.origin), pyr.size,
                     ctypes.byref(V), ctypes.byref(P), _p(idx_arr), count, _p(D),
                     _p(S), _p(Vis), _p(L), _p(steps), _p(cones), _p(margin),
                     _p(hit_margin))
    out = {"D": D, "S": S, "Vis": Vis, "steps": steps, "cones": cones,
           "margin": float(margin[0]), "hit_margin": float(hit_margin[0])}
    if P.flags & SHADE:
        out["L"] = L
    return out


def trace_backward(pyr: Pyramid, view: dict, prm: dict, gD, gS, gV, idx=None, gL=None,
                   per_level: bool = False):
    """dL/d(level-0 grid) [n,n,n,4] for upstream gradients of the listed pixels
    (gL: of the shaded radiance [k,4], with the shading flag).  per_level:
    return instead dL/d(every texel of the pyramid), in the pyramid's layout
    (before the mip adjoint)."""
    keep: list = []
    V = _view_struct(view, keep)
    P = params_struct(prm)
    if pyr.aniso:
        P.flags |= ANISO
    if idx is None:
        count, idx_arr = V.width * V.height, None
    else:
        idx_arr = np.ascontiguousarray(idx, dtype=np.int64)
        count = len(idx_arr)
    gD, gS = _f64(gD).reshape(count, 4), _f64(gS).reshape(count, 4)
    gV = None if gV is None else _f64(gV).reshape(count)
    gL = None if gL is None else _f64(gL).reshape(count, 4)
    n = pyr.n
    scratch = np.empty(_lib().orc_aniso_offset(n, pyr.levels, 0) if pyr.aniso
                       else level_offset(n, pyr.levels))
    grad0 = np.zeros(n * n * n * 4)
    _lib().orc_trace_backward(_p(pyr.data), n, pyr.levels, _p(pyr.origin), pyr.size,
                              ctypes.byref(V), ctypes.byref(P), _p(idx_arr), count,
                              _p(gD), _p(gS), _p(gV), _p(gL), _p(scratch),
                              None if per_level else _p(grad0))
    return scratch if per_level else grad0.reshape(n, n, n, 4)


def voxelize(mesh: dict, n: int, origin=(0.0, 0.0, 0.0), size: float = 1.0,
             light: dict | None = None):
    """Voxelizes a triangle mesh (dict: vertices [V,3], indices [T,3], colors
    [T,3]; float32 / int32) into an n^3 grid.  light: dict(light_dir,
    light_color, ambient, diffuse_str).  Returns (grid [n,n,n,4] float64,
    owner [n,n,n] int32 (triangle index + 1, 0 empty), stats dict)."""
    light = light or {}
    verts = np.ascontiguousarray(mesh["vertices"], dtype=np.float32).reshape(-1, 3)
    idx = np.ascontiguousarray(mesh["indices"], dtype=np.int32).reshape(-1, 3)
    cols = np.ascontiguousarray(mesh["colors"], dtype=np.float32).reshape(-1, 3)
    assert cols.shape[0] == idx.shape[0]
    org = np.ascontiguousarray(origin, dtype=np.float32).reshape(3)
    ldir = _f64(light.get("light_dir", (0.0, 1.0, 0.0))).reshape(3)
    lcol = _f64(light.get("light_color", (1.0, 1.0, 1.0))).reshape(3)
    grid = np.empty((n, n, n, 4), dtype=np.float64)
    owner = np.empty((n, n, n), dtype=np.int32)
    stats = np.zeros(3, dtype=np.int64)
    _lib().orc_voxelize(_p(verts), verts.shape[0], _p(idx), idx.shape[0], _p(cols), int(n),
                        _p(org), float(np.float32(size)), _p(ldir), _p(lcol),
                        float(light.get("ambient", 0.0)), float(light.get("diffuse_str", 1.0)),
                        _p(grid), _p(owner), _p(stats))
    return grid, owner, {"fragments": int(stats[0]), "skipped": int(stats[1]),
                         "degenerate": int(stats[2])}


def gbuffer(mesh: dict, camera: dict, pixels=None):
    """G-buffer of a triangle mesh (dict as for voxelize) seen by a pinhole
    camera (dict: eye, forward, right, up, tan_half, width, height,
    frame_origin, frame_size; vectors as float32).  pixels: linear pixel
    indices (y * width + x) to evaluate, or None for all.  Returns dict of
    tri [P] int32 (-1 = no hit), position / normal / albedo [P,3] float64,
    mask [P] uint8 and the stats (skipped, degenerate)."""
    verts = np.ascontiguousarray(mesh["vertices"], dtype=np.float32).reshape(-1, 3)
    idx = np.ascontiguousarray(mesh["indices"], dtype=np.int32).reshape(-1, 3)
    cols = np.ascontiguousarray(mesh["colors"], dtype=np.float32).reshape(-1, 3)
    assert cols.shape[0] == idx.shape[0]
    f32 = [np.ascontiguousarray(camera[k], dtype=np.float32).reshape(3)
           for k in ("frame_origin", "eye", "forward", "right", "up")]
    W, H = int(camera["width"]), int(camera["height"])
    sel = None
    if pixels is not None:
        sel = np.ascontiguousarray(pixels, dtype=np.int64).reshape(-1)
        assert sel.size == 0 or (sel.min() >= 0 and sel.max() < W * H)
    count = W * H if sel is None else sel.size
    tri = np.empty(count, np.int32)
    pos, nrm, alb = (np.empty((count, 3), np.float64) for _ in range(3))
    mask = np.empty(count, np.uint8)
    stats = np.zeros(2, np.int64)
    rc = _lib().orc_gbuffer(_p(verts), verts.shape[0], _p(idx), idx.shape[0], _p(cols),
                            _p(f32[0]), float(np.float32(camera["frame_size"])), _p(f32[1]),
                            _p(f32[2]), _p(f32[3]), _p(f32[4]),
                            float(np.float32(camera["tan_half"])), W, H,
                            None if sel is None else _p(sel), count, _p(tri), _p(pos),
                            _p(nrm), _p(alb), _p(mask), _p(stats))
    if rc != 0:
        raise ValueError(f"orc_gbuffer failed ({rc}): camera outside the frame")
    return {"tri": tri, "position": pos, "normal": nrm, "albedo": alb, "mask": mask,
            "skipped": int(stats[0]), "degenerate": int(stats[1])}
