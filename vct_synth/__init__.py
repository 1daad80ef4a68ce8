"""Seeded synthetic inputs for the voxel-cone-tracing hot path.

Both the CUDA path and the FP64 oracle consume exactly the arrays made here;
this module holds no cone-tracing, sampling or mip arithmetic (only scene
synthesis: boxes, the Lambert-lit radiance injected into voxels, cameras,
G-buffers, and the cone tables / parameters, all of which are inputs).

Scene recipe (stands in for the thesis's scene files and scanned models, which
are not available; Ch. 5.4.4 and Ch. 6.3.2 describe the thesis's own scenes):

* The grid spans the unit cube; level 0 has ``n`` voxels per axis and the
  array layout is ``[z][y][x][rgba]`` float32.
* Boxes have integer voxel extents (so walls land exactly on voxel faces, the
  remedy for the voxelization inaccuracy discussed in Ch. 6.2): size per axis
  uniform in [n/16, n/4], min corner uniform in [0, n - size]; later boxes
  overwrite earlier ones.  Each box gets an RGB colour uniform in [0,1]^3.
* A directional light l, uniform on the sphere with l_y >= 0.3.
* Occupied voxels have opacity 1 (Ch. 4.4.3).  A voxel on a face with outward
  normal n_f gets colour * max(0, n_f . l) (max over the faces it lies on);
  interior voxels get RGB 0; empty voxels are (0,0,0,0).
* Optional room: one-voxel-thick walls on the six grid faces, facing inward,
  left wall red (0.75,0.2,0.2), right wall green (0.2,0.75,0.2), others grey.
"""
from __future__ import annotations

import ctypes
import hashlib
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LOCK = threading.Lock()
_LIB = None

RED = (0.75, 0.2, 0.2)
GREEN = (0.2, 0.75, 0.2)
GREY = (0.75, 0.75, 0.75)


# --------------------------------------------------------------------------
# native raycaster (input synthesis only)
# --------------------------------------------------------------------------
def _build_raycaster() -> str:
    src = os.path.join(_HERE, "raycast.c")
    with open(src, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, f"libvct_synth_{tag}.so")
    if not os.path.exists(so):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
               src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return so


def build() -> None:
    """Compile the raycaster (called by the repository build step)."""
    _lib()


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(_build_raycaster())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.vs_raycast.argtypes = [
                ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_double,
                ctypes.c_int, dp, ctypes.c_int, dp,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.vs_raycast.restype = None
            _LIB = lib
    return _LIB


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------
def random_light(rng: np.random.Generator) -> np.ndarray:
    while True:
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        if v[1] >= 0.3:
            return v


def random_boxes(n: int, count: int, rng: np.random.Generator):
    """Integer voxel boxes as (lo[3], hi[3], colour[3]) with hi exclusive, xyz order."""
    boxes = []
    smin, smax = max(1, n // 16), max(1, n // 4)
    for _ in range(count):
        size = rng.integers(smin, smax + 1, size=3)
        lo = np.array([rng.integers(0, n - s + 1) for s in size], dtype=np.int64)
        colour = rng.random(3)
        boxes.append((lo, lo + size, colour))
    return boxes


_FACES = [(0, -1), (0, +1), (1, -1), (1, +1), (2, -1), (2, +1)]


def _paint_solid(grid, lo, hi, face_colours, light):
    """Write one solid box: opacity 1, Lambert-lit shell, dark interior."""
    x0, y0, z0 = (int(v) for v in lo)
    x1, y1, z1 = (int(v) for v in hi)
    sub = np.zeros((z1 - z0, y1 - y0, x1 - x0, 4), dtype=np.float64)
    sub[..., 3] = 1.0
    for (axis, sign), col in zip(_FACES, face_colours):
        nf = np.zeros(3)
        nf[axis] = sign
        lam = max(0.0, float(nf @ light))
        val = np.asarray(col, dtype=np.float64) * lam
        sl = [slice(None)] * 3
        # array axes are (z, y, x) = (2, 1, 0)
        arr_axis = 2 - axis
        sl[arr_axis] = slice(0, 1) if sign < 0 else slice(-1, None)
        face = sub[tuple(sl)]
        np.maximum(face[..., :3], val, out=face[..., :3])
    grid[z0:z1, y0:y1, x0:x1] = sub.astype(np.float32)


def box_scene(n: int, n_boxes: int, seed: int, room: bool = False):
    """Seeded box scene; returns dict(grid, boxes, light, room)."""
    rng = np.random.default_rng(seed)
    light = random_light(rng)
    boxes = random_boxes(n, n_boxes, rng)
    grid = np.zeros((n, n, n, 4), dtype=np.float32)
    if room:
        _paint_room(grid, n, light)
    for lo, hi, col in boxes:
        _paint_solid(grid, lo, hi, [col] * 6, light)
    return {"n": n, "grid": grid, "boxes": boxes, "light": light, "room": room}


def _paint_room(grid, n, light):
    walls = [  # (axis, index, inward normal sign, colour)
        (0, 0, +1, RED), (0, n - 1, -1, GREEN),
        (1, 0, +1, GREY), (1, n - 1, -1, GREY),
        (2, 0, +1, GREY), (2, n - 1, -1, GREY)]
    rgb = np.zeros((n, n, n, 3), dtype=np.float64)
    solid = np.zeros((n, n, n), dtype=bool)
    for axis, idx, sign, col in walls:
        nf = np.zeros(3)
        nf[axis] = sign
        lam = max(0.0, float(nf @ light))
        sl = [slice(None)] * 3
        sl[2 - axis] = slice(idx, idx + 1)
        sl = tuple(sl)
        solid[sl] = True
        np.maximum(rgb[sl], np.asarray(col) * lam, out=rgb[sl])
    grid[..., :3] = np.where(solid[..., None], rgb, 0.0).astype(np.float32)
    grid[..., 3] = solid.astype(np.float32)


# --------------------------------------------------------------------------
# cameras and G-buffers
# --------------------------------------------------------------------------
def _inside_any(p, boxes, n, margin=0.0):
    q = np.asarray(p) * n
    for lo, hi, _ in boxes:
        if np.all(q >= lo - margin) and np.all(q <= hi + margin):
            return True
    return False


def interior_camera(rng, boxes, n, lo=0.12, hi=0.88):
    while True:
        p = lo + (hi - lo) * rng.random(3)
        if not _inside_any(p, boxes, n, margin=2.0):
            return p


def look_at(cam, target, up=(0.0, 1.0, 0.0)):
    f = np.asarray(target, dtype=np.float64) - cam
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    if np.linalg.norm(r) < 1e-6:
        r = np.cross(f, np.array([1.0, 0.0, 0.0]))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    return f, r, u


def raycast_gbuffer(scene, width, height, cam, target, fov_deg=60.0):
    """Pinhole G-buffer of a box scene: float32 pos/normal [H*W*3], uint8 mask."""
    n = scene["n"]
    f, r, u = look_at(cam, target)
    boxes = np.array([[*(lo / n), *(hi / n)] for lo, hi, _ in scene["boxes"]],
                     dtype=np.float64).reshape(-1, 6)
    room = np.array([1.0 / n] * 3 + [(n - 1.0) / n] * 3, dtype=np.float64)
    pos = np.empty(height * width * 3, dtype=np.float32)
    nrm = np.empty(height * width * 3, dtype=np.float32)
    mask = np.empty(height * width, dtype=np.uint8)
    cam = np.ascontiguousarray(cam, dtype=np.float64)
    f, r, u = (np.ascontiguousarray(v, dtype=np.float64) for v in (f, r, u))
    _lib().vs_raycast(width, height, _dptr(cam), _dptr(f), _dptr(r), _dptr(u),
                      math.tan(math.radians(fov_deg) / 2), len(boxes),
                      _dptr(np.ascontiguousarray(boxes)), int(scene["room"]),
                      _dptr(room), pos.ctypes.data, nrm.ctypes.data,
                      mask.ctypes.data)
    return pos, nrm, mask


def surface_gbuffer(scene, count, rng):
    """Seeded points on exposed box faces: each pixel picks a face by area,
    then a uniform point on it whose outside neighbourhood is empty."""
    n = scene["n"]
    faces = []
    for lo, hi, _ in scene["boxes"]:
        for axis, sign in _FACES:
            o1, o2 = [a for a in range(3) if a != axis]
            area = float((hi[o1] - lo[o1]) * (hi[o2] - lo[o2]))
            faces.append((lo, hi, axis, sign, o1, o2, area))
    areas = np.array([fc[6] for fc in faces])
    prob = areas / areas.sum()
    pos = np.empty((count, 3), dtype=np.float32)
    nrm = np.zeros((count, 3), dtype=np.float32)
    filled = 0
    while filled < count:
        k = rng.choice(len(faces), p=prob)
        lo, hi, axis, sign, o1, o2, _ = faces[k]
        q = np.empty(3)
        q[axis] = lo[axis] if sign < 0 else hi[axis]
        q[o1] = lo[o1] + rng.random() * (hi[o1] - lo[o1])
        q[o2] = lo[o2] + rng.random() * (hi[o2] - lo[o2])
        probe = q.copy()
        probe[axis] += 0.5 * sign
        if np.any(probe <= 0) or np.any(probe >= n):
            continue
        if _inside_any(probe / n, scene["boxes"], n):
            continue
        pos[filled] = (q / n).astype(np.float32)
        nrm[filled, axis] = sign
        filled += 1
    return pos.reshape(-1), nrm.reshape(-1), np.ones(count, dtype=np.uint8)


# --------------------------------------------------------------------------
# cone tables and trace parameters (inputs to both sides)
# --------------------------------------------------------------------------
def _sph(theta_deg, phi_deg):
    t, p = math.radians(theta_deg), math.radians(phi_deg)
    v = (math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t))
    return tuple(0.0 if abs(c) < 1e-12 else c for c in v)


def cone_table_ring6():
    """Front cone + five cones at 60 degrees polar; weights ~ cos(theta)."""
    dirs = [(0.0, 0.0, 1.0)] + [_sph(60.0, 72.0 * k) for k in range(5)]
    w = np.array([1.0] + [0.5] * 5)
    return np.array(dirs), w / w.sum()


def cone_table_thesis9():
    """The thesis's diffuse set (Ch. 5.4.4, cone configurations): front cone,
    four intermediate cones at 45 degrees, four side cones at 90 degrees on
    the same azimuths; equal weights 1/9."""
    dirs = [(0.0, 0.0, 1.0)]
    dirs += [_sph(45.0, 90.0 * k) for k in range(4)]
    dirs += [_sph(90.0, 90.0 * k) for k in range(4)]
    return np.array(dirs), np.full(9, 1.0 / 9.0)


def trace_params(dirs, weights, diffuse_aperture, spec_enable=True,
                 spec_aperture_min=math.radians(10.0),
                 spec_aperture_max=None, roughness_min=0.05, occ_enable=False,
                 occ_aperture=0.55, light=(0.0, 1.0, 0.0), beta=0.5,
                 t0_voxels=1.0, normal_offset_voxels=1.0, t_max=1.0):
    """Plain-dict trace parameters, float32-rounded as both sides see them."""
    f32 = lambda v: float(np.float32(v))
    return {
        "n_diffuse": int(len(dirs)),
        "diffuse_dir": np.asarray(dirs, dtype=np.float32).reshape(-1, 3),
        "diffuse_weight": np.asarray(weights, dtype=np.float32).reshape(-1),
        "diffuse_aperture": f32(diffuse_aperture),
        "spec_enable": int(bool(spec_enable)),
        "spec_aperture_min": f32(spec_aperture_min),
        "spec_aperture_max": f32(spec_aperture_min if spec_aperture_max is None
                                 else spec_aperture_max),
        "roughness_min": f32(roughness_min),
        "occ_enable": int(bool(occ_enable)),
        "occ_aperture": f32(occ_aperture),
        "light_dir": np.asarray(light, dtype=np.float32).reshape(3),
        "beta": f32(beta),
        "t0_voxels": f32(t0_voxels),
        "normal_offset_voxels": f32(normal_offset_voxels),
        "t_max": f32(t_max),
    }


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def view_dict(pos, nrm, mask, width, height, cam, roughness=None, pyramid=0):
    return {"width": width, "height": height, "position": pos, "normal": nrm,
            "mask": mask, "roughness": roughness,
            "camera": np.asarray(cam, dtype=np.float32), "pyramid": pyramid}


def config_small_fp32(n=64, n_boxes=12, width=128, height=128, seed=1):
    """64^3 grid, 12 boxes, 128x128 surface samples, 6 diffuse cones of 60
    degrees (cos-weighted) + one 10 degree specular cone, no occlusion cone."""
    rng = np.random.default_rng(seed)
    scene = box_scene(n, n_boxes, seed)
    pos, nrm, mask = surface_gbuffer(scene, width * height, rng)
    d = rng.normal(size=3)
    cam = 0.5 + 1.2 * d / np.linalg.norm(d)
    dirs, w = cone_table_ring6()
    prm = trace_params(dirs, w, math.radians(60.0), spec_enable=True,
                       spec_aperture_min=math.radians(10.0), occ_enable=False,
                       light=scene["light"])
    return {"name": f"{n}^3 {n_boxes} boxes, {width}x{height} surface samples, "
                    "6x60deg diffuse + 10deg specular",
            "scenes": [scene], "views": [view_dict(pos, nrm, mask, width, height, cam)],
            "params": prm}


def interior_view(scene, width, height, rng, with_roughness=True):
    n = scene["n"]
    cam = interior_camera(rng, scene["boxes"], n)
    target = interior_camera(rng, scene["boxes"], n)
    while np.linalg.norm(target - cam) < 0.2:
        target = interior_camera(rng, scene["boxes"], n)
    pos, nrm, mask = raycast_gbuffer(scene, width, height, cam, target)
    rough = None
    if with_roughness:
        rough = rng.uniform(0.05, 1.0, size=width * height).astype(np.float32)
    v = view_dict(pos, nrm, mask, width, height, cam, roughness=rough)
    v["target"] = np.asarray(target, dtype=np.float64)
    return v


def camera(eye, target, width, height, fov_deg=60.0, frame_origin=(0.0, 0.0, 0.0),
           frame_size=1.0):
    """Pinhole camera of the G-buffer pass: eye, unit forward / right / up
    (look_at, world up +y) and tan of half the vertical field of view, as
    float32; frame_origin / frame_size set the fixed-point frame the hit
    tests run in (the scene must lie within two frame sizes of the origin)."""
    eye = np.asarray(eye, dtype=np.float64)
    f, r, u = look_at(eye, target)
    f32 = lambda a: np.asarray(a, dtype=np.float32).reshape(3)  # noqa: E731
    return {"eye": f32(eye), "forward": f32(f), "right": f32(r), "up": f32(u),
            "tan_half": float(np.float32(math.tan(math.radians(fov_deg) / 2.0))),
            "width": int(width), "height": int(height), "frame_origin": f32(frame_origin),
            "frame_size": float(np.float32(frame_size))}


def box_mesh(scene, tess=1):
    """The boxes that raycast_gbuffer intersects, as triangles with faces on
    the box bounds (no inset): boxes outward, the room inward on
    [1/n, (n-1)/n]^3; scene units; colour per box (room walls grey)."""
    n = scene["n"]
    V, I, C = [], [], []
    count = 0

    def add(faces, colour):
        nonlocal count
        for cs, _, _ in faces:
            verts, tris = _quad_grid(*cs, tess)
            V.append(verts)
            I.append(tris + count)
            C.append(np.broadcast_to(np.asarray(colour, np.float64), (len(tris), 3)))
            count += len(verts)

    if scene.get("room"):
        add(_box_faces(np.full(3, 1.0), np.full(3, n - 1.0), 0.0, False), GREY)
    for lo, hi, col in scene["boxes"]:
        add(_box_faces(np.asarray(lo, np.float64), np.asarray(hi, np.float64), 0.0, True), col)
    return {"vertices": (np.concatenate(V) / n).astype(np.float32),
            "indices": np.concatenate(I).astype(np.int32),
            "colors": np.concatenate(C).astype(np.float32)}


# --------------------------------------------------------------------------
# triangle meshes (input of the voxelizer)
# --------------------------------------------------------------------------
def _quad_grid(c0, c1, c2, c3, tess):
    """tess x tess grid of quads over the bilinear patch c0 c1 c2 c3 (counter-
    clockwise seen from the side the face looks at): vertices, triangles."""
    t = np.linspace(0.0, 1.0, tess + 1)
    u, v = np.meshgrid(t, t, indexing="xy")
    u, v = u[..., None], v[..., None]
    p = ((1 - u) * (1 - v) * c0 + u * (1 - v) * c1 + u * v * c2 + (1 - u) * v * c3)
    verts = p.reshape(-1, 3)
    a, b = np.meshgrid(np.arange(tess), np.arange(tess), indexing="xy")
    i00 = (b * (tess + 1) + a).ravel()
    i10, i01 = i00 + 1, i00 + tess + 1
    i11 = i01 + 1
    tris = np.concatenate([np.stack([i00, i10, i11], 1), np.stack([i00, i11, i01], 1)])
    return verts, tris


def _box_faces(a, b, e, outward):
    """Six faces of the box with planes through a and b (voxel units), each
    extended in-plane to [a - e, b + e]; normals outward or inward."""
    faces = []
    for axis in range(3):
        u, v = [x for x in range(3) if x != axis]
        for side, pos in ((-1.0, a[axis]), (1.0, b[axis])):
            cs = []
            for cu, cv in ((a[u] - e, a[v] - e), (b[u] + e, a[v] - e), (b[u] + e, b[v] + e),
                           (a[u] - e, b[v] + e)):
                p = np.zeros(3)
                p[axis], p[u], p[v] = pos, cu, cv
                cs.append(p)
            nrm = np.zeros(3)
            nrm[axis] = side if outward else -side
            if np.cross(cs[1] - cs[0], cs[2] - cs[0]) @ nrm < 0:
                cs = [cs[0], cs[3], cs[2], cs[1]]
            faces.append((cs, axis, side))
    return faces


def _uv_sphere(c, r, stacks, slices):
    th = np.linspace(0.0, math.pi, stacks + 1)
    ph = np.linspace(0.0, 2.0 * math.pi, slices + 1)
    T, Ph = np.meshgrid(th, ph, indexing="ij")
    p = np.stack([np.sin(T) * np.cos(Ph), np.cos(T), np.sin(T) * np.sin(Ph)], -1)
    verts = (c + r * p).reshape(-1, 3)
    a, b = np.meshgrid(np.arange(slices), np.arange(stacks), indexing="xy")
    i00 = (b * (slices + 1) + a).ravel()
    i10, i01 = i00 + 1, i00 + slices + 1
    i11 = i01 + 1
    # outward: (p10 - p00) x (p11 - p00) points away from the centre
    tris = np.concatenate([np.stack([i00, i11, i10], 1), np.stack([i00, i01, i11], 1)])
    return verts, tris


def scene_mesh(scene, tess=1, n_spheres=0, sphere_res=(32, 64), seed=0):
    """Triangle mesh of a box scene: every box as six faces whose planes run
    through the centres of its outermost voxel layers (in-plane inset 1/4
    voxel), the room as six inward walls through the centres of the wall
    voxels, each face a tess x tess grid of quads; plus n_spheres UV spheres
    (random centre, radius n/24 .. n/10, random colour).  Scene units: the
    grid spans [0, 1]^3.  Returns dict(vertices float32 [V,3], indices int32
    [T,3], colors float32 [T,3])."""
    n = scene["n"]
    V, I, C = [], [], []
    count = 0

    def add(verts, tris, colour):
        nonlocal count
        V.append(verts)
        I.append(tris + count)
        C.append(np.broadcast_to(np.asarray(colour, np.float64), (len(tris), 3)))
        count += len(verts)

    if scene.get("room"):
        walls = {(0, -1.0): RED, (0, 1.0): GREEN}
        for cs, axis, side in _box_faces(np.full(3, 0.5), np.full(3, n - 0.5), 0.25, False):
            add(*_quad_grid(*cs, tess), walls.get((axis, side), GREY))
    for lo, hi, col in scene["boxes"]:
        for cs, _, _ in _box_faces(np.asarray(lo) + 0.5, np.asarray(hi) - 0.5, 0.25, True):
            add(*_quad_grid(*cs, tess), col)
    rng = np.random.default_rng(seed)
    for _ in range(n_spheres):
        r = rng.uniform(n / 24.0, n / 10.0)
        c = rng.uniform(r + 1.0, n - r - 1.0, size=3)
        add(*_uv_sphere(c, r, *sphere_res), rng.random(3))
    verts = np.concatenate(V) / n
    return {"vertices": verts.astype(np.float32), "indices": np.concatenate(I).astype(np.int32),
            "colors": np.concatenate(C).astype(np.float32)}


def albedo(width, height, seed):
    """Per-pixel material colour in [0.2, 1] (float32 [H*W, 3])."""
    rng = np.random.default_rng(seed)
    return (0.2 + 0.8 * rng.random((width * height, 3))).astype(np.float32)


def variant_params(prm, flags):
    """Parameters of the thesis's modified cones and shading (Ch. 5.4.4):
    occlusion fade-in over the first 0.3 scene units (shadow strength 1),
    Phong exponent 32 (angular grace 0.256 pi) with falloff 2, material
    ratios 0.8 / 0.6 and a warm light colour."""
    return dict(prm, flags=flags, shadow_str=1.0, occ_max_dist=0.3, shininess=32.0,
                shininess_falloff=2.0, diffuse_str=0.8, specular_str=0.6,
                light_color=(1.0, 0.9, 0.7))


def params_room9(light):
    dirs, w = cone_table_thesis9()
    return trace_params(dirs, w, 0.55, spec_enable=True,
                        spec_aperture_min=math.radians(5.0),
                        spec_aperture_max=math.radians(60.0), roughness_min=0.05,
                        occ_enable=True, occ_aperture=0.55, light=light)


def config_room_1080p(n=256, n_boxes=32, width=1920, height=1080, seed=2):
    """256^3 room with 32 boxes, 1920x1080 raycast G-buffer with per-pixel
    roughness in [0.05,1] (specular aperture 5..60 degrees), the thesis's nine
    0.55 rad diffuse cones, one specular and one 0.55 rad occlusion cone."""
    rng = np.random.default_rng(seed)
    scene = box_scene(n, n_boxes, seed, room=True)
    view = interior_view(scene, width, height, rng)
    return {"name": f"{n}^3 room + {n_boxes} boxes, {width}x{height}, 9 diffuse + "
                    "1 specular + 1 occlusion cone",
            "scenes": [scene], "views": [view], "params": params_room9(scene["light"])}


def config_room_mesh(n=256, n_boxes=32, seed=2, tess=24, n_spheres=4, width=1920,
                     height=1080):
    """The 256^3 room of config_room_1080p as a triangle mesh for per-frame
    revoxelization: tess 24 quads per face edge and four UV spheres, about
    244K triangles (a high-polygon scene), plus the 1080p view of the room."""
    c = config_room_1080p(n=n, n_boxes=n_boxes, width=width, height=height, seed=seed)
    scene = c["scenes"][0]
    c["mesh"] = scene_mesh(scene, tess=tess, n_spheres=n_spheres, seed=seed + 100)
    c["light"] = {"light_dir": np.asarray(scene["light"], np.float64),
                  "light_color": (1.0, 1.0, 1.0), "ambient": 0.0, "diffuse_str": 1.0}
    c["name"] += f", mesh of {len(c['mesh']['indices'])} triangles"
    return c


def config_batched(grids=(128, 256, 256, 512), views_per_scene=64, n_boxes=32,
                   scene_seeds=(41, 42, 43, 44), view_seed=45,
                   res_lo=(256, 256), res_hi=(1920, 1080)):
    """Several room scenes with many interior views of uneven resolution."""
    scenes = [box_scene(n, n_boxes, s, room=True) for n, s in zip(grids, scene_seeds)]
    rng = np.random.default_rng(view_seed)
    views = []
    for si, sc in enumerate(scenes):
        for _ in range(views_per_scene):
            w = int(rng.integers(res_lo[0], res_hi[0] + 1))
            h = int(rng.integers(res_lo[1], res_hi[1] + 1))
            v = interior_view(sc, w, h, rng)
            v["pyramid"] = si
            views.append(v)
    # one light for the batch: the first scene's (cone parameters are shared)
    return {"name": f"{len(scenes)} scenes {list(grids)} x {views_per_scene} views",
            "scenes": scenes, "views": views, "params": params_room9(scenes[0]["light"])}


def config_learnable(n=128, n_views=32, width=512, height=512, gt_seed=51,
                     view_seed=52, n_boxes=32, init=0.1):
    """Learnable grid at a constant value, views of a ground-truth box scene;
    cone set: the 6x60 degree diffuse ring, a 10 degree specular cone and a
    0.55 rad occlusion cone, so all three outputs carry gradient."""
    gt = box_scene(n, n_boxes, gt_seed, room=True)
    rng = np.random.default_rng(view_seed)
    views = [interior_view(gt, width, height, rng, with_roughness=False)
             for _ in range(n_views)]
    dirs, w = cone_table_ring6()
    prm = trace_params(dirs, w, math.radians(60.0), spec_enable=True,
                       spec_aperture_min=math.radians(10.0), occ_enable=True,
                       occ_aperture=0.55, light=gt["light"])
    learn = np.full((n, n, n, 4), init, dtype=np.float32)
    return {"name": f"learnable {n}^3 at {init}, {n_views} views {width}x{height}",
            "scenes": [gt], "learnable": learn, "views": views, "params": prm}
