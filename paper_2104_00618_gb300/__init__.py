"""GB300 voxel cone tracing: Python binding of libvct (argument marshalling only).

Every step of the hot path runs in the CUDA kernels behind ``include/vct.h``;
this module allocates caller-owned device buffers with PyTorch, fills the C
structs and calls the C ABI on PyTorch's current stream.  There is no
fallback: if libvct cannot be built or loaded, every call raises.

Main entry points
    build_mips(level0, ...)          -> Pyramid            (Ch. 4.3.3 mipmaps)
    trace(pyramids, views, params)   -> per-view outputs   (Ch. 4.2, 4.3.2, 4.5)
    trace_backward(...)              -> dL/d level-0 grid   (adjoint of both)
    voxelize(mesh, n, ...)           -> dense level-0 grid  (Ch. 4.4)
    TraceFn / render(...)            -> torch.autograd wrapper
"""
from __future__ import annotations

import ctypes
import dataclasses
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _abi
from ._abi import (FLAG_DIFFUSE_FIRST_HIT, FLAG_OCC_SMOOTH, FLAG_PREMULTIPLIED, FLAG_SHADE,
                   FLAG_SHADE_IMPL, FLAG_SPEC_GRACE, VCT_F16, VCT_F32, VctCamera, VctError,
                   VctGbufferStats, VctLaunchConfig, VctMesh,
                   VctPyramid, VctTraceParams, VctTraceStats, VctView, VctViewGrad,
                   VctVoxelizeStats, VctVoxelLight, check, load)

__all__ = ["Pyramid", "build_mips", "read_level", "read_volume", "pyramid_status", "make_params", "trace",
           "trace_backward", "autotune", "read_stats", "TraceFn", "render", "VctError",
           "launch_config", "num_levels", "lib", "FLAG_OCC_SMOOTH", "FLAG_SPEC_GRACE",
           "FLAG_DIFFUSE_FIRST_HIT", "FLAG_SHADE", "FLAG_SHADE_IMPL", "FLAG_PREMULTIPLIED",
           "Mesh", "voxelize",
           "voxelize_workspace", "read_voxelize_stats", "voxel_owner", "plan_bricks",
           "Pipeline", "gbuffer", "gbuffer_workspace", "read_gbuffer_stats", "gbuffer_view",
           "camera_struct"]

DTYPES = {"f32": VCT_F32, "f16": VCT_F16, VCT_F32: VCT_F32, VCT_F16: VCT_F16}
LAYOUTS = {"dense": _abi.LAYOUT_DENSE, "bricks": _abi.LAYOUT_BRICKS, "aniso": _abi.LAYOUT_ANISO,
           _abi.LAYOUT_ANISO: _abi.LAYOUT_ANISO,
           _abi.LAYOUT_DENSE: _abi.LAYOUT_DENSE, _abi.LAYOUT_BRICKS: _abi.LAYOUT_BRICKS}


def lib():
    return load()


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def num_levels(n: int) -> int:
    return n.bit_length()


def launch_config(tile_w=8, tile_h=8, lanes_per_pixel=1, ctas_per_sm=0) -> VctLaunchConfig:
    return VctLaunchConfig(tile_w, tile_h, lanes_per_pixel, ctas_per_sm)


# ---------------------------------------------------------------------------
# pyramids
# ---------------------------------------------------------------------------
class Pyramid:
    """A pyramid in a caller-owned (PyTorch) device buffer.  Dense by default;
    a brick pyramid (layout="bricks") needs the number of occupied bricks it
    will hold (see plan_bricks); layout="aniso" holds six directional
    volumes per coarse level (float32 only)."""

    def __init__(self, n: int, levels: int | None = None, dtype="f32",
                 origin=(0.0, 0.0, 0.0), size: float = 1.0, device=None,
                 layout: str = "dense", occupied: int | None = None):
        self.n = int(n)
        self.levels = num_levels(n) if levels is None else int(levels)
        self.dtype = DTYPES[dtype]
        self.origin = tuple(float(v) for v in origin)
        self.size = float(size)
        self.layout = LAYOUTS[layout]
        if self.layout == _abi.LAYOUT_BRICKS:
            if occupied is None:
                raise VctError(_abi.VCT_ERR_INVALID_ARG, "a brick pyramid needs `occupied`")
            nbytes = lib().vct_pyramid_bytes_bricks(self.n, self.levels, self.dtype,
                                                    int(occupied))
        elif self.layout == _abi.LAYOUT_ANISO:
            nbytes = lib().vct_pyramid_bytes_aniso(self.n, self.levels, self.dtype)
        else:
            nbytes = lib().vct_pyramid_bytes(self.n, self.levels, self.dtype)
        if nbytes == 0:
            raise VctError(_abi.VCT_ERR_INVALID_ARG,
                           f"invalid pyramid shape n={n} levels={levels} dtype={dtype}")
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.storage = torch.empty(nbytes, dtype=torch.uint8, device=dev)

    def struct(self) -> VctPyramid:
        return VctPyramid(self.n, self.levels, self.dtype, self.layout,
                          (ctypes.c_float * 3)(*self.origin), self.size,
                          self.storage.data_ptr(), self.storage.numel())

    def occupied_bricks(self) -> int:
        """Occupied-brick count recorded by the last build (brick layout)."""
        return int(self.storage[8:16].cpu().numpy().view(np.uint64)[0])

    def level_offset(self, level: int) -> int:
        return int(lib().vct_pyramid_level_offset(self.n, self.levels, self.dtype, level))


def _check_level0(level0):
    if level0.dtype != torch.float32 or not level0.is_cuda or level0.dim() != 4 \
            or level0.shape[3] != 4 or not level0.is_contiguous():
        raise VctError(_abi.VCT_ERR_INVALID_ARG,
                       "level0 must be a contiguous CUDA float32 tensor [n, n, n, 4]")


def plan_bricks(level0: torch.Tensor, levels: int | None = None, dtype="f32",
                stream=None) -> tuple[int, int]:
    """(occupied bricks, bytes) of a brick pyramid of this grid (synchronises)."""
    _check_level0(level0)
    n = level0.shape[0]
    levels = num_levels(n) if levels is None else int(levels)
    dt = DTYPES[dtype]
    sb = lib().vct_pyramid_plan_scratch_bytes(n, levels, dt)
    scratch = torch.empty(max(sb, 256), dtype=torch.uint8, device=level0.device)
    occ, nbytes = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().vct_pyramid_plan_bricks(_ptr(level0), n, levels, dt, _ptr(scratch), sb,
                                        ctypes.byref(occ), ctypes.byref(nbytes),
                                        _stream(stream)), "vct_pyramid_plan_bricks")
    return int(occ.value), int(nbytes.value)


def build_mips(level0: torch.Tensor, levels: int | None = None, dtype="f32",
               origin=(0.0, 0.0, 0.0), size: float = 1.0, out: Pyramid | None = None,
               stream=None, layout: str = "dense") -> Pyramid:
    """Morton-pack a dense float32 [n,n,n,4] (z,y,x,c) grid and build its mips
    (layout="bricks": plan the brick pool first, then build into it)."""
    _check_level0(level0)
    n = level0.shape[0]
    if out is None and LAYOUTS[layout] == _abi.LAYOUT_BRICKS:
        occ, _ = plan_bricks(level0, levels, dtype, stream)
        out = Pyramid(n, levels, dtype, origin, size, level0.device, "bricks", occ)
    pyr = out if out is not None else Pyramid(n, levels, dtype, origin, size, level0.device,
                                              layout)
    p = pyr.struct()
    check(lib().vct_build_mips(_ptr(level0), ctypes.byref(p), _stream(stream)), "vct_build_mips")
    return pyr


def read_level(pyr: Pyramid, level: int, stream=None) -> torch.Tensor:
    m = pyr.n >> level
    out = torch.empty((m, m, m, 4), dtype=torch.float32, device=pyr.storage.device)
    p = pyr.struct()
    check(lib().vct_pyramid_read_level(ctypes.byref(p), level, _ptr(out), _stream(stream)),
          "vct_pyramid_read_level")
    return out


def read_volume(pyr: Pyramid, level: int, direction: int, stream=None) -> torch.Tensor:
    """Volume `direction` (0..5 = +x, -x, +y, -y, +z, -z) of level `level` of
    an anisotropic pyramid as a dense [m,m,m,4] grid (direction 0 otherwise)."""
    m = pyr.n >> level
    out = torch.empty((m, m, m, 4), dtype=torch.float32, device=pyr.storage.device)
    p = pyr.struct()
    check(lib().vct_pyramid_read_volume(ctypes.byref(p), level, direction, _ptr(out),
                                        _stream(stream)), "vct_pyramid_read_volume")
    return out


def pyramid_status(pyr: Pyramid, stream=None) -> None:
    p = pyr.struct()
    check(lib().vct_pyramid_status(ctypes.byref(p), _stream(stream)), "vct_pyramid_status")


# ---------------------------------------------------------------------------
# parameters and views
# ---------------------------------------------------------------------------
def make_params(prm: dict) -> VctTraceParams:
    """vct_trace_params from a plain dict (keys as in include/vct.h)."""
    P = VctTraceParams()
    nd = int(prm["n_diffuse"])
    P.n_diffuse = nd
    dirs = torch.as_tensor(prm["diffuse_dir"], dtype=torch.float32).reshape(-1, 3)
    wts = torch.as_tensor(prm["diffuse_weight"], dtype=torch.float32).reshape(-1)
    for k in range(min(nd, _abi.MAX_DIFFUSE)):
        for a in range(3):
            P.diffuse_dir[k][a] = float(dirs[k, a])
        P.diffuse_weight[k] = float(wts[k])
    P.diffuse_aperture = float(prm["diffuse_aperture"])
    P.spec_enable = int(prm["spec_enable"])
    P.occ_enable = int(prm["occ_enable"])
    P.flags = int(prm.get("flags", 0))
    P.spec_aperture_min = float(prm["spec_aperture_min"])
    P.spec_aperture_max = float(prm["spec_aperture_max"])
    P.roughness_min = float(prm["roughness_min"])
    P.occ_aperture = float(prm["occ_aperture"])
    light = torch.as_tensor(prm["light_dir"], dtype=torch.float32).reshape(3)
    for a in range(3):
        P.light_dir[a] = float(light[a])
    P.beta = float(prm["beta"])
    P.t0_voxels = float(prm["t0_voxels"])
    P.normal_offset_voxels = float(prm["normal_offset_voxels"])
    P.t_max = float(prm["t_max"])
    P.shadow_str = float(prm.get("shadow_str", 1.0))
    P.occ_max_dist = float(prm.get("occ_max_dist", 1.0))
    P.shininess = float(prm.get("shininess", 32.0))
    P.shininess_falloff = float(prm.get("shininess_falloff", 1.0))
    P.diffuse_str = float(prm.get("diffuse_str", 1.0))
    P.specular_str = float(prm.get("specular_str", 1.0))
    lc = torch.as_tensor(prm.get("light_color", (1.0, 1.0, 1.0)), dtype=torch.float32).reshape(3)
    for a in range(3):
        P.light_color[a] = float(lc[a])
    return P


@dataclass
class View:
    """Device G-buffer of one view plus its output buffers."""
    width: int
    height: int
    position: torch.Tensor
    normal: torch.Tensor
    camera: tuple
    roughness: torch.Tensor | None = None
    mask: torch.Tensor | None = None
    pyramid: int = 0
    out_diffuse: torch.Tensor | None = None
    out_specular: torch.Tensor | None = None
    out_visibility: torch.Tensor | None = None
    albedo: torch.Tensor | None = None
    out_radiance: torch.Tensor | None = None
    cone_state: torch.Tensor | None = None
    keep: list = field(default_factory=list)

    @staticmethod
    def from_host(v: dict, device="cuda", outputs=True, non_blocking=False) -> "View":
        """Copies a host G-buffer dict (numpy/tensors) to the device."""
        def dev(a, dt):
            if a is None:
                return None
            t = torch.as_tensor(a)
            return t.to(device=device, dtype=dt, non_blocking=non_blocking).contiguous()
        w, h = int(v["width"]), int(v["height"])
        view = View(w, h, dev(v["position"], torch.float32), dev(v["normal"], torch.float32),
                    tuple(float(c) for c in v["camera"]),
                    dev(v.get("roughness"), torch.float32), dev(v.get("mask"), torch.uint8),
                    int(v.get("pyramid", 0)))
        view.albedo = dev(v.get("albedo"), torch.float32)
        if outputs:
            view.alloc_outputs()
        return view

    def alloc_outputs(self, diffuse=True, specular=True, visibility=True, radiance=False):
        dev = self.position.device
        npx = self.width * self.height
        self.out_diffuse = torch.empty((npx, 4), device=dev) if diffuse else None
        self.out_specular = torch.empty((npx, 4), device=dev) if specular else None
        self.out_visibility = torch.empty((npx,), device=dev) if visibility else None
        self.out_radiance = torch.empty((npx, 4), device=dev) if radiance else None
        return self

    def struct(self) -> VctView:
        return VctView(self.width, self.height, self.pyramid, 0, _ptr(self.position),
                       _ptr(self.normal), _ptr(self.roughness), _ptr(self.mask),
                       (ctypes.c_float * 3)(*self.camera), 0.0, _ptr(self.out_diffuse),
                       _ptr(self.out_specular), _ptr(self.out_visibility), _ptr(self.albedo),
                       _ptr(self.out_radiance), _ptr(self.cone_state))

    def alloc_cone_state(self, params) -> "View":
        """Buffer for the per-cone march state that vct_trace writes and
        vct_trace_backward reads (8 bytes per cone and pixel)."""
        P = params if isinstance(params, VctTraceParams) else make_params(params)
        n_cones = P.n_diffuse + P.spec_enable + P.occ_enable
        self.cone_state = torch.empty((n_cones, self.width * self.height, 2), dtype=torch.int32,
                                      device=self.position.device)
        return self


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.zeros(max(256, nbytes), dtype=torch.uint8, device=device)


def read_stats(workspace: torch.Tensor) -> dict:
    raw = workspace[:ctypes.sizeof(VctTraceStats)].cpu().numpy().tobytes()
    st = VctTraceStats.from_buffer_copy(raw)
    return {"samples": list(st.samples), "cones": list(st.cones), "status": int(st.status)}


def trace(pyramids, views, params, cfg: VctLaunchConfig | None = None,
          workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Traces every view into its output buffers; returns the workspace
    (read it with read_stats after the stream has reached this call)."""
    pyrs = list(pyramids) if isinstance(pyramids, (list, tuple)) else [pyramids]
    vs = list(views) if isinstance(views, (list, tuple)) else [views]
    P = params if isinstance(params, VctTraceParams) else make_params(params)
    parr = (VctPyramid * len(pyrs))(*[p.struct() for p in pyrs])
    varr = (VctView * len(vs))(*[v.struct() for v in vs])
    dev = pyrs[0].storage.device
    ws = workspace if workspace is not None else _workspace(lib().vct_trace_workspace_bytes(), dev)
    check(lib().vct_trace(parr, len(pyrs), varr, len(vs), ctypes.byref(P),
                          None if cfg is None else ctypes.byref(cfg), _ptr(ws), ws.numel(),
                          _stream(stream)), "vct_trace")
    return ws


def autotune(pyramids, views, params, workspace=None, stream=None) -> VctLaunchConfig:
    pyrs = list(pyramids) if isinstance(pyramids, (list, tuple)) else [pyramids]
    vs = list(views) if isinstance(views, (list, tuple)) else [views]
    P = params if isinstance(params, VctTraceParams) else make_params(params)
    parr = (VctPyramid * len(pyrs))(*[p.struct() for p in pyrs])
    varr = (VctView * len(vs))(*[v.struct() for v in vs])
    ws = workspace if workspace is not None else _workspace(
        lib().vct_trace_workspace_bytes(), pyrs[0].storage.device)
    best = VctLaunchConfig()
    check(lib().vct_autotune_trace(parr, len(pyrs), varr, len(vs), ctypes.byref(P), _ptr(ws),
                                   ws.numel(), _stream(stream), ctypes.byref(best)),
          "vct_autotune_trace")
    return best


def backward_workspace(pyr: Pyramid, deterministic: bool = False) -> torch.Tensor:
    p = pyr.struct()
    f = (lib().vct_trace_backward_deterministic_workspace_bytes if deterministic
         else lib().vct_trace_backward_workspace_bytes)
    nbytes = f(ctypes.byref(p))
    return torch.empty(nbytes, dtype=torch.uint8, device=pyr.storage.device)


def trace_backward(pyr: Pyramid, views, grads, params, grad_level0: torch.Tensor | None = None,
                   cfg: VctLaunchConfig | None = None, workspace: torch.Tensor | None = None,
                   stream=None, deterministic: bool = False) -> torch.Tensor:
    """Accumulates dL/d(level-0 grid) into grad_level0 ([n,n,n,4] float32).
    grads: per view (grad_D [H*W,4] | None, grad_S | None, grad_Vis [H*W] | None
    [, grad_L [H*W,4] | None]), grad_L the gradient of the shaded radiance.
    deterministic: the reproducible fixed-point accumulation
    (vct_trace_backward_deterministic)."""
    vs = list(views) if isinstance(views, (list, tuple)) else [views]
    P = params if isinstance(params, VctTraceParams) else make_params(params)
    if grad_level0 is None:
        grad_level0 = torch.zeros((pyr.n,) * 3 + (4,), dtype=torch.float32,
                                  device=pyr.storage.device)
    elif (tuple(grad_level0.shape) != (pyr.n,) * 3 + (4,) or grad_level0.dtype != torch.float32
          or not grad_level0.is_contiguous() or grad_level0.device != pyr.storage.device):
        raise ValueError(f"grad_level0 must be a contiguous float32 [{pyr.n}]^3 x 4 tensor on "
                         f"{pyr.storage.device}, got {tuple(grad_level0.shape)} "
                         f"{grad_level0.dtype} on {grad_level0.device}")
    ws = workspace if workspace is not None else backward_workspace(pyr, deterministic)
    p = pyr.struct()
    varr = (VctView * len(vs))(*[v.struct() for v in vs])
    keep = []
    garr = (VctViewGrad * len(vs))()
    for i, g in enumerate(grads):
        g = tuple(g) + (None,) * (4 - len(g))
        gd, gs, gv, gl = (None if t is None else t.contiguous() for t in g)
        keep.extend(t for t in (gd, gs, gv, gl) if t is not None)
        garr[i] = VctViewGrad(_ptr(gd), _ptr(gs), _ptr(gv), _ptr(gl))
    fn = lib().vct_trace_backward_deterministic if deterministic else lib().vct_trace_backward
    check(fn(ctypes.byref(p), varr, garr, len(vs), ctypes.byref(P),
             None if cfg is None else ctypes.byref(cfg), _ptr(grad_level0), _ptr(ws), ws.numel(),
             _stream(stream)), "vct_trace_backward")
    return grad_level0


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------
class TraceFn(torch.autograd.Function):
    """(level-0 grid) -> (D, S, Vis, L) of one view; backward through the
    cone march (any variant), the shading epilogue and the mip box filter by
    the hand-written adjoint kernels.  L is an empty tensor unless the
    params carry VCT_FLAG_SHADE."""

    @staticmethod
    def forward(ctx, level0, view: View, params, levels, origin, size, dtype, layout,
                deterministic):
        pyr = build_mips(level0.detach().contiguous(), levels, dtype, origin, size,
                         layout=layout)
        v = dataclasses.replace(view, keep=[])
        shade = bool(params.flags & FLAG_SHADE)
        v.alloc_outputs(radiance=shade)
        v.alloc_cone_state(params)  # lets the adjoint skip its forward march
        trace(pyr, [v], params)
        ctx.pyr, ctx.view, ctx.params, ctx.det = pyr, v, params, deterministic
        L = v.out_radiance if shade else torch.empty(0, device=level0.device)
        return v.out_diffuse, v.out_specular, v.out_visibility, L

    @staticmethod
    def backward(ctx, gD, gS, gV, gL):
        gl = gL if (ctx.params.flags & FLAG_SHADE) and gL is not None and gL.numel() else None
        grad = trace_backward(ctx.pyr, [ctx.view], [(gD, gS, gV, gl)], ctx.params,
                              deterministic=ctx.det)
        return grad, None, None, None, None, None, None, None, None


def render(level0: torch.Tensor, view: View, params, levels=None, origin=(0.0, 0.0, 0.0),
           size: float = 1.0, dtype: str = "f32", layout: str = "dense",
           deterministic: bool = False):
    """Differentiable (D, S, Vis) of one view from a level-0 grid, plus the
    shaded radiance L when the params carry the shading flag.  dtype /
    layout: the pyramid's storage (the gradient is always float32, dense);
    deterministic: the reproducible fixed-point adjoint."""
    P = params if isinstance(params, VctTraceParams) else make_params(params)
    D, S, V, L = TraceFn.apply(level0, view, P, levels, origin, size, dtype, layout,
                               deterministic)
    return (D, S, V, L) if P.flags & FLAG_SHADE else (D, S, V)


# ---------------------------------------------------------------------------
# voxelization
# ---------------------------------------------------------------------------
@dataclass
class Mesh:
    """Triangle mesh on the device: vertices [V,3] float32, indices [T,3]
    int32, colors [T,3] float32 (material colour per triangle)."""
    vertices: torch.Tensor
    indices: torch.Tensor
    colors: torch.Tensor

    @staticmethod
    def from_host(m: dict, device="cuda") -> "Mesh":
        def dev(a, dt):
            return torch.as_tensor(a).to(device=device, dtype=dt).contiguous()
        return Mesh(dev(m["vertices"], torch.float32).reshape(-1, 3),
                    dev(m["indices"], torch.int32).reshape(-1, 3),
                    dev(m["colors"], torch.float32).reshape(-1, 3))

    def struct(self) -> VctMesh:
        return VctMesh(_ptr(self.vertices), _ptr(self.indices), _ptr(self.colors),
                       self.vertices.shape[0], self.indices.shape[0])


def voxelize_workspace(n: int, n_triangles: int, device="cuda") -> torch.Tensor:
    nbytes = lib().vct_voxelize_workspace_bytes(int(n), int(n_triangles))
    if nbytes == 0:
        raise VctError(_abi.VCT_ERR_INVALID_ARG, f"invalid voxelize size n={n}")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def voxelize(mesh: Mesh, n: int, origin=(0.0, 0.0, 0.0), size: float = 1.0,
             light: dict | None = None, out: torch.Tensor | None = None,
             workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Voxelizes the mesh into a dense float32 [n,n,n,4] grid (z,y,x,rgba).
    light: dict(light_dir, light_color, ambient, diffuse_str)."""
    light = light or {}
    L = VctVoxelLight()
    ld = [float(v) for v in light.get("light_dir", (0.0, 1.0, 0.0))]
    lc = [float(v) for v in light.get("light_color", (1.0, 1.0, 1.0))]
    for a in range(3):
        L.light_dir[a], L.light_color[a] = ld[a], lc[a]
    L.ambient = float(light.get("ambient", 0.0))
    L.diffuse_str = float(light.get("diffuse_str", 1.0))
    dev = mesh.vertices.device
    if out is None:
        out = torch.empty((n, n, n, 4), dtype=torch.float32, device=dev)
    ws = workspace if workspace is not None else voxelize_workspace(n, mesh.indices.shape[0], dev)
    m = mesh.struct()
    org = (ctypes.c_float * 3)(*[float(v) for v in origin])
    check(lib().vct_voxelize(ctypes.byref(m), int(n), org, float(size), ctypes.byref(L),
                             _ptr(out), _ptr(ws), ws.numel(), _stream(stream)), "vct_voxelize")
    return out


def read_voxelize_stats(workspace: torch.Tensor) -> dict:
    raw = workspace[:ctypes.sizeof(VctVoxelizeStats)].cpu().numpy().tobytes()
    st = VctVoxelizeStats.from_buffer_copy(raw)
    return {"fragments": int(st.fragments), "skipped": int(st.skipped),
            "degenerate": int(st.degenerate), "large_triangles": int(st.large_triangles),
            "large_items": int(st.large_items)}


def voxel_owner(workspace: torch.Tensor, n: int) -> torch.Tensor:
    """The owner grid of the last vct_voxelize on this workspace: [n,n,n]
    int32, triangle index + 1 per voxel (0 = empty)."""
    return workspace[256:256 + 4 * n * n * n].view(torch.int32).reshape(n, n, n)


# ---------------------------------------------------------------------------
# camera G-buffer
# ---------------------------------------------------------------------------
def camera_struct(cam: dict) -> VctCamera:
    """dict(eye, forward, right, up, tan_half, width, height, frame_origin,
    frame_size) -> vct_camera."""
    c = VctCamera()
    for k, f in (("eye", "eye"), ("forward", "forward"), ("right", "right"), ("up", "up"),
                 ("frame_origin", "frame_origin")):
        v = [float(x) for x in cam[k]]
        for a in range(3):
            getattr(c, f)[a] = v[a]
    c.tan_half_fov = float(cam["tan_half"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.frame_size = float(cam.get("frame_size", 1.0))
    return c


def gbuffer_workspace(width: int, height: int, n_triangles: int, pair_capacity: int | None = None,
                      device="cuda") -> torch.Tensor:
    """Workspace of vct_gbuffer; by default room for 8 (tile, triangle)
    pairs per triangle plus 64 per 16x16 tile."""
    if pair_capacity is None:
        tiles = ((width + 15) // 16) * ((height + 15) // 16)
        pair_capacity = 8 * n_triangles + 64 * tiles
    nbytes = lib().vct_gbuffer_workspace_bytes(int(width), int(height), int(n_triangles),
                                               int(pair_capacity))
    if nbytes == 0:
        raise VctError(_abi.VCT_ERR_INVALID_ARG, f"invalid G-buffer size {width}x{height}")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def read_gbuffer_stats(workspace: torch.Tensor) -> dict:
    raw = workspace[:ctypes.sizeof(VctGbufferStats)].cpu().numpy().tobytes()
    st = VctGbufferStats.from_buffer_copy(raw)
    return {k: int(getattr(st, k)) for k in ("pairs", "pair_capacity", "skipped", "degenerate",
                                             "culled", "wide", "overflow")}


def gbuffer(mesh: Mesh, cam: dict, out: dict | None = None, workspace: torch.Tensor | None = None,
            verify: bool = True, stream=None) -> dict:
    """Draws the mesh into a G-buffer (vct_gbuffer).  Returns dict of device
    tensors position / normal / albedo [H*W,3] float32, mask [H*W] uint8,
    triangle [H*W] int32 and the workspace.  verify: read the stats back
    (synchronises) and, if the tile lists overflowed, redo the call with a
    workspace of the needed size."""
    W, H = int(cam["width"]), int(cam["height"])
    dev = mesh.vertices.device
    if out is None:
        out = {"position": torch.empty((W * H, 3), device=dev),
               "normal": torch.empty((W * H, 3), device=dev),
               "albedo": torch.empty((W * H, 3), device=dev),
               "mask": torch.empty((W * H,), dtype=torch.uint8, device=dev),
               "triangle": torch.empty((W * H,), dtype=torch.int32, device=dev)}
    nt = mesh.indices.shape[0]
    ws = workspace if workspace is not None else gbuffer_workspace(W, H, nt, device=dev)
    c, m = camera_struct(cam), mesh.struct()
    for _ in range(2):
        check(lib().vct_gbuffer(ctypes.byref(m), ctypes.byref(c), _ptr(out["position"]),
                                _ptr(out["normal"]), _ptr(out.get("albedo")),
                                _ptr(out.get("mask")), _ptr(out.get("triangle")), _ptr(ws),
                                ws.numel(), _stream(stream)), "vct_gbuffer")
        if not verify:
            break
        st = read_gbuffer_stats(ws)
        if not st["overflow"]:
            break
        ws = gbuffer_workspace(W, H, nt, st["pairs"], device=dev)
    out["workspace"] = ws
    return out


def gbuffer_view(g: dict, cam: dict, roughness: torch.Tensor | None = None,
                 pyramid: int = 0) -> View:
    """A View over the buffers of gbuffer() (position, normal, mask, albedo)."""
    v = View(int(cam["width"]), int(cam["height"]), g["position"], g["normal"],
             tuple(float(x) for x in cam["eye"]), roughness, g.get("mask"), pyramid)
    v.albedo = g.get("albedo")
    return v.alloc_outputs()


# ---------------------------------------------------------------------------
# host-buffer frame pipeline
# ---------------------------------------------------------------------------
class Pipeline:
    """Frames whose inputs and outputs live in (page-locked) host memory:
    copies in, mip build + trace, copies out, overlapped across two device
    slots by the library (vct_pipeline_*).  Host tensors passed to submit()
    must stay alive and unchanged until join() has been reached."""

    def __init__(self, n: int, width: int, height: int, params, levels: int | None = None,
                 dtype="f32", origin=(0.0, 0.0, 0.0), size: float = 1.0,
                 has_roughness=True, has_mask=True, outputs=7):
        d = _abi.VctPipelineDesc()
        d.n, d.levels, d.dtype = int(n), num_levels(n) if levels is None else int(levels), \
            DTYPES[dtype]
        d.width, d.height = int(width), int(height)
        d.has_roughness, d.has_mask, d.outputs = int(has_roughness), int(has_mask), int(outputs)
        for a in range(3):
            d.origin[a] = float(origin[a])
        d.size = float(size)
        self.desc = d
        self.params = params if isinstance(params, VctTraceParams) else make_params(params)
        self._h = ctypes.c_void_p()
        check(lib().vct_pipeline_create(ctypes.byref(d), ctypes.byref(self.params),
                                        ctypes.byref(self._h)), "vct_pipeline_create")
        self._keep = []

    def submit(self, level0, position, normal, camera, out_diffuse=None, out_specular=None,
               out_visibility=None, roughness=None, mask=None, stream=None):
        f = _abi.VctHostFrame()
        f.level0, f.position, f.normal = _ptr(level0), _ptr(position), _ptr(normal)
        f.roughness, f.mask = _ptr(roughness), _ptr(mask)
        for a in range(3):
            f.camera[a] = float(camera[a])
        f.out_diffuse, f.out_specular = _ptr(out_diffuse), _ptr(out_specular)
        f.out_visibility = _ptr(out_visibility)
        self._keep.append((level0, position, normal, roughness, mask, out_diffuse, out_specular,
                           out_visibility))
        check(lib().vct_pipeline_submit(self._h, ctypes.byref(f), _stream(stream)),
              "vct_pipeline_submit")

    def join(self, stream=None):
        """Makes `stream` (default: the current one) wait for every frame so far."""
        check(lib().vct_pipeline_join(self._h, _stream(stream)), "vct_pipeline_join")

    def wait(self):
        """Blocks until every submitted frame is done; host outputs are final."""
        s = torch.cuda.current_stream()
        self.join(s)
        s.synchronize()
        self._keep = []

    def stats(self, slot: int) -> dict:
        st = VctTraceStats()
        check(lib().vct_pipeline_stats(self._h, int(slot), ctypes.byref(st)),
              "vct_pipeline_stats")
        return {"samples": list(st.samples), "cones": list(st.cones)}

    def close(self):
        if self._h:
            lib().vct_pipeline_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
