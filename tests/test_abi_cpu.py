"""The C ABI library builds, loads and exports every declared entry point;
host-side validation and layout queries work without a GPU."""
import ctypes
import os
import re

import pytest

import paper_2104_00618_gb300 as vct
from paper_2104_00618_gb300 import _abi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "vct.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vct_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return _abi.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_abi.EXPORTS), "binding and header disagree"


def test_struct_sizes_match_header_layout():
    assert ctypes.sizeof(_abi.VctPyramid) == 48
    assert ctypes.sizeof(_abi.VctView) == 112
    assert ctypes.sizeof(_abi.VctLaunchConfig) == 16
    assert ctypes.sizeof(_abi.VctTraceStats) == 56
    assert ctypes.sizeof(_abi.VctTraceParams) == 16 + 32 * 12 + 32 * 4 + 4 * 5 + 12 + 16 + 4 * 9


def test_pyramid_layout(lib):
    for n in (2, 8, 64, 256, 1024):
        L = n.bit_length()
        for dt, tb in ((0, 16), (1, 8)):
            off = 256
            for l in range(L):
                assert lib.vct_pyramid_level_offset(n, L, dt, l) == off
                m = n >> l
                off += (m ** 3 * tb + 255) // 256 * 256
            total = lib.vct_pyramid_bytes(n, L, dt)
            assert total >= off
            if dt == 0:
                assert total == off
    assert lib.vct_pyramid_bytes(3, 1, 0) == 0        # not a power of two
    assert lib.vct_pyramid_bytes(2048, 12, 0) == 0    # too large
    assert lib.vct_pyramid_bytes(64, 8, 0) == 0       # too many levels
    assert lib.vct_pyramid_bytes(64, 7, 2) == 0       # bad dtype


def test_status_strings(lib):
    assert lib.vct_status_string(0) == b"VCT_OK"
    assert lib.vct_status_string(5) == b"VCT_ERR_TIMEOUT"
    assert lib.vct_version() == 1


def test_validation_without_gpu(lib):
    # every one of these is rejected before any CUDA call
    assert lib.vct_build_mips(None, None, None) == _abi.VCT_ERR_INVALID_ARG
    p = _abi.VctPyramid(64, 7, 0, 0, (ctypes.c_float * 3)(0, 0, 0), 1.0, 256, 10)
    assert lib.vct_build_mips(None, ctypes.byref(p), None) == _abi.VCT_ERR_INVALID_ARG
    assert b"bytes" in lib.vct_last_error()
    assert lib.vct_trace(None, 0, None, 0, None, None, None, 0, None) == _abi.VCT_ERR_INVALID_ARG
    prm = vct.make_params({"n_diffuse": 1, "diffuse_dir": [[0, 0, 1]], "diffuse_weight": [1],
                           "diffuse_aperture": 0.0, "spec_enable": 0, "occ_enable": 0,
                           "spec_aperture_min": 0.1, "spec_aperture_max": 0.1,
                           "roughness_min": 0.05, "occ_aperture": 0.5, "light_dir": [0, 1, 0],
                           "beta": 0.5, "t0_voxels": 1.0, "normal_offset_voxels": 1.0,
                           "t_max": 1.0})
    p = _abi.VctPyramid(64, 7, 0, 0, (ctypes.c_float * 3)(0, 0, 0), 1.0, 256,
                        lib.vct_pyramid_bytes(64, 7, 0))
    v = _abi.VctView()
    v.width, v.height, v.position, v.normal, v.out_diffuse = 4, 4, 1024, 2048, 4096
    st = lib.vct_trace(ctypes.byref(p), 1, ctypes.byref(v), 1, ctypes.byref(prm), None,
                       None, 0, None)
    assert st == _abi.VCT_ERR_INVALID_ARG and b"aperture" in lib.vct_last_error()
    prm.diffuse_aperture = 0.5
    st = lib.vct_trace(ctypes.byref(p), 1, ctypes.byref(v), 1, ctypes.byref(prm), None,
                       None, 0, None)
    assert st == _abi.VCT_ERR_WORKSPACE
    p16 = _abi.VctPyramid(64, 7, 1, 0, (ctypes.c_float * 3)(0, 0, 0), 1.0, 256,
                          lib.vct_pyramid_bytes(64, 7, 1))
    g = _abi.VctViewGrad()
    st = lib.vct_trace_backward(ctypes.byref(p16), ctypes.byref(v), ctypes.byref(g), 1,
                                ctypes.byref(prm), None, None, None, 0, None)
    assert st == _abi.VCT_ERR_INVALID_ARG and b"grad_level0" in lib.vct_last_error()
    assert lib.vct_debug_wait_probe(None, 10, None) == _abi.VCT_ERR_INVALID_ARG


def test_variant_flag_validation_without_gpu(lib):
    """Flag combinations the library refuses before any CUDA call."""
    base = {"n_diffuse": 1, "diffuse_dir": [[0, 0, 1]], "diffuse_weight": [1],
            "diffuse_aperture": 0.5, "spec_enable": 1, "occ_enable": 1,
            "spec_aperture_min": 0.1, "spec_aperture_max": 0.3, "roughness_min": 0.05,
            "occ_aperture": 0.5, "light_dir": [0, 1, 0], "beta": 0.5, "t0_voxels": 1.0,
            "normal_offset_voxels": 1.0, "t_max": 1.0}
    p = _abi.VctPyramid(64, 7, 0, 0, (ctypes.c_float * 3)(0, 0, 0), 1.0, 256,
                        lib.vct_pyramid_bytes(64, 7, 0))
    v = _abi.VctView()
    v.width, v.height, v.position, v.normal, v.out_diffuse = 4, 4, 1024, 2048, 4096

    def run(flags, view=v, **kw):
        prm = vct.make_params(dict(base, flags=flags, **kw))
        return lib.vct_trace(ctypes.byref(p), 1, ctypes.byref(view), 1, ctypes.byref(prm),
                             None, None, 0, None)

    assert run(64) == _abi.VCT_ERR_INVALID_ARG and b"unknown flags" in lib.vct_last_error()
    assert run(_abi.FLAG_SHADE_IMPL) == _abi.VCT_ERR_INVALID_ARG
    assert run(_abi.FLAG_OCC_SMOOTH, occ_max_dist=0.0) == _abi.VCT_ERR_INVALID_ARG
    assert run(_abi.FLAG_SPEC_GRACE, shininess=-1.0) == _abi.VCT_ERR_INVALID_ARG
    assert run(_abi.FLAG_SHADE, light_dir=[0, 0, 0]) == _abi.VCT_ERR_INVALID_ARG
    assert run(_abi.FLAG_SHADE, light_color=[1, float("nan"), 1]) == _abi.VCT_ERR_INVALID_ARG
    # radiance output only with the shading flag; width/height are 16-bit
    vr = _abi.VctView.from_buffer_copy(v)
    vr.out_radiance = 8192
    assert run(0, view=vr) == _abi.VCT_ERR_INVALID_ARG and b"out_radiance" in lib.vct_last_error()
    vr.out_radiance = 8200
    assert run(_abi.FLAG_SHADE, view=vr) == _abi.VCT_ERR_INVALID_ARG  # misaligned
    vw = _abi.VctView.from_buffer_copy(v)
    vw.width = 65536
    assert run(0, view=vw) == _abi.VCT_ERR_INVALID_ARG
    # every valid combination passes validation (and stops at the workspace)
    vr.out_radiance = 8192
    for flags in range(64):
        if flags & _abi.FLAG_SHADE_IMPL and not flags & _abi.FLAG_SHADE:
            continue
        view = vr if flags & _abi.FLAG_SHADE else v
        assert run(flags, view=view) == _abi.VCT_ERR_WORKSPACE, (flags, lib.vct_last_error())
    # the adjoint takes every flag (validation then stops at the missing gradient grid)
    g = _abi.VctViewGrad()
    for flags, want in [(_abi.FLAG_OCC_SMOOTH, _abi.VCT_ERR_INVALID_ARG),
                        (_abi.FLAG_DIFFUSE_FIRST_HIT, _abi.VCT_ERR_INVALID_ARG),
                        (_abi.FLAG_SPEC_GRACE, _abi.VCT_ERR_INVALID_ARG),
                        (_abi.FLAG_PREMULTIPLIED, _abi.VCT_ERR_INVALID_ARG),
                        (_abi.FLAG_SHADE, _abi.VCT_ERR_INVALID_ARG)]:
        prm = vct.make_params(dict(base, flags=flags))
        st = lib.vct_trace_backward(ctypes.byref(p), ctypes.byref(v), ctypes.byref(g), 1,
                                    ctypes.byref(prm), None, None, None, 0, None)
        assert st == want, (flags, lib.vct_last_error())


def test_voxelize_structs_and_validation(lib):
    assert ctypes.sizeof(_abi.VctMesh) == 32
    assert ctypes.sizeof(_abi.VctVoxelLight) == 32
    assert ctypes.sizeof(_abi.VctVoxelizeStats) == 40
    n = 64
    assert lib.vct_voxelize_workspace_bytes(n, 0) == 256 + 4 * n ** 3
    assert lib.vct_voxelize_workspace_bytes(n, 1000) == 256 + 4 * n ** 3 + 16128 + 2 * 8192
    assert lib.vct_voxelize_workspace_bytes(48, 10) == 0
    assert lib.vct_voxelize_workspace_bytes(2048, 10) == 0
    m = _abi.VctMesh(1024, 2048, 4096, 3, 1)
    L = _abi.VctVoxelLight((ctypes.c_float * 3)(0, 1, 0), (ctypes.c_float * 3)(1, 1, 1), 0.0, 1.0)
    org = (ctypes.c_float * 3)(0, 0, 0)
    ws_need = lib.vct_voxelize_workspace_bytes(n, 1)

    def run(mesh=m, nn=n, size=1.0, out=8192, ws=1 << 20, ws_bytes=ws_need):
        return lib.vct_voxelize(ctypes.byref(mesh), nn, org, size, ctypes.byref(L), out, ws,
                                ws_bytes, None)

    assert run(nn=48) == _abi.VCT_ERR_INVALID_ARG
    assert run(size=0.0) == _abi.VCT_ERR_INVALID_ARG
    assert run(out=8200) == _abi.VCT_ERR_INVALID_ARG
    assert run(ws_bytes=ws_need - 1) == _abi.VCT_ERR_WORKSPACE
    assert run(ws=(1 << 20) + 8) == _abi.VCT_ERR_WORKSPACE
    bad = _abi.VctMesh(1024, 0, 4096, 3, 1)
    assert run(mesh=bad) == _abi.VCT_ERR_INVALID_ARG
    neg = _abi.VctMesh(1024, 2048, 4096, -1, 1)
    assert run(mesh=neg) == _abi.VCT_ERR_INVALID_ARG
    L.light_dir[1] = float("inf")
    assert run() == _abi.VCT_ERR_INVALID_ARG


def test_gbuffer_structs_and_validation(lib):
    """Camera G-buffer: workspace layout (stats, tile offsets and cursors,
    96-byte triangle records, pairs) and every argument check that needs no
    GPU."""
    assert ctypes.sizeof(_abi.VctCamera) == 76
    assert ctypes.sizeof(_abi.VctGbufferStats) == 48

    def al(x):
        return (x + 255) // 256 * 256
    W, H, nt = 100, 40, 1000
    T = 7 * 3
    fixed = 256 + al((T + 1) * 4) + al(T * 4) + al(nt * 96)
    assert lib.vct_gbuffer_workspace_bytes(W, H, nt, 0) == fixed
    assert lib.vct_gbuffer_workspace_bytes(W, H, nt, 1000) == fixed + al(4000)
    assert lib.vct_gbuffer_workspace_bytes(0, H, nt, 0) == 0
    assert lib.vct_gbuffer_workspace_bytes(W, 16385, nt, 0) == 0
    assert lib.vct_gbuffer_workspace_bytes(W, H, nt, (1 << 31) + 1) == 0
    m = _abi.VctMesh(1024, 2048, 4096, 3, 1)
    f3 = lambda *v: (ctypes.c_float * 3)(*v)  # noqa: E731

    def cam(**kw):
        c = _abi.VctCamera(f3(0.5, 0.5, 0.1), f3(0, 0, 1), f3(-1, 0, 0), f3(0, 1, 0), 0.577, W,
                           H, f3(0, 0, 0), 1.0)
        for k, v in kw.items():
            setattr(c, k, v)
        return c

    need = lib.vct_gbuffer_workspace_bytes(W, H, 1, 0)

    def run(c=None, mesh=m, pos=8192, nrm=16384, ws=1 << 20, ws_bytes=need):
        c = c or cam()
        return lib.vct_gbuffer(ctypes.byref(mesh), ctypes.byref(c), pos, nrm, None, None, None,
                               ws, ws_bytes, None)

    bad = _abi.VCT_ERR_INVALID_ARG
    assert run(cam(width=0)) == bad
    assert run(cam(tan_half_fov=0.0)) == bad
    assert run(cam(tan_half_fov=1.5)) == bad                 # tx + ty > 2.99 at 100x40
    assert run(cam(frame_size=-1.0)) == bad
    assert run(cam(eye=f3(0.5, 0.5, 2.5))) == bad            # beyond two frame sizes
    assert run(cam(forward=f3(0, 0, 1.01))) == bad           # component > 1 + 2^-10
    assert run(cam(up=f3(0, 0, 1))) == bad                   # basis det 0
    assert run(pos=0) == bad and run(nrm=16386) == bad
    assert run(mesh=_abi.VctMesh(1024, 0, 4096, 3, 1)) == bad
    assert run(ws_bytes=need - 1) == _abi.VCT_ERR_WORKSPACE
    assert run(ws=(1 << 20) + 16) == _abi.VCT_ERR_WORKSPACE


def test_debug_bounds_variant_loads(lib):
    """The bounds-checked variant exports the same entry points; the release
    library reports that it has no bounds checks."""
    dbg = _abi.open_library("debug_bounds")
    for name in _abi.EXPORTS:
        assert hasattr(dbg, name), name
    out = ctypes.c_uint32(5)
    assert lib.vct_debug_bounds_flags(ctypes.byref(out), 0) == _abi.VCT_ERR_UNSUPPORTED
    assert out.value == 0
    assert lib.vct_debug_bounds_probe(8192, 10, 1, None) == _abi.VCT_ERR_UNSUPPORTED
    assert lib.vct_debug_bounds_probe(8192, 10, 0, None) == _abi.VCT_ERR_INVALID_ARG
    assert dbg.vct_debug_bounds_probe(8192, 0, 1, None) == _abi.VCT_ERR_INVALID_ARG


def test_brick_layout_sizes_and_validation(lib):
    """Brick layout: per bricked level a uint32 slot table, small levels
    dense, FP32 staging, then the pool (zero brick + occupied bricks)."""
    def al(x):
        return (x + 255) // 256 * 256
    n, levels = 64, 7
    for dtype, tb in ((0, 16), (1, 8)):
        fixed = 256
        for l in range(levels):
            m = n >> l
            fixed += al((m ** 3 // 512) * 4) if m >= 16 else al(m ** 3 * tb)
        fixed += al((n // 16) ** 3 * 16) + al((n // 32) ** 3 * 16)  # staging (block 16)
        assert lib.vct_pyramid_plan_scratch_bytes(n, levels, dtype) == fixed
        assert lib.vct_pyramid_bytes_bricks(n, levels, dtype, 0) == fixed + 512 * tb
        assert lib.vct_pyramid_bytes_bricks(n, levels, dtype, 10) == fixed + 11 * 512 * tb
    assert lib.vct_pyramid_bytes_bricks(48, 3, 0, 5) == 0
    p = _abi.VctPyramid(64, 7, 0, 2, (ctypes.c_float * 3)(0, 0, 0), 1.0, 256,
                        lib.vct_pyramid_bytes(64, 7, 0))
    assert lib.vct_build_mips(1024, ctypes.byref(p), None) == _abi.VCT_ERR_INVALID_ARG
    p.layout = _abi.LAYOUT_BRICKS
    p.bytes = lib.vct_pyramid_plan_scratch_bytes(64, 7, 0)  # no room for the zero brick
    assert lib.vct_build_mips(1024, ctypes.byref(p), None) == _abi.VCT_ERR_INVALID_ARG
    occ, nb = ctypes.c_uint64(), ctypes.c_uint64()
    st = lib.vct_pyramid_plan_bricks(1024, 64, 7, 0, 256, 100, ctypes.byref(occ),
                                     ctypes.byref(nb), None)
    assert st == _abi.VCT_ERR_WORKSPACE


def test_aniso_layout_and_adjoint_workspace_sizes(lib):
    """Anisotropic pyramids: level 0 as dense, six volumes per level >= 1
    (each level 256-byte aligned after a 256-byte header); FP32 only.  The
    adjoint's float32 gradient pyramid takes the same layout, and the
    reproducible mode adds 4 x uint64 per texel of every volume."""
    al = lambda x: (x + 255) // 256 * 256
    for n in (2, 8, 64, 256):
        L = n.bit_length()
        levels = [(n >> l) ** 3 * (6 if l >= 1 else 1) for l in range(L)]
        total = 256 + sum(al(t * 16) for t in levels)
        assert lib.vct_pyramid_bytes_aniso(n, L, 0) == total
        p = _abi.VctPyramid(n, L, 0, _abi.LAYOUT_ANISO)
        assert lib.vct_trace_backward_workspace_bytes(ctypes.byref(p)) == total
        det = lib.vct_trace_backward_deterministic_workspace_bytes(ctypes.byref(p))
        assert det == al(total) + sum(al(t * 32) for t in levels)
        d = _abi.VctPyramid(n, L, 0, _abi.LAYOUT_DENSE)
        assert lib.vct_trace_backward_workspace_bytes(ctypes.byref(d)) == lib.vct_pyramid_bytes(n, L, 0)
    assert lib.vct_pyramid_bytes_aniso(64, 7, 1) == 0  # FP16 is not offered
    assert lib.vct_pyramid_bytes_aniso(48, 6, 0) == 0  # not a power of two


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the compiled library the binding raises, and a
    failed build raises rather than leaving a stale or empty library."""
    from paper_2104_00618_gb300 import build as _build
    monkeypatch.setattr(_build, "library_file", lambda variant="release": str(tmp_path / "none.so"))
    with pytest.raises(RuntimeError, match="not found"):
        _abi.open_library("release", build_if_missing=False)

    def no_nvcc():
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvct")
    monkeypatch.setattr(_build, "nvcc", no_nvcc)
    with pytest.raises(RuntimeError):
        _build.build(force=True)
