"""The bounds-checked build (-DVCT_DEBUG_BOUNDS, libvct_debug_bounds.so) on
small cases: grids of 2 .. 32 voxels per axis with hand-placed single
voxels, 1 .. 4 pixels on the domain's edges, every entry point and layout
(dense, bricks, anisotropic).
No index may leave its array (flag word 0), and the outputs must equal the
release library's (the checks change no arithmetic).  The probe checks that
a planted out-of-range index is caught and its write skipped."""
import numpy as np
import pytest
import torch

import paper_2104_00618_gb300 as vct
import vct_synth as vs

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16, 1), (8, 8, 2), (4, 8, 4), (8, 4, 8)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vct.lib()


def flags(lib, reset=True):
    import ctypes
    out = ctypes.c_uint32(0)
    assert lib.vct_debug_bounds_flags(ctypes.byref(out), 1 if reset else 0) == vct._abi.VCT_OK
    return out.value


def single_voxel_grid(n, spots, seed):
    rng = np.random.default_rng(seed)
    g = np.zeros((n, n, n, 4), np.float32)
    for (x, y, z) in spots:
        g[z, y, x] = (*rng.uniform(0.2, 1.0, 3), 1.0)
    return g


def edge_view(n, count, seed):
    """Pixels on the faces and corners of the grid (border-zero lookups),
    normals pointing inwards, roughness over its range."""
    rng = np.random.default_rng(seed)
    eps = 1e-4
    pts = [((0.5 + eps) / n, 0.5, 0.5, 1, 0, 0), (1 - (0.5 + eps) / n, 0.5, 0.5, -1, 0, 0),
           (eps, eps, eps, 0, 1, 0), (0.5, 1 - eps, 0.5, 0, -1, 0)][:count]
    pos = np.array([p[:3] for p in pts], np.float32).ravel()
    nrm = np.array([p[3:] for p in pts], np.float32).ravel()
    view = vs.view_dict(pos, nrm, np.ones(count, np.uint8), count, 1, (0.5, 0.5, 2.0),
                        roughness=rng.uniform(0.05, 1.0, count).astype(np.float32))
    return view


def small_cases():
    cases = []
    for n, spots in ((2, [(0, 0, 0)]), (4, [(3, 3, 3), (0, 2, 1)]), (8, [(0, 0, 0), (7, 7, 7)]),
                     (16, [(15, 0, 8)]), (32, [(0, 31, 31), (16, 16, 16)])):
        cases.append((n, single_voxel_grid(n, spots, n)))
    return cases


def run_everything():
    """Every entry point on the small cases; returns host arrays by name."""
    out = {}
    prm = vs.params_room9((0.36, 0.8, -0.48))
    prm["t_max"] = 1.0
    for n, grid in small_cases():
        level0 = torch.from_numpy(grid).cuda()
        for dtype in ("f32", "f16"):
            for layout in ("dense", "bricks"):
                P = vct.build_mips(level0, dtype=dtype, layout=layout)
                for l in range(P.levels):
                    out[f"lvl{n}{dtype}{layout}{l}"] = vct.read_level(P, l).cpu().numpy()
                for count in (1, 4):
                    view = edge_view(n, count, n + count)
                    for shape in SHAPES:
                        v = vct.View.from_host(view)
                        vct.trace([P], [v], prm, cfg=vct.launch_config(*shape))
                        key = f"tr{n}{dtype}{layout}{count}{shape}"
                        out[key + "D"] = v.out_diffuse.cpu().numpy()
                        out[key + "S"] = v.out_specular.cpu().numpy()
                        out[key + "V"] = v.out_visibility.cpu().numpy()
                    if dtype == "f32" and layout == "dense":
                        v = vct.View.from_host(view)
                        vct.trace([P], [v], prm)
                        gl = vct.trace_backward(P, [v], [(torch.ones_like(v.out_diffuse),
                                                          torch.ones_like(v.out_specular),
                                                          torch.ones_like(v.out_visibility))], prm)
                        out[f"bw{n}{count}"] = gl.cpu().numpy()
        # anisotropic mips: every directional volume, traces under all shapes
        P = vct.build_mips(level0, layout="aniso")
        out[f"an{n}lvl0"] = vct.read_level(P, 0).cpu().numpy()
        for l in range(1, P.levels):
            for d in range(6):
                out[f"an{n}lvl{l}d{d}"] = vct.read_volume(P, l, d).cpu().numpy()
        for count in (1, 4):
            view = edge_view(n, count, n + count)
            for shape in SHAPES:
                v = vct.View.from_host(view)
                vct.trace([P], [v], prm, cfg=vct.launch_config(*shape))
                key = f"an{n}{count}{shape}"
                out[key + "D"] = v.out_diffuse.cpu().numpy()
                out[key + "S"] = v.out_specular.cpu().numpy()
                out[key + "V"] = v.out_visibility.cpu().numpy()
            v = vct.View.from_host(view)
            vct.trace([P], [v], prm)
            gl = vct.trace_backward(P, [v], [(torch.ones_like(v.out_diffuse),
                                              torch.ones_like(v.out_specular),
                                              torch.ones_like(v.out_visibility))], prm)
            out[f"bwan{n}{count}"] = gl.cpu().numpy()
    # voxelizer and G-buffer on a few triangles, one crossing the grid border
    mesh = {"vertices": np.array([[-0.2, 0.1, 0.5], [1.2, 0.3, 0.55], [0.4, 1.1, 0.45],
                                  [0.1, 0.1, 0.9], [0.9, 0.1, 0.9], [0.5, 0.9, 0.9]], np.float32),
            "indices": np.array([[0, 1, 2], [3, 4, 5]], np.int32),
            "colors": np.array([[1, 0, 0], [0, 1, 0]], np.float32)}
    m = vct.Mesh.from_host(mesh)
    for n in (2, 8):
        out[f"vox{n}"] = vct.voxelize(m, n, light={"light_dir": (0.0, 0.0, -1.0)}).cpu().numpy()
    for W, H in ((1, 1), (4, 3), (33, 17)):
        cam = vs.camera((0.5, 0.5, 0.1), (0.5, 0.5, 1.0), W, H)
        g = vct.gbuffer(m, cam)
        for k in ("position", "normal", "albedo", "mask", "triangle"):
            out[f"gb{W}x{H}{k}"] = g[k].cpu().numpy()
    torch.cuda.synchronize()
    return out


def test_small_cases_in_bounds_and_identical():
    with vct._abi.using_variant("debug_bounds") as lib:
        flags(lib)
        dbg = run_everything()
        f = flags(lib)
    assert f == 0, f"bounds check tripped: flags 0x{f:x}"
    rel = run_everything()
    assert dbg.keys() == rel.keys()
    for k in rel:
        if k.startswith("bw"):  # float atomics: summation order differs between runs
            np.testing.assert_allclose(dbg[k], rel[k], rtol=1e-5, atol=1e-7 * np.abs(rel[k]).max(),
                                       err_msg=k)
        else:
            assert np.array_equal(dbg[k], rel[k]), k


def test_probe_is_caught():
    import ctypes
    declared, extra = 1000, 37
    with vct._abi.using_variant("debug_bounds") as lib:
        flags(lib)
        buf = torch.full((declared + extra,), -1, dtype=torch.int32, device="cuda")
        st = lib.vct_debug_bounds_probe(ctypes.c_void_p(buf.data_ptr()), declared, extra,
                                        torch.cuda.current_stream().cuda_stream)
        assert st == vct._abi.VCT_OK
        f = flags(lib)
        assert f == 64, f"flags 0x{f:x}"
        b = buf.cpu().numpy()
        assert np.array_equal(b[:declared], np.arange(declared)) and np.all(b[declared:] == -1)
        assert flags(lib) == 0  # cleared by the previous read
    rel = vct.lib()
    assert rel.vct_debug_bounds_probe(ctypes.c_void_p(buf.data_ptr()), declared, extra,
                                      None) == vct._abi.VCT_ERR_UNSUPPORTED
    out = ctypes.c_uint32(7)
    assert rel.vct_debug_bounds_flags(ctypes.byref(out), 0) == vct._abi.VCT_ERR_UNSUPPORTED
    assert out.value == 0
