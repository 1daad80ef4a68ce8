"""Mesh voxelization (Ch. 4.4) on the CUDA path against the oracle: the
owner of every voxel bit for bit, the stored colours within the FP32 bound."""
import numpy as np
import pytest
import torch

import oracle
import paper_2104_00618_gb300 as vct
import vct_synth as vs
from gpu_cases import FP32_BOUND, gpu_trace
from metrics import report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vct.lib()


def gpu_voxelize(mesh_host, n, origin=(0.0, 0.0, 0.0), size=1.0, light=None):
    m = vct.Mesh.from_host(mesh_host)
    ws = vct.voxelize_workspace(n, m.indices.shape[0])
    grid = vct.voxelize(m, n, origin, size, light, workspace=ws)
    torch.cuda.synchronize()
    return grid.cpu().numpy(), vct.voxel_owner(ws, n).cpu().numpy(), vct.read_voxelize_stats(ws)


def check_same(mesh, n, origin=(0.0, 0.0, 0.0), size=1.0, light=None):
    g, o, st = gpu_voxelize(mesh, n, origin, size, light)
    rg, ro, rst = oracle.voxelize(mesh, n, origin, size, light)
    diff = int((o != ro).sum())
    assert diff == 0, f"{diff} voxels with another owner"
    for k in ("fragments", "skipped", "degenerate"):
        assert st[k] == rst[k], (k, st, rst)
    assert np.array_equal(g[..., 3], rg[..., 3])
    err = report(g.reshape(-1, 4)[:, :3], rg.reshape(-1, 4)[:, :3])[0]
    assert err.max() <= FP32_BOUND, err
    return st, err


def random_mesh(rng, n, small=2000, large=12):
    """Small triangles (half of them on the half-voxel lattice, so that edges
    run through pixel centres), triangles crossing the grid boundary, large
    ones taking the warp path, and a few degenerate / out-of-range / badly
    indexed triangles."""
    V, I, C = [], [], []

    def add(tri, col=None):
        I.append([len(V), len(V) + 1, len(V) + 2])
        V.extend(np.asarray(tri, np.float64))
        C.append(rng.uniform(0.1, 1.0, 3) if col is None else col)

    for t in range(small):
        c = rng.uniform(-1.0, n + 1.0, size=3)
        tri = c + rng.uniform(-2.5, 2.5, size=(3, 3))
        if t % 2 == 0:
            tri = np.round(tri * 2.0) / 2.0
        if t % 7 == 3:
            tri[:, t % 3] = np.floor(tri[0, t % 3]) + 0.5
        add(tri / n)
    for _ in range(large):
        add(rng.uniform(-0.2, 1.2, size=(3, 3)))
    add([[0.1, 0.1, 0.1], [0.2, 0.2, 0.2], [0.3, 0.3, 0.3]])       # degenerate
    add([[0.1, 0.1, 0.1], [3e6, 0.2, 0.2], [0.3, 0.5, 0.3]])       # out of range
    mesh = {"vertices": np.asarray(V, np.float32), "indices": np.asarray(I, np.int32),
            "colors": np.asarray(C, np.float32)}
    mesh["indices"] = np.concatenate([mesh["indices"], [[0, 1, len(V) + 5]]]).astype(np.int32)
    mesh["colors"] = np.concatenate([mesh["colors"], [[1, 1, 1]]]).astype(np.float32)
    return mesh


LIGHT = {"light_dir": (0.36, 0.8, -0.48), "light_color": (1.0, 0.9, 0.75), "ambient": 0.05,
         "diffuse_str": 0.9}


@pytest.mark.parametrize("n", [8, 32, 128])
def test_random_mesh_bit_exact(n):
    rng = np.random.default_rng(n)
    mesh = random_mesh(rng, n)
    st, err = check_same(mesh, n, light=LIGHT)
    print(n, st, float(err.max()))
    assert st["skipped"] == 2 and st["degenerate"] >= 1
    assert st["fragments"] > 0 and (n * n <= 64 or st["large_triangles"] > 0)


def test_other_origin_and_size():
    rng = np.random.default_rng(5)
    n = 64
    mesh = random_mesh(rng, n, small=1500, large=6)
    origin, size = np.array([-3.0, 0.5, 2.25], np.float32), 4.0
    mesh["vertices"] = (origin + size * mesh["vertices"].astype(np.float64)).astype(np.float32)
    check_same(mesh, n, origin=origin, size=size, light=LIGHT)


def test_edge_cases():
    n = 16
    empty = {"vertices": np.zeros((0, 3), np.float32), "indices": np.zeros((0, 3), np.int32),
             "colors": np.zeros((0, 3), np.float32)}
    g, o, st = gpu_voxelize(empty, n)
    assert not g.any() and not o.any() and st["fragments"] == 0
    # one triangle covering the whole viewport: many warp items; n = 2 grid
    big = {"vertices": np.array([[-1, -1, 0.3], [3, -1, 0.6], [-1, 3, 0.4]], np.float32),
           "indices": np.array([[0, 1, 2]], np.int32), "colors": np.ones((1, 3), np.float32)}
    for m in (2, 16, 256):
        st, _ = check_same(big, m, light=LIGHT)
        assert st["fragments"] == m * m
    # the same workspace twice: the second call starts from a cleared grid
    rng = np.random.default_rng(1)
    a, b = random_mesh(rng, n, small=300, large=2), random_mesh(rng, n, small=300, large=2)
    ma, mb = vct.Mesh.from_host(a), vct.Mesh.from_host(b)
    ws = vct.voxelize_workspace(n, max(ma.indices.shape[0], mb.indices.shape[0]))
    vct.voxelize(ma, n, workspace=ws)
    gb = vct.voxelize(mb, n, workspace=ws).cpu().numpy()
    rg, ro, _ = oracle.voxelize(b, n)
    assert np.array_equal(vct.voxel_owner(ws, n).cpu().numpy(), ro)
    assert np.array_equal(gb[..., 3], rg[..., 3])


def test_room_mesh_full_size():
    """The 256^3 room as a mesh of about 244K triangles (the revoxelized
    workload): every voxel's owner bit for bit."""
    c = vs.config_room_mesh()
    st, err = check_same(c["mesh"], 256, light=c["light"])
    print("room mesh:", st, float(err.max()))
    assert st["fragments"] > 500_000 and st["degenerate"] > 0


def test_voxelize_then_trace():
    """Voxelize -> mips -> trace on the GPU against the same three steps in
    the oracle."""
    scene, n = vs.box_scene(64, 8, 17, room=True), 64
    mesh = vs.scene_mesh(scene, tess=3, n_spheres=2, sphere_res=(12, 24), seed=4)
    light = {"light_dir": scene["light"]}
    rng = np.random.default_rng(3)
    view = vs.interior_view(scene, 97, 61, rng)
    prm = vs.params_room9(scene["light"])
    g = vct.voxelize(vct.Mesh.from_host(mesh), n, light=light)
    P = vct.build_mips(g)
    (out,), _ = gpu_trace([P], [view], prm)
    rg, _, _ = oracle.voxelize(mesh, n, light=light)
    ref = oracle.trace(oracle.build_mips(rg), view, prm)
    for k, o in zip(("D", "S", "Vis"), out):
        e = report(o, ref[k])[0].max()
        assert e <= FP32_BOUND, (k, e)
