"""Camera G-buffer (the geometry pass before cone tracing, Ch. 5.4) on the
CUDA path against the oracle: the triangle seen by every pixel bit for bit,
positions and normals within float32 rounding, colours exactly."""
import numpy as np
import pytest
import torch

import oracle
import oracle_pins as pins
import paper_2104_00618_gb300 as vct
import vct_synth as vs
from gpu_cases import FP32_BOUND, gpu_trace
from metrics import report

pytestmark = pytest.mark.gpu

POS_TOL = 4e-6  # frame sizes: float32 t, t * D, / s and + origin
NRM_TOL = 1e-5  # unit normals from float32 edges and a fused cross product


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vct.lib()


def run_gpu(mesh_host, cam, pair_capacity=None, verify=True):
    m = vct.Mesh.from_host(mesh_host)
    ws = None
    if pair_capacity is not None:
        ws = vct.gbuffer_workspace(cam["width"], cam["height"], m.indices.shape[0], pair_capacity)
    g = vct.gbuffer(m, cam, workspace=ws, verify=verify)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in g.items() if k != "workspace"}
    out["stats"] = vct.read_gbuffer_stats(g["workspace"])
    return out


def check_same(mesh, cam, pixels=None, g=None):
    """GPU G-buffer against the oracle on all pixels (or the listed ones)."""
    g = g or run_gpu(mesh, cam)
    ref = oracle.gbuffer(mesh, cam, pixels=pixels)
    sel = slice(None) if pixels is None else np.asarray(pixels)
    tri = g["triangle"][sel]
    diff = int((tri != ref["tri"]).sum())
    assert diff == 0, f"{diff} pixels see another triangle"
    assert np.array_equal(g["mask"][sel], ref["mask"])
    hit = ref["mask"].astype(bool)
    size = float(cam["frame_size"])
    if hit.any():
        ep = np.abs(g["position"][sel][hit] - ref["position"][hit]).max() / size
        en = np.abs(g["normal"][sel][hit] - ref["normal"][hit]).max()
        assert ep <= POS_TOL and en <= NRM_TOL, (ep, en)
    assert np.array_equal(g["albedo"][sel], ref["albedo"].astype(np.float32))
    for k in ("position", "normal"):
        assert not g[k][sel][~hit].any(), k
    if pixels is None:
        assert (g["stats"]["skipped"], g["stats"]["degenerate"]) == (ref["skipped"],
                                                                    ref["degenerate"])
    return g, ref


def look(eye, target, W, H, fov=60.0, origin=(0.0, 0.0, 0.0), size=1.0):
    return vs.camera(np.asarray(eye, np.float64), np.asarray(target, np.float64), W, H, fov,
                     origin, size)


def soup(rng, count, big=20):
    """Overlapping random triangles around the unit cube: small and large,
    some crossing the eye's plane or lying behind it, a few coincident ones
    (exact depth ties), degenerate and out-of-frame ones."""
    V, I, C = [], [], []

    def add(tri):
        I.append([len(V), len(V) + 1, len(V) + 2])
        V.extend(np.asarray(tri, np.float64))
        C.append(rng.uniform(0.05, 1.0, 3))

    for _ in range(count):
        c = rng.uniform(-0.2, 1.2, 3)
        add(c + rng.normal(0.0, rng.choice([0.01, 0.05, 0.2]), (3, 3)))
    for _ in range(big):
        add(rng.uniform(-1.5, 1.9, (3, 3)))
    add(V[-3:])                                              # coincident with the last one
    add([[0.2, 0.2, 0.2], [0.4, 0.4, 0.4], [0.6, 0.6, 0.6]])  # degenerate
    add([[0.2, 0.2, 0.2], [2.5, 0.4, 0.4], [0.6, 0.9, 0.6]])  # beyond the frame
    return {"vertices": np.asarray(V, np.float32), "indices": np.asarray(I, np.int32),
            "colors": np.asarray(C, np.float32)}


def test_pin_scenes_bit_exact():
    """The oracle's pin scenes (closed-form plane, depth order, coincident
    triangles, the shared-edge diamond) on the CUDA path."""
    cam = pins._gb_camera((0.5, 0.5, 0.1), (0, 0, 1), (-1, 0, 0), (0, 1, 0), 25, 15)
    A, B = (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)
    near, far, behind = pins._plane_quad(0.5), pins._plane_quad(0.8), pins._plane_quad(-0.3)
    for quads in ([far, near], [near, far], [near, near], [behind, far], [behind]):
        check_same(pins._gb_mesh(quads, [A, B][:len(quads)]), cam)
    top, right, bot, left = (0.5, 0.9, 0.7), (0.8, 0.5, 0.7), (0.5, 0.1, 0.7), (0.2, 0.5, 0.7)
    for tris in ([[top, right, bot], [top, bot, left]], [[top, bot, left], [top, right, bot]]):
        mesh = {"vertices": np.asarray(tris, np.float32).reshape(-1, 3),
                "indices": np.arange(6, dtype=np.int32).reshape(2, 3),
                "colors": np.asarray([A, B], np.float32)}
        g, _ = check_same(mesh, cam)
        assert np.all(g["triangle"][np.arange(15) * 25 + 12] == 0)
    for origin, size, flip in (((0, 0, 0), 1.0, False), ((-0.5, 0.25, -1.0), 4.0, True)):
        cam = pins._gb_camera((0.5, 0.5, 0.1), (0, 0, 1), (-1, 0, 0), (0, 1, 0), 24, 16,
                              origin, size)
        check_same(pins._gb_mesh([pins._plane_quad(0.7, flip=flip)], [A]), cam)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_triangle_soup_bit_exact(seed):
    """Random soups seen from random eyes, ragged image sizes (partial tiles)."""
    rng = np.random.default_rng(seed)
    mesh = soup(rng, 3000)
    sizes = [(97, 61), (16, 16), (130, 33)]
    for k in range(3):
        eye = rng.uniform(0.2, 0.8, 3)
        target = eye + rng.normal(size=3)
        W, H = sizes[k]
        g, ref = check_same(mesh, look(eye, target, W, H, fov=rng.uniform(30, 60)))
        st = g["stats"]
        print(seed, k, st, int(ref["mask"].sum()))
        assert st["overflow"] == 0 and ref["mask"].any()


def test_room_mesh_boxes_and_slab_raycaster():
    """Box scene as exact box faces, interior views: the GPU mask and face
    normals equal the slab raycaster's (independent double-precision
    intersection) except at pixels grazing a box edge."""
    scene = vs.box_scene(64, 12, 9, room=True)
    mesh = vs.box_mesh(scene, tess=4)
    rng = np.random.default_rng(5)
    for _ in range(3):
        eye = vs.interior_camera(rng, scene["boxes"], 64)
        target = vs.interior_camera(rng, scene["boxes"], 64)
        cam = vs.camera(eye, target, 160, 90)
        g, _ = check_same(mesh, cam)
        pos, nrm, mask = vs.raycast_gbuffer(scene, 160, 90, eye, target)
        assert np.array_equal(g["mask"], mask)
        same = np.all(g["normal"] == nrm.reshape(-1, 3), axis=1)
        assert same.mean() > 0.99, same.mean()


def test_room_mesh_full_size_sampled():
    """The 244K-triangle room at 1920x1080 (the revoxelized bench scene):
    every pixel hits (closed room, eye inside), the sampled pixels equal the
    oracle's, and the pair count stays within the default workspace."""
    c = vs.config_room_mesh()
    v = c["views"][0]
    cam = vs.camera(v["camera"], v["target"], 1920, 1080)
    g = run_gpu(c["mesh"], cam)
    st = g["stats"]
    print("room 1080p:", st)
    assert st["overflow"] == 0 and g["mask"].all()
    rng = np.random.default_rng(1)
    pixels = np.unique(np.concatenate([rng.integers(0, 1920 * 1080, 1500),
                                       np.arange(0, 1920 * 1080, 1920 * 1080 // 97)]))
    check_same(c["mesh"], cam, pixels=pixels, g=g)


def test_overflow_and_edge_cases():
    rng = np.random.default_rng(4)
    mesh = soup(rng, 500, big=5)
    cam = look((0.5, 0.5, -0.3), (0.5, 0.5, 1.0), 64, 48)
    # pairs beyond the workspace: every pixel empty, the needed count reported
    g = run_gpu(mesh, cam, pair_capacity=10, verify=False)
    assert g["stats"]["overflow"] == 1 and g["stats"]["pairs"] > 10
    assert not g["mask"].any() and np.all(g["triangle"] == -1)
    # the binding grows the workspace and redoes the call
    g = run_gpu(mesh, cam, pair_capacity=10, verify=True)
    assert g["stats"]["overflow"] == 0
    check_same(mesh, cam, g=g)
    # no triangles; one pixel; a one-row image
    empty = {"vertices": np.zeros((0, 3), np.float32), "indices": np.zeros((0, 3), np.int32),
             "colors": np.zeros((0, 3), np.float32)}
    g = run_gpu(empty, cam)
    assert not g["mask"].any() and np.all(g["triangle"] == -1)
    for W, H, fov in ((1, 1, 60.0), (300, 1, 1.0), (1, 77, 60.0)):
        check_same(mesh, look((0.5, 0.5, -0.3), (0.5, 0.5, 1.0), W, H, fov=fov))


def test_eye_close_to_triangles():
    """Triangles passing within a few fixed-point units of the eye (binned to
    every tile) and ones crossing the eye's plane."""
    eye = np.array([0.5, 0.5, 0.5])
    V = [[0.5 - 1e-5, 0.3, 0.2], [0.5 + 1e-5, 0.3, 0.9], [0.5, 0.8, 0.6],   # near the eye
         [0.1, 0.45, 0.3], [0.9, 0.45, 0.3], [0.5, 0.45, 0.9],             # below, crossing
         [0.0, 0.0, 0.95], [1.0, 0.0, 0.95], [0.5, 1.0, 0.95]]
    mesh = {"vertices": np.asarray(V, np.float32),
            "indices": np.arange(9, dtype=np.int32).reshape(3, 3),
            "colors": np.eye(3, dtype=np.float32)}
    for target in ((0.5, 0.5, 1.0), (0.52, 0.3, 1.0), (0.5, 0.5, 0.0), (1.0, 0.5, 0.5)):
        g, _ = check_same(mesh, look(eye, target, 81, 47, fov=80.0))
        print(target, g["stats"])


def test_gbuffer_then_trace():
    """Mesh -> voxelize -> mips -> G-buffer -> trace on the GPU against the
    same chain in the oracle."""
    scene, n = vs.box_scene(64, 8, 17, room=True), 64
    mesh = vs.scene_mesh(scene, tess=3, n_spheres=2, sphere_res=(12, 24), seed=4)
    light = {"light_dir": scene["light"]}
    rng = np.random.default_rng(3)
    eye = vs.interior_camera(rng, scene["boxes"], n)
    target = vs.interior_camera(rng, scene["boxes"], n)
    cam = vs.camera(eye, target, 97, 61)
    prm = vs.params_room9(scene["light"])
    m = vct.Mesh.from_host(mesh)
    P = vct.build_mips(vct.voxelize(m, n, light=light))
    g = vct.gbuffer(m, cam)
    view = vct.gbuffer_view(g, cam)
    vct.trace([P], [view], prm)
    out = [t.cpu().numpy() for t in (view.out_diffuse, view.out_specular, view.out_visibility)]
    rg, _, _ = oracle.voxelize(mesh, n, light=light)
    rb = oracle.gbuffer(mesh, cam)
    host = vs.view_dict(rb["position"].astype(np.float32).ravel(),
                        rb["normal"].astype(np.float32).ravel(), rb["mask"], 97, 61,
                        cam["eye"])
    ref = oracle.trace(oracle.build_mips(rg), host, prm)
    assert np.array_equal(g["mask"].cpu().numpy(), rb["mask"])
    for k, o in zip(("D", "S", "Vis"), out):
        e = report(o, ref[k])[0].max()
        assert e <= FP32_BOUND, (k, e)
    # the GPU's own G-buffer traced again through the host path gives the same
    (again,), _ = gpu_trace([P], [dict(host, position=g["position"].cpu().numpy().ravel(),
                                        normal=g["normal"].cpu().numpy().ravel(),
                                        mask=g["mask"].cpu().numpy())], prm)
    for a, b in zip(again, out):
        assert np.array_equal(a, b)
