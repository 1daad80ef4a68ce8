"""vct_trace_backward_noalloc: the adjoint for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).  Checked
through the C ABI against vct_trace_backward with a caller-owned workspace,
on two calls in a row (the shared scratch must not carry anything over), at
the largest grids its array accepts (64^3 dense, 32^3 anisotropic), and in
contexts other than the device's primary one (a child process that creates
and destroys driver contexts).

This file is named to be collected last."""
import ctypes
import math
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import paper_2104_00618_gb300 as vct
import vct_synth as vs
from paper_2104_00618_gb300 import _abi

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def _case(n, seed=5, random_grid=False):
    gt = vs.box_scene(n, 5, seed, room=True)
    rng = np.random.default_rng(seed)
    views = [vs.interior_view(gt, 40, 30, rng, with_roughness=True) for _ in range(2)]
    dirs, w = vs.cone_table_ring6()
    prm = vs.trace_params(dirs, w, math.radians(60), spec_enable=True,
                          spec_aperture_min=math.radians(10),
                          spec_aperture_max=math.radians(40), occ_enable=True,
                          occ_aperture=0.55, light=gt["light"])
    if random_grid:
        grid = rng.uniform(0.05, 0.3, (n, n, n, 4)).astype(np.float32)
    else:
        grid = np.full((n, n, n, 4), 0.1, np.float32)
    grads = []
    for v in views:
        npx = v["width"] * v["height"]
        grads.append((rng.standard_normal((npx, 4)).astype(np.float32),
                      rng.standard_normal((npx, 4)).astype(np.float32),
                      rng.standard_normal(npx).astype(np.float32)))
    return grid, views, prm, grads


def _noalloc(P, views, grads, prm):
    lib = vct.lib()
    out = torch.zeros((P.n,) * 3 + (4,), dtype=torch.float32, device="cuda")
    p = P.struct()
    varr = (_abi.VctView * len(views))(*[v.struct() for v in views])
    garr = (_abi.VctViewGrad * len(views))(
        *[_abi.VctViewGrad(g[0].data_ptr(), g[1].data_ptr(), g[2].data_ptr()) for g in grads])
    P_ = vct.make_params(prm)
    st = lib.vct_trace_backward_noalloc(ctypes.byref(p), varr, garr, len(views),
                                        ctypes.byref(P_), None, ctypes.c_void_p(out.data_ptr()),
                                        torch.cuda.current_stream().cuda_stream)
    return st, out


@pytest.mark.parametrize("n,layout", [(32, "dense"), (64, "dense"), (32, "aniso")])
def test_noalloc_adjoint_matches_workspace_adjoint_twice(n, layout):
    grid, hviews, prm, hgrads = _case(n, random_grid=(layout == "aniso"))
    P = vct.build_mips(torch.from_numpy(grid).cuda(), layout=layout)
    if n == 64:  # the largest dense pyramid the array accepts
        assert vct.lib().vct_trace_backward_workspace_bytes(ctypes.byref(P.struct())) > 4 << 20
    views = [vct.View.from_host(v) for v in hviews]
    grads = [tuple(torch.from_numpy(a).cuda() for a in g) for g in hgrads]
    for _ in range(2):
        ref = vct.trace_backward(P, views, grads, prm)  # caller-owned workspace
        st, got = _noalloc(P, views, grads, prm)
        assert st == _abi.VCT_OK, vct.lib().vct_last_error()
        torch.cuda.synchronize()
        scale = ref.abs().max().item()
        assert scale > 0
        # same arithmetic; only the order of the scatter's float atomics differs
        assert (got - ref).abs().max().item() <= 1e-6 * scale


@pytest.mark.parametrize("n,layout,limit", [(128, "dense", b"dense and bricked grids up to 64^3"),
                                            (64, "aniso", b"anisotropic grids up to 32^3")])
def test_noalloc_adjoint_rejects_pyramids_beyond_its_scratch(n, layout, limit):
    grid, hviews, prm, hgrads = _case(n, seed=6)
    P = vct.build_mips(torch.from_numpy(grid).cuda(), layout=layout)
    views = [vct.View.from_host(v) for v in hviews]
    grads = [tuple(torch.from_numpy(a).cuda() for a in g) for g in hgrads]
    st, _ = _noalloc(P, views, grads, prm)
    assert st == _abi.VCT_ERR_WORKSPACE
    msg = vct.lib().vct_last_error()
    need = vct.lib().vct_trace_backward_workspace_bytes(ctypes.byref(P.struct()))
    assert limit in msg and str(need).encode() in msg, msg


def test_noalloc_adjoint_in_created_contexts():
    """A child process calls the entry point in the primary context, in a
    context created with cuCtxCreate, in the primary context again after
    that one is destroyed, and in a second created context; each result
    equals the workspace adjoint's."""
    r = subprocess.run([sys.executable, os.path.join(HERE, "noalloc_context_child.py")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), (r.stdout, r.stderr)
