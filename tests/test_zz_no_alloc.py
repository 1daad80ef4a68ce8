"""vct_trace_backward_noalloc: the adjoint for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).  Checked
through the C ABI against vct_trace_backward with a caller-owned workspace,
on two calls in a row (the shared scratch must not carry anything over).

This file is named to be collected last."""
import ctypes
import math

import numpy as np
import pytest
import torch

import paper_2104_00618_gb300 as vct
import vct_synth as vs
from paper_2104_00618_gb300 import _abi

pytestmark = pytest.mark.gpu


def _case(n, seed=5):
    gt = vs.box_scene(n, 5, seed, room=True)
    rng = np.random.default_rng(seed)
    views = [vs.interior_view(gt, 40, 30, rng, with_roughness=True) for _ in range(2)]
    dirs, w = vs.cone_table_ring6()
    prm = vs.trace_params(dirs, w, math.radians(60), spec_enable=True,
                          spec_aperture_min=math.radians(10),
                          spec_aperture_max=math.radians(40), occ_enable=True,
                          occ_aperture=0.55, light=gt["light"])
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


def test_noalloc_adjoint_matches_workspace_adjoint_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    grid, hviews, prm, hgrads = _case(32)
    P = vct.build_mips(torch.from_numpy(grid).cuda())
    views = [vct.View.from_host(v) for v in hviews]
    grads = [tuple(torch.from_numpy(a).cuda() for a in g) for g in hgrads]
    for _ in range(2):
        ref = vct.trace_backward(P, views, grads, prm)  # caller-owned workspace
        st, got = _noalloc(P, views, grads, prm)
        assert st == _abi.VCT_OK, vct.lib().vct_last_error()
        torch.cuda.synchronize()
        scale = ref.abs().max().item()
        assert scale > 0
        # same arithmetic; only the order of the scatter atomics differs
        assert (got - ref).abs().max().item() <= 1e-4 * scale


def test_noalloc_adjoint_rejects_pyramids_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    grid, hviews, prm, hgrads = _case(128, seed=6)
    P = vct.build_mips(torch.from_numpy(grid).cuda())
    views = [vct.View.from_host(v) for v in hviews]
    grads = [tuple(torch.from_numpy(a).cuda() for a in g) for g in hgrads]
    st, _ = _noalloc(P, views, grads, prm)
    assert st == _abi.VCT_ERR_WORKSPACE
    assert b"64^3" in vct.lib().vct_last_error()
