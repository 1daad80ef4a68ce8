"""Child process of tests/test_zz_no_alloc.py (not collected by pytest).

Calls vct_trace_backward_noalloc in three CUDA contexts one after another:
the device's primary context, then a context created with the driver API
(cuCtxCreate) and made current, then the primary context again after the
created one is destroyed, and once more in a second created context.  In
each, the result must equal vct_trace_backward with a caller-owned
workspace.  The scratch array's device address differs from context to
context, so an address kept from an earlier context would be wrong there.

Only the driver API and libvct are used (no PyTorch CUDA state): buffers
come from cuMemAlloc in the current context.  Prints "OK" on success."""
import ctypes
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import vct_synth as vs  # noqa: E402
from paper_2104_00618_gb300 import _abi  # noqa: E402
from paper_2104_00618_gb300 import make_params  # noqa: E402

cu = ctypes.CDLL("libcuda.so.1")
_u64 = ctypes.c_uint64


def ck(r, what):
    if r != 0:
        raise RuntimeError(f"{what} failed: CUresult {r}")


class Ctx:
    """Buffers of one context (device pointers from cuMemAlloc)."""

    def __init__(self):
        self.bufs = []

    def alloc(self, nbytes):
        p = _u64(0)
        ck(cu.cuMemAlloc_v2(ctypes.byref(p), ctypes.c_size_t(max(int(nbytes), 256))),
           "cuMemAlloc")
        self.bufs.append(p.value)
        return p.value

    def upload(self, a):
        a = np.ascontiguousarray(a)
        p = self.alloc(a.nbytes)
        ck(cu.cuMemcpyHtoD_v2(_u64(p), a.ctypes.data_as(ctypes.c_void_p),
                              ctypes.c_size_t(a.nbytes)), "cuMemcpyHtoD")
        return p

    def zeros(self, nbytes):
        p = self.alloc(nbytes)
        ck(cu.cuMemsetD8_v2(_u64(p), ctypes.c_ubyte(0), ctypes.c_size_t(nbytes)), "cuMemsetD8")
        return p

    def download(self, p, shape, dtype):
        out = np.empty(shape, dtype)
        ck(cu.cuMemcpyDtoH_v2(out.ctypes.data_as(ctypes.c_void_p), _u64(p),
                              ctypes.c_size_t(out.nbytes)), "cuMemcpyDtoH")
        return out

    def free(self):
        for p in self.bufs:
            cu.cuMemFree_v2(_u64(p))
        self.bufs = []


def case():
    n = 16
    scene = vs.box_scene(n, 3, 9, room=True)
    rng = np.random.default_rng(9)
    view = vs.interior_view(scene, 24, 16, rng)
    dirs, w = vs.cone_table_ring6()
    prm = vs.trace_params(dirs, w, math.radians(60), spec_enable=True,
                          spec_aperture_min=math.radians(10),
                          spec_aperture_max=math.radians(40), occ_enable=True,
                          occ_aperture=0.55, light=scene["light"])
    grid = (0.1 + 0.8 * rng.random((n, n, n, 4))).astype(np.float32)
    npx = view["width"] * view["height"]
    g = (rng.standard_normal((npx, 4)).astype(np.float32),
         rng.standard_normal((npx, 4)).astype(np.float32),
         rng.standard_normal(npx).astype(np.float32))
    return n, grid, view, prm, g


def run_in_current_context(lib, n, grid, view, prm, g):
    """Both adjoints in the current context; returns (noalloc, workspace)."""
    c = Ctx()
    try:
        levels = n.bit_length()
        nbytes = lib.vct_pyramid_bytes(n, levels, _abi.VCT_F32)
        P = _abi.VctPyramid(n, levels, _abi.VCT_F32, _abi.LAYOUT_DENSE, (0.0, 0.0, 0.0), 1.0,
                            c.alloc(nbytes), nbytes)
        lvl0 = c.upload(grid)
        ck(lib.vct_build_mips(ctypes.c_void_p(lvl0), ctypes.byref(P), None), "vct_build_mips")
        npx = view["width"] * view["height"]
        V = _abi.VctView()
        V.width, V.height = view["width"], view["height"]
        V.position = c.upload(view["position"])
        V.normal = c.upload(view["normal"])
        V.roughness = c.upload(view["roughness"])
        V.mask = c.upload(view["mask"])
        for a in range(3):
            V.camera[a] = float(view["camera"][a])
        G = _abi.VctViewGrad(c.upload(g[0]), c.upload(g[1]), c.upload(g[2]))
        params = make_params(prm)
        out_ws = c.zeros(n ** 3 * 16)
        out_na = c.zeros(n ** 3 * 16)
        wsb = lib.vct_trace_backward_workspace_bytes(ctypes.byref(P))
        ws = c.alloc(wsb)
        st = lib.vct_trace_backward(ctypes.byref(P), ctypes.byref(V), ctypes.byref(G), 1,
                                    ctypes.byref(params), None, ctypes.c_void_p(out_ws),
                                    ctypes.c_void_p(ws), ctypes.c_size_t(wsb), None)
        ck(st, f"vct_trace_backward ({lib.vct_last_error()})")
        st = lib.vct_trace_backward_noalloc(ctypes.byref(P), ctypes.byref(V), ctypes.byref(G),
                                            1, ctypes.byref(params), None,
                                            ctypes.c_void_p(out_na), None)
        ck(st, f"vct_trace_backward_noalloc ({lib.vct_last_error()})")
        ck(cu.cuCtxSynchronize(), "cuCtxSynchronize")
        a = c.download(out_na, (n, n, n, 4), np.float32)
        b = c.download(out_ws, (n, n, n, 4), np.float32)
        del npx
        return a, b
    finally:
        c.free()


def main():
    lib = _abi.load()
    ck(cu.cuInit(0), "cuInit")
    dev = ctypes.c_int(0)
    ck(cu.cuDeviceGet(ctypes.byref(dev), 0), "cuDeviceGet")
    primary = ctypes.c_void_p(0)
    ck(cu.cuDevicePrimaryCtxRetain(ctypes.byref(primary), dev), "cuDevicePrimaryCtxRetain")
    ck(cu.cuCtxSetCurrent(primary), "cuCtxSetCurrent")
    n, grid, view, prm, g = case()
    results = []
    results.append(("primary", run_in_current_context(lib, n, grid, view, prm, g)))
    for name in ("created-1", "primary-again", "created-2"):
        if name.startswith("created"):
            ctx = ctypes.c_void_p(0)
            ck(cu.cuCtxCreate_v2(ctypes.byref(ctx), 0, dev), "cuCtxCreate")
            results.append((name, run_in_current_context(lib, n, grid, view, prm, g)))
            ck(cu.cuCtxDestroy_v2(ctx), "cuCtxDestroy")
            ck(cu.cuCtxSetCurrent(primary), "cuCtxSetCurrent")
        else:
            results.append((name, run_in_current_context(lib, n, grid, view, prm, g)))
    ref = results[0][1][1]
    scale = float(np.abs(ref).max())
    assert scale > 0
    for name, (na, ws) in results:
        err = float(np.abs(na.astype(np.float64) - ws).max())
        assert err <= 1e-6 * scale, (name, err / scale)
        assert float(np.abs(ws.astype(np.float64) - ref).max()) <= 1e-6 * scale, name
    cu.cuDevicePrimaryCtxRelease_v2(dev)
    print("OK")


if __name__ == "__main__":
    main()
