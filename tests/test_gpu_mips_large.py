"""Mip build of a 512^3 float32 grid (Ch. 4.3.3), the size where the dense
streaming build takes several patches along x and hands its level 4 to the
level-group kernel: every level must equal, bit for bit, the one the TMA
pack kernel builds for the brick layout (every brick of a random grid is
occupied), and sampled texels of every level must equal the FP64 mean of
their 2^l cube of level-0 voxels (the definition of the box-filter pyramid),
computed on the host texel by texel; the top level is the mean of the grid.
"""
import numpy as np
import pytest
import torch

import paper_2104_00618_gb300 as vct

pytestmark = pytest.mark.gpu

N = 512


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vct.lib()
    yield
    torch.cuda.empty_cache()


def test_mips_512_streamed_equal_tma_and_sampled_means():
    rng = np.random.default_rng(512)
    g = rng.random((N, N, N, 4), dtype=np.float32)
    level0 = torch.from_numpy(g).cuda()
    dense = vct.build_mips(level0)
    bricks = vct.build_mips(level0, layout="bricks")
    vct.pyramid_status(bricks)
    assert dense.levels == 10
    for l in range(dense.levels):
        a = vct.read_level(dense, l)
        b = vct.read_level(bricks, l)
        assert torch.equal(a, b), l
        del b
        if 1 <= l <= 6:
            m = N >> l
            s = 1 << l
            got = a.cpu().numpy()
            for x, y, z in rng.integers(0, m, size=(48, 3)):
                cube = g[z * s:(z + 1) * s, y * s:(y + 1) * s, x * s:(x + 1) * s]
                want = cube.reshape(-1, 4).astype(np.float64).mean(0)
                assert np.allclose(got[z, y, x], want, rtol=2e-6, atol=0), (l, x, y, z)
        del a
    top = vct.read_level(dense, dense.levels - 1).cpu().numpy().reshape(4)
    mean = np.zeros(4)
    for z0 in range(0, N, 64):
        mean += g[z0:z0 + 64].reshape(-1, 4).astype(np.float64).sum(0)
    mean /= N ** 3
    assert np.allclose(top, mean, rtol=1e-5, atol=0), (top, mean)
