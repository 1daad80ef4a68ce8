"""Host-buffer frame pipeline: frames submitted back to back (alternating
scenes and views, so both device slots and every event edge are used) give
exactly the outputs of the direct device-buffer calls."""
import numpy as np
import pytest
import torch

import paper_2104_00618_gb300 as vct
from gpu_cases import room_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vct.lib()


def test_pipeline_frames_equal_direct_calls():
    cases = [room_case(n=64, width=96, height=64, seed=s) for s in (1, 2, 3)]
    prm = cases[0][2]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    pipe = vct.Pipeline(64, 96, 64, prm)
    frames = []
    for i in range(7):
        scene, view, _ = cases[i % 3]
        npx = 96 * 64
        outs = (torch.empty((npx, 4)).pin_memory(), torch.empty((npx, 4)).pin_memory(),
                torch.empty((npx,)).pin_memory())
        inputs = (pin(scene["grid"]), pin(view["position"]), pin(view["normal"]),
                  pin(view["roughness"]), pin(view["mask"]))
        pipe.submit(inputs[0], inputs[1], inputs[2], view["camera"], *outs,
                    roughness=inputs[3], mask=inputs[4])
        frames.append((i % 3, outs, inputs))
    pipe.wait()
    ref = []
    for scene, view, _ in cases:
        P = vct.build_mips(torch.from_numpy(scene["grid"]).cuda())
        v = vct.View.from_host(view)
        vct.trace([P], [v], prm)
        ref.append((v.out_diffuse.cpu(), v.out_specular.cpu(), v.out_visibility.cpu()))
    for k, outs, _ in frames:
        for a, b in zip(outs, ref[k]):
            assert torch.equal(a, b)
    st = pipe.stats(0)
    assert sum(st["samples"]) > 0
    pipe.close()


def test_pipeline_rejects_bad_descriptions():
    _, _, prm = room_case(n=32, width=8, height=8)
    with pytest.raises(vct.VctError):
        vct.Pipeline(48, 8, 8, prm)
    with pytest.raises(vct.VctError):
        vct.Pipeline(32, 8, 8, prm, outputs=0)
    with pytest.raises(vct.VctError):
        vct.Pipeline(32, 8, 8, dict(prm, flags=vct.FLAG_SHADE))
