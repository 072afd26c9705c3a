"""GPU parity of the propagated variance V = sum w^2 max(img, 0) (az_integrate_variance)
against the oracle: FP32 compensated within 1e-5 relative (bins above 1e-3 of the largest)
and normwise; one frame gives the bits of the same frame in a batch."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1412_6367_gb300 import synth
from gpu_common import Case, needs_gpu, rel_err, small_workload, to_dev

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.mark.parametrize("split", [0, 1, 2])
@pytest.mark.parametrize("npt_azim", [0, 24])
@pytest.mark.parametrize("dtype", ["uint32", "float32"])
def test_variance_matches_oracle(split, npt_azim, dtype):
    w = small_workload(77, 93, split=split, npt=60, npt_azim=npt_azim, unit=0,
                       seed=3 * split + npt_azim + len(dtype))
    c = Case(w, with_corrections=False)
    gpu = c.gpu_from_oracle_positions()
    if dtype == "uint32":
        frames = np.stack([synth.uniform_image(77, 93, seed=s, lo=0, hi=5000, dtype=np.uint32)
                           for s in range(11)])
    else:  # some negative values: clipped at 0
        frames = np.stack([synth.uniform_image(77, 93, seed=s, lo=-500, hi=5000) for s in range(11)])
    V = gpu.variance(to_dev(frames))
    for k in (0, 5, 10):
        per, norm = rel_err(V[k].cpu().numpy(), O.variance(c.A, frames[k]))
        assert per <= 1e-5 and norm <= 1e-5, (k, per, norm)
        one = gpu.variance(to_dev(frames[k]))
        assert torch.equal(one, V[k])


def test_variance_pilatus_full_size():
    w = synth.pilatus_workload()
    c = Case(w, with_corrections=False)
    gpu = c.gpu_from_geometry()
    frames = np.stack([synth.ring_image(c.crad, seed=s, dtype=np.uint32) for s in range(3)])
    V = gpu.variance(to_dev(frames))
    for k in range(3):
        per, norm = rel_err(V[k].cpu().numpy(), O.variance(c.A, frames[k]))
        assert per <= 1e-5 and norm <= 1e-5, (k, per, norm)
