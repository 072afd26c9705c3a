"""The frame-pair staging of the batched frames kernel: with 8 frames per stage, frames F and
F + 4 of a stage share a region of shared memory and one 3D tensor copy per row class moves
both; a last partial stage goes through the plain layout.  Every frame must keep the bits of
the single-frame path whatever the tile shape (with or without a pair layout), the frame
count (whole stages, a remainder, more than one launch) and the alignment of the batch."""
import numpy as np
import pytest
import torch

from paper_1412_6367_gb300 import synth
from gpu_common import Case, needs_gpu, rel_err, small_workload, to_dev

pytestmark = [pytest.mark.gpu, needs_gpu]


def _frames(c, n, seed0):
    return np.stack([synth.ring_image(c.crad, seed=seed0 + k, dtype=np.uint32) for k in range(n)])


# (8, 224): pair pitch 248; (16, 96): 116; (4, 64): 112; (32, 64) and (4, 232): no pair pitch
@pytest.mark.parametrize("tile", [(8, 224), (16, 96), (4, 64), (32, 64), (4, 232)])
def test_pairs_keep_single_frame_bits(tile):
    w = small_workload(117, 251, split=2, npt=120, seed=61)  # odd frame size
    c = Case(w)
    g = c.gpu_from_oracle_positions()
    g.set_tuning(tile_h=tile[0], tile_w=tile[1], frames_per_pass=8)
    corr = c.corrections_dev()
    fr = _frames(c, 21, 300)
    fd = to_dev(fr)
    singles = [g.integrate(fd[k], *corr, precision="fp32") for k in range(fr.shape[0])]
    for n in (8, 13, 16, 21):
        out = g.integrate_batch(fd[:n].contiguous(), *corr)
        for k in range(n):
            assert torch.equal(out.I[k], singles[k].I), (tile, n, k)
            assert torch.equal(out.sum_signal[k], singles[k].sum_signal), (tile, n, k)
        assert torch.equal(out.sum_norm, singles[0].sum_norm)
        assert torch.equal(out.count, singles[0].count)
    ref = c.oracle(fr[11])
    for name, got, r in zip("ISNC", (out.I[11], out.sum_signal[11], out.sum_norm, out.count), ref):
        per, norm = rel_err(got.double().cpu().numpy(), r)
        assert per <= 1e-5 and norm <= 1e-5, (tile, name, per, norm)
    assert g.status() == 0


@pytest.mark.parametrize("off", [1, 2, 3])
def test_pairs_misaligned_batch_and_two_launches(off):
    """A batch that starts 4 * off bytes past a 16-byte boundary (every frame's word phase
    moves) and is longer than one launch (64 frames, then 5 in a partial stage)."""
    w = small_workload(53, 67, split=2, npt=60, seed=62)
    c = Case(w)
    g = c.gpu_from_oracle_positions()
    g.set_tuning(tile_h=8, tile_w=64, frames_per_pass=8)
    corr = c.corrections_dev()
    n, npix = 69, 53 * 67
    fr = _frames(c, n, 400)
    buf = torch.zeros(n * npix + 4, dtype=torch.int32, device="cuda")
    buf[off:off + n * npix] = torch.from_numpy(fr.reshape(-1).view(np.int32)).cuda()
    fd = buf[off:off + n * npix].view(n, 53, 67).view(torch.uint32)
    out = g.integrate_batch(fd, *corr)
    for k in (0, 3, 4, 7, 8, 31, 63, 64, 68):
        one = g.integrate(fd[k], *corr, precision="fp32")
        assert torch.equal(out.I[k], one.I), (off, k)
        assert torch.equal(out.sum_signal[k], one.sum_signal), (off, k)
    g.set_corrections(*corr)
    bound = g.integrate_batch_bound(fd)
    assert all(torch.equal(x, y) for x, y in zip(bound, out))
    assert g.status() == 0
