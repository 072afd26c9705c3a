"""Edge cases of the CUDA path against the oracle: degenerate and ragged detector shapes,
single bins and single azimuthal bins, nearly empty masks, more bins than pixels, tiles
larger than the detector, frame counts around the per-launch and per-stage sizes, empty
batches, and a work item cut out of a heavy tile.  Tolerances as in the forward tests."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1412_6367_gb300 import synth
from gpu_common import Case, api, needs_gpu, rel_err, small_workload, to_dev

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def check(res, ref, precision, what, tol=None):
    tol = TOL[precision] if tol is None else tol
    for name, got, r in zip("ISNC", res, ref):
        per, norm = rel_err(got.reshape(-1).cpu().numpy(), r)
        assert per <= tol and norm <= tol, (what, precision, name, per, norm)


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (29, 1), (3, 5), (13, 251), (250, 9)])
@pytest.mark.parametrize("split", [0, 1, 2])
def test_degenerate_shapes(shape, split):
    ny, nx = shape
    if split == 0 and ny * nx == 1:
        pytest.skip("one pixel without splitting spans no range")
    w = small_workload(ny, nx, split=split, npt=7, seed=ny * 131 + nx + split)
    c = Case(w, image=synth.uniform_image(ny, nx, seed=5, lo=1, hi=100, dtype=np.float32))
    gpu = c.gpu_from_oracle_positions()
    for precision in ("fp64", "fp32"):
        res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision=precision)
        check(res, c.oracle(), precision, "shape %s" % (shape,))
    out = gpu.integrate_batch(to_dev(np.stack([c.image] * 3)), *c.corrections_dev())
    check((out.I[2], out.sum_signal[2], out.sum_norm, out.count), c.oracle(), "fp32", "batch")


def test_more_bins_than_pixels():
    w = small_workload(12, 10, split=2, npt=2000, seed=9)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision="fp64")
    check(res, c.oracle(), "fp64", "bins > pixels")
    C = res.count.cpu().numpy()
    assert np.all(res.I.cpu().numpy()[C == 0] == 0.0)


@pytest.mark.parametrize("npt, npt_azim", [(1, 0), (1, 1), (5, 1), (1, 36)])
def test_single_bins(npt, npt_azim):
    w = small_workload(40, 50, split=2, npt=npt, npt_azim=npt_azim, unit=0, seed=npt + npt_azim)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    for precision in ("fp64", "fp32"):
        res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision=precision)
        check(res, c.oracle(), precision, "bins %d x %d" % (npt, npt_azim))


def test_one_unmasked_pixel_and_all_masked():
    ny, nx = 30, 40
    w = small_workload(ny, nx, split=1, npt=5, seed=4)
    mask = np.ones((ny, nx), np.uint8)
    mask[17, 23] = 0
    c = Case(w, mask=mask)
    gpu = c.gpu_from_oracle_positions()
    res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision="fp64")
    check(res, c.oracle(), "fp64", "one pixel")
    from paper_1412_6367_gb300 import _lib as L
    with pytest.raises(L.AzError) as e:
        api().Integrator.from_positions((ny, nx), c.dev(c.rad), c.dev(c.chi), 5, 0, "bbox",
                                        np.ones((ny, nx), np.uint8))
    assert e.value.code == -8  # AZ_ERANGE: nothing unmasked


@pytest.mark.parametrize("nf", [0, 1, 2, 7, 8, 9, 63, 64, 65, 130])
def test_batch_frame_counts(nf):
    w = small_workload(45, 67, split=2, npt=40, seed=8)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    corr = c.corrections_dev()
    imgs = [synth.ring_image(c.crad, seed=s, dtype=np.uint32) for s in range(5)]
    frames = np.stack([imgs[k % 5] for k in range(nf)]) if nf else np.zeros((0, 45, 67), np.uint32)
    out = gpu.integrate_batch(to_dev(frames), *corr)
    assert out.I.shape == (nf, gpu.nrows)
    for k in sorted({0, nf // 2, nf - 1}) if nf else []:
        one = gpu.integrate(to_dev(frames[k]), *corr, precision="fp32")
        assert torch.equal(out.I[k], one.I) and torch.equal(out.sum_signal[k], one.sum_signal)
    if nf:
        check((out.I[nf - 1], out.sum_signal[nf - 1], out.sum_norm, out.count),
              c.oracle(frames[nf - 1]), "fp32", "frames %d" % nf)


def test_tile_larger_than_detector():
    w = small_workload(11, 13, split=2, npt=9, seed=21)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    gpu.set_tuning(16, 128, 0, 8)
    res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision="fp32")
    check(res, c.oracle(), "fp32", "big tile")


def test_heavy_tile_is_cut_into_items():
    """2D around the beam centre: the pixels at the centre reach every azimuthal bin, so the
    tile holding them has far more entries than the others; the layout cuts it into several
    work items at segment boundaries.  Results must not change."""
    p = synth.GeometryParams(dist=0.005, poni1=64 * 100e-6, poni2=64 * 100e-6, pixel1=100e-6,
                             pixel2=100e-6)
    w = synth.Workload("centre", 128, 128, p, synth.UNIT_2TH_DEG, synth.SPLIT_FULL, 300, 720,
                       corrections=True)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    ref = c.oracle()
    for tile in ((32, 64), (8, 64)):
        gpu.set_tuning(tile[0], tile[1], 0, 8)
        if tile == (32, 64):
            assert gpu.info["n_items"] > gpu.info["n_tiles"]  # the centre tile was cut
        # FP64 bar of 2D full split with small cell fragments, as for the cake workload
        for precision, tol in (("fp32", 1e-5), ("fp64", 1e-10)):
            res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision=precision)
            check(res, ref, precision, "tile %s" % (tile,), tol)
        out = gpu.integrate_batch(to_dev(np.stack([c.image] * 9)), *c.corrections_dev())
        check((out.I[8], out.sum_signal[8], out.sum_norm, out.count), ref, "fp32", "batch")
