"""The look-up-table layout (Sec. 5.2) on the GPU against the oracle's table.

- the table: built from the oracle's positions, its pixel indices and width are bit-exact
  with the oracle's table of the oracle's matrix; its FP64 coefficients are the GPU matrix's
  weights placed bit for bit (and within the weight tolerance of the matrix tests of the
  oracle's), its FP32 coefficients their rounding to float;
- the forward through it: FP64 within 1e-12 and FP32 compensated within 1e-5 of the oracle's
  forward through its table (per output, normwise), 1D and 2D, every image dtype, with and
  without corrections, more bins than pixels (empty rows), masks, and at the full Pilatus 6M
  and cake sizes; bit-identical across runs;
- az_set_layout routes az_integrate1d/2d through it; az_autotune picks a layout and the
  results stay within the bars.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1412_6367_gb300 import synth
from gpu_common import Case, needs_gpu, rel_err, small_workload, random_mask, to_dev

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def oracle_lut_forward(c, image=None):
    idx, coef = O.lut_from_csr(c.A)
    img = c.image if image is None else image
    return O.integrate_lut(idx, coef, img, c.dark, c.flat, c.sa, c.pol)


def check(res, ref, precision, what, tol=None):
    tol = TOL[precision] if tol is None else tol
    for name, got, r in zip("ISNC", res, ref):
        per, norm = rel_err(got.reshape(-1).double().cpu().numpy(), r)
        assert per <= tol and norm <= tol, (what, precision, name, per, norm)


@pytest.mark.parametrize("npt_azim", [0, 24])
@pytest.mark.parametrize("split", [synth.SPLIT_BBOX, synth.SPLIT_FULL])
def test_table_matches_oracle(split, npt_azim):
    w = small_workload(60, 83, split=split, npt=70, npt_azim=npt_azim, seed=31 + split)
    c = Case(w, mask=random_mask(60, 83, 5))
    gpu = c.gpu_from_oracle_positions()
    gpu.lut_build("fp64")
    gpu.lut_build("fp32")
    pix, c64 = gpu.lut_export("fp64")
    pix32, c32 = gpu.lut_export("fp32")
    idx, coef = O.lut_from_csr(c.A)
    assert gpu.info["lut_width"] == idx.shape[1]
    assert np.array_equal(pix, idx) and np.array_equal(pix32, idx)
    # coefficients: the GPU matrix's own weights in the table's slots, bit for bit
    indptr, indices, data = gpu.export_csr()
    want = np.zeros_like(c64)
    for b in range(gpu.nrows):
        n = indptr[b + 1] - indptr[b]
        want[b, :n] = data[indptr[b]:indptr[b + 1]]
    assert np.array_equal(c64, want)
    assert np.array_equal(c32, want.astype(np.float32))
    assert np.max(np.abs(c64 - coef)) <= 1e-10


@pytest.mark.parametrize("dtype", ["uint32", "float32", "int32"])
@pytest.mark.parametrize("npt_azim", [0, 36])
@pytest.mark.parametrize("corrections", [True, False])
def test_forward_matches_oracle(dtype, npt_azim, corrections):
    w = small_workload(97, 131, npt=90, npt_azim=npt_azim, seed=3, corrections=corrections,
                       dtype="float32" if dtype == "float32" else "uint32")
    c = Case(w)
    if dtype == "int32":
        c.image = c.image.astype(np.int32) - 40  # some negative counts
    gpu = c.gpu_from_oracle_positions()
    ref = oracle_lut_forward(c)
    for precision in ("fp64", "fp32"):
        res = gpu.integrate_lut(to_dev(c.image), *c.corrections_dev(), precision=precision)
        check(res, ref, precision, "lut %s %d" % (dtype, npt_azim))
        again = gpu.integrate_lut(to_dev(c.image), *c.corrections_dev(), precision=precision)
        for a, b in zip(res, again):
            assert torch.equal(a, b)
    assert gpu.status() == 0


def test_more_bins_than_pixels_and_empty_rows():
    w = small_workload(12, 10, split=synth.SPLIT_FULL, npt=2000, seed=9)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    ref = oracle_lut_forward(c)
    for precision in ("fp64", "fp32"):
        res = gpu.integrate_lut(c.image_dev(), *c.corrections_dev(), precision=precision)
        check(res, ref, precision, "empty rows")
        C = res.count.cpu().numpy()
        assert np.all(res.I.cpu().numpy()[C == 0] == 0.0)


def test_layout_routes_single_frame_forward():
    w = small_workload(80, 64, npt=50, seed=12)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    img, corr = c.image_dev(), c.corrections_dev()
    tiled = gpu.integrate(img, *corr, precision="fp32")
    gpu.set_layout("lut")
    assert gpu.info["layout"] == 1
    for precision in ("fp32", "fp64"):
        routed = gpu.integrate(img, *corr, precision=precision)
        direct = gpu.integrate_lut(img, *corr, precision=precision)
        for a, b in zip(routed, direct):
            assert torch.equal(a, b)
    gpu.set_layout("tiled")
    back = gpu.integrate(img, *corr, precision="fp32")
    for a, b in zip(back, tiled):
        assert torch.equal(a, b)
    ref = c.oracle()
    check(back, ref, "fp32", "tiled")


def test_autotune_picks_a_layout():
    w = small_workload(256, 300, npt=300, seed=14)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    gpu.autotune(4)
    assert gpu.info["layout"] in (0, 1)
    res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision="fp32")
    check(res, c.oracle(), "fp32", "after autotune")


def test_pilatus_full_size():
    c = Case(synth.pilatus_workload())
    gpu = c.gpu_from_oracle_positions()
    ref = oracle_lut_forward(c)
    for precision in ("fp64", "fp32"):
        res = gpu.integrate_lut(c.image_dev(), *c.corrections_dev(), precision=precision)
        check(res, ref, precision, "pilatus lut")
    info = gpu.refresh_info()  # the table was built by the first call
    assert info["lut_width"] >= info["nnz"] / info["nrows"]


def test_cake_full_size():
    c = Case(synth.cake_workload())
    gpu = c.gpu_from_geometry()
    # FP64 bar of the 2D full split as in the cake tests (the split weights, not the sums)
    ref = oracle_lut_forward(c)
    for precision, tol in (("fp64", 1e-10), ("fp32", 1e-5)):
        res = gpu.integrate_lut(c.image_dev(), *c.corrections_dev(), precision=precision)
        assert res.I.shape == (360, 500)
        check(res, ref, precision, "cake lut", tol)
