"""az_csr_import: a host CSR matrix (scipy layout, Sec. 5.2.1) brought into an integrator.

- export -> import -> export gives the same three arrays bit for bit, and the imported
  integrator's forward (FP64, FP32, batch) and adjoint give the bits of the original;
- the oracle's own matrix, imported, separates the GPU's summation from its split weights:
  on the full-size 2048 x 2048 cake (500 x 360 bins, full split, corrections) the FP64 sums
  agree with the oracle's within 1e-12 per bin, FP32 compensated within 1e-5, and the FP64
  adjoint agrees pixel by pixel with the oracle's transpose product within 1e-12 of each
  pixel's sum of absolute terms.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1412_6367_gb300 import synth
from gpu_common import Case, api, needs_gpu, rel_err, small_workload, to_dev, SPLIT_NAMES

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.mark.parametrize("npt_azim", [0, 24])
def test_export_import_round_trip(npt_azim):
    w = small_workload(90, 110, npt=70, npt_azim=npt_azim, seed=21)
    c = Case(w)
    g = c.gpu_from_geometry()
    ip, ix, dv = g.export_csr()
    info = g.info
    h = api().Integrator.from_csr((w.ny, w.nx), ip, ix, dv, w.npt_rad, w.npt_azim, info["lo"], info["hi"],
                                  split=SPLIT_NAMES[w.split])
    ip2, ix2, dv2 = h.export_csr()
    assert np.array_equal(ip, ip2) and np.array_equal(ix, ix2)
    assert np.array_equal(dv.view(np.uint64), dv2.view(np.uint64))
    for k in ("nnz", "nrows", "n_unmasked", "lo", "hi", "delta", "tile_h", "tile_w", "n_segments"):
        assert h.info[k] == info[k], k
    assert np.array_equal(h.radial_axis(), g.radial_axis())
    corr = c.corrections_dev()
    img = c.image_dev()
    for prec in ("fp64", "fp32"):
        a, b = g.integrate(img, *corr, precision=prec), h.integrate(img, *corr, precision=prec)
        for x, y in zip(a, b):
            assert torch.equal(x, y), prec
        if prec == "fp64":
            ga = g.backward(torch.ones_like(a.I), a.I, a.sum_norm, corr[2], corr[3], "fp64")
            gb = h.backward(torch.ones_like(b.I), b.I, b.sum_norm, corr[2], corr[3], "fp64")
            rel = max(float((x - y).abs().max() / y.abs().max()) for x, y in zip(ga, gb))
            assert rel <= 1e-15, rel  # each pixel's (few) terms, possibly in another order
    frames = torch.stack([img.view(torch.int32)] * 3).view(torch.uint32)
    a, b = g.integrate_batch(frames, *corr), h.integrate_batch(frames, *corr)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert h.status() == 0


@pytest.fixture(scope="module")
def cake():
    w = synth.cake_workload()
    c = Case(w)
    A = c.A
    h = api().Integrator.from_csr((w.ny, w.nx), A.indptr.astype(np.int32), A.indices, A.data,
                                  w.npt_rad, w.npt_azim, A.lo, A.hi, unit="2th_deg", split="full")
    return c, h


def test_cake_oracle_matrix_fp64_within_1e12(cake):
    c, h = cake
    assert h.info["nnz"] == c.A.nnz and h.info["nrows"] == 500 * 360
    ref = c.oracle()
    res = h.integrate(c.image_dev(), *c.corrections_dev(), precision="fp64")
    for name, got, r in zip("ISNC", res, ref):
        per, norm = rel_err(got.reshape(-1).cpu().numpy(), r)
        assert per <= 1e-12 and norm <= 1e-12, (name, per, norm)
    res = h.integrate(c.image_dev(), *c.corrections_dev(), precision="fp32")
    for name, got, r in zip("ISNC", res, ref):
        per, norm = rel_err(got.reshape(-1).double().cpu().numpy(), r)
        assert per <= 1e-5 and norm <= 1e-5, (name, per, norm)
    assert h.status() == 0


def test_cake_oracle_matrix_adjoint_fp64(cake):
    c, h = cake
    res = h.integrate(c.image_dev(), *c.corrections_dev(), precision="fp64")
    I, N = (t.reshape(-1).cpu().numpy() for t in (res.I, res.sum_norm))
    g = np.random.default_rng(4).normal(size=I.shape)
    gi, gf = h.backward(torch.from_numpy(g).cuda(), res.I.reshape(-1), res.sum_norm.reshape(-1),
                        c.dev(c.sa), c.dev(c.pol), "fp64")
    gi_ref, gf_ref = O.backward(c.A, g, I, N, c.sa, c.pol)
    gi_abs, gf_abs = O.backward(c.A, np.abs(g), np.abs(I), N, c.sa, c.pol)
    for got, ref, absref in ((gi, gi_ref, gi_abs), (gf, gf_ref, gf_abs)):
        got = got.cpu().numpy().ravel()
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(absref) + 1e-300)
