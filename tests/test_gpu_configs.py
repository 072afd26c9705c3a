"""GPU parity at the full sizes of the five workloads, in the launch configuration the
benchmark times (default tiles and frames per pass, frames batched 64 per launch).

- Pilatus 6M (2527 x 2463 uint32, module-gap mask, 1000 q bins, full split, corrections):
  matrix indices bit-exact with the oracle's, from the oracle's positions and end to end;
  FP64 one frame within 1e-12; a 140-frame batch (two full 64-frame launches and a ragged one)
  within 1e-5 of the oracle on sampled frames, and bit-identical to the single-frame FP32
  path.
- Cake (2048 x 2048 float32, 500 2theta x 360 chi bins, full split, PONI on a pixel corner):
  FP32 within 1e-5 per bin; FP64 within 1e-10 per bin.  The FP64 bar is set by the split
  weights, not by the sums: the GPU integrates the cell edges of each pixel (Sec. 4.2) where
  the oracle clips polygons, both in FP64 on bin coordinates up to 500 (2theta) and 360 (chi),
  whose ulps (5.7e-14, 5.7e-14) divided by the area of the small cell fragments of a 2D split
  (down to ~1e-3 of a bin cell) bound the weight differences near 1e-11.

Split weights of the two sides agree to 1e-10 absolute and 1e-13 on average for the same
reason.
- Batching: 64 instances of three detector shapes and 500 / 2000 / 5000 bins in one
  graph-captured launch, identical to one launch per instance, three instances against the
  oracle and every instance against the count invariant; a stream of 2167 x 2070 frames
  through one matrix from host buffers against the oracle.
- Differentiation: the Pilatus gradient of sum (I - T)^2 for image and flat field against
  the oracle's explicit transpose product within 1e-5.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_1412_6367_gb300 import synth
from gpu_common import (Case, api, gpu_geometry, needs_gpu, oracle_geometry, rel_err, to_dev,
                        UNIT_NAMES, SPLIT_NAMES)

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def check(res, ref, precision, what, tol=None):
    tol = TOL[precision] if tol is None else tol
    for name, got, r in zip("ISNC", res, ref):
        per, norm = rel_err(np.asarray(got.cpu() if torch.is_tensor(got) else got), r)
        assert per <= tol and norm <= tol, (what, precision, name, per, norm)


@pytest.fixture(scope="module")
def pilatus():
    w = synth.pilatus_workload()
    return Case(w)


@pytest.fixture(scope="module")
def pilatus_gpu(pilatus):
    return pilatus.gpu_from_geometry()


def test_pilatus_indices_bit_exact(pilatus, pilatus_gpu):
    c = pilatus
    indptr, indices, data = pilatus_gpu.export_csr()
    assert np.array_equal(indptr.astype(np.int64), c.A.indptr)
    assert np.array_equal(indices, c.A.indices)
    # weights: different area methods on the two sides (see the module docstring)
    dw = np.abs(data - c.A.data)
    assert dw.max() <= 1e-10 and dw.mean() <= 1e-13, (dw.max(), dw.mean())
    g2 = c.gpu_from_oracle_positions()
    indptr2, indices2, _ = g2.export_csr()
    assert np.array_equal(indices2, c.A.indices)
    assert np.array_equal(indptr2.astype(np.int64), c.A.indptr)


def test_pilatus_fp64_single_frame(pilatus, pilatus_gpu):
    c = pilatus
    res = pilatus_gpu.integrate(c.image_dev(), *c.corrections_dev(), precision="fp64")
    check(res, c.oracle(), "fp64", "pilatus fp64")


def test_pilatus_batch_140_frames(pilatus, pilatus_gpu):
    c = pilatus
    n = 140
    base = [synth.ring_image(c.crad, seed=100 + k, dtype=np.uint32) for k in range(5)]
    frames = np.stack([base[k % 5] for k in range(n)])
    corr = c.corrections_dev()
    out = pilatus_gpu.integrate_batch(to_dev(frames), *corr)
    torch.cuda.synchronize()
    for k in (0, 63, 127, 128, 139):
        ref = c.oracle(frames[k])
        got = (out.I[k], out.sum_signal[k], out.sum_norm, out.count)
        check(got, ref, "fp32", "pilatus batch frame %d" % k)
        one = pilatus_gpu.integrate(to_dev(frames[k]), *corr, precision="fp32")
        assert torch.equal(one.I, out.I[k]) and torch.equal(one.sum_signal, out.sum_signal[k])
    assert pilatus_gpu.status() == 0


def test_cake_full_size():
    w = synth.cake_workload()
    c = Case(w)
    gpu = c.gpu_from_geometry()
    corr = c.corrections_dev()
    ref = c.oracle()
    for precision, tol in (("fp32", 1e-5), ("fp64", 1e-10)):
        res = gpu.integrate(c.image_dev(), *corr, precision=precision)
        assert res.I.shape == (360, 500)
        check([t.reshape(-1) for t in res], ref, precision, "cake", tol)


def test_batching_64_instances():
    ws = synth.batch_instances()
    gpus, imgs, crads = [], [], []
    for w in ws:
        g = gpu_geometry(w.geometry)
        gpus.append(api().Integrator.build(g, (w.ny, w.nx), w.npt_rad, 0, UNIT_NAMES[w.unit],
                                           SPLIT_NAMES[w.split]))
        crad, _ = g.positions(w.ny, w.nx, UNIT_NAMES[w.unit], "centres", chi=False)
        img = synth.ring_image(crad.cpu().numpy(), seed=w.seed, dtype=np.uint32)
        imgs.append(to_dev(img))
    plan = api().MultiPlan(gpus, imgs)
    outs = plan.launch(use_graph=True)
    outs = plan.launch(use_graph=True)  # replay of the captured graph
    torch.cuda.synchronize()
    checked_shapes = set()
    for w, g, img, o in zip(ws, gpus, imgs, outs):
        one = g.integrate(img, precision="fp32")
        for a, b in zip(o, one):
            assert torch.equal(a, b)
        # every unmasked pixel's weights sum to 1: the counts add up to the pixel count
        assert abs(float(o.count.double().sum()) - w.ny * w.nx) <= 1e-4 * w.ny * w.nx
        if (w.ny, w.nx) not in checked_shapes:
            checked_shapes.add((w.ny, w.nx))
            c = Case(w, image=img.view(torch.int32).cpu().numpy().view(np.uint32), with_corrections=False)
            check(o, c.oracle(), "fp32", "instance %s" % w.name)
    assert len(checked_shapes) == 3


def test_batching_instances_with_corrections():
    """The many-instance launch with dark, flat, solid angle and polarisation per instance:
    every (shape, bin count) pair of the 64-instance workload is checked against the oracle
    per bin, and every instance against its own single-frame FP32 integration."""
    ws = synth.batch_instances()
    pairs = {}
    for k, w in enumerate(ws):
        pairs.setdefault((w.ny, w.nx, w.npt_rad), k)
    sel = sorted(pairs.values())
    cases, gpus, imgs, corrs = [], [], [], []
    for k in sel:
        c = Case(ws[k], with_corrections=True)
        cases.append(c)
        gpus.append(c.gpu_from_geometry())
        imgs.append(c.image_dev())
        corrs.append(c.corrections_dev())
    plan = api().MultiPlan(gpus, imgs, darks=[x[0] for x in corrs], flats=[x[1] for x in corrs],
                           solid_angles=[x[2] for x in corrs], polarizations=[x[3] for x in corrs])
    outs = plan.launch(use_graph=True)
    outs = plan.launch(use_graph=True)
    torch.cuda.synchronize()
    for c, g, img, corr, o in zip(cases, gpus, imgs, corrs, outs):
        check(o, c.oracle(), "fp32", "instance %s" % c.w.name)
        one = g.integrate(img, *corr, precision="fp32")
        check(o, [t.double().cpu().numpy() for t in one], "fp32", "single %s" % c.w.name)
        assert g.status() == 0


def test_stream_through_one_matrix_from_host():
    w = synth.stream_workload()
    c = Case(w, with_corrections=False)
    gpu = c.gpu_from_geometry()
    base = [synth.ring_image(c.crad, seed=s, dtype=np.uint32) for s in range(5)]
    frames = np.stack([base[(3 * k) % 5] for k in range(40)])
    I, S = gpu.integrate_batch_host(to_dev(frames, pinned=True))
    for k in (0, 17, 39):
        ref = c.oracle(frames[k])
        for name, got, r in (("I", I[k], ref[0]), ("S", S[k], ref[1])):
            per, norm = rel_err(got.numpy(), r)
            assert per <= 1e-5 and norm <= 1e-5, (k, name, per, norm)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_differentiation_full_size(pilatus, pilatus_gpu, precision):
    from paper_1412_6367_gb300.autograd import AzimuthalIntegrate
    c = pilatus
    img2 = synth.ring_image(c.crad, seed=2, dtype=np.uint32)
    T = c.oracle(img2)[0]
    dt = torch.float64 if precision == "fp64" else torch.float32
    img = torch.from_numpy(c.image.astype(np.float32)).cuda().requires_grad_(True)
    flat = torch.from_numpy(c.flat).cuda().requires_grad_(True)
    dark, sa, pol = c.dev(c.dark), c.dev(c.sa), c.dev(c.pol)
    I = AzimuthalIntegrate.apply(img, flat, pilatus_gpu, dark, sa, pol, precision)
    loss = torch.sum((I.to(torch.float64) - torch.from_numpy(T).cuda()) ** 2)
    loss.backward()
    # the oracle's explicit transpose product with the oracle's own forward quantities
    Io, So, No, Co = c.oracle(c.image.astype(np.float32))
    g = 2.0 * (Io - T)
    gi_ref, gf_ref = O.backward(c.A, g, Io, No, c.sa, c.pol)
    for got, ref in ((img.grad, gi_ref), (flat.grad, gf_ref)):
        per, norm = rel_err(got.double().cpu().numpy(), ref)
        assert norm <= 1e-5, (precision, per, norm)
    # pixel by pixel: the oracle's transpose product over the GPU's own matrix (its split
    # weights differ from the oracle's by up to 1e-10, see the module docstring) with the GPU
    # forward's own I and N.  The upstream gradient 2 (I - T) changes sign between bins, so
    # each pixel is bounded by the tolerance times its sum over absolute values.
    ip, ix, dv = pilatus_gpu.export_csr()
    Ag = dataclasses.replace(c.A, indptr=ip.astype(np.int64), indices=ix, data=dv)
    res = pilatus_gpu.integrate(img.detach(), dark, flat.detach(), sa, pol, precision=precision)
    Ig, Ng = (t.double().cpu().numpy() for t in (res.I, res.sum_norm))
    gg = 2.0 * (Ig - T)
    gi_ref, gf_ref = O.backward(Ag, gg, Ig, Ng, c.sa, c.pol)
    gi_abs, gf_abs = O.backward(Ag, np.abs(gg), np.abs(Ig), Ng, c.sa, c.pol)
    if precision == "fp64":
        # the FP64 adjoint itself; the autograd gradients are those values rounded to the
        # float32 of the image and flat tensors
        gd, gfd = pilatus_gpu.backward(torch.from_numpy(gg).cuda(), res.I, res.sum_norm, sa, pol, "fp64")
        pairs = ((gd, gi_ref, gi_abs), (gfd, gf_ref, gf_abs))
        tol = 1e-12
        for a32, a64 in ((img.grad, gd), (flat.grad, gfd)):
            a32, a64 = a32.double().cpu().numpy().ravel(), a64.cpu().numpy().ravel()
            assert np.all(np.abs(a32 - a64) <= 2.0 ** -24 * np.abs(a64)), "float32 rounding"
    else:
        pairs = ((img.grad, gi_ref, gi_abs), (flat.grad, gf_ref, gf_abs))
        tol = 1e-5
    for got, ref, absref in pairs:
        got = got.double().cpu().numpy().ravel()
        bad = np.abs(got - ref) > tol * np.abs(absref) + 1e-300
        assert not bad.any(), (precision, int(bad.sum()))


def test_largest_size_flat_image():
    """The largest image of the size sweep (4096 x 4096 int32, 1000 q bins, bounding-box
    split): a flat image of ones integrates to I = 1 exactly in every bin with counts, through
    the batch, the single-frame and the look-up-table forms, and the counts add up to the
    pixel count (every pixel's weights sum to 1)."""
    w = synth.size_sweep_workloads()[-1]
    assert (w.ny, w.nx) == (4096, 4096)
    g = gpu_geometry(w.geometry)
    ig = api().Integrator.build(g, (w.ny, w.nx), w.npt_rad, 0, UNIT_NAMES[w.unit], SPLIT_NAMES[w.split])
    ones = torch.ones((3, w.ny, w.nx), dtype=torch.int32, device="cuda")
    out = ig.integrate_batch(ones)
    one = ig.integrate(ones[0], precision="fp32")
    lut = ig.integrate_lut(ones[0], precision="fp32")
    C = out.count.cpu().numpy()
    has = C > 0
    for I in (out.I[0], out.I[2], one.I, lut.I):
        I = I.cpu().numpy()
        assert np.all(I[has] == 1.0) and np.all(I[~has] == 0.0)
    assert abs(float(out.count.double().sum()) - w.ny * w.nx) <= 1e-6 * w.ny * w.nx
    assert ig.status() == 0
