"""GPU parity of the adjoint kernel and the autograd Function.

- against the oracle's explicit transpose product: FP64 within 1e-12, FP32 within 1e-5,
  pixel by pixel.  Each pixel's gradient is a short signed sum over its bins, so the bound
  of a pixel is the tolerance times that sum taken over absolute values (its condition),
  with the transpose product formed from the GPU forward's own I and N; with an upstream
  gradient of one sign (no cancellation) the plain relative error of every pixel above
  1e-3 of the maximum is held to the same tolerance;
- central finite differences in float64 of L = sum (I - T)^2 on a 64 x 64 detector with 50
  bins, through torch.autograd (exactly representable float32 perturbations, so that the
  float64 differences are those of the forward alone).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1412_6367_gb300 import synth
from gpu_common import Case, needs_gpu, rel_err, small_workload

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("split", [1, 2])
def test_adjoint_matches_oracle_transpose(precision, split):
    w = small_workload(90, 120, split=split, npt=80, seed=61 + split)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    I, S, N, C = c.oracle()
    gI = np.random.default_rng(1).normal(size=I.shape)
    gi_ref, gf_ref = O.backward(c.A, gI, I, N, c.sa, c.pol)
    dt = torch.float64 if precision == "fp64" else torch.float32
    res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision=precision)
    tol = 1e-12 if precision == "fp64" else 1e-5
    Ig, Ng = (t.double().cpu().numpy() for t in (res.I, res.sum_norm))
    # a signed upstream gradient and one of a single sign
    for gI, signed in ((gI, True), (np.random.default_rng(2).uniform(0.5, 1.5, size=I.shape), False)):
        g = torch.from_numpy(gI).to(dt).cuda()
        gi, gf = gpu.backward(g, res.I, res.sum_norm, c.dev(c.sa), c.dev(c.pol), precision)
        gi, gf = gi.double().cpu().numpy().ravel(), gf.double().cpu().numpy().ravel()
        if signed:  # end to end against the oracle's own forward: normwise
            gi_ref, gf_ref = O.backward(c.A, gI, I, N, c.sa, c.pol)
            for got, ref in ((gi, gi_ref), (gf, gf_ref)):
                per, norm = rel_err(got, ref)
                assert norm <= tol, (precision, per, norm)
        # pixel by pixel against the transpose product of the GPU forward's I and N
        gi_ref, gf_ref = O.backward(c.A, gI, Ig, Ng, c.sa, c.pol)
        gi_abs, gf_abs = O.backward(c.A, np.abs(gI), np.abs(Ig), Ng, c.sa, c.pol)
        for got, ref, absref in ((gi, gi_ref, np.abs(gi_abs)), (gf, gf_ref, np.abs(gf_abs))):
            assert np.all(np.abs(got - ref) <= tol * absref + 1e-300), (precision, signed)
            if not signed:
                per, norm = rel_err(got, ref)
                assert per <= tol and norm <= tol, (precision, per, norm)


def _loss(gpu, img, flat, sa, pol, target):
    I = gpu.integrate(img, None, flat, sa, pol, precision="fp64").I
    return float(torch.sum((I - target) ** 2))


def test_finite_differences_64x64():
    from paper_1412_6367_gb300.autograd import AzimuthalIntegrate
    p = synth.GeometryParams(dist=0.01, poni1=32.3e-4, poni2=30.1e-4, rot1=0.02, pixel1=100e-6,
                             pixel2=100e-6)
    w = synth.Workload("fd", 64, 64, p, synth.UNIT_2TH_DEG, synth.SPLIT_FULL, 50)
    c = Case(w, with_corrections=True)
    gpu = c.gpu_from_oracle_positions()
    img = torch.from_numpy(synth.uniform_image(64, 64, 3, 100, 200)).cuda().requires_grad_(True)
    flat = torch.from_numpy(c.flat).cuda().requires_grad_(True)
    sa, pol = c.dev(c.sa), c.dev(c.pol)
    target = torch.from_numpy(np.random.default_rng(2).uniform(100, 200, 50)).cuda()
    I = AzimuthalIntegrate.apply(img, flat, gpu, None, sa, pol, "fp64")
    loss = torch.sum((I - target) ** 2)
    loss.backward()
    # the same gradient in float64 straight from the adjoint kernel
    res = gpu.integrate(img.detach(), None, flat.detach(), sa, pol, precision="fp64")
    gd, gfd = gpu.backward(2 * (res.I - target), res.I, res.sum_norm, sa, pol, "fp64")
    assert torch.allclose(img.grad.double(), gd, rtol=1e-6, atol=0)
    assert torch.allclose(flat.grad.double(), gfd, rtol=1e-6, atol=1e-12)
    g_img, g_flat = gd.cpu().numpy(), gfd.cpu().numpy()
    rng = np.random.default_rng(0)
    hi, hf = 0.25, 2.0 ** -12  # exact in float32 at these magnitudes
    base_img, base_flat = img.detach().clone(), flat.detach().clone()
    for p_ in rng.choice(64 * 64, 30, replace=False):
        i, j = divmod(int(p_), 64)
        a, b = base_img.clone(), base_img.clone()
        a[i, j] += hi
        b[i, j] -= hi
        fd = (_loss(gpu, a, base_flat, sa, pol, target) - _loss(gpu, b, base_flat, sa, pol, target)) / (2 * hi)
        assert abs(fd - g_img[i, j]) <= 1e-7 * max(1.0, abs(fd)), (i, j, fd, g_img[i, j])
        a, b = base_flat.clone(), base_flat.clone()
        a[i, j] += hf
        b[i, j] -= hf
        fd = (_loss(gpu, base_img, a, sa, pol, target) - _loss(gpu, base_img, b, sa, pol, target)) / (2 * hf)
        assert abs(fd - g_flat[i, j]) <= 1e-4 * max(1.0, abs(fd)), (i, j, fd, g_flat[i, j])


def test_autograd_fp32_matches_fp64():
    from paper_1412_6367_gb300.autograd import integrate
    w = small_workload(80, 90, split=2, npt=60, seed=8)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    grads = {}
    for prec in ("fp64", "fp32"):
        img = torch.from_numpy(c.image.astype(np.float32)).cuda().requires_grad_(True)
        flat = c.dev(c.flat).requires_grad_(True)
        I = integrate(img, flat, gpu, c.dev(c.dark), c.dev(c.sa), c.dev(c.pol), prec)
        (I.double() ** 2).sum().backward()
        grads[prec] = (img.grad.double().cpu().numpy(), flat.grad.double().cpu().numpy())
    # L = sum I^2 with I > 0: gradients of one sign, no cancellation inside a pixel's sum
    for a, b in zip(grads["fp32"], grads["fp64"]):
        per, norm = rel_err(a, b)
        assert per <= 1e-5 and norm <= 1e-5, (per, norm)
