"""Pins of the oracle's forward integration and its adjoint (CPU only).

Sec. 3.3 writes the integral as a ratio of two histograms; Sec. 5.2 as a sparse
matrix-vector product over a scipy-compatible CSR matrix.  Pins: a flat image with unit
corrections integrates to exactly 1; signal and pixel conservation (Sec. 4); the product
equals scipy.sparse's; the adjoint equals central finite differences of the forward and
scipy's transpose product.
"""
import numpy as np
import pytest

import oracle as O
from paper_1412_6367_gb300 import synth


def _case(seed, ny=36, nx=44, npt=60, npt_azim=0, split=O.SPLIT_FULL, unit=O.UNIT_Q_NM):
    rng = np.random.default_rng(seed)
    g = O.Geometry(*synth.random_geometry(rng, ny, nx).astuple())
    rad, chi = O.positions_for(g, ny, nx, unit, split, npt_azim)
    mask = (rng.random((ny, nx)) < 0.07).astype(np.uint8)
    A = O.csr_build(ny, nx, rad, chi, mask, npt, npt_azim, split)
    img = rng.poisson(200.0, size=(ny, nx)).astype(np.float32)
    dark = rng.normal(10, 1, size=(ny, nx)).astype(np.float32)
    flat = rng.uniform(0.95, 1.05, size=(ny, nx)).astype(np.float32)
    sa = O.solid_angle(g, ny, nx).astype(np.float32)
    pol = O.polarization(g, ny, nx, 0.99).astype(np.float32)
    return g, A, mask, img, dark, flat, sa, pol


@pytest.mark.parametrize("npt_azim", [0, 24])
@pytest.mark.parametrize("split", [O.SPLIT_NONE, O.SPLIT_BBOX, O.SPLIT_FULL])
def test_flat_image_integrates_to_one(split, npt_azim):
    g, A, mask, *_ = _case(1, split=split, npt_azim=npt_azim)
    ones = np.ones((A.ny, A.nx), np.float32)
    I, S, N, C = O.integrate(A, ones)
    pop = C > 0
    assert np.all(I[pop] == 1.0)
    assert np.all(I[~pop] == 0.0)
    # explicit unit corrections give the same bits
    I2, *_ = O.integrate(A, ones, np.zeros_like(ones), ones, ones, ones)
    assert np.array_equal(I, I2)


@pytest.mark.parametrize("split", [O.SPLIT_NONE, O.SPLIT_BBOX, O.SPLIT_FULL])
def test_conservation(split):
    """Sum of the weighted histogram = sum of the image; sum of the unweighted = number of
    pixels (Sec. 4)."""
    g, A, mask, img, dark, *_ = _case(2, split=split)
    I, S, N, C = O.integrate(A, img, dark)
    keep = mask == 0
    v = img.astype(np.float64) - dark
    assert abs(S.sum() - v[keep].sum()) <= 1e-12 * np.abs(v[keep]).sum()
    assert abs(C.sum() - keep.sum()) <= 1e-11


@pytest.mark.parametrize("npt_azim", [0, 30])
def test_forward_matches_scipy_sparse(npt_azim):
    g, A, mask, img, dark, flat, sa, pol = _case(3, npt_azim=npt_azim)
    I, S, N, C = O.integrate(A, img, dark, flat, sa, pol)
    M = A.scipy()
    v = img.astype(np.float64).ravel() - dark.astype(np.float64).ravel()
    n = flat.astype(np.float64).ravel() * sa.astype(np.float64).ravel() * pol.astype(np.float64).ravel()
    S_ref, N_ref, C_ref = M @ v, M @ n, M @ np.ones(M.shape[1])
    assert np.allclose(S, S_ref, rtol=1e-13, atol=1e-9)
    assert np.allclose(N, N_ref, rtol=1e-13, atol=1e-12)
    assert np.allclose(C, C_ref, rtol=1e-13, atol=1e-12)
    ref_I = np.where(N_ref != 0, S_ref / np.where(N_ref != 0, N_ref, 1), 0)
    assert np.allclose(I, ref_I, rtol=1e-12, atol=0)


def _loss(A, img, flat, sa, pol, target):
    I, S, N, C = O.integrate(A, img, None, flat, sa, pol)
    return np.sum((I - target) ** 2), I, N


@pytest.mark.parametrize("split", [O.SPLIT_BBOX, O.SPLIT_FULL])
def test_adjoint_matches_finite_differences(split):
    """L = sum (I - T)^2; dL/dimage and dL/dflat by central differences in float64."""
    rng = np.random.default_rng(4)
    ny = nx = 10
    g = O.Geometry(dist=0.05, poni1=2e-4, poni2=-3e-4, rot1=0.02, pixel1=100e-6, pixel2=100e-6)
    rad, chi = O.corner_positions(g, ny, nx, O.UNIT_2TH_DEG)
    A = O.csr_build(ny, nx, rad, chi, None, 12, 0, split)
    img = rng.uniform(50, 150, (ny, nx))
    flat = rng.uniform(0.9, 1.1, (ny, nx))
    sa = O.solid_angle(g, ny, nx)
    pol = O.polarization(g, ny, nx, 0.99)
    target = rng.uniform(50, 150, A.nrows)
    L0, I, N = _loss(A, img, flat, sa, pol, target)
    gI = 2 * (I - target)
    g_img, g_flat = O.backward(A, gI, I, N, sa, pol)
    h_img, h_flat = 1e-4, 1e-7
    for p in rng.choice(ny * nx, 25, replace=False):
        e = np.zeros(ny * nx)
        e[p] = 1
        e = e.reshape(ny, nx)
        fd = (_loss(A, img + h_img * e, flat, sa, pol, target)[0]
              - _loss(A, img - h_img * e, flat, sa, pol, target)[0]) / (2 * h_img)
        assert abs(fd - g_img[p]) <= 1e-6 * max(1.0, abs(fd))
        fd = (_loss(A, img, flat + h_flat * e, sa, pol, target)[0]
              - _loss(A, img, flat - h_flat * e, sa, pol, target)[0]) / (2 * h_flat)
        assert abs(fd - g_flat[p]) <= 1e-5 * max(1.0, abs(fd))


def test_adjoint_matches_scipy_transpose():
    g, A, mask, img, dark, flat, sa, pol = _case(5, ny=50, nx=40, npt=70)
    I, S, N, C = O.integrate(A, img, dark, flat, sa, pol)
    gI = np.random.default_rng(0).normal(size=A.nrows)
    g_img, g_flat = O.backward(A, gI, I, N, sa, pol)
    u = np.where(N != 0, gI / np.where(N != 0, N, 1), 0)
    M = A.scipy()
    assert np.allclose(g_img, M.T @ u, rtol=1e-13, atol=1e-16)
    ref = -sa.astype(np.float64).ravel() * pol.astype(np.float64).ravel() * (M.T @ (u * I))
    assert np.allclose(g_flat, ref, rtol=1e-13, atol=1e-16)
