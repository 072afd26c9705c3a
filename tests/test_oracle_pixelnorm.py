"""Pins of the oracle's per-pixel-corrected normalisation (the paper's correction pass then
integration, Sec. 6.4): I = sum w c / sum w with c = (img - dark) / (flat Omega P).

- the corrected sums equal scipy.sparse's product with the corrected image;
- with flat Omega P == 1 it equals the ratio-of-sums form: U = S and, where N = C, I agrees;
- a corrected image of ones (img - dark = flat Omega P) integrates to exactly 1;
- counts C agree with the ratio-of-sums form's C.
"""
import numpy as np
import pytest

import oracle as O
from paper_1412_6367_gb300 import synth


def _case(seed, npt_azim=0, split=O.SPLIT_FULL):
    rng = np.random.default_rng(seed)
    ny, nx = 30, 34
    g = O.Geometry(*synth.random_geometry(rng, ny, nx).astuple())
    rad, chi = O.positions_for(g, ny, nx, O.UNIT_Q_NM, split, npt_azim)
    A = O.csr_build(ny, nx, rad, chi, None, 40, npt_azim, split)
    img = rng.poisson(300.0, size=(ny, nx)).astype(np.float32)
    dark = rng.normal(10, 1, size=(ny, nx)).astype(np.float32)
    flat = rng.uniform(0.9, 1.1, size=(ny, nx)).astype(np.float32)
    sa = O.solid_angle(g, ny, nx).astype(np.float32)
    pol = O.polarization(g, ny, nx, 0.99).astype(np.float32)
    return A, img, dark, flat, sa, pol


@pytest.mark.parametrize("npt_azim", [0, 16])
def test_pixelnorm_matches_scipy(npt_azim):
    A, img, dark, flat, sa, pol = _case(2, npt_azim)
    I, U, C = O.integrate_pixelnorm(A, img, dark, flat, sa, pol)
    M = A.scipy()
    c = (img.astype(np.float64) - dark) / (flat.astype(np.float64) * sa * pol)
    U_ref, C_ref = M @ c.ravel(), M @ np.ones(M.shape[1])
    assert np.allclose(U, U_ref, rtol=1e-13, atol=1e-9)
    assert np.allclose(C, C_ref, rtol=1e-13, atol=1e-12)
    assert np.allclose(I, np.where(C_ref > 0, U_ref / np.where(C_ref > 0, C_ref, 1), 0), rtol=1e-12)


@pytest.mark.parametrize("split", [O.SPLIT_NONE, O.SPLIT_BBOX, O.SPLIT_FULL])
def test_unit_normalisation_equals_ratio_of_sums(split):
    A, img, dark, *_ = _case(3, split=split)
    I, U, C = O.integrate_pixelnorm(A, img, dark)
    I2, S, N, C2 = O.integrate(A, img, dark)
    assert np.array_equal(U, S) and np.array_equal(C, C2) and np.array_equal(I, I2)


def test_corrected_ones_integrate_to_one():
    A, img, dark, flat, sa, pol = _case(4)
    one = (flat.astype(np.float64) * sa * pol)
    I, U, C = O.integrate_pixelnorm(A, one, None, flat, sa, pol)
    pop = C > 0
    assert np.all(np.abs(I[pop] - 1.0) <= 4e-16)
