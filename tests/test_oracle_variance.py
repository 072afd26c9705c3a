"""Pins of the oracle's propagated variance V_b = sum_p w_bp^2 max(img_p, 0) (Poisson counts,
constant dark; an extension: the paper states no error model).

- equals scipy.sparse's elementwise-squared matrix applied to the clipped image;
- without pixel splitting every weight is 1, so V equals the signal sum S of a non-negative
  image without dark;
- statistics: for independent Poisson pixels of mean lambda the variance over many draws of
  the signal sums S = A img equals V(lambda), within the sampling error of the estimate.
"""
import numpy as np
import pytest

import oracle as O
from paper_1412_6367_gb300 import synth


def _matrix(seed, ny=20, nx=24, npt=30, npt_azim=0, split=O.SPLIT_FULL):
    rng = np.random.default_rng(seed)
    g = O.Geometry(*synth.random_geometry(rng, ny, nx).astuple())
    rad, chi = O.positions_for(g, ny, nx, O.UNIT_Q_NM, split, npt_azim)
    return O.csr_build(ny, nx, rad, chi, None, npt, npt_azim, split), rng


@pytest.mark.parametrize("split", [O.SPLIT_BBOX, O.SPLIT_FULL])
@pytest.mark.parametrize("npt_azim", [0, 12])
def test_variance_matches_scipy(split, npt_azim):
    A, rng = _matrix(5 + split, split=split, npt_azim=npt_azim)
    img = rng.normal(50, 60, size=(A.ny, A.nx))  # some negative pixels: clipped at 0
    V = O.variance(A, img)
    M = A.scipy()
    ref = M.multiply(M) @ np.maximum(img.ravel(), 0.0)
    assert np.allclose(V, ref, rtol=1e-13, atol=1e-12)


def test_no_split_variance_is_signal():
    A, rng = _matrix(7, split=O.SPLIT_NONE)
    img = rng.poisson(30.0, size=(A.ny, A.nx)).astype(np.float64)
    V = O.variance(A, img)
    I, S, N, C = O.integrate(A, img)
    assert np.array_equal(V, S)


def test_variance_matches_poisson_statistics():
    A, rng = _matrix(11, ny=12, nx=14, npt=10)
    lam = rng.uniform(20.0, 200.0, size=(A.ny, A.nx))
    V = O.variance(A, lam)
    M = A.scipy()
    draws = rng.poisson(lam.ravel(), size=(40000, lam.size)).astype(np.float64)
    S = draws @ M.T.toarray()
    emp = S.var(axis=0, ddof=1)
    keep = V > 0
    # the sample variance of 40000 draws has a relative standard error of about 0.7 %
    assert np.all(np.abs(emp[keep] / V[keep] - 1.0) < 0.04)
