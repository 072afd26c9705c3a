"""Pins of the oracle's look-up-table layout (Sec. 5.2: per output bin, the (pixel index,
coefficient) pairs it gathers from, every bin padded to the same number of slots) and of the
forward through it.

- a hand-written three-bin matrix with an empty bin gives the table written out below;
- the table, scattered back into a dense matrix, equals scipy.sparse's dense form of the
  oracle's CSR matrix, for 1D and 2D, bbox and full split, with a mask;
- its width is the longest row, and every row is its entries then padding only;
- the forward through the table equals scipy.sparse's product of the corrected image within
  rounding, and the CSR forward bit for bit (both add a bin's entries in column order).
"""
import numpy as np
import pytest

import oracle as O
from paper_1412_6367_gb300 import synth


def _matrix(seed, ny=20, nx=24, npt=30, npt_azim=0, split=O.SPLIT_FULL, mask=None):
    rng = np.random.default_rng(seed)
    g = O.Geometry(*synth.random_geometry(rng, ny, nx).astuple())
    rad, chi = O.positions_for(g, ny, nx, O.UNIT_Q_NM, split, npt_azim)
    return O.csr_build(ny, nx, rad, chi, mask, npt, npt_azim, split), rng


def test_hand_example():
    # bin 0 <- 0.5 p1 + 0.25 p3, bin 1 empty, bin 2 <- 1.0 p0 + 0.125 p2 + 2.0 p3
    indptr = [0, 2, 2, 5]
    indices = [1, 3, 0, 2, 3]
    data = [0.5, 0.25, 1.0, 0.125, 2.0]
    idx, coef = O.lut_from_csr_arrays(indptr, indices, data)
    assert idx.tolist() == [[1, 3, -1], [-1, -1, -1], [0, 2, 3]]
    assert coef.tolist() == [[0.5, 0.25, 0.0], [0.0, 0.0, 0.0], [1.0, 0.125, 2.0]]
    img = np.array([8.0, 4.0, 16.0, 32.0])
    flat = np.array([1.0, 2.0, 0.5, 4.0])
    I, S, N, C = O.integrate_lut(idx, coef, img, flat=flat)
    assert S.tolist() == [0.5 * 4 + 0.25 * 32, 0.0, 8.0 + 0.125 * 16 + 2.0 * 32]
    assert N.tolist() == [0.5 * 2 + 0.25 * 4, 0.0, 1.0 + 0.125 * 0.5 + 2.0 * 4]
    assert C.tolist() == [0.75, 0.0, 3.125]
    assert I.tolist() == [10.0 / 2.0, 0.0, 74.0 / 9.0625]


@pytest.mark.parametrize("split", [O.SPLIT_BBOX, O.SPLIT_FULL])
@pytest.mark.parametrize("npt_azim", [0, 12])
def test_table_is_the_matrix(split, npt_azim):
    ny, nx = 22, 27
    mask = np.zeros((ny, nx), np.uint8)
    mask[5:9, 3:20] = 1
    A, _ = _matrix(3 + split + npt_azim, ny, nx, npt=25, npt_azim=npt_azim, split=split, mask=mask)
    idx, coef = O.lut_from_csr(A)
    M = A.scipy().toarray()
    nrows, width = idx.shape
    assert nrows == M.shape[0]
    assert width == int(np.max((M != 0).sum(axis=1)))  # the longest row
    dense = np.zeros_like(M)
    for b in range(nrows):
        real = idx[b] >= 0
        k = int(real.sum())
        assert np.all(real[:k]) and not np.any(real[k:])    # entries first, then padding
        assert np.all(coef[b, k:] == 0.0)
        assert np.all(np.diff(idx[b, :k]) > 0)              # column order
        dense[b, idx[b, :k]] = coef[b, :k]
    assert np.array_equal(dense, M)
    # the LUT holds width * nrows slots against nnz entries of the CSR form
    assert width * nrows >= A.nnz


@pytest.mark.parametrize("npt_azim", [0, 10])
def test_forward_through_table(npt_azim):
    A, rng = _matrix(17, npt=40, npt_azim=npt_azim)
    img = rng.poisson(200.0, size=(A.ny, A.nx)).astype(np.float64)
    dark = rng.normal(10.0, 1.0, size=img.shape)
    flat = rng.uniform(0.9, 1.1, size=img.shape)
    sa = rng.uniform(0.5, 1.0, size=img.shape)
    pol = rng.uniform(0.8, 1.0, size=img.shape)
    idx, coef = O.lut_from_csr(A)
    got = O.integrate_lut(idx, coef, img, dark, flat, sa, pol)
    M = A.scipy()
    S = M @ (img - dark).ravel()
    N = M @ (flat * sa * pol).ravel()
    C = M @ np.ones(img.size)
    for g, r in zip(got[1:], (S, N, C)):
        assert np.allclose(g, r, rtol=1e-13, atol=1e-12)
    ref = O.integrate(A, img, dark, flat, sa, pol)
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
