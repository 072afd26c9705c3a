"""The multi-core CPU baseline (oracle/azint_omp.c: the paper's per-thread histograms over the
pixels, Sec. 3.4.1) gives the oracle's sums: FP64, within 1e-12 of orc_integrate per bin
(another summation order), deterministic for a given thread count (CPU)."""
import numpy as np
import pytest

import oracle as O
from paper_1412_6367_gb300 import synth


@pytest.mark.parametrize("npt_azim", [0, 36])
def test_omp_baseline_equals_oracle(npt_azim):
    rng = np.random.default_rng(50 + npt_azim)
    ny, nx = 70, 90
    g = O.Geometry(*synth.random_geometry(rng, ny, nx).astuple())
    rad, chi = O.corner_positions(g, ny, nx, O.UNIT_Q_NM)
    mask = (rng.random((ny, nx)) < 0.1).astype(np.uint8)
    A = O.csr_build(ny, nx, rad, chi, mask, 80, npt_azim, O.SPLIT_FULL)
    img = rng.integers(0, 5000, size=(ny, nx)).astype(np.uint32)
    dark, flat = synth.dark_flat(ny, nx, 3)
    sa = O.solid_angle(g, ny, nx).astype(np.float32)
    pol = O.polarization(g, ny, nx, 0.99).astype(np.float32)
    ref = O.integrate(A, img, dark, flat, sa, pol)
    M = O.csc_of(A)
    got = O.omp_integrate(M, img, dark, flat, sa, pol)
    assert got[4] >= 1
    for r, x in zip(ref, got[:4]):
        scale = np.abs(r).max()
        assert np.max(np.abs(x - r)) <= 1e-12 * scale
    again = O.omp_integrate(M, img, dark, flat, sa, pol)
    for x, y in zip(got[:4], again[:4]):
        assert np.array_equal(x, y)
    # no corrections: S = sum w img, N = C
    I, S, N, C, _ = O.omp_integrate(M, img)
    assert np.array_equal(N, C)
