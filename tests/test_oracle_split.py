"""Pins of the oracle's binning and pixel splitting (CPU only).

- hand-derived weights (tests/golden/split_pixels.txt, Sec. 4.1 / 4.2);
- no-split counts bit-exact against numpy.histogram (Sec. 3.3);
- no-split means equal to the paper's naive loop + mean (Sec. 3.2);
- per-pixel fractions sum to 1, i.e. signal and pixel conservation (Sec. 4);
- full split converges to brute-force 64 x 64 sub-pixel sampling (Sec. 4.2);
- CSR structure: rows ascending by pixel, no duplicates, masked pixels absent (Sec. 5.2.1).
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from paper_1412_6367_gb300 import synth
from splitfix import column_entries, fixture_detector, load_fixtures


def _geom(p: synth.GeometryParams):
    return O.Geometry(*p.astuple())


@pytest.mark.parametrize("ndim", [1, 2])
@pytest.mark.parametrize("split", [O.SPLIT_BBOX, O.SPLIT_FULL])
def test_golden_split_weights(ndim, split):
    fx = [f for f in load_fixtures() if f["ndim"] == ndim and f["split"] == split]
    assert fx
    ny, nx, rad, chi, mask, cols = fixture_detector([f["corners"] for f in fx])
    A = O.csr_build(ny, nx, rad, chi, mask, 10, 360 if ndim == 2 else 0, split)
    assert (A.lo, A.hi, A.delta) == (0.0, 10.0, 1.0)
    for f, col in zip(fx, cols):
        got = column_entries(A.indptr, A.indices, A.data, col, 10, ndim)
        assert set(got) == set(f["entries"]), (f["id"], got)
        for k, w in f["entries"].items():
            assert abs(got[k] - w) <= 4e-16, (f["id"], k, got[k], w)


def _ambiguous(x, edges):
    """True where x lies within 4 ulp of a bin edge (either rounding may be right)."""
    k = np.clip(np.searchsorted(edges, x), 1, len(edges) - 1)
    d = np.minimum(np.abs(x - edges[k - 1]), np.abs(x - edges[k]))
    return d <= 4 * np.spacing(np.abs(x))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_no_split_counts_match_numpy_histogram(seed):
    rng = np.random.default_rng(seed)
    ny, nx, npt = 64, 80, int(rng.integers(10, 300))
    g = _geom(synth.random_geometry(rng, ny, nx))
    unit = int(rng.integers(0, 3))
    rad, _ = O.centre_positions(g, ny, nx, unit)
    mask = (rng.random((ny, nx)) < 0.1).astype(np.uint8)
    A = O.csr_build(ny, nx, rad, None, mask, npt, 0, O.SPLIT_NONE)
    x = rad[mask == 0]
    hist, edges = np.histogram(x, bins=npt, range=(x.min(), x.max()))
    counts = np.diff(A.indptr)
    assert A.lo == x.min() and A.hi == x.max()
    assert np.all(A.data == 1.0)
    amb = _ambiguous(x, edges)
    if not amb.any():
        assert np.array_equal(counts, hist)
    else:  # only bins next to an ambiguous value may differ, by at most those values
        assert np.abs(counts - hist).sum() <= 2 * amb.sum()


def _centres_scipy(g, ny, nx):
    """Pixel-centre 2theta (degrees) and chi (degrees in [-180, 180)) computed here with
    scipy's rotation, independently of the oracle: t = R (d1 - poni1, d2 - poni2, L),
    2theta = atan2(|t_12|, t3), chi = atan2(t1, t2) (Sec. 3 coordinate list)."""
    R = Rotation.from_euler("xyz", [g.rot1, g.rot2, g.rot3]).as_matrix()
    d1 = (np.arange(ny) + 0.5)[:, None] * g.pixel1 - g.poni1
    d2 = (np.arange(nx) + 0.5)[None, :] * g.pixel2 - g.poni2
    v = np.stack(np.broadcast_arrays(d1, d2, np.full((1, 1), g.dist)), axis=-1)
    t = v @ R.T
    tth = np.degrees(np.arctan2(np.hypot(t[..., 0], t[..., 1]), t[..., 2]))
    chi = np.degrees(np.arctan2(t[..., 0], t[..., 1]))
    chi = np.where(chi >= 180.0, chi - 360.0, chi)  # the chi range is [-180, 180)
    return tth, chi


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_no_split_2d_counts_match_numpy_histogram2d(seed):
    """The 2D histogram form of Sec. 3.3: with no splitting a pixel goes whole into the bin
    of its centre (radial bin from the data range, chi bin of 360 / npt_azim degrees from
    -180).  Counts per (chi, radial) bin equal numpy.histogram2d of the same centre values,
    except where a value lies within 4 ulp of a bin edge in either direction."""
    rng = np.random.default_rng(40 + seed)
    ny, nx = 60, 72
    npt, nch = int(rng.integers(10, 120)), int(rng.choice([4, 36, 90, 360]))
    g = _geom(synth.random_geometry(rng, ny, nx))
    tth, chi = _centres_scipy(g, ny, nx)
    mask = (rng.random((ny, nx)) < 0.1).astype(np.uint8)
    A = O.csr_build(ny, nx, tth, chi, mask, npt, nch, O.SPLIT_NONE)
    sel = mask == 0
    x, c = tth[sel], chi[sel]
    hist, ce, xe = np.histogram2d(c, x, bins=[nch, npt], range=[[-180.0, 180.0], [x.min(), x.max()]])
    counts = np.diff(A.indptr).reshape(nch, npt)  # row = chi_bin * npt + radial_bin
    assert A.lo == x.min() and A.hi == x.max()
    assert np.all(A.data == 1.0)
    amb = _ambiguous(x, xe) | _ambiguous(c, ce)
    if not amb.any():
        assert np.array_equal(counts, hist)
    else:
        assert np.abs(counts - hist).sum() <= 2 * amb.sum()
    # each pixel's entry: its own (chi, radial) bin, independently of the histogram's edges
    rows = np.repeat(np.arange(A.nrows), np.diff(A.indptr))
    kr = np.minimum(np.floor((tth.ravel() - x.min()) / ((x.max() - x.min()) / npt)), npt - 1)
    kc = np.floor((chi.ravel() + 180.0) / (360.0 / nch)).astype(np.int64) % nch
    want = (kc * npt + kr.astype(np.int64))[A.indices]
    ok = (want == rows) | np.concatenate([amb, [False]])[np.searchsorted(np.flatnonzero(sel), A.indices)]
    assert ok.all()


def test_no_split_equals_naive_loop_mean():
    """Sec. 3.2: per bin, the mean of the pixels whose radius lies in [r1, r2)."""
    p = synth.tiny_workload().geometry
    g = _geom(p)
    ny, nx, npt = 96, 128, 150
    rad, _ = O.centre_positions(g, ny, nx, O.UNIT_2TH_DEG)
    img = synth.tiny_image(rad, seed=4).astype(np.float64)
    A = O.csr_build(ny, nx, rad, None, None, npt, 0, O.SPLIT_NONE)
    I, S, N, C = O.integrate(A, img)
    lo, hi = rad.min(), rad.max()
    for i in range(npt):
        r1 = lo + (hi - lo) * i / npt
        r2 = lo + (hi - lo) * (i + 1) / npt
        sel = (r1 <= rad) & ((rad < r2) if i < npt - 1 else (rad <= r2))
        if sel.sum() == 0:
            assert C[i] == 0 and I[i] == 0
            continue
        assert C[i] == sel.sum()
        assert abs(I[i] - img[sel].mean()) <= 1e-12 * abs(img[sel].mean())


@pytest.mark.parametrize("ndim", [1, 2])
@pytest.mark.parametrize("split", [O.SPLIT_BBOX, O.SPLIT_FULL])
def test_fractions_sum_to_one(ndim, split):
    rng = np.random.default_rng(10 + ndim + split)
    for _ in range(3):
        ny, nx = 40, 52
        g = _geom(synth.random_geometry(rng, ny, nx))
        rad, chi = O.corner_positions(g, ny, nx, O.UNIT_Q_NM)
        mask = (rng.random((ny, nx)) < 0.05).astype(np.uint8)
        A = O.csr_build(ny, nx, rad, chi, mask, 77, 36 if ndim == 2 else 0, split)
        colsum = np.bincount(A.indices, weights=A.data, minlength=ny * nx)
        assert np.all(colsum[mask.reshape(-1) == 1] == 0)
        assert np.max(np.abs(colsum[mask.reshape(-1) == 0] - 1.0)) <= 1e-14
        assert np.all(A.data > 0)
        # pixel conservation: sum of the unweighted histogram = number of pixels (Sec. 4)
        assert abs(A.data.sum() - (mask == 0).sum()) <= 1e-10


@pytest.mark.parametrize("ndim", [1, 2])
def test_csr_structure(ndim):
    rng = np.random.default_rng(99)
    ny, nx = 30, 45
    g = _geom(synth.random_geometry(rng, ny, nx))
    rad, chi = O.corner_positions(g, ny, nx, O.UNIT_2TH_DEG)
    mask = (rng.random((ny, nx)) < 0.2).astype(np.uint8)
    A = O.csr_build(ny, nx, rad, chi, mask, 64, 18 if ndim == 2 else 0, O.SPLIT_FULL)
    assert A.indptr[0] == 0 and A.indptr[-1] == A.nnz
    for r in range(A.nrows):
        row = A.indices[A.indptr[r]:A.indptr[r + 1]]
        assert np.all(np.diff(row) > 0)
    assert not np.any(mask.reshape(-1)[A.indices])
    # scipy accepts it as a canonical CSR matrix (Sec. 5.2.1)
    M = A.scipy()
    assert M.has_canonical_format


def _numpy_positions(g, d1, d2, unit):
    """Independent vectorised geometry (scipy rotation) for the brute-force sampler."""
    R = Rotation.from_euler("xyz", [g.rot1, g.rot2, g.rot3]).as_matrix()
    x = np.stack([d1 - g.poni1, d2 - g.poni2, np.full_like(d1, g.dist)], axis=-1)
    t = x @ R.T
    tth = np.arctan2(np.hypot(t[..., 0], t[..., 1]), t[..., 2])
    if unit == O.UNIT_2TH_DEG:
        return np.degrees(tth)
    return 4 * np.pi * np.sin(tth / 2) / g.wavelength * 1e-9


def _brute_force_counts(g, ny, nx, unit, A, sub=64):
    """Each of sub x sub sample points of every pixel adds 1/sub^2 to the bin of its own
    radial value (same bin rule as the no-split histogram, Sec. 3.3)."""
    u = (np.arange(sub) + 0.5) / sub
    counts = np.zeros(A.nrows)
    for i in range(ny):
        d1 = (i + u[:, None, None]) * g.pixel1 + 0 * u[None, None, :]
        for j in range(nx):
            d2 = (j + u[None, None, :]) * g.pixel2 + 0 * u[:, None, None]
            x = _numpy_positions(g, np.broadcast_to(d1, (sub, 1, sub)).reshape(-1),
                                 np.broadcast_to(d2, (sub, 1, sub)).reshape(-1), unit)
            f = (x - A.lo) / A.delta
            b = np.clip(np.floor(f).astype(int), 0, A.npt_rad - 1)
            counts += np.bincount(b, minlength=A.nrows) / (sub * sub)
    return counts


def test_full_split_converges_to_subpixel_sampling():
    """Full split uses straight edges in the (radial, chi) plane (Sec. 4.2); true pixels
    are curved there, by an amount that shrinks as the pixel gets smaller relative to its
    distance from the beam centre.  The per-bin count must approach the brute-force
    count, and the error must shrink as that ratio grows."""
    errs = []
    ny = nx = 12
    for R_pix in (6, 12, 24):
        p = 100e-6
        g = O.Geometry(dist=0.1, poni1=-R_pix * p, poni2=-0.5 * R_pix * p, pixel1=p, pixel2=p)
        rad, chi = O.corner_positions(g, ny, nx, O.UNIT_2TH_DEG)
        A = O.csr_build(ny, nx, rad, chi, None, 20, 0, O.SPLIT_FULL)
        C = np.bincount(np.repeat(np.arange(A.nrows), np.diff(A.indptr)), weights=A.data,
                        minlength=A.nrows)
        ref = _brute_force_counts(g, ny, nx, O.UNIT_2TH_DEG, A)
        sel = ref > 0.5
        errs.append(np.max(np.abs(C[sel] - ref[sel]) / ref[sel]))
    assert max(errs) < 1e-2, errs
    assert errs[0] > errs[1] > errs[2], errs


def test_full_split_beats_bbox_against_sampling():
    """Sec. 4.1: the bounding box over-estimates the pixel and blurs; the full split is the
    closer of the two to the sampled truth."""
    ny = nx = 10
    p = 100e-6
    g = O.Geometry(dist=0.1, poni1=-40 * p, poni2=-25 * p, rot3=0.3, pixel1=p, pixel2=p)
    rad, chi = O.corner_positions(g, ny, nx, O.UNIT_2TH_DEG)
    out = {}
    for split in (O.SPLIT_BBOX, O.SPLIT_FULL):
        A = O.csr_build(ny, nx, rad, chi, None, 25, 0, split)
        C = np.bincount(np.repeat(np.arange(A.nrows), np.diff(A.indptr)), weights=A.data,
                        minlength=A.nrows)
        out[split] = (A, C)
    ref = _brute_force_counts(g, ny, nx, O.UNIT_2TH_DEG, out[O.SPLIT_FULL][0])
    e_full = np.abs(out[O.SPLIT_FULL][1] - ref).sum()
    e_bbox = np.abs(out[O.SPLIT_BBOX][1] - ref).sum()
    assert e_full < 0.25 * e_bbox


def test_edge_cases():
    g = O.Geometry(dist=0.1, poni1=1e-3, poni2=1e-3)
    rad, chi = O.corner_positions(g, 4, 4, O.UNIT_2TH_DEG)
    crad, cchi = O.centre_positions(g, 4, 4, O.UNIT_2TH_DEG)
    with pytest.raises(O.OracleError) as e:   # every pixel masked
        O.csr_build(4, 4, rad, chi, np.ones((4, 4), np.uint8), 10, 0, O.SPLIT_BBOX)
    assert e.value.code == -8
    with pytest.raises(O.OracleError) as e:   # no bins
        O.csr_build(4, 4, rad, chi, None, 0, 0, O.SPLIT_BBOX)
    assert e.value.code == -1
    with pytest.raises(O.OracleError) as e:   # one unmasked pixel, no split: zero range
        m = np.ones((4, 4), np.uint8)
        m[1, 2] = 0
        O.csr_build(4, 4, crad, None, m, 10, 0, O.SPLIT_NONE)
    assert e.value.code == -8
    # one pixel, split: the pixel spans the whole range and every bin
    r1, c1 = O.corner_positions(g, 1, 1, O.UNIT_2TH_DEG)
    A = O.csr_build(1, 1, r1, c1, None, 5, 0, O.SPLIT_BBOX)
    assert A.nnz == 5 and abs(A.data.sum() - 1) < 1e-15
    # one azimuthal bin: every chi bin index wraps onto bin 0, duplicates are merged
    A = O.csr_build(4, 4, rad, chi, None, 6, 1, O.SPLIT_BBOX)
    colsum = np.bincount(A.indices, weights=A.data, minlength=16)
    assert np.allclose(colsum, 1.0, atol=1e-15)
    for r in range(A.nrows):
        assert np.all(np.diff(A.indices[A.indptr[r]:A.indptr[r + 1]]) > 0)
