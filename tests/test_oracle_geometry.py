"""Pins of the oracle's geometry against closed forms and library routines (CPU only).

Sec. 3 lists the coordinates (r, chi, 2theta, q); the tilted-detector convention is a
reading (t = Rz(rot3) Ry(rot2) Rx(rot1) (x1, x2, L)), pinned here against scipy's rotation
routine, the PONI identity, the rot3 azimuth shift, the exact solid angle of a rectangle
and the dot-product form of the polarisation factor.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O


def rel_close(a, b, rtol, atol=0.0):
    a, b = np.asarray(a), np.asarray(b)
    return np.all(np.abs(a - b) <= atol + rtol * np.maximum(np.abs(a), np.abs(b)))


def det_coords(ny, nx, p1, p2, corners=True):
    if corners:
        a, b = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        return a * p1, b * p2
    i, j = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return (i + 0.5) * p1, (j + 0.5) * p2


def scipy_lab(g, d1, d2):
    R = Rotation.from_euler("xyz", [g.rot1, g.rot2, g.rot3]).as_matrix()
    x = np.stack([d1 - g.poni1, d2 - g.poni2, np.full_like(d1, g.dist)], axis=-1)
    return x @ R.T


def test_rotation_matches_scipy_extrinsic_xyz():
    rng = np.random.default_rng(11)
    for _ in range(20):
        r = rng.uniform(-np.pi, np.pi, 3)
        R = O.rotation(*r)
        ref = Rotation.from_euler("xyz", r).as_matrix()
        assert np.allclose(R, ref, atol=1e-15, rtol=0)


@pytest.mark.parametrize("corners", [True, False])
def test_untilted_closed_forms(corners):
    """rot = 0: r = sqrt(x^2 + y^2), chi = atan(y/x) (y = dim1), 2theta = atan(r/d),
    q = 4 pi sin(2theta/2)/lambda (Sec. 3 coordinate list)."""
    g = O.Geometry(dist=0.1, poni1=12.03e-3, poni2=12.85e-3, pixel1=100e-6, pixel2=100e-6,
                   wavelength=1.0e-10)
    ny, nx = 40, 56
    d1, d2 = det_coords(ny, nx, g.pixel1, g.pixel2, corners)
    x1, x2 = d1 - g.poni1, d2 - g.poni2
    r = np.hypot(x1, x2)
    tth = np.arctan(r / g.dist)
    fn = O.corner_positions if corners else O.centre_positions
    tth_deg, chi = fn(g, ny, nx, O.UNIT_2TH_DEG)
    assert rel_close(tth_deg, np.degrees(tth), 1e-14)
    assert rel_close(chi, np.degrees(np.arctan2(x1, x2)), 1e-14, 1e-12)
    q, _ = fn(g, ny, nx, O.UNIT_Q_NM)
    assert rel_close(q, 4 * np.pi * np.sin(tth / 2) / g.wavelength * 1e-9, 1e-14)
    rmm, _ = fn(g, ny, nx, O.UNIT_R_MM)
    assert rel_close(rmm, r * 1e3, 1e-13)


def test_tilted_positions_match_scipy_rotation():
    rng = np.random.default_rng(5)
    for _ in range(8):
        g = O.Geometry(dist=rng.uniform(0.05, 0.5), poni1=rng.uniform(0, 0.01),
                       poni2=rng.uniform(0, 0.01), rot1=rng.uniform(-0.3, 0.3),
                       rot2=rng.uniform(-0.3, 0.3), rot3=rng.uniform(-3, 3),
                       pixel1=150e-6, pixel2=120e-6, wavelength=0.8e-10)
        ny, nx = 33, 47
        d1, d2 = det_coords(ny, nx, g.pixel1, g.pixel2, True)
        t = scipy_lab(g, d1, d2)
        tth_ref = np.arctan2(np.hypot(t[..., 0], t[..., 1]), t[..., 2])
        tth, chi = O.corner_positions(g, ny, nx, O.UNIT_2TH_DEG)
        assert rel_close(tth, np.degrees(tth_ref), 1e-13, 1e-13)
        assert rel_close(chi, np.degrees(np.arctan2(t[..., 0], t[..., 1])), 1e-13, 1e-11)
        # independent angle formula where it is well conditioned
        far = tth_ref > 0.05
        cos_ref = t[..., 2] / np.linalg.norm(t, axis=-1)
        assert rel_close(np.radians(tth[far]), np.arccos(cos_ref[far]), 1e-11)


def test_two_theta_at_poni():
    """At the PONI, 2theta = arccos(cos rot1 cos rot2) whatever rot3 is."""
    rng = np.random.default_rng(7)
    for _ in range(25):
        p = 100e-6
        a, b = int(rng.integers(1, 30)), int(rng.integers(1, 30))
        r1, r2, r3 = rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(-3, 3)
        g = O.Geometry(dist=0.2, poni1=a * p, poni2=b * p, rot1=r1, rot2=r2, rot3=r3,
                       pixel1=p, pixel2=p)
        tth, _ = O.corner_positions(g, 31, 31, O.UNIT_2TH_DEG)
        ref = np.degrees(np.arccos(np.cos(r1) * np.cos(r2)))
        assert abs(tth[a, b] - ref) <= 1e-11 * max(ref, 1e-3)


def test_rot3_shifts_chi_and_keeps_two_theta():
    g0 = O.Geometry(dist=0.15, poni1=3.1e-3, poni2=2.2e-3)
    for r3 in (0.3, -1.2, 2.9):
        g = O.Geometry(dist=0.15, poni1=3.1e-3, poni2=2.2e-3, rot3=r3)
        t0, c0 = O.corner_positions(g0, 50, 60, O.UNIT_2TH_DEG)
        t1, c1 = O.corner_positions(g, 50, 60, O.UNIT_2TH_DEG)
        assert rel_close(t1, t0, 1e-14, 1e-13)
        d = (c1 - (c0 - np.degrees(r3)) + 180.0) % 360.0 - 180.0
        assert np.max(np.abs(d)) < 1e-10


def test_four_fold_symmetry_centred():
    p = 100e-6
    g = O.Geometry(dist=0.1, poni1=32 * p, poni2=32 * p, pixel1=p, pixel2=p)
    tth, _ = O.centre_positions(g, 64, 64, O.UNIT_2TH_DEG)
    assert rel_close(tth, tth[::-1, :], 1e-14)
    assert rel_close(tth, tth[:, ::-1], 1e-14)
    assert rel_close(tth, tth.T, 1e-14)


def _rect_solid_angle(xa, xb, ya, yb, L):
    F = lambda x, y: np.arctan(x * y / (L * np.sqrt(x * x + y * y + L * L)))
    return F(xb, yb) - F(xa, yb) - F(xb, ya) + F(xa, ya)


@pytest.mark.parametrize("rot", [(0.0, 0.0, 0.0), (0.2, -0.1, 0.7)])
def test_solid_angle_matches_exact_rectangle(rot):
    """Omega_p relative to the PONI equals the exact solid angle of the pixel rectangle
    times L^2 / pixel area, up to O((pixel/L)^2).  A cos^2 or cos^4 law would fail."""
    p, L = 100e-6, 0.05
    ny, nx = 24, 30
    g = O.Geometry(dist=L, poni1=-8e-3, poni2=5e-3, rot1=rot[0], rot2=rot[1], rot3=rot[2],
                   pixel1=p, pixel2=p)
    sa = O.solid_angle(g, ny, nx)
    i, j = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    xa, xb = i * p - g.poni1, (i + 1) * p - g.poni1
    ya, yb = j * p - g.poni2, (j + 1) * p - g.poni2
    ref = _rect_solid_angle(xa, xb, ya, yb, L) * L * L / (p * p)
    assert rel_close(sa, ref, 2e-5)
    # the cos^2 alternative differs far more than that tolerance
    assert np.max(np.abs(sa ** (2 / 3) - ref) / ref) > 1e-2


def test_solid_angle_is_one_at_poni():
    p = 100e-6
    g = O.Geometry(dist=0.1, poni1=10.5 * p, poni2=3.5 * p, rot1=0.3, pixel1=p, pixel2=p)
    sa = O.solid_angle(g, 20, 20)
    assert sa[10, 3] == 1.0


@pytest.mark.parametrize("f", [0.99, 0.0, 1.0, -0.5])
def test_polarization_matches_dot_product_form(f):
    """P(f) = (1+f)/2 (1 - (e2.s)^2) + (1-f)/2 (1 - (e1.s)^2): the textbook intensity of a
    dipole along lab axis 2 / axis 1, mixed by the polarisation factor."""
    g = O.Geometry(dist=0.08, poni1=1.1e-3, poni2=2.4e-3, rot1=0.05, rot2=-0.03, rot3=0.4,
                   pixel1=172e-6, pixel2=172e-6)
    ny, nx = 30, 26
    pol = O.polarization(g, ny, nx, f)
    d1, d2 = det_coords(ny, nx, g.pixel1, g.pixel2, corners=False)
    t = scipy_lab(g, d1, d2)
    s = t / np.linalg.norm(t, axis=-1, keepdims=True)
    ref = (1 + f) / 2 * (1 - s[..., 1] ** 2) + (1 - f) / 2 * (1 - s[..., 0] ** 2)
    assert rel_close(pol, ref, 1e-13)
    if f == 0.0:
        tth, _ = O.centre_positions(g, ny, nx, O.UNIT_2TH_DEG)
        assert rel_close(pol, (1 + np.cos(np.radians(tth)) ** 2) / 2, 1e-13)
