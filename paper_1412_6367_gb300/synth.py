"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the integration arithmetic: it draws geometries, masks,
correction arrays and Poisson images.  Ring images are shaped on a radial (and azimuthal)
coordinate array that the CALLER computes and passes in, so the same image can be fed to
the CUDA path and to the oracle.  The paper's own test images (a simulated gold-powder
pattern and pyFAI test-suite frames) are not available; these seeded frames stand in for
them with the same detector shapes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

UNIT_2TH_DEG, UNIT_Q_NM, UNIT_R_MM = 0, 1, 2
SPLIT_NONE, SPLIT_BBOX, SPLIT_FULL = 0, 1, 2


@dataclass(frozen=True)
class GeometryParams:
    dist: float
    poni1: float
    poni2: float
    rot1: float = 0.0
    rot2: float = 0.0
    rot3: float = 0.0
    pixel1: float = 100e-6
    pixel2: float = 100e-6
    wavelength: float = 1.0e-10

    def astuple(self):
        return (self.dist, self.poni1, self.poni2, self.rot1, self.rot2, self.rot3,
                self.pixel1, self.pixel2, self.wavelength)


@dataclass(frozen=True)
class Workload:
    name: str
    ny: int
    nx: int
    geometry: GeometryParams
    unit: int
    split: int
    npt_rad: int
    npt_azim: int = 0
    image_dtype: str = "float32"        # "float32" | "uint32"
    masked: bool = False
    corrections: bool = False           # dark, flat, solid angle, polarisation
    polarization_factor: float = 0.99
    seed: int = 0
    extra: dict = field(default_factory=dict)


def tiny_workload() -> Workload:
    """256 x 256 float32, 100 um pixels, 100 mm, beam centre at (col 128.5, row 120.3),
    2theta in degrees, 200 bins, bounding-box split, no mask, no corrections."""
    g = GeometryParams(dist=0.1, poni1=120.3 * 100e-6, poni2=128.5 * 100e-6)
    return Workload("tiny-256x256-bbox-200", 256, 256, g, UNIT_2TH_DEG, SPLIT_BBOX, 200,
                    image_dtype="float32", seed=0)


def pilatus_workload(seed: int = 1, split: int = SPLIT_FULL, npt: int = 1000) -> Workload:
    """Pilatus-6M shape: 2527 x 2463 uint32, 172 um pixels, 300 mm, PONI at the detector
    centre +- U(-5, 5) mm per axis, rot1 = 0.02, rot2 = 0.01, q in nm^-1, 1000 bins,
    full split, module-gap mask, dark/flat/solid-angle/polarisation (f = 0.99)."""
    rng = np.random.default_rng(seed)
    ny, nx, px = 2527, 2463, 172e-6
    off = rng.uniform(-5e-3, 5e-3, size=2)
    g = GeometryParams(dist=0.3, poni1=ny * px / 2 + off[0], poni2=nx * px / 2 + off[1],
                       rot1=0.02, rot2=0.01, rot3=0.0, pixel1=px, pixel2=px,
                       wavelength=1.0e-10)
    return Workload("pilatus6m-2527x2463-q-full-%d" % npt, ny, nx, g, UNIT_Q_NM, split, npt,
                    image_dtype="uint32", masked=True, corrections=True, seed=seed)


def pilatus1m_workload(seed: int = 1, split: int = SPLIT_BBOX, npt: int = 1000) -> Workload:
    """Pilatus-1M shape of the paper's stage timings (Sec. 6.4: 981 x 1043 signed 32-bit
    pixels): 1043 rows x 981 columns (5 x 2 modules of 195 x 487 pixels, gaps of 17 rows and
    7 columns), int32, 172 um, 200 mm, PONI at the centre +- U(-5, 5) mm per axis,
    rot1 = 0.02, rot2 = 0.01, q in nm^-1, 1000 bins, bounding-box split (the paper's
    benchmarks split by bounding box, Sec. 6), module-gap mask, corrections."""
    rng = np.random.default_rng(seed)
    ny, nx, px = 1043, 981, 172e-6
    off = rng.uniform(-5e-3, 5e-3, size=2)
    g = GeometryParams(dist=0.2, poni1=ny * px / 2 + off[0], poni2=nx * px / 2 + off[1],
                       rot1=0.02, rot2=0.01, rot3=0.0, pixel1=px, pixel2=px,
                       wavelength=1.0e-10)
    return Workload("pilatus1m-1043x981-q-bbox-%d" % npt, ny, nx, g, UNIT_Q_NM, split, npt,
                    image_dtype="int32", masked=True, corrections=True, seed=seed)


SWEEP_SHAPES = ((1024, 1024), (1448, 1448), (2048, 2048), (2527, 2463), (3456, 3456), (4096, 4096))


def size_sweep_workloads(npt: int = 1000):
    """The image sizes of the paper's benchmarks (Sec. 6: 1, 2, 4, 6, 12 and 16 Mpixel):
    square detectors of 1024^2, 1448^2, 2048^2, 3456^2 and 4096^2 pixels and the Pilatus-6M
    shape, int32 counts, 100 um pixels, 100 mm, beam centred, no tilt, q in nm^-1, `npt`
    bins, bounding-box split (the split of those benchmarks), no mask, no corrections."""
    out = []
    for ny, nx in SWEEP_SHAPES:
        g = GeometryParams(dist=0.1, poni1=ny * 100e-6 / 2, poni2=nx * 100e-6 / 2,
                           pixel1=100e-6, pixel2=100e-6, wavelength=1.0e-10)
        out.append(Workload("sweep-%dx%d-bbox-%d" % (ny, nx, npt), ny, nx, g, UNIT_Q_NM, SPLIT_BBOX,
                            npt, image_dtype="int32"))
    return out


def cake_workload(seed: int = 2) -> Workload:
    """2048 x 2048 float32, 50 um, 150 mm, rot1 = 0.05, PONI at the detector centre (a pixel
    corner), 500 2theta x 360 chi bins, full split, corrections as the Pilatus case."""
    g = GeometryParams(dist=0.15, poni1=2048 * 50e-6 / 2, poni2=2048 * 50e-6 / 2, rot1=0.05,
                       pixel1=50e-6, pixel2=50e-6, wavelength=1.0e-10)
    return Workload("cake-2048x2048-500x360-full", 2048, 2048, g, UNIT_2TH_DEG, SPLIT_FULL,
                    500, 360, image_dtype="float32", corrections=True, seed=seed)


BATCH_SHAPES = ((512, 1028, 75e-6), (1679, 1475, 172e-6), (2167, 2070, 75e-6))
BATCH_BINS = (500, 2000, 5000)


def batch_instances(n: int = 64, seed: int = 3, shapes=BATCH_SHAPES, bins=BATCH_BINS):
    """Heterogeneous instances: shape and bin count drawn from the three detector shapes and
    {500, 2000, 5000}; distance U(0.1, 0.5) m, rotations U(-0.05, 0.05) rad, PONI near the
    centre, q in nm^-1, full split, no mask."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        ny, nx, px = shapes[int(rng.integers(len(shapes)))]
        npt = int(bins[int(rng.integers(len(bins)))])
        off = rng.uniform(-2e-3, 2e-3, size=2)
        rot = rng.uniform(-0.05, 0.05, size=3)
        g = GeometryParams(dist=float(rng.uniform(0.1, 0.5)), poni1=ny * px / 2 + off[0],
                           poni2=nx * px / 2 + off[1], rot1=rot[0], rot2=rot[1], rot3=rot[2],
                           pixel1=px, pixel2=px, wavelength=1.0e-10)
        out.append(Workload("batch-%d-%dx%d-%d" % (k, ny, nx, npt), ny, nx, g, UNIT_Q_NM,
                            SPLIT_FULL, npt, image_dtype="uint32", seed=seed * 1000 + k))
    return out


def stream_workload() -> Workload:
    """One shared geometry for the multi-frame stream: 2167 x 2070 uint32, 75 um, 200 mm,
    centred, 2000 q bins, full split."""
    ny, nx, px = 2167, 2070, 75e-6
    g = GeometryParams(dist=0.2, poni1=ny * px / 2, poni2=nx * px / 2, pixel1=px, pixel2=px,
                       wavelength=1.0e-10)
    return Workload("stream-2167x2070-q-full-2000", ny, nx, g, UNIT_Q_NM, SPLIT_FULL, 2000,
                    image_dtype="uint32", seed=0)


def differentiation_workload() -> Workload:
    return pilatus_workload(seed=1)


# --------------------------------------------------------------------------------------
# masks, corrections and images
# --------------------------------------------------------------------------------------

def pilatus_module_mask(ny: int = 2527, nx: int = 2463, mod_rows: int = 195,
                        mod_cols: int = 487, gap_rows: int = 17, gap_cols: int = 7):
    """uint8 mask (1 = masked) of the inter-module gaps of a modular detector."""
    rows = (np.arange(ny) % (mod_rows + gap_rows)) >= mod_rows
    cols = (np.arange(nx) % (mod_cols + gap_cols)) >= mod_cols
    return (rows[:, None] | cols[None, :]).astype(np.uint8)


def dark_flat(ny: int, nx: int, seed: int):
    """dark ~ N(10, 1), flat ~ U(0.95, 1.05), both float32."""
    rng = np.random.default_rng(seed + 7919)
    dark = rng.normal(10.0, 1.0, size=(ny, nx)).astype(np.float32)
    flat = rng.uniform(0.95, 1.05, size=(ny, nx)).astype(np.float32)
    return dark, flat


def tiny_image(tth_deg_centre: np.ndarray, seed: int = 0) -> np.ndarray:
    """Poisson(100 + sum_k 500 exp(-(2theta - theta_k)^2 / (2 * 0.05^2))),
    theta_k = 5, 10, 15, 20, 25 degrees, as float32."""
    rng = np.random.default_rng(seed)
    lam = np.full(tth_deg_centre.shape, 100.0)
    for tk in (5.0, 10.0, 15.0, 20.0, 25.0):
        lam += 500.0 * np.exp(-(tth_deg_centre - tk) ** 2 / (2 * 0.05 ** 2))
    return rng.poisson(lam).astype(np.float32)


def ring_image(radial_centre: np.ndarray, seed: int, n_rings: int = 20, amplitude: float = 2000.0,
               sigma: float = 0.05, background: float = 1000.0, dtype=np.uint32,
               chi_deg_centre: np.ndarray | None = None, modulation: float = 0.0,
               floor: float = 0.05):
    """Poisson(background / x + sum_k A exp(-(x - x_k)^2 / (2 sigma^2))) on the radial value
    x of each pixel centre, x_k evenly spaced in (0.1 x_max, 0.9 x_max); optionally times
    (1 + modulation cos 2chi).  x is floored at `floor` to keep the 1/x background finite."""
    rng = np.random.default_rng(seed)
    x = np.maximum(radial_centre, floor)
    xmax = float(radial_centre.max())
    lam = background / x
    for xk in np.linspace(0.1 * xmax, 0.9 * xmax, n_rings):
        lam = lam + amplitude * np.exp(-(x - xk) ** 2 / (2 * sigma ** 2))
    if chi_deg_centre is not None and modulation:
        lam = lam * (1.0 + modulation * np.cos(np.deg2rad(2.0 * chi_deg_centre)))
    return rng.poisson(lam).astype(dtype)


def uniform_image(ny, nx, seed, lo=0.0, hi=1000.0, dtype=np.float32):
    rng = np.random.default_rng(seed)
    if np.dtype(dtype).kind in "ui":
        return rng.integers(int(lo), int(hi), size=(ny, nx)).astype(dtype)
    return rng.uniform(lo, hi, size=(ny, nx)).astype(dtype)


def random_geometry(rng: np.random.Generator, ny: int, nx: int, pixel: float = 100e-6,
                    tilt: float = 0.05, dist=(0.05, 0.5)):
    """A random PONI geometry whose beam centre lies somewhere on or near the detector."""
    return GeometryParams(dist=float(rng.uniform(*dist)),
                          poni1=float(rng.uniform(-0.2, 1.2) * ny * pixel),
                          poni2=float(rng.uniform(-0.2, 1.2) * nx * pixel),
                          rot1=float(rng.uniform(-tilt, tilt)), rot2=float(rng.uniform(-tilt, tilt)),
                          rot3=float(rng.uniform(-np.pi, np.pi)), pixel1=pixel, pixel2=pixel,
                          wavelength=float(rng.uniform(0.5e-10, 1.5e-10)))
