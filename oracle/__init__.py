"""Azimuthal-integration ORACLE -- test infrastructure, not product code.

A plain, slow, double-precision CPU statement of the method of Kieffer & Ashiotis,
"PyFAI: a Python library for high performance azimuthal integration on GPU" (EuroSciPy
2014).  The arithmetic lives in ``azint_oracle.c`` (plain C, compiled without FMA
contraction); this module only builds it with gcc, loads it with ctypes and converts
NumPy arrays.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline arm of
``bench.py`` may import it.  It shares no code with the CUDA package and never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

UNIT_2TH_DEG, UNIT_Q_NM, UNIT_R_MM = 0, 1, 2
SPLIT_NONE, SPLIT_BBOX, SPLIT_FULL = 0, 1, 2
UNITS = {"2th_deg": UNIT_2TH_DEG, "q_nm^-1": UNIT_Q_NM, "r_mm": UNIT_R_MM}
SPLITS = {"none": SPLIT_NONE, "bbox": SPLIT_BBOX, "full": SPLIT_FULL}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "azint_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_OMP_SRC = os.path.join(_HERE, "azint_omp.c")
_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None


def _compile(src, path, force, extra=()):
    if not force and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(src):
        return path
    tmp = path + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", *extra, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, no FMA contraction) and the multi-core CPU baseline
    (the same, with OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    _compile(_OMP_SRC, _OMP_PATH, force, ("-fopenmp",))
    return _compile(_SRC, _LIB_PATH, force)


class _Geom(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("dist", "poni1", "poni2", "rot1", "rot2", "rot3", "pixel1", "pixel2",
                 "wavelength")]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        G = ctypes.POINTER(_Geom)
        vp = ctypes.c_void_p
        lib.orc_rotation.argtypes = [ctypes.c_double] * 3 + [D]
        lib.orc_position_at.argtypes = [G, ctypes.c_int, ctypes.c_double, ctypes.c_double, D, D]
        for name in ("orc_corner_positions", "orc_centre_positions"):
            getattr(lib, name).argtypes = [G, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
        lib.orc_solid_angle.argtypes = [G, ctypes.c_int, ctypes.c_int, vp]
        lib.orc_polarization.argtypes = [G, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp]
        lib.orc_csr_build.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.orc_csr_build.restype = vp
        lib.orc_csr_free.argtypes = [vp]
        lib.orc_csr_nnz.argtypes = [vp]
        lib.orc_csr_nnz.restype = ctypes.c_int64
        lib.orc_csr_nrows.argtypes = [vp]
        lib.orc_csr_range.argtypes = [vp, D]
        lib.orc_csr_copy.argtypes = [vp, vp, vp, vp]
        lib.orc_integrate.argtypes = [ctypes.c_int] + [vp] * 12
        lib.orc_backward.argtypes = [ctypes.c_int, ctypes.c_int64] + [vp] * 10
        lib.orc_variance.argtypes = [ctypes.c_int] + [vp] * 5
        lib.orc_integrate_pixelnorm.argtypes = [ctypes.c_int] + [vp] * 11
        lib.orc_lut_width.argtypes = [ctypes.c_int, vp]
        lib.orc_lut_width.restype = ctypes.c_int64
        lib.orc_lut_from_csr.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.c_int64, vp, vp]
        lib.orc_integrate_lut.argtypes = [ctypes.c_int, ctypes.c_int64] + [vp] * 11
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


@dataclass(frozen=True)
class Geometry:
    """PONI-style detector geometry: distances and pixel sizes in metres, angles in rad."""
    dist: float
    poni1: float
    poni2: float
    rot1: float = 0.0
    rot2: float = 0.0
    rot3: float = 0.0
    pixel1: float = 100e-6
    pixel2: float = 100e-6
    wavelength: float = 1.0e-10

    def _c(self):
        return _Geom(self.dist, self.poni1, self.poni2, self.rot1, self.rot2, self.rot3,
                     self.pixel1, self.pixel2, self.wavelength)


def rotation(rot1, rot2, rot3):
    R = np.zeros(9)
    _load().orc_rotation(rot1, rot2, rot3, R.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return R.reshape(3, 3)


def position_at(geom: Geometry, unit: int, d1: float, d2: float):
    r, c = ctypes.c_double(), ctypes.c_double()
    g = geom._c()
    _load().orc_position_at(ctypes.byref(g), unit, d1, d2, ctypes.byref(r), ctypes.byref(c))
    return r.value, c.value


def corner_positions(geom: Geometry, ny: int, nx: int, unit: int):
    rad = np.empty((ny + 1, nx + 1))
    chi = np.empty((ny + 1, nx + 1))
    g = geom._c()
    _load().orc_corner_positions(ctypes.byref(g), ny, nx, unit, _ptr(rad), _ptr(chi))
    return rad, chi


def centre_positions(geom: Geometry, ny: int, nx: int, unit: int):
    rad = np.empty((ny, nx))
    chi = np.empty((ny, nx))
    g = geom._c()
    _load().orc_centre_positions(ctypes.byref(g), ny, nx, unit, _ptr(rad), _ptr(chi))
    return rad, chi


def solid_angle(geom: Geometry, ny: int, nx: int):
    out = np.empty((ny, nx))
    g = geom._c()
    _load().orc_solid_angle(ctypes.byref(g), ny, nx, _ptr(out))
    return out


def polarization(geom: Geometry, ny: int, nx: int, factor: float):
    out = np.empty((ny, nx))
    g = geom._c()
    _load().orc_polarization(ctypes.byref(g), ny, nx, factor, _ptr(out))
    return out


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__("oracle error %d" % code)
        self.code = code


@dataclass
class Csr:
    """bins x pixels weight matrix in scipy-compatible CSR form (Sec. 5.2.1)."""
    indptr: np.ndarray   # int64 [nrows + 1]
    indices: np.ndarray  # int32 [nnz], ascending within a row
    data: np.ndarray     # float64 [nnz]
    nrows: int
    ny: int
    nx: int
    npt_rad: int
    npt_azim: int
    lo: float
    hi: float
    delta: float

    @property
    def nnz(self):
        return int(self.indices.shape[0])

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.data, self.indices, self.indptr),
                             shape=(self.nrows, self.ny * self.nx))


def csr_build(ny, nx, rad, chi, mask, npt_rad, npt_azim, split) -> Csr:
    """Build the weight matrix from positions: pixel-centre arrays (ny, nx) for split NONE,
    corner arrays (ny+1, nx+1) otherwise.  ``chi`` may be None for 1D NONE/BBOX."""
    lib = _load()
    rad = _f64(rad)
    chi = _f64(chi)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    err = ctypes.c_int(0)
    h = lib.orc_csr_build(ny, nx, _ptr(rad), _ptr(chi), _ptr(m), npt_rad, npt_azim, split,
                          ctypes.byref(err))
    if not h:
        raise OracleError(err.value)
    try:
        nnz = lib.orc_csr_nnz(h)
        nrows = lib.orc_csr_nrows(h)
        rng = np.zeros(3)
        lib.orc_csr_range(h, rng.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        indptr = np.empty(nrows + 1, np.int64)
        indices = np.empty(max(nnz, 1), np.int32)
        data = np.empty(max(nnz, 1), np.float64)
        lib.orc_csr_copy(h, _ptr(indptr), _ptr(indices), _ptr(data))
    finally:
        lib.orc_csr_free(h)
    return Csr(indptr, indices[:nnz], data[:nnz], nrows, ny, nx, npt_rad, npt_azim,
               float(rng[0]), float(rng[1]), float(rng[2]))


def positions_for(geom: Geometry, ny, nx, unit, split, npt_azim):
    """The position arrays the split mode reads: (rad, chi) at centres or corners."""
    if split == SPLIT_NONE:
        return centre_positions(geom, ny, nx, unit)
    return corner_positions(geom, ny, nx, unit)


def build_from_geometry(geom: Geometry, ny, nx, unit, split, npt_rad, npt_azim=0,
                        mask=None) -> Csr:
    rad, chi = positions_for(geom, ny, nx, unit, split, npt_azim)
    return csr_build(ny, nx, rad, chi, mask, npt_rad, npt_azim, split)


def _csr_arrays(A: Csr):
    return (np.ascontiguousarray(A.indptr, dtype=np.int64),
            np.ascontiguousarray(A.indices, dtype=np.int32),
            np.ascontiguousarray(A.data, dtype=np.float64))


def integrate(A: Csr, image, dark=None, flat=None, solid_angle=None, polarization=None):
    """(I, S, N, C) per bin in float64; inputs are promoted exactly to float64."""
    lib = _load()
    img = _f64(np.asarray(image).reshape(-1))
    dark, flat, sa, pol = (None if a is None else _f64(np.asarray(a).reshape(-1))
                           for a in (dark, flat, solid_angle, polarization))
    I, S, N, C = (np.empty(A.nrows) for _ in range(4))
    ip, ix, dt = _csr_arrays(A)
    lib.orc_integrate(A.nrows, _ptr(ip), _ptr(ix), _ptr(dt), _ptr(img), _ptr(dark), _ptr(flat),
                      _ptr(sa), _ptr(pol), _ptr(I), _ptr(S), _ptr(N), _ptr(C))
    return I, S, N, C


def backward(A: Csr, grad_I, I, N, solid_angle=None, polarization=None):
    """(dL/dimage, dL/dflat) per pixel in float64 for upstream gradient dL/dI."""
    lib = _load()
    g, I, N = (_f64(np.asarray(a).reshape(-1)) for a in (grad_I, I, N))
    sa, pol = (None if a is None else _f64(np.asarray(a).reshape(-1))
               for a in (solid_angle, polarization))
    npix = A.ny * A.nx
    gi = np.empty(npix)
    gf = np.empty(npix)
    ip, ix, dt = _csr_arrays(A)
    lib.orc_backward(A.nrows, npix, _ptr(ip), _ptr(ix), _ptr(dt), _ptr(g), _ptr(I), _ptr(N),
                     _ptr(sa), _ptr(pol), _ptr(gi), _ptr(gf))
    return gi, gf


def integrate_pixelnorm(A: Csr, image, dark=None, flat=None, solid_angle=None, polarization=None):
    """The paper's per-pixel-corrected form: (I, U, C) with U = sum w (img - dark) / (flat
    solid_angle polarisation), C = sum w, I = U / C; float64."""
    lib = _load()
    img = _f64(np.asarray(image).reshape(-1))
    dark, flat, sa, pol = (None if a is None else _f64(np.asarray(a).reshape(-1))
                           for a in (dark, flat, solid_angle, polarization))
    I, U, C = (np.empty(A.nrows) for _ in range(3))
    ip, ix, dt = _csr_arrays(A)
    lib.orc_integrate_pixelnorm(A.nrows, _ptr(ip), _ptr(ix), _ptr(dt), _ptr(img), _ptr(dark),
                                _ptr(flat), _ptr(sa), _ptr(pol), _ptr(I), _ptr(U), _ptr(C))
    return I, U, C


def variance(A: Csr, image):
    """Propagated Poisson variance of each bin's signal sum, sum_p w^2 max(img_p, 0), float64."""
    lib = _load()
    img = _f64(np.asarray(image).reshape(-1))
    V = np.empty(A.nrows)
    ip, ix, dt = _csr_arrays(A)
    lib.orc_variance(A.nrows, _ptr(ip), _ptr(ix), _ptr(dt), _ptr(img), _ptr(V))
    return V


def lut_from_csr_arrays(indptr, indices, data):
    """The look-up table (Sec. 5.2) of a CSR matrix given as arrays: (idx int32, coef
    float64), both [nrows][width], width = the longest row; each row holds its entries in
    column order, then padding pairs (-1, 0.0)."""
    lib = _load()
    ip = np.ascontiguousarray(indptr, dtype=np.int64)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    dt = np.ascontiguousarray(data, dtype=np.float64)
    nrows = len(ip) - 1
    width = int(lib.orc_lut_width(nrows, _ptr(ip)))
    idx = np.empty((nrows, width), np.int32)
    coef = np.empty((nrows, width), np.float64)
    lib.orc_lut_from_csr(nrows, _ptr(ip), _ptr(ix), _ptr(dt), width, _ptr(idx), _ptr(coef))
    return idx, coef


def lut_from_csr(A: Csr):
    """The look-up table of the oracle's matrix A (see lut_from_csr_arrays)."""
    return lut_from_csr_arrays(*_csr_arrays(A))


def integrate_lut(idx, coef, image, dark=None, flat=None, solid_angle=None, polarization=None):
    """(I, S, N, C) per bin in float64 through a look-up table [nrows][width]."""
    lib = _load()
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    nrows, width = idx.shape
    img = _f64(np.asarray(image).reshape(-1))
    dark, flat, sa, pol = (None if a is None else _f64(np.asarray(a).reshape(-1))
                           for a in (dark, flat, solid_angle, polarization))
    I, S, N, C = (np.empty(nrows) for _ in range(4))
    lib.orc_integrate_lut(nrows, width, _ptr(idx), _ptr(coef), _ptr(img), _ptr(dark), _ptr(flat),
                          _ptr(sa), _ptr(pol), _ptr(I), _ptr(S), _ptr(N), _ptr(C))
    return I, S, N, C


def radial_axis(A: Csr):
    """Bin centres lo + (k + 1/2) delta of the radial axis."""
    return A.lo + (np.arange(A.npt_rad) + 0.5) * A.delta


# ---- multi-core CPU baseline (azint_omp.c) ---------------------------------------------
_omp = None


def _load_omp():
    global _omp
    with _lock:
        if _omp is not None:
            return _omp
        build()
        lib = ctypes.CDLL(_OMP_PATH)
        vp = ctypes.c_void_p
        lib.omp_threads.restype = ctypes.c_int
        lib.omp_integrate.argtypes = [ctypes.c_int, ctypes.c_int64] + [vp] * 12
        lib.omp_integrate.restype = ctypes.c_int
        _omp = lib
        return lib


@dataclass
class Csc:
    """The weight matrix pixel-major (column pointers, row indices, weights)."""
    colptr: np.ndarray  # int64 [npix + 1]
    rows: np.ndarray    # int32 [nnz]
    data: np.ndarray    # float64 [nnz]
    nrows: int
    npix: int


def csc_of(A: Csr) -> Csc:
    """The oracle's matrix A regrouped by pixel (scipy.sparse's CSR -> CSC conversion)."""
    M = A.scipy().tocsc()
    M.sort_indices()
    return Csc(np.ascontiguousarray(M.indptr, dtype=np.int64), np.ascontiguousarray(M.indices, dtype=np.int32),
               np.ascontiguousarray(M.data, dtype=np.float64), A.nrows, A.ny * A.nx)


def omp_threads() -> int:
    return int(_load_omp().omp_threads())


def omp_integrate(M: Csc, image_u32, dark=None, flat=None, solid_angle=None, polarization=None):
    """(I, S, N, C, threads) of the multi-core CPU baseline: the paper's per-thread histograms
    over the pixels (Sec. 3.4.1) in FP64.  image: uint32 [npix]; corrections float32 or None."""
    lib = _load_omp()
    img = np.ascontiguousarray(np.asarray(image_u32).reshape(-1), dtype=np.uint32)
    cs = [None if a is None else np.ascontiguousarray(np.asarray(a).reshape(-1), dtype=np.float32)
          for a in (dark, flat, solid_angle, polarization)]
    I, S, N, C = (np.empty(M.nrows) for _ in range(4))
    used = lib.omp_integrate(M.nrows, M.npix, _ptr(M.colptr), _ptr(M.rows), _ptr(M.data), _ptr(img),
                             *[_ptr(a) for a in cs], _ptr(I), _ptr(S), _ptr(N), _ptr(C))
    if used < 0:
        raise MemoryError("per-thread histograms")
    return I, S, N, C, used
