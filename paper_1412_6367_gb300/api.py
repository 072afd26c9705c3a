"""Python binding of the azint C ABI (argument marshalling only).

Every computation runs in the CUDA kernels of libazint.so; PyTorch provides device memory
and streams.  Device arrays are torch tensors on a CUDA device, C-contiguous; the current
torch stream of that device is passed to every call.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from ._lib import AzError, check  # noqa: F401  (re-exported)

UNITS = {"2th_deg": L.UNIT_2TH_DEG, "q_nm^-1": L.UNIT_Q_NM, "r_mm": L.UNIT_R_MM}
SPLITS = {"none": L.SPLIT_NONE, "bbox": L.SPLIT_BBOX, "full": L.SPLIT_FULL}
PRECISIONS = {"fp64": L.PREC_FP64, "fp32": L.PREC_FP32_COMP}
_DTYPES = {torch.float32: L.DTYPE_F32, torch.int32: L.DTYPE_I32}
if hasattr(torch, "uint32"):
    _DTYPES[torch.uint32] = L.DTYPE_U32


def _code(table, value, what):
    if isinstance(value, str):
        if value not in table:
            raise ValueError("unknown %s %r (choose from %s)" % (what, value, sorted(table)))
        return table[value]
    return int(value)


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev(t, name, dtype=None, numel=None):
    """Device pointer of a CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be C-contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (name, numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def image_dtype_code(t: torch.Tensor) -> int:
    """AZ_DTYPE_* of an image tensor: float32, int32, or 4-byte unsigned counts."""
    if t.dtype in _DTYPES:
        return _DTYPES[t.dtype]
    raise TypeError("image dtype %s not supported (float32, int32 or uint32)" % t.dtype)


class Geometry:
    """PONI geometry (Sec. 3); see az_geometry_create."""

    def __init__(self, dist, poni1, poni2, rot1=0.0, rot2=0.0, rot3=0.0, pixel1=100e-6,
                 pixel2=100e-6, wavelength=1.0e-10):
        self._lib = L.load()
        h = ctypes.c_void_p()
        check(self._lib.az_geometry_create(dist, poni1, poni2, rot1, rot2, rot3, pixel1, pixel2,
                                           wavelength, ctypes.byref(h)))
        self._h = h
        self.params = (dist, poni1, poni2, rot1, rot2, rot3, pixel1, pixel2, wavelength)

    @classmethod
    def from_params(cls, p):
        return cls(*p.astuple()) if hasattr(p, "astuple") else cls(*p)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.az_geometry_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def rotation(self) -> np.ndarray:
        R = np.zeros(9)
        check(self._lib.az_geometry_rotation(self._h, ctypes.c_void_p(R.ctypes.data)))
        return R.reshape(3, 3)

    def positions(self, ny, nx, unit="2th_deg", where="corners", chi=True, device="cuda"):
        corners = where == "corners"
        shape = (ny + 1, nx + 1) if corners else (ny, nx)
        rad = torch.empty(shape, dtype=torch.float64, device=device)
        ch = torch.empty(shape, dtype=torch.float64, device=device) if chi else None
        check(self._lib.az_geometry_positions(
            self._h, ny, nx, _code(UNITS, unit, "unit"),
            L.WHERE_CORNERS if corners else L.WHERE_CENTRES, _dev(rad, "rad"), _dev(ch, "chi"),
            _stream(rad.device)))
        return rad, ch

    def solid_angle(self, ny, nx, device="cuda"):
        out = torch.empty((ny, nx), dtype=torch.float32, device=device)
        check(self._lib.az_geometry_solid_angle(self._h, ny, nx, _dev(out, "out"),
                                                _stream(out.device)))
        return out

    def polarization(self, ny, nx, factor, device="cuda"):
        out = torch.empty((ny, nx), dtype=torch.float32, device=device)
        check(self._lib.az_geometry_polarization(self._h, ny, nx, float(factor), _dev(out, "out"),
                                                 _stream(out.device)))
        return out


@dataclass
class Result:
    I: torch.Tensor
    sum_signal: torch.Tensor
    sum_norm: torch.Tensor
    count: torch.Tensor

    def __iter__(self):
        return iter((self.I, self.sum_signal, self.sum_norm, self.count))


class Integrator:
    """A built bins x pixels matrix and the kernels that apply it (az_csr_build)."""

    def __init__(self, handle, device):
        self._lib = L.load()
        self._h = handle
        self.device = torch.device(device)
        self.info = self._info()

    @classmethod
    def build(cls, geometry: Geometry, shape, npt_rad, npt_azim=0, unit="2th_deg", split="bbox",
              mask=None, device="cuda"):
        ny, nx = shape
        lib = L.load()
        h = ctypes.c_void_p()
        m = None
        if mask is not None:
            m = torch.as_tensor(mask, device=device).to(torch.uint8).contiguous()
        check(lib.az_csr_build(geometry.handle, ny, nx, npt_rad, npt_azim,
                               _code(UNITS, unit, "unit"), _code(SPLITS, split, "split"),
                               _dev(m, "mask", torch.uint8, ny * nx), _stream(device),
                               ctypes.byref(h)))
        return cls(h, device)

    @classmethod
    def from_csr(cls, shape, indptr, indices, data, npt_rad, npt_azim=0, lo=0.0, hi=1.0,
                 unit="2th_deg", split="full", device="cuda"):
        """Import a host CSR matrix (scipy layout: indptr, indices, data) of nrows = npt_rad
        (1D) or npt_azim * npt_rad rows over ny * nx pixels (az_csr_import); lo, hi is the
        radial range of the bins."""
        ny, nx = shape
        lib = L.load()
        ip = np.ascontiguousarray(indptr, dtype=np.int32)
        ix = np.ascontiguousarray(indices, dtype=np.int32)
        dv = np.ascontiguousarray(data, dtype=np.float64)
        h = ctypes.c_void_p()
        check(lib.az_csr_import(ny, nx, npt_rad, npt_azim, _code(UNITS, unit, "unit"),
                                _code(SPLITS, split, "split"), ctypes.c_void_p(ip.ctypes.data),
                                ctypes.c_void_p(ix.ctypes.data), ctypes.c_void_p(dv.ctypes.data),
                                float(lo), float(hi), _stream(device), ctypes.byref(h)))
        return cls(h, device)

    @classmethod
    def from_positions(cls, shape, rad, chi, npt_rad, npt_azim=0, split="bbox", mask=None):
        """Build from FP64 positions (device tensors): centres for split 'none', corners
        otherwise (az_csr_build_from_positions)."""
        ny, nx = shape
        lib = L.load()
        device = rad.device
        h = ctypes.c_void_p()
        m = None
        if mask is not None:
            m = torch.as_tensor(mask, device=device).to(torch.uint8).contiguous()
        check(lib.az_csr_build_from_positions(
            ny, nx, _dev(rad, "rad", torch.float64), _dev(chi, "chi", torch.float64),
            npt_rad, npt_azim, _code(SPLITS, split, "split"),
            _dev(m, "mask", torch.uint8, ny * nx), _stream(device), ctypes.byref(h)))
        return cls(h, device)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.az_integrator_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def _info(self):
        info = L.Info()
        check(self._lib.az_integrator_info(self._h, ctypes.byref(info)))
        return {name: getattr(info, name) for name, _ in L.Info._fields_}

    def refresh_info(self):
        self.info = self._info()
        return self.info

    @property
    def nrows(self):
        return self.info["nrows"]

    @property
    def shape(self):
        return (self.info["ny"], self.info["nx"])

    def export_csr(self):
        """(indptr int32, indices int32, data float64) numpy arrays (scipy-compatible)."""
        nnz, nrows = self.info["nnz"], self.info["nrows"]
        indptr = np.empty(nrows + 1, np.int32)
        indices = np.empty(nnz, np.int32)
        data = np.empty(nnz, np.float64)
        check(self._lib.az_csr_export(self._h, ctypes.c_void_p(indptr.ctypes.data),
                                      ctypes.c_void_p(indices.ctypes.data),
                                      ctypes.c_void_p(data.ctypes.data)))
        return indptr, indices, data

    def radial_axis(self):
        out = np.empty(self.info["npt_rad"])
        check(self._lib.az_radial_axis(self._h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def status(self):
        return check(self._lib.az_integrator_status(self._h))

    def _corr(self, dark, flat, solid_angle, polarization):
        n = self.info["ny"] * self.info["nx"]
        return [_dev(a, name, torch.float32, n) for a, name in
                ((dark, "dark"), (flat, "flat"), (solid_angle, "solid_angle"),
                 (polarization, "polarization"))]

    def integrate(self, image, dark=None, flat=None, solid_angle=None, polarization=None,
                  precision="fp32", out=None) -> Result:
        """One frame (az_integrate1d / az_integrate2d); returns (I, S, N, C)."""
        prec = _code(PRECISIONS, precision, "precision")
        npix = self.info["ny"] * self.info["nx"]
        img = _dev(image, "image", numel=npix)
        dt = torch.float64 if prec == L.PREC_FP64 else torch.float32
        if out is None:
            out = Result(*(torch.empty(self.nrows, dtype=dt, device=image.device) for _ in range(4)))
        fn = self._lib.az_integrate2d if self.info["npt_azim"] else self._lib.az_integrate1d
        check(fn(self._h, img, image_dtype_code(image), *self._corr(dark, flat, solid_angle, polarization),
                 prec, _dev(out.I, "I", dt), _dev(out.sum_signal, "S", dt),
                 _dev(out.sum_norm, "N", dt), _dev(out.count, "C", dt), _stream(image.device)))
        if self.info["npt_azim"]:
            shp = (self.info["npt_azim"], self.info["npt_rad"])
            out = Result(*(t.view(shp) for t in out))
        return out

    def integrate_noalloc(self, image, dark=None, flat=None, solid_angle=None, polarization=None,
                          precision="fp32", out=None) -> Result:
        """One frame like integrate(), through az_integrate_noalloc: the call allocates no
        device memory itself (its partial sums use a fixed array inside the library).  Pass
        preallocated `out` tensors to keep the whole call free of allocation."""
        prec = _code(PRECISIONS, precision, "precision")
        npix = self.info["ny"] * self.info["nx"]
        img = _dev(image, "image", numel=npix)
        dt = torch.float64 if prec == L.PREC_FP64 else torch.float32
        if out is None:
            out = Result(*(torch.empty(self.nrows, dtype=dt, device=image.device) for _ in range(4)))
        check(self._lib.az_integrate_noalloc(
            self._h, img, image_dtype_code(image), *self._corr(dark, flat, solid_angle, polarization),
            prec, _dev(out.I, "I", dt), _dev(out.sum_signal, "S", dt),
            _dev(out.sum_norm, "N", dt), _dev(out.count, "C", dt), _stream(image.device)))
        if self.info["npt_azim"]:
            shp = (self.info["npt_azim"], self.info["npt_rad"])
            out = Result(*(t.view(shp) for t in out))
        return out

    def integrate_batch(self, frames, dark=None, flat=None, solid_angle=None, polarization=None,
                        out=None):
        """Many frames [n, ny, nx] through the matrix (az_integrate_batch, FP32 compensated).
        Returns (I [n, nrows], S [n, nrows], N [nrows], C [nrows])."""
        n = frames.shape[0]
        npix = self.info["ny"] * self.info["nx"]
        fr = _dev(frames, "frames", numel=n * npix)
        dev = frames.device
        if out is None:
            out = Result(torch.empty((n, self.nrows), dtype=torch.float32, device=dev),
                         torch.empty((n, self.nrows), dtype=torch.float32, device=dev),
                         torch.empty(self.nrows, dtype=torch.float32, device=dev),
                         torch.empty(self.nrows, dtype=torch.float32, device=dev))
        check(self._lib.az_integrate_batch(
            self._h, fr, n, image_dtype_code(frames), *self._corr(dark, flat, solid_angle, polarization),
            _dev(out.I, "I", torch.float32), _dev(out.sum_signal, "S", torch.float32),
            _dev(out.sum_norm, "N", torch.float32), _dev(out.count, "C", torch.float32),
            _stream(dev)))
        return out

    def set_corrections(self, dark=None, flat=None, solid_angle=None, polarization=None):
        """Bind the correction arrays once (az_set_corrections): per-entry darks, N and C are
        formed now and reused by integrate_batch_bound."""
        dev = next((t.device for t in (dark, flat, solid_angle, polarization) if t is not None),
                   self.device)
        check(self._lib.az_set_corrections(self._h, *self._corr(dark, flat, solid_angle, polarization),
                                           _stream(dev)))

    def integrate_batch_bound(self, frames, out=None):
        """Frames [n, ny, nx] through the corrections bound by set_corrections
        (az_integrate_batch_bound).  Returns (I [n, nrows], S [n, nrows], N [nrows], C [nrows])."""
        n = frames.shape[0]
        npix = self.info["ny"] * self.info["nx"]
        fr = _dev(frames, "frames", numel=n * npix)
        dev = frames.device
        if out is None:
            out = Result(torch.empty((n, self.nrows), dtype=torch.float32, device=dev),
                         torch.empty((n, self.nrows), dtype=torch.float32, device=dev),
                         torch.empty(self.nrows, dtype=torch.float32, device=dev),
                         torch.empty(self.nrows, dtype=torch.float32, device=dev))
        check(self._lib.az_integrate_batch_bound(
            self._h, fr, n, image_dtype_code(frames), _dev(out.I, "I", torch.float32),
            _dev(out.sum_signal, "S", torch.float32), _dev(out.sum_norm, "N", torch.float32),
            _dev(out.count, "C", torch.float32), _stream(dev)))
        return out

    def integrate_pixelnorm(self, frames, dark=None, flat=None, solid_angle=None, polarization=None):
        """The paper's per-pixel-corrected form (az_integrate_batch_pixelnorm) for frames
        [n, ny, nx] or one frame [ny, nx]: returns (I, U, C) with U = sum w (img - dark) /
        (flat solid_angle polarization), C = sum w, I = U / C."""
        one = frames.dim() == 2
        fr = frames.unsqueeze(0) if one else frames
        n = fr.shape[0]
        npix = self.info["ny"] * self.info["nx"]
        dev = fr.device
        I = torch.empty((n, self.nrows), dtype=torch.float32, device=dev)
        U = torch.empty((n, self.nrows), dtype=torch.float32, device=dev)
        C = torch.empty(self.nrows, dtype=torch.float32, device=dev)
        check(self._lib.az_integrate_batch_pixelnorm(
            self._h, _dev(fr, "frames", numel=n * npix), n, image_dtype_code(fr),
            *self._corr(dark, flat, solid_angle, polarization), _dev(I, "I", torch.float32),
            _dev(U, "U", torch.float32), _dev(C, "C", torch.float32), _stream(dev)))
        if one:
            I, U = I[0], U[0]
        return I, U, C

    def variance(self, frames, out=None):
        """Propagated Poisson variance of the bin sums, sum w^2 max(img, 0), of frames
        [n, ny, nx] or of one frame [ny, nx] (az_integrate_variance, FP32 compensated).
        Returns [n, nrows] (or [nrows] for one frame)."""
        one = frames.dim() == 2
        fr = frames.unsqueeze(0) if one else frames
        n = fr.shape[0]
        npix = self.info["ny"] * self.info["nx"]
        if out is None:
            out = torch.empty((n, self.nrows), dtype=torch.float32, device=fr.device)
        check(self._lib.az_integrate_variance(self._h, _dev(fr, "frames", numel=n * npix), n,
                                              image_dtype_code(fr), _dev(out, "out", torch.float32),
                                              _stream(fr.device)))
        return out[0] if one else out

    def integrate_batch_host(self, frames: torch.Tensor, dark=None, flat=None, solid_angle=None,
                             polarization=None, out_I=None, out_S=None):
        """End-to-end form on host buffers (az_integrate_batch_host): frames is a CPU tensor
        [n, ny, nx] (pinned for overlapped copies); returns host (I, S) [n, nrows]."""
        if frames.is_cuda:
            raise TypeError("frames must be a host tensor")
        n = frames.shape[0]
        frames = frames.contiguous()
        if out_I is None:
            out_I = torch.empty((n, self.nrows), dtype=torch.float32, pin_memory=frames.is_pinned())
        if out_S is None:
            out_S = torch.empty((n, self.nrows), dtype=torch.float32, pin_memory=frames.is_pinned())
        check(self._lib.az_integrate_batch_host(
            self._h, ctypes.c_void_p(frames.data_ptr()), n, image_dtype_code(frames),
            *self._corr(dark, flat, solid_angle, polarization),
            ctypes.c_void_p(out_I.data_ptr()), ctypes.c_void_p(out_S.data_ptr()),
            _stream(self.device)))
        return out_I, out_S

    def backward(self, grad_I, I, sum_norm, solid_angle=None, polarization=None,
                 precision="fp32", want_image=True, want_flat=True):
        """(dL/dimage, dL/dflat) for upstream gradient grad_I (az_integrate_backward)."""
        prec = _code(PRECISIONS, precision, "precision")
        dt = torch.float64 if prec == L.PREC_FP64 else torch.float32
        ny, nx = self.shape
        dev = grad_I.device
        gi = torch.empty((ny, nx), dtype=dt, device=dev) if want_image else None
        gf = torch.empty((ny, nx), dtype=dt, device=dev) if want_flat else None
        n = self.nrows
        check(self._lib.az_integrate_backward(
            self._h, _dev(grad_I.contiguous(), "grad_I", dt, n), _dev(I.contiguous(), "I", dt, n),
            _dev(sum_norm.contiguous(), "sum_norm", dt, n),
            _dev(solid_angle, "solid_angle", torch.float32, ny * nx),
            _dev(polarization, "polarization", torch.float32, ny * nx), prec,
            _dev(gi, "grad_image"), _dev(gf, "grad_flat"), _stream(dev)))
        return gi, gf

    def profile_enable(self, enable=True):
        check(self._lib.az_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        """{kind: (launches, total_ms)} since the last read (synchronises)."""
        p = L.Profile()
        check(self._lib.az_profile_read(self._h, ctypes.byref(p)))
        return {k: (int(p.launches[i]), float(p.total_ms[i])) for i, k in enumerate(L.PROFILE_KINDS)}

    def autotune(self, n_trial_frames=32):
        best = ctypes.c_double(0.0)
        check(self._lib.az_autotune(self._h, n_trial_frames, _stream(self.device), ctypes.byref(best)))
        self.refresh_info()
        return best.value

    def set_copy_engine(self, engine):
        """"tma" (one bulk copy per tile row) or "async" (16-byte cp.async copies)."""
        code = {"tma": 0, "async": 1}[engine] if isinstance(engine, str) else int(engine)
        check(self._lib.az_set_copy_engine(self._h, code))
        self.refresh_info()

    def set_tuning(self, tile_h=0, tile_w=0, rows_per_warp=0, frames_per_pass=0):
        check(self._lib.az_set_tuning(self._h, tile_h, tile_w, rows_per_warp, frames_per_pass))
        self.refresh_info()

    # ---- look-up-table layout (Sec. 5.2) ----
    def lut_build(self, precision="fp32"):
        """Build the look-up table of `precision` (az_lut_build); returns its width."""
        check(self._lib.az_lut_build(self._h, _code(PRECISIONS, precision, "precision"),
                                     _stream(self.device)))
        self.refresh_info()
        return self.info["lut_width"]

    def lut_export(self, precision="fp32"):
        """(pixel int32, coefficient) numpy arrays [nrows][width] of the table built for
        `precision` (float32 or float64 coefficients), padding (-1, 0) included."""
        width = ctypes.c_int64(0)
        check(self._lib.az_lut_export(self._h, ctypes.byref(width), None, None, None))
        shape = (self.nrows, width.value)
        pix = np.empty(shape, np.int32)
        fp64 = _code(PRECISIONS, precision, "precision") == L.PREC_FP64
        coef = np.empty(shape, np.float64 if fp64 else np.float32)
        c = ctypes.c_void_p(coef.ctypes.data)
        check(self._lib.az_lut_export(self._h, None, ctypes.c_void_p(pix.ctypes.data),
                                      None if fp64 else c, c if fp64 else None))
        return pix, coef

    def integrate_lut(self, image, dark=None, flat=None, solid_angle=None, polarization=None,
                      precision="fp32", out=None) -> Result:
        """One frame through the look-up table (az_integrate_lut); returns (I, S, N, C)
        shaped as integrate() returns them."""
        prec = _code(PRECISIONS, precision, "precision")
        npix = self.info["ny"] * self.info["nx"]
        img = _dev(image, "image", numel=npix)
        dt = torch.float64 if prec == L.PREC_FP64 else torch.float32
        if out is None:
            out = Result(*(torch.empty(self.nrows, dtype=dt, device=image.device) for _ in range(4)))
        check(self._lib.az_integrate_lut(
            self._h, img, image_dtype_code(image), *self._corr(dark, flat, solid_angle, polarization),
            prec, _dev(out.I, "I", dt), _dev(out.sum_signal, "S", dt),
            _dev(out.sum_norm, "N", dt), _dev(out.count, "C", dt), _stream(image.device)))
        if self.info["npt_azim"]:
            shp = (self.info["npt_azim"], self.info["npt_rad"])
            out = Result(*(t.view(shp) for t in out))
        return out

    def set_layout(self, layout):
        """The single-frame layout of integrate(): "tiled" or "lut" (az_set_layout)."""
        code = {"tiled": 0, "lut": 1}[layout] if isinstance(layout, str) else int(layout)
        check(self._lib.az_set_layout(self._h, code))
        self.refresh_info()


def selftest_wait(arrive=False, limit_cycles=2_000_000, device=None):
    """Run the bounded-wait self-test (az_selftest_wait) on the current CUDA device; returns
    the status the kernel wrote: 0 (AZ_OK) or -7 (AZ_ETIMEOUT)."""
    lib = L.load()
    st = ctypes.c_int(1)
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    check(lib.az_selftest_wait(1 if arrive else 0, int(limit_cycles), ctypes.byref(st), _stream(dev)))
    return st.value


class MultiPlan:
    """Several integrators of uneven shape in one persistent launch (az_multi_create)."""

    def __init__(self, integrators, images, darks=None, flats=None, solid_angles=None,
                 polarizations=None):
        self._lib = L.load()
        n = len(integrators)
        self.integrators = list(integrators)
        self.images = list(images)
        dev = images[0].device
        self.outputs = [Result(*(torch.empty(ig.nrows, dtype=torch.float32, device=dev)
                                 for _ in range(4))) for ig in integrators]

        def arr(items, name, dtype=None):
            if items is None:
                return None
            a = (ctypes.c_void_p * n)()
            for k, t in enumerate(items):
                p = _dev(t, name, dtype)
                a[k] = p.value if p is not None else None
            return ctypes.cast(a, L.PP), a

        dtc = image_dtype_code(images[0])
        keep = []
        ptrs = []
        for items, name, dtype in ((integrators, "h", None), (images, "image", None),
                                   (darks, "dark", torch.float32), (flats, "flat", torch.float32),
                                   (solid_angles, "sa", torch.float32),
                                   (polarizations, "pol", torch.float32)):
            if name == "h":
                a = (ctypes.c_void_p * n)(*[ig.handle.value for ig in integrators])
                keep.append(a)
                ptrs.append(ctypes.cast(a, L.PP))
                continue
            r = arr(items, name, dtype)
            if r is None:
                ptrs.append(None)
            else:
                ptrs.append(r[0])
                keep.append(r[1])
        outs = []
        for k in range(4):
            a = (ctypes.c_void_p * n)(*[o.__dict__[f].data_ptr() for o in self.outputs
                                        for f in [("I", "sum_signal", "sum_norm", "count")[k]]])
            keep.append(a)
            outs.append(ctypes.cast(a, L.PP))
        h = ctypes.c_void_p()
        check(self._lib.az_multi_create(ptrs[0], n, ptrs[1], dtc, ptrs[2], ptrs[3], ptrs[4],
                                        ptrs[5], *outs, ctypes.byref(h)))
        self._keep = keep
        self._inputs = (darks, flats, solid_angles, polarizations)
        self._h = h

    def launch(self, use_graph=False):
        check(self._lib.az_multi_launch(self._h, 1 if use_graph else 0,
                                        _stream(self.images[0].device)))
        return self.outputs

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.az_multi_destroy(h)
            self._h = None
