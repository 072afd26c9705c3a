"""Shared helpers for the GPU parity tests: build the same workload for the CUDA path and
the oracle from the same seeded inputs."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1412_6367_gb300 import synth

needs_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")
SPLIT_NAMES = {0: "none", 1: "bbox", 2: "full"}
UNIT_NAMES = {0: "2th_deg", 1: "q_nm^-1", 2: "r_mm"}


def api():
    from paper_1412_6367_gb300 import api as A
    return A


def to_dev(a, pinned=False):
    """numpy -> torch (CUDA, or pinned host); uint32 data moves as int32 and is viewed back
    as uint32 (torch's uint32 support is limited to same-size views)."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        t = torch.from_numpy(a.view(np.int32))
        t = t.pin_memory() if pinned else t.cuda()
        return t.view(torch.uint32)
    t = torch.from_numpy(a)
    return t.pin_memory() if pinned else t.cuda()


def oracle_geometry(p: synth.GeometryParams):
    return O.Geometry(*p.astuple())


def gpu_geometry(p: synth.GeometryParams):
    return api().Geometry(*p.astuple())


def rel_err(got, ref, floor_frac=1e-3):
    """max |got - ref| / |ref| over entries with |ref| > floor_frac * max|ref|, and the
    normwise ||got - ref||_inf / ||ref||_inf."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    scale = np.max(np.abs(ref)) if ref.size else 0.0
    if scale == 0:
        return float(np.max(np.abs(got))) if got.size else 0.0, 0.0
    sel = np.abs(ref) > floor_frac * scale
    per = np.max(np.abs(got[sel] - ref[sel]) / np.abs(ref[sel])) if sel.any() else 0.0
    norm = np.max(np.abs(got - ref)) / scale
    return float(per), float(norm)


class Case:
    """A workload with its oracle matrix, inputs and oracle results."""

    def __init__(self, w: synth.Workload, image=None, with_corrections=None, mask=None,
                 frame_seed=None):
        self.w = w
        g = oracle_geometry(w.geometry)
        self.og = g
        ny, nx = w.ny, w.nx
        self.rad, self.chi = O.positions_for(g, ny, nx, w.unit, w.split, w.npt_azim)
        crad, cchi = O.centre_positions(g, ny, nx, w.unit)
        self.crad, self.cchi = crad, cchi
        if mask is None and w.masked:
            mask = synth.pilatus_module_mask(ny, nx)
        self.mask = mask
        self.A = O.csr_build(ny, nx, self.rad, self.chi, mask, w.npt_rad, w.npt_azim, w.split)
        corr = w.corrections if with_corrections is None else with_corrections
        if corr:
            self.dark, self.flat = synth.dark_flat(ny, nx, w.seed)
            self.sa = O.solid_angle(g, ny, nx).astype(np.float32)
            self.pol = O.polarization(g, ny, nx, w.polarization_factor).astype(np.float32)
        else:
            self.dark = self.flat = self.sa = self.pol = None
        if image is None:
            seed = w.seed if frame_seed is None else frame_seed
            if w.image_dtype == "uint32":
                image = synth.ring_image(crad, seed=seed, dtype=np.uint32,
                                         chi_deg_centre=cchi if w.npt_azim else None,
                                         modulation=0.3 if w.npt_azim else 0.0)
            else:
                image = synth.ring_image(crad, seed=seed, dtype=np.float32,
                                         chi_deg_centre=cchi if w.npt_azim else None,
                                         modulation=0.3 if w.npt_azim else 0.0)
        self.image = image

    def oracle(self, image=None):
        img = self.image if image is None else image
        return O.integrate(self.A, img, self.dark, self.flat, self.sa, self.pol)

    def dev(self, a, dtype=None):
        if a is None:
            return None
        t = to_dev(a)
        return t if dtype is None else t.to(dtype)

    def corrections_dev(self):
        return [self.dev(a) for a in (self.dark, self.flat, self.sa, self.pol)]

    def image_dev(self, image=None):
        img = self.image if image is None else image
        return to_dev(img)

    def gpu_from_oracle_positions(self):
        rad = self.dev(self.rad)
        chi = self.dev(self.chi)
        return api().Integrator.from_positions((self.w.ny, self.w.nx), rad, chi, self.w.npt_rad,
                                               self.w.npt_azim, SPLIT_NAMES[self.w.split],
                                               self.mask)

    def gpu_from_geometry(self):
        g = gpu_geometry(self.w.geometry)
        return api().Integrator.build(g, (self.w.ny, self.w.nx), self.w.npt_rad, self.w.npt_azim,
                                      UNIT_NAMES[self.w.unit], SPLIT_NAMES[self.w.split],
                                      self.mask)


def small_workload(ny=70, nx=90, split=synth.SPLIT_FULL, npt=60, npt_azim=0, unit=synth.UNIT_Q_NM,
                   seed=0, masked=False, corrections=True, dtype="uint32", tilt=0.05):
    rng = np.random.default_rng(seed)
    p = synth.GeometryParams(dist=float(rng.uniform(0.02, 0.08)),
                             poni1=float(rng.uniform(0.2, 0.8) * ny * 100e-6),
                             poni2=float(rng.uniform(0.2, 0.8) * nx * 100e-6),
                             rot1=float(rng.uniform(-tilt, tilt)), rot2=float(rng.uniform(-tilt, tilt)),
                             rot3=float(rng.uniform(-1, 1)), pixel1=100e-6, pixel2=100e-6,
                             wavelength=1e-10)
    return synth.Workload("small", ny, nx, p, unit, split, npt, npt_azim, image_dtype=dtype,
                          masked=False, corrections=corrections, seed=seed)


def random_mask(ny, nx, seed, frac=0.1):
    return (np.random.default_rng(seed + 77).random((ny, nx)) < frac).astype(np.uint8)
