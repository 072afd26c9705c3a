"""Corrections bound once (az_set_corrections) and batches through them
(az_integrate_batch_bound): the bits of az_integrate_batch with the same corrections, against
the oracle per bin, a snapshot that neither later unbound calls nor changes to the caller's
arrays disturb, replaced by a new binding and dropped by a change of the tiled layout."""
import numpy as np
import pytest
import torch

from paper_1412_6367_gb300 import synth
from gpu_common import Case, api, needs_gpu, rel_err, small_workload, to_dev

pytestmark = [pytest.mark.gpu, needs_gpu]


def _frames(c, n, seed0):
    return np.stack([synth.ring_image(c.crad, seed=seed0 + k, dtype=np.uint32) for k in range(n)])


def _same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("engine", ["tma", "async"])
def test_bound_equals_per_call_and_oracle(engine):
    w = small_workload(120, 150, npt=90, seed=31)
    c = Case(w)
    g = c.gpu_from_geometry()
    g.set_copy_engine(engine)
    fr = _frames(c, 20, 500)
    frames = to_dev(fr)
    A = c.corrections_dev()
    dB, fB = (torch.from_numpy(x).cuda() for x in synth.dark_flat(w.ny, w.nx, w.seed + 1))
    B = [dB, fB, A[2], A[3]]
    g.set_corrections(*A)
    bound_a = g.integrate_batch_bound(frames)
    per_call_a = g.integrate_batch(frames, *A)
    assert _same(bound_a, per_call_a)
    for k in (0, 13, 19):
        ref = c.oracle(fr[k])
        for name, got, r in zip("ISNC", (bound_a.I[k], bound_a.sum_signal[k], bound_a.sum_norm,
                                         bound_a.count), ref):
            per, norm = rel_err(got.double().cpu().numpy(), r)
            assert per <= 1e-5 and norm <= 1e-5, (name, per, norm)
    # a new binding replaces the old one
    g.set_corrections(*B)
    bound_b = g.integrate_batch_bound(frames)
    assert _same(bound_b, g.integrate_batch(frames, *B))
    assert not torch.equal(bound_b.sum_signal, bound_a.sum_signal)
    # unbound calls with other corrections, and changes to the bound arrays, leave it intact
    g.integrate_batch(frames, *A)
    dB.add_(3.0)
    fB.mul_(1.5)
    assert _same(g.integrate_batch_bound(frames), bound_b)
    assert g.status() == 0


def test_layout_change_drops_the_binding():
    from paper_1412_6367_gb300 import _lib as L
    w = small_workload(64, 96, npt=40, seed=32)
    c = Case(w)
    g = c.gpu_from_geometry()
    g.set_corrections(*c.corrections_dev())
    frames = to_dev(_frames(c, 3, 700))
    g.integrate_batch_bound(frames)
    g.set_tuning(8, 64, 0, 0)
    with pytest.raises(L.AzError) as e:
        g.integrate_batch_bound(frames)
    assert e.value.code == -1
    g.set_corrections(*c.corrections_dev())
    assert _same(g.integrate_batch_bound(frames), g.integrate_batch(frames, *c.corrections_dev()))


def test_bound_without_corrections():
    w = small_workload(64, 80, npt=50, seed=33, corrections=False)
    c = Case(w)
    g = c.gpu_from_geometry()
    g.set_corrections()
    frames = to_dev(_frames(c, 4, 800))
    assert _same(g.integrate_batch_bound(frames), g.integrate_batch(frames))


def test_bound_2d_and_zero_frames():
    """A 2D (radial x chi) integrator, whose rows have few segments (the per-thread phase 2),
    and a call with no frames, which only hands back the bound N and C."""
    w = small_workload(96, 110, npt=40, npt_azim=36, seed=34)
    c = Case(w)
    g = c.gpu_from_geometry()
    corr = c.corrections_dev()
    g.set_corrections(*corr)
    fr = _frames(c, 18, 900)
    frames = to_dev(fr)
    bound = g.integrate_batch_bound(frames)
    assert _same(bound, g.integrate_batch(frames, *corr))
    ref = c.oracle(fr[5])
    for name, got, r in zip("ISNC", (bound.I[5], bound.sum_signal[5], bound.sum_norm, bound.count), ref):
        per, norm = rel_err(got.double().cpu().numpy(), r)
        assert per <= 1e-5 and norm <= 1e-5, (name, per, norm)
    empty = torch.empty((0, w.ny, w.nx), dtype=torch.int32, device="cuda").view(torch.uint32)
    none = g.integrate_batch_bound(empty)
    assert torch.equal(none.sum_norm, bound.sum_norm) and torch.equal(none.count, bound.count)
    assert g.status() == 0
