"""az_integrate_noalloc: the single-frame forward for callers that may not allocate device
memory while they run (a plugin whose host program's memory pool has reserved the GPU, an
acquisition loop that forbids allocations after set-up).  Its partial sums live in a fixed
array inside the library instead of the integrator's own buffer, so it must give what
az_integrate1d / az_integrate2d give, call after call, with the array keeping whatever the
previous call left in it -- and the calls themselves must leave the device's free memory
unchanged.

This file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest
import torch

from paper_1412_6367_gb300 import synth
from gpu_common import Case, api, gpu_geometry, needs_gpu, rel_err, small_workload, to_dev

pytestmark = [pytest.mark.gpu, needs_gpu]

# the forward tests' tolerances: FP64 to rounding, FP32 compensated within 1e-5 relative
TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _outputs(ig, precision):
    dt = torch.float64 if precision == "fp64" else torch.float32
    return api().Result(*(torch.full((ig.nrows,), float("nan"), dtype=dt, device="cuda")
                        for _ in range(4)))


def _close(got, ref, tol):
    for g, r in zip(got, ref):
        g = g.double().cpu().numpy().ravel()
        r = r.double().cpu().numpy().ravel()
        assert np.all(np.isfinite(g) == np.isfinite(r))
        fin = np.isfinite(r)
        scale = max(np.max(np.abs(r[fin])), 1e-300) if fin.any() else 1.0
        assert np.max(np.abs(g[fin] - r[fin]), initial=0.0) <= tol * scale


@pytest.mark.parametrize("npt_azim", [0, 36])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_integrate_two_calls(precision, npt_azim):
    w = small_workload(ny=96, nx=131, npt=80, npt_azim=npt_azim, seed=11)
    case = Case(w)
    ig = case.gpu_from_geometry()
    corr = case.corrections_dev()
    # two different frames, one after the other: the second call runs on whatever the
    # first one left in the library's fixed array
    frames = [case.image, synth.ring_image(case.crad, seed=12, dtype=np.uint32)]
    dimgs = [to_dev(img) for img in frames]
    refs = [ig.integrate(d, *corr, precision=precision) for d in dimgs]
    outs = [_outputs(ig, precision) for _ in frames]
    torch.cuda.synchronize()
    # everything the calls read or write exists now: the calls themselves allocate nothing
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    got = [ig.integrate_noalloc(d, *corr, precision=precision, out=o) for d, o in zip(dimgs, outs)]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    for img, g, ref in zip(frames, got, refs):
        g = [t.view(ref.I.shape) for t in g]
        _close(g, ref, TOL[precision])
        # and per bin against the oracle
        for name, gg, oo in zip("ISNC", g, case.oracle(img)):
            per, norm = rel_err(gg.double().cpu().numpy(), oo)
            assert per <= TOL[precision] and norm <= TOL[precision], (name, per, norm)
    assert ig.status() == 0


def test_noalloc_refuses_more_than_its_array():
    # 4 x 4 pixel tiles on a 2048 x 2048 detector with 2000 bins: far more segments than the
    # fixed array holds in FP64 (8 MiB / 24 bytes per segment)
    from paper_1412_6367_gb300 import _lib as L
    w = small_workload(ny=2048, nx=2048, npt=2000, seed=3, corrections=False)
    ig = api().Integrator.build(gpu_geometry(w.geometry), (2048, 2048), 2000, 0, "q_nm^-1", "full")
    ig.set_tuning(4, 4, 0, 0)
    need = 3 * ig.info["n_segments"] * 8
    assert need > (8 << 20)
    img = torch.zeros((2048, 2048), dtype=torch.int32, device="cuda")
    with pytest.raises(L.AzError) as e:
        ig.integrate_noalloc(img, precision="fp64", out=_outputs(ig, "fp64"))
    assert e.value.code == -2  # AZ_ESHAPE
    assert "fixed buffer" in str(e.value)
