"""GPU parity of the fused correction + sparse matrix-vector product against the oracle.

Tolerances: FP64 path within 1e-12 relative per bin; FP32 Kahan-compensated path within
1e-5 relative per bin (bins with |ref| above 1e-3 of the largest) and normwise, stated for
I, S (sum_signal), N (sum_norm) and C (count).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1412_6367_gb300 import synth
from gpu_common import Case, api, needs_gpu, random_mask, rel_err, small_workload, to_dev

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def check_outputs(res, ref, precision, what=""):
    for name, got, r in zip("ISNC", res, ref):
        per, norm = rel_err(got.cpu().numpy(), r)
        tol = TOL[precision]
        assert per <= tol and norm <= tol, (what, precision, name, per, norm)


def tiny_case():
    w = synth.tiny_workload()
    g = O.Geometry(*w.geometry.astuple())
    crad, _ = O.centre_positions(g, w.ny, w.nx, w.unit)
    return Case(w, image=synth.tiny_image(crad, seed=0))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tiny_config(precision):
    """256 x 256 float32, bbox, 200 bins, no corrections: indices bit-exact, I within 1e-12
    (FP64)."""
    c = tiny_case()
    gpu = c.gpu_from_geometry()
    res = gpu.integrate(c.image_dev(), precision=precision)
    check_outputs(res, c.oracle(), precision, "tiny")
    indptr, indices, _ = gpu.export_csr()
    assert np.array_equal(indices, c.A.indices)
    assert np.array_equal(indptr.astype(np.int64), c.A.indptr)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("split", [0, 1, 2])
@pytest.mark.parametrize("dtype", ["uint32", "float32", "int32"])
def test_small_with_corrections(precision, split, dtype):
    w = small_workload(83, 117, split=split, npt=75, seed=split * 7 + len(dtype), dtype="float32")
    c = Case(w, mask=random_mask(83, 117, split))
    img = synth.uniform_image(83, 117, seed=4, lo=0, hi=5000,
                              dtype={"uint32": np.uint32, "float32": np.float32, "int32": np.int32}[dtype])
    gpu = c.gpu_from_oracle_positions()
    res = gpu.integrate(c.image_dev(img), *c.corrections_dev(), precision=precision)
    check_outputs(res, c.oracle(img), precision, "small")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("split", [0, 1, 2])
def test_cake_2d(precision, split):
    w = small_workload(96, 128, split=split, npt=50, npt_azim=72, unit=0, seed=31 + split,
                       dtype="float32")
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision=precision)
    assert res.I.shape == (72, 50)
    check_outputs([t.reshape(-1) for t in res], c.oracle(), precision, "cake")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("npt_azim", [0, 36])
def test_flat_image_is_exactly_one(precision, npt_azim):
    w = small_workload(90, 110, split=2, npt=64, npt_azim=npt_azim, unit=0, seed=2)
    c = Case(w, mask=random_mask(90, 110, 3), with_corrections=False)
    gpu = c.gpu_from_oracle_positions()
    ones = torch.ones((90, 110), dtype=torch.float32, device="cuda")
    res = gpu.integrate(ones, precision=precision)
    I, C = res.I.reshape(-1).cpu().numpy(), res.count.reshape(-1).cpu().numpy()
    assert np.all(I[C > 0] == 1.0)
    assert np.all(I[C == 0] == 0.0)
    if npt_azim == 0:
        u = to_dev(np.ones((3, 90, 110), np.uint32))
        out = gpu.integrate_batch(u)
        Ib = out.I.cpu().numpy()
        assert np.all(Ib[:, C > 0] == 1.0)


def test_deterministic():
    w = small_workload(128, 160, split=2, npt=100, seed=13)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    img = c.image_dev()
    corr = c.corrections_dev()
    a = [t.clone() for t in gpu.integrate(img, *corr, precision="fp32")]
    for _ in range(3):
        b = gpu.integrate(img, *corr, precision="fp32")
        for x, y in zip(a, b):
            assert torch.equal(x, y)


def test_batch_equals_single_frame():
    """The batched path (N and C once, frames_per_pass frames per matrix read) performs the
    same operations per frame as the single-frame path: identical bits."""
    w = small_workload(101, 141, split=2, npt=90, seed=17)  # odd frame size: frames misaligned
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    corr = c.corrections_dev()
    frames = np.stack([synth.ring_image(c.crad, seed=s, dtype=np.uint32) for s in range(11)])
    fd = to_dev(frames)
    for fpp in (1, 2, 4, 8, 16, 32):
        gpu.set_tuning(frames_per_pass=fpp)
        out = gpu.integrate_batch(fd, *corr)
        for k in range(frames.shape[0]):
            one = gpu.integrate(fd[k], *corr, precision="fp32")
            assert torch.equal(out.I[k], one.I), (fpp, k)
            assert torch.equal(out.sum_signal[k], one.sum_signal)
        assert torch.equal(out.sum_norm, one.sum_norm)
        assert torch.equal(out.count, one.count)
        ref = c.oracle(frames[3])
        per, norm = rel_err(out.I[3].cpu().numpy(), ref[0])
        assert per <= 1e-5 and norm <= 1e-5


def test_cake_batch_equals_single_frame():
    """2D: the batched path (and its one-thread-per-row finalisation for rows of few
    segments) gives the single-frame bits; N and C again on a second call (cached C)."""
    w = small_workload(96, 128, split=2, npt=40, npt_azim=90, unit=0, seed=29, dtype="float32")
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    corr = c.corrections_dev()
    frames = np.stack([synth.uniform_image(96, 128, seed=s, lo=0, hi=3000) for s in range(7)])
    fd = to_dev(frames)
    for call in range(2):
        out = gpu.integrate_batch(fd, *corr)
        for k in range(frames.shape[0]):
            one = gpu.integrate(fd[k], *corr, precision="fp32")
            assert torch.equal(out.I[k], one.I.reshape(-1)), (call, k)
            assert torch.equal(out.sum_signal[k], one.sum_signal.reshape(-1))
        assert torch.equal(out.sum_norm, one.sum_norm.reshape(-1))
        assert torch.equal(out.count, one.count.reshape(-1))
    ref = c.oracle(frames[4])
    for got, r in zip((out.I[4], out.sum_signal[4], out.sum_norm, out.count), ref):
        per, norm = rel_err(got.cpu().numpy(), r)
        assert per <= 1e-5 and norm <= 1e-5


@pytest.mark.parametrize("tile", [(16, 64), (32, 32), (64, 64), (16, 128), (8, 256)])
@pytest.mark.parametrize("rpw", [1, 4, 32])
def test_tunings_give_same_answer(tile, rpw):
    w = small_workload(150, 190, split=2, npt=140, seed=41)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    gpu.set_tuning(tile_h=tile[0], tile_w=tile[1], rows_per_warp=rpw)
    res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision="fp64")
    check_outputs(res, c.oracle(), "fp64", "tuning")
    res = gpu.integrate(c.image_dev(), *c.corrections_dev(), precision="fp32")
    check_outputs(res, c.oracle(), "fp32", "tuning")


@pytest.mark.parametrize("tile", [(16, 128), (8, 256), (32, 64)])
def test_copy_engines_identical(tile):
    """TMA bulk row copies and 16-byte cp.async copies stage the same bytes: identical
    results for the single-frame (FP64 and FP32) and batched paths."""
    w = small_workload(143, 301, split=2, npt=130, seed=43)
    c = Case(w, mask=random_mask(143, 301, 4))
    gpu = c.gpu_from_oracle_positions()
    gpu.set_tuning(tile_h=tile[0], tile_w=tile[1])
    corr = c.corrections_dev()
    frames = to_dev(np.stack([synth.ring_image(c.crad, seed=s, dtype=np.uint32) for s in range(9)]))
    res = {}
    for eng in ("tma", "async"):
        gpu.set_copy_engine(eng)
        a = [t.clone() for t in gpu.integrate(c.image_dev(), *corr, precision="fp64")]
        b = [t.clone() for t in gpu.integrate(c.image_dev(), *corr, precision="fp32")]
        o = [t.clone() for t in gpu.integrate_batch(frames, *corr)]
        res[eng] = a + b + o
    for x, y in zip(res["tma"], res["async"]):
        assert torch.equal(x, y)
    check_outputs(res["async"][:4], c.oracle(), "fp64", "engine")


def test_batch_host_matches_device():
    w = small_workload(120, 100, split=1, npt=70, seed=23)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    corr = c.corrections_dev()
    frames = np.stack([synth.ring_image(c.crad, seed=s, dtype=np.uint32) for s in range(37)])
    fh = to_dev(frames, pinned=True)
    I_h, S_h = gpu.integrate_batch_host(fh, *corr)
    out = gpu.integrate_batch(to_dev(frames), *corr)
    assert torch.equal(I_h, out.I.cpu())
    assert torch.equal(S_h, out.sum_signal.cpu())


def test_multi_instance_matches_single():
    rng = np.random.default_rng(5)
    cases, gpus, imgs = [], [], []
    for k in range(6):
        ny, nx = int(rng.integers(40, 160)), int(rng.integers(40, 160))
        w = small_workload(ny, nx, split=2, npt=int(rng.integers(20, 200)), seed=50 + k)
        c = Case(w)
        cases.append(c)
        gpus.append(c.gpu_from_oracle_positions())
        imgs.append(c.image_dev())
    corr = [c.corrections_dev() for c in cases]
    plan = api().MultiPlan(gpus, imgs, [x[0] for x in corr], [x[1] for x in corr],
                           [x[2] for x in corr], [x[3] for x in corr])
    for use_graph in (False, True, True):
        outs = plan.launch(use_graph=use_graph)
        torch.cuda.synchronize()
        for c, g, img, cr, o in zip(cases, gpus, imgs, corr, outs):
            one = g.integrate(img, *cr, precision="fp32")
            for a, b in zip(o, one):
                assert torch.equal(a, b)
            check_outputs(o, c.oracle(), "fp32", "multi")


def test_misaligned_views():
    """Arrays whose start is 4-byte but not 16-byte aligned are staged from the aligned-down
    address; results must not change."""
    w = small_workload(61, 77, split=2, npt=50, seed=3, dtype="float32")
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    ref = c.oracle()
    n = 61 * 77
    for off in (1, 2, 3):
        buf = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
        buf[off:off + n] = to_dev(c.image.reshape(-1))
        corr = []
        for a in (c.dark, c.flat, c.sa, c.pol):
            b = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
            b[3 - off + 1:3 - off + 1 + n] = to_dev(a.reshape(-1))
            corr.append(b[3 - off + 1:3 - off + 1 + n].view(61, 77))
        res = gpu.integrate(buf[off:off + n].view(61, 77), *corr, precision="fp64")
        check_outputs(res, ref, "fp64", "offset %d" % off)


def test_forward_errors():
    import ctypes
    A = api()
    from paper_1412_6367_gb300 import _lib
    w = small_workload(30, 40, split=1, npt=20, seed=1)
    c = Case(w)
    gpu = c.gpu_from_oracle_positions()
    img = c.image_dev()
    with pytest.raises(TypeError):
        gpu.integrate(img.double())
    with pytest.raises(ValueError):
        gpu.integrate(img.reshape(-1)[:10])
    raw = torch.zeros(30 * 40 * 4 + 8, dtype=torch.uint8, device="cuda")
    rc = _lib.load().az_integrate1d(gpu.handle, ctypes.c_void_p(raw.data_ptr() + 2), 0, None,
                                    None, None, None, 1, None, None, None, None, None)
    assert rc == -1   # AZ_EINVAL: not 4-byte aligned
    rc = _lib.load().az_integrate1d(gpu.handle, ctypes.c_void_p(raw.data_ptr()), 9, None,
                                    None, None, None, 1, None, None, None, None, None)
    assert rc == -1   # bad dtype
    rc = _lib.load().az_integrate1d(gpu.handle, ctypes.c_void_p(raw.data_ptr()), 0, None,
                                    None, None, None, 5, None, None, None, None, None)
    assert rc == -1   # bad precision
    rc = _lib.load().az_integrate2d(gpu.handle, ctypes.c_void_p(raw.data_ptr()), 0, None,
                                    None, None, None, 1, None, None, None, None, None)
    assert rc == -2   # 1D integrator
    assert gpu.status() == 0
