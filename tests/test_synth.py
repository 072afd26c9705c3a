"""The seeded synthetic inputs match the recipes stated in the design notes (CPU): shapes,
module-gap masks, corrections, batch instances and the size sweep; the generators are
deterministic and hold none of the method's arithmetic."""
import numpy as np

from paper_1412_6367_gb300 import synth


def test_pilatus6m_recipe():
    w = synth.pilatus_workload()
    assert (w.ny, w.nx, w.npt_rad, w.split, w.unit) == (2527, 2463, 1000, synth.SPLIT_FULL, synth.UNIT_Q_NM)
    m = synth.pilatus_module_mask(w.ny, w.nx)
    # 12 x 5 modules of 195 x 487 pixels, gaps of 17 rows and 7 columns
    assert int(m.sum()) == 526101 and int((m == 0).sum()) == 5697900
    assert w.geometry.pixel1 == w.geometry.pixel2 == 172e-6 and w.geometry.dist == 0.3


def test_pilatus1m_recipe():
    w = synth.pilatus1m_workload()
    assert (w.ny, w.nx, w.image_dtype, w.split) == (1043, 981, "int32", synth.SPLIT_BBOX)
    m = synth.pilatus_module_mask(w.ny, w.nx)
    # 5 x 2 modules: 4 gaps of 17 rows, 1 gap of 7 columns
    assert int((m == 0).sum()) == 5 * 2 * 195 * 487


def test_dark_flat_distributions_and_determinism():
    d, f = synth.dark_flat(300, 400, seed=1)
    d2, f2 = synth.dark_flat(300, 400, seed=1)
    assert np.array_equal(d, d2) and np.array_equal(f, f2)
    assert d.dtype == np.float32 and f.dtype == np.float32
    assert abs(float(d.mean()) - 10.0) < 0.02 and abs(float(d.std()) - 1.0) < 0.02
    assert f.min() >= 0.95 and f.max() <= 1.05


def test_batch_instances_recipe():
    ws = synth.batch_instances()
    assert len(ws) == 64
    assert {(w.ny, w.nx) for w in ws} == {(s[0], s[1]) for s in synth.BATCH_SHAPES}
    assert {w.npt_rad for w in ws} <= set(synth.BATCH_BINS)
    again = synth.batch_instances()
    assert [w.geometry for w in ws] == [w.geometry for w in again]
    for w in ws:
        assert 0.1 <= w.geometry.dist <= 0.5
        for r in (w.geometry.rot1, w.geometry.rot2, w.geometry.rot3):
            assert abs(r) <= 0.05


def test_size_sweep_covers_1_to_16_mpixel():
    sizes = [w.ny * w.nx / 1e6 for w in synth.size_sweep_workloads()]
    assert sizes == sorted(sizes)
    assert 1.0 <= sizes[0] < 1.1 and 16.0 <= sizes[-1] < 17.0
    assert any(abs(s - 6.2) < 0.1 for s in sizes)  # the Pilatus-6M shape


def test_ring_image_is_seeded_counts():
    w = synth.pilatus_workload()
    q = np.linspace(0.5, 40.0, 1000).reshape(20, 50)
    a = synth.ring_image(q, seed=3)
    b = synth.ring_image(q, seed=3)
    c = synth.ring_image(q, seed=4)
    assert a.dtype == np.uint32 and np.array_equal(a, b) and not np.array_equal(a, c)
