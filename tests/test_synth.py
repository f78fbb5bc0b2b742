"""The seeded synthetic volumes that stand in for the F3 block (Sec. 3)."""
import numpy as np

from paper_1901_11095_gb300 import synth


def test_deterministic_and_shaped():
    a = synth.make_volume((40, 33, 29), seed=0)
    b = synth.make_volume((40, 33, 29), seed=0)
    c = synth.make_volume((40, 33, 29), seed=1)
    assert a.shape == (40, 33, 29) and a.dtype == np.float32 and a.flags.c_contiguous
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_snr_close_to_10db():
    clean = synth.make_volume((64, 48, 48), seed=3, noise=False)
    noisy = synth.make_volume((64, 48, 48), seed=3)
    ps = np.mean(clean.astype(np.float64) ** 2)
    pn = np.mean((noisy - clean).astype(np.float64) ** 2)
    assert abs(10 * np.log10(ps / pn) - 10.0) < 0.2


def test_f3_kind_has_zero_dome_interior():
    v = synth.make_volume((64, 60, 60), seed=1, kind="f3", noise=False)
    assert (v == 0).mean() > 0.01          # the salt-like body has zero amplitude


def test_ricker_peak_and_symmetry():
    w = synth.ricker()
    assert len(w) == 33 and w[16] == 1.0 and np.allclose(w, w[::-1])


def test_batch_shapes_range():
    s = synth.batch_shapes()
    assert len(s) == 64 and all(32 <= v <= 192 for sh in s for v in sh)
    assert s == synth.batch_shapes()
