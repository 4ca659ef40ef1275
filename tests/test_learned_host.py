"""Host-side pieces of the learned pre-decoder's training loop (no GPU):
parameter initialisation, the learning-rate schedule, weight files, and the
committed trained weights."""
import os

import numpy as np

import paper_2212_06985_gb300 as t3d
from paper_2212_06985_gb300 import learned

WEIGHTS = os.path.join(os.path.dirname(t3d.__file__), "weights", "cnn_L12_p04.npz")


def test_init_params_shape_and_scale():
    p = learned.init_params(3)
    assert p.dtype == np.float32 and p.size == t3d.toric3d_cnn_param_count() == 16515
    w1 = p[:16 * 6 * 27]
    assert abs(w1.std() - np.sqrt(2.0 / (6 * 27))) < 0.02    # He-normal fan-in 6 x 27
    assert np.array_equal(learned.init_params(3), p)


def test_lr_schedule():
    lr = [learned.lr_at(s, 1000, 1e-3) for s in range(1, 1001)]
    assert lr[0] == 1e-5 and abs(lr[99] - 1e-3) < 1e-12          # linear warm-up over 100 steps
    assert all(a >= b for a, b in zip(lr[99:], lr[100:]))          # then non-increasing
    assert abs(lr[-1] - 5e-5) < 1e-12                              # ends at 5% of lr


def test_weight_file_roundtrip(tmp_path):
    p = learned.init_params(1)
    f = str(tmp_path / "w.npz")
    learned.save_params(f, p, steps=7)
    assert np.array_equal(learned.load_params(f), p)


def test_committed_weights_load():
    p = learned.load_params(WEIGHTS)
    assert np.isfinite(p).all() and np.abs(p).max() < 100
