"""Host side of the threshold experiments: the ansatz fit recovers a known
crossing from synthetic failure rates (no GPU)."""
import numpy as np
import pytest

pytest.importorskip("scipy")

from paper_2212_06985_gb300 import threshold


def test_fit_recovers_crossing():
    pth, nu, a = 0.0546, 1.1, (0.08, 1.6, 3.0)
    rng = np.random.default_rng(0)
    points = []
    for L in (14, 18, 24, 32):
        for p in (0.053, 0.054, 0.055, 0.056):
            x = (p - pth) * L ** (1 / nu)
            f = a[0] + a[1] * x + a[2] * x * x
            n = 200000
            points.append({"L": L, "p": p, "samples": n, "fail_q0": int(rng.binomial(n, f))})
    fit = threshold.fit_threshold(points)
    assert abs(fit["p_th"] - pth) < 3e-4
    assert fit["p_th_err"] < 3e-4


def test_presets_follow_the_paper():
    assert threshold.PRESETS["flip"]["T"] == 1000 and threshold.PRESETS["flip"]["schedule"] == "F"
    assert threshold.PRESETS["bp"]["bp_iters"] == 30 and threshold.PRESETS["bp"]["T"] == 500
    assert threshold.PRESETS["pbp"]["bp_iters"] == 20 and threshold.PRESETS["pbp"]["schedule"] == "PFFPFF"
    assert threshold.PRESETS["table1"]["T"] == 1000 and not threshold.PRESETS["table1"]["use_bp"]


def test_crossing_guess_brackets_the_crossing():
    pts = [{"L": L, "p": p, "samples": 1000, "fail_q0": f}
           for L, row in ((14, (10, 300, 900)), (24, (1, 150, 950))) for p, f in zip((0.040, 0.041, 0.042), row)]
    assert threshold.crossing_guess(pts) == 0.0415
