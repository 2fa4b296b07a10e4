"""The truth-recovery scorer: a catalog equal to the truth scores zero error, and known offsets
come back as the errors the definitions give."""
import numpy as np

import synth
from synth.metrics import truth_recovery


def _truth_theta(sc):
    tr = sc.truth
    th = np.zeros((sc.n_sources, 27))
    th[:, 0:2] = tr["u"]
    g = tr["is_gal"]
    th[:, 6] = np.where(g, 8.0, -8.0)
    th[:, 7] = th[:, 9] = tr["log_r"]
    th[:, 11:15] = th[:, 19:23] = tr["colors"]
    logit = lambda p: np.log(p) - np.log1p(-p)
    th[:, 2] = logit(np.clip(tr["shape"][:, 0], 1e-6, 1 - 1e-6))
    th[:, 3] = logit(np.clip(tr["shape"][:, 1], 1e-6, 1 - 1e-6))
    th[:, 4] = tr["shape"][:, 2]
    th[:, 5] = np.log(tr["shape"][:, 3])
    return th


def test_truth_scores_zero_and_offsets_come_back():
    sc = synth.tiny(seed=4, n_sources=6, n_images=2, H=60, W=64)
    th = _truth_theta(sc)
    r = truth_recovery(sc, th)
    assert r["position_px_median"] < 1e-12 and r["mag_r_median"] < 1e-12 and r["type_error_rate"] == 0.0
    th2 = th.copy()
    th2[:, 0] += 0.3
    th2[:, 7] += 0.1
    th2[:, 9] += 0.1
    r2 = truth_recovery(sc, th2)
    assert abs(r2["position_px_median"] - 0.3) < 1e-12
    assert abs(r2["mag_r_median"] - 2.5 / np.log(10) * 0.1) < 1e-12
