"""The survey-mosaic generator (input generation only): its batched renderer against the per-source
renderer of the other scenes, and the shape of a small mosaic (exposures per source, radii)."""
import numpy as np
import torch

import synth
from synth import mosaic as M


def test_batched_renderer_matches_per_source_renderer():
    sc = synth.tiny(seed=5, n_sources=6, n_images=3, H=60, W=70, noise=False)   # rendered with window 40
    tr = sc.truth
    for im in sc.images:
        pos = np.array([im.wcs[:4].reshape(2, 2) @ u + im.wcs[4:] for u in tr["u"]])
        fl = np.exp(tr["log_r"][:, None] + tr["colors"] @ synth.COLOR_MIX.T)[:, im.band]
        rate = M.render_image_rate(im, pos, tr["is_gal"], tr["shape"], fl, torch.device("cpu"), window=40).numpy()
        # the stored images are float32
        assert np.abs(rate - im.pixels).max() <= 1e-7 * im.pixels.max()


def test_small_mosaic_shape():
    sc = M.mosaic(seed=3, fields_x=3, fields_y=2, n_sources=400, field_W=500, field_H=400, device="cpu")
    n = sc.truth["n_images"]
    assert n.min() >= 1 and n.max() <= 12
    assert sc.radius.min() >= 8 and sc.radius.max() <= 64
    assert len(sc.images) >= 6 and all(im.pixels.dtype == np.float32 for im in sc.images)
    # exposures per field: 1-3 bands, distinct within a field
    assert 6 <= len(sc.images) <= 18
    again = M.mosaic(seed=3, fields_x=3, fields_y=2, n_sources=400, field_W=500, field_H=400, device="cpu")
    np.testing.assert_array_equal(sc.theta0, again.theta0)
    np.testing.assert_array_equal(sc.radius, again.radius)
