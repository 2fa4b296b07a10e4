"""Truth-recovery errors of a catalog against the seeded truth (the error definitions of the
paper's comparison table, Sec. "Experimental results": position, brightness, colours, galaxy
shape, star/galaxy type), for reports on synthetic scenes.  Scoring only: no inference."""
import numpy as np


def _sig(x):
    return 1.0 / (1.0 + np.exp(-x))


def truth_recovery(scene, theta):
    """theta: [S, 27] catalog (free parameters).  Returns a dict of error summaries."""
    th = np.asarray(theta, np.float64)
    tr = scene.truth
    gal = np.asarray(tr["is_gal"], bool)
    p_gal = _sig(th[:, 6])
    pred_gal = p_gal > 0.5
    # the type's own brightness means
    r_mean = np.where(pred_gal, th[:, 9], th[:, 7])
    c_mean = np.where(pred_gal[:, None], th[:, 19:23], th[:, 11:15])
    pos_err = np.hypot(*(th[:, 0:2] - tr["u"]).T)
    mag_err = 2.5 / np.log(10.0) * np.abs(r_mean - tr["log_r"])          # reference band r
    col_err = np.abs(c_mean - tr["colors"])                                 # log flux ratios
    out = {
        "sources": int(len(th)),
        "position_px_median": float(np.median(pos_err)), "position_px_p90": float(np.percentile(pos_err, 90)),
        "mag_r_median": float(np.median(mag_err)),
        "color_median": [float(v) for v in np.median(col_err, 0)],
        "type_error_rate": float(np.mean(pred_gal != gal)),
    }
    both = gal & pred_gal
    if both.any():
        shp = tr["shape"][both]
        dev = _sig(th[both, 2])
        axis = _sig(th[both, 3])
        ang = np.abs(np.remainder(th[both, 4] - shp[:, 2] + np.pi / 2, np.pi) - np.pi / 2)
        scale = np.exp(th[both, 5])
        out.update({"galaxy_fracdev_median": float(np.median(np.abs(dev - shp[:, 0]))),
                    "galaxy_axis_median": float(np.median(np.abs(axis - shp[:, 1]))),
                    "galaxy_angle_deg_median": float(np.degrees(np.median(ang[shp[:, 1] < 0.9]))) if
                    (shp[:, 1] < 0.9).any() else None,
                    "galaxy_scale_px_median": float(np.median(np.abs(scale - shp[:, 3])))})
    return out
