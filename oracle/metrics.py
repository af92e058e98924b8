"""Error metrics for the oracle (float64).  Test infrastructure only.

* Relative XYZ error of a result against a reference image:
  max_p |XYZ(p) - XYZ_ref(p)|_inf / max(|XYZ_ref(p)|_inf, 1e-3 max_q |XYZ_ref(q)|_inf)
  (the floor keeps pixels that all lights miss from dividing by zero).
* Delta E statistics of the latent render against the n-sample render: both
  images are divided by Y_ref = max_p Y of the n-sample image, converted to
  CIELAB with white T @ 1, and Delta E 2000 (also 94, 76) is taken per pixel;
  reported as the mean and the nearest-rank 95th percentile (sort ascending,
  index ceil(0.95 N) - 1).  The paper compares colours by CIE94 (Sec. 4.5) and
  Delta E 76 (Sec. 5.2); Delta E 2000 is added as the primary statistic.

Pins: the nearest-rank percentile against a hand-sorted list; the statistics
of identical images are zero.
"""
from __future__ import annotations

import math

import numpy as np

from . import cmf


def rel_xyz_error(xyz, xyz_ref, floor_frac=1e-3):
    xyz = np.asarray(xyz, dtype=np.float64)
    ref = np.asarray(xyz_ref, dtype=np.float64)
    if ref.size == 0:
        return 0.0
    mag = np.abs(ref).max(axis=1)
    den = np.maximum(mag, floor_frac * mag.max())
    den = np.where(den > 0, den, 1.0)
    return float((np.abs(xyz - ref).max(axis=1) / den).max())


def nearest_rank(values, q=0.95):
    v = np.sort(np.asarray(values, dtype=np.float64))
    if v.size == 0:
        return 0.0
    idx = max(int(math.ceil(q * v.size)) - 1, 0)
    return float(v[idx])


def delta_e_stats(xyz_latent, xyz_spectral, T):
    """Mean and p95 of Delta E 2000 (and means of 94 / 76) of the latent image
    against the spectral one, exposure set by the spectral image's max Y."""
    white = np.asarray(T, dtype=np.float64).sum(axis=1)
    ys = np.asarray(xyz_spectral, dtype=np.float64)
    yl = np.asarray(xyz_latent, dtype=np.float64)
    yref = ys[:, 1].max()
    if yref <= 0:
        yref = 1.0
    lab_s = cmf.xyz_to_lab(ys / yref, white)
    lab_l = cmf.xyz_to_lab(yl / yref, white)
    d00 = cmf.delta_e2000(lab_s, lab_l)
    d94 = cmf.delta_e94(lab_s, lab_l)
    d76 = cmf.delta_e76(lab_s, lab_l)
    return {"de2000_mean": float(d00.mean()), "de2000_p95": nearest_rank(d00, 0.95),
            "de94_mean": float(d94.mean()), "de76_mean": float(d76.mean()),
            "y_ref": float(yref), "per_pixel_de2000": d00}
