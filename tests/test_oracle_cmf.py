"""Pins of the oracle's colorimetry against facts outside its own code."""
import json
import os

import numpy as np
import pytest

import hsc_inputs as hi
from oracle import cmf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "colorimetry_points.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("grid_spec", [hi.GRID_31, hi.GRID_81])
def test_equal_energy_white_is_near_one_third(grid_spec):
    # The CIE 1931 observer puts the equal-energy illuminant at x = y = 1/3;
    # the analytic fit is within its ~1% lobe error of that.  Dropping the
    # negative x-bar lobe moves x by ~0.008 and fails this.
    T = cmf.cmf_weights(*grid_spec)
    w = T.sum(axis=1)
    xy = w[:2] / w.sum()
    assert abs(xy[0] - 1 / 3) < 1e-3 and abs(xy[1] - 1 / 3) < 1e-3
    assert abs(w[1] - 1.0) < 1e-14          # Y of the unit spectrum is 1


def test_ybar_peak_is_photopic_555():
    # ybar is the photopic luminous efficiency V(lambda): maximum 1 near 555 nm.
    lam = np.arange(380.0, 781.0, 0.5)
    y = cmf.ybar(lam)
    assert 550.0 <= lam[np.argmax(y)] <= 560.0
    assert abs(y.max() - 1.0) < 0.01
    assert abs(cmf.ybar(555.0) - 1.0) < 0.01


def test_cmf_lobe_shapes():
    # each lobe is exactly 1 at its centre and has the stated one-sided widths
    assert cmf._lobe(599.8, 599.8, 37.9, 31.0) == 1.0
    assert abs(cmf._lobe(599.8 - 37.9, 599.8, 37.9, 31.0) - np.exp(-0.5)) < 1e-15
    assert abs(cmf._lobe(599.8 + 31.0, 599.8, 37.9, 31.0) - np.exp(-0.5)) < 1e-15
    # x-bar has its main peak near 600 nm and a secondary one near 445 nm; z-bar peaks near 445 nm
    lam = np.arange(380.0, 781.0, 1.0)
    x = cmf.xbar(lam)
    assert 590 <= lam[np.argmax(x)] <= 605
    z = cmf.zbar(lam)
    assert 440 <= lam[np.argmax(z)] <= 450


def test_srgb_matrix_maps_d65_to_equal_rgb():
    g = _golden()["srgb"]
    rgb = np.array([g["d65_xyz"]]) @ cmf.XYZ_TO_SRGB.T
    assert np.allclose(rgb, 1.0, atol=2e-4)


def test_srgb_transfer_points():
    g = _golden()["srgb"]
    # continuity at the segment join and the fixed points 0 and 1
    t = 0.0031308
    assert abs(12.92 * t - (1.055 * t ** (1 / 2.4) - 0.055)) < 1e-6
    assert cmf.srgb_oetf(0.0) == 0.0
    assert abs(cmf.srgb_oetf(1.0) - 1.0) < 1e-12
    assert abs(cmf.srgb_oetf(0.5) - g["oetf_half"]) < 1e-5


def test_lab_reference_points():
    g = _golden()["lab"]
    white = np.array([0.9, 1.0, 1.1])
    lab = cmf.xyz_to_lab(white[None, :], white)
    assert np.allclose(lab, [[100.0, 0.0, 0.0]], atol=1e-12)
    grey = cmf.xyz_to_lab((0.18 * white)[None, :], white)
    assert abs(grey[0, 0] - g["L_of_18pct_grey"]) < 1e-3
    assert abs(grey[0, 1]) < 1e-12 and abs(grey[0, 2]) < 1e-12
    dark = cmf.xyz_to_lab((1e-3 * white)[None, :], white)
    assert abs(dark[0, 0] - g["kappa"] * 1e-3) < 1e-9
    # the two branches of f meet at (6/29)^3
    e = (6 / 29) ** 3
    lo = cmf.xyz_to_lab((e * (1 - 1e-12) * white)[None, :], white)[0, 0]
    hi_ = cmf.xyz_to_lab((e * (1 + 1e-12) * white)[None, :], white)[0, 0]
    assert abs(lo - hi_) < 1e-8


def _rand_lab(rng, n):
    return np.stack([rng.uniform(0, 100, n), rng.uniform(-80, 80, n), rng.uniform(-80, 80, n)], axis=1)


def test_delta_e_identity_and_symmetry():
    rng = np.random.default_rng(1)
    a, b = _rand_lab(rng, 500), _rand_lab(rng, 500)
    for f in (cmf.delta_e2000, cmf.delta_e76):
        assert np.all(f(a, a) < 1e-12)
        assert np.allclose(f(a, b), f(b, a), atol=1e-12)
    assert np.all(cmf.delta_e94(a, a) < 1e-12)
    assert np.all(cmf.delta_e2000(a, b) >= 0)


def test_delta_e2000_neutral_pairs_reduce_to_lightness_term():
    # a* = b* = 0: chroma and hue terms vanish, dE00 = |dL| / S_L, with S_L = 1 at mean L = 50
    L1 = np.array([45.0, 40.0, 20.0, 70.0])
    L2 = np.array([55.0, 60.0, 35.0, 90.0])
    z = np.zeros(4)
    d = cmf.delta_e2000(np.stack([L1, z, z], 1), np.stack([L2, z, z], 1))
    assert abs(d[0] - 10.0) < 1e-12 and abs(d[1] - 20.0) < 1e-12
    Lm = 0.5 * (L1 + L2)
    SL = 1 + 0.015 * (Lm - 50) ** 2 / np.sqrt(20 + (Lm - 50) ** 2)
    assert np.allclose(d, np.abs(L2 - L1) / SL, atol=1e-12)
    assert np.allclose(cmf.delta_e94(np.stack([L1, z, z], 1), np.stack([L2, z, z], 1)), np.abs(L2 - L1))
    assert np.allclose(cmf.delta_e76(np.stack([L1, z, z], 1), np.stack([L2, z, z], 1)), np.abs(L2 - L1))


def test_delta_e2000_small_differences_are_below_delta_e76_scale():
    # for a given small Lab step the CIEDE2000 weights (S_L, S_C, S_H >= 1 at
    # mean L = 50) never enlarge it much beyond dE76
    rng = np.random.default_rng(3)
    a = _rand_lab(rng, 1000)
    a[:, 0] = 50.0
    b = a + rng.normal(0, 0.05, size=a.shape)
    b[:, 0] = 50.0
    d00 = cmf.delta_e2000(a, b)
    d76 = cmf.delta_e76(a, b)
    assert np.all(d00 <= 1.5 * d76 + 1e-12)


SHARMA = os.path.join(os.path.dirname(__file__), "golden", "ciede2000_sharma2005.json")


def test_delta_e2000_published_conformance_pairs():
    # the 34 published CIEDE2000 test pairs (Sharma, Wu and Dalal 2005), in
    # both orders; they exercise every term, including the hue-angle and
    # mean-hue branches at 180 degrees
    with open(SHARMA) as fh:
        pairs = json.load(fh)["pairs"]
    a = np.array([p["lab1"] for p in pairs], dtype=np.float64)
    b = np.array([p["lab2"] for p in pairs], dtype=np.float64)
    want = np.array([p["de00"] for p in pairs])
    assert len(pairs) == 34
    assert np.all(np.abs(cmf.delta_e2000(a, b) - want) < 5e-5)
    assert np.all(np.abs(cmf.delta_e2000(b, a) - want) < 5e-5)


def test_delta_e94_and_76_on_pure_chroma_and_hue_steps():
    # Delta E 76 is the Euclidean Lab distance: a 3-4-5 triangle
    assert abs(cmf.delta_e76(np.array([[50.0, 3.0, 4.0]]), np.array([[50.0, 0.0, 0.0]]))[0] - 5.0) < 1e-12
    ref = np.array([[50.0, 30.0, 0.0], [50.0, 30.0, 0.0], [50.0, 0.0, 30.0]])
    # a pure chroma step of 10 at C_ref = 30: 10 / (1 + 0.045 * 30)
    # a 90-degree hue turn at constant C = 30: chord 2 C sin(45 deg) / (1 + 0.015 * 30)
    # the same turn with the weights taken from the other colour (C_ref = 30 too) is unchanged
    oth = np.array([[50.0, 40.0, 0.0], [50.0, 0.0, 30.0], [50.0, 30.0, 0.0]])
    want = [10.0 / 2.35, 60.0 * np.sin(np.pi / 4) / 1.45, 60.0 * np.sin(np.pi / 4) / 1.45]
    assert np.allclose(cmf.delta_e94(ref, oth), want, rtol=1e-12, atol=0)
    # CIE94 is asymmetric: the weights come from the reference colour
    back = cmf.delta_e94(oth[:1], ref[:1])[0]
    assert abs(back - 10.0 / (1 + 0.045 * 40)) < 1e-12


def test_cmf_fit_follows_the_cie_1931_table():
    # the analytic fit against the tabulated observer at five wavelengths; a
    # dropped, shifted or mis-scaled lobe moves some value by far more
    g = _golden()["cie1931_2deg"]
    lam = np.asarray(g["nm"], dtype=np.float64)
    for name in ("xbar", "ybar", "zbar"):
        fit = getattr(cmf, name)(lam)
        assert np.max(np.abs(fit - np.asarray(g[name]))) < 0.012, name
