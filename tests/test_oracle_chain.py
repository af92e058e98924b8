"""Pins of the multi-bounce chain oracle (Sec. 4.5 proxy)."""
import numpy as np

import hsc_inputs as hi
from oracle import chain, cmf


def _sets(n=31, seed=1):
    lam = hi.grid(400.0, 300.0 / (n - 1), n)
    rng = np.random.default_rng(seed)
    R = hi.smooth_reflectances(rng, lam, 12)
    L = np.concatenate([hi.blackbody(lam, [3000.0, 6500.0]), hi.narrowband(lam, [500.0], [15.0])])
    return R, L, cmf.cmf_weights(400.0, 300.0 / (n - 1), n)


def test_identity_codec_gives_zero_error():
    R, L, T = _sets(n=30)
    E = np.eye(30)
    rng = np.random.default_rng(0)
    cl = rng.integers(0, 3, 20)
    cr = rng.integers(0, 12, (20, 3))
    out = chain.chain_delta_e(R, L, E, E.T, T, cl, cr)
    assert np.abs(out["de2000"]).max() < 1e-9 and np.abs(out["de94"]).max() < 1e-9


def test_constant_reflectance_closed_form():
    # equal-energy light of any intensity, S(b) = rho^b: Y / Y(light) = rho^b,
    # neutral colour; the codec is exact for flat spectra at k = n
    n = 30
    _, _, T = _sets(n)
    L = np.full((2, n), 3.0)
    R = np.full((1, n), 0.5)
    E = np.eye(n)
    out = chain.chain_delta_e(R, L, E, E.T, T, [0, 1], [[0, 0, 0], [0, 0, 0]])
    xs, _, light = chain.chain_xyz(R, L, E, E.T, T, [0, 1], [[0, 0, 0], [0, 0, 0]])
    white = T.sum(axis=1)
    for b in range(3):
        lab = cmf.xyz_to_lab(xs[:, b] / light[:, 1:2], white)
        y = 0.5 ** (b + 1)
        assert np.allclose(lab[:, 0], 116.0 * y ** (1 / 3) - 16.0, atol=1e-10)
        assert np.allclose(lab[:, 1:], 0.0, atol=1e-10)
    assert np.abs(out["de2000"]).max() < 1e-9


def test_all_ones_chain_is_the_white():
    n = 31
    _, _, T = _sets(n)
    L = np.full((1, n), 0.25)
    R = np.ones((1, n))
    xs, _, light = chain.chain_xyz(R, L, np.eye(n)[:3], np.eye(n)[:, :3], T, [0], [[0, 0]])
    lab = cmf.xyz_to_lab(xs[:, 1] / light[:, 1:2], T.sum(axis=1))
    assert np.allclose(lab, [[100.0, 0.0, 0.0]], atol=1e-10)


def test_brute_force_matches_vectorised():
    R, L, T = _sets(n=16, seed=3)
    rng = np.random.default_rng(5)
    E = rng.uniform(0, 0.3, (6, 16))
    D = rng.uniform(0, 1.0, (16, 6))
    cl = [1, 2]
    cr = [[3, 4, 5], [0, 11, 7]]
    xs, xl, _ = chain.chain_xyz(R, L, E, D, T, cl, cr)
    for c in range(2):
        bs, bl = chain.brute_force_chain_xyz(R, L, E, D, T, cl[c], cr[c])
        assert np.allclose(xs[c], bs, rtol=1e-13) and np.allclose(xl[c], bl, rtol=1e-13)


def test_exposure_maps_light_peak_to_one_and_is_intensity_invariant():
    R, L, T = _sets(n=31, seed=4)
    lam = hi.grid(400.0, 10.0, 31)
    # narrow bands at both ends of the grid have X or Z far above Y
    L = np.concatenate([L, hi.narrowband(lam, [400.0, 700.0], [10.0, 10.0])])
    light = L @ T.T
    s = chain.exposure(light)
    assert np.allclose((light * s[:, None]).max(axis=1), 1.0, rtol=1e-14)
    assert chain.exposure(np.zeros((1, 3)))[0] == 0.0
    rng = np.random.default_rng(9)
    E = rng.uniform(0, 0.3, (6, 31))
    D = rng.uniform(0, 0.5, (31, 6))
    cl = rng.integers(0, L.shape[0], 40)
    cr = rng.integers(0, R.shape[0], (40, 3))
    a = chain.chain_delta_e(R, L, E, D, T, cl, cr)
    b = chain.chain_delta_e(R, 7.5 * L, E, D, T, cl, cr)
    assert np.allclose(a["de94"], b["de94"], rtol=1e-10, atol=1e-12)
    assert np.allclose(a["de2000"], b["de2000"], rtol=1e-10, atol=1e-12)
    # reflectances in [0, 1]: every scaled spectral colour stays inside the unit cube
    xs, _, lx = chain.chain_xyz(R, L, E, D, T, cl, cr)
    sc = chain.exposure(lx)
    assert (xs * sc[:, None, None]).max() <= 1.0 + 1e-12
