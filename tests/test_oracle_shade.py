"""Pins of the oracle's shading against closed forms, brute force and the
identity codec."""
import math

import numpy as np
import pytest

import hsc_inputs as hi
from oracle import cmf, codec, shade


def _tiny(seed, w=4, h=4, secondary=True, grid=hi.GRID_31, lights=3, n_smooth=5, n_saw=2):
    return hi.make_frame(seed, w, h, grid, n_smooth=n_smooth, n_saw=n_saw, lights=lights,
                         secondary=secondary)


def _frame_from(pos1, nrm1, mat1, spectra, lpos, linten, spd, pos2=None, nrm2=None, mat2=None,
                grid=(400.0, 10.0, 31)):
    g1 = hi.GBuffer(np.asarray(nrm1, np.float32), np.asarray(pos1, np.float32), np.asarray(mat1, np.int32))
    g2 = None
    if pos2 is not None:
        g2 = hi.GBuffer(np.asarray(nrm2, np.float32), np.asarray(pos2, np.float32), np.asarray(mat2, np.int32))
    P = g1.pixels
    return hi.Frame(P, 1, grid, np.asarray(spectra, np.float32), np.asarray(spd, np.float32),
                    np.asarray(lpos, np.float32), np.asarray(linten, np.float32), g1, g2)


def test_single_light_closed_form():
    # Lambert surface rho/pi under a point light of intensity I at height h
    # straight above: radiance rho I / (pi h^2) at every wavelength.
    n = 31
    rho, I, h = 0.5, 1.5, 2.0
    f = _frame_from([[0, 0, 0]], [[0, 0, 1]], [0], np.full((1, n), rho),
                    [[0, 0, h]], [I], np.ones((1, n)))
    S, xyz = shade.shade_spectral(f)
    expect = rho * I / (math.pi * h * h)
    assert np.allclose(S, expect, rtol=1e-15)
    T = cmf.cmf_weights(*f.grid)
    assert np.allclose(xyz[0], expect * T.sum(axis=1), rtol=1e-14)
    assert abs(xyz[0, 1] - expect) < 1e-15       # Y of a flat spectrum is its value


def test_oblique_light_and_back_facing_closed_form():
    n = 31
    f = _frame_from([[0, 0, 0], [0, 0, 0]], [[0, 0, 1], [0, 0, -1]], [0, 0], np.full((1, n), 1.0),
                    [[1.0, 0.0, 0.5]], [1.0], np.ones((1, n)))
    S, _ = shade.shade_spectral(f)
    g = 0.5 / 1.25 ** 1.5                         # cos * r / r^3 with n.d = 0.5, r^2 = 1.25
    assert np.allclose(S[0], g / math.pi, rtol=1e-15)
    assert np.all(S[1] == 0.0)                    # light behind the surface


def test_two_point_bounce_closed_form():
    # x1 = 0 facing +z, x2 = (0,0,1) facing -z: d = (0,0,1), h12 = 1.
    # One light at (1, 0, 0.5) sees both points with n.d = 0.5, r^2 = 1.25.
    n = 31
    rho1, rho2, I = 0.7, 0.4, 2.0
    f = _frame_from([[0, 0, 0]], [[0, 0, 1]], [0], [np.full(n, rho1), np.full(n, rho2)],
                    [[1.0, 0.0, 0.5]], [I], np.ones((1, n)),
                    pos2=[[0, 0, 1]], nrm2=[[0, 0, -1]], mat2=[1])
    g = 0.5 / 1.25 ** 1.5
    expect = (rho1 / math.pi) * (I * g + 1.0 * (rho2 / math.pi) * I * g)
    S, _ = shade.shade_spectral(f)
    assert np.allclose(S, expect, rtol=1e-14)


def test_bounce_clamp_closed_form():
    # facing unit normals along d: n1.d = -n2.d = |d|, so h12 = 1 / max(|d|^2, eps).
    # Secondary point 0.05 above: |d|^2 = 0.0025 < eps = 0.01, clamped to h12 = 100.
    x1 = np.array([[0.0, 0.0, 0.0]])
    h = shade.bounce_factor(x1, [[0, 0, 1]], [[0.0, 0.0, 0.05]], [[0, 0, -1]])
    assert abs(h[0] - 100.0) < 1e-10
    # not clamped above eps: 0.5 above gives 1 / 0.25 = 4
    h2 = shade.bounce_factor(x1, [[0, 0, 1]], [[0, 0, 0.5]], [[0, 0, -1]])
    assert abs(h2[0] - 4.0) < 1e-12
    # back-facing secondary normal: no transfer
    h3 = shade.bounce_factor(x1, [[0, 0, 1]], [[0, 0, 0.5]], [[0, 0, 1]])
    assert h3[0] == 0.0


@pytest.mark.parametrize("secondary", [False, True])
def test_brute_force_spectral_matches_vectorised(secondary):
    f = _tiny(11, secondary=secondary)
    S, _ = shade.shade_spectral(f)
    B = shade.brute_force_spectral(f)
    assert np.max(np.abs(S - B) / np.maximum(np.abs(B), 1e-300)) < 1e-13


@pytest.mark.parametrize("secondary", [False, True])
def test_brute_force_latent_matches_vectorised(secondary):
    f = _tiny(12, secondary=secondary)
    rng = np.random.default_rng(0)
    E = rng.uniform(0, 0.2, (6, f.n))
    z = shade.shade_latent(f, E)
    B = shade.brute_force_latent(f, E)
    assert np.max(np.abs(z - B) / np.maximum(np.abs(B), 1e-300)) < 1e-13


@pytest.mark.parametrize("grid_spec,k", [(hi.GRID_81, 81), (hi.GRID_31, 33)])
def test_identity_codec_makes_latent_equal_spectral(grid_spec, k):
    # Sec. 3.1: at k = n the identity is an exact algebra-preserving codec, so
    # latent shading must reproduce spectral shading (n = 31 padded to k = 33).
    f = _tiny(13, w=8, h=5, grid=grid_spec, lights=6)
    n = f.n
    E = np.zeros((k, n))
    E[:n, :n] = np.eye(n)
    D = E.T.copy()
    z = shade.shade_latent(f, E)
    S, xyz_s = shade.shade_spectral(f)
    assert np.max(np.abs(codec.decode(D, z) - S)) <= 1e-13 * np.abs(S).max()
    T = cmf.cmf_weights(*f.grid)
    xyz_l = shade.decode_xyz(z, D, T)
    assert np.max(np.abs(xyz_l - xyz_s)) <= 1e-13 * np.abs(xyz_s).max()


def test_passes_equal_fused():
    f = _tiny(14, w=9, h=7, lights=5)
    E = np.random.default_rng(1).uniform(0, 0.2, (9, f.n))
    z = shade.shade_latent(f, E)
    passes, zr = shade.shade_latent_passes(f, E)
    assert len(passes) == 3 and all(p.shape == (63, 3) for p in passes)
    assert np.max(np.abs(z - zr)) <= 1e-14 * np.abs(z).max()
    for b in range(3):
        assert np.array_equal(zr[:, 3 * b:3 * b + 3], passes[b])


def test_non_negativity():
    # Sec. 4.3: non-negative weights and spectra keep codes, latent images
    # and decoded spectra non-negative.
    f = _tiny(15, w=16, h=16)
    rng = np.random.default_rng(2)
    E = rng.uniform(0, 0.2, (6, f.n))
    D = rng.uniform(0, 1.0, (f.n, 6))
    assert shade.material_codes(E, f).min() >= 0 and shade.light_codes(E, f).min() >= 0
    z = shade.shade_latent(f, E)
    assert z.min() >= 0 and codec.decode(D, z).min() >= 0


def test_light_sum_is_linear_in_lights():
    # exact addition (Sec. 4.1): shading with two lights equals the sum of
    # shading with each alone, in latent space too
    f = _tiny(16, lights=2)
    E = np.random.default_rng(3).uniform(0, 0.2, (6, f.n))
    z = shade.shade_latent(f, E)
    parts = []
    for l in range(2):
        g = hi.Frame(f.width, f.height, f.grid, f.mat_spectra, f.light_spd[l:l + 1],
                     f.light_pos[l:l + 1], f.light_intensity[l:l + 1], f.g1, f.g2)
        parts.append(shade.shade_latent(g, E))
    assert np.max(np.abs(z - parts[0] - parts[1])) <= 1e-14 * np.abs(z).max()
