"""Pins of the code-space path-tracing oracle."""
import json
import os

import numpy as np

import hsc_inputs as hi
from oracle import cmf, codec
from oracle import pathtrace as pt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")


def test_philox_known_answers():
    with open(GOLDEN) as fh:
        vectors = json.load(fh)["vectors"]
    for v in vectors:
        c = [np.array([int(x, 16)], np.uint32) for x in v["ctr"]]
        out = pt.philox4x32_10(*c, int(v["key"][0], 16), int(v["key"][1], 16))
        assert [f"{int(o[0]):08x}" for o in out] == v["out"]


def test_u01_is_exact_and_in_range():
    x = np.array([0, 255, 256, 0xFFFFFFFF], np.uint32)
    u = pt.u01(x)
    assert u.dtype == np.float32
    assert u[0] == 0.0 and u[1] == 0.0 and u[2] == np.float32(2.0 ** -24)
    assert u[3] == np.float32(1.0 - 2.0 ** -24) and u[3] < 1.0


def test_sincos_polynomials():
    u = (np.arange(100000, dtype=np.float64) / 100000.0).astype(np.float32)
    s, c = pt.sincos_turn(u)
    ang = 2.0 * np.pi * u.astype(np.float64)
    assert np.max(np.abs(s - np.sin(ang))) < 1e-6 and np.max(np.abs(c - np.cos(ang))) < 1e-6


def test_orthonormal_frames():
    rng = np.random.default_rng(0)
    n = rng.normal(size=(2000, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n = np.concatenate([n, [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [0, -1, 0]]]).astype(np.float32)
    b1, b2 = pt.onb(n[:, 0], n[:, 1], n[:, 2])
    B1 = np.stack(b1, axis=1).astype(np.float64)
    B2 = np.stack(b2, axis=1).astype(np.float64)
    N = n.astype(np.float64)
    for a, b in ((B1, B2), (B1, N), (B2, N)):
        assert np.max(np.abs((a * b).sum(axis=1))) < 1e-6
    for a in (B1, B2):
        assert np.max(np.abs(np.linalg.norm(a, axis=1) - 1.0)) < 1e-6


def test_cosine_weighted_mean_cosine():
    # E[cos theta] = 2/3 for cosine-weighted directions; mean of z = sqrt(1 - u1)
    r = pt.philox4x32_10(np.arange(200000, dtype=np.uint32), np.zeros(200000, np.uint32),
                         np.ones(200000, np.uint32), np.zeros(200000, np.uint32), 7, 0)
    z = np.sqrt(np.float32(1.0) - pt.u01(r[2])).astype(np.float64)
    assert abs(z.mean() - 2.0 / 3.0) < 4 * np.sqrt(1.0 / 18.0 / 200000)


def test_closed_form_hits():
    sc = hi.cornell_scene(4, 4)
    # straight down from the centre: the floor at t = 0.5 (the emitter is not above x = 0.5, z = 0.2)
    t, kind, idx = pt.intersect(sc, [0.5], [0.5], [0.2], [0.0], [-1.0], [0.0])
    assert kind[0] == 0 and idx[0] == 0 and t[0] == np.float32(0.5)
    # along +z through the sphere at (0.28, 0.18, 0.62), r = 0.18: first hit at z = 0.44
    t, kind, idx = pt.intersect(sc, [0.28], [0.18], [0.0], [0.0], [0.0], [1.0])
    assert kind[0] == 1 and idx[0] == 0 and abs(float(t[0]) - 0.44) < 1e-6
    # straight up under the emitter
    t, kind, idx = pt.intersect(sc, [0.5], [0.5], [0.55], [0.0], [1.0], [0.0])
    assert kind[0] == 0 and sc.quads[idx[0], 7] < 0 and abs(float(t[0]) - 0.498) < 1e-6


def test_scalar_tracer_gives_the_same_paths():
    sc = hi.cornell_scene(12, 9)
    paths = pt.trace(sc, 12, 9, 3, 4, seed=11)
    for lin in range(0, 12 * 9 * 3, 5):
        end, mats = pt.brute_force_path(sc, 12, 9, 3, 4, 11, lin // 3, lin % 3)
        assert end == paths.end[lin]
        m = paths.mats[lin]
        if end >= 0:
            assert mats[:end] == list(m[:end])
        else:
            assert mats == [x for x in m if x >= 0]


def test_direct_view_of_the_emitter_and_monotone_depth():
    W, H = 24, 18
    sc = hi.cornell_scene(W, H)
    T = cmf.cmf_weights(*sc.grid)
    p0 = pt.trace(sc, W, H, 4, 0, seed=3)
    x0 = pt.render_spectral(p0, sc, T)
    # with no reflections a sample is E when it sees the emitter, else 0
    frac = (p0.end.reshape(W * H, 4) == 0).mean(axis=1)
    assert np.allclose(x0, frac[:, None] * (T @ sc.emit)[None, :], rtol=1e-12, atol=1e-12)
    assert frac.max() > 0
    prev = x0
    for D in (1, 2, 3):
        xd = pt.render_spectral(pt.trace(sc, W, H, 4, D, seed=3), sc, T)
        assert np.all(xd[:, 1] >= prev[:, 1] - 1e-12)
        prev = xd


def test_identity_codec_latent_equals_spectral():
    g = (400.0, 10.0, 30)
    W, H = 16, 12
    sc = hi.cornell_scene(W, H, grid_spec=g)
    T = cmf.cmf_weights(*g)
    paths = pt.trace(sc, W, H, 2, 3, seed=5)
    E = np.eye(30)
    z, xl = pt.render_latent(paths, codec.encode(E, sc.refl), codec.encode(E, sc.emit[None, :])[0], E.T, T)
    xs = pt.render_spectral(paths, sc, T)
    assert np.allclose(xl, xs, rtol=1e-12, atol=1e-14)


def test_shared_float32_constants():
    # the kernel spells these as bit patterns; both sides must round them alike
    bits = lambda v: int(np.float32(v).view(np.uint32))
    assert bits(pt.HALF_PI) == 0x3FC90FDB and bits(pt.T_MIN) == 0x38D1B717 and bits(pt.OFFSET) == 0x3A83126F
    assert [bits(v) for v in pt._S] == [0x3E2AAAAB, 0x3C088889, 0x39500D01, 0x3638EF1D, 0x32D7322B]
    assert [bits(v) for v in pt._C] == [0x3F000000, 0x3D2AAAAB, 0x3AB60B61, 0x37D00D01, 0x3493F27E, 0x310F76C7]


def _enclosure_expectation(rho, f, depth, E=1.0):
    """Mean and variance of one path's value in the spherical room: every
    reflection happens on the sphere, and from any point on a sphere a
    cosine-weighted direction meets the sphere at a uniformly distributed
    point (the form factor between two area elements of a sphere's inside is
    dA / (4 pi R^2) whatever their positions).  The emitter square hides
    exactly the cap above z0 from the rest of the sphere (a chord from below
    the plane to the cap crosses the plane inside the sphere), so every
    bounce ends on the emitter with probability f = cap area / sphere area,
    independently of where it starts.  A path that makes j reflections and
    then meets the emitter carries E rho^j, with probability (1 - f)^(j-1) f
    for j = 1 .. depth (the camera sees only the sphere below z0)."""
    j = np.arange(1, depth + 1)
    p = (1.0 - f) ** (j - 1) * f
    mean = float(np.sum(p * E * rho ** j))
    second = float(np.sum(p * (E * rho ** j) ** 2))
    return mean, second - mean * mean


def test_spherical_room_matches_the_closed_form():
    # the estimator's expectation pinned by geometry alone (not by the traced
    # float32 paths): mean over 128 x 128 pixels x 24 samples of the room's
    # radiance against E sum_j rho^j (1 - f)^(j-1) f, with f = (1 - z0) / 2,
    # within five standard errors plus 0.4% for the 1e-3 offset of each new
    # ray off the sphere (the uniform-hit property holds on the sphere itself)
    W = H = 128
    spp = 24
    for z0, rho, depth in ((0.6, 0.8, 1), (0.6, 0.8, 3), (0.2, 0.7, 8), (0.6, 1.0, 8)):
        sc = hi.sphere_enclosure_scene(W, H, z0=z0, rho=rho)
        paths = pt.trace(sc, W, H, spp, depth, seed=21 + depth)
        assert np.all(paths.end != 0)                   # the camera never sees the emitter
        vals = pt.path_products(paths, sc.refl, sc.emit)[:, 0]
        mean, var = _enclosure_expectation(rho, (1.0 - z0) / 2.0, depth)
        se = np.sqrt(var / vals.size)
        assert abs(vals.mean() - mean) <= 5 * se + 4e-3 * mean, (z0, rho, depth, vals.mean(), mean)
        # the first bounce ends on the emitter with probability f
        f = (1.0 - z0) / 2.0
        assert abs(np.mean(paths.end == 1) - f) <= 5 * np.sqrt(f * (1 - f) / paths.end.size) + 4e-3 * f


def test_spherical_room_rays_stay_inside():
    # with inward normals every bounce stays in the room: after any number of
    # reflections a path either met the emitter or is still going at the
    # depth bound; no path leaves the scene
    sc = hi.sphere_enclosure_scene(32, 32, z0=-0.2, rho=0.5)
    paths = pt.trace(sc, 32, 32, 8, 12, seed=4)
    lost = (paths.end < 0) & (paths.mats[:, -1] < 0)
    assert not lost.any()
