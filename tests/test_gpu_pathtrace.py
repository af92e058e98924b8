"""Path tracing with per-channel throughput against the FP64 oracle.

The oracle traces the same paths (float32 geometry in the same rounding
order, the same Philox4x32-10 random numbers), so the GPU and the oracle
differ only in the radiance arithmetic along a path (FP32 products and sums
against FP64): 1e-5 relative XYZ per pixel, floored at 1e-3 of the image
maximum, like the other FP32 paths.  A single path traced differently would
move its pixel by a whole sample's contribution and fail the bound."""
import numpy as np
import pytest

import hsc_inputs as hi
from oracle import cmf, codec, metrics
from oracle import pathtrace as pt

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2602_18741_gb300 as hsc
    ctx = hsc.Context(0)
    yield hsc, ctx, torch.device("cuda:0")
    ctx.close()


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)


def _gpu(hsc, ctx, dev, sc, W, H, spp, depth, seed, mats, emit, to_xyz, want_chan=False):
    import torch
    xyz = torch.full((W * H, 3), float("nan"), device=dev)
    C = emit.shape[0]
    ch = torch.full((W * H, C), float("nan"), device=dev) if want_chan else None
    hsc.hsc_path_trace(ctx, _t(sc.quads, dev), _t(sc.spheres, dev), _t(sc.cam, dev), W, H, spp, depth, seed,
                       _t(mats, dev), _t(emit, dev), _t(to_xyz, dev), xyz, ch)
    hsc.hsc_sync(ctx)
    return xyz.cpu().numpy(), (ch.cpu().numpy() if want_chan else None)


@pytest.mark.parametrize("W,H,spp,depth,light", [(40, 30, 4, 3, "blackbody"), (37, 23, 1, 0, "blackbody"),
                                                 (24, 18, 3, 8, "narrowband"), (17, 9, 5, 1, "blackbody")])
def test_spectral_and_latent_match_oracle(env, W, H, spp, depth, light):
    hsc, ctx, dev = env
    sc = hi.cornell_scene(W, H, light=light)
    T = cmf.cmf_weights(*sc.grid)
    seed = 1000 + depth
    paths = pt.trace(sc, W, H, spp, depth, seed)
    xs_ref = pt.render_spectral(paths, sc, T)
    xs, _ = _gpu(hsc, ctx, dev, sc, W, H, spp, depth, seed, sc.refl, sc.emit, T)
    assert metrics.rel_xyz_error(xs, xs_ref) <= TOL
    E, D = hi.load_codec(6, 81)
    E64, D64 = E.astype(np.float64), D.astype(np.float64)
    zr = codec.encode(E64, sc.refl)
    ze = codec.encode(E64, sc.emit[None, :])[0]
    M = T @ D64
    z_ref, xl_ref = pt.render_latent(paths, zr, ze, D64, T)
    xl, z = _gpu(hsc, ctx, dev, sc, W, H, spp, depth, seed, zr, ze, M, want_chan=True)
    assert metrics.rel_xyz_error(xl, xl_ref) <= TOL
    scale = np.abs(z_ref).max()
    assert np.max(np.abs(z - z_ref)) <= TOL * max(scale, 1e-30) or np.allclose(z, z_ref, rtol=TOL, atol=1e-7 * scale)


def test_limits_and_errors(env):
    hsc, ctx, dev = env
    import torch
    sc = hi.cornell_scene(8, 8)
    T = cmf.cmf_weights(*sc.grid)
    # an empty image is fine
    xyz = torch.empty(0, 3, device=dev)
    hsc.hsc_path_trace(ctx, _t(sc.quads, dev), _t(sc.spheres, dev), _t(sc.cam, dev), 0, 0, 1, 2, 1,
                       _t(sc.refl, dev), _t(sc.emit, dev), _t(T, dev), xyz)
    with pytest.raises(Exception):  # depth beyond the limit
        hsc.hsc_path_trace(ctx, _t(sc.quads, dev), _t(sc.spheres, dev), _t(sc.cam, dev), 8, 8, 1, 17, 1,
                           _t(sc.refl, dev), _t(sc.emit, dev), _t(T, dev), torch.empty(64, 3, device=dev))
    # a material index past the table sets the error word
    bad = sc.quads.copy()
    bad[0, 7] = 9
    hsc.hsc_path_trace(ctx, _t(bad, dev), _t(sc.spheres, dev), _t(sc.cam, dev), 8, 8, 2, 2, 1, _t(sc.refl, dev),
                       _t(sc.emit, dev), _t(T, dev), torch.empty(64, 3, device=dev))
    with pytest.raises(hsc.HscError) as ei:
        hsc.hsc_sync(ctx)
    assert ei.value.status == hsc.HSC_ERR_DEVICE_CHECK


def test_spherical_room_inward_sphere(env):
    # the closed spherical room (a sphere with a negative radius, normals
    # inward) whose mean radiance the oracle pins to a closed form: the
    # kernel traces the same paths and gives the oracle's pixels
    hsc, ctx, dev = env
    W, H, spp, depth = 48, 40, 6, 8
    sc = hi.sphere_enclosure_scene(W, H, z0=0.2, rho=0.7, grid_spec=hi.GRID_31)
    T = cmf.cmf_weights(*sc.grid)
    paths = pt.trace(sc, W, H, spp, depth, seed=77)
    xs_ref = pt.render_spectral(paths, sc, T)
    xs, ch = _gpu(hsc, ctx, dev, sc, W, H, spp, depth, 77, sc.refl, sc.emit, T)
    assert metrics.rel_xyz_error(xs, xs_ref) <= TOL
    assert xs_ref[:, 1].min() > 0.0     # every pixel gathers light from the emitter
