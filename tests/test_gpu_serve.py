"""Continuous-batching server on the GPU: every request's result is the same
bits as rendering it alone, whatever it was batched with; requests that
arrive while others are on the GPU share launches, and several launches are
in flight at once."""
import numpy as np
import pytest

import hsc_inputs as hi

pytestmark = pytest.mark.gpu

SIZES = ((64, 48), (128, 96), (200, 150), (37, 29))


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2602_18741_gb300 as hsc
    from paper_2602_18741_gb300 import serve
    ctx = hsc.Context(0)
    dev = torch.device("cuda:0")
    scenes = serve.ResidentScenes(hsc, ctx, dev, scenes=2, sizes=SIZES, n_mat=64, pool=40)
    yield hsc, serve, ctx, dev, scenes
    ctx.close()


@pytest.fixture(scope="module")
def big_scenes(env):
    hsc, serve, ctx, dev, _ = env
    return serve.ResidentScenes(hsc, ctx, dev, scenes=2, sizes=BIG_SIZES, n_mat=64, pool=128)


BIG_SIZES = ((1024, 1024), (1536, 1024))


def _solo_latent(hsc, ctx, dev, scenes, r):
    import torch
    g1, lights, zm, zl, M = scenes.frame_inputs(r)
    lat = torch.empty(r.width * r.height, r.k, device=dev)
    xyz = torch.empty(r.width * r.height, 3, device=dev)
    hsc.hsc_shade_latent(ctx, g1, None, zm, lights, zl, hsc.HSC_FUSED, lat, xyz_out=xyz, M_xyz=M)
    hsc.hsc_sync(ctx)
    return xyz


def _stream(n=60):
    return hi.request_stream(seed=11, rate_hz=3000.0, duration_s=1.0, sizes=SIZES, min_lights=4, max_lights=40,
                             scenes=2)[:n]


def test_latent_serving_matches_requests_alone(env):
    hsc, serve, ctx, dev, scenes = env
    import torch
    reqs = _stream()
    stats, backend = serve.serve(hsc, ctx, scenes, reqs, mode="latent", keep_outputs=True, max_batch=16)
    s = stats.summary()
    assert s["requests"] == len(reqs) and s["launches"] >= 1
    for r in reqs:
        assert torch.equal(backend.outputs[r.rid], _solo_latent(hsc, ctx, dev, scenes, r)), r


def test_latent_burst_shares_launches_that_overlap(env, big_scenes):
    # 32 requests arrive together (1-1.5 Mpx, 96-128 lights, every k and n):
    # the scheduler admits them 8 to a launch, and each launch (~1 ms of GPU
    # work) is still running when the host submits the next, so launches
    # share requests and are in flight together; every result is still the
    # bits of rendering the request alone
    hsc, serve, ctx, dev, _ = env
    import torch
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(32):
        w, h = BIG_SIZES[i % 2]
        reqs.append(hi.Request(i, 0.0, w, h, (6, 9)[(i // 2) % 2], (31, 81)[(i // 4) % 2],
                               int(rng.integers(96, 129)), int(rng.integers(0, 2)), i))
    stats, backend = serve.serve(hsc, ctx, big_scenes, reqs, mode="latent", keep_outputs=True, max_batch=8)
    s = stats.summary()
    assert s["requests"] == len(reqs)
    assert s["max_batch"] == 8 and s["launches"] == 4 and s["batch_hist"] == {"8": 4}, s
    assert s["max_inflight_launches"] >= 2, s
    for r in reqs:
        assert torch.equal(backend.outputs[r.rid], _solo_latent(hsc, ctx, dev, big_scenes, r)), r


def test_spectral_serving_matches_requests_alone(env):
    hsc, serve, ctx, dev, scenes = env
    import torch
    reqs = _stream(30)
    stats, backend = serve.serve(hsc, ctx, scenes, reqs, mode="spectral", keep_outputs=True)
    assert stats.summary()["requests"] == len(reqs)
    for r in reqs:
        g1 = scenes.gbuf[(r.scene, r.width, r.height)]
        lpos, linten = scenes.lights[r.scene]
        lights = hsc.Lights(lpos[:r.lights], linten[:r.lights])
        xyz = torch.empty(r.width * r.height, 3, device=dev)
        hsc.hsc_shade_spectral(ctx, g1, None, scenes.mats[(r.scene, r.n)], lights, scenes.spd[(r.scene, r.n)][:r.lights],
                               scenes.T[r.n], xyz)
        hsc.hsc_sync(ctx)
        assert torch.equal(backend.outputs[r.rid], xyz), r
