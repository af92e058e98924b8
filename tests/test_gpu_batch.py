"""Batched persistent launch over frames of uneven size, light count, k and
codec: every frame's output must be bit-identical to shading the frame alone
(the per-channel arithmetic is the same code), and match the oracle."""
import numpy as np
import pytest

import hsc_inputs as hi
from oracle import cmf, metrics, shade

from helpers import rel_err_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2602_18741_gb300 as hsc
    ctx = hsc.Context(0)
    yield hsc, ctx, torch.device("cuda:0")
    ctx.close()


def _device_frame(hsc, ctx, dev, spec, dtype):
    import torch
    f = hi.frame_from_spec(spec, n_smooth=10, n_saw=3)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    g1 = hsc.GBuffer(t(f.g1.normal), t(f.g1.pos), t(f.g1.mat))
    g2 = hsc.GBuffer(t(f.g2.normal), t(f.g2.pos), t(f.g2.mat)) if f.g2 is not None else None
    lights = hsc.Lights(t(f.light_pos), t(f.light_intensity))
    k = spec.k
    zm = torch.empty(f.mat_spectra.shape[0], k, device=dev, dtype=dtype)
    zl = torch.empty(f.lights, k, device=dev, dtype=dtype)
    hsc.hsc_encode(ctx, t(spec.E), t(f.mat_spectra), zm)
    hsc.hsc_encode(ctx, t(spec.E), t(f.light_spd), zl)
    T = torch.empty(3, f.n, device=dev)
    hsc.hsc_cmf_weights(ctx, f.n, f.grid[0], f.grid[1], T)
    M = torch.empty(3, k, device=dev)
    hsc.hsc_fold_xyz(ctx, T, t(spec.D), M)
    return f, g1, g2, lights, zm, zl, M


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_is_bit_identical_to_single_frames(env, autotune):
    hsc, ctx, dev = env
    import torch
    specs = hi.batched_frame_specs(seed=77, count=10, min_side=7, max_side=150, min_lights=2, max_lights=300)
    for i, s in enumerate(specs):
        s.secondary = (i % 3 == 0)
    bctx = hsc.Context(0)
    hsc.hsc_set_autotune(bctx, autotune)
    frames, singles, refs = [], [], []
    for i, s in enumerate(specs):
        dt = torch.bfloat16 if i % 4 == 1 else torch.float32
        f, g1, g2, lights, zm, zl, M = _device_frame(hsc, bctx, dev, s, dt)
        xyz = torch.full((f.pixels, 3), -1.0, device=dev)
        lat = torch.full((f.pixels, s.k), -1.0, device=dev)
        frames.append(hsc.BatchFrame(g1, g2, zm, lights, zl, M, xyz, lat))
        lat1 = torch.empty(f.pixels, s.k, device=dev)
        xyz1 = torch.empty(f.pixels, 3, device=dev)
        hsc.hsc_shade_latent(ctx, g1, g2, zm, lights, zl, hsc.HSC_FUSED, lat1, xyz_out=xyz1, M_xyz=M)
        singles.append((lat1, xyz1))
        refs.append(f)
    batch = hsc.hsc_batch_create(bctx, frames)
    for _ in range(2):  # replays reset the tile queue
        hsc.hsc_batch_shade(bctx, batch)
        hsc.hsc_sync(bctx)
        for fr, (lat1, xyz1) in zip(frames, singles):
            assert torch.equal(fr.keep[7], lat1)
            assert torch.equal(fr.keep[6], xyz1)
    if autotune:
        assert "batch of 10 frames" in hsc.hsc_tune_report(bctx)
    # oracle check of two frames (fp32 codes)
    for i in (0, 2):
        f = refs[i]
        s = specs[i]
        z = shade.shade_latent(f, s.E.astype(np.float64))
        x = shade.decode_xyz(z, s.D.astype(np.float64), cmf.cmf_weights(*f.grid))
        assert rel_err_rows(frames[i].keep[7].cpu().numpy(), z) <= 1e-5
        assert metrics.rel_xyz_error(frames[i].keep[6].cpu().numpy(), x) <= 1e-5
    batch.close()
    bctx.close()


def test_batch_rejects_unsupported_k(env):
    hsc, ctx, dev = env
    import torch
    spec = hi.batched_frame_specs(seed=5, count=1, min_side=8, max_side=8, ks=(6,))[0]
    f, g1, g2, lights, zm, zl, M = _device_frame(hsc, ctx, dev, spec, torch.float32)
    zm3 = zm[:, :3].contiguous()
    zl3 = zl[:, :3].contiguous()
    bad = hsc.BatchFrame(g1, None, zm3, lights, zl3, M[:, :3].contiguous(), torch.empty(f.pixels, 3, device=dev))
    with pytest.raises(hsc.HscError) as ei:
        hsc.hsc_batch_create(ctx, [bad])
    assert ei.value.status == hsc.HSC_ERR_INVALID_ARG


def test_shade_frames_with_no_frames_only_prepares(env):
    hsc, ctx, dev = env
    import torch
    c2 = hsc.Context(0)
    hsc.hsc_shade_frames(c2, [])          # allocates the descriptor ring, launches nothing
    hsc.hsc_shade_frames(c2, [])
    spec = hi.batched_frame_specs(seed=6, count=1, min_side=9, max_side=9, ks=(6,))[0]
    f, g1, g2, lights, zm, zl, M = _device_frame(hsc, c2, dev, spec, torch.float32)
    xyz = torch.empty(f.pixels, 3, device=dev)
    hsc.hsc_shade_frames(c2, [hsc.BatchFrame(g1, g2, zm, lights, zl, M, xyz)])
    ref = torch.empty(f.pixels, 3, device=dev)
    lat = torch.empty(f.pixels, 6, device=dev)
    hsc.hsc_shade_latent(c2, g1, g2, zm, lights, zl, hsc.HSC_FUSED, lat, xyz_out=ref, M_xyz=M)
    hsc.hsc_sync(c2)
    assert torch.equal(xyz, ref)
    c2.close()
