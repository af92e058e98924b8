"""RGB-to-latent upsampling network (Sec. 5) on the tensor cores against the
FP64 oracle.

Tolerance: the kernel follows the oracle's f16 contract (forward_f16) except
for FP32 accumulation, the biases carried as f16 (hi, lo) pairs (about 2^-22
relative) and SiLU through the hardware tanh approximation (about 2^-11
relative) before the f16 rounding.  Those differences
can move a hidden activation to a neighbouring f16 value (2^-10 relative)
before the next layer; over 128 inputs per unit and two hidden layers that
stays below 5e-3 of the output scale per element on the random networks
(mean below 5e-4) and below 1e-2 on the fitted one, whose weights are larger.
The f16 contract itself sits several times closer to the exact network than
the bf16 one, so the distance to the exact network is asserted as well."""
import numpy as np
import pytest

import hsc_inputs as hi
from oracle import cmf, codec, upsample as up

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2602_18741_gb300 as hsc
    ctx = hsc.Context(0)
    yield hsc, ctx, torch.device("cuda:0")
    ctx.close()


def _dev(p: up.Params, dev):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev) for a in p.arrays()]


def _run(hsc, ctx, dev, p, C):
    import torch
    W = _dev(p, dev)
    rgb = torch.from_numpy(np.ascontiguousarray(C, dtype=np.float32)).to(dev)
    z = torch.full((C.shape[0], p.W3.shape[0]), float("nan"), device=dev)
    hsc.hsc_upsample_rgb(ctx, rgb, *W, z)
    hsc.hsc_sync(ctx)
    return z.cpu().numpy().astype(np.float64)


def _f32(p: up.Params) -> up.Params:
    return up.Params(*[np.asarray(a, dtype=np.float32).astype(np.float64) for a in p.arrays()])


@pytest.mark.parametrize("k,P", [(6, 1000), (9, 333), (16, 129), (1, 1), (6, 128 * 152 * 2 + 77)])
def test_random_network_matches_f16_contract(env, k, P):
    hsc, ctx, dev = env
    p = _f32(up.init_params(k, seed=k + P))
    C = np.random.default_rng(P).uniform(0.0, 1.0, (P, 3))
    z = _run(hsc, ctx, dev, p, C)
    ref = up.forward_f16(p, np.asarray(C, dtype=np.float32).astype(np.float64))
    scale = np.abs(ref).max()
    err = np.abs(z - ref)
    assert np.isfinite(z).all()
    assert err.max() <= 5e-3 * scale, err.max() / scale
    if err.size >= 64:  # a mean over a handful of values is just their maximum
        assert err.mean() <= 5e-4 * scale, err.mean() / scale
    # and within 1 % of the exact network (the bf16 contract alone is 0.5 %)
    assert np.abs(z - up.forward(p, C)).max() <= 1e-2 * scale


def test_trained_network_on_palette_colours(env):
    hsc, ctx, dev = env
    w = hi.load_upsampler(6, 81)
    p = up.Params(*[w[n].astype(np.float64) for n in ("W1", "b1", "W2", "b2", "W3", "b3")])
    T = cmf.cmf_weights(*hi.GRID_81)
    S = hi.rgb_palette(count=3000)
    C = up.rgb_of_spectra(S, T)
    z = _run(hsc, ctx, dev, p, C)
    C32 = np.asarray(C, dtype=np.float32).astype(np.float64)
    ref_h = up.forward_f16(p, C32)
    ref = up.forward(p, C32)
    assert np.abs(z - ref_h).max() <= 1e-2 * np.abs(ref_h).max()
    assert np.abs(z - ref).max() <= 1e-2 * np.abs(ref).max()
    # closer to the exact network than the bf16 contract
    assert np.abs(z - ref).max() < np.abs(up.forward_bf16(p, C32) - ref).max()
    # colour of the decoded codes, Delta E 2000: GPU against the f16 contract
    # (kernel arithmetic only) and against the exact network (plus f16)
    _, D = hi.load_codec(6, 81)
    white = T.sum(axis=1)

    def xyz(zz):
        return codec.decode(D.astype(np.float64), zz) @ T.T

    y = max(xyz(ref)[:, 1].max(), 1e-12)

    def de(a, b):
        return cmf.delta_e2000(cmf.xyz_to_lab(xyz(a) / y, white), cmf.xyz_to_lab(xyz(b) / y, white))

    d_k = de(z, ref_h)
    d_x = de(z, ref)
    assert d_k.mean() < 0.05 and np.percentile(d_k, 95) < 0.1, (d_k.mean(), np.percentile(d_k, 95))
    assert d_x.mean() < 0.2, d_x.mean()


def test_empty_and_invalid(env):
    hsc, ctx, dev = env
    import torch
    p = _f32(up.init_params(6, seed=1))
    W = _dev(p, dev)
    hsc.hsc_upsample_rgb(ctx, torch.empty(0, 3, device=dev), *W, torch.empty(0, 6, device=dev))
    W17 = _dev(up.init_params(17, seed=1), dev)
    with pytest.raises(Exception):
        hsc.hsc_upsample_rgb(ctx, torch.zeros(4, 3, device=dev), *W17, torch.empty(4, 17, device=dev))
    hsc.hsc_sync(ctx)
