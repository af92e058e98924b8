"""Tensor-core spectral decode (tcgen05, BF16 operands, FP32 accumulation)
against the FP64 product of the same bf16-rounded operands.

The decode is s_hat = W_dec z (Eq. 4).  With bf16 operands every product is
exact in FP32, so the only error left is the FP32 accumulation of at most 16
terms; the bound used is the shading path's 1e-5 relative per pixel.
"""
import numpy as np
import pytest

from oracle import codec, quant

from helpers import rel_err_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2602_18741_gb300 as hsc
    ctx = hsc.Context(0)
    yield hsc, ctx, torch.device("cuda:0")
    ctx.close()


# 160,077 pixels: 1,251 tiles, several per persistent CTA, so the staging
# tiles are reused while earlier stores may still be in flight
@pytest.mark.parametrize("k,n,P", [(6, 81, 128), (6, 81, 4096 + 77), (9, 81, 3 * 128), (9, 31, 1000), (16, 128, 257),
                                   (3, 16, 5), (6, 1, 300), (12, 96, 131), (6, 81, 160_077), (16, 128, 160_077),
                                   (9, 81, 160_077)])   # odd k: element loads over many tiles
def test_decode_spectra_bf16(env, k, n, P):
    hsc, ctx, dev = env
    import torch
    rng = np.random.default_rng(k * 1000 + n + P)
    D = rng.uniform(0, 1, (n, k)).astype(np.float32)
    z = rng.gamma(1.0, 0.3, (P, k)).astype(np.float32)
    zb = torch.from_numpy(z).to(torch.bfloat16)
    out = torch.full((P, n), -1.0, device=dev)
    hsc.hsc_decode_spectra(ctx, zb.to(dev), torch.from_numpy(D).to(dev), out)
    hsc.hsc_sync(ctx)
    ref = codec.decode(quant.round_bf16(D), zb.float().numpy().astype(np.float64))
    assert rel_err_rows(out.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("k,n,P", [(6, 81, 8192 + 5), (9, 81, 640), (9, 31, 129), (6, 81, 160_077),
                                   (9, 81, 160_077), (3, 128, 70_001)])
def test_decode_spectra_fp8(env, k, n, P):
    hsc, ctx, dev = env
    import torch
    rng = np.random.default_rng(k + n + P)
    D = rng.uniform(0, 1, (n, k)).astype(np.float32)
    z = (rng.gamma(1.0, 0.3, (P, k)) * rng.uniform(0.1, 5, k)[None, :]).astype(np.float32)
    s = quant.fp8_channel_scales(z)
    bits, _ = quant.quantize_fp8(z, s)
    q = torch.from_numpy(bits).view(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    Ds = quant.round_bf16((D * s[None, :]).astype(np.float32))
    out = torch.full((P, n), -1.0, device=dev)
    hsc.hsc_decode_spectra(ctx, torch.from_numpy(bits).to(dev), torch.from_numpy(D).to(dev), out,
                           scales=torch.from_numpy(s).to(dev))
    hsc.hsc_sync(ctx)
    ref = codec.decode(Ds, q)
    assert rel_err_rows(out.cpu().numpy(), ref) <= 1e-5


def test_decode_spectra_tc_matches_fp32_path_on_bf16_inputs(env):
    # the same bf16 values decoded on CUDA cores in FP32 and on tensor cores
    hsc, ctx, dev = env
    import torch
    rng = np.random.default_rng(7)
    P, k, n = 20000, 9, 81
    D = quant.round_bf16(rng.uniform(0, 1, (n, k)).astype(np.float32)).astype(np.float32)
    z = torch.from_numpy(rng.gamma(1.0, 0.3, (P, k)).astype(np.float32)).to(torch.bfloat16)
    a = torch.empty(P, n, device=dev)
    b = torch.empty(P, n, device=dev)
    hsc.hsc_decode_spectra(ctx, z.to(dev), torch.from_numpy(D).to(dev), a)
    hsc.hsc_decode_spectra(ctx, z.float().contiguous().to(dev), torch.from_numpy(D).to(dev), b)
    hsc.hsc_sync(ctx)
    assert rel_err_rows(a.cpu().numpy(), b.cpu().numpy().astype(np.float64)) <= 1e-5
