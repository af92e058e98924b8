"""The allocation-free fp8 quantiser against the context-based one.

hsc_quantize_fp8_noalloc is for callers that may not allocate device memory
(a plugin under a host renderer that owns the GPU memory budget, a frame loop
that cannot afford cudaMalloc's device-wide synchronisation).  It keeps its
per-channel scratch in a static device array shared by every call, so the
test makes two calls in a row, the second on a latent whose channel maxima
are far below the first's: a stale maximum left in the array would change the
second call's scales and codes.  Quantisation is bit-exact, so both outputs
must equal hsc_quantize_fp8's exactly.

The file name sorts last so that a run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_quantizer_matches_context_quantizer_on_two_calls():
    import torch
    import paper_2602_18741_gb300 as hsc

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    ctx = hsc.Context(0)
    rng = np.random.default_rng(2026)
    P, k = 10_007, 9
    for call, gain in enumerate((50.0, 0.01)):
        z = (rng.gamma(1.0, 1.0, (P, k)) * gain * rng.uniform(0.2, 1.0, k)[None, :]).astype(np.float32)
        z[:, 7] = 0.0                       # an all-zero channel takes scale 1
        zd = torch.from_numpy(z).to(dev)
        ref_codes = torch.empty(P, k, device=dev, dtype=torch.uint8)
        ref_scales = torch.empty(k, device=dev)
        hsc.hsc_quantize_fp8(ctx, zd, ref_codes, ref_scales)
        codes = torch.full((P, k), 0xAB, device=dev, dtype=torch.uint8)
        scales = torch.full((k,), -1.0, device=dev)
        hsc.hsc_quantize_fp8_noalloc(zd, codes, scales)
        torch.cuda.synchronize()
        assert torch.equal(scales, ref_scales), f"call {call}: scales differ"
        assert torch.equal(codes, ref_codes), f"call {call}: codes differ"
        assert float(scales[7]) == 1.0
    ctx.close()


def test_noalloc_quantizer_rejects_too_many_channels():
    import torch
    import paper_2602_18741_gb300 as hsc

    dev = torch.device("cuda:0")
    z = torch.zeros(4, hsc.HSC_NOALLOC_MAX_K + 3, device=dev)
    with pytest.raises(hsc.HscError) as ei:
        hsc.hsc_quantize_fp8_noalloc(z, torch.empty(z.shape, device=dev, dtype=torch.uint8),
                                     torch.empty(z.shape[1], device=dev))
    assert ei.value.status == hsc.HSC_ERR_INVALID_ARG
    assert "maximum" in str(ei.value)
