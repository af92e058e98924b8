"""The allocation-free fp8 quantiser against the context-based one.

hsc_quantize_fp8_noalloc is for callers that may not allocate device memory
(a plugin under a host renderer that owns the GPU memory budget, a frame loop
that cannot afford cudaMalloc's device-wide synchronisation).  It keeps its
per-channel scratch in a static device array shared by every call, so the
test makes two calls in a row, the second on a latent whose channel maxima
are far below the first's: a stale maximum left in the array would change the
second call's scales and codes.  Quantisation is bit-exact, so both outputs
must equal hsc_quantize_fp8's exactly.

A caller that cannot allocate usually has no hsc context either, so one test
runs the entry point in a fresh process before any context exists, checks
it against the oracle's fp8 quantiser, and checks with cudaMemGetInfo that a
call after the first (which loads the kernels) leaves the device's free
memory unchanged.

The file name sorts last so that a run that stops at the first failure has
already run every other test.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

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


_NO_CONTEXT = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
import paper_2602_18741_gb300 as hsc
from oracle import quant
dev = torch.device("cuda:0")
torch.cuda.set_device(dev)
rng = np.random.default_rng(7)
P, k = 4099, 6
z = (rng.gamma(1.0, 1.0, (P, k)) * rng.uniform(0.1, 3.0, k)[None, :]).astype(np.float32)
zd = torch.from_numpy(z).to(dev)
codes = torch.empty(P, k, device=dev, dtype=torch.uint8)
scales = torch.empty(k, device=dev)
hsc.hsc_quantize_fp8_noalloc(zd, codes, scales)        # no hsc context in this process
torch.cuda.synchronize()
want_scales = quant.fp8_channel_scales(z)
want_codes, _ = quant.quantize_fp8(z, want_scales)
first = (np.array_equal(scales.cpu().numpy(), want_scales), np.array_equal(codes.cpu().numpy(), want_codes))
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
hsc.hsc_quantize_fp8_noalloc(zd, codes, scales)
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
second = np.array_equal(codes.cpu().numpy(), want_codes)
print(json.dumps({"scales_equal": bool(first[0]), "codes_equal": bool(first[1]), "second_equal": bool(second),
                  "free_before": int(free0), "free_after": int(free1)}))
"""


def test_noalloc_quantizer_without_any_context_allocates_nothing():
    r = subprocess.run([sys.executable, "-c", _NO_CONTEXT, ROOT], capture_output=True, text=True, cwd=ROOT,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["scales_equal"] and res["codes_equal"] and res["second_equal"], res
    assert res["free_after"] == res["free_before"], res
