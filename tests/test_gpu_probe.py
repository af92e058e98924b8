"""The FP32 issue-rate probe that sits beside the ALU roofline: it runs the
FMA recurrences it claims (values against the closed form) and reports the
lane-operation count of its launch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_probe_counts_and_values():
    import paper_2602_18741_gb300 as hsc
    ctx = hsc.Context(0)
    dev = torch.device("cuda:0")
    ctas, iters = 3, 5
    sink = torch.full((ctas * 256,), float("nan"), device=dev)
    ops = hsc.hsc_fp32_peak_probe(ctx, sink, iters, ctas=ctas)
    hsc.hsc_sync(ctx)
    assert ops == ctas * 256 * iters * 32
    # each of the 8 chains runs a <- 0.999 a + 1e-3 for 32 x iters steps from
    # a0 = tid * 1e-3 + c: a_N = m^N a0 + s (1 - m^N) / (1 - m)
    m, s, N = 0.999, 1e-3, 4 * iters
    tid = np.tile(np.arange(256), ctas)
    a0 = (np.float32(tid * 1e-3)[:, None] + np.arange(8)[None, :]).astype(np.float64)
    want = (m ** N * a0 + s * (1 - m ** N) / (1 - m)).sum(axis=1)
    got = sink.cpu().numpy().astype(np.float64)
    assert np.allclose(got, want, rtol=2e-6, atol=0)
    ctx.close()


def test_probe_rejects_bad_arguments():
    import paper_2602_18741_gb300 as hsc
    ctx = hsc.Context(0)
    sink = torch.empty(256, device="cuda:0")
    with pytest.raises(Exception):
        hsc.hsc_fp32_peak_probe(ctx, sink, 0, ctas=1)
    with pytest.raises(Exception):
        hsc.hsc_fp32_peak_probe(ctx, sink, 4, ctas=2)    # sink too small
    ctx.close()


def test_tanh_probe_counts_and_values():
    # each of the 8 recurrences a <- tanh(a + 1/4) (hardware tanh, about
    # 2^-11 relative) stays within 1e-3 of the FP64 recurrence: tanh is a
    # contraction, so the per-step errors do not grow
    import paper_2602_18741_gb300 as hsc
    ctx = hsc.Context(0)
    dev = torch.device("cuda:0")
    ctas, iters = 2, 3
    sink = torch.full((ctas * 256,), float("nan"), device=dev)
    ops = hsc.hsc_tanh_peak_probe(ctx, sink, iters, ctas=ctas)
    hsc.hsc_sync(ctx)
    assert ops == ctas * 256 * iters * 32
    tid = np.tile(np.arange(256), ctas)
    a = (np.float32(tid * 1e-3)[:, None] + np.float32(np.arange(8) * 0.1)[None, :]).astype(np.float64)
    for _ in range(4 * iters):
        a = np.tanh(a + 0.25)
    got = sink.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - a.sum(axis=1))) < 8e-3
    ctx.close()


def test_tanh_probe_packed_f16_pairs():
    # the f16x2 form: two recurrences per register (the second starts 0.05
    # higher), f16 rounding each step (2^-11) plus the approximation; the
    # contraction keeps the sum of the 16 values within 3e-2 of FP64
    import paper_2602_18741_gb300 as hsc
    ctx = hsc.Context(0)
    dev = torch.device("cuda:0")
    ctas, iters = 2, 3
    sink = torch.full((ctas * 256,), float("nan"), device=dev)
    ops = hsc.hsc_tanh_peak_probe(ctx, sink, iters, ctas=ctas, packed=True)
    hsc.hsc_sync(ctx)
    assert ops == ctas * 256 * iters * 32 * 2
    tid = np.tile(np.arange(256), ctas)
    lo = (np.float32(tid * 1e-3)[:, None] + np.float32(np.arange(8) * 0.1)[None, :]).astype(np.float64)
    a = np.concatenate([lo, lo + 0.05], axis=1)
    for _ in range(4 * iters):
        a = np.tanh(a + 0.25)
    got = sink.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - a.sum(axis=1))) < 3e-2
    with pytest.raises(Exception):
        hsc.hsc_tanh_peak_probe(ctx, sink, iters, ctas=ctas, packed=2)
    ctx.close()
