"""Storage rounding for reduced-precision variants.  Test infrastructure only.

The paper stores codes in RGB images (Fig. 2b) without naming a precision.
The reduced-precision variants store codes and light codes in bf16 or fp16 and
the latent image in fp8 e4m3 with one scale per channel; every rounding is
round-to-nearest-even, fp8 saturating at +-448.  The per-channel scale is
scale_c = max_p z_c(p) / 448 in float32 and the stored code is
q = fp8(z * (1 / scale_c)) with the reciprocal and product in float32;
dequantisation is q * scale_c in float32.

Rounding goes through torch's CPU casts.  Pins (tests/test_oracle_quant.py):
hand-derived values of each format's definition: exactly representable values
survive, ties go to the even neighbour, the e4m3 maximum is 448, the bf16 /
fp16 spacing at 1.0 is 2^-7 / 2^-10.
"""
from __future__ import annotations

import numpy as np
import torch

FP8_MAX = 448.0


def round_bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def round_f16(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.float16).to(torch.float64).numpy()


def round_fp8_e4m3(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    t = torch.clamp(t, -FP8_MAX, FP8_MAX)
    return t.to(torch.float8_e4m3fn).to(torch.float64).numpy()


def fp8_e4m3_bits(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    t = torch.clamp(t, -FP8_MAX, FP8_MAX)
    return t.to(torch.float8_e4m3fn).view(torch.uint8).numpy()


def fp8_channel_scales(z_f32):
    """scale_c = max_p z_c / 448 in float32 (channels with max 0 get scale 1)."""
    z = np.asarray(z_f32, dtype=np.float32)
    mx = z.max(axis=0) if z.shape[0] else np.zeros(z.shape[1], np.float32)
    s = (mx / np.float32(FP8_MAX)).astype(np.float32)
    return np.where(s > 0, s, np.float32(1.0)).astype(np.float32)


def quantize_fp8(z_f32, scales):
    """Codes (bits) and dequantised float32 values of a float32 latent image."""
    z = np.asarray(z_f32, dtype=np.float32)
    inv = (np.float32(1.0) / np.asarray(scales, dtype=np.float32)).astype(np.float32)
    scaled = (z * inv[None, :]).astype(np.float32)
    bits = fp8_e4m3_bits(scaled)
    deq = (round_fp8_e4m3(scaled).astype(np.float32) * np.asarray(scales, np.float32)[None, :]).astype(np.float32)
    return bits, deq
