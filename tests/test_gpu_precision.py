"""Reduced-precision variants on the 3840x2160 frame (n = 81, k = 6 and 9,
64 lights, primary + secondary): codes in BF16 / FP16, latent image in FP8
E4M3 with per-channel scales, spectral decode on tensor cores.  Each result is
compared with the FP64 oracle (unrounded codes) on 2000 sampled pixels, by
relative XYZ error and by CIEDE2000 of the variant against the oracle's latent
image.  The errors are written to a JSON report (set HSC_PRECISION_REPORT to a
path) and checked against loose bounds: FP32 must meet the 1e-5 parity bar,
the storage formats their own rounding scale."""
import json
import os

import numpy as np
import pytest

import hsc_inputs as hi
from oracle import cmf, codec, metrics, shade

from helpers import subset_frame, upload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [6, 9])
def test_precision_variants_against_oracle(k):
    import torch
    import paper_2602_18741_gb300 as hsc
    dev = torch.device("cuda:0")
    ctx = hsc.Context(0)
    f = hi.frame_config3()
    E, D = hi.load_codec(k, 81)
    df = upload(hsc, ctx, f, dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    Ed, Dd = t(E), t(D)
    M = torch.empty(3, k, device=dev)
    hsc.hsc_fold_xyz(ctx, df.T, Dd, M)
    rng = np.random.default_rng(k)
    idx = np.unique(rng.integers(0, f.pixels, 2000))
    tidx = torch.from_numpy(idx).to(dev)
    sf = subset_frame(f, idx)
    T64 = cmf.cmf_weights(*f.grid)
    z_ref = shade.shade_latent(sf, E.astype(np.float64))
    x_ref = shade.decode_xyz(z_ref, D.astype(np.float64), T64)
    S_ref = codec.decode(D.astype(np.float64), z_ref)

    def de(xyz):
        st = metrics.delta_e_stats(xyz, x_ref, T64)
        return st["de2000_mean"], st["de2000_p95"]

    report = {}
    for name, dt, lat_dt in (("f32", torch.float32, torch.float32), ("bf16_codes", torch.bfloat16, torch.float32),
                             ("f16_codes", torch.float16, torch.float32), ("bf16_codes_fp8_latent", torch.bfloat16, torch.uint8)):
        zm = torch.empty(f.mat_spectra.shape[0], k, device=dev, dtype=dt)
        zl = torch.empty(f.light_spd.shape[0], k, device=dev, dtype=dt)
        hsc.hsc_encode(ctx, Ed, df.mats, zm)
        hsc.hsc_encode(ctx, Ed, df.spd, zl)
        lat = torch.empty(f.pixels, k, device=dev, dtype=lat_dt)
        scales = torch.empty(k, device=dev) if lat_dt == torch.uint8 else None
        xyz = torch.empty(f.pixels, 3, device=dev)
        if lat_dt == torch.uint8:
            hsc.hsc_shade_latent(ctx, df.g1, df.g2, zm, df.lights, zl, hsc.HSC_FUSED, lat, latent_scales=scales)
            hsc.hsc_decode_xyz(ctx, lat, M, xyz, scales=scales)
            spec = torch.empty(f.pixels, 81, device=dev)
            hsc.hsc_decode_spectra(ctx, lat, Dd, spec, scales=scales)
        else:
            hsc.hsc_shade_latent(ctx, df.g1, df.g2, zm, df.lights, zl, hsc.HSC_FUSED, lat, xyz_out=xyz, M_xyz=M)
            spec = torch.empty(f.pixels, 81, device=dev)
            hsc.hsc_decode_spectra(ctx, lat.to(torch.bfloat16) if name != "f32" else lat, Dd, spec)
        hsc.hsc_sync(ctx)
        xs = xyz[tidx].cpu().numpy()
        sp = spec[tidx].cpu().numpy()
        m, p95 = de(xs)
        report[name] = {"rel_xyz": metrics.rel_xyz_error(xs, x_ref),
                        "rel_spectra": float(np.max(np.abs(sp - S_ref)) / np.abs(S_ref).max()),
                        "de2000_mean": m, "de2000_p95": p95,
                        "spectral_decode": "f32 tensor cores (bf16 three-part split)" if name == "f32" else "bf16 tensor cores"}
    ctx.close()
    path = os.environ.get("HSC_PRECISION_REPORT")
    if path:
        old = {}
        if os.path.exists(path):
            with open(path) as fh:
                old = json.load(fh)
        old[f"k{k}"] = report
        with open(path, "w") as fh:
            json.dump(old, fh, indent=1)
    assert report["f32"]["rel_xyz"] <= 1e-5
    assert report["f32"]["de2000_mean"] < 1e-3
    assert report["bf16_codes"]["rel_xyz"] < 0.1 and report["bf16_codes"]["de2000_mean"] < 1.0
    assert report["f16_codes"]["rel_xyz"] < 5e-3 and report["f16_codes"]["de2000_mean"] < 0.2
    assert report["bf16_codes_fp8_latent"]["rel_xyz"] < 0.5 and report["bf16_codes_fp8_latent"]["de2000_mean"] < 5.0
