"""Shared plumbing for the GPU tests: upload a seeded frame, run the library,
and compute the oracle on the same inputs."""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

import hsc_inputs as hi


def subset_frame(f: hi.Frame, idx: np.ndarray) -> hi.Frame:
    """The frame restricted to pixels ``idx`` (for sampled oracle checks)."""
    g1 = hi.GBuffer(f.g1.normal[idx], f.g1.pos[idx], f.g1.mat[idx])
    g2 = None if f.g2 is None else hi.GBuffer(f.g2.normal[idx], f.g2.pos[idx], f.g2.mat[idx])
    return hi.Frame(len(idx), 1, f.grid, f.mat_spectra, f.light_spd, f.light_pos, f.light_intensity, g1, g2)


@dataclass
class DevFrame:
    g1: object
    g2: Optional[object]
    lights: object
    mats: object
    spd: object
    T: object
    P: int
    n: int


def upload(hsc, ctx, f: hi.Frame, dev):
    import torch

    def t(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    g1 = hsc.GBuffer(t(f.g1.normal), t(f.g1.pos), t(f.g1.mat))
    g2 = None if f.g2 is None else hsc.GBuffer(t(f.g2.normal), t(f.g2.pos), t(f.g2.mat))
    lights = hsc.Lights(t(f.light_pos), t(f.light_intensity))
    T = torch.empty(3, f.n, device=dev)
    hsc.hsc_cmf_weights(ctx, f.n, f.grid[0], f.grid[1], T)
    return DevFrame(g1, g2, lights, t(f.mat_spectra), t(f.light_spd), T, f.pixels, f.n)


def encode_all(hsc, ctx, df: DevFrame, E, dtype=None):
    import torch
    dtype = dtype or torch.float32
    dev = df.mats.device
    Ed = torch.from_numpy(np.ascontiguousarray(E, dtype=np.float32)).to(dev)
    k = E.shape[0]
    zm = torch.empty(df.mats.shape[0], k, device=dev, dtype=dtype)
    zl = torch.empty(df.spd.shape[0], k, device=dev, dtype=dtype)
    hsc.hsc_encode(ctx, Ed, df.mats, zm)
    hsc.hsc_encode(ctx, Ed, df.spd, zl)
    return zm, zl


def rel_err_rows(got, ref, floor_frac=1e-3):
    """max_p |got - ref|_inf / max(|ref(p)|_inf, floor * max|ref|) over rows."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return 0.0
    mag = np.abs(ref).max(axis=1)
    den = np.maximum(mag, floor_frac * mag.max())
    den = np.where(den > 0, den, 1.0)
    return float((np.abs(got - ref).max(axis=1) / den).max())


def assert_srgb8(got, srgb_ref, margin: float = 0.2):
    """8-bit sRGB bytes against the oracle's display values (FP64, [0, 1]
    after the clamp).  A byte whose unrounded code v * 255 + 0.5 lies more than
    `margin` of a code from a rounding boundary must equal the oracle's byte
    exactly (FP32 XYZ within 1e-5 relative moves the unrounded code by at most
    ~0.13, and by ~0.005 at the errors the kernels show); the others may round
    the other way, so they lie within one code."""
    x = np.clip(np.asarray(srgb_ref, dtype=np.float64), 0.0, 1.0) * 255.0 + 0.5
    want = np.floor(x)
    frac = x - want
    clear = (frac > margin) & (frac < 1.0 - margin)
    d = np.abs(np.asarray(got).astype(np.int64) - want.astype(np.int64))
    assert int(d.max()) <= 1
    assert np.all(d[clear] == 0), int(np.count_nonzero(d[clear]))
    return float(np.mean(clear))


def _oracle_band(args):
    """Worker: the oracle's XYZ of one band of a frame, n-sample and latent
    for each codec (runs in a spawned process)."""
    sf, codecs = args
    from oracle import cmf, shade
    T = cmf.cmf_weights(*sf.grid)
    out = {"spectral": shade.shade_spectral(sf, want_spectra=False)[1]}
    for k, (E, D) in codecs.items():
        z = shade.shade_latent(sf, np.asarray(E, dtype=np.float64))
        out[k] = shade.decode_xyz(z, np.asarray(D, dtype=np.float64), T)
    return out


def oracle_xyz_whole_frame(f: hi.Frame, codecs: dict, band_rows: int = 32, workers: int = 0) -> dict:
    """The FP64 oracle's XYZ of every pixel of a frame: the n-sample render
    ("spectral") and the latent render of each codec (key k, value (E, D)),
    computed band by band of `band_rows` rows in a pool of spawned processes
    with one BLAS thread each (the host memory per band stays bounded)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    step = band_rows * f.width
    bands = [np.arange(p0, min(p0 + step, f.pixels)) for p0 in range(0, f.pixels, step)]
    workers = workers or max(1, min(16, os.cpu_count() or 1, len(bands)))
    saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    out = {"spectral": np.empty((f.pixels, 3))}
    for k in codecs:
        out[k] = np.empty((f.pixels, 3))
    # the workers start on the first submission and read the thread setting
    # from the environment then; this process's BLAS is already set up
    for v in saved:
        os.environ[v] = "1"
    try:
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            jobs = ex.map(_oracle_band, [(subset_frame(f, b), codecs) for b in bands])
            for idx, res in zip(bands, jobs):
                for key, xyz in res.items():
                    out[key][idx] = xyz
    finally:
        for v, old in saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old
    return out
