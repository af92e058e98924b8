"""Fit and store the RGB-to-latent upsampling networks used by the tests and
the bench.
Test infrastructure (input data generation), not part of the product path.

Trains the oracle's network (Sec. 5: 3 -> 128 -> 128 -> k, SiLU) on the
linear RGB colours and codes of the seeded training reflectances under the
stored k = 6 and k = 9 codecs on the 81-sample grid, and writes
``hsc_inputs/upsampler/upsampler_k{k}_n{n}.npz`` (float32 W1, b1, W2, b2, W3,
b3 and the loss log).  Calls only ``oracle`` and ``hsc_inputs``.

    python -m oracle.make_upsampler [--steps 3000]
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

import hsc_inputs as hi
from oracle import cmf, codec, upsample


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=3000)
    args = ap.parse_args()
    os.makedirs(hi.UPSAMPLER_DIR, exist_ok=True)
    for k in (6, 9):
        g = hi.GRID_81
        E, _ = hi.load_codec(k, g[2])
        R = hi.training_set(g).R
        C = upsample.rgb_of_spectra(R, cmf.cmf_weights(*g))
        Z = codec.encode(E.astype(np.float64), R)
        t0 = time.time()
        p, log = upsample.fit(C, Z, k, steps=args.steps, seed=k)
        arrs = {n: a.astype(np.float32) for n, a in zip(("W1", "b1", "W2", "b2", "W3", "b3"), p.arrays())}
        np.savez(hi.upsampler_path(k, g[2]), **arrs, losses=np.asarray(log.losses, dtype=np.float64))
        print(f"k={k} n={g[2]}: loss {log.losses[0]:.4g} -> {log.losses[-1]:.4g} in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
