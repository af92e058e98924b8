"""Fit and store the codecs (E, D) used as inputs by the tests and the bench.
Test infrastructure (input data generation), not part of the product path.

Runs the oracle's projected-gradient fit of Eq. 8 (paper weights, Sec. 4.5)
on the seeded synthetic training set for k in {6, 9} and n in {31, 81}, and
writes ``hsc_inputs/codecs/codec_k{k}_n{n}.npz`` holding float32 E (k, n) and
D (n, k) plus the fit log.  Calls only ``oracle`` and ``hsc_inputs``.

    python -m oracle.make_codecs [--iters 3000]
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

import hsc_inputs as hi
from oracle import cmf, codec


def fit_one(k: int, grid_spec, iters: int):
    ts = hi.training_set(grid_spec)
    batch = codec.make_batch(ts, cmf.cmf_weights(*grid_spec))
    t0 = time.time()
    r = codec.projected_gradient_fit(batch, k, iters=iters)
    parts = codec.losses(r.E, r.D, batch)
    return r, parts, time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--only", default="", help="e.g. 6x81")
    args = ap.parse_args()
    os.makedirs(hi.CODEC_DIR, exist_ok=True)
    for k in (6, 9):
        for g in (hi.GRID_31, hi.GRID_81):
            if args.only and args.only != f"{k}x{g[2]}":
                continue
            r, parts, dt = fit_one(k, g, args.iters)
            path = hi.codec_path(k, g[2])
            np.savez(path, E=r.E.astype(np.float32), D=r.D.astype(np.float32),
                     k=k, n=g[2], lambda0=g[0], dlambda=g[1], iterations=r.iterations,
                     loss_history=np.asarray(r.history), proj_grad_inf=r.proj_grad_inf,
                     **{f"loss_{key}": val for key, val in parts.items()})
            print(f"k={k} n={g[2]}: {r.iterations} it, loss {r.history[0]:.6g} -> "
                  f"{r.history[-1]:.6g} ({dt:.0f} s) -> {path}", flush=True)


if __name__ == "__main__":
    main()
