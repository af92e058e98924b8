"""Codec hyper-parameter sweep on the GPU (Sec. 4.5).

Every variant (one setting of the four loss weights of Eq. 8) is a codec
E = softplus(E~), D = softplus(D~) trained with Adam on shared mini-batches;
all variants advance together, one launch per mini-batch
(hsc_codec_fit_step), are validated after every epoch (hsc_codec_fit_eval)
and stop early once their validation loss has not improved for `patience`
epochs (hsc_codec_fit_track, which also keeps each variant's best
parameters).  The kept codecs are then scored by the multi-bounce proxy
(hsc_chain_eval: mean CIE94 of latent against spectral chains, averaged over
the depths) and the lowest score is selected.

This module only sequences the launches: the training arithmetic, the
validation, the early-stopping state and the chain errors all run in the
library's kernels; the host reads one count per epoch (to end the loop when
every variant has stopped) and the per-variant chain statistics at the end.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Dict, Optional

import numpy as np


def band_init_raw(k: int, n: int, floor: float = 1e-3, beta: float = 10.0):
    """Raw parameters (E~ (k, n), D~ (n, k)), float32, whose softplus is the
    band initialisation: the n samples split into k contiguous bands, row i
    of E the mean over band i, column i of D its indicator, every other
    weight `floor`."""
    edges = np.linspace(0, n, k + 1)
    E = np.full((k, n), floor)
    D = np.full((n, k), floor)
    for i in range(k):
        lo = int(round(edges[i]))
        hi = max(int(round(edges[i + 1])), lo + 1)
        E[i, lo:hi] = max(1.0 / (hi - lo), floor)
        D[lo:hi, i] = 1.0
    # x with log(1 + exp(beta x)) / beta = y
    inv = lambda y: (beta * y + np.log(-np.expm1(-beta * y))) / beta
    return inv(E).astype(np.float32), inv(D).astype(np.float32)


@dataclass
class SweepResult:
    best_Et: object            # (V, k, n) kept raw parameters
    best_Dt: object            # (V, n, k)
    best_loss: object          # (V,) validation loss of the kept parameters
    epochs: object             # (V,) int32 epochs trained
    history: object            # (epochs_run, V, 5) validation loss terms per epoch (NaN once stopped)
    epochs_run: int = 0
    steps: int = 0             # mini-batch launches
    variant_steps: int = 0     # sum over variants of the steps each trained
    seconds: Dict[str, float] = field(default_factory=dict)
    E: object = None           # (V, k, n) softplus(best_Et)
    D: object = None
    kept_loss: object = None   # (V, 5) loss terms of the kept parameters on the validation batch
    chain_stats: Optional[np.ndarray] = None   # (V, depth, 4) {mean dE94, p95, mean dE2000, p95}
    scores: Optional[np.ndarray] = None        # (V,) mean over depths of mean dE94
    selected: int = -1


def fit_variants(hsc, ctx, R_all, L_all, T, weights, train, val, Et0, Dt0, epochs: int, patience: int = 15,
                 lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                 softplus_beta: float = 10.0, stream=None) -> SweepResult:
    """Train every variant.  R_all, L_all: device (rows, n); T: device (3, n);
    weights: device (V, 4); train: device (pair_r, pair_l, pair_scale), each
    (epochs_max, batches, batch); val: device (pair_r, pair_l, pair_scale) of
    the validation batch; Et0 (V, k, n), Dt0 (V, n, k): device initial raw
    parameters (copied, not modified)."""
    import torch
    V, k, n = Et0.shape
    dev = Et0.device
    tr, tl, ts_ = train
    if tr.shape[0] < epochs:
        raise ValueError("the schedule holds fewer epochs than requested")
    nb = tr.shape[1]
    Et, Dt = Et0.clone(), Dt0.clone()
    best_Et, best_Dt = Et0.clone(), Dt0.clone()
    mom = [torch.zeros_like(Et), torch.zeros_like(Et), torch.zeros_like(Dt), torch.zeros_like(Dt)]
    best = torch.full((V,), math.inf, device=dev)
    wait = torch.zeros(V, dtype=torch.int32, device=dev)
    active = torch.ones(V, dtype=torch.int32, device=dev)
    ep = torch.zeros(V, dtype=torch.int32, device=dev)
    n_active = torch.empty(1, dtype=torch.int32, device=dev)
    hist = torch.full((max(epochs, 1), V, 5), math.nan, device=dev)
    host_n = torch.empty(1, dtype=torch.int32, pin_memory=True)
    vr, vl, vs = val
    step = 0
    run = 0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for e in range(epochs):
        for b in range(nb):
            step += 1
            hsc.hsc_codec_fit_step(ctx, R_all, L_all, tr[e, b], tl[e, b], ts_[e, b], T, weights, Et, Dt, *mom,
                                   step=step, lr=lr, beta1=beta1, beta2=beta2, eps=eps,
                                   softplus_beta=softplus_beta, active=active, stream=stream)
        hsc.hsc_codec_fit_eval(ctx, R_all, L_all, vr, vl, vs, T, weights, Et, Dt, softplus_beta=softplus_beta,
                               active=active, losses_out=hist[e], stream=stream)
        hsc.hsc_codec_fit_track(ctx, hist[e], Et, Dt, best_Et, best_Dt, best, wait, active, patience, epochs=ep,
                                n_active_out=n_active, stream=stream)
        run = e + 1
        host_n.copy_(n_active, non_blocking=True)
        torch.cuda.synchronize(dev)
        if int(host_n[0]) == 0:
            break
    hsc.hsc_sync(ctx)
    t1 = time.perf_counter()
    res = SweepResult(best_Et, best_Dt, best, ep, hist[:run], epochs_run=run, steps=step)
    res.variant_steps = int(ep.sum().item()) * nb
    res.seconds["train"] = t1 - t0
    return res


def score_variants(hsc, ctx, res: SweepResult, R_all, L_all, T, weights, val, refl, lights, chain_light,
                   chain_refl, softplus_beta: float = 10.0, stream=None) -> SweepResult:
    """Score every kept codec by the multi-bounce proxy and select the lowest
    score (NaN scores never win).  refl, lights: device spectra of the chains;
    chain_light (C,), chain_refl (C, depth): device int32 indices."""
    import torch
    V, k, n = res.best_Et.shape
    dev = res.best_Et.device
    vr, vl, vs = val
    E = torch.empty(V, k, n, device=dev)
    D = torch.empty(V, n, k, device=dev)
    kept = torch.empty(V, 5, device=dev)
    C, depth = chain_refl.shape
    d94 = torch.empty(depth, C, device=dev)
    d00 = torch.empty(depth, C, device=dev)
    stats = torch.zeros(V, depth * 4, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    hsc.hsc_codec_fit_eval(ctx, R_all, L_all, vr, vl, vs, T, weights, res.best_Et, res.best_Dt,
                           softplus_beta=softplus_beta, losses_out=kept, E_out=E, D_out=D, stream=stream)
    for v in range(V):
        hsc.hsc_chain_eval(ctx, refl, lights, E[v], D[v], T, chain_light, chain_refl, d94, d00, stats[v],
                           stream=stream)
    hsc.hsc_sync(ctx)
    st = stats.cpu().numpy().reshape(V, depth, 4)
    res.seconds["score"] = time.perf_counter() - t0
    res.E, res.D = E, D
    res.kept_loss = kept
    res.chain_stats = st
    res.scores = st[:, :, 0].mean(axis=1)
    s = np.where(np.isnan(res.scores), np.inf, res.scores)
    res.selected = -1 if np.all(np.isnan(res.scores)) else int(np.argmin(s))
    return res
