"""The codec hyper-parameter sweep of Sec. 4.5 (float64).  Test infrastructure
only.

Sec. 4.5 trains one codec per setting of the four loss weights of Eq. 8, all
with the same data, architecture and optimiser (Adam, lr 1e-3, mini-batches
of 128 pairs, at most 150 epochs, early stopping with patience 15), scores
every trained codec with the multi-bounce proxy (CIE94 of the latent chain
against the spectral chain at depths 1-3) and keeps the setting that does best
across the depths.

Readings where the paper is silent:

* An epoch is one pass over the training pairs in a seeded shuffled order,
  cut into whole mini-batches; the Adam step counter runs on across epochs.
* The validation loss of a variant is its own weighted Eq. 8 total on one
  fixed validation batch, taken after every epoch.  An epoch improves on the
  best so far only when its loss is strictly lower (a NaN never improves);
  after ``patience`` epochs in a row without improvement the variant stops, and
  the parameters it keeps are those of its best epoch.
* The selection score is the mean over the depths of the mean CIE94; the
  lowest score wins, ties to the lower index.
* Every variant starts from the same raw parameters: the band initialisation
  (row i of E averages band i, column i of D is its indicator), with zeros
  raised to ``floor`` so that the softplus inverse exists.

Pins (tests/test_oracle_sweep.py): the early-stopping rule on hand-made loss
sequences (stop exactly ``patience`` epochs after the last improvement, ties
and NaN are no improvement, a falling sequence never stops, stopped variants
are left alone); the softplus of the initial parameters is the band
initialisation; the kept parameters are those of the epoch with the lowest
validation loss, re-evaluating them gives that loss, and a variant stops
exactly ``patience`` epochs after that epoch; zero epochs keep the initial
parameters; the selection takes the arg-min of the score and passes over NaN
scores; the identity codec scores 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import chain, codec


@dataclass
class EarlyStop:
    best: np.ndarray          # (V,) best validation loss so far (+inf before the first epoch)
    wait: np.ndarray          # (V,) epochs since the last improvement
    active: np.ndarray        # (V,) bool
    epochs: np.ndarray        # (V,) epochs evaluated while active


def early_stop_init(V: int) -> EarlyStop:
    return EarlyStop(np.full(V, np.inf), np.zeros(V, np.int64), np.ones(V, bool), np.zeros(V, np.int64))


def early_stop_update(st: EarlyStop, val, patience: int) -> np.ndarray:
    """One epoch's update of every active variant; returns the mask of the
    variants whose loss improved (their parameters become the kept ones)."""
    val = np.asarray(val)
    improved = np.zeros(len(st.best), bool)
    for v in range(len(st.best)):
        if not st.active[v]:
            continue
        st.epochs[v] += 1
        if val[v] < st.best[v]:          # False for NaN
            st.best[v] = val[v]
            st.wait[v] = 0
            improved[v] = True
        else:
            st.wait[v] += 1
            if st.wait[v] >= patience:
                st.active[v] = False
    return improved


def band_init_raw(k: int, n: int, floor: float = 1e-3, beta: float = codec.SOFTPLUS_BETA):
    """Raw parameters (E~, D~) whose softplus is the band initialisation with
    zeros raised to ``floor``."""
    E0, D0 = codec.band_init(k, n)
    return (codec.softplus_inverse(np.maximum(E0, floor), beta),
            codec.softplus_inverse(np.maximum(D0, floor), beta))


def _pairs(R, L, r, l, s, T) -> codec.Batch:
    return codec.Batch(R[np.asarray(r)], L[np.asarray(l)] * np.asarray(s, np.float64)[:, None], T)


@dataclass
class VariantResult:
    Et: np.ndarray            # kept raw parameters
    Dt: np.ndarray
    best: float               # validation loss of the kept parameters
    epochs: int               # epochs trained
    history: List[float] = field(default_factory=list)


def train_variant(R, L, T, w, sched, Et0, Dt0, epochs: int, patience: int, lr: float = 1e-3,
                  beta: float = codec.SOFTPLUS_BETA) -> VariantResult:
    """Train one variant with weights ``w`` (e2e, rec, code, col) over the
    schedule's mini-batches, validating after every epoch."""
    R = np.asarray(R, np.float64)
    L = np.asarray(L, np.float64)
    T = np.asarray(T, np.float64)
    wd = {"e2e": float(w[0]), "rec": float(w[1]), "code": float(w[2]), "col": float(w[3])}
    val = _pairs(R, L, sched.val_r, sched.val_l, sched.val_s, T)
    Et, Dt = np.array(Et0, np.float64), np.array(Dt0, np.float64)
    st = codec.adam_init(Et, Dt)
    es = early_stop_init(1)
    keep = (Et.copy(), Dt.copy())
    hist = []
    for e in range(epochs):
        if not es.active[0]:
            break
        for b in range(sched.train_r.shape[1]):
            batch = _pairs(R, L, sched.train_r[e, b], sched.train_l[e, b], sched.train_s[e, b], T)
            Et, Dt, st, _ = codec.adam_softplus_step(Et, Dt, st, batch, wd, lr=lr, beta=beta)
        v = codec.losses(codec.softplus(Et, beta), codec.softplus(Dt, beta), val, wd)["total"]
        hist.append(v)
        if early_stop_update(es, [v], patience)[0]:
            keep = (Et.copy(), Dt.copy())
    return VariantResult(keep[0], keep[1], float(es.best[0]), int(es.epochs[0]), hist)


def selection_scores(R, L, T, codecs, chain_light, chain_refl, beta: float = codec.SOFTPLUS_BETA) -> np.ndarray:
    """Mean over the depths of the mean CIE94 of every codec (E~, D~) on the
    given chains."""
    out = []
    for Et, Dt in codecs:
        r = chain.chain_delta_e(R, L, codec.softplus(Et, beta), codec.softplus(Dt, beta), T, chain_light, chain_refl)
        out.append(float(np.mean(r["de94_mean"])))
    return np.asarray(out)


def select(scores) -> int:
    """Index of the lowest score (the first of equal ones); a NaN score never
    wins.  -1 when every score is NaN."""
    s = np.asarray(scores, np.float64)
    if s.size == 0 or np.all(np.isnan(s)):
        return -1
    return int(np.argmin(np.where(np.isnan(s), np.inf, s)))
