"""RGB-to-latent upsampling network (float64).  Test infrastructure only.

Sec. 5 of the paper maps a linear RGB colour to a k-dimensional latent code
with a per-pixel multilayer perceptron of three fully connected layers, hidden
width 128 and SiLU activations:

    h1 = silu(W1 c + b1),   h2 = silu(W2 h1 + b2),   z = W3 h2 + b3,
    silu(x) = x / (1 + exp(-x)).

Training pairs are the linear RGB colour of each training spectrum s and its
code z_gt = E s under the frozen codec.  The paper's objective adds to the
code MSE 0.3 times the batch mean of the per-sample maximum absolute code
error, plus 0.05 times the CIE76 difference of the decoded colours.

Readings where the paper is silent or the build differs:

* linear RGB: the IEC 61966-2-1 matrix applied to XYZ = T s (unclipped);
* the fit (``fit``) is full-batch Adam in float64 on the two latent terms
  only (MSE + 0.3 mean max-abs), PyTorch-style uniform initialisation, a
  fixed step count and a step size halved on plateaus; the colour term and
  the paper's AdamW schedule are not reproduced.  The weights are data for
  the inference kernel, not a parity target;
* kernel precision contract (``forward_f16``): the GPU runs the three layers
  on FP16 tensor cores with FP32 accumulation, so the colour, the three
  weight matrices and both hidden activations are rounded to f16
  (round-to-nearest-even from float32) before the layer that reads them, and
  the biases stay float32 (the kernel carries each as an f16 pair whose sum
  is the float32 value to about 2^-22 relative, far below the roundings
  here).  ``forward_f16`` applies the same roundings to the float64
  computation.  ``forward_bf16`` is the same contract with bf16 roundings (a
  coarser format that the kernel used to follow; kept as the bound the f16
  contract must beat).

Pins (tests/test_oracle_upsample.py): SiLU at closed-form points; brute-force
loops over a small network against the matrix form; zero output weights give
the output bias; a one-hidden-unit network evaluated by hand; central finite
differences of the loss gradient; the fit lowers the loss; forward_bf16 and
forward_f16 with the rounding switched off equal forward, and with it on stay
within their formats' error bounds of forward (f16's several times tighter).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import cmf, quant

HIDDEN = 128
MAXABS_WEIGHT = 0.3


def silu(x):
    """x * sigmoid(x), evaluated without overflow for large |x|."""
    x = np.asarray(x, dtype=np.float64)
    e = np.exp(-np.abs(x))
    sig = np.where(x >= 0, 1.0 / (1.0 + e), e / (1.0 + e))
    return x * sig


def silu_grad(x):
    x = np.asarray(x, dtype=np.float64)
    e = np.exp(-np.abs(x))
    sig = np.where(x >= 0, 1.0 / (1.0 + e), e / (1.0 + e))
    return sig * (1.0 + x * (1.0 - sig))


@dataclass
class Params:
    W1: np.ndarray  # (H, 3)
    b1: np.ndarray  # (H,)
    W2: np.ndarray  # (H, H)
    b2: np.ndarray  # (H,)
    W3: np.ndarray  # (k, H)
    b3: np.ndarray  # (k,)

    def arrays(self):
        return [self.W1, self.b1, self.W2, self.b2, self.W3, self.b3]


def init_params(k: int, hidden: int = HIDDEN, seed: int = 0) -> Params:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    rng = np.random.default_rng(seed)

    def lin(o, i):
        bound = 1.0 / np.sqrt(i)
        return rng.uniform(-bound, bound, (o, i)), rng.uniform(-bound, bound, o)

    W1, b1 = lin(hidden, 3)
    W2, b2 = lin(hidden, hidden)
    W3, b3 = lin(k, hidden)
    return Params(W1, b1, W2, b2, W3, b3)


def rgb_of_spectra(S, T):
    """Linear sRGB of row spectra S (m, n): XYZ_TO_SRGB (T s), unclipped."""
    return (np.asarray(S, dtype=np.float64) @ np.asarray(T, dtype=np.float64).T) @ cmf.XYZ_TO_SRGB.T


def forward(p: Params, C, keep=False):
    """z (m, k) for colours C (m, 3); with ``keep`` also the pre-activations
    and activations of both hidden layers."""
    C = np.asarray(C, dtype=np.float64)
    a1 = C @ p.W1.T + p.b1
    h1 = silu(a1)
    a2 = h1 @ p.W2.T + p.b2
    h2 = silu(a2)
    z = h2 @ p.W3.T + p.b3
    return (z, (a1, h1, a2, h2)) if keep else z


def forward_f16(p: Params, C, rounding: bool = True):
    """The kernel's precision contract (see the module docstring)."""
    return _forward_rounded(p, C, quant.round_f16, rounding)


def forward_bf16(p: Params, C, rounding: bool = True):
    """The same contract with bf16 roundings (see the module docstring)."""
    return _forward_rounded(p, C, quant.round_bf16, rounding)


def _forward_rounded(p: Params, C, rnd, rounding: bool):
    r = rnd if rounding else (lambda x: np.asarray(x, dtype=np.float64))
    b32 = (lambda x: np.asarray(x, dtype=np.float32).astype(np.float64)) if rounding else \
        (lambda x: np.asarray(x, dtype=np.float64))
    h1 = r(silu(r(C) @ r(p.W1).T + b32(p.b1)))
    h2 = r(silu(h1 @ r(p.W2).T + b32(p.b2)))
    return h2 @ r(p.W3).T + b32(p.b3)


def loss(p: Params, C, Z, maxabs=MAXABS_WEIGHT):
    """MSE over all code elements + maxabs * mean over samples of max_i |dz_i|."""
    d = forward(p, C) - np.asarray(Z, dtype=np.float64)
    return float(np.mean(d * d) + maxabs * np.mean(np.max(np.abs(d), axis=1)))


def gradient(p: Params, C, Z, maxabs=MAXABS_WEIGHT) -> Params:
    """Analytic gradient of ``loss`` (the max-abs term by its subgradient at
    the arg max of each sample)."""
    C = np.asarray(C, dtype=np.float64)
    z, (a1, h1, a2, h2) = forward(p, C, keep=True)
    d = z - np.asarray(Z, dtype=np.float64)
    m, k = d.shape
    dz = 2.0 * d / (m * k)
    j = np.argmax(np.abs(d), axis=1)
    dz[np.arange(m), j] += maxabs / m * np.sign(d[np.arange(m), j])
    gW3 = dz.T @ h2
    gb3 = dz.sum(axis=0)
    da2 = (dz @ p.W3) * silu_grad(a2)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    da1 = (da2 @ p.W2) * silu_grad(a1)
    gW1 = da1.T @ C
    gb1 = da1.sum(axis=0)
    return Params(gW1, gb1, gW2, gb2, gW3, gb3)


@dataclass
class FitLog:
    losses: list
    steps: int


def fit(C, Z, k: int, steps: int = 3000, lr: float = 2e-3, seed: int = 0, hidden: int = HIDDEN,
        plateau: int = 200):
    """Full-batch Adam (beta 0.9 / 0.999) on ``loss``; the step size halves
    when the loss has not improved for ``plateau`` steps."""
    p = init_params(k, hidden, seed)
    ms = [np.zeros_like(a) for a in p.arrays()]
    vs = [np.zeros_like(a) for a in p.arrays()]
    b1, b2, eps = 0.9, 0.999, 1e-8
    log, best, since = [], np.inf, 0
    for t in range(1, steps + 1):
        g = gradient(p, C, Z)
        new = []
        for a, ga, m_, v_ in zip(p.arrays(), g.arrays(), ms, vs):
            m_ *= b1
            m_ += (1 - b1) * ga
            v_ *= b2
            v_ += (1 - b2) * ga * ga
            mh = m_ / (1 - b1 ** t)
            vh = v_ / (1 - b2 ** t)
            new.append(a - lr * mh / (np.sqrt(vh) + eps))
        p = Params(*new)
        L = loss(p, C, Z)
        log.append(L)
        if L < best - 1e-12:
            best, since = L, 0
        else:
            since += 1
            if since >= plateau:
                lr *= 0.5
                since = 0
    return p, FitLog(log, steps)


def brute_force_forward(p: Params, c):
    """One colour through the network by explicit loops (small networks)."""
    H = len(p.b1)
    h1 = []
    for j in range(H):
        a = float(p.b1[j]) + sum(float(p.W1[j][i]) * float(c[i]) for i in range(3))
        h1.append(a / (1.0 + np.exp(-a)))
    h2 = []
    for j in range(H):
        a = float(p.b2[j]) + sum(float(p.W2[j][i]) * h1[i] for i in range(H))
        h2.append(a / (1.0 + np.exp(-a)))
    return [float(p.b3[o]) + sum(float(p.W3[o][j]) * h2[j] for j in range(H)) for o in range(len(p.b3))]
