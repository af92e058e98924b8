"""Linear non-negative Hadamard codec (float64).  Test infrastructure only.

Follows Sec. 4 of the paper:

* Eq. 4 (linear codec): z = E(s) = W_enc s with W_enc in R^{k x n};
  s_hat = D(z) = W_dec z with W_dec in R^{n x k}.
* Eq. 6 (blockwise Hadamard product): codes of length k = 3B are split into B
  blocks of three and multiplied block by block, the blocks concatenated.
* Eq. 8 (total loss) with its four terms L_e2e, L_rec, L_code, L_col
  (Sec. 4.3) and the selected weights lambda_e2e = 0.5, lambda_rec = 0.75,
  lambda_code = 1.0, lambda_col = 0.5 (Sec. 4.5).

Readings where the paper is silent:

* MSE is the mean over every element of the batch; the cosine in L_e2e is
  taken per sample along wavelength and averaged over the batch, and L_e2e is
  the product of the two batch means, as the formula is printed.
* Non-negativity: the paper parameterises W = softplus(W~) (Eq. 5) and trains
  with Adam; here E, D are kept non-negative by projection onto the
  non-negative orthant inside a projected-gradient method with Armijo
  backtracking, full batch, float64.  Both give non-negative weights; the fit
  output is data for the shading path, not a parity target.
* Initialisation: the n samples are split into k contiguous bands; row i of E
  averages band i and column i of D is band i's indicator (for k = n this is
  the identity, a fixed point with zero loss).

The paper's own parameterisation (softplus with beta = 10, Adam) is given by
``adam_softplus_step``: one bias-corrected Adam step on the raw parameters,
the gradient through the softplus by the chain rule.

Pins (tests/test_oracle_codec.py): exact linearity of encode/decode; the
blockwise product equals the element-wise product on R^k; central finite
differences of the total loss against the analytic gradient; monotone descent;
the identity codec at k = n has zero loss and stays put; weights and codes stay
non-negative; softplus closed forms and its inverse; finite differences of the
loss through the softplus; the first Adam step moves every parameter with a
non-zero gradient by lr against its sign.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

PAPER_WEIGHTS = {"e2e": 0.5, "rec": 0.75, "code": 1.0, "col": 0.5}


def encode(E, S):
    """Eq. 4 encoder on row spectra: S (m, n) -> codes (m, k)."""
    return np.asarray(S, dtype=np.float64) @ np.asarray(E, dtype=np.float64).T


def decode(D, Z):
    """Eq. 4 decoder on row codes: Z (m, k) -> spectra (m, n)."""
    return np.asarray(Z, dtype=np.float64) @ np.asarray(D, dtype=np.float64).T


def blockwise_hadamard(zr, zl):
    """Eq. 6: split both codes into B = k/3 blocks of three, multiply
    block-by-block and concatenate the blocks."""
    zr = np.asarray(zr, dtype=np.float64)
    zl = np.asarray(zl, dtype=np.float64)
    k = zr.shape[-1]
    if k % 3:
        raise ValueError("code length must be a multiple of 3")
    blocks = [zr[..., 3 * i:3 * i + 3] * zl[..., 3 * i:3 * i + 3] for i in range(k // 3)]
    return np.concatenate(blocks, axis=-1)


def band_init(k: int, n: int):
    """Band initialisation: n samples split into k contiguous bands."""
    edges = np.linspace(0, n, k + 1)
    E = np.zeros((k, n))
    D = np.zeros((n, k))
    for i in range(k):
        lo, hi = int(round(edges[i])), int(round(edges[i + 1]))
        hi = max(hi, lo + 1)
        E[i, lo:hi] = 1.0 / (hi - lo)
        D[lo:hi, i] = 1.0
    return E, D


@dataclass
class Batch:
    """Training pairs: reflectance rows R, scaled light rows L, and the CMF
    weights T (3, n) used by the colour term."""
    R: np.ndarray
    L: np.ndarray
    T: np.ndarray


def make_batch(ts, T) -> Batch:
    R = ts.R[ts.pair_r].astype(np.float64)
    L = ts.L[ts.pair_l].astype(np.float64) * ts.pair_scale[:, None]
    return Batch(R, L, np.asarray(T, dtype=np.float64))


def _mse(a, b):
    return float(np.mean((a - b) ** 2))


def _rowcos(a, b):
    na = np.linalg.norm(a, axis=1)
    nb = np.linalg.norm(b, axis=1)
    return (a * b).sum(axis=1) / (na * nb)


def losses(E, D, batch: Batch, w=PAPER_WEIGHTS):
    """Eq. 8 and its four terms (Sec. 4.3) on a batch of pairs."""
    R, L, T = batch.R, batch.L, batch.T
    zR, zL = encode(E, R), encode(E, L)
    zRL = blockwise_hadamard(zR, zL)
    S_hat = decode(D, zRL)
    Y = R * L
    e2e = _mse(S_hat, Y) * (2.0 - float(np.mean(_rowcos(S_hat, Y))))
    rec = _mse(decode(D, zR), R) + _mse(decode(D, zL), L)
    code = _mse(zRL, encode(E, Y))
    col = _mse(S_hat @ T.T, Y @ T.T)
    total = w["e2e"] * e2e + w["rec"] * rec + w["code"] * code + w["col"] * col
    return {"total": total, "e2e": e2e, "rec": rec, "code": code, "col": col}


def total_loss(E, D, batch, w=PAPER_WEIGHTS):
    return losses(E, D, batch, w)["total"]


def gradient(E, D, batch: Batch, w=PAPER_WEIGHTS):
    """Analytic gradient of Eq. 8 with respect to (E, D), by the chain rule
    through S_hat = D(E R (.) E L) and the four terms."""
    R, L, T = batch.R, batch.L, batch.T
    P, n = R.shape
    k = E.shape[0]
    zR, zL = R @ E.T, L @ E.T
    zRL = zR * zL
    S = zRL @ D.T
    Y = R * L
    N = P * n
    gE = np.zeros_like(E)
    gD = np.zeros_like(D)

    # L_e2e = m * (2 - c),  m = MSE(S, Y),  c = mean_p cos(S_p, Y_p)
    e = S - Y
    m = float(np.sum(e * e)) / N
    nS = np.linalg.norm(S, axis=1)
    nY = np.linalg.norm(Y, axis=1)
    cos = (S * Y).sum(axis=1) / (nS * nY)
    c = float(np.mean(cos))
    dm_dS = 2.0 * e / N
    dc_dS = (Y / (nS * nY)[:, None] - cos[:, None] * S / (nS ** 2)[:, None]) / P
    gS = w["e2e"] * ((2.0 - c) * dm_dS - m * dc_dS)

    # L_col = MSE(S T^T, Y T^T) over (P, 3)
    gS += w["col"] * 2.0 * ((S - Y) @ T.T) @ T / (3 * P)

    # S = zRL D^T
    gD += gS.T @ zRL
    g_zRL = gS @ D

    # L_code = MSE(zRL, Y E^T) over (P, k)
    rc = zRL - Y @ E.T
    g_rc = w["code"] * 2.0 * rc / (P * k)
    g_zRL += g_rc
    gE -= g_rc.T @ Y

    g_zR = g_zRL * zL
    g_zL = g_zRL * zR

    # L_rec = MSE(zR D^T, R) + MSE(zL D^T, L)
    for z, X, gz in ((zR, R, g_zR), (zL, L, g_zL)):
        r = z @ D.T - X
        g_r = w["rec"] * 2.0 * r / N
        gD += g_r.T @ z
        gz += g_r @ D

    gE += g_zR.T @ R + g_zL.T @ L
    return gE, gD


@dataclass
class FitResult:
    E: np.ndarray
    D: np.ndarray
    history: list
    iterations: int
    proj_grad_inf: float


def projected_gradient_fit(batch: Batch, k: int, iters: int = 5000, w=PAPER_WEIGHTS,
                           tol: float = 1e-8, armijo_c: float = 1e-4, shrink: float = 0.5,
                           E0=None, D0=None, step0: float = 1.0) -> FitResult:
    """Minimise Eq. 8 over E >= 0, D >= 0 by projected gradient with Armijo
    backtracking along the projection arc.  The trial step of each iteration
    is the Barzilai-Borwein step <s,s>/<s,y> of the last accepted move (first
    iteration: ``step0``); it is halved until
    f(P(x - a g)) <= f(x) + c g.(P(x - a g) - x), so the loss never increases.
    Stops when the projected-gradient infinity norm drops below ``tol`` times
    its initial value or after ``iters`` iterations."""
    n = batch.R.shape[1]
    E, D = (band_init(k, n) if E0 is None else (np.array(E0, float), np.array(D0, float)))
    f = total_loss(E, D, batch, w)
    hist = [f]
    step = step0
    pg0 = None
    pg = 0.0
    it = 0
    gE, gD = gradient(E, D, batch, w)
    for it in range(1, iters + 1):
        # projected gradient: drop components that push out of the orthant at a bound
        pE = np.where((E <= 0) & (gE > 0), 0.0, gE)
        pD = np.where((D <= 0) & (gD > 0), 0.0, gD)
        pg = max(np.abs(pE).max(), np.abs(pD).max())
        if pg0 is None:
            pg0 = pg
        if pg0 == 0.0 or pg <= tol * pg0:
            break
        a = step
        while True:
            En = np.maximum(E - a * gE, 0.0)
            Dn = np.maximum(D - a * gD, 0.0)
            fn = total_loss(En, Dn, batch, w)
            dec = float((gE * (En - E)).sum() + (gD * (Dn - D)).sum())
            if fn <= f + armijo_c * dec or a < 1e-30:
                break
            a *= shrink
        if a < 1e-30 or dec == 0.0:
            break
        gEn, gDn = gradient(En, Dn, batch, w)
        sy = float(((En - E) * (gEn - gE)).sum() + ((Dn - D) * (gDn - gD)).sum())
        ss = float(((En - E) ** 2).sum() + ((Dn - D) ** 2).sum())
        step = min(max(ss / sy, 1e-10), 1e10) if sy > 0 else a * 2.0
        E, D, f, gE, gD = En, Dn, fn, gEn, gDn
        hist.append(f)
    return FitResult(E, D, hist, it, float(pg))


# ----------------------------------------------------------------------------
# The paper's parameterisation (Sec. 4.1-4.5): W = softplus_beta(W~) with
# beta = 10, Adam on mini-batches.  One step, as the batched GPU sweep takes it.
# ----------------------------------------------------------------------------

SOFTPLUS_BETA = 10.0


def softplus(x, beta=SOFTPLUS_BETA):
    """log(1 + exp(beta x)) / beta, evaluated without overflow."""
    bx = beta * np.asarray(x, dtype=np.float64)
    return (np.maximum(bx, 0.0) + np.log1p(np.exp(-np.abs(bx)))) / beta


def softplus_grad(x, beta=SOFTPLUS_BETA):
    """d softplus / dx = sigmoid(beta x)."""
    bx = beta * np.asarray(x, dtype=np.float64)
    e = np.exp(-np.abs(bx))
    return np.where(bx >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def softplus_inverse(y, beta=SOFTPLUS_BETA):
    """x with softplus(x) = y > 0."""
    by = beta * np.asarray(y, dtype=np.float64)
    return (by + np.log(-np.expm1(-by))) / beta


@dataclass
class AdamState:
    mE: np.ndarray
    vE: np.ndarray
    mD: np.ndarray
    vD: np.ndarray
    t: int = 0


def adam_init(Et, Dt) -> AdamState:
    return AdamState(np.zeros_like(Et), np.zeros_like(Et), np.zeros_like(Dt), np.zeros_like(Dt), 0)


def adam_softplus_step(Et, Dt, st: AdamState, batch: Batch, w=PAPER_WEIGHTS, lr: float = 1e-3,
                       b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8, beta: float = SOFTPLUS_BETA):
    """One Adam step (bias-corrected moments) on the raw parameters (E~, D~)
    of E = softplus(E~), D = softplus(D~) for the Eq. 8 loss on ``batch``;
    returns the new (E~, D~, state) and the loss terms at the old parameters."""
    E, D = softplus(Et, beta), softplus(Dt, beta)
    parts = losses(E, D, batch, w)
    gE, gD = gradient(E, D, batch, w)
    g = (gE * softplus_grad(Et, beta), gD * softplus_grad(Dt, beta))
    t = st.t + 1
    out = []
    moments = ((st.mE, st.vE), (st.mD, st.vD))
    new_m = []
    for x, gx, (m, v) in zip((Et, Dt), g, moments):
        m = b1 * m + (1 - b1) * gx
        v = b2 * v + (1 - b2) * gx * gx
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        out.append(x - lr * mh / (np.sqrt(vh) + eps))
        new_m.append((m, v))
    return out[0], out[1], AdamState(new_m[0][0], new_m[0][1], new_m[1][0], new_m[1][1], t), parts
