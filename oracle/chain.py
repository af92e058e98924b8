"""Multi-bounce chains in spectral and latent space (float64).
Test infrastructure only.

Sec. 4.5 of the paper selects its codec with a synthetic b-bounce proxy: a
light L is multiplied by a fresh reflectance at every bounce,
S(1) = R(1) (.) L, S(b) = R(b) (.) S(b-1), the same recurrence runs in latent
space with the blockwise product of Eq. 6, and the two are compared per depth
by CIE94 colour difference.  Here both chains are taken to colour with the
CMF weights T; the latent chain is decoded with D first (T (D z)).

Reading where the paper is silent: each chain's colours are scaled by
1 / max(T L), so that the largest tristimulus value of its light is 1, and
converted to CIELAB with the equal-energy white T @ 1 (Yn = 1).  The paper's
chain errors are a few Delta E, which presumes colours in a bounded range:
taking the light's own T L as the white makes Lab degenerate for narrow-band
lights near the ends of the grid (X or Z near zero), and scaling by the
luminance Y(T L) alone leaves such lights with X / Y or Z / Y in the
hundreds.  A light with max(T L) <= 0 has no colour; its chains get Delta E 0.
CIE94 takes the spectral chain as reference; Delta E 2000 and the
nearest-rank p95 are reported beside the means.

Pins (tests/test_oracle_chain.py): the identity codec (k = n) makes every
latent chain equal its spectral chain (Delta E 0); the exposure maps every
light's largest tristimulus value to 1 and is invariant to the light's
intensity, so Delta E is too; constant reflectances rho
under an equal-energy light give S(b) = rho^b, whose L* is 116 (rho^b)^(1/3)
- 16 with a* = b* = 0; an all-ones chain under that light is the white
(100, 0, 0); brute-force loops on tiny inputs.
"""
from __future__ import annotations

import numpy as np

from . import cmf, codec


def chain_xyz(R, L, E, D, T, chain_light, chain_refl):
    """XYZ of every chain at every depth.

    R (N_R, n), L (N_L, n): spectra; chain_light (C,), chain_refl (C, depth):
    indices.  Returns xyz_spec (C, depth, 3), xyz_lat (C, depth, 3),
    white (C, 3) = T L."""
    R = np.asarray(R, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    cl = np.asarray(chain_light)
    cr = np.asarray(chain_refl)
    C, depth = cr.shape
    zR = codec.encode(E, R)
    zL = codec.encode(E, L)
    s = L[cl]
    z = zL[cl]
    xs = np.empty((C, depth, 3))
    xl = np.empty((C, depth, 3))
    for b in range(depth):
        s = R[cr[:, b]] * s
        z = codec.blockwise_hadamard(zR[cr[:, b]], z)
        xs[:, b] = s @ T.T
        xl[:, b] = codec.decode(D, z) @ T.T
    return xs, xl, L[cl] @ T.T


def exposure(light_xyz):
    """Per-chain colour scale 1 / max(X, Y, Z) of the light; 0 for a light
    with no positive tristimulus value."""
    m = np.asarray(light_xyz, dtype=np.float64).max(axis=1)
    return np.where(m > 0.0, 1.0 / np.where(m > 0.0, m, 1.0), 0.0)


def chain_delta_e(R, L, E, D, T, chain_light, chain_refl):
    """Per-depth Delta E of the latent chain against the spectral chain:
    dict with (depth, C) arrays 'de94', 'de2000' and per-depth lists of the
    means and nearest-rank p95s."""
    from . import metrics
    xs, xl, light_xyz = chain_xyz(R, L, E, D, T, chain_light, chain_refl)
    C, depth, _ = xs.shape
    white = np.asarray(T, dtype=np.float64).sum(axis=1)
    scale = exposure(light_xyz)
    de94 = np.empty((depth, C))
    de00 = np.empty((depth, C))
    for b in range(depth):
        lab_s = cmf.xyz_to_lab(xs[:, b] * scale[:, None], white)
        lab_l = cmf.xyz_to_lab(xl[:, b] * scale[:, None], white)
        de94[b] = cmf.delta_e94(lab_s, lab_l)
        de00[b] = cmf.delta_e2000(lab_s, lab_l)
    return {"de94": de94, "de2000": de00,
            "de94_mean": [float(de94[b].mean()) for b in range(depth)],
            "de2000_mean": [float(de00[b].mean()) for b in range(depth)],
            "de94_p95": [metrics.nearest_rank(de94[b]) for b in range(depth)],
            "de2000_p95": [metrics.nearest_rank(de00[b]) for b in range(depth)]}


def brute_force_chain_xyz(R, L, E, D, T, light, refls):
    """One chain by explicit loops: returns (xyz_spec, xyz_lat) per depth."""
    n = len(L[light])
    k = len(E)
    s = [float(v) for v in L[light]]
    z = [sum(float(E[c][i]) * s[i] for i in range(n)) for c in range(k)]
    out_s, out_l = [], []
    for r in refls:
        s = [float(R[r][i]) * s[i] for i in range(n)]
        zr = [sum(float(E[c][i]) * float(R[r][i]) for i in range(n)) for c in range(k)]
        z = [zr[c] * z[c] for c in range(k)]
        spec = [sum(float(D[i][c]) * z[c] for c in range(k)) for i in range(n)]
        out_s.append([sum(float(T[j][i]) * s[i] for i in range(n)) for j in range(3)])
        out_l.append([sum(float(T[j][i]) * spec[i] for i in range(n)) for j in range(3)])
    return out_s, out_l
