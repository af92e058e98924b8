"""Deferred G-buffer shading in spectral and latent space (float64).
Test infrastructure only.

The paper renders with an unmodified path tracer (Sec. 6.1): the spectral
ground truth propagates all n wavelength samples; the latent render packs the
k-code into k/3 RGB triplets, renders k/3 passes, reassembles the k-channel
latent image and decodes it once (Fig. 2b).  Light-material interaction is the
element-wise product (Sec. 3 item 3), which Eq. 6 replaces by the blockwise
Hadamard product of codes; light sums and scalings stay exact because the codec
is linear (Eq. 4).

The paper does not fix a shading model for a G-buffer.  Read here as:

* point lights l at p_l with intensity I_l and unit-peak SPD spd_l, Lambert
  BRDF rho/pi, inverse-square falloff, no visibility (a G-buffer carries
  none):  E_s(x, n) = sum_l I_l max(0, n.(p_l - x)) / |p_l - x|^3 spd_l;
* one indirect bounce through a secondary G-buffer point (x2, n2, m2) treated
  as a virtual point light with clamp eps = 1e-2:
  h12 = max(0, n1.d) max(0, -n2.d) / (|d|^2 max(|d|^2, eps)),  d = x2 - x1;
* spectral radiance  S = (R_m1/pi) (.) [E_s(x1,n1) + h12 (R_m2/pi) (.) E_s(x2,n2)];
* latent radiance: the same formula with every spectrum replaced by its code
  (R -> E R, spd -> E spd) and (.) by the blockwise product of Eq. 6;
  XYZ_latent = T (D z), decoded unfolded.

Pins (tests/test_oracle_shade.py): k = n identity codec makes latent equal
spectral; one light above a facing pixel with constant spectra gives the closed
form rho I / (pi h^2), and a hand-built two-point bounce gives its closed form;
brute-force per-pixel loops of the unfactored sum match the vectorised forms on
4x4 images; the k/3-pass form equals the fused form; codes, latent image and
decoded spectra are non-negative.
"""
from __future__ import annotations

import math

import numpy as np

from . import codec

EPS_BOUNCE = 1e-2


def geometry(x, nrm, light_pos):
    """g[p, l] = max(0, n_p.(p_l - x_p)) / |p_l - x_p|^3, shape (P, L)."""
    x = np.asarray(x, dtype=np.float64)
    nrm = np.asarray(nrm, dtype=np.float64)
    lp = np.asarray(light_pos, dtype=np.float64)
    d = lp[None, :, :] - x[:, None, :]
    r2 = (d * d).sum(axis=2)
    cosang = np.maximum(0.0, (nrm[:, None, :] * d).sum(axis=2))
    return cosang / (r2 * np.sqrt(r2))


def bounce_factor(x1, n1, x2, n2, eps=EPS_BOUNCE):
    """Virtual-point-light transfer from the secondary point to the primary."""
    x1 = np.asarray(x1, dtype=np.float64)
    x2 = np.asarray(x2, dtype=np.float64)
    d = x2 - x1
    dd = (d * d).sum(axis=1)
    c1 = np.maximum(0.0, (np.asarray(n1, dtype=np.float64) * d).sum(axis=1))
    c2 = np.maximum(0.0, -(np.asarray(n2, dtype=np.float64) * d).sum(axis=1))
    return c1 * c2 / (dd * np.maximum(dd, eps))


def irradiance(x, nrm, light_pos, light_intensity, light_vals):
    """E_s at each point: sum_l I_l g_l light_vals_l, shape (P, C) for light
    values of C channels (spectral samples or code channels)."""
    g = geometry(x, nrm, light_pos) * np.asarray(light_intensity, dtype=np.float64)[None, :]
    return g @ np.asarray(light_vals, dtype=np.float64)


def _radiance(refl1, irr1, h12=None, refl2=None, irr2=None, product=np.multiply):
    """(R1/pi) (.) [E1 + h12 (R2/pi) (.) E2] with a pluggable product."""
    inner = irr1
    if h12 is not None:
        inner = irr1 + h12[:, None] * product(refl2 / math.pi, irr2)
    return product(refl1 / math.pi, inner)


def shade_spectral(frame, want_spectra=True):
    """Naive n-sample shading of a frame: returns (S (P,n) or None, XYZ (P,3))."""
    from . import cmf
    mats = frame.mat_spectra.astype(np.float64)
    spd = frame.light_spd.astype(np.float64)
    g1 = frame.g1
    irr1 = irradiance(g1.pos, g1.normal, frame.light_pos, frame.light_intensity, spd)
    if frame.g2 is not None:
        g2 = frame.g2
        irr2 = irradiance(g2.pos, g2.normal, frame.light_pos, frame.light_intensity, spd)
        h12 = bounce_factor(g1.pos, g1.normal, g2.pos, g2.normal)
        S = _radiance(mats[g1.mat], irr1, h12, mats[g2.mat], irr2)
    else:
        S = _radiance(mats[g1.mat], irr1)
    T = cmf.cmf_weights(*frame.grid)
    return (S if want_spectra else None), S @ T.T


def material_codes(E, frame):
    return codec.encode(E, frame.mat_spectra)


def light_codes(E, frame):
    return codec.encode(E, frame.light_spd)


def shade_latent(frame, E, zmat=None, zlight=None):
    """Fused k-channel latent shading: returns the latent image z (P, k).
    ``zmat``/``zlight`` override the codes (e.g. storage-rounded codes)."""
    zm = material_codes(E, frame) if zmat is None else np.asarray(zmat, dtype=np.float64)
    zl = light_codes(E, frame) if zlight is None else np.asarray(zlight, dtype=np.float64)
    g1 = frame.g1
    a1 = irradiance(g1.pos, g1.normal, frame.light_pos, frame.light_intensity, zl)
    if frame.g2 is None:
        return _radiance(zm[g1.mat], a1, product=codec.blockwise_hadamard)
    g2 = frame.g2
    a2 = irradiance(g2.pos, g2.normal, frame.light_pos, frame.light_intensity, zl)
    h12 = bounce_factor(g1.pos, g1.normal, g2.pos, g2.normal)
    return _radiance(zm[g1.mat], a1, h12, zm[g2.mat], a2, product=codec.blockwise_hadamard)


def shade_latent_passes(frame, E, zmat=None, zlight=None):
    """k/3-pass form (Fig. 2b): pass b shades code channels 3b..3b+2 as an RGB
    image; returns the list of B pass images (P, 3) and their reassembly into
    the k-channel latent image."""
    zm = material_codes(E, frame) if zmat is None else np.asarray(zmat, dtype=np.float64)
    zl = light_codes(E, frame) if zlight is None else np.asarray(zlight, dtype=np.float64)
    B = zm.shape[1] // 3
    passes = []
    g1 = frame.g1
    for b in range(B):
        sl = slice(3 * b, 3 * b + 3)
        a1 = irradiance(g1.pos, g1.normal, frame.light_pos, frame.light_intensity, zl[:, sl])
        if frame.g2 is None:
            img = _radiance(zm[g1.mat][:, sl], a1)
        else:
            g2 = frame.g2
            a2 = irradiance(g2.pos, g2.normal, frame.light_pos, frame.light_intensity, zl[:, sl])
            h12 = bounce_factor(g1.pos, g1.normal, g2.pos, g2.normal)
            img = _radiance(zm[g1.mat][:, sl], a1, h12, zm[g2.mat][:, sl], a2)
        passes.append(img)
    return passes, reassemble(passes)


def reassemble(passes):
    """B images (P, 3) -> latent image (P, 3B): pass b fills channels 3b..3b+2."""
    P = passes[0].shape[0]
    z = np.empty((P, 3 * len(passes)))
    for b, img in enumerate(passes):
        z[:, 3 * b:3 * b + 3] = img
    return z


def decode_xyz(z, D, T):
    """XYZ of a latent image, decoded to spectra first: T (D z)."""
    return codec.decode(D, z) @ np.asarray(T, dtype=np.float64).T


# ----------------------------------------------------------------------------
# Brute force (pure Python loops, unfactored) for tiny frames
# ----------------------------------------------------------------------------

def brute_force_spectral(frame):
    """Per pixel, per light, per wavelength, unfactored:
    S(lam) = sum_l [R1 I_l g_l(x1) spd_l / pi] + h12 sum_l [R1 R2 I_l g_l(x2) spd_l / pi^2]."""
    n = frame.n
    P = frame.pixels
    out = np.zeros((P, n))
    for p in range(P):
        x1 = [float(v) for v in frame.g1.pos[p]]
        n1 = [float(v) for v in frame.g1.normal[p]]
        m1 = int(frame.g1.mat[p])
        if frame.g2 is not None:
            x2 = [float(v) for v in frame.g2.pos[p]]
            n2 = [float(v) for v in frame.g2.normal[p]]
            m2 = int(frame.g2.mat[p])
            d = [x2[i] - x1[i] for i in range(3)]
            dd = sum(v * v for v in d)
            h = max(0.0, sum(n1[i] * d[i] for i in range(3))) * \
                max(0.0, -sum(n2[i] * d[i] for i in range(3))) / (dd * max(dd, EPS_BOUNCE))
        for lam in range(n):
            s = 0.0
            for l in range(frame.lights):
                pl = [float(v) for v in frame.light_pos[l]]
                I = float(frame.light_intensity[l])
                sp = float(frame.light_spd[l, lam])
                r1 = float(frame.mat_spectra[m1, lam])
                dv = [pl[i] - x1[i] for i in range(3)]
                r2 = sum(v * v for v in dv)
                c = max(0.0, sum(n1[i] * dv[i] for i in range(3)))
                s += r1 * I * c / r2 ** 1.5 * sp / math.pi
                if frame.g2 is not None:
                    rr2 = float(frame.mat_spectra[m2, lam])
                    dv2 = [pl[i] - x2[i] for i in range(3)]
                    q2 = sum(v * v for v in dv2)
                    c2 = max(0.0, sum(n2[i] * dv2[i] for i in range(3)))
                    s += h * r1 * rr2 * I * c2 / q2 ** 1.5 * sp / math.pi ** 2
            out[p, lam] = s
    return out


def brute_force_latent(frame, E):
    """Per pixel, per light, per code channel, unfactored, with codes
    computed by explicit sums z_c = sum_i E[c, i] s_i."""
    k, n = E.shape
    E = np.asarray(E, dtype=np.float64)

    def code(s):
        return [sum(float(E[c, i]) * float(s[i]) for i in range(n)) for c in range(k)]

    zm = [code(frame.mat_spectra[m]) for m in range(frame.mat_spectra.shape[0])]
    zl = [code(frame.light_spd[l]) for l in range(frame.lights)]
    P = frame.pixels
    out = np.zeros((P, k))
    for p in range(P):
        x1 = [float(v) for v in frame.g1.pos[p]]
        n1 = [float(v) for v in frame.g1.normal[p]]
        m1 = int(frame.g1.mat[p])
        if frame.g2 is not None:
            x2 = [float(v) for v in frame.g2.pos[p]]
            n2 = [float(v) for v in frame.g2.normal[p]]
            m2 = int(frame.g2.mat[p])
            d = [x2[i] - x1[i] for i in range(3)]
            dd = sum(v * v for v in d)
            h = max(0.0, sum(n1[i] * d[i] for i in range(3))) * \
                max(0.0, -sum(n2[i] * d[i] for i in range(3))) / (dd * max(dd, EPS_BOUNCE))
        for c in range(k):
            s = 0.0
            for l in range(frame.lights):
                pl = [float(v) for v in frame.light_pos[l]]
                I = float(frame.light_intensity[l])
                dv = [pl[i] - x1[i] for i in range(3)]
                r2 = sum(v * v for v in dv)
                cc = max(0.0, sum(n1[i] * dv[i] for i in range(3)))
                s += zm[m1][c] * I * cc / r2 ** 1.5 * zl[l][c] / math.pi
                if frame.g2 is not None:
                    dv2 = [pl[i] - x2[i] for i in range(3)]
                    q2 = sum(v * v for v in dv2)
                    c2 = max(0.0, sum(n2[i] * dv2[i] for i in range(3)))
                    s += h * zm[m1][c] * zm[m2][c] * I * c2 / q2 ** 1.5 * zl[l][c] / math.pi ** 2
            out[p, c] = s
    return out
