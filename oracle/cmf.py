"""Colorimetry for the oracle (float64).  Test infrastructure only.

The paper projects spectra to colour with the CIE colour matching functions
(T_cmf in the colour loss, Sec. 4.3) and compares colours in CIELAB with
Delta E 76 (upsampler loss, Sec. 5.2) and CIE94 (codec selection, Sec. 4.5).
It does not say which CMF tabulation, white point or exposure it uses.  Read
here as:

* CMFs: the analytic multi-lobe piecewise-Gaussian fit of the CIE 1931 2-degree
  observer of Wyman, Sloan and Shirley, "Simple Analytic Approximations to the
  CIE XYZ Color Matching Functions", JCGT 2(2), 2013.
* Integration weights T[c, i] = cmf_c(lambda_i) * dlambda / sum_j ybar(lambda_j)
  * dlambda, so the constant unit spectrum has Y = 1 (equal-energy white).
* Lab reference white = T @ 1; Delta E 2000 per CIE 142-2001 as written out by
  Sharma, Wu and Dalal (2005), kL = kC = kH = 1; CIE94 with the graphic-arts
  constants (kL = 1, K1 = 0.045, K2 = 0.015), the first colour as reference.
* sRGB: the IEC 61966-2-1 XYZ -> linear sRGB matrix and transfer function.

Pins (tests/test_oracle_cmf.py): equal-energy white chromaticity near (1/3,
1/3) and ybar(555) near 1 (catch a dropped or mis-signed lobe); the fit within
0.012 of the tabulated CIE 1931 observer at five wavelengths; the sRGB matrix
maps D65 to equal RGB and the transfer function is continuous; Lab of the white
is (100, 0, 0), 18% grey has L* = 49.5, the linear segment has slope 903.3;
Delta E vanishes on equal colours, is symmetric (2000, 76), reduces to
|dL|/S_L on neutral pairs, and Delta E 2000 reproduces, in both orders, the
34 published conformance pairs of Sharma, Wu and Dalal (2005, Table 1;
tests/golden/ciede2000_sharma2005.json), which exercise the chroma, hue and
rotation terms and the hue-angle branch points.
"""
from __future__ import annotations

import numpy as np

# (amplitude, mu [nm], sigma below mu, sigma above mu) per lobe, from the
# multi-lobe fit of Wyman, Sloan and Shirley (2013).
XBAR_LOBES = ((1.056, 599.8, 37.9, 31.0), (0.362, 442.0, 16.0, 26.7), (-0.065, 501.1, 20.4, 26.2))
YBAR_LOBES = ((0.821, 568.8, 46.9, 40.5), (0.286, 530.9, 16.3, 31.1))
ZBAR_LOBES = ((1.217, 437.0, 11.8, 36.0), (0.681, 459.0, 26.0, 13.8))


def _lobe(lam, mu, s_lo, s_hi):
    lam = np.asarray(lam, dtype=np.float64)
    sigma = np.where(lam < mu, s_lo, s_hi)
    return np.exp(-0.5 * ((lam - mu) / sigma) ** 2)


def _cmf(lam, lobes):
    return sum(a * _lobe(lam, mu, s1, s2) for (a, mu, s1, s2) in lobes)


def xbar(lam):
    return _cmf(lam, XBAR_LOBES)


def ybar(lam):
    return _cmf(lam, YBAR_LOBES)


def zbar(lam):
    return _cmf(lam, ZBAR_LOBES)


def cmf_weights(lambda0: float, dlambda: float, n: int) -> np.ndarray:
    """T (3, n): CMFs at the grid samples times dlambda, divided by the
    Y-integral of the unit spectrum, so that Y(T @ 1) = 1."""
    lam = lambda0 + dlambda * np.arange(n, dtype=np.float64)
    raw = np.stack([xbar(lam), ybar(lam), zbar(lam)]) * dlambda
    return raw / raw[1].sum()


# IEC 61966-2-1: CIE XYZ -> linear sRGB.
XYZ_TO_SRGB = np.array([[3.2406, -1.5372, -0.4986],
                        [-0.9689, 1.8758, 0.0415],
                        [0.0557, -0.2040, 1.0570]], dtype=np.float64)


def srgb_oetf(c):
    """IEC 61966-2-1 transfer function for linear values in [0, 1]."""
    c = np.asarray(c, dtype=np.float64)
    lo = 12.92 * c
    hi = 1.055 * np.power(np.maximum(c, 0.0031308), 1.0 / 2.4) - 0.055
    return np.where(c <= 0.0031308, lo, hi)


def xyz_to_srgb(xyz):
    """(P,3) XYZ -> display sRGB in [0,1]: matrix, clamp to [0,1], transfer."""
    lin = np.asarray(xyz, dtype=np.float64) @ XYZ_TO_SRGB.T
    return srgb_oetf(np.clip(lin, 0.0, 1.0))


def srgb_to_u8(srgb):
    """Round-half-up quantisation of [0,1] display values to 0..255."""
    return np.floor(np.clip(srgb, 0.0, 1.0) * 255.0 + 0.5).astype(np.uint8)


# ----------------------------------------------------------------------------
# CIELAB and colour differences
# ----------------------------------------------------------------------------

_DELTA = 6.0 / 29.0


def _lab_f(t):
    t = np.asarray(t, dtype=np.float64)
    return np.where(t > _DELTA ** 3, np.cbrt(t), t / (3.0 * _DELTA ** 2) + 4.0 / 29.0)


def xyz_to_lab(xyz, white):
    """CIE 1976 L*a*b* of (P,3) XYZ relative to the reference white (3,)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    fx = _lab_f(xyz[:, 0] / white[0])
    fy = _lab_f(xyz[:, 1] / white[1])
    fz = _lab_f(xyz[:, 2] / white[2])
    return np.stack([116.0 * fy - 16.0, 500.0 * (fx - fy), 200.0 * (fy - fz)], axis=1)


def xyz_to_lab_rows(xyz, whites):
    """CIE 1976 L*a*b* of (P,3) XYZ, each row relative to its own white (P,3)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    w = np.asarray(whites, dtype=np.float64)
    fx = _lab_f(xyz[:, 0] / w[:, 0])
    fy = _lab_f(xyz[:, 1] / w[:, 1])
    fz = _lab_f(xyz[:, 2] / w[:, 2])
    return np.stack([116.0 * fy - 16.0, 500.0 * (fx - fy), 200.0 * (fy - fz)], axis=1)


def delta_e76(lab1, lab2):
    return np.sqrt(((np.asarray(lab1) - np.asarray(lab2)) ** 2).sum(axis=1))


def delta_e94(lab_ref, lab):
    """CIE94, graphic-arts weights; ``lab_ref`` is the reference colour."""
    L1, a1, b1 = lab_ref[:, 0], lab_ref[:, 1], lab_ref[:, 2]
    L2, a2, b2 = lab[:, 0], lab[:, 1], lab[:, 2]
    C1 = np.hypot(a1, b1)
    C2 = np.hypot(a2, b2)
    dL = L1 - L2
    dC = C1 - C2
    dH2 = np.maximum((a1 - a2) ** 2 + (b1 - b2) ** 2 - dC ** 2, 0.0)
    SC = 1.0 + 0.045 * C1
    SH = 1.0 + 0.015 * C1
    return np.sqrt(dL ** 2 + (dC / SC) ** 2 + dH2 / SH ** 2)


def delta_e2000(lab1, lab2):
    """CIEDE2000 with kL = kC = kH = 1, hue angles in degrees."""
    L1, a1, b1 = [np.asarray(lab1[:, i], dtype=np.float64) for i in range(3)]
    L2, a2, b2 = [np.asarray(lab2[:, i], dtype=np.float64) for i in range(3)]
    C1 = np.hypot(a1, b1)
    C2 = np.hypot(a2, b2)
    Cbar = 0.5 * (C1 + C2)
    Cbar7 = Cbar ** 7
    G = 0.5 * (1.0 - np.sqrt(Cbar7 / (Cbar7 + 25.0 ** 7)))
    ap1 = (1.0 + G) * a1
    ap2 = (1.0 + G) * a2
    Cp1 = np.hypot(ap1, b1)
    Cp2 = np.hypot(ap2, b2)
    hp1 = np.where((ap1 == 0) & (b1 == 0), 0.0, np.degrees(np.arctan2(b1, ap1)) % 360.0)
    hp2 = np.where((ap2 == 0) & (b2 == 0), 0.0, np.degrees(np.arctan2(b2, ap2)) % 360.0)

    dLp = L2 - L1
    dCp = Cp2 - Cp1
    prod = Cp1 * Cp2
    dh = hp2 - hp1
    dhp = np.where(prod == 0, 0.0,
                   np.where(np.abs(dh) <= 180.0, dh,
                            np.where(dh > 180.0, dh - 360.0, dh + 360.0)))
    dHp = 2.0 * np.sqrt(prod) * np.sin(np.radians(dhp) / 2.0)

    Lbp = 0.5 * (L1 + L2)
    Cbp = 0.5 * (Cp1 + Cp2)
    hsum = hp1 + hp2
    hbp = np.where(prod == 0, hsum,
                   np.where(np.abs(hp1 - hp2) <= 180.0, 0.5 * hsum,
                            np.where(hsum < 360.0, 0.5 * (hsum + 360.0), 0.5 * (hsum - 360.0))))
    T = (1.0 - 0.17 * np.cos(np.radians(hbp - 30.0)) + 0.24 * np.cos(np.radians(2.0 * hbp))
         + 0.32 * np.cos(np.radians(3.0 * hbp + 6.0)) - 0.20 * np.cos(np.radians(4.0 * hbp - 63.0)))
    dtheta = 30.0 * np.exp(-(((hbp - 275.0) / 25.0) ** 2))
    Cbp7 = Cbp ** 7
    RC = 2.0 * np.sqrt(Cbp7 / (Cbp7 + 25.0 ** 7))
    SL = 1.0 + 0.015 * (Lbp - 50.0) ** 2 / np.sqrt(20.0 + (Lbp - 50.0) ** 2)
    SC = 1.0 + 0.045 * Cbp
    SH = 1.0 + 0.015 * Cbp * T
    RT = -np.sin(np.radians(2.0 * dtheta)) * RC
    tL = dLp / SL
    tC = dCp / SC
    tH = dHp / SH
    return np.sqrt(np.maximum(tL ** 2 + tC ** 2 + tH ** 2 + RT * tC * tH, 0.0))
