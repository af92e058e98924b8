"""Path tracing in spectral and in latent code space.  Test infrastructure only.

The paper renders its latent images with a path tracer (Sec. 6.1; multi-bounce
results, Fig. of 1, 2, 3 and unbounded bounces): every spectrum is replaced by
its code, the path throughput is multiplied by the material codes with the
blockwise product (Eq. 6) at each interaction, the emission is added where a
path meets a light, and the image is decoded once at the end.  This module
traces a Cornell-box stand-in (hsc_inputs.cornell_scene):

* Lambertian surfaces and one emitting rectangle (emission only, no
  reflection); camera rays through jittered pixel positions;
* cosine-weighted bounce directions, so every reflection multiplies the
  throughput by the reflectance exactly (estimator weight rho);
* a path ends when it meets the emitter (after j reflections, j >= 0), leaves
  the box, or has made D reflections without meeting the emitter;
* pixel value = mean over samples of E (.) rho_{m_0} (.) ... (.) rho_{m_{j-1}}
  for paths that met the emitter; the latent form uses the codes and the
  blockwise product, then XYZ = T (D z).

Reading where the paper is silent: no Russian roulette and no next-event
estimation (the paper's path tracer settings are Mitsuba's; the simplest
unbiased estimator is taken here); a depth bound D in place of Mitsuba's
maxDepth.

Determinism shared with the CUDA kernel (so both trace identical paths and
only the radiance along them is compared):

* geometry in IEEE float32 with every operation rounded to nearest, in a fixed
  order, without fused multiply-adds; square roots and divisions correctly
  rounded;
* random numbers from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), one
  call per path vertex with counter (pixel, sample, vertex, 0) and key
  (seed, 0); u = (x >> 8) * 2^-24;
* the bounce direction: r = sqrt(u1), phi = 2 pi u2 with sin and cos of phi
  from Taylor polynomials on a quarter turn, rotated by quadrant;
* the tangent frame of a normal by the branchless construction of Duff et
  al., "Building an Orthonormal Basis, Revisited", JCGT 6(1), 2017;
* the nearest hit with t > 1e-4 over the rectangles then the spheres in
  order, strict comparison; a new ray starts 1e-3 along the normal.

Pins (tests/test_oracle_pathtrace.py): Philox known-answer vectors
(tests/golden/philox4x32_10_kat.json); the sin/cos polynomials against the
library within 1e-6; orthonormal frames; the mean cosine of cosine-weighted
samples is 2/3; closed-form ray-plane and ray-sphere hits; a per-path scalar
tracer written with explicit loops gives the same paths; pixels that see the
emitter directly equal T E; one more bounce never lowers a pixel; the
identity codec makes the latent image equal the spectral one.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

F = np.float32
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)
T_MIN = F(1e-4)
OFFSET = F(1e-3)
STREAM = np.uint32(0)  # fourth counter word


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 arrays (counter words c0..c3, key
    words k0, k1); returns the four output words."""
    c = [np.asarray(x, dtype=np.uint32).copy() for x in (c0, c1, c2, c3)]
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    mask = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = np.uint32((int(k0) + int(PHILOX_W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(PHILOX_W1)) & 0xFFFFFFFF)
        p0 = PHILOX_M0 * c[0].astype(np.uint64)
        p1 = PHILOX_M1 * c[2].astype(np.uint64)
        hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
        lo0 = (p0 & mask).astype(np.uint32)
        hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
        lo1 = (p1 & mask).astype(np.uint32)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def u01(x):
    """uint32 -> float32 in [0, 1): the top 24 bits times 2^-24 (exact)."""
    return (np.asarray(x, dtype=np.uint32) >> np.uint32(8)).astype(F) * F(1.0 / 16777216.0)


# Taylor coefficients of sin and cos as float32 quotients (rounded once).
_S = [F(1.0) / F(6.0), F(1.0) / F(120.0), F(1.0) / F(5040.0), F(1.0) / F(362880.0), F(1.0) / F(39916800.0)]
_C = [F(1.0) / F(2.0), F(1.0) / F(24.0), F(1.0) / F(720.0), F(1.0) / F(40320.0), F(1.0) / F(3628800.0),
      F(1.0) / F(479001600.0)]
HALF_PI = F(np.pi / 2)


def sincos_turn(u):
    """(sin, cos) of 2 pi u for float32 u in [0, 1): quarter-turn quadrant
    q = floor(4u), angle (4u - q) pi/2 on Taylor polynomials (Horner form,
    alternating signs), rotated by q."""
    u = np.asarray(u, dtype=F)
    x4 = u * F(4.0)
    q = np.floor(x4).astype(np.int32)
    th = (x4 - q.astype(F)) * HALF_PI
    t2 = th * th
    s = F(1.0) - t2 * (_S[0] - t2 * (_S[1] - t2 * (_S[2] - t2 * (_S[3] - t2 * _S[4]))))
    s = th * s
    c = F(1.0) - t2 * (_C[0] - t2 * (_C[1] - t2 * (_C[2] - t2 * (_C[3] - t2 * (_C[4] - t2 * _C[5])))))
    sn = np.where(q == 0, s, np.where(q == 1, c, np.where(q == 2, -s, -c)))
    cs = np.where(q == 0, c, np.where(q == 1, -s, np.where(q == 2, -c, s)))
    return sn.astype(F), cs.astype(F)


def onb(nx, ny, nz):
    """Tangents (b1, b2) of unit normals, Duff et al. 2017, float32."""
    nx, ny, nz = (np.asarray(v, dtype=F) for v in (nx, ny, nz))
    sign = np.where(nz >= F(0.0), F(1.0), F(-1.0)).astype(F)
    a = F(-1.0) / (sign + nz)
    b = nx * ny * a
    b1 = (F(1.0) + sign * (nx * nx) * a, sign * b, -(sign * nx))
    b2 = (b, sign + (ny * ny) * a, -ny)
    return b1, b2


def intersect(scene, ox, oy, oz, dx, dy, dz):
    """Nearest hit with t > T_MIN: (t, kind, index) with kind 0 = rectangle,
    1 = sphere, -1 = none; float32, objects in order, strict comparison."""
    o = [np.asarray(v, dtype=F) for v in (ox, oy, oz)]
    d = [np.asarray(v, dtype=F) for v in (dx, dy, dz)]
    n = o[0].shape
    best = np.full(n, np.inf, dtype=F)
    kind = np.full(n, -1, dtype=np.int32)
    idx = np.full(n, -1, dtype=np.int32)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        for i, qd in enumerate(scene.quads):
            ax = int(qd[0])
            ua, va = [a for a in range(3) if a != ax]
            t = (F(qd[1]) - o[ax]) / d[ax]
            pu = o[ua] + t * d[ua]
            pv = o[va] + t * d[va]
            ok = (t > T_MIN) & (t < best) & (pu >= F(qd[2])) & (pu <= F(qd[3])) & (pv >= F(qd[4])) & (pv <= F(qd[5]))
            best = np.where(ok, t, best)
            kind = np.where(ok, 0, kind)
            idx = np.where(ok, i, idx)
        for i, sp in enumerate(scene.spheres):
            ocx, ocy, ocz = o[0] - F(sp[0]), o[1] - F(sp[1]), o[2] - F(sp[2])
            A = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
            B = (ocx * d[0] + ocy * d[1]) + ocz * d[2]
            C = ((ocx * ocx + ocy * ocy) + ocz * ocz) - F(sp[3]) * F(sp[3])
            disc = B * B - A * C
            sq = np.sqrt(np.maximum(disc, F(0.0)))
            t0 = (-B - sq) / A
            t1 = (-B + sq) / A
            t = np.where(t0 > T_MIN, t0, t1)
            ok = (disc >= F(0.0)) & (t > T_MIN) & (t < best)
            best = np.where(ok, t, best)
            kind = np.where(ok, 1, kind)
            idx = np.where(ok, i, idx)
    return best, kind, idx


@dataclass
class Paths:
    """Per (pixel, sample): ``end`` = number of reflections before meeting the
    emitter (-1: never met), ``mats`` (N, D) material indices of the
    reflections (-1 past the end)."""
    end: np.ndarray
    mats: np.ndarray
    width: int
    height: int
    spp: int


def trace(scene, width: int, height: int, spp: int, depth: int, seed: int) -> Paths:
    """Traces every (pixel, sample) path; pixel index = y * width + x with y
    up from the bottom row."""
    N = width * height * spp
    lin = np.arange(N, dtype=np.int64)
    pix = (lin // spp).astype(np.uint32)
    smp = (lin % spp).astype(np.uint32)
    px = (pix.astype(np.int64) % width).astype(F)
    py = (pix.astype(np.int64) // width).astype(F)
    cam = scene.cam.astype(F)
    key0 = np.uint32(seed & 0xFFFFFFFF)
    r = philox4x32_10(pix, smp, np.zeros(N, np.uint32), np.full(N, STREAM, np.uint32), key0, 0)
    jx, jy = u01(r[0]), u01(r[1])
    fx = (px + jx) / F(width)
    fy = (py + jy) / F(height)
    ox = np.full(N, cam[0, 0], F)
    oy = np.full(N, cam[0, 1], F)
    oz = np.full(N, cam[0, 2], F)
    dx = ((cam[1, 0] + fx * cam[2, 0]) + fy * cam[3, 0]) - cam[0, 0]
    dy = ((cam[1, 1] + fx * cam[2, 1]) + fy * cam[3, 1]) - cam[0, 1]
    dz = ((cam[1, 2] + fx * cam[2, 2]) + fy * cam[3, 2]) - cam[0, 2]
    end = np.full(N, -1, np.int32)
    mats = np.full((N, depth), -1, np.int32)
    alive = np.ones(N, bool)
    for v in range(depth + 1):
        t, kind, idx = intersect(scene, ox, oy, oz, dx, dy, dz)
        qi = np.clip(idx, 0, len(scene.quads) - 1)
        si = np.clip(idx, 0, len(scene.spheres) - 1)
        miss = kind < 0
        alive &= ~miss
        is_light = alive & (kind == 0) & (scene.quads[qi, 7] < 0)
        end = np.where(is_light, v, end)
        alive &= ~is_light
        if v == depth:
            break
        mat = np.where(kind == 0, scene.quads[qi, 7].astype(np.int32), scene.spheres[si, 4].astype(np.int32))
        mats[:, v] = np.where(alive, mat, -1)
        # hit point and normal
        hx, hy, hz = ox + t * dx, oy + t * dy, oz + t * dz
        nxq = np.zeros(N, F)
        nyq = np.zeros(N, F)
        nzq = np.zeros(N, F)
        qa = scene.quads[qi, 0].astype(np.int32)
        qs = scene.quads[qi, 6].astype(F)
        nxq = np.where(qa == 0, qs, nxq)
        nyq = np.where(qa == 1, qs, nyq)
        nzq = np.where(qa == 2, qs, nzq)
        sp = scene.spheres[si].astype(F)
        with np.errstate(divide="ignore", invalid="ignore"):
            nxs = (hx - sp[:, 0]) / sp[:, 3]
            nys = (hy - sp[:, 1]) / sp[:, 3]
            nzs = (hz - sp[:, 2]) / sp[:, 3]
        nx = np.where(kind == 1, nxs, nxq).astype(F)
        ny = np.where(kind == 1, nys, nyq).astype(F)
        nz = np.where(kind == 1, nzs, nzq).astype(F)
        # cosine-weighted direction around the normal
        r = philox4x32_10(pix, smp, np.full(N, v + 1, np.uint32), np.full(N, STREAM, np.uint32), key0, 0)
        u1, u2 = u01(r[2]), u01(r[3])
        rad = np.sqrt(u1)
        sn, cs = sincos_turn(u2)
        lx, ly, lz = rad * cs, rad * sn, np.sqrt(F(1.0) - u1)
        b1, b2 = onb(nx, ny, nz)
        ndx = (lx * b1[0] + ly * b2[0]) + lz * nx
        ndy = (lx * b1[1] + ly * b2[1]) + lz * ny
        ndz = (lx * b1[2] + ly * b2[2]) + lz * nz
        ox = np.where(alive, hx + OFFSET * nx, ox).astype(F)
        oy = np.where(alive, hy + OFFSET * ny, oy).astype(F)
        oz = np.where(alive, hz + OFFSET * nz, oz).astype(F)
        dx = np.where(alive, ndx, dx).astype(F)
        dy = np.where(alive, ndy, dy).astype(F)
        dz = np.where(alive, ndz, dz).astype(F)
    return Paths(end, mats, width, height, spp)


def path_products(paths: Paths, refl, emit, product=np.multiply):
    """Per path: emit (.) refl[m_0] (.) ... (.) refl[m_{end-1}] (zero if the
    path never met the emitter); rows of ``refl`` / ``emit`` are spectra or
    codes, ``product`` the element-wise or blockwise product."""
    refl = np.asarray(refl, dtype=np.float64)
    emit = np.asarray(emit, dtype=np.float64)
    N = paths.end.shape[0]
    out = np.zeros((N, emit.shape[-1]))
    hit = paths.end >= 0
    acc = np.tile(emit, (N, 1))
    D = paths.mats.shape[1]
    for v in range(D):
        take = hit & (paths.end > v)
        m = np.maximum(paths.mats[:, v], 0)
        acc = np.where(take[:, None], product(refl[m], acc), acc)
    out[hit] = acc[hit]
    return out


def pixel_means(paths: Paths, per_path):
    P = paths.width * paths.height
    return per_path.reshape(P, paths.spp, -1).mean(axis=1)


def render_spectral(paths: Paths, scene, T):
    """(P, 3) XYZ of the spectral render."""
    S = pixel_means(paths, path_products(paths, scene.refl, scene.emit))
    return S @ np.asarray(T, dtype=np.float64).T


def render_latent(paths: Paths, zrefl, zemit, D, T):
    """(P, k) latent image and its (P, 3) XYZ, T (D z)."""
    from . import codec
    z = pixel_means(paths, path_products(paths, zrefl, zemit, product=codec.blockwise_hadamard))
    return z, codec.decode(D, z) @ np.asarray(T, dtype=np.float64).T


def brute_force_path(scene, width, height, spp, depth, seed, pixel, sample):
    """One path by scalar float32 loops: (end, material list)."""
    def f(v):
        return F(v)
    x, y = pixel % width, pixel // width
    r = philox4x32_10([pixel], [sample], [0], [0], seed & 0xFFFFFFFF, 0)
    jx, jy = u01(r[0])[0], u01(r[1])[0]
    cam = scene.cam.astype(F)
    fx = (f(x) + jx) / f(width)
    fy = (f(y) + jy) / f(height)
    o = [cam[0, i] for i in range(3)]
    d = [((cam[1, i] + fx * cam[2, i]) + fy * cam[3, i]) - cam[0, i] for i in range(3)]
    mats = []
    for v in range(depth + 1):
        t, kind, idx = intersect(scene, [o[0]], [o[1]], [o[2]], [d[0]], [d[1]], [d[2]])
        t, kind, idx = t[0], int(kind[0]), int(idx[0])
        if kind < 0:
            return -1, mats
        if kind == 0 and scene.quads[idx, 7] < 0:
            return v, mats
        if v == depth:
            return -1, mats
        h = [o[i] + t * d[i] for i in range(3)]
        if kind == 0:
            nrm = [f(0.0), f(0.0), f(0.0)]
            nrm[int(scene.quads[idx, 0])] = f(scene.quads[idx, 6])
            mats.append(int(scene.quads[idx, 7]))
        else:
            sp = scene.spheres[idx]
            nrm = [(h[i] - f(sp[i])) / f(sp[3]) for i in range(3)]
            mats.append(int(sp[4]))
        r = philox4x32_10([pixel], [sample], [v + 1], [0], seed & 0xFFFFFFFF, 0)
        u1, u2 = u01(r[2])[0], u01(r[3])[0]
        rad = np.sqrt(u1)
        sn, cs = sincos_turn([u2])
        lx, ly, lz = rad * cs[0], rad * sn[0], np.sqrt(f(1.0) - u1)
        b1, b2 = onb([nrm[0]], [nrm[1]], [nrm[2]])
        d = [(lx * b1[i][0] + ly * b2[i][0]) + lz * nrm[i] for i in range(3)]
        o = [h[i] + OFFSET * nrm[i] for i in range(3)]
    return -1, mats
