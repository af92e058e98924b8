"""Seeded synthetic inputs for the Hadamard-spectral-code shading path.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
no arithmetic of the method itself (no encoding, shading, decoding or colour
science): only seeded random draws and the closed-form spectra that stand in
for the paper's measured data.  The paper trains and renders with Munsell
reflectances, LSPDD lamp spectra and Mitsuba scenes (Sec. 4.4, Sec. 6.1), none
of which is available here; every array below is a synthetic stand-in with the
shapes and value ranges those data have.

Conventions
-----------
* Spectra are sampled on a uniform grid ``lambda_i = lambda0 + i * dlambda``.
* Every array handed to a device is float32 (int32 for material indices); the
  oracle reads the same float32 values and widens them to float64, so both
  sides start from bit-identical inputs.
* All randomness flows from ``numpy.random.SeedSequence(seed)``; each consumer
  takes its own spawned stream so adding a draw in one place does not shift
  another.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

MASTER_SEED = 2602_18741

# Wavelength grids (lambda0 [nm], dlambda [nm], n).
GRID_31 = (400.0, 10.0, 31)   # 400..700 nm at 10 nm
GRID_81 = (380.0, 5.0, 81)    # 380..780 nm at 5 nm

CODEC_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "codecs")


def streams(seed: int, count: int) -> list:
    """``count`` independent numpy Generators spawned from one seed."""
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(count)]


def grid(lambda0: float, dlambda: float, n: int) -> np.ndarray:
    """Wavelength samples in nm (float64)."""
    return lambda0 + dlambda * np.arange(n, dtype=np.float64)


# ----------------------------------------------------------------------------
# Spectra
# ----------------------------------------------------------------------------

def smooth_reflectances(rng, lam: np.ndarray, count: int) -> np.ndarray:
    """Sum of three Gaussians (centre U[400,700] nm, std U[20,80] nm, amplitude
    U[0,1]) clipped to [0, 1]: a smooth, Munsell-like reflectance."""
    c = rng.uniform(400.0, 700.0, size=(count, 3, 1))
    w = rng.uniform(20.0, 80.0, size=(count, 3, 1))
    a = rng.uniform(0.0, 1.0, size=(count, 3, 1))
    s = (a * np.exp(-0.5 * ((lam[None, None, :] - c) / w) ** 2)).sum(axis=1)
    return np.clip(s, 0.0, 1.0)


def sawtooth_reflectances(rng, lam: np.ndarray, count: int) -> np.ndarray:
    """High-frequency reflectances: clip(a + b*frac((lambda - phi)/period), 0, 1)
    with period U[10,40] nm, phase U[0,period], a U[0,0.3], b U[0.4,0.7]."""
    period = rng.uniform(10.0, 40.0, size=(count, 1))
    phi = rng.uniform(0.0, 1.0, size=(count, 1)) * period
    a = rng.uniform(0.0, 0.3, size=(count, 1))
    b = rng.uniform(0.4, 0.7, size=(count, 1))
    t = (lam[None, :] - phi) / period
    return np.clip(a + b * (t - np.floor(t)), 0.0, 1.0)


# SI-exact constants (2019 SI definitions).
_H = 6.62607015e-34
_C = 299792458.0
_KB = 1.380649e-23


def blackbody(lam: np.ndarray, temperature_k) -> np.ndarray:
    """Planck radiance at the grid wavelengths, normalised to unit peak on the
    grid (the paper normalises its lights to unit peak, Sec. 4.4)."""
    t = np.atleast_1d(np.asarray(temperature_k, dtype=np.float64))[:, None]
    lm = lam[None, :] * 1e-9
    b = (2.0 * _H * _C ** 2) / (lm ** 5 * np.expm1(_H * _C / (lm * _KB * t)))
    return b / b.max(axis=1, keepdims=True)


def narrowband(lam: np.ndarray, mu, sigma) -> np.ndarray:
    """Unit-peak Gaussian band(s), standard deviation ``sigma`` nm."""
    mu = np.atleast_1d(np.asarray(mu, dtype=np.float64))[:, None]
    sigma = np.atleast_1d(np.asarray(sigma, dtype=np.float64))[:, None]
    return np.exp(-0.5 * ((lam[None, :] - mu) / sigma) ** 2)


# ----------------------------------------------------------------------------
# Geometry
# ----------------------------------------------------------------------------

def _unit_hemisphere_z(rng, count: int) -> np.ndarray:
    z = rng.uniform(0.0, 1.0, size=count)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=count)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _unit_sphere(rng, count: int) -> np.ndarray:
    z = rng.uniform(-1.0, 1.0, size=count)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=count)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _normalize_f32(v: np.ndarray) -> np.ndarray:
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    return v.astype(np.float32)


@dataclass
class GBuffer:
    """Per-pixel shading points: unit normal (P,3), position (P,3), material (P,)."""
    normal: np.ndarray
    pos: np.ndarray
    mat: np.ndarray

    @property
    def pixels(self) -> int:
        return int(self.mat.shape[0])


def gbuffers(rng, pixels: int, n_mat: int, secondary: bool):
    """Primary G-buffer (normals uniform on the +z hemisphere, positions
    U[0,1]^3, material index uniform) and, optionally, a secondary G-buffer:
    the point one indirect bounce reaches, at U[0,1]^3 with a normal drawn
    around the direction back to the primary point, so most pairs face each
    other."""
    n1 = _normalize_f32(_unit_hemisphere_z(rng, pixels))
    x1 = rng.uniform(0.0, 1.0, size=(pixels, 3)).astype(np.float32)
    m1 = rng.integers(0, n_mat, size=pixels, dtype=np.int32)
    g1 = GBuffer(n1, x1, m1)
    if not secondary:
        return g1, None
    x2 = rng.uniform(0.0, 1.0, size=(pixels, 3)).astype(np.float32)
    back = x1.astype(np.float64) - x2.astype(np.float64)
    back /= np.maximum(np.linalg.norm(back, axis=1, keepdims=True), 1e-6)
    n2 = _normalize_f32(back + 0.8 * _unit_sphere(rng, pixels))
    m2 = rng.integers(0, n_mat, size=pixels, dtype=np.int32)
    return g1, GBuffer(n2, x2, m2)


def light_positions(rng, count: int):
    """Point lights above the unit cube: x, y U[-0.5,1.5], z U[1.5,2.5]
    (so every light is at least 0.5 from every shading point); intensity
    U[0.5,2]."""
    pos = np.stack([rng.uniform(-0.5, 1.5, size=count),
                    rng.uniform(-0.5, 1.5, size=count),
                    rng.uniform(1.5, 2.5, size=count)], axis=1).astype(np.float32)
    inten = rng.uniform(0.5, 2.0, size=count).astype(np.float32)
    return pos, inten


# ----------------------------------------------------------------------------
# Frames
# ----------------------------------------------------------------------------

@dataclass
class Frame:
    """One G-buffer frame with its spectral assets (all float32 / int32)."""
    width: int
    height: int
    grid: tuple                       # (lambda0, dlambda, n)
    mat_spectra: np.ndarray           # (m, n) reflectances in [0,1]
    light_spd: np.ndarray             # (L, n) unit-peak SPDs
    light_pos: np.ndarray             # (L, 3)
    light_intensity: np.ndarray       # (L,)
    g1: GBuffer
    g2: Optional[GBuffer] = None
    meta: dict = field(default_factory=dict)

    @property
    def pixels(self) -> int:
        return self.width * self.height

    @property
    def n(self) -> int:
        return int(self.grid[2])

    @property
    def lights(self) -> int:
        return int(self.light_pos.shape[0])

    @property
    def evals(self) -> int:
        """Pixel-light evaluations: one (shading point, light) pair each."""
        return self.pixels * self.lights * (2 if self.g2 is not None else 1)


def make_frame(seed: int, width: int, height: int, grid_spec=GRID_81,
               n_smooth: int = 256, n_saw: int = 32,
               lights: int = 64, secondary: bool = True,
               spd_kinds=None) -> Frame:
    """General seeded frame.  Lights: the first half blackbodies at U[2000,
    10000] K, the second half Gaussian bands (centre U[400,700] nm, std
    U[5,20] nm), unless ``spd_kinds`` gives explicit SPDs."""
    r_geo, r_mat, r_light, r_spd = streams(seed, 4)
    lam = grid(*grid_spec)
    mats = np.concatenate([smooth_reflectances(r_mat, lam, n_smooth),
                           sawtooth_reflectances(r_mat, lam, n_saw)], axis=0)
    if spd_kinds is not None:
        spd = spd_kinds(lam)
        lights = spd.shape[0]
    else:
        n_bb = lights // 2
        n_nb = lights - n_bb
        spd = np.concatenate([
            blackbody(lam, r_spd.uniform(2000.0, 10000.0, size=n_bb)),
            narrowband(lam, r_spd.uniform(400.0, 700.0, size=n_nb),
                       r_spd.uniform(5.0, 20.0, size=n_nb))], axis=0)
    lpos, linten = light_positions(r_light, lights)
    g1, g2 = gbuffers(r_geo, width * height, mats.shape[0], secondary)
    return Frame(width, height, tuple(grid_spec), mats.astype(np.float32),
                 spd.astype(np.float32), lpos, linten, g1, g2)


def _config1_spds(lam):
    return np.concatenate([blackbody(lam, [2700.0, 6500.0]),
                           narrowband(lam, [450.0, 610.0], [15.0, 15.0])], axis=0)


def frame_config1(seed: int = MASTER_SEED) -> Frame:
    """256x256, n=31 (400-700 nm @ 10 nm), 16 smooth materials, 4 lights
    (blackbody 2700 K and 6500 K, Gaussian bands of std 15 nm at 450 and
    610 nm), direct lighting only."""
    f = make_frame(seed, 256, 256, GRID_31, n_smooth=16, n_saw=0,
                   secondary=False, spd_kinds=_config1_spds)
    f.meta["name"] = "256x256 n=31 L=4 direct"
    return f


def frame_config2(seed: int = MASTER_SEED + 2, width: int = 1920, height: int = 1080) -> Frame:
    """1920x1080, n=81 (380-780 nm @ 5 nm), 256 smooth + 32 saw-tooth
    materials, 64 lights (32 blackbody, 32 Gaussian bands), primary plus one
    indirect bounce from a secondary G-buffer."""
    f = make_frame(seed, width, height, GRID_81, 256, 32, 64, True)
    f.meta["name"] = f"{width}x{height} n=81 L=64 direct+indirect"
    return f


def frame_config3(seed: int = MASTER_SEED + 3) -> Frame:
    """3840x2160 with the 1920x1080 frame's scene model."""
    f = make_frame(seed, 3840, 2160, GRID_81, 256, 32, 64, True)
    f.meta["name"] = "3840x2160 n=81 L=64 direct+indirect"
    return f


# ----------------------------------------------------------------------------
# Codec training set and stored codecs
# ----------------------------------------------------------------------------

@dataclass
class TrainingSet:
    R: np.ndarray        # (N_R, n) reflectances
    L: np.ndarray        # (N_L, n) unit-peak lights
    pair_r: np.ndarray   # (P,) index into R
    pair_l: np.ndarray   # (P,) index into L
    pair_scale: np.ndarray  # (P,) light scale augmentation U[0.5, 1]


def training_set(grid_spec, seed: int = MASTER_SEED + 100, n_smooth: int = 1024,
                 n_saw: int = 128, n_bb: int = 256, n_nb: int = 256,
                 pairs: int = 4096) -> TrainingSet:
    """Seeded stand-in for the paper's training spectra (Sec. 4.4): smooth and
    saw-tooth reflectances, blackbody (2000-10000 K) and narrow-band (std 5-20
    nm) unit-peak lights, random reflectance-light pairs with a light scale
    augmentation U[0.5, 1]."""
    r_ref, r_light, r_pair = streams(seed, 3)
    lam = grid(*grid_spec)
    R = np.concatenate([smooth_reflectances(r_ref, lam, n_smooth),
                        sawtooth_reflectances(r_ref, lam, n_saw)], axis=0)
    L = np.concatenate([
        blackbody(lam, r_light.uniform(2000.0, 10000.0, size=n_bb)),
        narrowband(lam, r_light.uniform(lam[0], lam[-1], size=n_nb),
                   r_light.uniform(5.0, 20.0, size=n_nb))], axis=0)
    pr = r_pair.integers(0, R.shape[0], size=pairs)
    pl = r_pair.integers(0, L.shape[0], size=pairs)
    ps = r_pair.uniform(0.5, 1.0, size=pairs)
    return TrainingSet(R, L, pr, pl, ps)


def sweep_weight_grid() -> np.ndarray:
    """The loss-weight grid of the codec sweep (Sec. 4.5) as (700, 4) float32
    rows (lambda_e2e, lambda_rec, lambda_code, lambda_col): e2e 0-2 by 0.5, rec
    0-3 by 0.5, code 0-1 by 0.25, col 0.25-1 by 0.25.  The grid as printed has
    7 x 5 x 5 x 5 = 875 points but is said to give 700 variants; leaving out
    lambda_col = 0 gives exactly 700 (and no variant without a colour term)."""
    e2e = np.arange(5) * 0.5
    rec = np.arange(7) * 0.5
    code = np.arange(5) * 0.25
    col = (np.arange(4) + 1) * 0.25
    g = np.stack(np.meshgrid(e2e, rec, code, col, indexing="ij"), axis=-1).reshape(-1, 4)
    return g.astype(np.float32)


@dataclass
class SweepSchedule:
    """Mini-batches of every epoch and the validation batch of a codec sweep.
    train_r, train_l: (epochs, batches, batch) int32 rows of R and L;
    train_s: the same shape, float32 light scales; val_r, val_l, val_s: the
    validation pairs (new pairings of the training spectra)."""
    train_r: np.ndarray
    train_l: np.ndarray
    train_s: np.ndarray
    val_r: np.ndarray
    val_l: np.ndarray
    val_s: np.ndarray


def sweep_schedule(ts: TrainingSet, epochs: int, batch: int = 128, val_pairs: int = 256,
                   seed: int = MASTER_SEED + 300) -> SweepSchedule:
    """Seeded shuffles of the training pairs, one per epoch, cut into
    ``len(pairs) // batch`` whole mini-batches (a trailing partial batch is
    dropped), and ``val_pairs`` validation pairs drawn like the training pairs
    (reflectance and light rows uniform, light scale U[0.5, 1])."""
    r_shuffle, r_val = streams(seed, 2)
    P = len(ts.pair_r)
    nb = P // batch
    order = np.stack([r_shuffle.permutation(P)[:nb * batch].reshape(nb, batch) for _ in range(epochs)])
    vr = r_val.integers(0, ts.R.shape[0], size=val_pairs)
    vl = r_val.integers(0, ts.L.shape[0], size=val_pairs)
    vs = r_val.uniform(0.5, 1.0, size=val_pairs)
    return SweepSchedule(ts.pair_r[order].astype(np.int32), ts.pair_l[order].astype(np.int32),
                         ts.pair_scale[order].astype(np.float32), vr.astype(np.int32), vl.astype(np.int32),
                         vs.astype(np.float32))


UPSAMPLER_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "upsampler")


def upsampler_path(k: int, n: int) -> str:
    return os.path.join(UPSAMPLER_DIR, f"upsampler_k{k}_n{n}.npz")


def load_upsampler(k: int, n: int):
    """Stored RGB-to-latent network for code length k over n samples: a dict
    of float32 W1 (128, 3), b1, W2 (128, 128), b2, W3 (k, 128), b3.  Written by
    the oracle's upsampler-fitting script."""
    with np.load(upsampler_path(k, n)) as z:
        return {name: z[name].astype(np.float32) for name in ("W1", "b1", "W2", "b2", "W3", "b3")}


def rgb_palette(seed: int = MASTER_SEED + 6, grid_spec=GRID_81, count: int = 4096):
    """Seeded reflectances standing in for the spectra behind an RGB texture:
    smooth and saw-tooth spectra in the training set's proportions (the caller
    takes their colours and codes)."""
    r_s, r_t = streams(seed, 2)
    lam = grid(*grid_spec)
    n_saw = count // 9
    return np.concatenate([smooth_reflectances(r_s, lam, count - n_saw), sawtooth_reflectances(r_t, lam, n_saw)])


def codec_path(k: int, n: int) -> str:
    return os.path.join(CODEC_DIR, f"codec_k{k}_n{n}.npz")


def load_codec(k: int, n: int):
    """Stored (E, D) for code length k over n samples, float32 (k,n) and (n,k).
    The files are written by the oracle's codec-fitting script."""
    with np.load(codec_path(k, n)) as z:
        return z["E"].astype(np.float32), z["D"].astype(np.float32)


# ----------------------------------------------------------------------------
# Batched frames and request streams
# ----------------------------------------------------------------------------

@dataclass
class FrameSpec:
    """Parameters of one frame of a batch (materialised by make_frame or on
    the device by torch_frame)."""
    width: int
    height: int
    grid: tuple
    lights: int
    k: int
    seed: int
    E: np.ndarray
    D: np.ndarray
    secondary: bool = False

    @property
    def pixels(self) -> int:
        return self.width * self.height


def batched_frame_specs(seed: int = MASTER_SEED + 4, count: int = 64, min_side: int = 256,
                        max_side: int = 2048, min_lights: int = 4, max_lights: int = 256,
                        ks=(6, 9), grids=(GRID_31, GRID_81), secondary: bool = False):
    """Frames of uneven size for a batched launch: W, H independent uniform
    integers in [min_side, max_side], L uniform in [min_lights, max_lights],
    k and n uniform over the given choices; each frame carries its own codec,
    a stored base codec times a seeded multiplicative jitter U[0.9, 1.1]
    (which keeps it non-negative)."""
    (r,) = streams(seed, 1)
    out = []
    for _ in range(count):
        w = int(r.integers(min_side, max_side + 1))
        h = int(r.integers(min_side, max_side + 1))
        L = int(r.integers(min_lights, max_lights + 1))
        k = int(ks[r.integers(0, len(ks))])
        g = grids[r.integers(0, len(grids))]
        fseed = int(r.integers(0, 2**31 - 1))
        E, D = load_codec(k, g[2])
        jE = r.uniform(0.9, 1.1, size=E.shape).astype(np.float32)
        jD = r.uniform(0.9, 1.1, size=D.shape).astype(np.float32)
        out.append(FrameSpec(w, h, tuple(g), L, k, fseed, (E * jE).astype(np.float32),
                             (D * jD).astype(np.float32), secondary))
    return out


def frame_assets(spec: FrameSpec, n_smooth: int = 48, n_saw: int = 16):
    """The spectral assets and lights of a batch frame (the same draws as
    frame_from_spec, without the G-buffer): materials (m, n), light SPDs
    (L, n), light positions (L, 3), intensities (L,)."""
    _, r_mat, r_light, r_spd = streams(spec.seed, 4)
    lam = grid(*spec.grid)
    mats = np.concatenate([smooth_reflectances(r_mat, lam, n_smooth),
                           sawtooth_reflectances(r_mat, lam, n_saw)], axis=0)
    n_bb = spec.lights // 2
    n_nb = spec.lights - n_bb
    spd = np.concatenate([
        blackbody(lam, r_spd.uniform(2000.0, 10000.0, size=n_bb)),
        narrowband(lam, r_spd.uniform(400.0, 700.0, size=n_nb), r_spd.uniform(5.0, 20.0, size=n_nb))], axis=0)
    lpos, linten = light_positions(r_light, spec.lights)
    return mats.astype(np.float32), spd.astype(np.float32), lpos, linten


def frame_from_spec(spec: FrameSpec, n_smooth: int = 48, n_saw: int = 16) -> Frame:
    """Host (numpy) frame of a batch spec."""
    f = make_frame(spec.seed, spec.width, spec.height, spec.grid, n_smooth=n_smooth, n_saw=n_saw,
                   lights=spec.lights, secondary=spec.secondary)
    f.meta.update(k=spec.k, E=spec.E, D=spec.D)
    return f


def torch_gbuffers(gen, pixels: int, n_mat: int, secondary: bool, device):
    """The gbuffers() recipe drawn with a torch generator on a device (for
    large benchmark batches, where drawing on the host would dominate).
    Returns (normal, pos, mat) tuples for the primary and, optionally, the
    secondary G-buffer, float32 / int32."""
    import torch
    kw = dict(generator=gen, device=device)

    def hemi(count):
        z = torch.rand(count, **kw)
        phi = torch.rand(count, **kw) * (2.0 * math.pi)
        r = torch.sqrt(torch.clamp(1.0 - z * z, min=0.0))
        return torch.stack([r * torch.cos(phi), r * torch.sin(phi), z], dim=1)

    def sphere(count):
        z = torch.rand(count, **kw) * 2.0 - 1.0
        phi = torch.rand(count, **kw) * (2.0 * math.pi)
        r = torch.sqrt(torch.clamp(1.0 - z * z, min=0.0))
        return torch.stack([r * torch.cos(phi), r * torch.sin(phi), z], dim=1)

    def unit(v):
        return (v / torch.linalg.norm(v, dim=1, keepdim=True)).float().contiguous()

    n1 = unit(hemi(pixels))
    x1 = torch.rand(pixels, 3, **kw).float().contiguous()
    m1 = torch.randint(0, n_mat, (pixels,), **kw, dtype=torch.int32)
    if not secondary:
        return (n1, x1, m1), None
    x2 = torch.rand(pixels, 3, **kw).float().contiguous()
    back = x1 - x2
    back = back / torch.clamp(torch.linalg.norm(back, dim=1, keepdim=True), min=1e-6)
    n2 = unit(back + 0.8 * sphere(pixels))
    m2 = torch.randint(0, n_mat, (pixels,), **kw, dtype=torch.int32)
    return (n1, x1, m1), (n2, x2, m2)


# ----------------------------------------------------------------------------
# Path-traced scene (a Cornell-box stand-in for the paper's Mitsuba scenes)
# ----------------------------------------------------------------------------

@dataclass
class PTScene:
    """Geometry in float32, spectra in float64.

    quads:   (Q, 8) rows (axis, c, u0, u1, v0, v1, normal sign, material):
             the rectangle {x[axis] = c, u0 <= x[u] <= u1, v0 <= x[v] <= v1}
             with (u, v) the other two axes in increasing order, its normal
             along +/- axis; material -1 marks the emitter.
    spheres: (S, 5) rows (cx, cy, cz, radius, material); the normal is
             (hit - centre) / radius, so a negative radius gives a sphere
             whose normals point inward (a closed room seen from inside).
    refl:    (M, n) reflectances of the materials; emit: (n,) emitted
             radiance of the emitter (SPD times intensity).
    cam:     (4, 3) pinhole origin, image-plane lower-left corner, horizontal
             and vertical spans (pixel (x, y) maps to
             ll + (x + jx)/W * hor + (y + jy)/H * ver, y up)."""
    quads: np.ndarray
    spheres: np.ndarray
    refl: np.ndarray
    emit: np.ndarray
    cam: np.ndarray
    grid: tuple


def cornell_scene(width: int, height: int, grid_spec=GRID_81, light: str = "blackbody",
                  seed: int = MASTER_SEED + 8, intensity: float = 12.0) -> PTScene:
    """The unit box [0,1]^3 open towards the camera (z = 0): white floor,
    ceiling and back wall, red left wall, green right wall, an emitting
    rectangle just below the ceiling, a smooth and a saw-tooth sphere.  The
    emitter is a 4000 K blackbody (``light='blackbody'``) or a 20 nm-wide band
    at 590 nm (``'narrowband'``), unit peak times ``intensity``."""
    lam = grid(*grid_spec)
    r_s, r_t = streams(seed, 2)
    white = np.full_like(lam, 0.78)
    red = 0.05 + 0.70 * np.exp(-0.5 * ((lam - 640.0) / 40.0) ** 2)
    green = 0.05 + 0.60 * np.exp(-0.5 * ((lam - 535.0) / 35.0) ** 2)
    refl = np.stack([white, red, green, smooth_reflectances(r_s, lam, 1)[0], sawtooth_reflectances(r_t, lam, 1)[0]])
    spd = blackbody(lam, [4000.0])[0] if light == "blackbody" else narrowband(lam, [590.0], [20.0])[0]
    quads = np.array([
        [1, 0.0, 0.0, 1.0, 0.0, 1.0, +1, 0],      # floor      y = 0
        [1, 1.0, 0.0, 1.0, 0.0, 1.0, -1, 0],      # ceiling    y = 1
        [2, 1.0, 0.0, 1.0, 0.0, 1.0, -1, 0],      # back wall  z = 1
        [0, 0.0, 0.0, 1.0, 0.0, 1.0, +1, 1],      # left wall  x = 0 (red)
        [0, 1.0, 0.0, 1.0, 0.0, 1.0, -1, 2],      # right wall x = 1 (green)
        [1, 0.998, 0.35, 0.65, 0.40, 0.70, -1, -1],  # emitter under the ceiling
    ], dtype=np.float32)
    spheres = np.array([[0.28, 0.18, 0.62, 0.18, 3], [0.70, 0.25, 0.38, 0.22, 4]], dtype=np.float32)
    aspect = width / height
    cam = np.array([[0.5, 0.5, -1.4], [0.5 - 0.5 * aspect, 0.0, 0.0], [aspect, 0.0, 0.0], [0.0, 1.0, 0.0]],
                   dtype=np.float32)
    return PTScene(quads, spheres, refl, intensity * spd, cam, tuple(grid_spec))


def sphere_enclosure_scene(width: int, height: int, z0: float = 0.6, rho: float = 0.8, emission: float = 1.0,
                           grid_spec=(400.0, 100.0, 4)) -> PTScene:
    """A closed spherical room seen from inside: the unit sphere with inward
    normals (a negative radius) of constant reflectance ``rho``, cut by an
    emitting square in the plane z = z0 that covers the sphere's cross-section
    there, so the part of the sphere above z0 is hidden behind the emitter.
    The camera sits at (0, 0, -0.3) and looks down the -z axis at the lower
    part of the sphere.  Constant spectra (``emission`` everywhere) on a small
    grid."""
    lam = grid(*grid_spec)
    refl = np.full((1, lam.size), float(rho))
    quads = np.array([[2, z0, -1.25, 1.25, -1.25, 1.25, -1, -1]], dtype=np.float32)
    spheres = np.array([[0.0, 0.0, 0.0, -1.0, 0]], dtype=np.float32)
    aspect = width / height
    cam = np.array([[0.0, 0.0, -0.3], [-0.25 * aspect, -0.25, -0.8], [0.5 * aspect, 0.0, 0.0], [0.0, 0.5, 0.0]],
                   dtype=np.float32)
    return PTScene(quads, spheres, refl, np.full(lam.size, float(emission)), cam, tuple(grid_spec))


SERVE_SIZES = ((512, 512), (1024, 1024), (1920, 1080), (2048, 2048), (3840, 2160))


@dataclass
class Request:
    rid: int
    arrival_s: float
    width: int
    height: int
    k: int
    n: int
    lights: int
    scene: int
    seed: int


def request_stream(seed: int = MASTER_SEED + 5, rate_hz: float = 200.0,
                   duration_s: float = 30.0, sizes=SERVE_SIZES, ks=(6, 9),
                   ns=(31, 81), min_lights: int = 16, max_lights: int = 128,
                   scenes: int = 8):
    """Poisson arrivals (exponential gaps, mean 1/rate) of render-plus-decode
    requests over ``duration_s``; size, k, n, light count and scene uniform."""
    (r,) = streams(seed, 1)
    t = 0.0
    out = []
    while True:
        t += float(r.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        w, h = sizes[r.integers(0, len(sizes))]
        out.append(Request(len(out), t, int(w), int(h), int(ks[r.integers(0, len(ks))]),
                           int(ns[r.integers(0, len(ns))]),
                           int(r.integers(min_lights, max_lights + 1)),
                           int(r.integers(0, scenes)), int(r.integers(0, 2**31 - 1))))
    return out
