"""Python binding of libhsc: Hadamard-spectral-code G-buffer shading on GB300.

Thin ctypes layer over the C ABI in ``include/hsc.h``: every function here
has the C entry point's name, takes torch CUDA tensors, checks shapes and
dtypes, and passes raw device pointers and the current CUDA stream to the
library.  All arithmetic runs in the library's CUDA kernels; there is no
fallback.  Importing raises ``ImportError`` when ``libhsc.so`` has not been
built (``python paper_2602_18741_gb300/build.py``).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhsc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhsc.so is not built at {LIB_PATH}; run `python paper_2602_18741_gb300/build.py`")

_lib = ctypes.CDLL(LIB_PATH)

# --------------------------------------------------------------------- enums
HSC_OK, HSC_ERR_INVALID_ARG, HSC_ERR_CUDA, HSC_ERR_OOM, HSC_ERR_UNSUPPORTED, HSC_ERR_TIMEOUT, \
    HSC_ERR_DEVICE_CHECK = range(7)
HSC_F32, HSC_BF16, HSC_F16, HSC_FP8_E4M3 = range(4)
HSC_PASSES, HSC_FUSED = range(2)
HSC_MAX_K = 96
HSC_NOALLOC_MAX_K = 96
HSC_MAX_FRAMES_PER_CALL = 512
HSC_MAX_N = 128
HSC_QUEUE_SLOTS = 256
HSC_ASSETS_MAX_CODES = 4096
HSC_ASSETS_MAX_LIGHTS = 256

STATUS_NAMES = {0: "HSC_OK", 1: "HSC_ERR_INVALID_ARG", 2: "HSC_ERR_CUDA", 3: "HSC_ERR_OOM",
                4: "HSC_ERR_UNSUPPORTED", 5: "HSC_ERR_TIMEOUT", 6: "HSC_ERR_DEVICE_CHECK"}

_DT_OF_TORCH = {torch.float32: HSC_F32, torch.bfloat16: HSC_BF16, torch.float16: HSC_F16,
                torch.float8_e4m3fn: HSC_FP8_E4M3, torch.uint8: HSC_FP8_E4M3}


class HscError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class _GBuffer(ctypes.Structure):
    _fields_ = [("normal", ctypes.c_void_p), ("pos", ctypes.c_void_p), ("mat", ctypes.c_void_p)]


class _Lights(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("intensity", ctypes.c_void_p), ("count", ctypes.c_int32)]


class _Frame(ctypes.Structure):
    _fields_ = [("g1", _GBuffer), ("g2", _GBuffer), ("has_g2", ctypes.c_int32), ("pixels", ctypes.c_int64),
                ("mat_codes", ctypes.c_void_p), ("n_mat", ctypes.c_int32), ("lights", _Lights),
                ("light_codes", ctypes.c_void_p), ("k", ctypes.c_int32), ("code_dt", ctypes.c_int),
                ("M_xyz", ctypes.c_void_p), ("xyz_out", ctypes.c_void_p), ("latent_out", ctypes.c_void_p)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int
_i64 = ctypes.c_int64
_f32 = ctypes.c_float
_GB = ctypes.POINTER(_GBuffer)
_LI = ctypes.POINTER(_Lights)

_SIGS = {
    "hsc_create": ([ctypes.POINTER(_vp), _i32], _i32),
    "hsc_destroy": ([_vp], None),
    "hsc_last_error": ([], ctypes.c_char_p),
    "hsc_sync": ([_vp, _vp], _i32),
    "hsc_reserve": ([_vp, ctypes.c_size_t], _i32),
    "hsc_shade_latent_scratch_bytes": ([_i64, _i32, _i32, _i32], ctypes.c_size_t),
    "hsc_set_autotune": ([_vp, _i32], _i32),
    "hsc_tune_report": ([_vp], ctypes.c_char_p),
    "hsc_tune_save": ([_vp, ctypes.c_char_p, ctypes.c_size_t], _i32),
    "hsc_tune_load": ([_vp, ctypes.c_char_p], _i32),
    "hsc_force_launch_config": ([_vp, _i32, _i32, _i32, _i32, _i32], _i32),
    "hsc_fp32_peak_probe": ([_vp, _i32, _i32, _vp, ctypes.POINTER(_i64), _vp], _i32),
    "hsc_tanh_peak_probe": ([_vp, _i32, _i32, _i32, _vp, ctypes.POINTER(_i64), _vp], _i32),
    "hsc_cmf_weights": ([_vp, _i32, _f32, _f32, _vp, _vp], _i32),
    "hsc_fold_xyz": ([_vp, _vp, _vp, _i32, _i32, _vp, _vp], _i32),
    "hsc_encode": ([_vp, _vp, _i32, _i32, _vp, _i32, _vp, _i32, _vp], _i32),
    "hsc_encode_assets": ([_vp, _vp, _i32, _i32, _vp, _i32, _vp, _vp, _i32, _vp, _i32, _vp], _i32),
    "hsc_shade_pass": ([_vp, _GB, _GB, _i64, _vp, _i32, _LI, _vp, _i32, _i32, _i32, _vp, _vp], _i32),
    "hsc_reassemble": ([_vp, ctypes.POINTER(_vp), _i32, _i64, _vp, _vp], _i32),
    "hsc_shade_latent": ([_vp, _GB, _GB, _i64, _vp, _i32, _LI, _vp, _i32, _i32, _i32, _vp, _i32, _vp, _vp, _vp,
                          _vp, _vp], _i32),
    "hsc_shade_latent_assets": ([_vp, _GB, _GB, _i64, _vp, _i32, _i32, _vp, _i32, _LI, _vp, _vp, _vp, _vp, _vp,
                                 _vp], _i32),
    "hsc_quantize_fp8": ([_vp, _vp, _i64, _i32, _vp, _vp, _vp], _i32),
    "hsc_quantize_fp8_noalloc": ([_vp, _i64, _i32, _vp, _vp, _vp], _i32),
    "hsc_decode_xyz": ([_vp, _vp, _i32, _vp, _i64, _i32, _vp, _vp, _vp, _vp], _i32),
    "hsc_decode_spectra": ([_vp, _vp, _i32, _vp, _i64, _i32, _vp, _i32, _vp, _vp], _i32),
    "hsc_shade_spectral": ([_vp, _GB, _GB, _i64, _vp, _i32, _LI, _vp, _i32, _vp, _vp, _vp, _vp], _i32),
    "hsc_delta_e": ([_vp, _vp, _vp, _i64, _vp, _i32, _vp, _vp, _vp], _i32),
    "hsc_chain_eval": ([_vp, _vp, _i32, _vp, _i32, _vp, _vp, _i32, _i32, _vp, _vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp],
                       _i32),
    "hsc_upsample_rgb": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp], _i32),
    "hsc_path_trace": ([_vp, _vp, _i32, _vp, _i32, _vp, _i32, _i32, _i32, _i32, ctypes.c_uint32, _vp, _i32, _vp,
                        _i32, _vp, _vp, _vp, _vp], _i32),
    "hsc_codec_fit_step": ([_vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                            _vp, _i32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                            _vp, _vp, _vp, _vp], _i32),
    "hsc_codec_fit_eval": ([_vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp,
                            ctypes.c_float, _vp, _vp, _vp, _vp, _vp], _i32),
    "hsc_codec_fit_track": ([_vp, _i32, _i32, _i32, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp,
                             _vp], _i32),
    "hsc_batch_create": ([_vp, ctypes.POINTER(_Frame), _i32, ctypes.POINTER(_vp)], _i32),
    "hsc_batch_shade": ([_vp, _vp, _vp], _i32),
    "hsc_batch_destroy": ([_vp], None),
    "hsc_shade_frames": ([_vp, ctypes.POINTER(_Frame), _i32, _vp], _i32),
}

for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


def _check(status: int):
    if status != HSC_OK:
        raise HscError(status, _lib.hsc_last_error().decode(errors="replace"))


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dt(t: torch.Tensor) -> int:
    try:
        return _DT_OF_TORCH[t.dtype]
    except KeyError:
        raise ValueError(f"unsupported dtype {t.dtype}") from None


class Context:
    """Owns an ``hsc_ctx`` (scratch, error word) on one CUDA device."""

    def __init__(self, device: int = 0):
        self._h = _vp()
        _check(_lib.hsc_create(ctypes.byref(self._h), int(device)))
        self.device = int(device)
        self.autotune = False

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.hsc_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GBuffer:
    """Device G-buffer: normal (P,3) f32, pos (P,3) f32, mat (P,) int32."""

    def __init__(self, normal: torch.Tensor, pos: torch.Tensor, mat: torch.Tensor):
        for t, nm in ((normal, "normal"), (pos, "pos")):
            if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 3:
                raise ValueError(f"{nm} must be (P,3) float32")
        if mat.dtype != torch.int32 or mat.dim() != 1:
            raise ValueError("mat must be (P,) int32")
        if not (normal.shape[0] == pos.shape[0] == mat.shape[0]):
            raise ValueError("G-buffer arrays disagree on P")
        self.normal, self.pos, self.mat = normal, pos, mat
        self._s = _GBuffer(_ptr(normal), _ptr(pos), _ptr(mat))

    @property
    def pixels(self) -> int:
        return int(self.mat.shape[0])


class Lights:
    """Device point lights: pos (L,3) f32, intensity (L,) f32."""

    def __init__(self, pos: torch.Tensor, intensity: torch.Tensor):
        if pos.dtype != torch.float32 or pos.dim() != 2 or pos.shape[1] != 3:
            raise ValueError("light pos must be (L,3) float32")
        if intensity.dtype != torch.float32 or intensity.shape != (pos.shape[0],):
            raise ValueError("light intensity must be (L,) float32")
        self.pos, self.intensity = pos, intensity
        self._s = _Lights(_ptr(pos), _ptr(intensity), int(pos.shape[0]))

    @property
    def count(self) -> int:
        return int(self.pos.shape[0])


def _gb(g: Optional[GBuffer]):
    return ctypes.byref(g._s) if g is not None else None


# ------------------------------------------------------------------- calls

def hsc_sync(ctx: Context, stream=None):
    _check(_lib.hsc_sync(ctx.handle, _stream(stream)))


def hsc_reserve(ctx: Context, nbytes: int):
    _check(_lib.hsc_reserve(ctx.handle, int(nbytes)))


def hsc_set_autotune(ctx: Context, enable: bool = True):
    _check(_lib.hsc_set_autotune(ctx.handle, 1 if enable else 0))
    ctx.autotune = bool(enable)


def hsc_tune_report(ctx: Context) -> str:
    return _lib.hsc_tune_report(ctx.handle).decode(errors="replace")


def hsc_tune_save(ctx: Context) -> str:
    n = _lib.hsc_tune_save(ctx.handle, None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    _lib.hsc_tune_save(ctx.handle, buf, n + 1)
    return buf.value.decode()


def hsc_tune_load(ctx: Context, text: str):
    _check(_lib.hsc_tune_load(ctx.handle, text.encode()))


def hsc_force_launch_config(ctx: Context, ppt: int = 0, block: int = 128, waves: int = 1, vec: int = 1,
                            chunk: int = 0):
    _check(_lib.hsc_force_launch_config(ctx.handle, int(ppt), int(block), int(waves), int(vec), int(chunk)))


def hsc_fp32_peak_probe(ctx: Context, sink: torch.Tensor, iters: int, ctas: int = 0, stream=None) -> int:
    """One launch of the FP32 FFMA probe; returns its FMA lane-operations.
    sink: device float32 with at least ctas x 256 elements (ctas <= 0: 8 per SM)."""
    n = int(ctas) if ctas > 0 else 8 * torch.cuda.get_device_properties(sink.device).multi_processor_count
    if sink.dtype != torch.float32 or sink.numel() < n * 256 or not sink.is_cuda:
        raise ValueError("sink must be a device float32 tensor of at least ctas x 256 elements")
    ops = ctypes.c_int64(0)
    _check(_lib.hsc_fp32_peak_probe(ctx.handle, n, int(iters), _ptr(sink), ctypes.byref(ops), _stream(stream)))
    return int(ops.value)


def hsc_tanh_peak_probe(ctx: Context, sink: torch.Tensor, iters: int, ctas: int = 0, packed: bool = False,
                        stream=None) -> int:
    """One launch of the MUFU tanh probe; returns its tanh results (FP32, or
    f16 pairs when packed).  sink: device float32 with at least ctas x 256
    elements (ctas <= 0: 8 per SM)."""
    n = int(ctas) if ctas > 0 else 8 * torch.cuda.get_device_properties(sink.device).multi_processor_count
    if sink.dtype != torch.float32 or sink.numel() < n * 256 or not sink.is_cuda:
        raise ValueError("sink must be a device float32 tensor of at least ctas x 256 elements")
    ops = ctypes.c_int64(0)
    _check(_lib.hsc_tanh_peak_probe(ctx.handle, n, int(iters), int(packed), _ptr(sink), ctypes.byref(ops),
                                    _stream(stream)))
    return int(ops.value)


def hsc_shade_latent_scratch_bytes(pixels: int, k: int, mode: int, latent_dt: int) -> int:
    return int(_lib.hsc_shade_latent_scratch_bytes(int(pixels), int(k), int(mode), int(latent_dt)))


def hsc_cmf_weights(ctx: Context, n: int, lambda0: float, dlambda: float, T_out: torch.Tensor, stream=None):
    if T_out.dtype != torch.float32 or T_out.shape != (3, n):
        raise ValueError("T_out must be (3, n) float32")
    _check(_lib.hsc_cmf_weights(ctx.handle, int(n), float(lambda0), float(dlambda), _ptr(T_out), _stream(stream)))


def hsc_fold_xyz(ctx: Context, T: torch.Tensor, D: torch.Tensor, M_out: torch.Tensor, stream=None):
    n, k = D.shape
    if T.shape != (3, n) or M_out.shape != (3, k):
        raise ValueError("shapes: T (3,n), D (n,k), M_out (3,k)")
    _check(_lib.hsc_fold_xyz(ctx.handle, _ptr(T), _ptr(D), int(k), int(n), _ptr(M_out), _stream(stream)))


def hsc_encode(ctx: Context, E: torch.Tensor, spectra: torch.Tensor, codes_out: torch.Tensor, stream=None):
    k, n = E.shape
    m = spectra.shape[0]
    if spectra.shape != (m, n) or codes_out.shape != (m, k):
        raise ValueError("shapes: E (k,n), spectra (m,n), codes_out (m,k)")
    if E.dtype != torch.float32 or spectra.dtype != torch.float32:
        raise ValueError("E and spectra must be float32")
    _check(_lib.hsc_encode(ctx.handle, _ptr(E), int(k), int(n), _ptr(spectra), int(m), _ptr(codes_out),
                           _dt(codes_out), _stream(stream)))


def hsc_encode_assets(ctx: Context, E: torch.Tensor, mat_spectra: torch.Tensor, mat_codes_out: torch.Tensor,
                      light_spd: torch.Tensor, light_codes_out: torch.Tensor, stream=None):
    k, n = E.shape
    nm, nl = mat_spectra.shape[0], light_spd.shape[0]
    if (mat_spectra.shape != (nm, n) or light_spd.shape != (nl, n) or mat_codes_out.shape != (nm, k)
            or light_codes_out.shape != (nl, k)):
        raise ValueError("shapes: E (k,n), mat_spectra (n_mat,n), light_spd (L,n), codes (n_mat,k) and (L,k)")
    if E.dtype != torch.float32 or mat_spectra.dtype != torch.float32 or light_spd.dtype != torch.float32:
        raise ValueError("E and spectra must be float32")
    if mat_codes_out.dtype != light_codes_out.dtype:
        raise ValueError("material and light codes must have one dtype")
    _check(_lib.hsc_encode_assets(ctx.handle, _ptr(E), int(k), int(n), _ptr(mat_spectra), int(nm),
                                  _ptr(mat_codes_out), _ptr(light_spd), int(nl), _ptr(light_codes_out),
                                  _dt(mat_codes_out), _stream(stream)))


def hsc_shade_pass(ctx: Context, g1: GBuffer, g2: Optional[GBuffer], mat_codes: torch.Tensor, lights: Lights,
                   light_codes: torch.Tensor, b: int, rgb_out: torch.Tensor, stream=None):
    k = mat_codes.shape[1]
    if rgb_out.shape != (g1.pixels, 3) or rgb_out.dtype != torch.float32:
        raise ValueError("rgb_out must be (P,3) float32")
    _check(_lib.hsc_shade_pass(ctx.handle, _gb(g1), _gb(g2), g1.pixels, _ptr(mat_codes), int(mat_codes.shape[0]),
                               ctypes.byref(lights._s), _ptr(light_codes), int(k), _dt(mat_codes), int(b),
                               _ptr(rgb_out), _stream(stream)))


def hsc_reassemble(ctx: Context, passes: Sequence[torch.Tensor], latent_out: torch.Tensor, stream=None):
    B = len(passes)
    P = latent_out.shape[0]
    arr = (_vp * B)(*[_ptr(p) for p in passes])
    _check(_lib.hsc_reassemble(ctx.handle, arr, B, int(P), _ptr(latent_out), _stream(stream)))


def hsc_shade_latent(ctx: Context, g1: GBuffer, g2: Optional[GBuffer], mat_codes: torch.Tensor, lights: Lights,
                     light_codes: torch.Tensor, mode: int, latent_out: torch.Tensor,
                     latent_scales: Optional[torch.Tensor] = None, xyz_out: Optional[torch.Tensor] = None,
                     M_xyz: Optional[torch.Tensor] = None, stream=None, srgb8_out: Optional[torch.Tensor] = None):
    k = mat_codes.shape[1]
    if light_codes.shape != (lights.count, k) or light_codes.dtype != mat_codes.dtype:
        raise ValueError("light_codes must be (L,k) with the material codes' dtype")
    if latent_out.shape != (g1.pixels, k):
        raise ValueError("latent_out must be (P,k)")
    if srgb8_out is not None and (srgb8_out.shape != (g1.pixels, 3) or srgb8_out.dtype != torch.uint8):
        raise ValueError("srgb8_out must be (P,3) uint8")
    _check(_lib.hsc_shade_latent(ctx.handle, _gb(g1), _gb(g2), g1.pixels, _ptr(mat_codes), int(mat_codes.shape[0]),
                                 ctypes.byref(lights._s), _ptr(light_codes), int(k), _dt(mat_codes), int(mode),
                                 _ptr(latent_out), _dt(latent_out), _ptr(latent_scales), _ptr(xyz_out),
                                 _ptr(srgb8_out), _ptr(M_xyz), _stream(stream)))


def hsc_shade_latent_assets(ctx: Context, g1: GBuffer, g2: Optional[GBuffer], E: torch.Tensor,
                            mat_spectra: torch.Tensor, lights: Lights, light_spd: torch.Tensor,
                            latent_out: torch.Tensor, xyz_out: Optional[torch.Tensor] = None,
                            M_xyz: Optional[torch.Tensor] = None, srgb8_out: Optional[torch.Tensor] = None,
                            stream=None):
    """One-launch latent frame from spectral assets (the encode in the shading
    prologue); see include/hsc.h."""
    k, n = E.shape
    if E.dtype != torch.float32 or mat_spectra.dtype != torch.float32 or light_spd.dtype != torch.float32:
        raise ValueError("E and the spectra must be float32")
    if mat_spectra.shape[1] != n or light_spd.shape != (lights.count, n):
        raise ValueError("spectra must be (n_mat, n) and (L, n)")
    if latent_out.shape != (g1.pixels, k) or latent_out.dtype != torch.float32:
        raise ValueError("latent_out must be (P, k) float32")
    if srgb8_out is not None and (srgb8_out.shape != (g1.pixels, 3) or srgb8_out.dtype != torch.uint8):
        raise ValueError("srgb8_out must be (P,3) uint8")
    _check(_lib.hsc_shade_latent_assets(ctx.handle, _gb(g1), _gb(g2), g1.pixels, _ptr(E), int(k), int(n),
                                        _ptr(mat_spectra), int(mat_spectra.shape[0]), ctypes.byref(lights._s),
                                        _ptr(light_spd), _ptr(latent_out), _ptr(xyz_out), _ptr(srgb8_out),
                                        _ptr(M_xyz), _stream(stream)))


def hsc_quantize_fp8(ctx: Context, latent: torch.Tensor, codes_out: torch.Tensor, scales_out: torch.Tensor,
                     stream=None):
    P, k = latent.shape
    _check(_lib.hsc_quantize_fp8(ctx.handle, _ptr(latent), int(P), int(k), _ptr(codes_out), _ptr(scales_out),
                                 _stream(stream)))


def hsc_quantize_fp8_noalloc(latent: torch.Tensor, codes_out: torch.Tensor, scales_out: torch.Tensor, stream=None):
    """Same result as hsc_quantize_fp8, for callers that may not allocate:
    needs no Context, runs on the current device, scratch in a static array."""
    P, k = latent.shape
    _check(_lib.hsc_quantize_fp8_noalloc(_ptr(latent), int(P), int(k), _ptr(codes_out), _ptr(scales_out),
                                         _stream(stream)))


def hsc_decode_xyz(ctx: Context, latent: torch.Tensor, M_xyz: torch.Tensor, xyz_out: torch.Tensor,
                   scales: Optional[torch.Tensor] = None, srgb8_out: Optional[torch.Tensor] = None, stream=None):
    P, k = latent.shape
    if (xyz_out is not None and xyz_out.shape != (P, 3)) or M_xyz.shape != (3, k):
        raise ValueError("shapes: latent (P,k), M_xyz (3,k), xyz_out (P,3)")
    _check(_lib.hsc_decode_xyz(ctx.handle, _ptr(latent), _dt(latent), _ptr(scales), int(P), int(k), _ptr(M_xyz),
                               _ptr(xyz_out), _ptr(srgb8_out), _stream(stream)))


def hsc_decode_spectra(ctx: Context, latent: torch.Tensor, D: torch.Tensor, spectra_out: torch.Tensor,
                       scales: Optional[torch.Tensor] = None, stream=None):
    P, k = latent.shape
    n = D.shape[0]
    if D.shape != (n, k) or spectra_out.shape != (P, n):
        raise ValueError("shapes: latent (P,k), D (n,k), spectra_out (P,n)")
    _check(_lib.hsc_decode_spectra(ctx.handle, _ptr(latent), _dt(latent), _ptr(scales), int(P), int(k), _ptr(D),
                                   int(n), _ptr(spectra_out), _stream(stream)))


def hsc_shade_spectral(ctx: Context, g1: GBuffer, g2: Optional[GBuffer], mat_spectra: torch.Tensor, lights: Lights,
                       light_spd: torch.Tensor, T: torch.Tensor, xyz_out: torch.Tensor,
                       spectra_out: Optional[torch.Tensor] = None, stream=None):
    n = mat_spectra.shape[1]
    if light_spd.shape != (lights.count, n) or T.shape != (3, n) or xyz_out.shape != (g1.pixels, 3):
        raise ValueError("shapes: mat_spectra (m,n), light_spd (L,n), T (3,n), xyz_out (P,3)")
    _check(_lib.hsc_shade_spectral(ctx.handle, _gb(g1), _gb(g2), g1.pixels, _ptr(mat_spectra),
                                   int(mat_spectra.shape[0]), ctypes.byref(lights._s), _ptr(light_spd), int(n),
                                   _ptr(T), _ptr(xyz_out), _ptr(spectra_out), _stream(stream)))


def hsc_delta_e(ctx: Context, xyz_test: torch.Tensor, xyz_ref: torch.Tensor, T: torch.Tensor,
                stats_out: torch.Tensor, de_out: Optional[torch.Tensor] = None, stream=None):
    P = xyz_ref.shape[0]
    if stats_out.dtype != torch.float64 or stats_out.numel() < 8:
        raise ValueError("stats_out must hold 8 float64")
    _check(_lib.hsc_delta_e(ctx.handle, _ptr(xyz_test), _ptr(xyz_ref), int(P), _ptr(T), int(T.shape[1]),
                            _ptr(de_out), _ptr(stats_out), _stream(stream)))


# ------------------------------------------------------------------- batches

class BatchFrame:
    """One frame of a batched launch (see hsc_frame in include/hsc.h).  Keeps
    references to its tensors so they outlive the batch."""

    def __init__(self, g1: GBuffer, g2: Optional[GBuffer], mat_codes: torch.Tensor, lights: Lights,
                 light_codes: torch.Tensor, M_xyz: torch.Tensor, xyz_out: torch.Tensor,
                 latent_out: Optional[torch.Tensor] = None):
        k = int(mat_codes.shape[1])
        if light_codes.shape != (lights.count, k) or light_codes.dtype != mat_codes.dtype:
            raise ValueError("light_codes must be (L,k) with the material codes' dtype")
        if M_xyz.shape != (3, k) or xyz_out.shape != (g1.pixels, 3):
            raise ValueError("shapes: M_xyz (3,k), xyz_out (P,3)")
        if latent_out is not None and latent_out.shape != (g1.pixels, k):
            raise ValueError("latent_out must be (P,k)")
        self.keep = (g1, g2, mat_codes, lights, light_codes, M_xyz, xyz_out, latent_out)
        self.s = _Frame()
        self.s.g1 = g1._s
        if g2 is not None:
            self.s.g2 = g2._s
        self.s.has_g2 = 1 if g2 is not None else 0
        self.s.pixels = g1.pixels
        self.s.mat_codes = _ptr(mat_codes)
        self.s.n_mat = int(mat_codes.shape[0])
        self.s.lights = lights._s
        self.s.light_codes = _ptr(light_codes)
        self.s.k = k
        self.s.code_dt = _dt(mat_codes)
        self.s.M_xyz = _ptr(M_xyz)
        self.s.xyz_out = _ptr(xyz_out)
        self.s.latent_out = _ptr(latent_out)


class Batch:
    def __init__(self, ctx: Context, frames: Sequence[BatchFrame]):
        self.ctx = ctx
        self.frames = list(frames)
        arr = (_Frame * len(self.frames))(*[f.s for f in self.frames])
        self._h = _vp()
        _check(_lib.hsc_batch_create(ctx.handle, arr, len(self.frames), ctypes.byref(self._h)))

    def close(self):
        if self._h:
            _lib.hsc_batch_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hsc_batch_create(ctx: Context, frames: Sequence[BatchFrame]) -> Batch:
    return Batch(ctx, frames)


def hsc_batch_shade(ctx: Context, batch: Batch, stream=None):
    _check(_lib.hsc_batch_shade(ctx.handle, batch._h, _stream(stream)))


def hsc_batch_destroy(batch: Batch):
    batch.close()


def hsc_shade_frames(ctx: Context, frames: Sequence[BatchFrame], stream=None):
    """Asynchronous one-shot batched launch (continuous batching)."""
    arr = (_Frame * len(frames))(*[f.s for f in frames])
    _check(_lib.hsc_shade_frames(ctx.handle, arr, len(frames), _stream(stream)))


def hsc_upsample_rgb(ctx: Context, rgb: torch.Tensor, W1: torch.Tensor, b1: torch.Tensor, W2: torch.Tensor,
                     b2: torch.Tensor, W3: torch.Tensor, b3: torch.Tensor, z_out: torch.Tensor, stream=None):
    """RGB-to-latent upsampling network (Sec. 5); see include/hsc.h."""
    P = rgb.shape[0]
    k = W3.shape[0]
    if rgb.shape != (P, 3) or W1.shape != (128, 3) or W2.shape != (128, 128) or W3.shape != (k, 128) \
            or b1.shape != (128,) or b2.shape != (128,) or b3.shape != (k,) or z_out.shape != (P, k):
        raise ValueError("shapes: rgb (P,3), W1 (128,3), W2 (128,128), W3 (k,128), biases, z_out (P,k)")
    for t in (rgb, W1, b1, W2, b2, W3, b3, z_out):
        if t.dtype != torch.float32:
            raise ValueError("all tensors must be float32")
    _check(_lib.hsc_upsample_rgb(ctx.handle, _ptr(rgb), int(P), _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2), _ptr(W3),
                                 _ptr(b3), int(k), _ptr(z_out), _stream(stream)))


def hsc_path_trace(ctx: Context, quads: torch.Tensor, spheres: torch.Tensor, camera: torch.Tensor, width: int,
                   height: int, spp: int, depth: int, seed: int, materials: torch.Tensor, emit: torch.Tensor,
                   to_xyz: torch.Tensor, xyz_out: torch.Tensor, channels_out: Optional[torch.Tensor] = None,
                   stream=None):
    """Path tracing with per-channel throughput (spectra or codes); see include/hsc.h."""
    C = emit.shape[0]
    P = width * height
    if quads.shape[1:] != (8,) or spheres.shape[1:] != (5,) or camera.shape != (4, 3) or \
            materials.shape[1:] != (C,) or to_xyz.shape != (3, C) or xyz_out.shape != (P, 3):
        raise ValueError("shapes: quads (Q,8), spheres (S,5), camera (4,3), materials (M,C), to_xyz (3,C), xyz (P,3)")
    if channels_out is not None and channels_out.shape != (P, C):
        raise ValueError("channels_out must be (P, C)")
    _check(_lib.hsc_path_trace(ctx.handle, _ptr(quads), int(quads.shape[0]), _ptr(spheres), int(spheres.shape[0]),
                               _ptr(camera), int(width), int(height), int(spp), int(depth), int(seed) & 0xFFFFFFFF,
                               _ptr(materials), int(materials.shape[0]), _ptr(emit), int(C), _ptr(to_xyz),
                               _ptr(xyz_out), _ptr(channels_out), _stream(stream)))


def hsc_codec_fit_step(ctx: Context, R_all: torch.Tensor, L_all: torch.Tensor, pair_r: torch.Tensor,
                       pair_l: torch.Tensor, pair_scale: torch.Tensor, T: torch.Tensor, weights: torch.Tensor,
                       Et: torch.Tensor, Dt: torch.Tensor, mE: torch.Tensor, vE: torch.Tensor, mD: torch.Tensor,
                       vD: torch.Tensor, step: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                       eps: float = 1e-8, softplus_beta: float = 10.0, active: Optional[torch.Tensor] = None,
                       losses_out: Optional[torch.Tensor] = None, grad_out: Optional[torch.Tensor] = None,
                       stream=None):
    """One Adam step of the softplus-parameterised codec for every variant; see include/hsc.h."""
    V, k, n = _fit_shapes(R_all, L_all, pair_r, pair_l, pair_scale, T, weights, Et, Dt, active)
    P = pair_r.shape[0]
    for m in (mE, vE):
        if m.shape != Et.shape:
            raise ValueError("moments of E~ must match Et")
    for m in (mD, vD):
        if m.shape != Dt.shape:
            raise ValueError("moments of D~ must match Dt")
    _check(_lib.hsc_codec_fit_step(ctx.handle, int(V), int(k), int(n), _ptr(R_all), _ptr(L_all), _ptr(pair_r),
                                   _ptr(pair_l), _ptr(pair_scale), int(P), _ptr(T), _ptr(weights), _ptr(Et),
                                   _ptr(Dt), _ptr(mE), _ptr(vE), _ptr(mD), _ptr(vD), int(step), float(lr),
                                   float(beta1), float(beta2), float(eps), float(softplus_beta), _ptr(active),
                                   _ptr(losses_out), _ptr(grad_out), _stream(stream)))


def _fit_shapes(R_all, L_all, pair_r, pair_l, pair_scale, T, weights, Et, Dt, active):
    V, k, n = Et.shape
    P = pair_r.shape[0]
    if Dt.shape != (V, n, k) or weights.shape != (V, 4) or T.shape != (3, n) or R_all.shape[1] != n \
            or L_all.shape[1] != n or pair_l.shape != (P,) or pair_scale.shape != (P,):
        raise ValueError("shapes: Et (V,k,n), Dt (V,n,k), weights (V,4), T (3,n), rows of n, pairs (P,)")
    if pair_r.dtype != torch.int32 or pair_l.dtype != torch.int32:
        raise ValueError("pair indices must be int32")
    if active is not None and (active.shape != (V,) or active.dtype != torch.int32):
        raise ValueError("active: (V,) int32")
    return V, k, n


def hsc_codec_fit_eval(ctx: Context, R_all: torch.Tensor, L_all: torch.Tensor, pair_r: torch.Tensor,
                       pair_l: torch.Tensor, pair_scale: torch.Tensor, T: torch.Tensor, weights: torch.Tensor,
                       Et: torch.Tensor, Dt: torch.Tensor, softplus_beta: float = 10.0,
                       active: Optional[torch.Tensor] = None, losses_out: Optional[torch.Tensor] = None,
                       E_out: Optional[torch.Tensor] = None, D_out: Optional[torch.Tensor] = None, stream=None):
    """Loss terms (and softplus(E~), softplus(D~)) of every active variant, no step; see include/hsc.h."""
    V, k, n = _fit_shapes(R_all, L_all, pair_r, pair_l, pair_scale, T, weights, Et, Dt, active)
    if (losses_out is not None and losses_out.shape != (V, 5)) or (E_out is not None and E_out.shape != (V, k, n)) \
            or (D_out is not None and D_out.shape != (V, n, k)):
        raise ValueError("outputs: losses (V,5), E (V,k,n), D (V,n,k)")
    _check(_lib.hsc_codec_fit_eval(ctx.handle, int(V), int(k), int(n), _ptr(R_all), _ptr(L_all), _ptr(pair_r),
                                   _ptr(pair_l), _ptr(pair_scale), int(pair_r.shape[0]), _ptr(T), _ptr(weights),
                                   _ptr(Et), _ptr(Dt), float(softplus_beta), _ptr(active), _ptr(losses_out),
                                   _ptr(E_out), _ptr(D_out), _stream(stream)))


def hsc_codec_fit_track(ctx: Context, val_loss: torch.Tensor, Et: torch.Tensor, Dt: torch.Tensor,
                        best_Et: torch.Tensor, best_Dt: torch.Tensor, best_loss: torch.Tensor, wait: torch.Tensor,
                        active: torch.Tensor, patience: int, epochs: Optional[torch.Tensor] = None,
                        n_active_out: Optional[torch.Tensor] = None, stream=None):
    """Early-stopping update of every variant; val_loss is (V,) or the (V, 5) loss table (column 0 is used);
    see include/hsc.h."""
    V, k, n = Et.shape
    if Dt.shape != (V, n, k) or best_Et.shape != Et.shape or best_Dt.shape != Dt.shape:
        raise ValueError("best parameters must match Et (V,k,n) and Dt (V,n,k)")
    if best_loss.shape != (V,) or wait.shape != (V,) or active.shape != (V,) or wait.dtype != torch.int32 \
            or active.dtype != torch.int32:
        raise ValueError("best_loss (V,) float32; wait, active (V,) int32")
    if epochs is not None and (epochs.shape != (V,) or epochs.dtype != torch.int32):
        raise ValueError("epochs: (V,) int32")
    if val_loss.shape == (V,):
        stride = 1
    elif val_loss.dim() == 2 and val_loss.shape[0] == V:
        stride = val_loss.shape[1]
    else:
        raise ValueError("val_loss: (V,) or (V, m)")
    _check(_lib.hsc_codec_fit_track(ctx.handle, int(V), int(k), int(n), _ptr(val_loss), int(stride), _ptr(Et),
                                    _ptr(Dt), _ptr(best_Et), _ptr(best_Dt), _ptr(best_loss), _ptr(wait),
                                    _ptr(active), _ptr(epochs), int(patience), _ptr(n_active_out),
                                    _stream(stream)))


def hsc_chain_eval(ctx: Context, refl: torch.Tensor, lights: torch.Tensor, E: torch.Tensor, D: torch.Tensor,
                   T: torch.Tensor, chain_light: torch.Tensor, chain_refl: torch.Tensor, de94_out: torch.Tensor,
                   de2000_out: torch.Tensor, stats_out: torch.Tensor, stream=None):
    """Multi-bounce chain errors (Sec. 4.5 proxy); see include/hsc.h."""
    k, n = E.shape
    chains, depth = chain_refl.shape
    if de94_out.shape != (depth, chains) or de2000_out.shape != (depth, chains) or stats_out.numel() < 4 * depth:
        raise ValueError("outputs: de (depth, chains), stats 4*depth doubles")
    _check(_lib.hsc_chain_eval(ctx.handle, _ptr(refl), int(refl.shape[0]), _ptr(lights), int(lights.shape[0]),
                               _ptr(E), _ptr(D), int(k), int(n), _ptr(T), _ptr(chain_light), _ptr(chain_refl),
                               int(chains), int(depth), _ptr(de94_out), _ptr(de2000_out), _ptr(stats_out),
                               _stream(stream)))
