"""CPU checks of the C ABI: the library builds, loads, exports exactly the
entry points include/hsc.h declares, and fails cleanly without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hsc.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^HSC_API\s+[\w\s\*]+?\b(hsc_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    return __graft_entry__._build_module().build()


def test_header_declares_the_entry_points():
    names = _declared()
    for must in ("hsc_encode", "hsc_shade_latent", "hsc_decode_xyz", "hsc_decode_spectra", "hsc_shade_spectral",
                 "hsc_shade_pass", "hsc_reassemble", "hsc_cmf_weights", "hsc_fold_xyz", "hsc_quantize_fp8",
                 "hsc_delta_e", "hsc_create", "hsc_destroy", "hsc_sync"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (hsc_\w+)", out))
    declared = set(_declared())
    assert declared <= exported, declared - exported
    # nothing beyond the header leaks out of the library
    assert exported <= declared, exported - declared
    lib = ctypes.CDLL(lib_path)
    for name in declared:
        assert getattr(lib, name) is not None


def test_binding_covers_the_header(lib_path):
    import paper_2602_18741_gb300 as hsc
    assert set(hsc.EXPORTED) == set(_declared())


def test_host_only_calls_work_without_gpu(lib_path):
    import paper_2602_18741_gb300 as hsc
    assert hsc.hsc_shade_latent_scratch_bytes(1000, 6, hsc.HSC_FUSED, hsc.HSC_F32) == 0
    assert hsc.hsc_shade_latent_scratch_bytes(1000, 6, hsc.HSC_PASSES, hsc.HSC_F32) == 24000
    assert hsc.hsc_shade_latent_scratch_bytes(1000, 9, hsc.HSC_PASSES, hsc.HSC_FP8_E4M3) == 72000
    lib = ctypes.CDLL(lib_path)
    lib.hsc_last_error.restype = ctypes.c_char_p
    assert lib.hsc_last_error() is not None


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="checks the no-GPU failure path")
def test_create_fails_cleanly_without_gpu(lib_path):
    import paper_2602_18741_gb300 as hsc
    with pytest.raises(hsc.HscError) as ei:
        hsc.Context(0)
    assert ei.value.status in (hsc.HSC_ERR_CUDA, hsc.HSC_ERR_INVALID_ARG)


def test_null_context_is_rejected(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.hsc_sync.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.hsc_sync(None, None) == 1     # HSC_ERR_INVALID_ARG
    lib.hsc_encode.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] * 2 + [ctypes.c_void_p, ctypes.c_int,
                                                                            ctypes.c_void_p, ctypes.c_int,
                                                                            ctypes.c_void_p]
    assert lib.hsc_encode(None, None, 6, 31, None, 4, None, 0, None) == 1
    lib.hsc_encode_assets.argtypes = ([ctypes.c_void_p] * 2 + [ctypes.c_int] * 2 +
                                      [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p] * 2 +
                                      [ctypes.c_int, ctypes.c_void_p])
    assert lib.hsc_encode_assets(None, None, 6, 81, None, 288, None, None, 64, None, 0, None) == 1
