"""Pins of storage rounding (format definitions) and of the error statistics."""
import numpy as np

import hsc_inputs as hi
from oracle import metrics, quant, shade


def test_bf16_rounding_by_definition():
    # bf16: 8 significand bits, spacing 2^-7 on [1, 2); ties to even.
    x = np.array([1.0, 1 + 2 ** -7, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20], np.float32)
    assert list(quant.round_bf16(x)) == [1.0, 1 + 2 ** -7, 1.0, 1 + 2 ** -6, 1 + 2 ** -7]


def test_f16_rounding_by_definition():
    x = np.array([1.0, 1 + 2 ** -11, 1 + 3 * 2 ** -11, 65504.0], np.float32)
    assert list(quant.round_f16(x)) == [1.0, 1.0, 1 + 2 ** -9, 65504.0]


def test_fp8_e4m3_rounding_by_definition():
    # e4m3 (bias 7, 3 mantissa bits, no infinities): spacing 1/8 on [1, 2);
    # max finite 448 = 1.75 * 2^8; min normal 2^-6; subnormal spacing 2^-9.
    x = np.array([1.0, 1.0625, 1.1875, 448.0, 2 ** -6, 2 ** -9, 2 ** -10, 3 * 2 ** -10, 500.0], np.float32)
    assert list(quant.round_fp8_e4m3(x)) == [1.0, 1.0, 1.25, 448.0, 2 ** -6, 2 ** -9, 0.0, 2 ** -8, 448.0]
    bits = quant.fp8_e4m3_bits(np.array([1.0, 448.0, 0.0, 2 ** -9], np.float32))
    assert list(bits) == [0x38, 0x7E, 0x00, 0x01]


def test_fp8_channel_scale_maps_max_to_448():
    rng = np.random.default_rng(0)
    z = rng.uniform(0, 3, (1000, 6)).astype(np.float32)
    z[:, 4] = 0.0
    s = quant.fp8_channel_scales(z)
    assert s[4] == 1.0
    bits, deq = quant.quantize_fp8(z, s)
    top = np.argmax(z, axis=0)
    for c in (0, 1, 2, 3, 5):
        assert bits[top[c], c] in (0x7E, 0x7F - 1)      # the channel max lands on 448
        # relative error of fp8 e4m3 with RNE is at most 2^-4 for normal values
        big = z[:, c] > 2 ** -6 * s[c]
        assert np.all(np.abs(deq[big, c] - z[big, c]) <= 2 ** -4 * z[big, c] * 1.0001)


def test_nearest_rank_percentile():
    v = [5.0, 1.0, 4.0, 2.0, 3.0]
    assert metrics.nearest_rank(v, 0.95) == 5.0
    assert metrics.nearest_rank(v, 0.5) == 3.0
    assert metrics.nearest_rank(list(range(1, 101)), 0.95) == 95.0
    assert metrics.nearest_rank([7.0], 0.95) == 7.0


def test_rel_xyz_error_floor_and_scale():
    ref = np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 0.0]])
    assert metrics.rel_xyz_error(ref, ref) == 0.0
    got = ref.copy()
    got[0, 2] += 3e-6
    assert abs(metrics.rel_xyz_error(got, ref) - 1e-6) < 1e-15
    got = ref.copy()
    got[1, 0] = 3e-6          # dark pixel: denominator floored at 1e-3 * 3
    assert abs(metrics.rel_xyz_error(got, ref) - 1e-3) < 1e-12


def test_delta_e_stats_of_identical_images_are_zero():
    f = hi.make_frame(3, 8, 8, hi.GRID_31, n_smooth=4, n_saw=0, lights=3, secondary=False)
    _, xyz = shade.shade_spectral(f)
    from oracle import cmf
    st = metrics.delta_e_stats(xyz, xyz, cmf.cmf_weights(*f.grid))
    assert st["de2000_mean"] == 0.0 and st["de2000_p95"] == 0.0 and st["de94_mean"] == 0.0
