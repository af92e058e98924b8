"""Pins of the RGB-to-latent upsampling oracle (Sec. 5)."""
import numpy as np

from oracle import upsample as up


def test_silu_closed_forms():
    assert up.silu(0.0) == 0.0
    # x / (1 + e^-x) at x = +-1 and 2, written from e = 2.718281828459045
    e = 2.718281828459045
    assert np.isclose(up.silu(1.0), 1.0 / (1.0 + 1.0 / e), rtol=1e-15)
    assert np.isclose(up.silu(-1.0), -1.0 / (1.0 + e), rtol=1e-15)
    assert np.isclose(up.silu(2.0), 2.0 / (1.0 + 1.0 / (e * e)), rtol=1e-15)
    # no overflow far out; silu(x) -> x and -> 0-
    assert np.isclose(up.silu(800.0), 800.0) and -1e-300 < up.silu(-800.0) <= 0.0
    # the derivative by central differences
    x = np.linspace(-6, 6, 25)
    h = 1e-6
    assert np.allclose(up.silu_grad(x), (up.silu(x + h) - up.silu(x - h)) / (2 * h), atol=1e-8)


def test_brute_force_loops_match_matrix_form():
    p = up.init_params(5, hidden=7, seed=3)
    rng = np.random.default_rng(1)
    C = rng.uniform(0, 1, (4, 3))
    z = up.forward(p, C)
    for i in range(4):
        assert np.allclose(z[i], up.brute_force_forward(p, C[i]), rtol=1e-13, atol=1e-15)


def test_zero_output_weights_give_the_bias():
    p = up.init_params(6, seed=2)
    p.W3[:] = 0.0
    C = np.random.default_rng(0).uniform(0, 1, (10, 3))
    assert np.array_equal(up.forward(p, C), np.tile(p.b3, (10, 1)))


def test_one_hidden_unit_by_hand():
    # W1 = [2, 0, 0], b1 = -1, W2 = [[3]], b2 = 0.5, W3 = [[1], [-2]], b3 = [0, 1]
    p = up.Params(np.array([[2.0, 0.0, 0.0]]), np.array([-1.0]), np.array([[3.0]]), np.array([0.5]),
                  np.array([[1.0], [-2.0]]), np.array([0.0, 1.0]))
    c = np.array([[0.75, 0.3, 0.9]])
    a1 = 2.0 * 0.75 - 1.0                      # 0.5
    h1 = a1 / (1.0 + np.exp(-a1))
    a2 = 3.0 * h1 + 0.5
    h2 = a2 / (1.0 + np.exp(-a2))
    assert np.allclose(up.forward(p, c), [[h2, 1.0 - 2.0 * h2]], rtol=1e-15)


def test_gradient_by_central_differences():
    p = up.init_params(4, hidden=6, seed=5)
    rng = np.random.default_rng(7)
    C = rng.uniform(0, 1, (9, 3))
    Z = rng.normal(0, 0.3, (9, 4))
    g = up.gradient(p, C, Z)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a = getattr(p, name)
        ga = getattr(g, name)
        for idx in list(np.ndindex(a.shape))[:12]:
            old = a[idx]
            a[idx] = old + h
            lp = up.loss(p, C, Z)
            a[idx] = old - h
            lm = up.loss(p, C, Z)
            a[idx] = old
            assert np.isclose(ga[idx], (lp - lm) / (2 * h), rtol=1e-5, atol=1e-8), (name, idx)


def test_fit_lowers_the_loss():
    rng = np.random.default_rng(11)
    C = rng.uniform(0, 1, (64, 3))
    M = rng.uniform(0, 1, (3, 6))
    Z = C @ M + 0.1 * np.sin(3 * C[:, :1])
    p0 = up.init_params(6, hidden=32, seed=0)
    p, log = up.fit(C, Z, 6, steps=400, hidden=32, seed=0)
    assert log.losses[-1] < 0.1 * up.loss(p0, C, Z)


def test_bf16_contract_reduces_and_stays_within_its_bound():
    p = up.init_params(6, seed=9)
    C = np.random.default_rng(4).uniform(0, 1, (50, 3))
    z = up.forward(p, C)
    assert np.array_equal(up.forward_bf16(p, C, rounding=False), z)
    zb = up.forward_bf16(p, C)
    # each rounding is at most 2^-9 relative; a few layers of them stay well
    # inside 3 % of the output scale
    assert np.max(np.abs(zb - z)) <= 0.03 * np.max(np.abs(z))
    assert np.max(np.abs(zb - z)) > 0.0


def test_f16_contract_reduces_and_is_tighter_than_bf16():
    p = up.init_params(6, seed=9)
    C = np.random.default_rng(4).uniform(0, 1, (50, 3))
    z = up.forward(p, C)
    assert np.array_equal(up.forward_f16(p, C, rounding=False), z)
    zh = up.forward_f16(p, C)
    zb = up.forward_bf16(p, C)
    # each f16 rounding is at most 2^-11 relative, 8 times below bf16's 2^-8:
    # a few layers of them stay inside 0.5 % of the output scale and below the
    # bf16 contract's own distance from the exact network
    err_h = np.max(np.abs(zh - z))
    assert 0.0 < err_h <= 0.005 * np.max(np.abs(z))
    assert err_h < np.max(np.abs(zb - z))
    # the two contracts round at different places: a planted bf16 rounding in
    # the f16 path would show up as a distance of bf16 size
    assert not np.array_equal(zh, zb)
