"""Pins of the oracle's codec (Eq. 4-8) against properties the paper fixes."""
import numpy as np

import hsc_inputs as hi
from oracle import cmf, codec


def _small_batch(n=31, pairs=48, seed=5):
    ts = hi.training_set((400.0, 300.0 / (n - 1), n), seed=seed, n_smooth=40, n_saw=8,
                         n_bb=16, n_nb=16, pairs=pairs)
    return codec.make_batch(ts, cmf.cmf_weights(400.0, 300.0 / (n - 1), n))


def test_linearity_is_exact():
    # Eq. 4: a linear codec keeps scaling and addition exact (Sec. 4.1).
    rng = np.random.default_rng(0)
    E = rng.uniform(0, 1, (9, 81))
    D = rng.uniform(0, 1, (81, 9))
    x, y = rng.uniform(0, 1, (2, 81))
    a, b = 0.37, 2.5
    lhs = codec.encode(E, (a * x + b * y)[None])[0]
    rhs = a * codec.encode(E, x[None])[0] + b * codec.encode(E, y[None])[0]
    assert np.max(np.abs(lhs - rhs) / np.abs(rhs)) < 1e-14
    z1, z2 = rng.uniform(0, 1, (2, 9))
    lhs = codec.decode(D, (a * z1 + b * z2)[None])[0]
    rhs = a * codec.decode(D, z1[None])[0] + b * codec.decode(D, z2[None])[0]
    assert np.max(np.abs(lhs - rhs) / np.abs(rhs)) < 1e-14


def test_blockwise_product_is_elementwise():
    # Eq. 6 concatenates per-block products of 3-vectors: on R^k that is the
    # element-wise product, so k/3 RGB passes and one k-channel pass agree.
    rng = np.random.default_rng(1)
    a, b = rng.uniform(0, 1, (2, 10, 9))
    assert np.array_equal(codec.blockwise_hadamard(a, b), a * b)
    for i in range(3):
        assert np.array_equal(codec.blockwise_hadamard(a, b)[:, 3 * i:3 * i + 3],
                              a[:, 3 * i:3 * i + 3] * b[:, 3 * i:3 * i + 3])


def test_band_init_identity_at_k_equals_n():
    E, D = codec.band_init(81, 81)
    assert np.array_equal(E, np.eye(81)) and np.array_equal(D, np.eye(81))
    E, D = codec.band_init(6, 31)
    assert np.allclose(E.sum(axis=1), 1.0)       # each row averages its band
    assert np.allclose(D.sum(axis=1), 1.0)       # every sample in exactly one band
    assert np.allclose(E @ D, np.eye(6))


def test_identity_codec_has_zero_loss_and_is_a_fixed_point():
    # Sec. 3.1: with k = n the coordinate projection (identity) preserves all
    # three operations exactly, so every term of Eq. 8 vanishes.
    b = _small_batch(n=30)
    E, D = codec.band_init(30, 30)
    parts = codec.losses(E, D, b)
    for key in ("e2e", "rec", "code", "col", "total"):
        assert abs(parts[key]) < 1e-28
    gE, gD = codec.gradient(E, D, b)
    assert np.abs(gE).max() < 1e-18 and np.abs(gD).max() < 1e-18
    r = codec.projected_gradient_fit(b, 30, iters=10)
    assert np.array_equal(r.E, E) and np.array_equal(r.D, D)


def test_gradient_matches_central_differences():
    b = _small_batch(n=31, pairs=40)
    rng = np.random.default_rng(2)
    E = rng.uniform(0.05, 0.4, (6, 31))
    D = rng.uniform(0.05, 0.4, (31, 6))
    gE, gD = codec.gradient(E, D, b)
    h = 1e-6
    for (M, G) in ((E, gE), (D, gD)):
        idx = [tuple(rng.integers(0, s) for s in M.shape) for _ in range(25)]
        for ij in idx:
            old = M[ij]
            M[ij] = old + h
            fp = codec.total_loss(E, D, b)
            M[ij] = old - h
            fm = codec.total_loss(E, D, b)
            M[ij] = old
            fd = (fp - fm) / (2 * h)
            assert abs(fd - G[ij]) <= 1e-6 * max(abs(G[ij]), 1e-3 * np.abs(G).max()), (ij, fd, G[ij])


def test_each_loss_term_gradient_separately():
    # a dropped or mis-weighted term would only show in its own weight's direction
    b = _small_batch(n=31, pairs=32, seed=9)
    rng = np.random.default_rng(4)
    E = rng.uniform(0.05, 0.4, (6, 31))
    D = rng.uniform(0.05, 0.4, (31, 6))
    for term in ("e2e", "rec", "code", "col"):
        w = {k: (1.0 if k == term else 0.0) for k in codec.PAPER_WEIGHTS}
        gE, gD = codec.gradient(E, D, b, w)
        h = 1e-6
        ij = (2, 7)
        E[ij] += h
        fp = codec.total_loss(E, D, b, w)
        E[ij] -= 2 * h
        fm = codec.total_loss(E, D, b, w)
        E[ij] += h
        assert abs((fp - fm) / (2 * h) - gE[ij]) <= 1e-6 * max(abs(gE[ij]), 1e-9), term
        ij = (11, 3)
        D[ij] += h
        fp = codec.total_loss(E, D, b, w)
        D[ij] -= 2 * h
        fm = codec.total_loss(E, D, b, w)
        D[ij] += h
        assert abs((fp - fm) / (2 * h) - gD[ij]) <= 1e-6 * max(abs(gD[ij]), 1e-9), term


def test_projected_gradient_descends_and_stays_non_negative():
    b = _small_batch(n=31, pairs=64)
    r = codec.projected_gradient_fit(b, 6, iters=60)
    h = np.asarray(r.history)
    assert np.all(np.diff(h) <= 1e-15)
    assert h[-1] < h[0]
    assert r.E.min() >= 0 and r.D.min() >= 0
    z = codec.encode(r.E, b.R)
    assert z.min() >= 0 and codec.decode(r.D, z).min() >= 0


def test_loss_terms_follow_their_definitions_on_a_tiny_case():
    # one pair, n = 3, k = 3, E = D = 0.5 I: every quantity by hand
    R = np.array([[0.2, 0.4, 0.6]])
    L = np.array([[1.0, 0.5, 0.25]])
    T = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    b = codec.Batch(R, L, T)
    E = 0.5 * np.eye(3)
    D = 0.5 * np.eye(3)
    Y = R * L                                # (0.2, 0.2, 0.15)
    S = 0.5 * (0.5 * R) * (0.5 * L)          # D(E R . E L) = Y / 8
    mse = np.mean((S - Y) ** 2)
    e2e = mse * (2 - 1.0)                    # S parallel to Y: cos = 1
    rec = np.mean((0.25 * R - R) ** 2) + np.mean((0.25 * L - L) ** 2)
    code = np.mean((0.25 * Y - 0.5 * Y) ** 2)
    col = mse                                # T = I
    parts = codec.losses(E, D, b)
    assert abs(parts["e2e"] - e2e) < 1e-15
    assert abs(parts["rec"] - rec) < 1e-15
    assert abs(parts["code"] - code) < 1e-15
    assert abs(parts["col"] - col) < 1e-15
    assert abs(parts["total"] - (0.5 * e2e + 0.75 * rec + 1.0 * code + 0.5 * col)) < 1e-15


def test_softplus_closed_forms_and_inverse():
    b = codec.SOFTPLUS_BETA
    assert np.isclose(codec.softplus(0.0), np.log(2.0) / b, rtol=1e-15)
    assert np.isclose(codec.softplus(5.0), 5.0, rtol=1e-15)       # beta x = 50: exp(-50) below the last bit
    assert 0.0 < codec.softplus(-5.0) < 1e-22
    y = np.array([1e-4, 0.01, 0.3, 1.0, 3.0])
    assert np.allclose(codec.softplus(codec.softplus_inverse(y)), y, rtol=1e-12)
    x = np.linspace(-1, 1, 41)
    h = 1e-6
    assert np.allclose(codec.softplus_grad(x), (codec.softplus(x + h) - codec.softplus(x - h)) / (2 * h), atol=1e-8)


def _rand_batch(seed=0, P=24, n=12):
    rng = np.random.default_rng(seed)
    R = rng.uniform(0, 1, (P, n))
    L = rng.uniform(0.2, 1, (P, n))
    T = rng.uniform(0, 0.1, (3, n))
    return codec.Batch(R, L, T)


def test_gradient_through_softplus_by_finite_differences():
    bt = _rand_batch()
    rng = np.random.default_rng(3)
    Et = rng.normal(-0.1, 0.2, (6, 12))
    Dt = rng.normal(0.0, 0.2, (12, 6))
    gE, gD = codec.gradient(codec.softplus(Et), codec.softplus(Dt), bt)
    gEt, gDt = gE * codec.softplus_grad(Et), gD * codec.softplus_grad(Dt)
    f = lambda a, b: codec.total_loss(codec.softplus(a), codec.softplus(b), bt)
    h = 1e-6
    for (X, G, which) in ((Et, gEt, 0), (Dt, gDt, 1)):
        for idx in [(0, 0), (2, 5), (5, 11)] if which == 0 else [(0, 0), (7, 3), (11, 5)]:
            Xp, Xm = X.copy(), X.copy()
            Xp[idx] += h
            Xm[idx] -= h
            num = (f(Xp, Dt) - f(Xm, Dt)) / (2 * h) if which == 0 else (f(Et, Xp) - f(Et, Xm)) / (2 * h)
            assert np.isclose(G[idx], num, rtol=1e-5, atol=1e-9)


def test_first_adam_step_moves_by_lr():
    bt = _rand_batch(1)
    rng = np.random.default_rng(4)
    Et = rng.normal(-0.1, 0.2, (6, 12))
    Dt = rng.normal(0.0, 0.2, (12, 6))
    st = codec.adam_init(Et, Dt)
    lr = 1e-3
    E2, D2, st2, parts = codec.adam_softplus_step(Et, Dt, st, bt, lr=lr, eps=0.0)
    gE, gD = codec.gradient(codec.softplus(Et), codec.softplus(Dt), bt)
    # with bias correction m_hat / sqrt(v_hat) = sign(g) after one step
    assert np.allclose(E2 - Et, -lr * np.sign(gE), rtol=1e-12, atol=1e-15)
    assert np.allclose(D2 - Dt, -lr * np.sign(gD), rtol=1e-12, atol=1e-15)
    assert st2.t == 1 and parts["total"] == codec.total_loss(codec.softplus(Et), codec.softplus(Dt), bt)
