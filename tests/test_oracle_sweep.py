"""Pins of the codec-sweep oracle (Sec. 4.5): early stopping, training with
validation, selection."""
import numpy as np

import hsc_inputs as hi
from oracle import cmf, codec
from oracle import sweep as sw


def _run(seq, patience):
    st = sw.early_stop_init(1)
    imp = []
    for v in seq:
        imp.append(bool(sw.early_stop_update(st, [v], patience)[0]))
    return st, imp


def test_stops_patience_epochs_after_the_last_improvement():
    st, imp = _run([5.0, 4.0, 4.5, 3.0, 3.0, 3.5, 9.0], patience=3)
    assert imp == [True, True, False, True, False, False, False]
    assert not st.active[0] and st.epochs[0] == 7 and st.best[0] == 3.0 and st.wait[0] == 3
    st, _ = _run([5.0, 4.0, 4.5, 3.0, 3.0, 3.5], patience=3)
    assert st.active[0] and st.wait[0] == 2


def test_ties_and_nan_never_improve():
    st, imp = _run([1.0, 1.0, np.nan, np.nan], patience=3)
    assert imp == [True, False, False, False] and not st.active[0] and st.best[0] == 1.0
    st, imp = _run([np.nan, 2.0], patience=5)
    assert imp == [False, True] and st.best[0] == 2.0


def test_falling_sequence_never_stops_and_stopped_variants_are_left_alone():
    st, imp = _run(list(np.arange(20, 0, -1.0)), patience=1)
    assert all(imp) and st.active[0] and st.epochs[0] == 20
    st = sw.early_stop_init(3)
    st.active[1] = False
    st.best[1] = 0.5
    imp = sw.early_stop_update(st, [1.0, 0.1, np.nan], patience=1)
    assert list(imp) == [True, False, False]
    assert st.best[1] == 0.5 and st.epochs[1] == 0 and not st.active[1]
    assert not st.active[2] and st.epochs[2] == 1


def test_band_initialisation_through_the_softplus():
    Et, Dt = sw.band_init_raw(6, 31)
    E, D = codec.softplus(Et), codec.softplus(Dt)
    E0, D0 = codec.band_init(6, 31)
    assert np.allclose(E, np.maximum(E0, 1e-3), rtol=1e-12, atol=0)
    assert np.allclose(D, np.maximum(D0, 1e-3), rtol=1e-12, atol=0)


def _tiny():
    g = (400.0, 20.0, 16)
    ts = hi.training_set(g, n_smooth=24, n_saw=8, n_bb=8, n_nb=8, pairs=96)
    sched = hi.sweep_schedule(ts, epochs=8, batch=32, val_pairs=40, seed=5)
    T = cmf.cmf_weights(*g)
    R = ts.R.astype(np.float32).astype(np.float64)
    L = ts.L.astype(np.float32).astype(np.float64)
    return g, ts, sched, T, R, L


def test_kept_parameters_are_the_best_epoch():
    g, ts, sched, T, R, L = _tiny()
    Et0, Dt0 = sw.band_init_raw(3, g[2])
    w = (0.5, 0.75, 1.0, 0.5)
    # a large learning rate makes the validation loss go up and down
    res = sw.train_variant(R, L, T, w, sched, Et0, Dt0, epochs=8, patience=2, lr=0.05)
    h = np.asarray(res.history)
    b = int(np.argmin(h))
    assert res.best == h[b]
    assert res.epochs == len(h)
    assert res.epochs == b + 1 + 2 < 8           # stopped early: exactly patience epochs after the best
    val = sw._pairs(R, L, sched.val_r, sched.val_l, sched.val_s, T)
    wd = {"e2e": 0.5, "rec": 0.75, "code": 1.0, "col": 0.5}
    assert codec.losses(codec.softplus(res.Et), codec.softplus(res.Dt), val, wd)["total"] == res.best
    # the training loss of a small step size goes down
    res2 = sw.train_variant(R, L, T, w, sched, Et0, Dt0, epochs=3, patience=5, lr=1e-3)
    assert res2.history[-1] < res2.history[0] and res2.epochs == 3


def test_zero_epochs_keep_the_initial_parameters():
    g, ts, sched, T, R, L = _tiny()
    Et0, Dt0 = sw.band_init_raw(3, g[2])
    res = sw.train_variant(R, L, T, (1, 1, 1, 1), sched, Et0, Dt0, epochs=0, patience=2)
    assert np.array_equal(res.Et, Et0) and np.array_equal(res.Dt, Dt0) and res.epochs == 0 and res.history == []


def test_selection():
    assert sw.select([3.0, 1.0, 1.0, 2.0]) == 1
    assert sw.select([np.nan, 2.0, np.nan, 0.5]) == 3
    assert sw.select([np.nan, np.nan]) == -1
    # the (numerically) identity codec scores ~0 and wins against the band codec
    g = (400.0, 10.0, 30)
    ts = hi.training_set(g, n_smooth=16, n_saw=4, n_bb=4, n_nb=4, pairs=8)
    T = cmf.cmf_weights(*g)
    rng = np.random.default_rng(1)
    cl = rng.integers(0, ts.L.shape[0], 50)
    cr = rng.integers(0, ts.R.shape[0], (50, 3))
    ident = (np.where(np.eye(30) > 0, codec.softplus_inverse(1.0), -10.0),) * 2
    band = sw.band_init_raw(6, 30)
    s = sw.selection_scores(ts.R, ts.L, T, [band, ident], cl, cr)
    assert s[1] < 1e-9 < s[0] and sw.select(s) == 1
