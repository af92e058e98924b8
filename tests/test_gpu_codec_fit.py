"""Batched codec fitting (softplus parameterisation, Adam; Sec. 4.1-4.5)
against the FP64 oracle.

The loss terms are FP32 sums over P x n = 10,368 elements (relative error a
few 1e-6), so they are compared at 1e-4 relative; the gradients are sums of
the same size, compared element-wise at 1e-4 of the largest component.  The
first Adam step moves a parameter by lr against the sign of its gradient, so
after one step the parameters agree wherever the gradient is not tiny."""
import numpy as np
import pytest

import hsc_inputs as hi
from oracle import cmf, codec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2602_18741_gb300 as hsc
    ctx = hsc.Context(0)
    yield hsc, ctx, torch.device("cuda:0")
    ctx.close()


def _setup(k, grid_spec, V, P, seed):
    ts = hi.training_set(grid_spec, n_smooth=96, n_saw=16, n_bb=24, n_nb=24, pairs=P)
    rng = np.random.default_rng(seed)
    n = grid_spec[2]
    E0, D0 = codec.band_init(k, n)
    Et = np.stack([codec.softplus_inverse(np.maximum(E0, 1e-3)) + rng.normal(0, 0.02, (k, n)) for _ in range(V)])
    Dt = np.stack([codec.softplus_inverse(np.maximum(D0, 1e-3)) + rng.normal(0, 0.02, (n, k)) for _ in range(V)])
    W = rng.uniform(0.2, 1.5, (V, 4))
    T = cmf.cmf_weights(*grid_spec)
    return ts, Et, Dt, W, T


def _dev(a, dev, dt=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt or np.float32)).to(dev)


def _weights(w):
    return {"e2e": w[0], "rec": w[1], "code": w[2], "col": w[3]}


@pytest.mark.parametrize("k,grid_spec,V,P", [(6, hi.GRID_81, 5, 128), (9, hi.GRID_31, 3, 77), (3, (400.0, 10.0, 16), 2, 256)])
def test_step_losses_gradients_and_update(env, k, grid_spec, V, P):
    hsc, ctx, dev = env
    import torch
    ts, Et, Dt, W, T = _setup(k, grid_spec, V, P, seed=k + P)
    Et32 = Et.astype(np.float32).astype(np.float64)
    Dt32 = Dt.astype(np.float32).astype(np.float64)
    d = dict(R_all=_dev(ts.R, dev), L_all=_dev(ts.L, dev), pair_r=_dev(ts.pair_r, dev, np.int32),
             pair_l=_dev(ts.pair_l, dev, np.int32), pair_scale=_dev(ts.pair_scale, dev), T=_dev(T, dev),
             weights=_dev(W, dev))
    gEt, gDt = _dev(Et32, dev), _dev(Dt32, dev)
    mom = [torch.zeros_like(gEt), torch.zeros_like(gEt), torch.zeros_like(gDt), torch.zeros_like(gDt)]
    losses = torch.empty(V, 5, device=dev)
    grad = torch.empty(V, 2 * k * grid_spec[2], device=dev)
    lr = 1e-3
    hsc.hsc_codec_fit_step(ctx, d["R_all"], d["L_all"], d["pair_r"], d["pair_l"], d["pair_scale"], d["T"],
                           d["weights"], gEt, gDt, *mom, step=1, lr=lr, losses_out=losses, grad_out=grad)
    hsc.hsc_sync(ctx)
    batch = codec.make_batch(ts, T)
    L = losses.cpu().numpy()
    G = grad.cpu().numpy()
    En_gpu, Dn_gpu = gEt.cpu().numpy(), gDt.cpu().numpy()
    n = grid_spec[2]
    for v in range(V):
        w = _weights(W[v].astype(np.float32).astype(np.float64))
        E, D = codec.softplus(Et32[v]), codec.softplus(Dt32[v])
        ref = codec.losses(E, D, batch, w)
        for j, key in enumerate(("total", "e2e", "rec", "code", "col")):
            assert abs(L[v, j] - ref[key]) <= 1e-4 * abs(ref[key]) + 1e-12, (v, key, L[v, j], ref[key])
        gE, gD = codec.gradient(E, D, batch, w)
        gEt_ref = gE * codec.softplus_grad(Et32[v])
        gDt_ref = gD * codec.softplus_grad(Dt32[v])
        g_ref = np.concatenate([gEt_ref.ravel(), gDt_ref.ravel()])
        scale = np.abs(g_ref).max()
        assert np.max(np.abs(G[v] - g_ref)) <= 1e-4 * scale, (v, np.max(np.abs(G[v] - g_ref)) / scale)
        st = codec.adam_init(Et32[v], Dt32[v])
        En, Dn, _, _ = codec.adam_softplus_step(Et32[v], Dt32[v], st, batch, w, lr=lr)
        big_E = np.abs(gEt_ref) > 1e-3 * scale
        big_D = np.abs(gDt_ref) > 1e-3 * scale
        assert np.allclose(En_gpu[v][big_E], En[big_E], rtol=0, atol=1e-6)
        assert np.allclose(Dn_gpu[v][big_D], Dn[big_D], rtol=0, atol=1e-6)
        assert n == Et.shape[2]


def test_steps_lower_the_loss_deterministically_and_variants_are_independent(env):
    hsc, ctx, dev = env
    import torch
    k, g, V, P = 6, hi.GRID_81, 4, 128
    ts, Et, Dt, W, T = _setup(k, g, V, P, seed=3)
    d = [_dev(ts.R, dev), _dev(ts.L, dev), _dev(ts.pair_r, dev, np.int32), _dev(ts.pair_l, dev, np.int32),
         _dev(ts.pair_scale, dev), _dev(T, dev)]

    def run(Wv, Ev, Dv, steps=40):
        e, dd = _dev(Ev, dev), _dev(Dv, dev)
        mom = [torch.zeros_like(e), torch.zeros_like(e), torch.zeros_like(dd), torch.zeros_like(dd)]
        lo = torch.empty(len(Wv), 5, device=dev)
        first = None
        for s in range(1, steps + 1):
            hsc.hsc_codec_fit_step(ctx, *d, _dev(Wv, dev), e, dd, *mom, step=s, lr=2e-3, losses_out=lo)
            if s == 1:
                first = lo.clone()
        hsc.hsc_sync(ctx)
        return e.cpu(), dd.cpu(), first.cpu(), lo.cpu()

    a = run(W, Et, Dt)
    b = run(W, Et, Dt)
    assert all(torch.equal(x, y) for x, y in zip(a, b))          # bit for bit run to run
    assert torch.all(a[3][:, 0] < a[2][:, 0])                      # the total loss went down
    one = run(W[2:3], Et[2:3], Dt[2:3])                            # variant 2 alone
    assert torch.equal(one[0][0], a[0][2]) and torch.equal(one[1][0], a[1][2])
