"""GPU checks of the learned warm start against the FP64 oracle: network forward
(bfloat16 weights and activations on both sides), gradients, the Adam step,
the feature maps, the solver integration, and what training gains."""

import numpy as np
import pytest

from oracle import cnn_oracle as CO
from oracle import dv_oracle as O
from tests.gpu_common import need_gpu, random_psfs, rel_l2

pytestmark = pytest.mark.gpu

CHANS = (5, 32, 32, 32, 32, 32, 1)


@pytest.fixture(scope="module")
def env():
    return need_gpu()


def oracle_params(flat, bf16_weights=True):
    out, off = [], 0
    for ci, co in zip(CHANS[:-1], CHANS[1:]):
        w = flat[off:off + 9 * ci * co].astype(np.float64).reshape(3, 3, ci, co)
        off += 9 * ci * co
        b = flat[off:off + co].astype(np.float64)
        off += co
        out.append((CO.bf16_round(w) if bf16_weights else w, b))
    return out


def _batch(g, N=2, H=37, W=45):
    x = g.uniform(0, 1, (N, H, W, 5)).astype(np.float32)
    t = g.uniform(-0.2, 0.2, (N, H, W)).astype(np.float32)
    return x, t


def test_forward_matches_oracle(env):
    torch, dv = env
    g = np.random.default_rng(0)
    net = dv.Cnn(seed=3)
    p, _ = net.get_params()
    # a nonzero last layer so the output is not tiny
    p = p * 1.0
    x, _ = _batch(g)
    out = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref, _, _ = CO.forward(oracle_params(p), CO.bf16_round(x), act_round=CO.bf16_round)
    assert rel_l2(out, ref) <= 2e-3
    net.close()


def test_gradients_match_oracle(env):
    torch, dv = env
    g = np.random.default_rng(1)
    net = dv.Cnn(seed=5)
    p, _ = net.get_params()
    x, t = _batch(g, N=2, H=33, W=40)
    grad, loss = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    ps = oracle_params(p)
    out, inputs, pre = CO.forward(ps, CO.bf16_round(x), act_round=CO.bf16_round)
    ref_loss, dout = CO.mse_loss(out, t.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    grads = CO.backward(ps, inputs, pre, dout)
    off = 0
    for (dw, db), ci, co in zip(grads, CHANS[:-1], CHANS[1:]):
        gw = grad[off:off + 9 * ci * co].reshape(3, 3, ci, co)
        off += 9 * ci * co
        gb = grad[off:off + co]
        off += co
        assert rel_l2(gw, dw) <= 3e-3
        assert rel_l2(gb, db) <= 3e-3
    net.close()


def test_adam_step_matches_oracle(env):
    torch, dv = env
    g = np.random.default_rng(2)
    net = dv.Cnn(seed=7)
    p0, _ = net.get_params()
    x, t = _batch(g, N=1, H=20, W=24)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    grad, _ = net.gradients(xd, td)
    net.train_step(xd, td, 1e-3)
    p1, step = net.get_params()
    assert step == 1
    ref, _, _ = CO.adam_step(p0.astype(np.float64), grad.astype(np.float64), 0.0, 0.0, 1, 1e-3)
    np.testing.assert_allclose(p1, ref, rtol=0, atol=2e-7)
    net.close()


def test_train_crops_equals_single_steps(env):
    """dv_cnn_train_crops (crop gather and the step loop inside libdv, no host
    synchronisation) gives the same parameters and losses, bit for bit, as one
    dv_cnn_train_step per step on the same crops; bad crops are refused."""
    torch, dv = env
    g = np.random.default_rng(5)
    P, H, W, crop, batch, steps = 3, 40, 36, 16, 4, 6
    feats = torch.from_numpy(g.uniform(0, 1, (P, H, W, 5)).astype(np.float32)).cuda()
    targets = torch.from_numpy(g.uniform(-0.2, 0.2, (P, H, W)).astype(np.float32)).cuda()
    crops = np.stack([g.integers(0, P, (steps, batch)), g.integers(0, H - crop + 1, (steps, batch)),
                      g.integers(0, W - crop + 1, (steps, batch))], axis=-1).astype(np.int32)
    lrs = np.linspace(2e-3, 5e-4, steps).astype(np.float32)
    a, b = dv.Cnn(seed=3), dv.Cnn(seed=3)
    la = a.train_crops(feats, targets, crops, crop, lrs)
    lb = []
    for t in range(steps):
        xb = torch.stack([feats[p, r:r + crop, c:c + crop] for p, r, c in crops[t]]).contiguous()
        tb = torch.stack([targets[p, r:r + crop, c:c + crop] for p, r, c in crops[t]]).contiguous()
        lb.append(b.train_step(xb, tb, float(lrs[t])))
    pa, sa = a.get_params()
    pb, sb = b.get_params()
    assert sa == sb == steps
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(la, np.array(lb))
    bad = crops.copy()
    bad[2, 1, 1] = H - crop + 1
    with pytest.raises(dv.DVError):
        a.train_crops(feats, targets, bad, crop, lrs)
    assert a.get_params()[1] == steps     # refused before any step
    a.close()
    b.close()


def test_features_match_oracle(env):
    torch, dv = env
    g = np.random.default_rng(3)
    K, hy, wy = 9, 50, 61
    psfs = random_psfs(g, (3, 2), K)
    y = g.uniform(0, 1, (hy, wy)).astype(np.float32)
    plan = dv.Plan(hy, wy, psfs, noise_sigma=0.004)
    f = torch.empty(plan.nx + (5,), device="cuda")
    dv.dv_warmstart_features(plan.handle, torch.from_numpy(y).cuda(), f)
    ref = CO.warmstart_features(y, psfs.astype(np.float64), 0.004,
                                O.bilinear_weights(plan.nx[0], 3), O.bilinear_weights(plan.nx[1], 2))
    assert rel_l2(f.cpu().numpy(), ref) <= 1e-6
    plan.close()


def test_warm_start_is_used_by_the_solver(env):
    """With n_outer = 0 the solve returns its start image, which must be
    max(0, y_pad + net(features)); the strip-wise evaluation inside the solve
    (several strips here) must equal a whole-image forward pass."""
    torch, dv = env
    g = np.random.default_rng(4)
    K, hy, wy = 5, 300, 14000
    psfs = random_psfs(g, (2, 2), K)
    y = torch.from_numpy(g.uniform(0, 1, (hy, wy)).astype(np.float32)).cuda()
    net = dv.Cnn(seed=11)
    plan = dv.Plan(hy, wy, psfs, n_outer=0, n_inner=0, use_warmstart=1, noise_sigma=0.01)
    with pytest.raises(dv.DVError):
        plan.solve(y, stats=False)     # no network attached yet
    dv.dv_plan_set_warmstart(plan.handle, net)
    x0, _ = plan.solve(y, stats=False)
    f = torch.empty(plan.nx + (5,), device="cuda")
    dv.dv_warmstart_features(plan.handle, y, f)
    d = net.forward(f[None].contiguous())[0]
    ref = torch.clamp(f[..., 0] + d, min=0.0)
    torch.cuda.synchronize()
    assert torch.equal(x0, ref)
    plan.close()
    net.close()


def test_training_gains_over_the_plain_start(env):
    """Train on pairs made by the plain method and check, on held-out cases,
    that the warm start begins closer to the plain method's converged image and
    reaches a lower objective after the same few outer iterations."""
    torch, dv = env
    from paper_1705_06603_gb300 import warmstart as WS
    pairs = []
    for s in range(32):
        f, t, *_ = WS.make_pair(s, size=96, K=15, n_outer=40)
        pairs.append((f, t))
    net = dv.Cnn(seed=1)
    losses = WS.train(net, pairs, steps=1500, batch=16, crop=64, lr=1e-3)
    assert np.mean(losses[-50:]) < 0.2 * np.mean(losses[:50])
    for s in (100, 101):
        f, t, y, psfs, sigma = WS.make_pair(s, size=96, K=15, n_outer=40)
        xconv = (t + f[..., 0]).cpu().numpy()
        res = {}
        for warm in (0, 1):
            plan = dv.Plan(96, 96, psfs, n_tiles=(2, 2), overlap=16, n_outer=3, n_inner=10,
                           use_warmstart=warm, noise_sigma=sigma)
            dv.dv_plan_set_warmstart(plan.handle, net)
            x3, st = plan.solve(y)
            p0 = dv.Plan(96, 96, psfs, n_outer=0, n_inner=0, use_warmstart=warm,
                         noise_sigma=sigma)
            dv.dv_plan_set_warmstart(p0.handle, net)
            xs, _ = p0.solve(y, stats=False)
            res[warm] = (rel_l2(xs.cpu().numpy(), xconv), st["objective"])
            plan.close()
            p0.close()
        assert res[1][0] < 0.8 * res[0][0]    # start closer to the converged image
        assert res[1][1] < res[0][1]          # lower objective after 3 outer iterations
    net.close()
