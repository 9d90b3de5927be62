"""The chosen form of the solve against the FP64 oracle (Algorithm 1, Sec. III-B).

The chosen form runs the tensor-core operator (BF16 operands) or the exact
FP32 operator in the inner iterations, starts from the learned warm start,
takes 3 projected-gradient steps per outer iteration with gamma 0.2 and
rho 1.8, and stops as soon as its FP64 objective F(x_hat) (evaluated with
the FP32 operator) reaches F* (1 + 1e-4), where F* is the oracle's objective
of the plain form (blurred-image start, the workload's gamma and rho, 30 outer
x 10 inner iterations).  gamma, rho and the inner step count change the route
of Douglas-Rachford, not its fixed point, so x_hat is compared with the
oracle's plain-form x_hat.

Tolerances: the objective reached, F <= F* (1 + 1e-4) (the benchmark's
target: at or below the plain form's converged objective within 1e-4; the
warm-started solve may land below F*, the plain form's 30 x 10 iterate not
being the minimiser), and the oracle's objective of the GPU's x_hat within 1e-5
of the value the GPU reports (the stopping test is judged right).  The objective is flat near its minimiser (a
small lambda, PSF nulls), so two images within 1e-4 of F* can differ by a few
per cent: x_hat is held to the bound measured per case below, and the route
itself -- gamma 0.2, rho 1.8, 3 inner steps from the blurred start, a fixed
iteration count -- is compared with the oracle running the same route, to
1e-3 with the FP32 operator (the final-image bound) and to the measured bound
of the rounded operator with BF16 operands."""

import dataclasses

import numpy as np
import pytest

from oracle import dv_oracle as O
from tests.gpu_common import assert_close, need_gpu, rel_l2

pytestmark = pytest.mark.gpu

AUTO, TENSOR = 0, 3
FP32, BF16 = 0, 2


@pytest.fixture(scope="module")
def env():
    return need_gpu()


def _case(name):
    from paper_1705_06603_gb300.synth import (WORKLOADS, gaussian_noise, moffat_psf_grid,
                                              psf_grid_for, scene_for, star_field)
    if name == "disks128":
        w = WORKLOADS["disks128"]
        psfs = psf_grid_for(w).astype(np.float32)
        x = scene_for(w)
    else:
        # 256 x 256 star field, 4 x 4 grid of 9 x 9 Moffat PSFs, 2 x 2 tiles
        w = dataclasses.replace(WORKLOADS["stars2048"], name="stars256", hy=256, wy=256, K=9,
                                grid=(4, 4), n_tiles=(2, 2), overlap=32, n_outer=30,
                                n_inner=10, scene_seed=12, noise_seed=13)
        psfs = moffat_psf_grid(4, 4, 9).astype(np.float32)
        x = star_field(w.nx, w.scene_seed, dtype=np.float64)
    wr = O.bilinear_weights(w.nx[0], w.grid[0])
    wc = O.bilinear_weights(w.nx[1], w.grid[1])
    y = O.apply_H(x, psfs.astype(np.float64), wr, wc)
    y = (y + gaussian_noise(y.shape, w.noise_sigma, w.noise_seed)).astype(np.float32)
    return w, psfs, y


def _network(dv, w, psfs):
    """A warm-start network trained on plain-method pairs of other seeded scenes
    with the case's PSF grid."""
    from paper_1705_06603_gb300 import warmstart as WS
    pairs = []
    for s in range(6):
        f, t, *_ = WS.make_pair(70_000 + s, size=128, K=w.K, grid=w.grid, n_tiles=(2, 2),
                                overlap=16, n_outer=w.n_outer, n_inner=w.n_inner, lam=w.lam,
                                delta=w.delta, gamma=w.gamma, psfs=psfs, sigma=w.noise_sigma)
        pairs.append((f, t))
    net = dv.Cnn(seed=3)
    WS.train(net, pairs, steps=3000, batch=16, crop=64, lr=1e-3, seed=3, schedule="cosine")
    return net


# relative RMSE of x_hat against the oracle's plain-form x_hat, per (workload,
# operator precision): the spread of images within 1e-4 of F*
# (measured on a GB300: 2.60e-2 / 4.15e-2 with either operator)
XTOL = {("disks128", FP32): 0.05, ("stars256", FP32): 0.08,
        ("disks128", BF16): 0.05, ("stars256", BF16): 0.08}
# the chosen route at a fixed iteration count against the oracle's same route
# (measured: 2.5e-7 / 2.2e-7 FP32, 3.7e-4 / 1.1e-3 BF16)
RTOL = {FP32: 1e-3, BF16: 3e-3}


@pytest.mark.parametrize("name", ["disks128", "stars256"])
@pytest.mark.parametrize("path,prec", [(AUTO, FP32), (TENSOR, BF16)])
def test_chosen_form_reaches_the_oracle_plain_form(env, name, path, prec):
    torch, dv = env
    w, psfs, y = _case(name)
    lay = O.make_layout(w.hy, w.wy, w.K, *w.n_tiles, w.overlap)
    ps64, y64 = psfs.astype(np.float64), y.astype(np.float64)
    xr, _ = O.solve(y64, ps64, lay, w.lam, w.delta, w.gamma, w.rho, w.n_outer, w.n_inner)
    f_star = O.objective(xr, y64, ps64, lay, w.lam, w.delta)[0]
    target = f_star * (1.0 + 1e-4)

    net = _network(dv, w, psfs)
    plan = dv.Plan(w.hy, w.wy, psfs, n_tiles=w.n_tiles, overlap=w.overlap, lam=w.lam,
                   delta=w.delta, gamma=0.2, rho=1.8, n_outer=4 * w.n_outer, n_inner=3,
                   precision=prec, path=path, use_warmstart=1, check_every=1,
                   target_objective=target, noise_sigma=w.noise_sigma)
    if path == TENSOR:
        assert plan.info.path == TENSOR
    dv.dv_plan_set_warmstart(plan.handle, net)
    xd, st = plan.solve(torch.from_numpy(y).cuda())
    torch.cuda.synchronize()
    xd = xd.cpu().numpy()
    plan.close()
    net.close()

    # the stop: reached within the run, judged on an objective the oracle agrees with
    assert st["outer_done"] < 4 * w.n_outer
    assert st["objective"] <= target
    F_gpu = O.objective(xd.astype(np.float64), y64, ps64, lay, w.lam, w.delta)[0]
    assert abs(F_gpu - st["objective"]) <= 1e-5 * F_gpu
    assert F_gpu <= target * (1.0 + 1e-5)
    # the image
    err = rel_l2(xd, xr)
    print(f"{name} prec {prec}: {st['outer_done']} outer x 3 inner, F {F_gpu:.8g} vs F* "
          f"{f_star:.8g} ({(F_gpu - f_star) / f_star:+.2e}), x_hat rel RMSE {err:.3e}")
    assert_close(xd, xr, XTOL[(name, prec)])
    assert xd.min() >= 0.0


@pytest.mark.parametrize("name", ["disks128", "stars256"])
@pytest.mark.parametrize("path,prec", [(AUTO, FP32), (TENSOR, BF16)])
def test_chosen_route_matches_the_oracle(env, name, path, prec):
    """gamma 0.2, rho 1.8, 3 projected-gradient steps per outer iteration,
    blurred-image start, 30 outer iterations: the GPU against the oracle on the
    same route (no warm start: its network is a GPU product)."""
    torch, dv = env
    w, psfs, y = _case(name)
    lay = O.make_layout(w.hy, w.wy, w.K, *w.n_tiles, w.overlap)
    ps64, y64 = psfs.astype(np.float64), y.astype(np.float64)
    n_outer = 30
    xr, info = O.solve(y64, ps64, lay, w.lam, w.delta, 0.2, 1.8, n_outer, 3)
    plan = dv.Plan(w.hy, w.wy, psfs, n_tiles=w.n_tiles, overlap=w.overlap, lam=w.lam,
                   delta=w.delta, gamma=0.2, rho=1.8, n_outer=n_outer, n_inner=3,
                   precision=prec, path=path)
    xd, st = plan.solve(torch.from_numpy(y).cuda())
    torch.cuda.synchronize()
    xd = xd.cpu().numpy()
    plan.close()
    F = O.objective(xr, y64, ps64, lay, w.lam, w.delta)[0]
    err = rel_l2(xd, xr)
    print(f"{name} prec {prec}: route x_hat rel RMSE {err:.3e}, objective {st['objective']:.8g} "
          f"vs {F:.8g}")
    assert_close(xd, xr, RTOL[prec])
    assert abs(st["objective"] - F) <= (1e-5 if prec == FP32 else 1e-3) * F
