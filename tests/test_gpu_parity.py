"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances (FP32 arithmetic against FP64): operator relative L2 <= 1e-5;
short solves relative L2 <= 1e-4; the full 30 x 10 solve relative RMSE <= 1e-3
and objective within 1e-4 relative (the precision targets of the method's
FP32 form)."""

import numpy as np
import pytest

from oracle import dv_oracle as O
from tests.gpu_common import (assert_close, need_gpu, oracle_solve, random_psfs, rel_l2,
                              workload_case)

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    return need_gpu()


def _apply_both(env, hy, wy, K, G, seed, negative=False, weights=None, path=1):
    torch, dv = env
    g = np.random.default_rng(seed)
    psfs = random_psfs(g, G, K, negative)
    nxr, nxc = hy + K - 1, wy + K - 1
    x = g.uniform(0, 1, (nxr, nxc)).astype(np.float32)
    r = g.standard_normal((hy, wy)).astype(np.float32)
    plan = dv.Plan(hy, wy, psfs, weights=weights, path=path)
    assert plan.info.path == path
    yd = plan.apply_H(torch.from_numpy(x).cuda())
    gd = plan.apply_Ht(torch.from_numpy(r).cuda())
    torch.cuda.synchronize()
    wr, wc = weights if weights is not None else (O.bilinear_weights(nxr, G[0]),
                                                  O.bilinear_weights(nxc, G[1]))
    wr, wc = np.asarray(wr, np.float64), np.asarray(wc, np.float64)
    ps = psfs.astype(np.float64)
    y_ref = O.apply_H(x.astype(np.float64), ps, wr, wc)
    g_ref = O.apply_Ht(r.astype(np.float64), ps, wr, wc)
    plan.close()
    return yd.cpu().numpy(), y_ref, gd.cpu().numpy(), g_ref, x, r


DIRECT, FFT = 1, 2


@pytest.mark.parametrize("path", [DIRECT, FFT])
@pytest.mark.parametrize("hy,wy,K,G", [
    (150, 133, 3, (3, 4)),     # several blocks, ragged tails
    (130, 70, 9, (3, 3)),
    (97, 140, 11, (2, 5)),     # run-time K kernel (direct)
    (200, 180, 31, (4, 3)),
    (250, 301, 31, (5, 6)),    # several 98x98 FFT blocks, straddling PSF cells
    (70, 75, 63, (2, 2)),
    (40, 33, 1, (2, 2)),       # 1x1 PSFs: H is pointwise, x and y share a size
    (66, 64, 5, (1, 1)),       # a single PSF: plain convolution
])
def test_operator_matches_oracle(env, hy, wy, K, G, path):
    yd, y_ref, gd, g_ref, x, r = _apply_both(env, hy, wy, K, G, seed=K * 7 + hy, path=path)
    assert_close(yd, y_ref, OP_TOL)
    assert_close(gd, g_ref, OP_TOL)


@pytest.mark.parametrize("path", [DIRECT, FFT])
def test_operator_signed_psfs_and_separable_weights(env, path):
    hy, wy, K, G = 90, 101, 7, (3, 3)
    g = np.random.default_rng(5)
    nxr, nxc = hy + K - 1, wy + K - 1
    # a non-tent first-order profile (still two neighbouring points at most)
    t = np.linspace(0, 1, nxr)
    wr = np.stack([np.clip(1 - 2 * t, 0, 1), 1 - np.abs(2 * t - 1), np.clip(2 * t - 1, 0, 1)])
    wc = O.bilinear_weights(nxc, 3) * 0.8
    yd, y_ref, gd, g_ref, *_ = _apply_both(env, hy, wy, K, G, 5, negative=True,
                                           weights=(wr.astype(np.float32), wc.astype(np.float32)),
                                           path=path)
    assert_close(yd, y_ref, OP_TOL)
    assert_close(gd, g_ref, OP_TOL)


@pytest.mark.parametrize("path", [DIRECT, FFT])
def test_adjoint_identity_on_gpu(env, path):
    yd, _, gd, _, x, r = _apply_both(env, 123, 77, 9, (3, 2), seed=99, path=path)
    lhs = np.vdot(yd.astype(np.float64), r.astype(np.float64))
    rhs = np.vdot(x.astype(np.float64), gd.astype(np.float64))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(yd) * np.linalg.norm(r)


def _gpu_solve(env, w, psfs, y, n_outer, n_inner, use_graphs=1, x0=None, **kw):
    torch, dv = env
    plan = dv.Plan(w.hy, w.wy, psfs, n_tiles=w.n_tiles, overlap=w.overlap,
                   tile_bounds=(w.yrows, w.ycols) if w.yrows is not None else None,
                   lam=w.lam, delta=w.delta, gamma=w.gamma, rho=w.rho, n_outer=n_outer,
                   n_inner=n_inner, use_graphs=use_graphs, **kw)
    xd, st = plan.solve(torch.from_numpy(y).cuda(),
                        None if x0 is None else torch.from_numpy(x0).cuda())
    torch.cuda.synchronize()
    return plan, xd.cpu().numpy(), st


@pytest.mark.parametrize("path", [DIRECT, FFT])
def test_short_solve_matches_oracle(env, path):
    w, psfs, y, _ = workload_case("disks128")
    plan, xd, st = _gpu_solve(env, w, psfs, y, 3, 2, path=path)
    lay, xr, info = oracle_solve(w, psfs, y, 3, 2)
    assert_close(xd, xr, 1e-5)
    F, data, prior = O.objective(xr, y.astype(np.float64), psfs.astype(np.float64), lay, w.lam,
                                 w.delta)
    assert abs(st["objective"] - F) <= 1e-5 * F
    assert abs(st["data_term"] - data) <= 1e-5 * data
    assert abs(st["prior_term"] - prior) <= 1e-5 * prior
    assert abs(st["primal_res"] - info.primal[-1]) <= 1e-3 * info.primal[-1]
    assert abs(st["dual_res"] - info.dual[-1]) <= 1e-3 * info.dual[-1]
    assert st["outer_done"] == 3 and st["inner_done"] == 6
    plan.close()


@pytest.mark.parametrize("path", [DIRECT, FFT])
def test_full_small_workload_matches_oracle(env, path):
    """The 128x128 workload, 30 consensus iterations x 10 inner steps."""
    w, psfs, y, _ = workload_case("disks128")
    plan, xd, st = _gpu_solve(env, w, psfs, y, w.n_outer, w.n_inner, path=path)
    lay, xr, info = oracle_solve(w, psfs, y, w.n_outer, w.n_inner)
    assert_close(xd, xr, 1e-3)
    F = O.objective(xr, y.astype(np.float64), psfs.astype(np.float64), lay, w.lam, w.delta)[0]
    assert abs(st["objective"] - F) <= 1e-4 * F
    assert xd.min() >= 0.0
    plan.close()


def test_graph_eager_host_and_repeat_are_bit_identical(env):
    torch, dv = env
    w, psfs, y, _ = workload_case("disks128")
    p1, x1, s1 = _gpu_solve(env, w, psfs, y, 4, 3, use_graphs=1)
    p2, x2, s2 = _gpu_solve(env, w, psfs, y, 4, 3, use_graphs=0)
    xh, sh = p1.solve_host(y)
    x3 = p1.solve(torch.from_numpy(y).cuda())[0].cpu().numpy()
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(x1, xh)
    np.testing.assert_array_equal(x1, x3)
    assert s1["objective"] == s2["objective"] == sh["objective"]
    p1.close()
    p2.close()


def test_checkpoint_resume_equals_uninterrupted(env):
    torch, dv = env
    w, psfs, y, _ = workload_case("disks128")
    plan, x_full, _ = _gpu_solve(env, w, psfs, y, 6, 4, inner_increment=2)
    p2, _, _ = _gpu_solve(env, w, psfs, y, 3, 4, inner_increment=2)
    n = p2.info.stack_elems
    xs = torch.empty(n, device="cuda")
    us = torch.empty(n, device="cuda")
    k = dv.dv_state_export(p2.handle, xs, us)
    assert k == 3
    p3 = dv.Plan(w.hy, w.wy, psfs, n_tiles=w.n_tiles, overlap=w.overlap, lam=w.lam,
                 delta=w.delta, gamma=w.gamma, n_outer=6, n_inner=4, inner_increment=2)
    dv.dv_state_import(p3.handle, xs, us, k)
    out = torch.empty(p3.nx, device="cuda")
    st = dv.dv_stats()
    dv.dv_consensus_continue(p3.handle, torch.from_numpy(y).cuda(), 3, out, st)
    np.testing.assert_array_equal(out.cpu().numpy(), x_full)
    assert st.outer_done == 6
    for p in (plan, p2, p3):
        p.close()


@pytest.mark.parametrize("case", ["one_tile", "no_inner", "no_outer", "uneven_tiles",
                                  "noise_weights", "no_prior", "paper_schedule", "independent"])
def test_edge_cases_match_oracle(env, case):
    torch, dv = env
    g = np.random.default_rng(17)
    K, G = 5, (2, 3)
    hy, wy = 70, 83
    psfs = random_psfs(g, G, K)
    nxr, nxc = hy + K - 1, wy + K - 1
    x = g.uniform(0, 1, (nxr, nxc))
    wr, wc = O.bilinear_weights(nxr, G[0]), O.bilinear_weights(nxc, G[1])
    y = (O.apply_H(x, psfs.astype(np.float64), wr, wc) +
         0.01 * g.standard_normal((hy, wy))).astype(np.float32)
    kw = dict(n_tiles=(2, 3), overlap=8, lam=0.01, delta=0.05, gamma=0.4, n_outer=4, n_inner=3)
    okw = {}
    W = None
    bounds = None
    if case == "one_tile":
        kw["n_tiles"] = (1, 1)
    elif case == "no_inner":
        kw["n_inner"] = 0
    elif case == "no_outer":
        kw["n_outer"] = 0
    elif case == "uneven_tiles":
        bounds = ([(0, 30), (22, 70)], [(0, 20), (12, 60), (50, 83)])
        kw["tile_bounds"] = bounds
    elif case == "noise_weights":
        W = g.uniform(0.2, 1.0, (hy, wy)).astype(np.float32)
        W[10:14, 20:30] = 0.0      # unmeasured pixels
        kw["noise_w"] = W
    elif case == "no_prior":
        kw["lam"] = 0.0
    elif case == "paper_schedule":
        kw["inner_increment"] = 2
        okw["inner_increment"] = 2
    elif case == "independent":
        # Sec. IV's "independent" method: tiles solved alone, then blended
        kw.update(gamma=1e-9, n_outer=1, n_inner=40)
    plan = dv.Plan(hy, wy, psfs, **kw)
    xd, st = plan.solve(torch.from_numpy(y).cuda())
    xd = xd.cpu().numpy()
    lay = O.make_layout(hy, wy, K, *kw["n_tiles"], kw["overlap"],
                        bounds[0] if bounds else None, bounds[1] if bounds else None)
    xr, info = O.solve(y.astype(np.float64), psfs.astype(np.float64), lay, kw["lam"], kw["delta"],
                       kw["gamma"], 1.0, kw["n_outer"], kw["n_inner"],
                       W=None if W is None else W.astype(np.float64), **okw)
    assert_close(xd, xr, 1e-5)
    F = O.objective(xr, y.astype(np.float64), psfs.astype(np.float64), lay, kw["lam"],
                    kw["delta"], None if W is None else W.astype(np.float64))[0]
    assert abs(st["objective"] - F) <= 1e-5 * F
    plan.close()


@pytest.mark.parametrize("path,prec", [(DIRECT, 0), (FFT, 0), (3, 2), (3, 1)])
def test_full_size_tile_step_matches_oracle(env, path, prec):
    """The 2048x2048 star-field workload in the benchmark's launch configuration:
    one inner step and one consensus step on all 16 tiles; an interior tile's
    x_i is compared element by element with the oracle's Local-Solver step
    (FP32 paths to 1e-5; the tensor path within its operator tolerance)."""
    torch, dv = env
    from paper_1705_06603_gb300.synth import WORKLOADS, psf_grid_for, scene_for, gaussian_noise
    w = WORKLOADS["stars2048"]
    psfs = psf_grid_for(w).astype(np.float32)
    rng = np.random.default_rng(3)
    y = (scene_for(w)[15:-15, 15:-15] * 0.9 +
         gaussian_noise((w.hy, w.wy), w.noise_sigma, w.noise_seed)).astype(np.float32)
    plan = dv.Plan(w.hy, w.wy, psfs, n_tiles=w.n_tiles, overlap=w.overlap, lam=w.lam,
                   delta=w.delta, gamma=w.gamma, n_outer=1, n_inner=1, path=path,
                   precision=prec)
    assert plan.info.path == path
    plan.solve(torch.from_numpy(y).cuda(), stats=False)
    xs = torch.empty(plan.info.stack_elems, device="cuda")
    us = torch.empty_like(xs)
    dv.dv_state_export(plan.handle, xs, us)
    xs = xs.cpu().numpy()
    lay = O.make_layout(w.hy, w.wy, w.K, *w.n_tiles, w.overlap)
    tr, tc = 1, 2
    n = tr * w.n_tiles[1] + tc
    # stack layout: tiles in row-major order, rows padded to 32 floats
    off = 0
    for t, (a, b) in enumerate(lay.tiles):
        rs, cs = lay.xslice(a, b)
        nr, nc = rs.stop - rs.start, cs.stop - cs.start
        pitch = -(-nc // 32) * 32
        if t == n:
            x_gpu = xs[off:off + nr * pitch].reshape(nr, pitch)[:, :nc]
            break
        off += -(-(nr * pitch) // 32) * 32
    x0 = O.start_image(y.astype(np.float64), w.K)
    rs, cs = lay.xslice(tr, tc)
    wr = O.bilinear_weights(lay.nx[0], w.grid[0])[:, rs]
    wc = O.bilinear_weights(lay.nx[1], w.grid[1])[:, cs]
    tau = O.tile_step(lay, tr, tc, psfs.astype(np.float64), None, w.lam, w.gamma)
    xi = O.local_solve(x0[rs, cs], x0[rs, cs], y.astype(np.float64)[lay.yslice(tr, tc)], None,
                       psfs.astype(np.float64), wr, wc, w.gamma * lay.omega(tr, tc), w.lam,
                       w.delta, tau, 1)
    assert_close(x_gpu, xi, {0: 1e-5, 2: 3e-3, 1: 5e-4}[prec])
    plan.close()


@pytest.mark.parametrize("use_graphs", [1, 0])
def test_kernel_timing_counts(env, use_graphs):
    """Per-kernel event timing sees every launch of the solve, in graphs and eagerly,
    and does not change the result."""
    torch, dv = env
    w, psfs, y, _ = workload_case("disks128")
    plan, x_ref, _ = _gpu_solve(env, w, psfs, y, 3, 4, use_graphs=use_graphs)
    dv.dv_plan_set_timing(plan.handle, 1)
    xd, _ = plan.solve(torch.from_numpy(y).cuda(), stats=False)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(xd.cpu().numpy(), x_ref)
    for kind, n in ((0, 12), (1, 12), (2, 3)):
        ms, cnt = dv.dv_plan_kernel_time(plan.handle, kind)
        assert cnt == n and ms > 0.0
    dv.dv_plan_set_timing(plan.handle, 0)
    plan.close()


def test_autotuner_times_both_paths_and_keeps_the_faster(env):
    torch, dv = env
    w, psfs, y, _ = workload_case("disks128")
    plan = dv.Plan(w.hy, w.wy, psfs, n_tiles=w.n_tiles, overlap=w.overlap, path=0)
    i = plan.info
    assert i.tune_ms_direct > 0 and i.tune_ms_fft > 0
    assert i.path == (FFT if i.tune_ms_fft < i.tune_ms_direct else DIRECT)
    plan.close()
    # a PSF too large for 128-point blocks keeps the direct path
    g = np.random.default_rng(0)
    big = random_psfs(g, (1, 1), 101)
    plan = dv.Plan(40, 40, big, path=0)
    assert plan.info.path == DIRECT and plan.info.tune_ms_fft == 0
    with pytest.raises(dv.DVError):
        dv.Plan(40, 40, big, path=FFT)
    plan.close()


TENSOR = 3
BF16, TF32 = 2, 1
# operator relative L2 with BF16 / TF32 operands and FP32 accumulation
TC_TOL = {BF16: 3e-3, TF32: 5e-4}


@pytest.mark.parametrize("prec", [BF16, TF32])
@pytest.mark.parametrize("hy,wy,K,G", [(130, 70, 9, (3, 3)), (200, 180, 31, (4, 3)),
                                       (150, 97, 63, (2, 2)), (66, 64, 15, (1, 1)),
                                       (300, 260, 15, (8, 8))])
def test_tensor_operator_matches_oracle(env, prec, hy, wy, K, G):
    """The tcgen05 operator on the global image: ragged 128 x 64 blocks, up to
    4 x 4 PSFs per block (8 x 8 grid), every supported K."""
    torch, dv = env
    g = np.random.default_rng(K + 1000)
    psfs = random_psfs(g, G, K)
    nxr, nxc = hy + K - 1, wy + K - 1
    x = g.uniform(0, 1, (nxr, nxc)).astype(np.float32)
    r = g.standard_normal((hy, wy)).astype(np.float32)
    plan = dv.Plan(hy, wy, psfs, precision=prec, path=TENSOR, tensor_h=1 if prec == BF16 else 0)
    assert plan.info.path == TENSOR and plan.info.block_side in (128, 256)
    assert plan.info.tensor_h_dft == 0
    yd = plan.apply_H(torch.from_numpy(x).cuda()).cpu().numpy()
    gd = plan.apply_Ht(torch.from_numpy(r).cuda()).cpu().numpy()
    wr, wc = O.bilinear_weights(nxr, G[0]), O.bilinear_weights(nxc, G[1])
    ps = psfs.astype(np.float64)
    assert_close(yd, O.apply_H(x.astype(np.float64), ps, wr, wc), TC_TOL[prec])
    assert_close(gd, O.apply_Ht(r.astype(np.float64), ps, wr, wc), TC_TOL[prec])
    plan.close()


@pytest.mark.parametrize("hy,wy,K,G", [(130, 70, 9, (3, 3)), (200, 180, 31, (4, 3)),
                                       (150, 97, 63, (2, 2)), (66, 64, 15, (1, 1)),
                                       (300, 260, 15, (8, 8)), (250, 301, 31, (5, 6)),
                                       (331, 203, 63, (4, 3))])
def test_block_dft_H_matches_oracle(env, hy, wy, K, G):
    """H as the block DFT on the tensor cores (FP16 operands, FP32 accumulation):
    several 128 x 128 overlap-save blocks with ragged edges, blocks straddling
    PSF cells (up to 3 x 3 PSFs per block on the 8 x 8 grid), every K of the
    tensor path, at the BF16 operator tolerance; H^T stays the banded form."""
    torch, dv = env
    g = np.random.default_rng(K + 2000)
    psfs = random_psfs(g, G, K)
    nxr, nxc = hy + K - 1, wy + K - 1
    x = g.uniform(0, 1, (nxr, nxc)).astype(np.float32)
    plan = dv.Plan(hy, wy, psfs, precision=BF16, path=TENSOR, tensor_h=2)
    assert plan.info.path == TENSOR and plan.info.tensor_h_dft == 1
    yd = plan.apply_H(torch.from_numpy(x).cuda()).cpu().numpy()
    wr, wc = O.bilinear_weights(nxr, G[0]), O.bilinear_weights(nxc, G[1])
    y_ref = O.apply_H(x.astype(np.float64), psfs.astype(np.float64), wr, wc)
    print(f"K {K} G {G}: rel L2 {rel_l2(yd, y_ref):.3e}")
    assert_close(yd, y_ref, TC_TOL[BF16])
    plan.close()


@pytest.mark.parametrize("hy,wy,K,G", [(130, 70, 9, (3, 3)), (200, 180, 31, (4, 3)),
                                       (150, 97, 63, (2, 2)), (66, 64, 15, (1, 1)),
                                       (300, 260, 15, (8, 8)), (250, 301, 31, (5, 6)),
                                       (331, 203, 63, (4, 3))])
def test_block_dft_Ht_matches_oracle(env, hy, wy, K, G):
    """H^T as the block DFT (tensor_h = 3): the correlation with each PSF on
    128 x 128 blocks of the residual reaching K - 1 above and left of the output
    block (zero outside the image), ragged edges, up to 3 x 3 PSFs per block,
    at the BF16 operator tolerance; H is the block DFT too."""
    torch, dv = env
    g = np.random.default_rng(K + 3000)
    psfs = random_psfs(g, G, K)
    nxr, nxc = hy + K - 1, wy + K - 1
    r = g.standard_normal((hy, wy)).astype(np.float32)
    x = g.uniform(0, 1, (nxr, nxc)).astype(np.float32)
    plan = dv.Plan(hy, wy, psfs, precision=BF16, path=TENSOR, tensor_h=3)
    assert plan.info.path == TENSOR and plan.info.tensor_h_dft == 1 and plan.info.tensor_ht_dft == 1
    gd = plan.apply_Ht(torch.from_numpy(r).cuda()).cpu().numpy()
    yd = plan.apply_H(torch.from_numpy(x).cuda()).cpu().numpy()
    wr, wc = O.bilinear_weights(nxr, G[0]), O.bilinear_weights(nxc, G[1])
    ps = psfs.astype(np.float64)
    g_ref = O.apply_Ht(r.astype(np.float64), ps, wr, wc)
    print(f"K {K} G {G}: H^T rel L2 {rel_l2(gd, g_ref):.3e}")
    assert_close(gd, g_ref, TC_TOL[BF16])
    assert_close(yd, O.apply_H(x.astype(np.float64), ps, wr, wc), TC_TOL[BF16])
    plan.close()


@pytest.mark.parametrize("mag", [1e-4, 3e3, 1e6])
def test_block_dft_scales_each_block(env, mag):
    """Inputs far from unit magnitude: each 128 x 128 block is scaled by a
    power of two into FP16 range before the transforms, so H x and H^T r keep
    the BF16 operator tolerance where unscaled FP16 operands would overflow
    (1e6) or lose their low bits (1e-4)."""
    torch, dv = env
    hy, wy, K, G = 200, 180, 31, (4, 3)
    g = np.random.default_rng(77)
    psfs = random_psfs(g, G, K)
    nxr, nxc = hy + K - 1, wy + K - 1
    x = (mag * g.uniform(0, 1, (nxr, nxc))).astype(np.float32)
    r = (mag * g.standard_normal((hy, wy))).astype(np.float32)
    plan = dv.Plan(hy, wy, psfs, precision=BF16, path=TENSOR, tensor_h=3)
    yd = plan.apply_H(torch.from_numpy(x).cuda()).cpu().numpy()
    gd = plan.apply_Ht(torch.from_numpy(r).cuda()).cpu().numpy()
    wr, wc = O.bilinear_weights(nxr, G[0]), O.bilinear_weights(nxc, G[1])
    ps = psfs.astype(np.float64)
    assert np.isfinite(yd).all() and np.isfinite(gd).all()
    assert_close(yd, O.apply_H(x.astype(np.float64), ps, wr, wc), TC_TOL[BF16])
    assert_close(gd, O.apply_Ht(r.astype(np.float64), ps, wr, wc), TC_TOL[BF16])
    plan.close()


def test_block_dft_both_solve_matches_oracle(env):
    """The 128x128 workload at the plain iteration count with H and H^T as
    block DFTs in the inner iterations (residual epilogue of H, projected
    gradient step fused into H^T, tile groups in the captured graphs): within
    the final-image bound 1e-3 of the oracle."""
    w, psfs, y, _ = workload_case("disks128")
    plan, xd, st = _gpu_solve(env, w, psfs, y, w.n_outer, w.n_inner, precision=BF16,
                              path=TENSOR, tensor_h=3)
    assert plan.info.tensor_h_dft == 1 and plan.info.tensor_ht_dft == 1
    lay, xr, info = oracle_solve(w, psfs, y, w.n_outer, w.n_inner)
    print(f"block-DFT H and H^T solve: x_hat rel L2 {rel_l2(xd, xr):.3e}")
    assert_close(xd, xr, 1e-3)
    F = O.objective(xr, y.astype(np.float64), psfs.astype(np.float64), lay, w.lam, w.delta)[0]
    assert abs(st["objective"] - F) <= 1e-3 * F
    plan.close()


def test_block_dft_solve_matches_oracle(env):
    """The 128x128 workload at the plain iteration count with H as the block
    DFT in the inner iterations (residual epilogue, tile groups in the
    captured graphs): within the final-image bound 1e-3 of the oracle."""
    w, psfs, y, _ = workload_case("disks128")
    plan, xd, st = _gpu_solve(env, w, psfs, y, w.n_outer, w.n_inner, precision=BF16,
                              path=TENSOR, tensor_h=2)
    assert plan.info.tensor_h_dft == 1
    lay, xr, info = oracle_solve(w, psfs, y, w.n_outer, w.n_inner)
    print(f"block-DFT solve: x_hat rel L2 {rel_l2(xd, xr):.3e}")
    assert_close(xd, xr, 1e-3)
    F = O.objective(xr, y.astype(np.float64), psfs.astype(np.float64), lay, w.lam, w.delta)[0]
    assert abs(st["objective"] - F) <= 1e-3 * F
    plan.close()


@pytest.mark.parametrize("prec", [BF16, TF32])
def test_tensor_solve_close_to_oracle(env, prec):
    """The 128x128 workload at the plain iteration count (30 x 10) with the
    tensor-core operator in the inner iterations: the objective is evaluated
    with the FP32 operator; the image is held to the final-image bound 1e-3 of
    the FP64 oracle (measured on a GB300: 4.1e-4 BF16, 8.2e-5 TF32) -- the
    iterates converge to the fixed point of the rounded operator, whose
    distance from the exact one the operator's rounding sets."""
    w, psfs, y, _ = workload_case("disks128")
    plan, xd, st = _gpu_solve(env, w, psfs, y, w.n_outer, w.n_inner, precision=prec, path=TENSOR)
    assert plan.info.path == TENSOR and plan.info.fp32_path in (DIRECT, FFT)
    lay, xr, info = oracle_solve(w, psfs, y, w.n_outer, w.n_inner)
    tol = 1e-3
    print(f"prec {prec}: x_hat rel L2 {rel_l2(xd, xr):.3e}")
    assert_close(xd, xr, tol)
    F = O.objective(xr, y.astype(np.float64), psfs.astype(np.float64), lay, w.lam, w.delta)[0]
    assert abs(st["objective"] - F) <= tol * F
    plan.close()


@pytest.mark.parametrize("path,prec,tol", [(DIRECT, 0, 1e-5), (FFT, 0, 1e-5), (TENSOR, BF16, 1e-2),
                                           (TENSOR, TF32, 2e-3)])
def test_paper_mode_solve_matches_oracle(env, path, prec, tol):
    """One PSF per block, the paper's own layout (reading R18): the 3 x 3 PSF
    grid of the 128^2 workload gives 3 x 3 blocks that overlap by half, each
    blurred by its own PSF; the increasing inner schedule 3 + 2k of Sec. IV-B.
    The GPU solve and its objective match the oracle on every operator path,
    and dv_apply_H keeps the interpolated model."""
    torch, dv = env
    w, psfs, y, _ = workload_case("disks128")
    G = psfs.shape[:2]
    plan = dv.Plan(w.hy, w.wy, psfs, n_tiles=G, weights="per_tile", lam=w.lam, delta=w.delta,
                   gamma=w.gamma, rho=w.rho, n_outer=4, n_inner=3, inner_increment=2, path=path,
                   precision=prec)
    assert plan.info.path == path
    xd, st = plan.solve(torch.from_numpy(y).cuda())
    torch.cuda.synchronize()
    lay = O.paper_layout(w.hy, w.wy, w.K, *G)
    ps, y64 = psfs.astype(np.float64), y.astype(np.float64)
    xr, info = O.solve(y64, ps, lay, w.lam, w.delta, w.gamma, w.rho, 4, 3, inner_increment=2,
                       weights="per_tile")
    assert_close(xd.cpu().numpy(), xr, tol)
    F = O.objective(xr, y64, ps, lay, w.lam, w.delta, weights="per_tile")[0]
    assert abs(st["objective"] - F) <= tol * F
    assert st["inner_done"] == 3 + 5 + 7 + 9
    g = np.random.default_rng(9)
    x = g.uniform(0, 1, plan.nx).astype(np.float32)
    hx = plan.apply_H(torch.from_numpy(x).cuda()).cpu().numpy()
    wr, wc = O.bilinear_weights(plan.nx[0], G[0]), O.bilinear_weights(plan.nx[1], G[1])
    assert_close(hx, O.apply_H(x.astype(np.float64), ps, wr, wc), max(tol, 1e-5))
    plan.close()


@pytest.mark.parametrize("shape,kind", [((11, 11), "uniform"), ((100, 77), "uniform"),
                                        ((531, 1040), "uniform"), ((300, 257), "stars")])
def test_image_quality_matches_oracle(env, shape, kind):
    """dv_image_quality (SNR over all pixels, mean SSIM over the 11 x 11
    windows, reading R19) against the FP64 oracle, on noise and on a blurred
    star field with a small perturbation."""
    torch, dv = env
    g = np.random.default_rng(shape[0])
    if kind == "uniform":
        ref = g.uniform(0, 1, shape).astype(np.float32)
        x = np.clip(ref + g.normal(0, 0.1, shape), 0, 1).astype(np.float32)
    else:
        from paper_1705_06603_gb300.synth import star_field
        ref = star_field(shape, 5).astype(np.float32)
        x = (ref + g.normal(0, 0.003, shape)).astype(np.float32)
    snr, ssim = dv.image_quality(torch.from_numpy(x).cuda(), torch.from_numpy(ref).cuda())
    x64, r64 = x.astype(np.float64), ref.astype(np.float64)
    assert snr == pytest.approx(O.snr_db(x64, r64), rel=1e-9)
    assert abs(ssim - O.ssim(x64, r64)) <= 2e-5
    s2, q2 = dv.image_quality(torch.from_numpy(ref).cuda(), torch.from_numpy(ref).cuda())
    assert s2 == float("inf") and abs(q2 - 1.0) <= 1e-5


@pytest.mark.parametrize("path", [DIRECT, FFT])
def test_vmlmb_solve_matches_oracle(env, path):
    """VMLM-B Local-Solver (reading R20: the paper's solver) through the C ABI:
    3 outer iterations of 4 VMLM-B iterations with 3 memory pairs on the 128^2
    workload, against the FP64 oracle running the same steps."""
    w, psfs, y, _ = workload_case("disks128")
    plan, xd, st = _gpu_solve(env, w, psfs, y, 3, 4, path=path, local_solver=1, vm_memory=3)
    assert st["inner_done"] == 12
    lay, xr, info = oracle_solve(w, psfs, y, 3, 4, local_solver="vmlmb", vm_memory=3,
                                 vm_stop_rel=1e-7)
    assert_close(xd, xr, 1e-4)
    F = O.objective(xr, y.astype(np.float64), psfs.astype(np.float64), lay, w.lam, w.delta)[0]
    assert abs(st["objective"] - F) <= 1e-5 * F
    assert 1.0 <= st["vm_tile_trials"] <= st["vm_trials_per_iter"] <= st["vm_trials_max"] <= 20
    plan.close()


def test_vmlmb_line_search_trials_stay_near_the_oracles(env):
    """The paper's schedule with VMLM-B (25 % of it: 6 outer iterations of
    10 + 10k iterations, one PSF per block) on the 128^2 workload: with the
    stop at the objective's resolution (reading R21, vm_stop_rel = 1e-7 on both
    sides) the batched line search needs about as many Armijo trials per
    iteration as the FP64 oracle's (about one), where without it the tiles
    near convergence spend up to 20 trials on rounding."""
    torch, dv = env
    w, psfs, y, _ = workload_case("disks128")
    G = psfs.shape[:2]
    kw = dict(n_tiles=G, weights="per_tile", lam=w.lam, delta=w.delta, gamma=w.gamma,
              rho=w.rho, n_outer=6, n_inner=10, inner_increment=10, path=DIRECT,
              local_solver=1, vm_memory=5)
    res = {}
    for stop in (1e-7, 0.0):
        plan = dv.Plan(w.hy, w.wy, psfs, vm_stop_rel=stop, **kw)
        xd, st = plan.solve(torch.from_numpy(y).cuda())
        torch.cuda.synchronize()
        res[stop] = (xd.cpu().numpy(), st)
        plan.close()
    lay = O.paper_layout(w.hy, w.wy, w.K, *G)
    ps, y64 = psfs.astype(np.float64), y.astype(np.float64)
    vst = {}
    xr, _ = O.solve(y64, ps, lay, w.lam, w.delta, w.gamma, w.rho, 6, 10, inner_increment=10,
                    weights="per_tile", local_solver="vmlmb", vm_memory=5, vm_stop_rel=1e-7,
                    vm_stats=vst)
    oracle_mean = float(np.mean(vst["trials"]))
    xd, st = res[1e-7]
    print(f"trials per iteration: GPU batched {st['vm_trials_per_iter']:.2f} (max "
          f"{st['vm_trials_max']}), GPU per tile {st['vm_tile_trials']:.2f}, oracle per tile "
          f"{oracle_mean:.2f}; without the stop: batched {res[0.0][1]['vm_trials_per_iter']:.2f}; "
          f"stops {st['vm_stops']}")
    assert oracle_mean <= 1.5
    assert st["vm_tile_trials"] <= oracle_mean + 0.5
    assert st["vm_trials_per_iter"] <= 2.5
    F = O.objective(xr, y64, ps, lay, w.lam, w.delta, weights="per_tile")[0]
    assert abs(st["objective"] - F) <= 1e-4 * F
    assert abs(res[0.0][1]["objective"] - F) <= 1e-4 * F


def test_grouped_tensor_solve_is_bit_identical_to_eager(env):
    """The captured local solve of the tensor path runs its tile groups on
    concurrent streams; the result equals one launch per operator over every
    tile (eager), and event timing counts whole local solves (kind 3)."""
    torch, dv = env
    w, psfs, y, _ = workload_case("disks128")
    p1, x1, s1 = _gpu_solve(env, w, psfs, y, 4, 3, use_graphs=1, path=TENSOR, precision=BF16)
    p2, x2, s2 = _gpu_solve(env, w, psfs, y, 4, 3, use_graphs=0, path=TENSOR, precision=BF16)
    assert p1.info.tile_groups == 4 and p2.info.tile_groups == 1
    np.testing.assert_array_equal(x1, x2)
    assert s1["objective"] == s2["objective"]
    dv.dv_plan_set_timing(p1.handle, 1)
    xd, _ = p1.solve(torch.from_numpy(y).cuda(), stats=False)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(xd.cpu().numpy(), x1)
    ms, cnt = dv.dv_plan_kernel_time(p1.handle, 3)
    assert cnt == 4 and ms > 0.0
    assert dv.dv_plan_kernel_time(p1.handle, 0)[1] == 0
    assert dv.dv_plan_kernel_time(p1.handle, 2)[1] == 4
    dv.dv_plan_set_timing(p1.handle, 0)
    p1.close()
    p2.close()


def test_autotuner_weighs_the_tensor_path(env):
    torch, dv = env
    w, psfs, y, _ = workload_case("disks128")
    plan = dv.Plan(w.hy, w.wy, psfs, n_tiles=w.n_tiles, overlap=w.overlap, path=0,
                   precision=BF16)
    i = plan.info
    assert i.tune_ms_tensor > 0 and i.fp32_path in (DIRECT, FFT)
    fp32_ms = i.tune_ms_fft if i.fp32_path == FFT else i.tune_ms_direct
    assert i.path == (TENSOR if i.tune_ms_tensor < fp32_ms else i.fp32_path)
    plan.close()


def test_unsupported_precisions_are_reported(env):
    torch, dv = env
    psfs = np.full((1, 1, 9, 9), 1 / 81.0, dtype=np.float32)
    with pytest.raises(dv.DVError) as e:
        dv.Plan(40, 40, psfs, path=TENSOR)            # FP32 has no tensor path
    assert e.value.code == dv.DV_ERR_INVALID_ARG
    p11 = np.full((1, 1, 11, 11), 1 / 121.0, dtype=np.float32)
    with pytest.raises(dv.DVError) as e:
        dv.Plan(40, 40, p11, precision=TF32, path=TENSOR)
    assert e.value.code == dv.DV_ERR_UNSUPPORTED
    plan = dv.Plan(40, 40, p11, precision=BF16)       # automatic: an FP32 path
    assert plan.info.path in (DIRECT, FFT) and plan.info.tune_ms_tensor == 0
    plan.close()
