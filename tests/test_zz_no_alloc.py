"""The allocation-free prior entry point, for callers that may not allocate device
memory (plug-ins inside a framework that owns all device memory, real-time
loops where a cudaMalloc could stall the device).

dv_prior_value_noalloc keeps its partial sums in a static device array instead
of allocating them.  Its value must equal the prior term the solver reports
(dv_consensus_solve's stats, computed with plan-allocated scratch) for a
one-tile plan, where both sum hub(|grad x|) over the same image.  Two calls in
a row, the second on a smaller image, check that what the first call leaves in
the shared array does not leak into the second.  This file is collected last."""

import numpy as np
import pytest

from tests.gpu_common import need_gpu, random_psfs

pytestmark = pytest.mark.gpu

TOL = 1e-5   # relative tolerance used for the solver's objective terms


def _solve_one_tile(torch, dv, hy, wy, seed):
    g = np.random.default_rng(seed)
    K = 5
    psfs = random_psfs(g, (2, 2), K)
    y = g.uniform(0, 1, (hy, wy)).astype(np.float32)
    plan = dv.Plan(hy, wy, psfs, n_tiles=(1, 1), lam=0.01, delta=0.05, gamma=0.4, n_outer=3,
                   n_inner=2)
    x, st = plan.solve(torch.from_numpy(y).cuda())
    torch.cuda.synchronize()
    plan.close()
    return x, st["prior_term"], 0.05


def test_noalloc_prior_matches_solver_prior_twice():
    torch, dv = need_gpu()
    xa, prior_a, delta = _solve_one_tile(torch, dv, 300, 260, seed=1)
    xb, prior_b, _ = _solve_one_tile(torch, dv, 90, 70, seed=2)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    dv.dv_prior_value_noalloc(xa, delta, out[0:1])
    dv.dv_prior_value_noalloc(xb, delta, out[1:2])
    torch.cuda.synchronize()
    va, vb = out.cpu().numpy()
    assert abs(va - prior_a) <= TOL * abs(prior_a)
    assert abs(vb - prior_b) <= TOL * abs(prior_b)


def test_noalloc_prior_rejects_oversize_images():
    torch, dv = need_gpu()
    x = torch.zeros((70000, 1), device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(dv.DVError) as e:
        dv.dv_prior_value_noalloc(x, 0.1, out)
    assert e.value.code == dv.DV_ERR_INVALID_ARG
    x = torch.zeros((4096, 257 * 16), device="cuda")
    with pytest.raises(dv.DVError, match="allocation-free scratch"):
        dv.dv_prior_value_noalloc(x, 0.1, out)
