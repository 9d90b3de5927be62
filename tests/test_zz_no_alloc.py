"""The allocation-free prior entry point, for callers that may not allocate device
memory (plug-ins inside a framework that owns all device memory, real-time
loops where a cudaMalloc could stall the device).

dv_prior_value_noalloc keeps its partial sums in a static device array instead
of allocating them.  Its value must equal the FP64 oracle's Huber prior on the
same image (both sum hub(|grad x|) in FP64 from the same FP32 pixels, so only
the summation order differs) and the prior term the solver reports through
dv_consensus_solve's stats (plan-allocated scratch) for a one-tile plan.  The
images cross the kernel's 256-column chunk edges with ragged tails.  Two calls
in a row, the second on a smaller image, check that what the first call leaves
in the shared array does not leak into the second; device memory is checked
to be unchanged by a call.  This file is collected last."""

import numpy as np
import pytest

from oracle import dv_oracle as O
from tests.gpu_common import need_gpu, random_psfs

pytestmark = pytest.mark.gpu

TOL_SOLVER = 1e-5   # relative tolerance of the solver's objective terms
TOL_ORACLE = 1e-10  # FP64 sums of the same terms in another order


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


def test_noalloc_prior_matches_oracle_and_solver_twice():
    torch, dv = need_gpu()
    # 304 x 260 x-pixels: one full 256-column chunk and a ragged 4-column tail
    xa, prior_a, delta = _solve_one_tile(torch, dv, 300, 256, seed=1)
    xb, prior_b, _ = _solve_one_tile(torch, dv, 90, 70, seed=2)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    dv.dv_prior_value_noalloc(xa, delta, out[0:1])
    dv.dv_prior_value_noalloc(xb, delta, out[1:2])
    torch.cuda.synchronize()
    va, vb = out.cpu().numpy()
    for v, x, prior in ((va, xa, prior_a), (vb, xb, prior_b)):
        ref = O.huber_value(x.cpu().numpy().astype(np.float64), delta)
        assert abs(v - ref) <= TOL_ORACLE * abs(ref)
        assert abs(v - prior) <= TOL_SOLVER * abs(prior)


def test_noalloc_prior_two_chunk_edges_and_no_device_allocation():
    torch, dv = need_gpu()
    g = np.random.default_rng(5)
    # 513 columns: two chunk edges and a one-column tail; then a single column
    imgs = [g.uniform(0, 1, (37, 513)).astype(np.float32),
            g.standard_normal((129, 1)).astype(np.float32)]
    xs = [torch.from_numpy(a).cuda() for a in imgs]
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    dv.dv_prior_value_noalloc(xs[0], 0.2, out[0:1])      # warm-up: module loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for i, (x, a) in enumerate(zip(xs, imgs)):
        dv.dv_prior_value_noalloc(x, 0.2, out[i:i + 1])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    for v, a in zip(out.cpu().numpy(), imgs):
        ref = O.huber_value(a.astype(np.float64), 0.2)
        assert abs(v - ref) <= TOL_ORACLE * abs(ref)


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
