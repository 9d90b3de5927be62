"""Failure detection on the GPU without a GPU fault: the bounded pipeline waits
of the tensor-core operator kernels.

With dv_plan_set_wait_test the banded BF16 kernels' bulk-copy lane issues none
of its operand copies, so the MMA lane's first wait on the copy ring can never
complete; the block-DFT kernels' loader warps load no window, so the staging
warps' first wait can never complete.  The wait gives up after the plan's wait limit (20 ms here), every
role of the CTA stops with nothing in flight, tensor memory is freed and the
kernel returns; the solve then reports DV_ERR_TIMEOUT.  The CUDA context stays
usable: the plan is destroyed and a fresh plan solves the same problem and
matches the FP64 oracle."""

import time

import numpy as np
import pytest

from tests.gpu_common import assert_close, need_gpu, oracle_solve, workload_case

pytestmark = pytest.mark.gpu

TENSOR, BF16 = 3, 2


def _plan(dv, w, psfs, **kw):
    return dv.Plan(w.hy, w.wy, psfs, n_tiles=w.n_tiles, overlap=w.overlap, lam=w.lam,
                   delta=w.delta, gamma=w.gamma, rho=w.rho, n_outer=2, n_inner=2,
                   precision=BF16, path=TENSOR, **kw)


@pytest.mark.parametrize("use_graphs,tensor_h", [(1, 1), (0, 1), (1, 3), (0, 3)])
def test_withheld_copies_time_out_and_the_context_survives(use_graphs, tensor_h):
    torch, dv = need_gpu()
    w, psfs, y, _ = workload_case("disks128")
    yd = torch.from_numpy(y).cuda()
    plan = _plan(dv, w, psfs, use_graphs=use_graphs, tensor_h=tensor_h)
    assert plan.info.path == TENSOR
    assert plan.info.tensor_ht_dft == (1 if tensor_h == 3 else 0)
    dv.dv_plan_set_wait_limit(plan.handle, 0.02)
    dv.dv_plan_set_wait_test(plan.handle, 1)
    t0 = time.perf_counter()
    with pytest.raises(dv.DVError) as e:
        plan.solve(yd)
    assert e.value.code == dv.DV_ERR_TIMEOUT
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 30.0
    plan.close()
    # the device and a new plan work normally
    z = torch.ones(1024, device="cuda").sum().item()
    assert z == 1024.0
    plan = _plan(dv, w, psfs, use_graphs=use_graphs, tensor_h=tensor_h)
    xd, st = plan.solve(yd)
    torch.cuda.synchronize()
    plan.close()
    _, xr, _ = oracle_solve(w, psfs, y, 2, 2)
    assert_close(xd.cpu().numpy(), xr, 3e-3)


def test_wait_settings_are_checked():
    torch, dv = need_gpu()
    w, psfs, _, _ = workload_case("disks128")
    plan = _plan(dv, w, psfs)
    for bad in (-1.0, 61.0, float("nan")):
        with pytest.raises(dv.DVError) as e:
            dv.dv_plan_set_wait_limit(plan.handle, bad)
        assert e.value.code == dv.DV_ERR_INVALID_ARG
    with pytest.raises(dv.DVError):
        dv.dv_plan_set_wait_test(plan.handle, 2)
    dv.dv_plan_set_wait_limit(plan.handle, 0.0)
    plan.close()
