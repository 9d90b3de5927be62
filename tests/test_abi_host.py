"""Host-only checks of the C ABI (no GPU needed): libdv.so loads, exports every
function include/dv.h declares, and its host-side layout logic (tiling,
consensus weights, local step sizes) agrees with the oracle; invalid problems
are rejected with DV_ERR_INVALID_ARG."""

import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import dv_oracle as O
from paper_1705_06603_gb300 import build as dvbuild
from paper_1705_06603_gb300.synth import WORKLOADS, psf_grid_for

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dv():
    dvbuild.build()
    from paper_1705_06603_gb300 import dv as mod
    return mod


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dv_[a-z_0-9A-Z]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("dv_plan_create", "dv_apply_H", "dv_apply_Ht", "dv_consensus_solve", "dv_destroy",
              "dv_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(dv):
    lib = C.CDLL(dv._LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) == set(dv.EXPORTED)


@pytest.mark.parametrize("name", ["disks128", "stars2048", "wide8192", "giga32768"])
def test_layout_and_steps_match_oracle(dv, name):
    w = WORKLOADS[name]
    psfs = psf_grid_for(w) if name != "giga32768" else np.full((2, 2, w.K, w.K), 1.0 / w.K**2)
    bounds = (w.yrows, w.ycols) if w.yrows is not None else None
    p, keep = dv.make_problem(w.hy, w.wy, psfs, n_tiles=w.n_tiles, overlap=w.overlap,
                              tile_bounds=bounds, lam=w.lam, delta=w.delta, gamma=w.gamma)
    rows, cols, tau = dv.dv_layout_query(p)
    lay = O.make_layout(w.hy, w.wy, w.K, *w.n_tiles, w.overlap, w.yrows, w.ycols)
    assert rows == [tuple(r) for r in lay.yrows]
    assert cols == [tuple(c) for c in lay.ycols]
    ps = psfs.astype(np.float32).astype(np.float64)
    for tr, tc in lay.tiles:
        ref = O.tile_step(lay, tr, tc, ps, None, w.lam, w.gamma)
        assert abs(tau[tr, tc] - ref) <= 1e-12 * ref


def test_layout_with_noise_weights(dv):
    g = np.random.default_rng(0)
    K = 5
    psfs = g.uniform(0, 1, (2, 2, K, K))
    psfs /= psfs.sum(axis=(2, 3), keepdims=True)
    W = g.uniform(0.1, 1.0, (40, 30)).astype(np.float32)
    p, keep = dv.make_problem(40, 30, psfs, n_tiles=(3, 2), overlap=6, noise_w=W, lam=0.01,
                              gamma=0.7)
    _, _, tau = dv.dv_layout_query(p)
    lay = O.make_layout(40, 30, K, 3, 2, 6)
    for tr, tc in lay.tiles:
        ref = O.tile_step(lay, tr, tc, psfs.astype(np.float32).astype(np.float64),
                          W.astype(np.float64), 0.01, 0.7)
        assert abs(tau[tr, tc] - ref) <= 1e-12 * ref


@pytest.mark.parametrize("change,needle", [
    (dict(K=4), "K must be odd"),
    (dict(rho=2.0), "rho"),
    (dict(gamma=0.0), "gamma"),
    (dict(delta=-1.0), "delta"),
    (dict(n_outer=-1), "iteration"),
    (dict(path=4), "operator path"),
    (dict(precision=3), "precision"),
    (dict(n_tc=1025), "tile grid"),
    (dict(local_solver=2), "local_solver"),
    (dict(vm_memory=33), "vm_memory"),
    (dict(weight_kind=3), "weight_kind"),
])
def test_invalid_problems_rejected(dv, change, needle):
    psfs = np.full((1, 1, 3, 3), 1 / 9.0)
    p, keep = dv.make_problem(20, 20, psfs)
    for k, v in change.items():
        setattr(p, k, v)
    with pytest.raises(dv.DVError) as e:
        dv.dv_layout_query(p)
    assert e.value.code == dv.DV_ERR_INVALID_ARG
    assert needle in str(e.value)


def test_bad_tilings_rejected(dv):
    psfs = np.full((1, 1, 3, 3), 1 / 9.0)
    # a gap between y-blocks
    p, keep = dv.make_problem(20, 20, psfs, n_tiles=(2, 1),
                              tile_bounds=([(0, 9), (10, 20)], [(0, 20)]))
    with pytest.raises(dv.DVError, match="gap"):
        dv.dv_layout_query(p)
    # x-tiles 0 and 2 overlap (each x-tile may only overlap its neighbours)
    p, keep = dv.make_problem(20, 20, psfs, n_tiles=(3, 1),
                              tile_bounds=([(0, 10), (5, 15), (10, 20)], [(0, 20)]))
    with pytest.raises(dv.DVError, match="overlap"):
        dv.dv_layout_query(p)


def test_separable_weights_validated(dv):
    K, hy, wy = 3, 10, 12
    psfs = np.full((3, 2, K, K), 1 / 9.0)
    wr = O.bilinear_weights(hy + K - 1, 3).astype(np.float32)
    wc = O.bilinear_weights(wy + K - 1, 2).astype(np.float32)
    p, keep = dv.make_problem(hy, wy, psfs, weights=(wr, wc))
    dv.dv_layout_query(p)
    bad = wr.copy()
    bad[:, 4] = 0.3        # three grid points nonzero at one coordinate
    p, keep = dv.make_problem(hy, wy, psfs, weights=(bad, wc))
    with pytest.raises(dv.DVError, match="at most two"):
        dv.dv_layout_query(p)


@pytest.mark.parametrize("path,prec", [(0, 0), (1, 0), (2, 0), (3, 1), (3, 2), (0, 2)])
def test_every_operator_path_is_a_valid_request(dv, path, prec):
    """Host-side validation accepts every dv_operator_path / dv_precision
    value (whether the tensor path applies to the PSF size is decided at plan
    creation)."""
    psfs = np.full((1, 1, 9, 9), 1 / 81.0)
    p, keep = dv.make_problem(20, 20, psfs, path=path, precision=prec)
    dv.dv_layout_query(p)


@pytest.mark.parametrize("hy,wy,K,G", [(128, 128, 9, (3, 3)), (2048, 2048, 31, (8, 8)),
                                       (200, 150, 15, (4, 2)), (97, 301, 9, (1, 5)),
                                       (8192, 8192, 63, (16, 16))])
def test_paper_layout_and_steps_match_oracle(dv, hy, wy, K, G):
    """One PSF per tile (reading R18): the library's blocks and per-tile steps
    equal the oracle's independent construction."""
    g = np.random.default_rng(K)
    psfs = g.uniform(0.0, 1.0, (G[0], G[1], K, K)).astype(np.float32)
    psfs /= psfs.sum(axis=(2, 3), keepdims=True)
    p, keep = dv.make_problem(hy, wy, psfs, n_tiles=G, weights="per_tile", lam=2e-3, gamma=0.3)
    rows, cols, tau = dv.dv_layout_query(p)
    lay = O.paper_layout(hy, wy, K, *G)
    assert rows == [tuple(r) for r in lay.yrows]
    assert cols == [tuple(c) for c in lay.ycols]
    ps = psfs.astype(np.float64)
    for tr, tc in lay.tiles:
        op = O.tile_operator(lay, tr, tc, ps, "per_tile")
        ref = O.tile_step(lay, tr, tc, op[0], None, 2e-3, 0.3)
        assert abs(tau[tr, tc] - ref) <= 1e-12 * ref


def test_per_tile_weights_need_the_tile_grid(dv):
    psfs = np.full((3, 3, 9, 9), 1.0 / 81, dtype=np.float32)
    p, keep = dv.make_problem(128, 128, psfs, n_tiles=(2, 3), weights="per_tile")
    with pytest.raises(dv.DVError, match="tile grid"):
        dv.dv_layout_query(p)


def test_per_tile_weights_take_no_arrays(dv):
    psfs = np.full((2, 2, 5, 5), 1 / 25.0, dtype=np.float32)
    wr = np.ones((2, 24), np.float32)
    p, keep = dv.make_problem(20, 20, psfs, n_tiles=(2, 2), weights=(wr, wr))
    p.weight_kind = dv.DV_WEIGHTS_PER_TILE
    with pytest.raises(dv.DVError, match="no weight arrays"):
        dv.dv_layout_query(p)


@pytest.mark.parametrize("rows,cols,L", [(10, 40, 1.0), (40, 10, 1.0), (40, 40, 0.0),
                                         (40, 40, float("inf"))])
def test_image_quality_arguments_checked_before_any_work(dv, rows, cols, L):
    """dv_image_quality refuses windows smaller than 11 x 11 and a bad dynamic
    range before touching device memory (the pointers here are never read)."""
    fake = C.c_void_p(16)
    rc = dv._lib.dv_image_quality(fake, fake, rows, cols, L, fake, fake, None)
    assert rc == dv.DV_ERR_INVALID_ARG
    assert dv._lib.dv_image_quality(None, fake, 40, 40, 1.0, fake, fake, None) == dv.DV_ERR_INVALID_ARG
    assert dv._lib.dv_image_quality_workspace(40, 70) == 3 * 3 * 3
