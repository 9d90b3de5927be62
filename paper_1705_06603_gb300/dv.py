"""Thin Python binding of libdv (the C ABI declared in include/dv.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Device buffers are torch CUDA tensors (float32, contiguous); streams are torch
CUDA streams.  Importing this module loads libdv.so and raises ImportError if
the library has not been built (python -m paper_1705_06603_gb300.build) or
cannot be loaded: there is no fallback implementation.

Names follow the C ABI: dv_plan_create, dv_apply_H, dv_apply_Ht,
dv_consensus_solve, dv_destroy, ...  `Plan` is a small convenience wrapper.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdv.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libdv.so is not built ({_LIB_PATH}); run python -m "
                      "paper_1705_06603_gb300.build (needs nvcc)")
try:
    _lib = C.CDLL(_LIB_PATH)
except OSError as e:  # pragma: no cover - depends on the machine
    raise ImportError(f"cannot load {_LIB_PATH}: {e}") from e

DV_OK, DV_ERR_INVALID_ARG, DV_ERR_CUDA, DV_ERR_OOM, DV_ERR_TIMEOUT, DV_ERR_UNSUPPORTED = range(6)
DV_PREC_FP32, DV_PREC_TF32, DV_PREC_BF16 = 0, 1, 2
DV_WEIGHTS_BILINEAR, DV_WEIGHTS_SEPARABLE, DV_WEIGHTS_PER_TILE = 0, 1, 2
DV_PATH_AUTO, DV_PATH_DIRECT, DV_PATH_FFT, DV_PATH_TENSOR = 0, 1, 2, 3
DV_SOLVER_PG, DV_SOLVER_VMLMB = 0, 1
KERNEL_H, KERNEL_HT_STEP, KERNEL_CONSENSUS = 0, 1, 2

_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)


class dv_problem(C.Structure):
    _fields_ = [("hy", C.c_int32), ("wy", C.c_int32),
                ("grid_r", C.c_int32), ("grid_c", C.c_int32), ("K", C.c_int32),
                ("psfs", _fp),
                ("weight_kind", C.c_int32), ("weights_r", _fp), ("weights_c", _fp),
                ("n_tr", C.c_int32), ("n_tc", C.c_int32),
                ("tile_r0", _ip), ("tile_r1", _ip), ("tile_c0", _ip), ("tile_c1", _ip),
                ("overlap", C.c_int32),
                ("noise_w", _fp),
                ("lambda_", C.c_double), ("delta", C.c_double), ("gamma", C.c_double),
                ("rho", C.c_double),
                ("n_outer", C.c_int32), ("n_inner", C.c_int32), ("inner_increment", C.c_int32),
                ("precision", C.c_int32), ("path", C.c_int32), ("use_warmstart", C.c_int32),
                ("check_every", C.c_int32), ("target_objective", C.c_double),
                ("use_graphs", C.c_int32), ("noise_sigma", C.c_double),
                ("local_solver", C.c_int32), ("vm_memory", C.c_int32),
                ("vm_stop_rel", C.c_double), ("tensor_h", C.c_int32),
                ("reserved", C.c_int32)]


class dv_stats(C.Structure):
    _fields_ = [("objective", C.c_double), ("data_term", C.c_double),
                ("prior_term", C.c_double), ("primal_res", C.c_double),
                ("dual_res", C.c_double), ("outer_done", C.c_int32), ("inner_done", C.c_int32),
                ("ms_total", C.c_double), ("kernel_launches", C.c_int64),
                ("vm_trials_per_iter", C.c_double), ("vm_tile_trials", C.c_double),
                ("vm_trials_max", C.c_int32), ("vm_stops", C.c_int32)]


class dv_plan_info(C.Structure):
    _fields_ = [("nx_r", C.c_int32), ("nx_c", C.c_int32), ("n_tiles", C.c_int32),
                ("path", C.c_int32), ("stack_elems", C.c_int64), ("device_bytes", C.c_int64),
                ("tau_min", C.c_double), ("tau_max", C.c_double),
                ("kernel_launches", C.c_int64), ("tune_ms_direct", C.c_double),
                ("tune_ms_fft", C.c_double), ("blocks", C.c_int64 * 2),
                ("block_psfs", C.c_int64 * 2), ("psf_pairs", C.c_int64 * 2),
                ("block_side", C.c_int32), ("fp32_path", C.c_int32),
                ("tune_ms_tensor", C.c_double), ("mma_ksteps", C.c_int64 * 2),
                ("tile_groups", C.c_int32), ("tensor_h_dft", C.c_int32),
                ("tune_ms_tensor_dft", C.c_double), ("tensor_ht_dft", C.c_int32),
                ("dft_h_rows", C.c_int32), ("tune_ms_tensor_dft2", C.c_double)]


_vp = C.c_void_p
_sigs = {
    "dv_problem_init": (None, [C.POINTER(dv_problem)]),
    "dv_layout_query": (C.c_int, [C.POINTER(dv_problem), _ip, _ip, _ip, _ip,
                                  C.POINTER(C.c_double)]),
    "dv_plan_create": (C.c_int, [C.POINTER(dv_problem), _vp, C.POINTER(_vp)]),
    "dv_apply_H": (C.c_int, [_vp, _vp, _vp, _vp]),
    "dv_apply_Ht": (C.c_int, [_vp, _vp, _vp, _vp]),
    "dv_consensus_solve": (C.c_int, [_vp, _vp, _vp, _vp, C.POINTER(dv_stats), _vp]),
    "dv_consensus_solve_host": (C.c_int, [_vp, _vp, _vp, _vp, C.POINTER(dv_stats), _vp]),
    "dv_consensus_continue": (C.c_int, [_vp, _vp, C.c_int32, _vp, C.POINTER(dv_stats), _vp]),
    "dv_state_export": (C.c_int, [_vp, _vp, _vp, _ip, _vp]),
    "dv_state_import": (C.c_int, [_vp, _vp, _vp, C.c_int32, _vp]),
    "dv_plan_get_info": (C.c_int, [_vp, C.POINTER(dv_plan_info)]),
    "dv_plan_set_timing": (C.c_int, [_vp, C.c_int32]),
    "dv_plan_set_wait_limit": (C.c_int, [_vp, C.c_double]),
    "dv_plan_set_wait_test": (C.c_int, [_vp, C.c_int32]),
    "dv_plan_kernel_time": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_double),
                                      C.POINTER(C.c_int64)]),
    "dv_prior_value_noalloc": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_double, _vp, _vp]),
    "dv_cnn_create": (C.c_int, [C.c_int32, C.c_int32, C.c_uint64, _vp, C.POINTER(_vp)]),
    "dv_cnn_param_count": (C.c_int64, [_vp]),
    "dv_cnn_get_params": (C.c_int, [_vp, _vp, C.c_int64, C.POINTER(C.c_int64)]),
    "dv_cnn_set_params": (C.c_int, [_vp, _vp, C.c_int64, _vp]),
    "dv_cnn_forward": (C.c_int, [_vp, _vp, C.c_int32, C.c_int32, C.c_int32, _vp, _vp]),
    "dv_cnn_gradients": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_int32, C.c_int32, _vp,
                                   C.POINTER(C.c_double), _vp]),
    "dv_cnn_train_step": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_int32, C.c_int32, C.c_float,
                                    C.POINTER(C.c_double), _vp]),
    "dv_cnn_train_crops": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_int32, C.c_int32, _vp,
                                     C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp]),
    "dv_cnn_destroy": (C.c_int, [_vp]),
    "dv_image_quality_workspace": (C.c_int64, [C.c_int32, C.c_int32]),
    "dv_image_quality": (C.c_int, [_vp, _vp, C.c_int32, C.c_int32, C.c_double, _vp, _vp, _vp]),
    "dv_plan_set_warmstart": (C.c_int, [_vp, _vp]),
    "dv_warmstart_features": (C.c_int, [_vp, _vp, _vp, _vp]),
    "dv_destroy": (C.c_int, [_vp]),
    "dv_last_error": (C.c_char_p, []),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sigs)


class DVError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdv error {code}: {msg}")
        self.code = code


def _check(code):
    if code != DV_OK:
        raise DVError(code, (_lib.dv_last_error() or b"").decode())


def dv_last_error() -> str:
    return (_lib.dv_last_error() or b"").decode()


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t, name, shape=None, writable=False):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


def _hptr(a, name, shape=None):
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous):
        raise TypeError(f"{name} must be a C-contiguous float32 numpy array")
    if shape is not None and tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {a.shape}, expected {tuple(shape)}")
    return C.c_void_p(a.ctypes.data)


def make_problem(hy, wy, psfs, n_tiles=(1, 1), overlap=16, tile_bounds=None, weights=None,
                 noise_w=None, lam=1e-3, delta=1.0 / 60.0, gamma=0.4, rho=1.0, n_outer=30,
                 n_inner=10, inner_increment=0, precision=DV_PREC_FP32, path=DV_PATH_AUTO,
                 use_warmstart=0, check_every=0, target_objective=0.0, use_graphs=1,
                 noise_sigma=0.0, local_solver=0, vm_memory=0, vm_stop_rel=None, tensor_h=0):
    """Builds a dv_problem.  weights: None (bilinear tents), (weights_r,
    weights_c) separable profiles, or "per_tile" (one PSF per tile, the PSF
    grid being the tile grid).  Returns (problem, keepalive) where keepalive
    holds the host arrays the struct points to until dv_plan_create has copied
    them."""
    p = dv_problem()
    _lib.dv_problem_init(C.byref(p))
    psfs = np.ascontiguousarray(psfs, dtype=np.float32)
    Gr, Gc, K, K2 = psfs.shape
    if K != K2:
        raise ValueError("PSFs must be square")
    keep = [psfs]
    p.hy, p.wy, p.grid_r, p.grid_c, p.K = hy, wy, Gr, Gc, K
    p.psfs = psfs.ctypes.data_as(_fp)
    if isinstance(weights, str):
        if weights != "per_tile":
            raise ValueError(f"unknown weights {weights!r}")
        p.weight_kind = DV_WEIGHTS_PER_TILE
    elif weights is not None:
        wr = np.ascontiguousarray(weights[0], dtype=np.float32)
        wc = np.ascontiguousarray(weights[1], dtype=np.float32)
        keep += [wr, wc]
        p.weight_kind = DV_WEIGHTS_SEPARABLE
        p.weights_r, p.weights_c = wr.ctypes.data_as(_fp), wc.ctypes.data_as(_fp)
    p.n_tr, p.n_tc = n_tiles
    p.overlap = overlap
    if tile_bounds is not None:
        arrs = [np.ascontiguousarray(np.asarray(v, dtype=np.int32)) for v in
                ([b[0] for b in tile_bounds[0]], [b[1] for b in tile_bounds[0]],
                 [b[0] for b in tile_bounds[1]], [b[1] for b in tile_bounds[1]])]
        keep += arrs
        p.tile_r0, p.tile_r1, p.tile_c0, p.tile_c1 = (a.ctypes.data_as(_ip) for a in arrs)
    if noise_w is not None:
        nw = np.ascontiguousarray(noise_w, dtype=np.float32)
        keep.append(nw)
        p.noise_w = nw.ctypes.data_as(_fp)
    p.lambda_, p.delta, p.gamma, p.rho = lam, delta, gamma, rho
    p.n_outer, p.n_inner, p.inner_increment = n_outer, n_inner, inner_increment
    p.precision, p.path, p.use_warmstart = precision, path, use_warmstart
    p.check_every, p.target_objective, p.use_graphs = check_every, target_objective, use_graphs
    p.noise_sigma = noise_sigma
    p.local_solver, p.vm_memory = local_solver, vm_memory
    if vm_stop_rel is not None:
        p.vm_stop_rel = vm_stop_rel
    p.tensor_h = tensor_h
    return p, keep


def dv_layout_query(problem):
    """Host-only: (row blocks, col blocks, tau[n_tr, n_tc]) the plan would use."""
    ntr, ntc = problem.n_tr, problem.n_tc
    r0, r1 = (C.c_int32 * ntr)(), (C.c_int32 * ntr)()
    c0, c1 = (C.c_int32 * ntc)(), (C.c_int32 * ntc)()
    tau = (C.c_double * (ntr * ntc))()
    _check(_lib.dv_layout_query(C.byref(problem), r0, r1, c0, c1, tau))
    return (list(zip(r0, r1)), list(zip(c0, c1)), np.array(tau[:]).reshape(ntr, ntc))


def dv_plan_create(problem, stream=None):
    h = C.c_void_p()
    _check(_lib.dv_plan_create(C.byref(problem), _stream_handle(stream), C.byref(h)))
    return h


def dv_apply_H(plan, x, y, stream=None):
    _check(_lib.dv_apply_H(plan, _dptr(x, "x"), _dptr(y, "y"), _stream_handle(stream)))


def dv_apply_Ht(plan, r, g, stream=None):
    _check(_lib.dv_apply_Ht(plan, _dptr(r, "r"), _dptr(g, "g"), _stream_handle(stream)))


def dv_consensus_solve(plan, y, x0, x_out, stats=None, stream=None):
    _check(_lib.dv_consensus_solve(plan, _dptr(y, "y"), _dptr(x0, "x0"), _dptr(x_out, "x_out"),
                                   C.byref(stats) if stats is not None else None,
                                   _stream_handle(stream)))


def dv_consensus_solve_host(plan, y, x0, x_out, stats=None, stream=None):
    _check(_lib.dv_consensus_solve_host(plan, _hptr(y, "y"), _hptr(x0, "x0"),
                                        _hptr(x_out, "x_out"),
                                        C.byref(stats) if stats is not None else None,
                                        _stream_handle(stream)))


def dv_consensus_continue(plan, y, n_outer, x_out, stats=None, stream=None):
    _check(_lib.dv_consensus_continue(plan, _dptr(y, "y"), int(n_outer), _dptr(x_out, "x_out"),
                                      C.byref(stats) if stats is not None else None,
                                      _stream_handle(stream)))


def dv_state_export(plan, x_stack, u_stack, stream=None):
    k = C.c_int32()
    _check(_lib.dv_state_export(plan, _dptr(x_stack, "x_stack"), _dptr(u_stack, "u_stack"),
                                C.byref(k), _stream_handle(stream)))
    return k.value


def dv_state_import(plan, x_stack, u_stack, outer_done, stream=None):
    _check(_lib.dv_state_import(plan, _dptr(x_stack, "x_stack"), _dptr(u_stack, "u_stack"),
                                int(outer_done), _stream_handle(stream)))


def dv_plan_get_info(plan):
    i = dv_plan_info()
    _check(_lib.dv_plan_get_info(plan, C.byref(i)))
    return i


def dv_plan_set_timing(plan, enable):
    _check(_lib.dv_plan_set_timing(plan, int(bool(enable))))


def dv_plan_set_wait_limit(plan, seconds):
    _check(_lib.dv_plan_set_wait_limit(plan, float(seconds)))


def dv_plan_set_wait_test(plan, withhold):
    _check(_lib.dv_plan_set_wait_test(plan, int(withhold)))


def dv_plan_kernel_time(plan, kind):
    ms, n = C.c_double(), C.c_int64()
    _check(_lib.dv_plan_kernel_time(plan, int(kind), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def image_quality_async(x, ref, work, out, dynamic_range=1.0, stream=None):
    """Stream-ordered dv_image_quality into out (float64 CUDA tensor of 2);
    work: float64 CUDA tensor of dv_image_quality_workspace(rows, cols)."""
    import torch
    rows, cols = ref.shape
    for t, name, n in ((work, "work", int(_lib.dv_image_quality_workspace(rows, cols))),
                       (out, "out", 2)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.is_contiguous() and t.numel() >= n):
            raise TypeError(f"{name} must be a contiguous float64 CUDA tensor of >= {n} elements")
    _check(_lib.dv_image_quality(_dptr(x, "x", (rows, cols)), _dptr(ref, "ref", (rows, cols)),
                                 rows, cols, float(dynamic_range), C.c_void_p(work.data_ptr()),
                                 C.c_void_p(out.data_ptr()), _stream_handle(stream)))


def image_quality(x, ref, dynamic_range=1.0, stream=None):
    """(SNR in dB, mean SSIM) of the 2-D float32 CUDA tensor x against ref."""
    import torch
    rows, cols = ref.shape
    work = torch.empty(max(1, int(_lib.dv_image_quality_workspace(rows, cols))),
                       dtype=torch.float64, device=ref.device)
    out = torch.empty(2, dtype=torch.float64, device=ref.device)
    image_quality_async(x, ref, work, out, dynamic_range, stream)
    snr, ssim = out.cpu().tolist()
    return snr, ssim


def dv_prior_value_noalloc(x, delta, value, stream=None):
    """Huber prior value of the 2-D image x written to value (a 1-element float64
    CUDA tensor on x's device), with no device allocation (see include/dv.h).
    The call is made with x's device current, on `stream` (default: that
    device's current stream)."""
    import torch
    if not (isinstance(value, torch.Tensor) and value.is_cuda and value.dtype == torch.float64
            and value.numel() >= 1):
        raise TypeError("value must be a float64 CUDA tensor with at least one element")
    _dptr(x, "x")
    if x.dim() != 2:
        raise ValueError("x must be a 2-D image")
    if value.device != x.device:
        raise ValueError(f"value is on {value.device}, x on {x.device}: both must be on one GPU")
    with torch.cuda.device(x.device):
        st = _stream_handle(stream if stream is not None else torch.cuda.current_stream(x.device))
        _check(_lib.dv_prior_value_noalloc(_dptr(x, "x"), int(x.shape[0]), int(x.shape[1]),
                                           float(delta), C.c_void_p(value.data_ptr()), st))


CNN_IN_CH = 5


class Cnn:
    """The learned warm-start network (dv_cnn_*): NHWC float32 CUDA tensors."""

    def __init__(self, seed=0, stream=None):
        self.stream = stream
        h = C.c_void_p()
        _check(_lib.dv_cnn_create(32, 6, seed, _stream_handle(stream), C.byref(h)))
        self._h = h
        self.nparam = int(_lib.dv_cnn_param_count(h))

    @property
    def handle(self):
        return self._h

    def get_params(self):
        out = np.empty(self.nparam, dtype=np.float32)
        step = C.c_int64()
        _check(_lib.dv_cnn_get_params(self._h, C.c_void_p(out.ctypes.data), self.nparam,
                                      C.byref(step)))
        return out, step.value

    def set_params(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        _check(_lib.dv_cnn_set_params(self._h, C.c_void_p(params.ctypes.data), params.size,
                                      _stream_handle(self.stream)))

    def forward(self, x, out=None):
        import torch
        N, H, W, Cc = x.shape
        assert Cc == CNN_IN_CH
        out = out if out is not None else torch.empty((N, H, W), device=x.device)
        _check(_lib.dv_cnn_forward(self._h, _dptr(x, "x"), N, H, W, _dptr(out, "out"),
                                   _stream_handle(self.stream)))
        return out

    def gradients(self, x, target):
        N, H, W, _ = x.shape
        g = np.empty(self.nparam, dtype=np.float32)
        loss = C.c_double()
        _check(_lib.dv_cnn_gradients(self._h, _dptr(x, "x"), _dptr(target, "target"), N, H, W,
                                     C.c_void_p(g.ctypes.data), C.byref(loss),
                                     _stream_handle(self.stream)))
        return g, loss.value

    def train_step(self, x, target, lr):
        N, H, W, _ = x.shape
        loss = C.c_double()
        _check(_lib.dv_cnn_train_step(self._h, _dptr(x, "x"), _dptr(target, "target"), N, H, W,
                                      float(lr), C.byref(loss), _stream_handle(self.stream)))
        return loss.value

    def train_crops(self, feats, targets, crops, crop, lrs):
        """len(lrs) Adam steps on crops of stacked pairs: feats [P][H][W][5] and
        targets [P][H][W] (float32 CUDA), crops int32 [steps][batch][3] =
        (pair, r0, c0), lrs float32 [steps]; returns the per-step losses."""
        P, H, W, _ = feats.shape
        _dptr(feats, "feats")
        _dptr(targets, "targets", (P, H, W))
        crops = np.ascontiguousarray(crops, dtype=np.int32)
        lrs = np.ascontiguousarray(lrs, dtype=np.float32)
        steps, batch, three = crops.shape
        if three != 3 or lrs.shape != (steps,):
            raise ValueError("crops must be [steps][batch][3] and lrs [steps]")
        losses = np.empty(steps, dtype=np.float64)
        _check(_lib.dv_cnn_train_crops(self._h, _dptr(feats, "feats"), _dptr(targets, "targets"),
                                       P, H, W, C.c_void_p(crops.ctypes.data), steps, batch,
                                       int(crop), C.c_void_p(lrs.ctypes.data),
                                       C.c_void_p(losses.ctypes.data), _stream_handle(self.stream)))
        return losses

    def close(self):
        if self._h is not None and self._h.value:
            _lib.dv_cnn_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dv_plan_set_warmstart(plan, cnn):
    _check(_lib.dv_plan_set_warmstart(plan, cnn.handle if cnn is not None else None))


def dv_warmstart_features(plan, y, feat, stream=None):
    _check(_lib.dv_warmstart_features(plan, _dptr(y, "y"), _dptr(feat, "feat"),
                                      _stream_handle(stream)))


def dv_destroy(plan):
    _check(_lib.dv_destroy(plan))


def stats_dict(s: dv_stats) -> dict:
    return {f: getattr(s, f) for f, _ in dv_stats._fields_}


class Plan:
    """Owns one dv_plan; the methods are the C-ABI calls on torch tensors."""

    def __init__(self, hy, wy, psfs, stream=None, **kw):
        import torch
        self.problem, keep = make_problem(hy, wy, psfs, **kw)
        self.hy, self.wy, self.K = hy, wy, self.problem.K
        self.nx = (hy + self.K - 1, wy + self.K - 1)
        self.stream = stream
        self._h = dv_plan_create(self.problem, stream)
        del keep
        self.info = dv_plan_get_info(self._h)
        self._torch = torch

    @property
    def handle(self):
        return self._h

    def apply_H(self, x, y=None):
        y = y if y is not None else self._torch.empty((self.hy, self.wy), device=x.device)
        _dptr(x, "x", self.nx)
        _dptr(y, "y", (self.hy, self.wy))
        dv_apply_H(self._h, x, y, self.stream)
        return y

    def apply_Ht(self, r, g=None):
        g = g if g is not None else self._torch.empty(self.nx, device=r.device)
        _dptr(r, "r", (self.hy, self.wy))
        _dptr(g, "g", self.nx)
        dv_apply_Ht(self._h, r, g, self.stream)
        return g

    def solve(self, y, x0=None, x_out=None, stats=True):
        x_out = x_out if x_out is not None else self._torch.empty(self.nx, device=y.device)
        _dptr(y, "y", (self.hy, self.wy))
        _dptr(x0, "x0", self.nx)
        _dptr(x_out, "x_out", self.nx)
        st = dv_stats() if stats else None
        dv_consensus_solve(self._h, y, x0, x_out, st, self.stream)
        return x_out, (stats_dict(st) if stats else None)

    def solve_host(self, y, x0=None, stats=True):
        y = np.ascontiguousarray(y, dtype=np.float32)
        out = np.empty(self.nx, dtype=np.float32)
        st = dv_stats() if stats else None
        dv_consensus_solve_host(self._h, y, x0, out, st, self.stream)
        return out, (stats_dict(st) if stats else None)

    def close(self):
        if self._h is not None and self._h.value:
            dv_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
