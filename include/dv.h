/*
 * dv.h -- C ABI of libdv, a GB300 (sm_103a) implementation of distributed
 * shift-variant deblurring by Douglas-Rachford consensus ("Distributed
 * Deblurring of Large Images of Wide Field-Of-View").
 *
 * Model (Eq. (2), Eq. (3), Sec. II-B):
 *   y = H x + noise,  H x = R sum_p h_p * (w_p . x)
 * where the PSFs h_p sit on a G_r x G_c field grid, w_p are first-order
 * interpolation weights (sum_p w_p = 1) and R keeps the "valid" part: the
 * observed image y is hy x wy, the unknown x is (hy + K - 1) x (wy + K - 1).
 * Convolution is centred at (K/2, K/2):
 *   (H x)(i, j) = sum_p sum_{ka,kb} h_p(ka, kb) w_p(i + K-1 - ka, j + K-1 - kb)
 *                                            x(i + K-1 - ka, j + K-1 - kb).
 *
 * Distributed formulation (Sec. III-A, Eq. (4)): the observed image is split
 * into overlapping y-blocks; tile i estimates the x-tile P_i = its y-block
 * dilated by K - 1 (so the local operator H_i is exact), with local cost
 *   f_i(x_i) = 1/2 ||y_i - H_i x_i||^2_W + lambda phi(D x_i) + indicator(x_i >= 0)
 * and phi the Huber function of the forward-difference gradient (Sec. IV-A).
 * Algorithm 1 (Sec. III-B) alternates, n_outer times:
 *   x_i  <- Local-Solver(u_i)         n_inner projected-gradient steps on
 *                                     f_i + 1/2 ||. - u_i||^2_alpha_i
 *   zbar <- sum_i alpha_i (2 x_i - u_i) / sum_i alpha_i     (Lemma 1)
 *   u_i  <- u_i + rho (zbar - x_i)
 * with alpha_i = gamma omega_i and omega_i the consensus weights of the tiles
 * (sum_i omega_i = 1).  The result is x_hat = sum_i omega_i x_i / sum_i omega_i.
 *
 * Conventions for every entry point:
 *   - Images are row-major float32, densely packed (row pitch = width).
 *   - "_dev" pointers are CUDA device pointers, borrowed for the call only;
 *     "_host" pointers are host memory (pageable or pinned), borrowed likewise.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All work is ordered on it; calls return when the work is enqueued unless
 *     stated otherwise.
 *   - Return codes only: nothing throws or aborts across the ABI.  After
 *     DV_ERR_INVALID_ARG or DV_ERR_UNSUPPORTED the plan is unchanged and usable.
 *     After DV_ERR_CUDA, DV_ERR_OOM (during a call) or DV_ERR_TIMEOUT only
 *     dv_destroy is valid on that plan.  dv_last_error() describes the last
 *     failure of the calling thread.
 *   - A plan is not thread-safe: calls on one plan must be serialised.
 */
#ifndef DV_H
#define DV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DV_ABI_VERSION 3

typedef enum dv_status {
  DV_OK = 0,
  DV_ERR_INVALID_ARG = 1,  /* bad argument; message in dv_last_error()       */
  DV_ERR_CUDA = 2,         /* a CUDA runtime call failed                      */
  DV_ERR_OOM = 3,          /* device or pinned-host allocation failed         */
  DV_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up              */
  DV_ERR_UNSUPPORTED = 5   /* valid request the library does not implement    */
} dv_status;

/* Lowest operand precision allowed for the blur operator H and its adjoint
 * (Sec. II-B) in the inner iterations.  BF16 / TF32 let the autotuner pick
 * the tensor-core path when it is faster; the objective, the stopping test
 * and every other step run in FP32 with FP64 reductions. */
typedef enum dv_precision {
  DV_PREC_FP32 = 0,        /* FP32 operands, FP32 accumulation                 */
  DV_PREC_TF32 = 1,        /* TF32 operands on tensor cores, FP32 accumulation */
  DV_PREC_BF16 = 2         /* BF16 operands on tensor cores, FP32 accumulation */
} dv_precision;

/* Interpolation weights w_p (Sec. II-B, Fig. 1). */
typedef enum dv_weight_kind {
  /* Tents on G equidistant grid points per axis, corners included: grid
   * point a sits at c_a = a (n - 1)/(G - 1) (x-pixel coordinates) and
   * w_a(t) = max(0, 1 - |t - c_a| / ((n - 1)/(G - 1))).  w_p = w_a(row) w_b(col). */
  DV_WEIGHTS_BILINEAR = 0,
  /* Caller-given separable profiles weights_r [G_r][hy+K-1] and
   * weights_c [G_c][wy+K-1]; at most two neighbouring grid points may be
   * nonzero at any coordinate (first-order interpolation). */
  DV_WEIGHTS_SEPARABLE = 1,
  /* One PSF per block, the paper's own layout (Sec. III-A, III-C): the PSF
   * grid is the tile grid (grid_r = n_tr, grid_c = n_tc) and tile (tr, tc)
   * blurs with PSF (tr, tc) alone, weight 1 on the whole tile (the local
   * operators H_i = C_i H_i of Sec. II-B).  Without explicit tile bounds,
   * x-tile i spans the grid points i - 1 .. i + 1 of the bilinear grid
   * (c_a = a (n - 1)/(G - 1)): [ceil(c_{i-1}), ceil(c_{i+1})) with c_{-1} = 0 and
   * c_G = n; the y-block is the x-tile less K - 1 at its end.  Neighbours then
   * overlap by half a block and the consensus weights omega_i are the
   * first-order interpolation tents.  dv_apply_H / dv_apply_Ht and the warm
   * start use the bilinear interpolation of the same PSFs (the paper's data
   * model, Sec. II-B).  No weight arrays. */
  DV_WEIGHTS_PER_TILE = 2
} dv_weight_kind;

/* How H and H^T are computed; all give the same operator. */
typedef enum dv_operator_path {
  DV_PATH_AUTO = 0,        /* plan-time autotuner picks the fastest allowed  */
  DV_PATH_DIRECT = 1,      /* spatial-domain correlation, FP32               */
  DV_PATH_FFT = 2,         /* block FFT (overlap-save), FP32                 */
  DV_PATH_TENSOR = 3       /* direct correlation on tensor cores (tcgen05)
                            * with BF16 / TF32 operands as set by precision
                            * (not FP32); K = 9, 15, 31 or 63               */
} dv_operator_path;

/* Local-Solver of Algorithm 1 (Sec. IV-B). */
typedef enum dv_local_solver {
  /* projected gradient with the step tau_i (the default; captured in CUDA
   * graphs, fused into the H^T kernels) */
  DV_SOLVER_PG = 0,
  /* VMLM-B, the paper's solver: limited-memory variable metric (vm_memory
   * pairs, reset at every local solve) on the free variables, projected
   * Armijo line search (c1 = 1e-4, halving, at most 20 trials); the
   * projected-gradient step when memory is empty or the direction is not a
   * descent direction.  One inner iteration = one VMLM-B iteration.  Runs
   * eagerly, driven from the host with per-tile scalars (use_graphs does not
   * apply).  Its objectives and gradients use the plan's inner operator path;
   * they are FP64 sums of per-pixel terms formed in FP32 (or from BF16 / TF32
   * operands), which resolve relative changes of about 1e-7 and no finer, so
   * near convergence the Armijo comparisons can fail on rounding alone.  A tile
   * therefore ends its local solve once the decrease a full step promises,
   * -g'd, is at most vm_stop_rel |Phi_i| (dv_problem.vm_stop_rel; 0 runs every
   * iteration).  dv_stats reports the Armijo trials. */
  DV_SOLVER_VMLMB = 1
} dv_local_solver;

typedef struct dv_problem {
  /* observed image size (Eq. (2)); x is (hy + K - 1) x (wy + K - 1) */
  int32_t hy, wy;
  /* PSF grid and odd PSF side (Sec. II-B) */
  int32_t grid_r, grid_c, K;
  /* host [grid_r][grid_c][K][K]; nonnegative with unit sum is expected by the
   * step-size bound but not enforced.  Deep-copied by dv_plan_create. */
  const float* psfs;
  /* dv_weight_kind; for DV_WEIGHTS_SEPARABLE the two host profiles below
   * (deep-copied), otherwise they must be NULL */
  int32_t weight_kind;
  const float* weights_r;
  const float* weights_c;
  /* tile grid (Sec. III-A, III-C): n_tr x n_tc y-blocks.  If the four bound
   * arrays are NULL the blocks are uniform: B = ceil((n + (count-1) overlap) / count)
   * and block i starts at round(i (n - B)/(count - 1)).  Otherwise host arrays
   * of n_tr (rows) / n_tc (cols) half-open y-block bounds, sorted, covering
   * [0, hy) x [0, wy) with no gaps, and with each x-tile overlapping only its
   * immediate neighbours along each axis.  n_tr, n_tc <= 1024; x may have at
   * most 65535 rows (hy + K - 1). */
  int32_t n_tr, n_tc;
  const int32_t* tile_r0;
  const int32_t* tile_r1;
  const int32_t* tile_c0;
  const int32_t* tile_c1;
  int32_t overlap;
  /* host [hy][wy] noise weights W (Eq. (3); 0 = unmeasured pixel), or NULL
   * for W = 1.  Deep-copied. */
  const float* noise_w;
  /* prior weight, Huber threshold (Sec. IV-A), alpha_i = gamma omega_i and the
   * relaxation rho in (0, 2) (Sec. III-B) */
  double lambda, delta, gamma, rho;
  /* Algorithm 1: n_outer D-R iterations; the local solve at outer iteration k
   * runs n_inner + k * inner_increment projected-gradient steps (Sec. IV-B) */
  int32_t n_outer, n_inner, inner_increment;
  int32_t precision;       /* dv_precision */
  int32_t path;            /* dv_operator_path */
  int32_t use_warmstart;   /* 0: blurred-image start; 1: learned warm start */
  /* if > 0, evaluate the objective after check_every outer iterations and
   * stop as soon as it is <= target_objective (when target_objective > 0);
   * without a target it is evaluated every check_every iterations, with one
   * the next evaluation comes where the decrease per outer iteration since the
   * previous evaluation would reach the target (0.9 of that estimate, between
   * 1 and 2 check_every iterations) */
  int32_t check_every;
  double target_objective;
  int32_t use_graphs;      /* 1: replay each outer iteration as a CUDA graph */
  /* noise standard deviation of y, an input of the learned warm start only */
  double noise_sigma;
  int32_t local_solver;    /* dv_local_solver */
  int32_t vm_memory;       /* VMLM-B memory pairs, 1..32 (0: 5) */
  /* VMLM-B: a tile ends its local solve once -g'd <= vm_stop_rel |Phi_i(w)|
   * (>= 0; dv_problem_init sets 1e-7, the resolution of the FP32-formed
   * objective; 0 runs every iteration) */
  double vm_stop_rel;
  /* tensor-core path, BF16 allowed, the form of the operators H and H^T of
   * the inner iterations: 0 = whichever of the forms below the plan-time
   * autotuner finds fastest, 1 = banded Toeplitz MMAs (BF16 operands) for
   * both, 2 = H as the block DFT and H^T banded, 3 = both as block DFTs.
   * Block DFT: 128 x 128 overlap-save blocks of real data (each block scaled
   * by a power of two into FP16 range) transformed by dense half-spectrum
   * DFT GEMMs with FP16 operands and FP32 accumulation, the PSF spectra
   * (conjugated for H^T) applied between the forward and inverse transforms
   * (K in 9, 15, 31, 63). */
  int32_t tensor_h;
  int32_t reserved;
} dv_problem;

typedef struct dv_stats {
  double objective;        /* F(x_hat) = sum_i f_i(C_i x_hat) without indicator */
  double data_term;        /* sum_i 1/2 ||y_i - H_i C_i x_hat||^2_W */
  double prior_term;       /* sum_i phi(D C_i x_hat) (times lambda in F) */
  double primal_res;       /* sqrt(sum_i ||x_i - C_i zbar||^2), last iteration */
  double dual_res;         /* ||zbar^k - zbar^{k-1}|| over x pixels, last iteration */
  int32_t outer_done;      /* outer iterations performed */
  int32_t inner_done;      /* projected-gradient steps per tile performed */
  double ms_total;         /* wall time of the solve on the stream (events) */
  int64_t kernel_launches; /* libdv kernels launched by the call */
  /* VMLM-B Local-Solver (0 for projected gradient): Armijo trials per
   * iteration of the batched line search (the maximum over the tiles still
   * iterating), averaged over the iterations of the call, and their maximum;
   * trials per iteration of one tile averaged over (tile, iteration); and the
   * number of (tile, local solve) pairs ended by the vm_stop_rel test */
  double vm_trials_per_iter;
  double vm_tile_trials;
  int32_t vm_trials_max;
  int32_t vm_stops;
} dv_stats;

typedef struct dv_plan dv_plan;

/* Learned warm start (an addition to the paper's method, which starts from a
 * given guess, Algorithm 1): a 6-layer 3x3 convolutional network with 32
 * channels, bfloat16 weights and activations and FP32 accumulation, maps
 * DV_CNN_IN_CH feature maps of the x grid -- the observed image edge-replicated
 * by K/2; RMS radius / 8 px, 10 x peak and fraction of |h| beyond 3 px of the
 * PSFs, interpolated with the weights w_p; 100 x noise_sigma -- to a
 * correction d, and the solve starts from x0 = max(0, y_pad + d).  Network
 * tensors are NHWC float32 at the interface: input [N][H][W][5], output
 * [N][H][W].  Parameters (float32, the layout of dv_cnn_get_params) are, for
 * each layer l in order, w_l[3][3][C_in][C_out] (correlation taps) then
 * b_l[C_out], with C = 5, 32, 32, 32, 32, 32, 1. */
#define DV_CNN_IN_CH 5
typedef struct dv_cnn dv_cnn;

/* Fills *p with defaults: the paper's rho = 1 and outer/inner schedule shape,
 * lambda = 1e-3, delta = 1/60, gamma = 0.4, 30 x 10 iterations, one tile,
 * one PSF, FP32, automatic path, graphs on.  Pointers are set to NULL. */
void dv_problem_init(dv_problem* p);

/* Host-only: validates *prob and writes the y-block bounds the plan would use
 * (tile_r0/r1: n_tr entries, tile_c0/c1: n_tc entries) and the local step
 * sizes tau (n_tr * n_tc entries, row-major over tiles).  Any output may be NULL. */
dv_status dv_layout_query(const dv_problem* prob, int32_t* tile_r0, int32_t* tile_r1,
                          int32_t* tile_c0, int32_t* tile_c1, double* tau);

/* Builds a plan (Sec. III-A "distribute blocks, PSFs and weights"): validates
 * the problem, lays out the tile-stacked iterates x_i, u_i and residuals in
 * HBM, uploads PSFs, weight tables, consensus weights and noise weights, and
 * (DV_PATH_AUTO) times the operator paths.  Allocates all device workspace;
 * uses stream for uploads and synchronises it before returning.
 * Errors: DV_ERR_INVALID_ARG, DV_ERR_UNSUPPORTED, DV_ERR_OOM, DV_ERR_CUDA. */
dv_status dv_plan_create(const dv_problem* prob, void* stream, dv_plan** out);

/* y_dev [hy][wy] = H x_dev [(hy+K-1)][(wy+K-1)]: the global shift-variant
 * operator of Sec. II-B.  x_dev and y_dev must not alias. */
dv_status dv_apply_H(dv_plan* plan, const float* x_dev, float* y_dev, void* stream);

/* g_dev [(hy+K-1)][(wy+K-1)] = H^T r_dev [hy][wy], the adjoint of dv_apply_H
 * (<H x, r> = <x, H^T r>).  r_dev and g_dev must not alias. */
dv_status dv_apply_Ht(dv_plan* plan, const float* r_dev, float* g_dev, void* stream);

/* Algorithm 1 on the observed image y_dev [hy][wy]: starts from
 * x_i = u_i = C_i x0 with x0 = x0_dev [(hy+K-1)][(wy+K-1)] if given, else the
 * learned warm start (use_warmstart = 1, network attached with
 * dv_plan_set_warmstart), else y edge-replicated by K/2; runs the
 * outer/inner schedule of the problem and writes x_hat to x_out_dev
 * [(hy+K-1)][(wy+K-1)].  If stats is not NULL the call synchronises the stream
 * and fills it (one extra operator pass for the objective).  The plan keeps
 * the final x_i, u_i (see dv_state_export). */
dv_status dv_consensus_solve(dv_plan* plan, const float* y_dev, const float* x0_dev,
                             float* x_out_dev, dv_stats* stats, void* stream);

/* dv_consensus_solve from host buffers: copies y_host (and x0_host if not
 * NULL) to plan-owned device memory, solves, copies x_hat back to x_out_host,
 * and synchronises the stream before returning. */
dv_status dv_consensus_solve_host(dv_plan* plan, const float* y_host, const float* x0_host,
                                  float* x_out_host, dv_stats* stats, void* stream);

/* Continues Algorithm 1 for n_outer more outer iterations from the plan's
 * current x_i, u_i (after a solve or dv_state_import), with y_dev as data,
 * then writes x_hat.  Outer-iteration numbering (for inner_increment)
 * continues from the state's count. */
dv_status dv_consensus_continue(dv_plan* plan, const float* y_dev, int32_t n_outer,
                                float* x_out_dev, dv_stats* stats, void* stream);

/* Checkpoint / resume of the D-R state (x_i, u_i, k): copies the tile-stacked
 * iterates to / from caller device buffers of dv_plan_info().stack_elems
 * floats each (tile after tile, row pitch stack_pitch of each tile), plus the
 * number of outer iterations done. */
dv_status dv_state_export(dv_plan* plan, float* x_stack_dev, float* u_stack_dev,
                          int32_t* outer_done, void* stream);
dv_status dv_state_import(dv_plan* plan, const float* x_stack_dev, const float* u_stack_dev,
                          int32_t outer_done, void* stream);

typedef struct dv_plan_info {
  int32_t nx_r, nx_c;      /* x size */
  int32_t n_tiles;
  int32_t path;            /* dv_operator_path of the inner iterations (never AUTO) */
  int64_t stack_elems;     /* floats in one x-shaped tile stack */
  int64_t device_bytes;    /* device memory owned by the plan */
  double tau_min, tau_max; /* local step sizes */
  int64_t kernel_launches; /* total libdv kernel launches on this plan */
  double tune_ms_direct;   /* autotuner: one H + one H^T apply, direct path (0 if not timed) */
  double tune_ms_fft;      /* same for the block-FFT path (0 if not timed / not available) */
  /* work scheduled by one tile-mode launch of the path in use: output blocks
   * and (block, active PSF) pairs for H [0] and H^T [1]; the FFT path runs
   * ceil(PSFs/2) packed transforms per block (psf_pairs) */
  int64_t blocks[2];
  int64_t block_psfs[2];
  int64_t psf_pairs[2];
  int32_t block_side;      /* output block rows: 64 (direct), 128 - K + 1 (FFT), 128 (tensor) */
  int32_t fp32_path;       /* FP32 operator of objective evaluations: DV_PATH_DIRECT or _FFT */
  double tune_ms_tensor;   /* autotuner: tensor-core path (0 if not timed / not available) */
  /* BF16 tensor-core path: k-steps per PSF tap row one tile-mode launch of H
   * [0] and H^T [1] issues, summed over (block, PSF) pairs -- each k-step is
   * one 128 x rows x 16 MMA per tap row, so K times this is the MMA count.
   * Steps where a PSF's column weight is zero on the whole step are skipped.
   * 0 on the other paths. */
  int64_t mma_ksteps[2];
  /* tile groups whose inner iterations the captured local solve runs on
   * concurrent streams (tensor path with CUDA graphs; 1 = one launch per
   * operator over every tile) */
  int32_t tile_groups;
  /* 1 when H runs as the block DFT on the tensor cores (dv_problem.tensor_h) */
  int32_t tensor_h_dft;
  /* autotuner: one block-DFT H + one banded H^T (0 if not timed) */
  double tune_ms_tensor_dft;
  /* 1 when H^T runs as the block DFT too (dv_problem.tensor_h) */
  int32_t tensor_ht_dft;
  /* block-DFT H: forward transforms along rows per tile-mode launch, one per
   * (block, active PSF grid row) (0 without the block-DFT work tables) */
  int32_t dft_h_rows;
  /* autotuner: one block-DFT H + one block-DFT H^T (0 if not timed) */
  double tune_ms_tensor_dft2;
} dv_plan_info;

dv_status dv_plan_get_info(const dv_plan* plan, dv_plan_info* info);

/* Per-kernel CUDA-event timing of the solve's launches (off by default).
 * kind: 0 = operator H with residual, 1 = operator H^T with fused prox step,
 * 2 = consensus + dual update, 3 = one whole local solve (n_inner x {H, H^T}
 * over every tile) when the captured local solve runs its tile groups
 * concurrently (dv_plan_info.tile_groups > 1; kinds 0 and 1 then see only
 * eager launches).  Reports the summed duration (ms) and the number of timed
 * launches (local solves for kind 3) since the last reset;
 * dv_consensus_solve must have returned (stats or a synchronised stream)
 * before reading. */
dv_status dv_plan_set_timing(dv_plan* plan, int32_t enable);
dv_status dv_plan_kernel_time(dv_plan* plan, int32_t kind, double* total_ms, int64_t* launches);

/* Bound, in seconds, of every pipeline wait (mbarrier) of the BF16
 * tensor-core operator kernels this plan launches from now on; 0 restores the
 * default of 2 s, at most 60.  A wait that runs out sets the plan's device
 * error word and makes every role of its CTA stop, wait (bounded) for the
 * copies and MMAs it issued, free its tensor memory and return, so the context
 * stays usable; the next call that synchronises (a solve with stats or
 * objective checks, a host-buffer solve) returns DV_ERR_TIMEOUT, after which
 * only dv_destroy is valid.  Drops the plan's captured CUDA graphs (they are
 * captured again with the new bound) and synchronises the device. */
dv_status dv_plan_set_wait_limit(dv_plan* plan, double seconds);

/* Test of that failure path, with no GPU fault, trap or hang: with
 * withhold = 1 the BF16 tensor-core kernels of this plan issue none of their
 * operand copies, so the first ring wait of every CTA's MMA lane runs out
 * (after the wait limit) with no copy or MMA in flight and the solve reports
 * DV_ERR_TIMEOUT; 0 turns it off.  Drops the captured graphs and synchronises
 * the device, like dv_plan_set_wait_limit. */
dv_status dv_plan_set_wait_test(dv_plan* plan, int32_t withhold);

/* Allocation-free Huber prior value (the paper has no counterpart; this is a
 * service for callers that may not allocate device memory, such as plug-ins
 * running inside a host framework that owns all device memory, or real-time
 * loops where a cudaMalloc could stall the device).  Writes to value_dev[0]
 * (device, one double) the FP64 sum over the rows x cols image x_dev of
 * hub_delta(|grad x|) with forward differences set to zero on the last row and
 * column -- the prior term phi(D x) of dv_stats for a one-tile plan.  Needs no
 * plan and allocates nothing: its per-block partial sums live in a static
 * device array of DV_NOALLOC_MAX_BLOCKS doubles (512 KiB) that every GPU
 * loading libdv keeps until the process exits.  One partial is used per row
 * and 256 columns, so rows * ceil(cols / 256) must not exceed
 * DV_NOALLOC_MAX_BLOCKS and rows must not exceed 65535; larger images are
 * rejected with DV_ERR_INVALID_ARG.  The first call on each device looks up
 * the array's device address (no allocation of its own); under CUDA's lazy
 * module loading that first call also loads this part of the library onto the
 * device, which places the array and the kernels in device memory, so make it
 * before a host framework reserves the device memory it manages, and before
 * any stream capture.  All calls share the array, so calls whose work overlaps
 * on the GPU (different streams, no ordering) race and give wrong sums; calls
 * ordered on one stream are safe.  Runs on the calling thread's current device
 * (x_dev and value_dev must be on it).  Enqueued on stream; returns without
 * synchronising. */
#define DV_NOALLOC_MAX_BLOCKS 65536
dv_status dv_prior_value_noalloc(const float* x_dev, int32_t rows, int32_t cols, double delta,
                                 double* value_dev, void* stream);

/* Image quality of x against a reference image, the measures of the
 * paper's evaluation (Sec. IV-C) on synthetic stand-ins: out_dev[0] = SNR =
 * 10 log10(sum ref^2 / sum (x - ref)^2) dB over all pixels (+inf if x == ref),
 * out_dev[1] = the mean structural similarity (Wang et al. 2004) over every
 * 11 x 11 window inside the image: separable unit-sum Gaussian window of
 * standard deviation 1.5, C1 = (0.01 L)^2, C2 = (0.03 L)^2 with
 * L = dynamic_range; local moments in FP32, sums in FP64 in a fixed order
 * (deterministic).  x_dev, ref_dev: device float32 [rows][cols], rows and
 * cols >= 11; work_dev: device scratch of dv_image_quality_workspace(rows,
 * cols) doubles; out_dev: device, two doubles.  Stream-ordered: no
 * allocation, no synchronisation. */
int64_t dv_image_quality_workspace(int32_t rows, int32_t cols);
dv_status dv_image_quality(const float* x_dev, const float* ref_dev, int32_t rows, int32_t cols,
                           double dynamic_range, double* work_dev, double* out_dev, void* stream);

/* Creates the warm-start network (width 32, depth 6 are the only supported
 * values) with He-normal weights drawn from seed; synchronises stream. */
dv_status dv_cnn_create(int32_t width, int32_t depth, uint64_t seed, void* stream, dv_cnn** out);
int64_t dv_cnn_param_count(const dv_cnn* cnn);
/* float32 parameters to / from host memory (n = dv_cnn_param_count); set also
 * resets the Adam state.  get also returns the number of training steps. */
dv_status dv_cnn_get_params(const dv_cnn* cnn, float* host, int64_t n, int64_t* step);
dv_status dv_cnn_set_params(dv_cnn* cnn, const float* host, int64_t n, void* stream);
/* out_dev [N][H][W] = network(in_dev [N][H][W][5]) (zero padding at the borders). */
dv_status dv_cnn_forward(dv_cnn* cnn, const float* in_dev, int32_t N, int32_t H, int32_t W,
                         float* out_dev, void* stream);
/* Loss 1/2 mean((out - target)^2) and its gradient (float32, parameter layout)
 * for one batch, without updating; synchronises stream. */
dv_status dv_cnn_gradients(dv_cnn* cnn, const float* in_dev, const float* target_dev, int32_t N,
                           int32_t H, int32_t W, float* grad_host, double* loss_host, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on one
 * batch; loss_host (optional) receives the loss before the step (synchronises). */
dv_status dv_cnn_train_step(dv_cnn* cnn, const float* in_dev, const float* target_dev, int32_t N,
                            int32_t H, int32_t W, float lr, double* loss_host, void* stream);
/* n_steps Adam steps on crops of a stack of training pairs, queued on stream
 * without host synchronisation between steps.  Step t trains on the batch of
 * the `batch` crops crops_host[t][b] = {pair, r0, c0} (host, int32), each
 * crop x crop pixels of feats_dev [n_pairs][H][W][5] and targets_dev
 * [n_pairs][H][W] (device, float32), with learning rate lr_host[t] (host).
 * The same as n_steps calls of dv_cnn_train_step on the gathered crops, bit
 * for bit.  losses_host (optional, n_steps doubles) receives each step's loss
 * before its update.  Synchronises stream once, at the end.  A crop outside
 * its pair or a pair index out of range: DV_ERR_INVALID_ARG before any work.
 * Allocates (and frees) device memory for the crop table and one batch. */
dv_status dv_cnn_train_crops(dv_cnn* cnn, const float* feats_dev, const float* targets_dev,
                             int32_t n_pairs, int32_t H, int32_t W, const int32_t* crops_host,
                             int32_t n_steps, int32_t batch, int32_t crop, const float* lr_host,
                             double* losses_host, void* stream);
dv_status dv_cnn_destroy(dv_cnn* cnn);
/* Attaches a network to the plan (borrowed; keep it alive while the plan
 * uses it).  With use_warmstart = 1 and no x0, dv_consensus_solve starts from
 * the network's x0. */
dv_status dv_plan_set_warmstart(dv_plan* plan, dv_cnn* cnn);
/* feat_dev [(hy+K-1)][(wy+K-1)][5] = the warm-start features of y_dev. */
dv_status dv_warmstart_features(dv_plan* plan, const float* y_dev, float* feat_dev, void* stream);

/* Releases everything the plan owns.  NULL is accepted. */
dv_status dv_destroy(dv_plan* plan);

/* Message of the calling thread's last failure ("" if none).  Valid until the
 * thread's next libdv call. */
const char* dv_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DV_H */
