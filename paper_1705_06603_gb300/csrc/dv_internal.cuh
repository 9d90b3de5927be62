// Internal declarations of libdv: device-side descriptors, the plan object and
// the kernel launchers shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dv.h"

namespace dv {

// ---------------------------------------------------------------------------
// Error reporting (thread-local message behind dv_last_error)
// ---------------------------------------------------------------------------
dv_status fail(dv_status code, const char* fmt, ...);
void clear_error();
dv_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define DV_TRY_CUDA(call)                                                     \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) return ::dv::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define DV_TRY(call)                         \
  do {                                       \
    dv_status s_ = (call);                   \
    if (s_ != DV_OK) return s_;              \
  } while (0)

// ---------------------------------------------------------------------------
// Device descriptors
// ---------------------------------------------------------------------------

// One tile: its y-block (global y coordinates) equals the origin of its x-tile
// in global x coordinates; the x-tile is the y-block grown by K - 1.
struct TileDesc {
  int32_t xr0, xc0;      // x-tile origin (global x) == y-block origin (global y)
  int32_t nyr, nyc;      // y-block extent
  int32_t nxr, nxc;      // x-tile extent (nyr + K - 1, nyc + K - 1)
  int32_t xpitch, ypitch;  // row pitch (floats) in x-shaped / y-shaped stacks
  int64_t xoff, yoff;    // element offset of (0,0) in x-shaped / y-shaped stacks
  int32_t omr_off, omc_off;  // offsets of this tile's consensus profiles
  int32_t tr, tc;
  float tau;             // local projected-gradient step
  int32_t wr0, wc0;      // index of x-tile row / column 0 in the weight tables
  int32_t pad;
};
static_assert(sizeof(TileDesc) == 80, "TileDesc layout");

// One CTA's output block of the direct operator kernels.
struct WorkItem {
  int32_t tile;          // tile index
  int32_t r0, c0;        // output block origin (tile-local: y coords for H, x for H^T)
  int32_t pad;
  int32_t a_lo, a_hi;    // active PSF grid rows  (inclusive)
  int32_t b_lo, b_hi;    // active PSF grid cols  (inclusive)
};
static_assert(sizeof(WorkItem) == 32, "WorkItem layout");

// Interpolation weights at one global x coordinate: grid index a0 has weight
// w0 and a0 + 1 has weight w1; every other grid index has weight 0.
struct WTab {
  int32_t a0;
  float w0, w1;
  int32_t pad;
};

__host__ __device__ inline float wsel(const WTab& t, int a) {
  return a == t.a0 ? t.w0 : (a == t.a0 + 1 ? t.w1 : 0.0f);
}

// Operator kernel modes
enum OpMode : int32_t {
  OP_PLAIN = 0,   // write H x (or H^T r) to a global image
  OP_RESID = 1,   // H: write r = W (H x - y) into the residual stack
  OP_OBJ = 2,     // H: FP64 partial of sum W (H x - y)^2, no write
  OP_STEP = 3     // H^T: fused projected-gradient step into w_next
};

// BF16 tensor-core path: PSF grid columns per work item with a k-step range
// of their own (further columns run every k-step)
constexpr int kTcMaxB = 16;

// Tile groups of the captured local solve: each group's H / H^T chain runs
// on a stream of its own, so one group's blocks fill the SMs another group's
// last blocks leave idle (the tiles are independent between consensus steps)
constexpr int kMaxGroups = 4;

struct OpArgs {
  const TileDesc* tiles;
  const WorkItem* work;
  int32_t n_work;
  int32_t mode;
  const WTab* wrow;
  const WTab* wcol;
  const float* psf;       // [Gr*Gc][K][KP]: flipped (H) or as given (H^T)
  int32_t Gc, K, KP;
  int32_t pad0;
  const float* in;        // x-shaped (H) or y-shaped (H^T) input base
  float* out;             // output base
  // H, OP_RESID / OP_OBJ: global observed image and noise weights (pitch wy)
  const float* y;
  const float* W;         // nullable
  int32_t wy;
  int32_t pad1;
  double* partials;       // OP_OBJ: one double per work item
  // H^T, OP_STEP: current iterate, dual variable, consensus profiles, prior
  const float* w;
  const float* u;
  const float* omr;
  const float* omc;
  float lambda, delta, gamma;
  int32_t pad2;
  const float2* spec;     // FFT path: [Gr*Gc][S][S] PSF spectra / S^2
  int* counter;           // FFT path: work counter, zeroed before each launch
  float2* scratch;        // FFT path: one S x S spectrum per CTA of the launch grid
  const unsigned char* tcop;  // tensor-core path: tall B operands [G][K] (shared-memory images)
  int32_t prec;           // tensor-core path: DV_PREC_BF16 or DV_PREC_TF32
  int32_t pad3;
  int* err;               // tensor-core path: nonzero after a bounded wait gave up
  const uint16_t* ksr;    // BF16 tensor-core path: [n_work][kTcMaxB] k-step ranges (lo | hi << 8)
  uint64_t wait_ns;       // BF16 tensor-core path: bound of a pipeline wait (0: 2 s)
  int32_t test_withhold;  // BF16 tensor-core path: issue no operand copy (dv_plan_set_test_fault)
  int32_t ctas;           // persistent kernels: CTAs of the launch (0: one per SM)
};

// One item of the consensus / assembly kernels: a rectangle of the global x
// grid (at most 2048 pixels, at most 512 columns wide) over which the covering tiles do not
// change, with per covering tile ("slot", tile rows outer, tile columns
// inner): the stack offset of (r0, global column 0), the row pitch, and the
// indices of global row 0 / column 0 in the consensus profiles.
struct ConsItem {
  int32_t r0, nrow, c0, ncol;
  int32_t ns, pad[3];
  int64_t base[4];
  int32_t pitch[4];
  int32_t obr[4];
  int32_t obc[4];
};
static_assert(sizeof(ConsItem) == 112, "ConsItem layout");

// Streaming kernels' shared view of the tile grid
struct GridArgs {
  const TileDesc* tiles;
  const int2* rowcov;     // per global x row: covering tile rows (second = -1 if none)
  const int2* colcov;     // per global x column: covering tile columns
  const float* omr;
  const float* omc;
  int32_t n_tc;
  int32_t nxr, nxc;
  int32_t n_citems;
  const ConsItem* citems;
};

// ---------------------------------------------------------------------------
// Launchers (stream-ordered; return cudaGetLastError of the launch)
// ---------------------------------------------------------------------------
cudaError_t launch_direct_H(const OpArgs& a, cudaStream_t s);
cudaError_t launch_direct_Ht(const OpArgs& a, cudaStream_t s);
int direct_tile_m();   // output block rows of the direct kernels
int direct_tile_n();   // output block cols

// start / gather: tile stacks from a global x image (x0 = NULL: y edge-padded);
// zg (nullable) also receives the global start image
cudaError_t launch_scatter(const GridArgs& g, int n_tiles, int max_nxr, int max_nxc,
                           const float* x0, const float* y, int hy, int wy, int rad,
                           float* w, float* u, cudaStream_t s, float* zg);
// consensus + dual update (Lemma 1, Sec. III-B); zbuf (nullable) holds the
// previous zbar and receives the new one; partials (nullable): 2 x n_blocks
cudaError_t launch_consensus(const GridArgs& g, const float* x, float* u, float gamma,
                             float rho, float* zbuf, double* partials, cudaStream_t s,
                             int* n_blocks_out);
int consensus_blocks(int n_citems);
// rows / columns of the largest consensus item
int cons_item_pixels();
int cons_item_cols();
// x_hat = sum omega_i x_i / sum omega_i
cudaError_t launch_assemble(const GridArgs& g, const float* x, float* out, cudaStream_t s);
// FP64 block partials of the Huber prior over the tile stacks
int huber_blocks(int n_tiles, int max_nxr, int max_nxc);
cudaError_t launch_huber_value(const TileDesc* tiles, int n_tiles, int max_nxr, int max_nxc,
                               const float* x, double delta, double* partials, cudaStream_t s);
// out[k] = sum_{i < counts[k]} parts[k][i] in a fixed order (one block), nk <= 8
cudaError_t launch_reduce(const double* const* parts, const int* counts, int nk, double* out,
                          cudaStream_t s);
size_t direct_smem_bytes(int K);
cudaError_t direct_prepare(int K);   // shared-memory limits of the direct kernels

// Block-FFT path (overlap-save, S = 128)
int fft_size();
int fft_block(int K);                 // valid outputs per block side, S - K + 1
bool fft_supported(int K);
cudaError_t fft_prepare();            // twiddles + shared-memory limits (plan time)
void fft_spectra(const float* psfs, int G, int K, std::vector<float2>& out);
cudaError_t launch_fft_H(const OpArgs& a, cudaStream_t s, int grid);
cudaError_t launch_fft_Ht(const OpArgs& a, cudaStream_t s, int grid);

// Block DFT of H on the tensor cores (FP16 operands; the FFT path's work tables)
bool dft_supported(int K);
cudaError_t dft_prepare();
void dft_constants(std::vector<uint8_t>& out);
void dft_spectra(const float* psfs, int G, int K, std::vector<uint32_t>& out);
cudaError_t launch_dft_H(const OpArgs& a, cudaStream_t s, int grid);
cudaError_t launch_dft_Ht(const OpArgs& a, cudaStream_t s, int grid);
int dft_Ht_kernels(int mode);   // kernels one block-DFT H^T launch runs

// Tensor-core path (tcgen05, BF16 / TF32 operands; its own work tables)
int tc_block_m();
int tc_block_n();
bool tc_supported(int K);
cudaError_t tc_prepare(int K, int prec);
void tc_operands(const float* psfs, int G, int K, int prec, bool flip, std::vector<uint8_t>& out);
cudaError_t launch_tc_H(const OpArgs& a, cudaStream_t s);
cudaError_t launch_tc_Ht(const OpArgs& a, cudaStream_t s);
// BF16 tensor-core path in the column-band layout: 128 output columns per
// block, up to tcT_max_rows(K) output rows (WorkItem.pad = the block's rows,
// a multiple of 16)
int tcT_block_cols();
int tcT_max_rows(int K);
cudaError_t tcT_prepare(int K);
void tcT_operands(const float* psfs, int G, int K, bool flip, std::vector<uint8_t>& out);
// k-step ranges of the items of one work table (kTcMaxB entries per item,
// lo | hi << 8); returns the k-steps per tap row summed over (item, PSF)
int64_t tcT_kstep_ranges(const std::vector<TileDesc>& tiles, const std::vector<WorkItem>& items,
                         const std::vector<WTab>& wcol, int K, bool adjoint,
                         std::vector<uint16_t>& out);
cudaError_t launch_tcT_H(const OpArgs& a, cudaStream_t s);
cudaError_t launch_tcT_Ht(const OpArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
// One captured outer iteration of Algorithm 1: the local solve (n_inner
// projected-gradient steps on all tiles), the consensus and dual update and,
// when due, the kernels and read-back of the FP64 objective reduction;
// replayed once per outer iteration.  With timing on, the timed units (every
// operator kernel, or the whole local solve when its tile groups run
// concurrently, and the consensus kernel) are bracketed by event-record nodes
// whose events are swapped before each launch.
struct GraphEntry {
  int n_inner = 0;
  int parity = 0;          // w buffer holding x_i when the local solve starts
  bool timed = false;
  int cons = 0;            // 0: local solve only; 1: + consensus; bit 1: zbar tracked;
                           // bit 2: residual partials; bit 3: objective reduction
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaGraphNode_t> ev_start, ev_end;  // per kernel node (timed only)
  std::vector<int> kinds;
};

struct Pending {
  int kind;
  int ev0, ev1;            // indices into the event pool
};

struct KernelTimer {
  std::vector<cudaEvent_t> pool;
  std::vector<cudaEvent_t> placeholders;
  std::vector<Pending> pending;
  size_t next = 0;
  double total_ms[4] = {0, 0, 0, 0};
  int64_t count[4] = {0, 0, 0, 0};
};

}  // namespace dv

namespace dv {
// Work tables of one operator path: tile mode (H over y-blocks, H^T over
// x-tiles) and the single global pseudo-tile of dv_apply_H / dv_apply_Ht.
struct OpTables {
  int64_t psfs[2] = {0, 0};    // sum over H / H^T items of active PSFs
  int64_t pairs[2] = {0, 0};   // sum of ceil(active PSFs / 2)
  int64_t rows[2] = {0, 0};    // sum over H / H^T items of active PSF grid rows
  WorkItem* H = nullptr;
  WorkItem* Ht = nullptr;
  WorkItem* Hg = nullptr;
  WorkItem* Htg = nullptr;
  int nH = 0, nHt = 0, nHg = 0, nHtg = 0;
  // BF16 tensor-core path: per-item k-step ranges and the k-steps one
  // tile-mode launch runs per tap row, summed over (block, PSF) pairs
  uint16_t* ksH = nullptr;
  uint16_t* ksHt = nullptr;
  uint16_t* ksHg = nullptr;
  uint16_t* ksHtg = nullptr;
  int64_t ksteps[2] = {0, 0};
  // host copy of the tile of every tile-mode H item (per-tile sums of its partials)
  std::vector<int32_t> tileH;
  // tile-mode items grouped by tile group: group g owns items [gH[g], gH[g + 1])
  int gH[kMaxGroups + 1] = {};
  int gHt[kMaxGroups + 1] = {};
};
}  // namespace dv

struct dv_plan {
  dv_problem prob;        // copy with host pointers cleared
  int hy, wy, K, rad, Gr, Gc, nxr, nxc, n_tr, n_tc, T;
  int path;               // operator of the inner iterations: DV_PATH_DIRECT, _FFT or _TENSOR
  int fpath;              // FP32 operator (objective, stopping test): DV_PATH_DIRECT or _FFT
  bool tensor_ok = false;  // tensor-core tables and operands were built
  dv::OpTables tab[3];    // [0] direct 64x64, [1] FFT b x b, [2] tensor 128x64 blocks
  bool fft_ok = false;
  bool dft_ok = false;             // H as the block DFT on the tensor cores is available
  bool dft_H = false;              // ... and used by the tensor path
  bool dft_Ht = false;             // H^T as the block DFT on the tensor path
  uint32_t* d_dspec = nullptr;     // its PSF spectra [G][128][128] (FP16 pairs), natural order, / 128
  unsigned char* d_dconst = nullptr;  // its constant operand [Fr; Fi] (FP16 panels)
  int* d_dcounter = nullptr;       // its work counters: [0] whole launches, [1 + g] group g
  float2* d_spec = nullptr;
  int* d_counter = nullptr;        // [0] H launches, [1] H^T launches (FFT path)
  float2* d_fft_scr = nullptr;     // FFT path: n_sm spectra of S x S
  int n_sm = 0;
  unsigned char* d_tcopH = nullptr;   // tensor-core B operands (flipped PSFs, for H)
  unsigned char* d_tcopHt = nullptr;  // tensor-core B operands (PSFs, for H^T)
  int* d_err = nullptr;               // device error word of the tensor-core kernels
  uint64_t wait_ns = 0;               // bound of the BF16 tensor kernels' waits (0: 2 s)
  int test_fault = 0;                 // dv_plan_set_test_fault kind
  double tune_ms[3] = {0.0, 0.0, 0.0};  // autotuner: one H + one H^T apply per path
  double tune_ms_dft = 0.0;             // ... tensor path with H as the block DFT
  double tune_ms_dft2 = 0.0;            // ... tensor path with H and H^T as block DFTs
  dv_cnn* cnn = nullptr;           // warm-start network (borrowed)
  float* d_desc = nullptr;         // per-PSF descriptors [G][3]
  float* d_feat = nullptr;         // warm-start features [nx][5] (lazy)
  float* d_wsd = nullptr;          // network output on the x grid (lazy)
  std::vector<int> yr0, yr1, yc0, yc1;
  std::vector<double> tau;
  std::vector<dv::TileDesc> h_tiles;
  int max_nxr, max_nxc;
  int64_t xstack, ystack;
  // device data
  float* d_psf_flip = nullptr;
  float* d_psf = nullptr;
  dv::WTab* d_wrow = nullptr;
  dv::WTab* d_wcol = nullptr;
  float* d_omr = nullptr;
  float* d_omc = nullptr;
  dv::TileDesc* d_tiles = nullptr;
  dv::TileDesc* d_gtile = nullptr;
  int2* d_rowcov = nullptr;
  int2* d_colcov = nullptr;
  dv::ConsItem* d_citems = nullptr;
  int n_citems = 0;
  float* d_w[2] = {nullptr, nullptr};
  float* d_u = nullptr;
  float* d_r = nullptr;
  float* d_y = nullptr;
  float* d_W = nullptr;
  float* d_z = nullptr;        // previous zbar (global x image)
  float* d_xg = nullptr;       // x_hat (global x image)
  double* d_part = nullptr;
  int64_t n_part = 0;
  double* d_scal = nullptr;
  double* h_scal = nullptr;    // pinned
  float* d_hx = nullptr;       // host-solve staging (x-sized), lazily allocated
  float* d_hy = nullptr;       // host-solve staging (y-sized)
  float* d_hx0 = nullptr;
  int64_t device_bytes = 0;
  int cur = 0;                 // w buffer holding x_i
  int outer_done = 0;
  int64_t launches = 0;
  bool timing = false;
  dv::KernelTimer timer;
  std::vector<dv::GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  int ngrp = 1;                       // tile groups of the captured local solve
  cudaStream_t grp_stream[dv::kMaxGroups] = {};
  cudaEvent_t grp_fork = nullptr, grp_join[dv::kMaxGroups] = {};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // VMLM-B Local-Solver (dv_problem.local_solver = DV_SOLVER_VMLMB), lazy
  int vm_m = 5;                          // memory pairs
  // Armijo trial counts of the current call (reset by the solve entry points)
  int64_t vm_iters = 0;                  // batched VMLM-B iterations run
  int64_t vm_trials = 0;                 // sum over iterations of the trials run
  int64_t vm_tile_iters = 0;             // (tile, iteration) pairs that searched
  int64_t vm_tile_trials = 0;            // their trials
  int vm_trials_max = 0;
  int vm_stops = 0;                      // (tile, local solve) pairs ended by vm_stop_rel
  float* d_vg = nullptr;                 // gradient at the iterate
  float* d_vgt = nullptr;                // gradient at the new iterate
  float* d_vd = nullptr;                 // search direction
  float* d_vq = nullptr;                 // two-loop work vector
  float* d_vht = nullptr;                // H_i^T r
  float* d_vs = nullptr;                 // [m] pairs s
  float* d_vy = nullptr;                 // [m] pairs y
  double* d_vpart = nullptr;             // [4] segments of per (tile, row chunk) partials
  double* d_vhub = nullptr;              // Huber partials per (tile, row block)
  float* d_vcoef = nullptr;              // ring of per-tile coefficient slots
  float* h_vcoef = nullptr;              // pinned staging of the ring
  double* h_vpart = nullptr;             // pinned landing of downloaded partials
  int64_t h_vpart_cap = 0;               // doubles in h_vpart
};

namespace dv {
// Named host range of one phase (solve, local solve, consensus, objective,
// warm start, plan, training) for profiler timelines; NVTX without an
// attached tool costs a few nanoseconds.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

dv_status warmstart_x0(dv_plan* P, cudaStream_t s, float* x0);
// VMLM-B Local-Solver: n_iter iterations on every tile (the projected-gradient
// solver's buffer convention: d_w[cur] in, d_w[cur ^ (n_iter & 1)] out)
dv_status vmlmb_local_solve(dv_plan* P, int n_iter, cudaStream_t s);
int tab_index_of(int path);
void psf_descriptors(const float* psfs, int G, int K, std::vector<float>& out);
// Operator launches on one path (DV_PATH_DIRECT, _FFT or _TENSOR; the args
// must come from op_args_* of the same path).  The H launch in OP_OBJ mode
// (FP32 paths) writes obj_parts(P) FP64 partials.
cudaError_t launch_op_H(const dv_plan* P, int path, const OpArgs& a, cudaStream_t s);
cudaError_t launch_op_Ht(const dv_plan* P, int path, const OpArgs& a, cudaStream_t s);
int obj_parts(const dv_plan* P);
dv::OpArgs op_args_H(const dv_plan* p, int path, int mode, const float* in, float* out, bool global);
dv::OpArgs op_args_Ht(const dv_plan* p, int path, int mode, const float* in, float* out,
                      bool global, const float* w, const float* u);
dv::GridArgs grid_args(const dv_plan* p);
// the tile-mode arguments restricted to the items of tile group g
dv::OpArgs group_args(const dv_plan* p, int path, dv::OpArgs a, bool adjoint, int g);
}  // namespace dv
