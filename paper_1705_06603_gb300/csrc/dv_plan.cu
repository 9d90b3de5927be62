// Plan construction for libdv: validation of the problem, tile layout
// (Sec. III-A, III-C), first-order interpolation weight tables (Sec. II-B),
// consensus weights omega_i and metric alpha_i = gamma omega_i (Sec. III-B),
// local step sizes, operator work tables and the HBM layout of the tile
// stacks.  Host code; every device buffer the plan uses is allocated here.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "dv_internal.cuh"

namespace dv {

static thread_local std::string g_err;

dv_status fail(dv_status code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

void clear_error() { g_err.clear(); }

dv_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  const dv_status code = (e == cudaErrorMemoryAllocation) ? DV_ERR_OOM : DV_ERR_CUDA;
  return fail(code, "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

namespace {

constexpr int kMaxK = 127;
constexpr int kMaxTileGrid = 1024;   // row kernels stage one tile row pair per block in shared memory
constexpr int kMaxRows = 65535;      // grid.y of the row kernels is one x row

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Equal blocks of B = ceil((n + (count-1) overlap) / count) pixels, block i
// starting at round(i (n - B) / (count - 1)).
void uniform_blocks(int n, int count, int overlap, std::vector<int>& s, std::vector<int>& e) {
  s.assign(count, 0);
  e.assign(count, n);
  if (count == 1) return;
  int64_t B = ((int64_t)n + (int64_t)(count - 1) * overlap + count - 1) / count;
  if (B > n) B = n;
  for (int i = 0; i < count; ++i) {
    const int64_t st = ((int64_t)i * (n - B) + (count - 1) / 2) / (count - 1);
    s[i] = (int)st;
    e[i] = (int)(st + B);
  }
}

dv_status check_blocks(const char* axis, int n, int K, const std::vector<int>& s,
                       const std::vector<int>& e) {
  const int cnt = (int)s.size();
  if (s[0] != 0 || e[cnt - 1] != n)
    return fail(DV_ERR_INVALID_ARG, "%s y-blocks must start at 0 and end at %d", axis, n);
  for (int i = 0; i < cnt; ++i) {
    if (s[i] < 0 || e[i] > n || s[i] >= e[i])
      return fail(DV_ERR_INVALID_ARG, "%s y-block %d = [%d, %d) is empty or out of range", axis,
                  i, s[i], e[i]);
    if (i + 1 < cnt) {
      if (s[i + 1] <= s[i] || e[i + 1] <= e[i])
        return fail(DV_ERR_INVALID_ARG, "%s y-blocks must be sorted", axis);
      if (s[i + 1] > e[i])
        return fail(DV_ERR_INVALID_ARG, "%s y-blocks %d and %d leave a gap", axis, i, i + 1);
    }
    // x-tile i = [s_i, e_i + K - 1); tile i + 2 must not reach into tile i
    if (i + 2 < cnt && s[i + 2] < e[i] + K - 1)
      return fail(DV_ERR_INVALID_ARG,
                  "%s x-tiles %d and %d overlap: each x-tile may only overlap its neighbours",
                  axis, i, i + 2);
  }
  return DV_OK;
}

// Per-tile 1-D consensus profiles on x-ranges [xs_i, xe_i): 1 where no other
// tile reaches, ramps (j + 1/2)/B across each band of width B shared with a
// neighbour, normalised so that the profiles sum to 1 at every coordinate.
std::vector<std::vector<double>> consensus_profiles(const std::vector<int>& xs,
                                                    const std::vector<int>& xe) {
  const int cnt = (int)xs.size();
  std::vector<std::vector<double>> t(cnt);
  for (int i = 0; i < cnt; ++i) t[i].assign(xe[i] - xs[i], 1.0);
  for (int i = 0; i + 1 < cnt; ++i) {
    const int B = xe[i] - xs[i + 1];
    for (int j = 0; j < B; ++j) {
      const double up = (j + 0.5) / B;
      t[i + 1][j] *= up;
      t[i][xs[i + 1] - xs[i] + j] *= 1.0 - up;
    }
  }
  std::vector<double> tot(xe[cnt - 1], 0.0);
  for (int i = 0; i < cnt; ++i)
    for (int j = 0; j < xe[i] - xs[i]; ++j) tot[xs[i] + j] += t[i][j];
  for (int i = 0; i < cnt; ++i)
    for (int j = 0; j < xe[i] - xs[i]; ++j) t[i][j] /= tot[xs[i] + j];
  return t;
}

// Interpolation weight table of one axis (n coordinates, G grid points).
dv_status weight_table(const char* axis, int n, int G, const float* prof, std::vector<WTab>& tab) {
  tab.assign(n, WTab{0, 0.f, 0.f, 0});
  if (!prof) {
    if (G == 1) {
      for (int t = 0; t < n; ++t) tab[t] = WTab{0, 1.f, 0.f, 0};
      return DV_OK;
    }
    const double D = (n - 1.0) / (G - 1.0);
    for (int t = 0; t < n; ++t) {
      int a0 = (int)std::floor(t / D);
      a0 = std::min(std::max(a0, 0), G - 2);
      const double w0 = std::max(0.0, 1.0 - std::fabs(t - a0 * D) / D);
      const double w1 = std::max(0.0, 1.0 - std::fabs(t - (a0 + 1) * D) / D);
      tab[t] = WTab{a0, (float)w0, (float)w1, 0};
    }
    return DV_OK;
  }
  for (int t = 0; t < n; ++t) {
    int first = -1, last = -1, cnt = 0;
    for (int a = 0; a < G; ++a) {
      const float v = prof[(size_t)a * n + t];
      if (!(v >= 0.f) || !std::isfinite(v))
        return fail(DV_ERR_INVALID_ARG, "%s weights must be finite and >= 0 (grid %d, t=%d)",
                    axis, a, t);
      if (v != 0.f) {
        if (first < 0) first = a;
        last = a;
        ++cnt;
      }
    }
    if (cnt > 2 || (cnt == 2 && last != first + 1))
      return fail(DV_ERR_INVALID_ARG,
                  "%s weights at coordinate %d: at most two neighbouring grid points may be "
                  "nonzero (first-order interpolation)", axis, t);
    if (cnt == 0) continue;
    int a0 = first;
    if (G == 1) a0 = 0;
    else if (a0 > G - 2) a0 = G - 2;
    tab[t] = WTab{a0, prof[(size_t)a0 * n + t], G > 1 ? prof[(size_t)(a0 + 1) * n + t] : 0.f, 0};
  }
  return DV_OK;
}

// Grid indices with a nonzero weight somewhere in [lo, hi).
void active_range(const std::vector<WTab>& tab, int lo, int hi, int& amin, int& amax) {
  amin = INT_MAX;
  amax = -1;
  for (int t = lo; t < hi; ++t) {
    if (tab[t].w0 != 0.f) {
      amin = std::min(amin, tab[t].a0);
      amax = std::max(amax, tab[t].a0);
    }
    if (tab[t].w1 != 0.f) {
      amin = std::min(amin, tab[t].a0 + 1);
      amax = std::max(amax, tab[t].a0 + 1);
    }
  }
  if (amax < 0) {
    amin = 0;
    amax = -1;
  }
}

struct Layout {
  std::vector<int> yr0, yr1, yc0, yc1;
  std::vector<std::vector<double>> omr, omc;
  // weight tables: the global x grid first, then (one PSF per tile) one table
  // per tile row / column; wr0[tr] / wc0[tc] = index of the tile's x row /
  // column 0 in them
  std::vector<WTab> wrow, wcol;
  std::vector<int> wr0, wc0;
  std::vector<double> tau;
};

// The paper's blocks on one axis (Sec. III-C) for one PSF per block: G equal
// cells of the x axis (n = ny + K - 1 coordinates), x-tile i spanning cells
// i - 1 .. i + 1, i.e. [(2i - 1) n / 2G, (2i + 3) n / 2G) clipped to [0, n);
// y-block i = the x-tile less K - 1 coordinates at its end.
void grid_blocks(int ny, int K, int G, std::vector<int>& s, std::vector<int>& e) {
  const int64_t n = (int64_t)ny + K - 1;
  s.assign(G, 0);
  e.assign(G, ny);
  for (int i = 0; i < G; ++i) {
    const int64_t x0 = std::max<int64_t>(0, (2 * (int64_t)i - 1) * n / (2 * G));
    const int64_t x1 = std::min<int64_t>(n, (2 * (int64_t)i + 3) * n / (2 * G));
    s[i] = (int)x0;
    e[i] = i == G - 1 ? ny : (int)(x1 - (K - 1));
  }
}

// One table per tile row (or column): every coordinate of the x-tile gives
// weight 1 to the tile's own PSF row (column) and 0 to the others.
void tile_tables(const std::vector<int>& y0, const std::vector<int>& y1, int K,
                 std::vector<WTab>& tab, std::vector<int>& off) {
  off.resize(y0.size());
  for (size_t t = 0; t < y0.size(); ++t) {
    off[t] = (int)tab.size();
    for (int c = 0; c < y1[t] - y0[t] + K - 1; ++c) tab.push_back(WTab{(int)t, 1.f, 0.f, 0});
  }
}

dv_status validate_and_layout(const dv_problem* p, Layout& L) {
  if (!p) return fail(DV_ERR_INVALID_ARG, "problem is NULL");
  if (p->hy < 1 || p->wy < 1) return fail(DV_ERR_INVALID_ARG, "image size must be >= 1");
  if (p->K < 1 || p->K % 2 == 0 || p->K > kMaxK)
    return fail(DV_ERR_INVALID_ARG, "K must be odd and in [1, %d]", kMaxK);
  if (p->grid_r < 1 || p->grid_c < 1) return fail(DV_ERR_INVALID_ARG, "PSF grid must be >= 1x1");
  if (!p->psfs) return fail(DV_ERR_INVALID_ARG, "psfs is NULL");
  if (p->n_tr < 1 || p->n_tc < 1) return fail(DV_ERR_INVALID_ARG, "tile grid must be >= 1x1");
  if (p->n_tr > kMaxTileGrid || p->n_tc > kMaxTileGrid)
    return fail(DV_ERR_INVALID_ARG, "tile grid must be at most %d x %d", kMaxTileGrid, kMaxTileGrid);
  if ((int64_t)p->hy + p->K - 1 > kMaxRows)
    return fail(DV_ERR_INVALID_ARG, "x must have at most %d rows", kMaxRows);
  if (!(p->lambda >= 0.0) || !(p->delta > 0.0) || !(p->gamma > 0.0))
    return fail(DV_ERR_INVALID_ARG, "need lambda >= 0, delta > 0, gamma > 0");
  if (!(p->rho > 0.0 && p->rho < 2.0)) return fail(DV_ERR_INVALID_ARG, "rho must be in (0, 2)");
  if (p->n_outer < 0 || p->n_inner < 0 || p->inner_increment < 0)
    return fail(DV_ERR_INVALID_ARG, "iteration counts must be >= 0");
  if (p->weight_kind != DV_WEIGHTS_BILINEAR && p->weight_kind != DV_WEIGHTS_SEPARABLE &&
      p->weight_kind != DV_WEIGHTS_PER_TILE)
    return fail(DV_ERR_INVALID_ARG, "unknown weight_kind %d", p->weight_kind);
  if (p->weight_kind == DV_WEIGHTS_SEPARABLE && (!p->weights_r || !p->weights_c))
    return fail(DV_ERR_INVALID_ARG, "separable weights need weights_r and weights_c");
  if (p->weight_kind != DV_WEIGHTS_SEPARABLE && (p->weights_r || p->weights_c))
    return fail(DV_ERR_INVALID_ARG, "bilinear and per-tile weights take no weight arrays");
  const bool per_tile = p->weight_kind == DV_WEIGHTS_PER_TILE;
  if (per_tile && (p->grid_r != p->n_tr || p->grid_c != p->n_tc))
    return fail(DV_ERR_INVALID_ARG,
                "one PSF per tile needs the PSF grid (%d x %d) to equal the tile grid (%d x %d)",
                p->grid_r, p->grid_c, p->n_tr, p->n_tc);
  if (p->precision != DV_PREC_FP32 && p->precision != DV_PREC_TF32 &&
      p->precision != DV_PREC_BF16)
    return fail(DV_ERR_INVALID_ARG, "unknown precision %d", p->precision);
  if (p->path < DV_PATH_AUTO || p->path > DV_PATH_TENSOR)
    return fail(DV_ERR_INVALID_ARG, "unknown operator path %d", p->path);
  if (p->overlap < 0) return fail(DV_ERR_INVALID_ARG, "overlap must be >= 0");
  if (p->check_every < 0) return fail(DV_ERR_INVALID_ARG, "check_every must be >= 0");
  if (p->local_solver != DV_SOLVER_PG && p->local_solver != DV_SOLVER_VMLMB)
    return fail(DV_ERR_INVALID_ARG, "unknown local_solver %d", p->local_solver);
  if (p->vm_memory < 0 || p->vm_memory > 32)
    return fail(DV_ERR_INVALID_ARG, "vm_memory must be in [0, 32] (0: 5)");
  if (!(p->vm_stop_rel >= 0.0) || !std::isfinite(p->vm_stop_rel))
    return fail(DV_ERR_INVALID_ARG, "vm_stop_rel must be finite and >= 0");
  if (p->tensor_h < 0 || p->tensor_h > 3)
    return fail(DV_ERR_INVALID_ARG, "tensor_h must be 0, 1, 2 or 3");
  if (!(p->noise_sigma >= 0.0)) return fail(DV_ERR_INVALID_ARG, "noise_sigma must be >= 0");

  const int K = p->K, nxr = p->hy + K - 1, nxc = p->wy + K - 1;
  if ((int64_t)nxr * nxc > (int64_t)1 << 40) return fail(DV_ERR_INVALID_ARG, "image too large");
  const bool given = p->tile_r0 || p->tile_r1 || p->tile_c0 || p->tile_c1;
  if (given) {
    if (!(p->tile_r0 && p->tile_r1 && p->tile_c0 && p->tile_c1))
      return fail(DV_ERR_INVALID_ARG, "give all four tile bound arrays or none");
    L.yr0.assign(p->tile_r0, p->tile_r0 + p->n_tr);
    L.yr1.assign(p->tile_r1, p->tile_r1 + p->n_tr);
    L.yc0.assign(p->tile_c0, p->tile_c0 + p->n_tc);
    L.yc1.assign(p->tile_c1, p->tile_c1 + p->n_tc);
  } else {
    if (p->n_tr > p->hy || p->n_tc > p->wy)
      return fail(DV_ERR_INVALID_ARG, "more tiles than pixels");
    if (per_tile) {
      grid_blocks(p->hy, K, p->n_tr, L.yr0, L.yr1);
      grid_blocks(p->wy, K, p->n_tc, L.yc0, L.yc1);
    } else {
      uniform_blocks(p->hy, p->n_tr, p->overlap, L.yr0, L.yr1);
      uniform_blocks(p->wy, p->n_tc, p->overlap, L.yc0, L.yc1);
    }
  }
  DV_TRY(check_blocks("row", p->hy, K, L.yr0, L.yr1));
  DV_TRY(check_blocks("column", p->wy, K, L.yc0, L.yc1));

  std::vector<int> xe(p->n_tr), xce(p->n_tc);
  for (int i = 0; i < p->n_tr; ++i) xe[i] = L.yr1[i] + K - 1;
  for (int i = 0; i < p->n_tc; ++i) xce[i] = L.yc1[i] + K - 1;
  L.omr = consensus_profiles(L.yr0, xe);
  L.omc = consensus_profiles(L.yc0, xce);

  DV_TRY(weight_table("row", nxr, p->grid_r,
                      p->weight_kind == DV_WEIGHTS_SEPARABLE ? p->weights_r : nullptr, L.wrow));
  DV_TRY(weight_table("column", nxc, p->grid_c,
                      p->weight_kind == DV_WEIGHTS_SEPARABLE ? p->weights_c : nullptr, L.wcol));
  if (per_tile) {
    tile_tables(L.yr0, L.yr1, K, L.wrow, L.wr0);
    tile_tables(L.yc0, L.yc1, K, L.wcol, L.wc0);
  } else {
    L.wr0 = L.yr0;
    L.wc0 = L.yc0;
  }

  // Lipschitz bound of the data gradient: ||H||^2 <= (max_p sum|h_p|)(sum_k max_p |h_p(k)|)
  const int G = p->grid_r * p->grid_c, KK = K * K;
  double colmax = 0.0, rowsum = 0.0;
  std::vector<double> kmax(KK, 0.0);
  for (int g = 0; g < G; ++g) {
    double s = 0.0;
    for (int k = 0; k < KK; ++k) {
      const double v = std::fabs((double)p->psfs[(size_t)g * KK + k]);
      if (!std::isfinite(v)) return fail(DV_ERR_INVALID_ARG, "PSF %d has a non-finite tap", g);
      s += v;
      kmax[k] = std::max(kmax[k], v);
    }
    colmax = std::max(colmax, s);
  }
  for (int k = 0; k < KK; ++k) rowsum += kmax[k];
  // one PSF per tile: the tile's own PSF alone, (sum |h_i|)^2
  auto tile_lh = [&](int tr, int tc) {
    if (!per_tile) return colmax * rowsum;
    double s1 = 0.0;
    for (int k = 0; k < KK; ++k) s1 += std::fabs((double)p->psfs[((size_t)tr * p->n_tc + tc) * KK + k]);
    return s1 * s1;
  };
  L.tau.assign((size_t)p->n_tr * p->n_tc, 0.0);
  for (int tr = 0; tr < p->n_tr; ++tr) {
    for (int tc = 0; tc < p->n_tc; ++tc) {
      double wmax = 1.0;
      if (p->noise_w) {
        wmax = 0.0;
        for (int i = L.yr0[tr]; i < L.yr1[tr]; ++i)
          for (int j = L.yc0[tc]; j < L.yc1[tc]; ++j) {
            const double v = p->noise_w[(size_t)i * p->wy + j];
            if (!(v >= 0.0) || !std::isfinite(v))
              return fail(DV_ERR_INVALID_ARG, "noise weights must be finite and >= 0");
            wmax = std::max(wmax, v);
          }
      }
      const double omax = *std::max_element(L.omr[tr].begin(), L.omr[tr].end()) *
                          *std::max_element(L.omc[tc].begin(), L.omc[tc].end());
      L.tau[(size_t)tr * p->n_tc + tc] =
          1.0 / (wmax * tile_lh(tr, tc) + 8.0 * p->lambda + p->gamma * omax);
    }
  }
  return DV_OK;
}

template <class T>
dv_status upload(dv_plan* P, T** dst, const T* src, size_t n, cudaStream_t s) {
  if (n == 0) n = 1;
  DV_TRY_CUDA(cudaMalloc((void**)dst, n * sizeof(T)));
  P->device_bytes += (int64_t)(n * sizeof(T));
  if (src) DV_TRY_CUDA(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, s));
  return DV_OK;
}

template <class T>
dv_status alloc(dv_plan* P, T** dst, size_t n) {
  if (n == 0) n = 1;
  DV_TRY_CUDA(cudaMalloc((void**)dst, n * sizeof(T)));
  P->device_bytes += (int64_t)(n * sizeof(T));
  return DV_OK;
}

// Work items of one operator over the given tiles: output blocks of bm x bn,
// with the PSF grid range active on the block's input (H) or output (H^T)
// region.  With max_rows > 0 the rows of each tile are split into the fewest
// blocks of at most max_rows rows, each a multiple of 16 rows, and the
// block's row count is stored in WorkItem.pad.
void make_work(const std::vector<TileDesc>& tiles, bool adjoint, int K, const Layout& L, int bm,
               int bn, std::vector<WorkItem>& out, int max_rows = 0) {
  out.clear();
  for (int t = 0; t < (int)tiles.size(); ++t) {
    const TileDesc& td = tiles[t];
    const int nr = adjoint ? td.nxr : td.nyr, nc = adjoint ? td.nxc : td.nyc;
    int bmt = bm;
    if (max_rows > 0) {
      const int nblk = (nr + max_rows - 1) / max_rows;
      bmt = (int)round_up((nr + nblk - 1) / nblk, 16);
    }
    for (int r0 = 0; r0 < nr; r0 += bmt) {
      for (int c0 = 0; c0 < nc; c0 += bn) {
        WorkItem w{};
        w.tile = t;
        w.r0 = r0;
        w.c0 = c0;
        if (max_rows > 0) w.pad = (int)std::min<int64_t>(bmt, round_up(nr - r0, 16));
        // weight-table coordinate range whose weights matter
        const int rlo = td.wr0 + r0, clo = td.wc0 + c0;
        const int rhi = td.wr0 + std::min(r0 + bmt, nr) + (adjoint ? 0 : K - 1);
        const int chi = td.wc0 + std::min(c0 + bn, nc) + (adjoint ? 0 : K - 1);
        active_range(L.wrow, rlo, rhi, w.a_lo, w.a_hi);
        active_range(L.wcol, clo, chi, w.b_lo, w.b_hi);
        out.push_back(w);
      }
    }
  }
}

}  // namespace

static int tab_index(int path) {
  return path == DV_PATH_FFT ? 1 : (path == DV_PATH_TENSOR ? 2 : 0);
}

int tab_index_of(int path) { return tab_index(path); }

// H / H^T as the block DFT: the tensor path with dft_H / dft_Ht set
static bool dft_h(const dv_plan* p, int path) { return path == DV_PATH_TENSOR && p->dft_H; }
static bool dft_ht(const dv_plan* p, int path) { return path == DV_PATH_TENSOR && p->dft_Ht; }

dv::OpArgs op_args_H(const dv_plan* p, int path, int mode, const float* in, float* out,
                     bool global) {
  OpArgs a{};
  const OpTables& tb = p->tab[dft_h(p, path) ? 1 : tab_index(path)];
  a.tiles = global ? p->d_gtile : p->d_tiles;
  a.work = global ? tb.Hg : tb.H;
  a.ksr = global ? tb.ksHg : tb.ksH;
  a.n_work = global ? tb.nHg : tb.nH;
  a.mode = mode;
  a.wrow = p->d_wrow;
  a.wcol = p->d_wcol;
  a.psf = p->d_psf_flip;
  a.Gc = p->Gc;
  a.K = p->K;
  a.KP = (p->K + 3) & ~3;
  a.in = in;
  a.out = out;
  a.y = p->d_y;
  a.W = p->d_W;
  a.wy = p->wy;
  a.partials = p->d_part;
  a.spec = p->d_spec;
  a.counter = p->d_counter;
  a.scratch = p->d_fft_scr;
  a.tcop = p->d_tcopH;
  a.prec = p->prob.precision;
  a.err = p->d_err;
  a.wait_ns = p->wait_ns;
  a.test_withhold = p->test_fault;
  a.lambda = (float)p->prob.lambda;
  a.delta = (float)p->prob.delta;
  a.gamma = (float)p->prob.gamma;
  if (dft_h(p, path)) {
    a.ksr = nullptr;
    a.spec = reinterpret_cast<const float2*>(p->d_dspec);
    a.tcop = p->d_dconst;
    a.counter = p->d_dcounter;
  }
  return a;
}

dv::OpArgs op_args_Ht(const dv_plan* p, int path, int mode, const float* in, float* out,
                      bool global, const float* w, const float* u) {
  OpArgs a = op_args_H(p, path, mode, in, out, global);
  const OpTables& tb = p->tab[dft_ht(p, path) ? 1 : tab_index(path)];
  a.spec = p->d_spec;
  a.tiles = global ? p->d_gtile : p->d_tiles;
  a.work = global ? tb.Htg : tb.Ht;
  a.ksr = global ? tb.ksHtg : tb.ksHt;
  a.n_work = global ? tb.nHtg : tb.nHt;
  a.psf = p->d_psf;
  a.counter = p->d_counter ? p->d_counter + 1 : nullptr;
  a.tcop = p->d_tcopHt;
  a.w = w;
  a.u = u;
  a.omr = p->d_omr;
  a.omc = p->d_omc;
  if (dft_ht(p, path)) {
    // block DFT: the block FFT's H^T work items; the counters of the H
    // launches (a group's H and H^T run in order on its stream)
    a.ksr = nullptr;
    a.spec = reinterpret_cast<const float2*>(p->d_dspec);
    a.tcop = p->d_dconst;
    a.counter = p->d_dcounter;
  }
  return a;
}

cudaError_t launch_op_H(const dv_plan* P, int path, const OpArgs& a, cudaStream_t s) {
  if (dft_h(P, path)) return launch_dft_H(a, s, a.ctas > 0 ? a.ctas : P->n_sm);
  if (path == DV_PATH_TENSOR)
    return P->prob.precision == DV_PREC_BF16 ? launch_tcT_H(a, s) : launch_tc_H(a, s);
  return path == DV_PATH_FFT ? launch_fft_H(a, s, P->n_sm) : launch_direct_H(a, s);
}

cudaError_t launch_op_Ht(const dv_plan* P, int path, const OpArgs& a, cudaStream_t s) {
  if (dft_ht(P, path)) return launch_dft_Ht(a, s, a.ctas > 0 ? a.ctas : P->n_sm);
  if (path == DV_PATH_TENSOR)
    return P->prob.precision == DV_PREC_BF16 ? launch_tcT_Ht(a, s) : launch_tc_Ht(a, s);
  return path == DV_PATH_FFT ? launch_fft_Ht(a, s, P->n_sm) : launch_direct_Ht(a, s);
}

int obj_parts(const dv_plan* P) { return P->tab[tab_index(P->fpath)].nH; }

dv::OpArgs group_args(const dv_plan* p, int path, dv::OpArgs a, bool adjoint, int g) {
  const bool dft = adjoint ? dft_ht(p, path) : dft_h(p, path);
  const OpTables& tb = p->tab[dft ? 1 : tab_index(path)];
  const int* b = adjoint ? tb.gHt : tb.gH;
  a.work += b[g];
  a.n_work = b[g + 1] - b[g];
  if (a.ksr) a.ksr += (size_t)b[g] * kTcMaxB;
  if (dft) {
    // persistent launches of the concurrent groups share the SMs
    a.counter = p->d_dcounter + 1 + g;
    a.ctas = std::max(1, p->n_sm / std::max(1, p->ngrp));
  }
  return a;
}

dv::GridArgs grid_args(const dv_plan* p) {
  GridArgs g{};
  g.tiles = p->d_tiles;
  g.rowcov = p->d_rowcov;
  g.colcov = p->d_colcov;
  g.citems = p->d_citems;
  g.n_citems = p->n_citems;
  g.omr = p->d_omr;
  g.omc = p->d_omc;
  g.n_tc = p->n_tc;
  g.nxr = p->nxr;
  g.nxc = p->nxc;
  return g;
}

dv_status release(dv_plan* P);

}  // namespace dv

using namespace dv;

extern "C" const char* dv_last_error(void) { return g_err.c_str(); }

extern "C" void dv_problem_init(dv_problem* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->hy = p->wy = 1;
  p->grid_r = p->grid_c = 1;
  p->K = 1;
  p->weight_kind = DV_WEIGHTS_BILINEAR;
  p->n_tr = p->n_tc = 1;
  p->overlap = 16;
  p->lambda = 1e-3;
  p->delta = 1.0 / 60.0;
  p->gamma = 0.4;
  p->rho = 1.0;
  p->n_outer = 30;
  p->n_inner = 10;
  p->precision = DV_PREC_FP32;
  p->path = DV_PATH_AUTO;
  p->use_graphs = 1;
  p->vm_stop_rel = 1e-7;
}

extern "C" dv_status dv_layout_query(const dv_problem* prob, int32_t* tile_r0, int32_t* tile_r1,
                                     int32_t* tile_c0, int32_t* tile_c1, double* tau) {
  clear_error();
  Layout L;
  DV_TRY(validate_and_layout(prob, L));
  for (int i = 0; i < prob->n_tr; ++i) {
    if (tile_r0) tile_r0[i] = L.yr0[i];
    if (tile_r1) tile_r1[i] = L.yr1[i];
  }
  for (int i = 0; i < prob->n_tc; ++i) {
    if (tile_c0) tile_c0[i] = L.yc0[i];
    if (tile_c1) tile_c1[i] = L.yc1[i];
  }
  if (tau) std::copy(L.tau.begin(), L.tau.end(), tau);
  return DV_OK;
}

namespace dv {
// Autotuner: times one H (with residual) and one H^T (with the fused step) on
// the plan's tile stacks for each candidate path.  The FP32 operator (used
// for the objective and, unless the tensor path wins, the inner iterations)
// is the faster of direct and block FFT; with BF16 / TF32 allowed the tensor
// path competes for the inner iterations.
static dv_status time_path(dv_plan* P, int path, cudaStream_t s, double& out) {
  double best = 1e30;
  for (int rep = 0; rep < 4; ++rep) {
    DV_TRY_CUDA(cudaEventRecord(P->ev0, s));
    DV_TRY_CUDA(launch_op_H(P, path, op_args_H(P, path, OP_RESID, P->d_w[0], P->d_r, false), s));
    DV_TRY_CUDA(launch_op_Ht(P, path, op_args_Ht(P, path, OP_STEP, P->d_r, P->d_w[1], false,
                                                 P->d_w[0], P->d_u), s));
    DV_TRY_CUDA(cudaEventRecord(P->ev1, s));
    DV_TRY_CUDA(cudaEventSynchronize(P->ev1));
    float ms = 0.f;
    DV_TRY_CUDA(cudaEventElapsedTime(&ms, P->ev0, P->ev1));
    if (rep > 0) best = std::min(best, (double)ms);   // first repetition warms up
  }
  out = best;
  return DV_OK;
}

static dv_status choose_path(dv_plan* P, int requested, cudaStream_t s) {
  if (requested == DV_PATH_DIRECT || requested == DV_PATH_FFT) {
    P->path = P->fpath = requested;
    return DV_OK;
  }
  P->fpath = DV_PATH_DIRECT;
  if (P->fft_ok) {
    DV_TRY(time_path(P, DV_PATH_DIRECT, s, P->tune_ms[0]));
    DV_TRY(time_path(P, DV_PATH_FFT, s, P->tune_ms[1]));
    if (P->tune_ms[1] < P->tune_ms[0]) P->fpath = DV_PATH_FFT;
  }
  P->path = P->fpath;
  // the tensor path's forms: banded Toeplitz MMAs for H and H^T, the block
  // DFT for H, or the block DFT for both (tensor_h)
  auto tensor_form = [&]() -> dv_status {
    P->dft_H = P->dft_Ht = false;
    if (!P->dft_ok) return DV_OK;
    if (P->prob.tensor_h >= 2) {
      P->dft_H = true;
      P->dft_Ht = P->prob.tensor_h == 3;
      return DV_OK;
    }
    if (P->tune_ms[2] == 0.0) DV_TRY(time_path(P, DV_PATH_TENSOR, s, P->tune_ms[2]));
    P->dft_H = true;
    DV_TRY(time_path(P, DV_PATH_TENSOR, s, P->tune_ms_dft));
    P->dft_Ht = true;
    DV_TRY(time_path(P, DV_PATH_TENSOR, s, P->tune_ms_dft2));
    const double best = std::min(P->tune_ms[2], std::min(P->tune_ms_dft, P->tune_ms_dft2));
    P->dft_Ht = best == P->tune_ms_dft2;
    P->dft_H = P->dft_Ht || best == P->tune_ms_dft;
    return DV_OK;
  };
  if (requested == DV_PATH_TENSOR) {
    P->path = DV_PATH_TENSOR;
    DV_TRY(tensor_form());
  } else if (P->tensor_ok) {
    DV_TRY(time_path(P, DV_PATH_TENSOR, s, P->tune_ms[2]));
    DV_TRY(tensor_form());
    const double fp32_ms = P->tune_ms[P->fpath == DV_PATH_FFT ? 1 : 0];
    if (fp32_ms == 0.0) DV_TRY(time_path(P, P->fpath, s, P->tune_ms[P->fpath == DV_PATH_FFT ? 1 : 0]));
    const double t_ms = P->dft_Ht ? P->tune_ms_dft2 : (P->dft_H ? P->tune_ms_dft : P->tune_ms[2]);
    if (t_ms < P->tune_ms[P->fpath == DV_PATH_FFT ? 1 : 0]) P->path = DV_PATH_TENSOR;
    else P->dft_H = P->dft_Ht = false;
  }
  return DV_OK;
}

static dv_status build_plan(const dv_problem* prob, cudaStream_t s, dv_plan* P) {
  Layout L;
  DV_TRY(validate_and_layout(prob, L));
  if (prob->path == DV_PATH_TENSOR && prob->precision == DV_PREC_FP32)
    return fail(DV_ERR_INVALID_ARG, "the tensor-core path needs precision BF16 or TF32");
  if (prob->path == DV_PATH_TENSOR && !tc_supported(prob->K))
    return fail(DV_ERR_UNSUPPORTED, "the tensor-core operator supports K = 9, 15, 31, 63");
  if (prob->path == DV_PATH_FFT && !fft_supported(prob->K))
    return fail(DV_ERR_UNSUPPORTED, "the FFT operator path needs K <= %d", fft_size() - 31);
  if (prob->tensor_h >= 2 && (prob->precision != DV_PREC_BF16 || !dft_supported(prob->K) ||
                              !tc_supported(prob->K) || prob->path == DV_PATH_DIRECT ||
                              prob->path == DV_PATH_FFT))
    return fail(DV_ERR_UNSUPPORTED,
                "the block-DFT forms of H and H^T need the tensor-core path with BF16 allowed "
                "and K in 9, 15, 31, 63");

  P->prob = *prob;
  P->vm_m = prob->vm_memory > 0 ? prob->vm_memory : 5;
  P->prob.psfs = nullptr;
  P->prob.weights_r = P->prob.weights_c = nullptr;
  P->prob.tile_r0 = P->prob.tile_r1 = P->prob.tile_c0 = P->prob.tile_c1 = nullptr;
  P->prob.noise_w = nullptr;
  P->hy = prob->hy;
  P->wy = prob->wy;
  P->K = prob->K;
  P->rad = prob->K / 2;
  P->Gr = prob->grid_r;
  P->Gc = prob->grid_c;
  P->nxr = prob->hy + prob->K - 1;
  P->nxc = prob->wy + prob->K - 1;
  P->n_tr = prob->n_tr;
  P->n_tc = prob->n_tc;
  P->T = P->n_tr * P->n_tc;
  P->path = DV_PATH_DIRECT;
  P->fpath = DV_PATH_DIRECT;
  P->tensor_ok = prob->precision != DV_PREC_FP32 && tc_supported(prob->K) &&
                 (prob->path == DV_PATH_AUTO || prob->path == DV_PATH_TENSOR);
  P->fft_ok = prob->path != DV_PATH_DIRECT && fft_supported(prob->K);
  P->dft_ok = P->tensor_ok && P->fft_ok && prob->precision == DV_PREC_BF16 &&
              dft_supported(prob->K) && prob->tensor_h != 1;
  {
    int dev = 0;
    DV_TRY_CUDA(cudaGetDevice(&dev));
    DV_TRY_CUDA(cudaDeviceGetAttribute(&P->n_sm, cudaDevAttrMultiProcessorCount, dev));
  }
  P->yr0 = L.yr0;
  P->yr1 = L.yr1;
  P->yc0 = L.yc0;
  P->yc1 = L.yc1;
  P->tau = L.tau;
  const int K = P->K, KP = (K + 3) & ~3;

  // PSFs as given and flipped, rows padded to KP
  const int G = P->Gr * P->Gc;
  std::vector<float> psf((size_t)G * K * KP, 0.f), flip((size_t)G * K * KP, 0.f);
  for (int g = 0; g < G; ++g)
    for (int a = 0; a < K; ++a)
      for (int b = 0; b < K; ++b) {
        const float v = prob->psfs[((size_t)g * K + a) * K + b];
        psf[((size_t)g * K + a) * KP + b] = v;
        flip[((size_t)g * K + (K - 1 - a)) * KP + (K - 1 - b)] = v;
      }
  DV_TRY(upload(P, &P->d_psf, psf.data(), psf.size(), s));
  {
    std::vector<float> desc;
    psf_descriptors(prob->psfs, G, K, desc);
    DV_TRY(upload(P, &P->d_desc, desc.data(), desc.size(), s));
  }
  DV_TRY(upload(P, &P->d_psf_flip, flip.data(), flip.size(), s));
  DV_TRY(upload(P, &P->d_wrow, L.wrow.data(), L.wrow.size(), s));
  DV_TRY(upload(P, &P->d_wcol, L.wcol.data(), L.wcol.size(), s));

  // consensus profiles, concatenated per tile row / column
  std::vector<float> omr, omc;
  std::vector<int> omr_off(P->n_tr), omc_off(P->n_tc);
  for (int i = 0; i < P->n_tr; ++i) {
    omr_off[i] = (int)omr.size();
    for (double v : L.omr[i]) omr.push_back((float)v);
  }
  for (int i = 0; i < P->n_tc; ++i) {
    omc_off[i] = (int)omc.size();
    for (double v : L.omc[i]) omc.push_back((float)v);
  }
  DV_TRY(upload(P, &P->d_omr, omr.data(), omr.size(), s));
  DV_TRY(upload(P, &P->d_omc, omc.data(), omc.size(), s));

  // tile descriptors and stack layout (rows padded to 32 floats)
  P->h_tiles.clear();
  int64_t xo = 0, yo = 0;
  P->max_nxr = P->max_nxc = 0;
  for (int tr = 0; tr < P->n_tr; ++tr) {
    for (int tc = 0; tc < P->n_tc; ++tc) {
      TileDesc d{};
      d.xr0 = L.yr0[tr];
      d.xc0 = L.yc0[tc];
      d.nyr = L.yr1[tr] - L.yr0[tr];
      d.nyc = L.yc1[tc] - L.yc0[tc];
      d.nxr = d.nyr + K - 1;
      d.nxc = d.nyc + K - 1;
      d.xpitch = (int)round_up(d.nxc, 32);
      d.ypitch = (int)round_up(d.nyc, 32);
      d.xoff = xo;
      d.yoff = yo;
      xo += round_up((int64_t)d.nxr * d.xpitch, 32);
      yo += round_up((int64_t)d.nyr * d.ypitch, 32);
      d.omr_off = omr_off[tr];
      d.omc_off = omc_off[tc];
      d.tr = tr;
      d.tc = tc;
      d.wr0 = L.wr0[tr];
      d.wc0 = L.wc0[tc];
      d.tau = (float)L.tau[(size_t)tr * P->n_tc + tc];
      P->max_nxr = std::max(P->max_nxr, d.nxr);
      P->max_nxc = std::max(P->max_nxc, d.nxc);
      P->h_tiles.push_back(d);
    }
  }
  P->xstack = xo;
  P->ystack = yo;
  DV_TRY(upload(P, &P->d_tiles, P->h_tiles.data(), P->h_tiles.size(), s));
  TileDesc gt{};
  gt.nyr = P->hy;
  gt.nyc = P->wy;
  gt.nxr = P->nxr;
  gt.nxc = P->nxc;
  gt.xpitch = P->nxc;
  gt.ypitch = P->wy;
  gt.omr_off = gt.omc_off = 0;
  gt.tau = 0.f;
  DV_TRY(upload(P, &P->d_gtile, &gt, 1, s));
  // host copy of the global tile for work-table construction
  std::vector<TileDesc> gtiles{gt};

  // work tables: direct path always, FFT and tensor paths when available
  std::vector<WorkItem> w;
  // tile groups of the captured local solve on the tensor path, balanced by
  // the tiles' (block, active PSF) pairs (largest tile to the lightest group)
  std::vector<int> tgroup(P->h_tiles.size(), 0);
  P->ngrp = (P->tensor_ok && prob->use_graphs) ? std::min<int>(kMaxGroups, (int)P->h_tiles.size()) : 1;
  if (P->ngrp > 1) {
    make_work(P->h_tiles, false, K, L, direct_tile_m(), direct_tile_n(), w);
    std::vector<int64_t> cost(P->h_tiles.size(), 0), load(P->ngrp, 0);
    for (const WorkItem& it : w) cost[it.tile] += (int64_t)(it.a_hi - it.a_lo + 1) * (it.b_hi - it.b_lo + 1);
    std::vector<int> idx(P->h_tiles.size());
    for (size_t t = 0; t < idx.size(); ++t) idx[t] = (int)t;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    for (int t : idx) {
      const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      tgroup[t] = g;
      load[g] += cost[t];
    }
  }
  for (int k = 0; k < 3; ++k) {
    if ((k == 1 && !P->fft_ok) || (k == 2 && !P->tensor_ok)) continue;
    // tensor path: BF16 column-band blocks (128 columns, rows per tile up to
    // tcT_max_rows) or the TF32 row-band blocks
    const bool band = k == 2 && prob->precision == DV_PREC_BF16;
    const int bm = k == 0 ? direct_tile_m() : (k == 1 ? fft_block(K) : tc_block_m());
    const int bn = k == 0 ? direct_tile_n()
                          : (k == 1 ? fft_block(K) : (band ? tcT_block_cols() : tc_block_n()));
    const int max_rows = band ? tcT_max_rows(K) : 0;
    OpTables& tb = P->tab[k];
    // FFT items are handed out dynamically, tensor items are long: heaviest
    // (most PSFs) first
    auto order = [&](std::vector<WorkItem>& v) {
      if (k >= 1)
        std::stable_sort(v.begin(), v.end(), [](const WorkItem& x, const WorkItem& y) {
          return (x.a_hi - x.a_lo + 1) * (x.b_hi - x.b_lo + 1) + 1 >
                 (y.a_hi - y.a_lo + 1) * (y.b_hi - y.b_lo + 1) + 1;
        });
    };
    // tensor path, tile mode: items grouped by tile group (heaviest first
    // within a group); bounds[g] = first item of group g
    auto group = [&](std::vector<WorkItem>& v, int* bounds) {
      std::fill(bounds, bounds + kMaxGroups + 1, (int)v.size());
      bounds[0] = 0;
      if (!(k == 2 || (k == 1 && P->dft_ok)) || P->ngrp <= 1) return;
      std::stable_sort(v.begin(), v.end(), [&](const WorkItem& x, const WorkItem& y) {
        return tgroup[x.tile] < tgroup[y.tile];
      });
      for (int g = 1; g <= P->ngrp; ++g)
        bounds[g] = (int)(std::partition_point(v.begin(), v.end(), [&](const WorkItem& x) {
                            return tgroup[x.tile] < g;
                          }) - v.begin());
    };
    auto count = [&](const std::vector<WorkItem>& v, int k2) {
      for (const WorkItem& it : v) {
        const int64_t np = (int64_t)(it.a_hi - it.a_lo + 1) * (it.b_hi - it.b_lo + 1);
        tb.psfs[k2] += np;
        tb.pairs[k2] += (np + 1) / 2;
        if (np > 0) tb.rows[k2] += it.a_hi - it.a_lo + 1;
      }
    };
    // BF16 tensor path: per-item k-step ranges of the PSF grid columns
    std::vector<uint16_t> ks;
    auto ranges = [&](const std::vector<TileDesc>& tl, bool adj, uint16_t** dst) -> dv_status {
      if (!band) return DV_OK;
      const int64_t steps = tcT_kstep_ranges(tl, w, L.wcol, K, adj, ks);
      if (&tl == &P->h_tiles) tb.ksteps[adj ? 1 : 0] = steps;
      return upload(P, dst, ks.data(), ks.size(), s);
    };
    make_work(P->h_tiles, false, K, L, bm, bn, w, max_rows);
    count(w, 0);
    order(w);
    group(w, tb.gH);
    tb.nH = (int)w.size();
    tb.tileH.resize(w.size());
    for (size_t i = 0; i < w.size(); ++i) tb.tileH[i] = w[i].tile;
    DV_TRY(upload(P, &tb.H, w.data(), w.size(), s));
    DV_TRY(ranges(P->h_tiles, false, &tb.ksH));
    make_work(P->h_tiles, true, K, L, bm, bn, w, max_rows);
    count(w, 1);
    order(w);
    group(w, tb.gHt);
    tb.nHt = (int)w.size();
    DV_TRY(upload(P, &tb.Ht, w.data(), w.size(), s));
    DV_TRY(ranges(P->h_tiles, true, &tb.ksHt));
    make_work(gtiles, false, K, L, bm, bn, w, max_rows);
    order(w);
    tb.nHg = (int)w.size();
    DV_TRY(upload(P, &tb.Hg, w.data(), w.size(), s));
    DV_TRY(ranges(gtiles, false, &tb.ksHg));
    make_work(gtiles, true, K, L, bm, bn, w, max_rows);
    order(w);
    tb.nHtg = (int)w.size();
    DV_TRY(upload(P, &tb.Htg, w.data(), w.size(), s));
    DV_TRY(ranges(gtiles, true, &tb.ksHtg));
  }
  if (P->tensor_ok) {
    std::vector<uint8_t> op;
    const bool bf16 = prob->precision == DV_PREC_BF16;
    for (int flip = 1; flip >= 0; --flip) {
      if (bf16)
        tcT_operands(prob->psfs, G, K, flip != 0, op);
      else
        tc_operands(prob->psfs, G, K, prob->precision, flip != 0, op);
      DV_TRY(upload(P, flip ? &P->d_tcopH : &P->d_tcopHt, op.data(), op.size(), s));
    }
    DV_TRY_CUDA(bf16 ? tcT_prepare(K) : tc_prepare(K, prob->precision));
  }
  DV_TRY(alloc(P, &P->d_err, 1));
  DV_TRY_CUDA(cudaMemsetAsync(P->d_err, 0, sizeof(int), s));
  if (P->dft_ok) {
    std::vector<uint8_t> cst;
    dft_constants(cst);
    DV_TRY(upload(P, &P->d_dconst, cst.data(), cst.size(), s));
    std::vector<uint32_t> dsp;
    dft_spectra(prob->psfs, G, K, dsp);
    DV_TRY(upload(P, &P->d_dspec, dsp.data(), dsp.size(), s));
    DV_TRY(alloc(P, &P->d_dcounter, 1 + kMaxGroups));
    DV_TRY_CUDA(dft_prepare());
  }
  if (P->fft_ok) {
    DV_TRY(alloc(P, &P->d_counter, 2));
    DV_TRY(alloc(P, &P->d_fft_scr, (size_t)P->n_sm * fft_size() * fft_size()));
    std::vector<float2> spec;
    fft_spectra(prob->psfs, G, K, spec);
    DV_TRY(upload(P, &P->d_spec, spec.data(), spec.size(), s));
    DV_TRY_CUDA(fft_prepare());
  }

  // tiles covering each global x row / column (at most two)
  std::vector<int2> rc(P->nxr, make_int2(-1, -1)), cc(P->nxc, make_int2(-1, -1));
  for (int tr = 0; tr < P->n_tr; ++tr)
    for (int R = L.yr0[tr]; R < L.yr1[tr] + K - 1; ++R) (rc[R].x < 0 ? rc[R].x : rc[R].y) = tr;
  for (int tc = 0; tc < P->n_tc; ++tc)
    for (int C = L.yc0[tc]; C < L.yc1[tc] + K - 1; ++C) (cc[C].x < 0 ? cc[C].x : cc[C].y) = tc;
  DV_TRY(upload(P, &P->d_rowcov, rc.data(), rc.size(), s));
  DV_TRY(upload(P, &P->d_colcov, cc.data(), cc.size(), s));
  // consensus / assembly items: rectangles of constant cover, cut into
  // pieces of at most cons_item_cols() columns and cons_item_pixels() pixels
  {
    std::vector<ConsItem> items;
    auto bands = [](const std::vector<int2>& cov) {
      std::vector<std::pair<int, int>> b;
      for (int i = 0; i < (int)cov.size();) {
        int e = i + 1;
        while (e < (int)cov.size() && cov[e].x == cov[i].x && cov[e].y == cov[i].y) ++e;
        b.push_back({i, e});
        i = e;
      }
      return b;
    };
    for (const auto& rb : bands(rc))
      for (const auto& cb : bands(cc))
        for (int c0 = cb.first; c0 < cb.second; c0 += cons_item_cols()) {
          const int ncol = std::min(cons_item_cols(), cb.second - c0);
          const int rows = std::max(1, cons_item_pixels() / ncol);
          for (int r0 = rb.first; r0 < rb.second; r0 += rows) {
            ConsItem it{};
            it.r0 = r0;
            it.nrow = std::min(rows, rb.second - r0);
            it.c0 = c0;
            it.ncol = ncol;
            const int trs[2] = {rc[r0].x, rc[r0].y}, tcs[2] = {cc[c0].x, cc[c0].y};
            for (int i = 0; i < 2; ++i)
              for (int j = 0; j < 2; ++j) {
                if (trs[i] < 0 || tcs[j] < 0) continue;
                const TileDesc& td = P->h_tiles[(size_t)trs[i] * P->n_tc + tcs[j]];
                const int sl = it.ns++;
                it.base[sl] = td.xoff + (int64_t)(r0 - td.xr0) * td.xpitch - td.xc0;
                it.pitch[sl] = td.xpitch;
                it.obr[sl] = td.omr_off - td.xr0;
                it.obc[sl] = td.omc_off - td.xc0;
              }
            items.push_back(it);
          }
        }
    P->n_citems = (int)items.size();
    DV_TRY(upload(P, &P->d_citems, items.data(), items.size(), s));
  }

  // iterates, dual variable, residuals, data, scratch
  DV_TRY(alloc(P, &P->d_w[0], P->xstack));
  DV_TRY(alloc(P, &P->d_w[1], P->xstack));
  DV_TRY(alloc(P, &P->d_u, P->xstack));
  DV_TRY(alloc(P, &P->d_r, P->ystack));
  DV_TRY(cudaMemsetAsync(P->d_w[0], 0, P->xstack * sizeof(float), s) == cudaSuccess
             ? DV_OK : fail(DV_ERR_CUDA, "memset"));
  DV_TRY(cudaMemsetAsync(P->d_w[1], 0, P->xstack * sizeof(float), s) == cudaSuccess
             ? DV_OK : fail(DV_ERR_CUDA, "memset"));
  DV_TRY(cudaMemsetAsync(P->d_u, 0, P->xstack * sizeof(float), s) == cudaSuccess
             ? DV_OK : fail(DV_ERR_CUDA, "memset"));
  DV_TRY(alloc(P, &P->d_y, (size_t)P->hy * P->wy));
  if (prob->noise_w) DV_TRY(upload(P, &P->d_W, prob->noise_w, (size_t)P->hy * P->wy, s));
  DV_TRY(alloc(P, &P->d_z, (size_t)P->nxr * P->nxc));
  DV_TRY(alloc(P, &P->d_xg, (size_t)P->nxr * P->nxc));
  const int64_t ncons = consensus_blocks(P->n_citems);
  const int64_t nhub = huber_blocks(P->T, P->max_nxr, P->max_nxc);
  P->n_part = std::max(std::max(P->tab[0].nH, P->tab[1].nH), P->tab[2].nH) + nhub + 2 * ncons;
  DV_TRY(alloc(P, &P->d_part, (size_t)P->n_part));
  DV_TRY(alloc(P, &P->d_scal, 8));
  DV_TRY_CUDA(cudaMallocHost((void**)&P->h_scal, 8 * sizeof(double)));
  DV_TRY_CUDA(direct_prepare(K));
  DV_TRY_CUDA(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  if (P->ngrp > 1) {
    DV_TRY_CUDA(cudaEventCreateWithFlags(&P->grp_fork, cudaEventDisableTiming));
    for (int g = 0; g < P->ngrp; ++g) {
      DV_TRY_CUDA(cudaStreamCreateWithFlags(&P->grp_stream[g], cudaStreamNonBlocking));
      DV_TRY_CUDA(cudaEventCreateWithFlags(&P->grp_join[g], cudaEventDisableTiming));
    }
  }
  DV_TRY_CUDA(cudaEventCreate(&P->ev0));
  DV_TRY_CUDA(cudaEventCreate(&P->ev1));
  DV_TRY_CUDA(cudaMemsetAsync(P->d_y, 0, (size_t)P->hy * P->wy * sizeof(float), s));
  DV_TRY_CUDA(cudaMemsetAsync(P->d_r, 0, (size_t)P->ystack * sizeof(float), s));
  DV_TRY(choose_path(P, prob->path, s));
  DV_TRY_CUDA(cudaStreamSynchronize(s));
  return DV_OK;
}
}  // namespace dv

extern "C" dv_status dv_plan_create(const dv_problem* prob, void* stream, dv_plan** out) {
  Range range("dv plan");
  clear_error();
  if (!out) return fail(DV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  dv_plan* P = new (std::nothrow) dv_plan();
  if (!P) return fail(DV_ERR_OOM, "host allocation of the plan failed");
  const dv_status st = build_plan(prob, (cudaStream_t)stream, P);
  if (st != DV_OK) {
    const std::string msg = g_err;
    release(P);
    g_err = msg;
    return st;
  }
  *out = P;
  return DV_OK;
}

namespace dv {
dv_status release(dv_plan* P) {
  if (!P) return DV_OK;
  for (auto& g : P->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  for (cudaEvent_t e : P->timer.pool) cudaEventDestroy(e);
  for (cudaEvent_t e : P->timer.placeholders) cudaEventDestroy(e);
  void* vbufs[] = {P->d_vg, P->d_vgt, P->d_vd, P->d_vq, P->d_vht, P->d_vs, P->d_vy,
                   P->d_vpart, P->d_vhub, P->d_vcoef};
  for (void* b : vbufs)
    if (b) cudaFree(b);
  if (P->h_vcoef) cudaFreeHost(P->h_vcoef);
  if (P->h_vpart) cudaFreeHost(P->h_vpart);
  void* bufs[] = {P->d_psf_flip, P->d_psf, P->d_wrow, P->d_wcol, P->d_omr, P->d_omc,
                  P->d_tiles, P->d_gtile, P->tab[0].H, P->tab[0].Ht, P->tab[0].Hg,
                  P->tab[0].Htg, P->tab[1].H, P->tab[1].Ht, P->tab[1].Hg, P->tab[1].Htg,
                  P->d_spec, P->d_counter, P->d_fft_scr, P->d_desc, P->d_feat, P->d_wsd,
                  P->tab[2].H, P->tab[2].Ht, P->tab[2].Hg, P->tab[2].Htg,
                  P->tab[2].ksH, P->tab[2].ksHt, P->tab[2].ksHg, P->tab[2].ksHtg,
                  P->d_tcopH, P->d_tcopHt, P->d_err, P->d_dspec, P->d_dconst, P->d_dcounter,
                  P->d_rowcov, P->d_colcov, P->d_citems, P->d_w[0], P->d_w[1], P->d_u, P->d_r, P->d_y,
                  P->d_W, P->d_z, P->d_xg, P->d_part, P->d_scal, P->d_hx, P->d_hy, P->d_hx0};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (P->h_scal) cudaFreeHost(P->h_scal);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  for (int g = 0; g < kMaxGroups; ++g) {
    if (P->grp_stream[g]) cudaStreamDestroy(P->grp_stream[g]);
    if (P->grp_join[g]) cudaEventDestroy(P->grp_join[g]);
  }
  if (P->grp_fork) cudaEventDestroy(P->grp_fork);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  delete P;
  return DV_OK;
}
}  // namespace dv

extern "C" dv_status dv_destroy(dv_plan* plan) {
  clear_error();
  return release(plan);
}

extern "C" dv_status dv_plan_get_info(const dv_plan* P, dv_plan_info* info) {
  clear_error();
  if (!P || !info) return fail(DV_ERR_INVALID_ARG, "plan or info is NULL");
  info->nx_r = P->nxr;
  info->nx_c = P->nxc;
  info->n_tiles = P->T;
  info->path = P->path;
  info->stack_elems = P->xstack;
  info->device_bytes = P->device_bytes;
  info->tau_min = *std::min_element(P->tau.begin(), P->tau.end());
  info->tau_max = *std::max_element(P->tau.begin(), P->tau.end());
  info->kernel_launches = P->launches;
  info->tune_ms_direct = P->tune_ms[0];
  info->tune_ms_fft = P->tune_ms[1];
  info->tune_ms_tensor = P->tune_ms[2];
  info->fp32_path = P->fpath;
  const int k = tab_index(P->path);
  info->blocks[0] = P->tab[k].nH;
  info->blocks[1] = P->tab[k].nHt;
  info->block_psfs[0] = P->tab[k].psfs[0];
  info->block_psfs[1] = P->tab[k].psfs[1];
  info->psf_pairs[0] = P->tab[k].pairs[0];
  info->psf_pairs[1] = P->tab[k].pairs[1];
  info->mma_ksteps[0] = P->tab[k].ksteps[0];
  info->mma_ksteps[1] = P->tab[k].ksteps[1];
  info->tile_groups = (P->ngrp > 1 && P->path == DV_PATH_TENSOR) ? P->ngrp : 1;
  info->tensor_h_dft = P->path == DV_PATH_TENSOR && P->dft_H ? 1 : 0;
  info->tensor_ht_dft = P->path == DV_PATH_TENSOR && P->dft_Ht ? 1 : 0;
  info->dft_h_rows = (int32_t)std::min<int64_t>(P->tab[1].rows[0], INT32_MAX);
  info->tune_ms_tensor_dft = P->tune_ms_dft;
  info->tune_ms_tensor_dft2 = P->tune_ms_dft2;
  if (info->tensor_h_dft) {
    info->blocks[0] = P->tab[1].nH;
    info->block_psfs[0] = P->tab[1].psfs[0];
    info->psf_pairs[0] = P->tab[1].pairs[0];
    info->mma_ksteps[0] = 0;
  }
  if (info->tensor_ht_dft) {
    info->blocks[1] = P->tab[1].nHt;
    info->block_psfs[1] = P->tab[1].psfs[1];
    info->psf_pairs[1] = P->tab[1].pairs[1];
    info->mma_ksteps[1] = 0;
  }
  info->block_side = k == 1 ? fft_block(P->K)
                            : (k == 2 ? (P->prob.precision == DV_PREC_BF16 ? tcT_max_rows(P->K)
                                                                          : tc_block_m())
                                      : direct_tile_m());
  return DV_OK;
}
