// Streaming (HBM-bound) kernels of libdv: start/gather of the tile stacks, the
// consensus prox and dual update (Lemma 1 and the explicit D-R updates of
// Sec. III-B), assembly of x_hat, FP64 partials of the Huber prior
// (Sec. IV-A) and a fixed-order FP64 reduction.
#include "dv_internal.cuh"

namespace dv {
namespace {

constexpr int NB = 256;  // threads per block of the streaming kernels

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v over the block (fixed order); valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// x_i = u_i = C_i x0 for every tile; x0 is the given global image or, if
// NULL, the observed image edge-replicated by rad.  Optionally also writes the
// global x0 (the "previous zbar" of the first dual residual).
__global__ void scatter_kernel(const TileDesc* __restrict__ tiles, const float* __restrict__ x0,
                               const float* __restrict__ y, int hy, int wy, int rad, int nxc_g,
                               float* __restrict__ w, float* __restrict__ u,
                               float* __restrict__ zg) {
  const TileDesc td = tiles[blockIdx.z];
  const int R = blockIdx.y;
  if (R >= td.nxr) return;
  for (int C = blockIdx.x * blockDim.x + threadIdx.x; C < td.nxc; C += gridDim.x * blockDim.x) {
    const int Rg = td.xr0 + R, Cg = td.xc0 + C;
    float v;
    if (x0) {
      v = x0[(int64_t)Rg * nxc_g + Cg];
    } else {
      const int ry = min(max(Rg - rad, 0), hy - 1), rx = min(max(Cg - rad, 0), wy - 1);
      v = y[(int64_t)ry * wy + rx];
    }
    const int64_t idx = td.xoff + (int64_t)R * td.xpitch + C;
    w[idx] = v;
    if (u) u[idx] = v;
    if (zg) zg[(int64_t)Rg * nxc_g + Cg] = v;
  }
}

// The consensus and assembly kernels run over items: rectangles of at most
// CI_PIX global pixels (at most CI_COLS wide) with a fixed set of covering tiles, so the
// tile offsets are uniform per block and every load of a pixel group is
// independent of the others.  The item's pixels are numbered row by row and
// thread t owns pixels t, t + 128, t + 256, ..., so every thread of a block
// has work whatever the item's shape (the overlap bands are narrow).
constexpr int NBR = 128;        // threads per block of the row kernels
constexpr int CI_PIX = 2048, CI_COLS = 512;   // pixels / columns per item at most

// Row and column of pixel p of an item with ncol columns (p < 2^20; inv =
// 1 / ncol in FP32, corrected to the exact quotient).
__device__ __forceinline__ void item_rc(int p, int ncol, float inv, int& r, int& c) {
  r = __float2int_rz((float)p * inv);
  if (r * ncol > p) --r;
  else if ((r + 1) * ncol <= p) ++r;
  c = p - r * ncol;
}
constexpr int HUB_ROWS = 4;     // tile rows per block of the prior kernel

// Per global x pixel: zbar = sum_i alpha_i (2 x_i - u_i) / sum_i alpha_i over
// the NS tiles covering it, then u_i <- u_i + rho (zbar - x_i).  With
// partials: FP64 block sums of (x_i - zbar)^2 and (zbar - zbar_prev)^2 (each
// thread adds a group's FP32 sum in FP64).
template <int NS>
__device__ __forceinline__ void consensus_item(const GridArgs& G, const ConsItem& it,
                                               const float* __restrict__ x, float* __restrict__ u,
                                               float gamma, float rho, float* __restrict__ zg,
                                               double& pp, double& dd) {
  constexpr int GP = 8 / NS;       // pixels per group
  const int tx = threadIdx.x;
  const int npix = it.nrow * it.ncol;
  const float inv = 1.f / (float)it.ncol;
  for (int p0 = 0; p0 < npix; p0 += GP * NBR) {
    float xs[GP][NS], us[GP][NS], as[GP][NS], zp[GP];
    int rs[GP], cs[GP];
#pragma unroll
    for (int g = 0; g < GP; ++g) {
      const int p = p0 + g * NBR + tx;
      const bool in = p < npix;
      item_rc(in ? p : 0, it.ncol, inv, rs[g], cs[g]);
      const int r = rs[g];
      const int R = it.r0 + r, C = it.c0 + cs[g];
      zp[g] = (in && zg) ? zg[(int64_t)R * G.nxc + C] : 0.f;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        xs[g][s] = us[g][s] = as[g][s] = 0.f;
        if (in) {
          const int64_t id = it.base[s] + (int64_t)r * it.pitch[s] + C;
          xs[g][s] = x[id];
          us[g][s] = u[id];
          // one covering tile: its weight cancels in the average
          if constexpr (NS > 1) as[g][s] = gamma * G.omr[it.obr[s] + R] * G.omc[it.obc[s] + C];
        }
      }
    }
    float pg = 0.f, dg = 0.f;
#pragma unroll
    for (int g = 0; g < GP; ++g) {
      if (p0 + g * NBR + tx >= npix) continue;
      const int r = rs[g];
      const int R = it.r0 + r, C = it.c0 + cs[g];
      float z;
      if constexpr (NS == 1) {
        z = 2.f * xs[g][0] - us[g][0];
      } else {
        float num = 0.f, den = 0.f;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          num += as[g][s] * (2.f * xs[g][s] - us[g][s]);
          den += as[g][s];
        }
        z = num / den;
      }
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        u[it.base[s] + (int64_t)r * it.pitch[s] + C] = us[g][s] + rho * (z - xs[g][s]);
        const float d = xs[g][s] - z;
        pg = fmaf(d, d, pg);
      }
      if (zg) {
        const float d = z - zp[g];
        dg = fmaf(d, d, dg);
        zg[(int64_t)R * G.nxc + C] = z;
      }
    }
    pp += (double)pg;
    dd += (double)dg;
  }
}

__global__ void __launch_bounds__(NBR, 6) consensus_kernel(const GridArgs G, const float* __restrict__ x,
                                                        float* __restrict__ u, float gamma, float rho,
                                                        float* __restrict__ zg,
                                                        double* __restrict__ partials) {
  __shared__ double red[NBR / 32];
  const ConsItem it = G.citems[blockIdx.x];
  double pp = 0.0, dd = 0.0;
  if (it.ns == 1)
    consensus_item<1>(G, it, x, u, gamma, rho, zg, pp, dd);
  else if (it.ns == 2)
    consensus_item<2>(G, it, x, u, gamma, rho, zg, pp, dd);
  else
    consensus_item<4>(G, it, x, u, gamma, rho, zg, pp, dd);
  if (partials) {
    const double sp = block_sum(pp, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = sp;
    const double sd = block_sum(dd, red);
    if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = sd;
  }
}

// x_hat = sum_i omega_i x_i / sum_i omega_i over the tiles covering each pixel.
template <int NS>
__device__ __forceinline__ void assemble_item(const GridArgs& G, const ConsItem& it,
                                              const float* __restrict__ x, float* __restrict__ out) {
  constexpr int GP = 16 / NS;
  const int tx = threadIdx.x;
  const int npix = it.nrow * it.ncol;
  const float inv = 1.f / (float)it.ncol;
  for (int p0 = 0; p0 < npix; p0 += GP * NBR) {
    float num[GP], den[GP];
    int rs[GP], cs[GP];
#pragma unroll
    for (int g = 0; g < GP; ++g) {
      const int p = p0 + g * NBR + tx;
      num[g] = den[g] = 0.f;
      item_rc(p < npix ? p : 0, it.ncol, inv, rs[g], cs[g]);
      if (p >= npix) continue;
      const int r = rs[g];
      const int R = it.r0 + r, C = it.c0 + cs[g];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const float om = G.omr[it.obr[s] + R] * G.omc[it.obc[s] + C];
        num[g] += om * x[it.base[s] + (int64_t)r * it.pitch[s] + C];
        den[g] += om;
      }
    }
#pragma unroll
    for (int g = 0; g < GP; ++g)
      if (p0 + g * NBR + tx < npix)
        out[(int64_t)(it.r0 + rs[g]) * G.nxc + it.c0 + cs[g]] = num[g] / den[g];
  }
}

__global__ void __launch_bounds__(NBR) assemble_kernel(const GridArgs G, const float* __restrict__ x,
                                                       float* __restrict__ out) {
  const ConsItem it = G.citems[blockIdx.x];
  if (it.ns == 1)
    assemble_item<1>(G, it, x, out);
  else if (it.ns == 2)
    assemble_item<2>(G, it, x, out);
  else
    assemble_item<4>(G, it, x, out);
}

// FP64 block partials of sum_l hub(|grad x(l)|) over every tile of the stack
// (forward differences, zero on each tile's last row / column).  A block owns
// HUB_ROWS rows of one tile; each pixel's term is formed in FP32 and each
// thread adds its FP32 row sum in FP64.
__global__ void __launch_bounds__(NBR) huber_value_kernel(const TileDesc* __restrict__ tiles,
                                                          const float* __restrict__ x, float delta,
                                                          double* __restrict__ partials) {
  __shared__ double red[NBR / 32];
  const TileDesc td = tiles[blockIdx.y];
  double acc = 0.0;
  const int r0 = blockIdx.x * HUB_ROWS, r1 = min(r0 + HUB_ROWS, td.nxr);
  for (int R = r0; R < r1; ++R) {
    const float* row = x + td.xoff + (int64_t)R * td.xpitch;
    const bool down = R + 1 < td.nxr;
    float racc = 0.f;
    for (int C = threadIdx.x; C < td.nxc; C += NBR) {
      const float c = row[C];
      const float dr = down ? row[C + td.xpitch] - c : 0.f;
      const float dc = (C + 1 < td.nxc) ? row[C + 1] - c : 0.f;
      const float s2 = dr * dr + dc * dc;
      racc += (s2 <= delta * delta) ? 0.5f * s2 : delta * (sqrtf(s2) - 0.5f * delta);
    }
    acc += (double)racc;
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

struct ReduceArgs {
  const double* parts[8];
  int counts[8];
  int nk;
  double* out;
};

__global__ void __launch_bounds__(NB) reduce_kernel(const ReduceArgs A) {
  __shared__ double red[NB / 32];
  for (int k = 0; k < A.nk; ++k) {
    double s = 0.0;
    for (int i = threadIdx.x; i < A.counts[k]; i += NB) s += A.parts[k][i];
    const double t = block_sum(s, red);
    if (threadIdx.x == 0) A.out[k] = t;
  }
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

}  // namespace

cudaError_t launch_scatter(const GridArgs& g, int n_tiles, int max_nxr, int max_nxc,
                           const float* x0, const float* y, int hy, int wy, int rad, float* w,
                           float* u, cudaStream_t s, float* zg) {
  dim3 grid(cdiv(max_nxc, NB), max_nxr, n_tiles);
  scatter_kernel<<<grid, NB, 0, s>>>(g.tiles, x0, y, hy, wy, rad, g.nxc, w, u, zg);
  return cudaGetLastError();
}

size_t row_smem(int n_tc) { return (size_t)2 * n_tc * (sizeof(int64_t) + 2 * sizeof(float)); }

cudaError_t launch_consensus(const GridArgs& g, const float* x, float* u, float gamma, float rho,
                             float* zbuf, double* partials, cudaStream_t s, int* n_blocks_out) {
  if (n_blocks_out) *n_blocks_out = g.n_citems;
  consensus_kernel<<<g.n_citems, NBR, 0, s>>>(g, x, u, gamma, rho, zbuf, partials);
  return cudaGetLastError();
}

int consensus_blocks(int n_citems) { return n_citems; }
int cons_item_pixels() { return CI_PIX; }
int cons_item_cols() { return CI_COLS; }

cudaError_t launch_assemble(const GridArgs& g, const float* x, float* out, cudaStream_t s) {
  assemble_kernel<<<g.n_citems, NBR, 0, s>>>(g, x, out);
  return cudaGetLastError();
}

int huber_blocks(int n_tiles, int max_nxr, int max_nxc) {
  (void)max_nxc;
  return cdiv(max_nxr, HUB_ROWS) * n_tiles;
}

cudaError_t launch_huber_value(const TileDesc* tiles, int n_tiles, int max_nxr, int max_nxc,
                               const float* x, double delta, double* partials, cudaStream_t s) {
  (void)max_nxc;
  dim3 grid(cdiv(max_nxr, HUB_ROWS), n_tiles);
  huber_value_kernel<<<grid, NBR, 0, s>>>(tiles, x, (float)delta, partials);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double* const* parts, const int* counts, int nk, double* out,
                          cudaStream_t s) {
  ReduceArgs A{};
  A.nk = nk < 8 ? nk : 8;
  for (int k = 0; k < A.nk; ++k) {
    A.parts[k] = parts[k];
    A.counts[k] = counts[k];
  }
  A.out = out;
  reduce_kernel<<<1, NB, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace dv
