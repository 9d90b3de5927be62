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

// The consensus, assembly and prior kernels work row-wise: a block owns one
// global x row (or a few tile rows) and NBR threads stride over its columns,
// so every warp touches 32 consecutive pixels of each tile stack it reads.
constexpr int NBR = 128;   // threads per block of the row kernels
constexpr int GRP = 4;     // pixels per thread and group: loads of a group are issued together
constexpr int HUB_ROWS = 4;  // tile rows per block of the prior kernel

// Column chunks of the row kernels: about 4096 columns each, a multiple of 32.
__host__ __device__ inline int row_chunks(int nxc) { return (nxc + 4095) / 4096; }
__host__ __device__ inline int row_chunk_width(int nxc) {
  const int n = row_chunks(nxc);
  return ((nxc + n - 1) / n + 31) / 32 * 32;
}

// Per block: for the (one or two) tile rows covering global row R and every
// tile column t, the stack offset of global column 0 on that row (sbase), the
// row factor of the profile times `scale` (srow) and the offset of global
// column 0 in the column profile (somc).  Returns the number of tile rows.
__device__ __forceinline__ int stage_row(const GridArgs& G, int R, float scale, int64_t* sbase,
                                         float* srow, int* somc) {
  const int2 rc = G.rowcov[R];
  const int nr = rc.y >= 0 ? 2 : 1;
  for (int e = threadIdx.x; e < nr * G.n_tc; e += blockDim.x) {
    const int i = e / G.n_tc, t = e - i * G.n_tc;
    const TileDesc td = G.tiles[(i ? rc.y : rc.x) * G.n_tc + t];
    const int lr = R - td.xr0;
    sbase[e] = td.xoff + (int64_t)lr * td.xpitch - td.xc0;
    srow[e] = scale * G.omr[td.omr_off + lr];
    somc[e] = td.omc_off - td.xc0;
  }
  __syncthreads();
  return nr;
}

// Per global x pixel: zbar = sum_i alpha_i (2 x_i - u_i) / sum_i alpha_i over
// the (at most 2 x 2) tiles covering it, then u_i <- u_i + rho (zbar - x_i).
// With partials: FP64 block sums of (x_i - zbar)^2 and (zbar - zbar_prev)^2
// (each thread adds a group's FP32 sum of at most 4 x 4 terms in FP64).
__global__ void __launch_bounds__(NBR) consensus_kernel(const GridArgs G, const float* __restrict__ x,
                                                        float* __restrict__ u, float gamma, float rho,
                                                        float* __restrict__ zg,
                                                        double* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red[NBR / 32];
  const int ntc = G.n_tc;
  int64_t* sbase = reinterpret_cast<int64_t*>(dsm);
  float* srow = reinterpret_cast<float*>(sbase + 2 * ntc);
  int* somc = reinterpret_cast<int*>(srow + 2 * ntc);
  const int R = blockIdx.y;
  const int nr = stage_row(G, R, gamma, sbase, srow, somc);
  const int cw = row_chunk_width(G.nxc);
  const int c0 = blockIdx.x * cw, c1 = min(c0 + cw, G.nxc);
  double pp = 0.0, dd = 0.0;
  for (int cb = c0 + threadIdx.x; cb < c1; cb += GRP * NBR) {
    float xs[GRP][4], us[GRP][4], as[GRP][4], zp[GRP];
    int2 cc[GRP];
#pragma unroll
    for (int k = 0; k < GRP; ++k) {
      const int C = cb + k * NBR;
      const bool in = C < c1;
      cc[k] = in ? G.colcov[C] : make_int2(-1, -1);
      zp[k] = (in && zg) ? zg[(int64_t)R * G.nxc + C] : 0.f;
#pragma unroll
      for (int sl = 0; sl < 4; ++sl) {
        const int i = sl >> 1, t = (sl & 1) ? cc[k].y : cc[k].x;
        xs[k][sl] = us[k][sl] = as[k][sl] = 0.f;
        if (in && i < nr && t >= 0) {
          const int e = i * ntc + t;
          const int64_t id = sbase[e] + C;
          xs[k][sl] = x[id];
          us[k][sl] = u[id];
          as[k][sl] = srow[e] * G.omc[somc[e] + C];
        }
      }
    }
    float pg = 0.f, dg = 0.f;
#pragma unroll
    for (int k = 0; k < GRP; ++k) {
      const int C = cb + k * NBR;
      if (C >= c1) continue;
      float num = 0.f, den = 0.f;
#pragma unroll
      for (int sl = 0; sl < 4; ++sl) {
        num += as[k][sl] * (2.f * xs[k][sl] - us[k][sl]);
        den += as[k][sl];
      }
      const float z = num / den;
#pragma unroll
      for (int sl = 0; sl < 4; ++sl) {
        if (as[k][sl] != 0.f) {
          const int e = (sl >> 1) * ntc + ((sl & 1) ? cc[k].y : cc[k].x);
          u[sbase[e] + C] = us[k][sl] + rho * (z - xs[k][sl]);
          const float d = xs[k][sl] - z;
          pg = fmaf(d, d, pg);
        }
      }
      if (zg) {
        const float d = z - zp[k];
        dg = fmaf(d, d, dg);
        zg[(int64_t)R * G.nxc + C] = z;
      }
    }
    pp += (double)pg;
    dd += (double)dg;
  }
  if (partials) {
    const int blk = blockIdx.y * gridDim.x + blockIdx.x, nblk = gridDim.x * gridDim.y;
    const double sp = block_sum(pp, red);
    if (threadIdx.x == 0) partials[blk] = sp;
    const double sd = block_sum(dd, red);
    if (threadIdx.x == 0) partials[nblk + blk] = sd;
  }
}

// x_hat = sum_i omega_i x_i / sum_i omega_i over the tiles covering each pixel.
__global__ void __launch_bounds__(NBR) assemble_kernel(const GridArgs G, const float* __restrict__ x,
                                                       float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int ntc = G.n_tc;
  int64_t* sbase = reinterpret_cast<int64_t*>(dsm);
  float* srow = reinterpret_cast<float*>(sbase + 2 * ntc);
  int* somc = reinterpret_cast<int*>(srow + 2 * ntc);
  const int R = blockIdx.y;
  const int nr = stage_row(G, R, 1.f, sbase, srow, somc);
  const int cw = row_chunk_width(G.nxc);
  const int c0 = blockIdx.x * cw, c1 = min(c0 + cw, G.nxc);
  for (int cb = c0 + threadIdx.x; cb < c1; cb += GRP * NBR) {
    float num[GRP], den[GRP];
#pragma unroll
    for (int k = 0; k < GRP; ++k) {
      const int C = cb + k * NBR;
      num[k] = den[k] = 0.f;
      if (C >= c1) continue;
      const int2 cc = G.colcov[C];
#pragma unroll
      for (int sl = 0; sl < 4; ++sl) {
        const int i = sl >> 1, t = (sl & 1) ? cc.y : cc.x;
        if (i < nr && t >= 0) {
          const int e = i * ntc + t;
          const float om = srow[e] * G.omc[somc[e] + C];
          num[k] += om * x[sbase[e] + C];
          den[k] += om;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < GRP; ++k) {
      const int C = cb + k * NBR;
      if (C < c1) out[(int64_t)R * G.nxc + C] = num[k] / den[k];
    }
  }
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
  dim3 grid(row_chunks(g.nxc), g.nxr);
  if (n_blocks_out) *n_blocks_out = grid.x * grid.y;
  consensus_kernel<<<grid, NBR, row_smem(g.n_tc), s>>>(g, x, u, gamma, rho, zbuf, partials);
  return cudaGetLastError();
}

int consensus_blocks(int nxr, int nxc) { return row_chunks(nxc) * nxr; }

cudaError_t launch_assemble(const GridArgs& g, const float* x, float* out, cudaStream_t s) {
  dim3 grid(row_chunks(g.nxc), g.nxr);
  assemble_kernel<<<grid, NBR, row_smem(g.n_tc), s>>>(g, x, out);
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
