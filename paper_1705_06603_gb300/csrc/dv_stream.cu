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

// Per global x pixel: zbar = sum_i alpha_i (2 x_i - u_i) / sum_i alpha_i over
// the (at most 2 x 2) tiles covering it, then u_i <- u_i + rho (zbar - x_i).
// With partials: FP64 block sums of (x_i - zbar)^2 and (zbar - zbar_prev)^2.
__global__ void __launch_bounds__(NB) consensus_kernel(const GridArgs G, const float* __restrict__ x,
                                                       float* __restrict__ u, float gamma, float rho,
                                                       float* __restrict__ zg,
                                                       double* __restrict__ partials) {
  __shared__ double red[NB / 32];
  const int R = blockIdx.y;
  const int C = blockIdx.x * blockDim.x + threadIdx.x;
  double pp = 0.0, dd = 0.0;
  if (C < G.nxc) {
    const int2 rc = G.rowcov[R], cc = G.colcov[C];
    const int trs[2] = {rc.x, rc.y}, tcs[2] = {cc.x, cc.y};
    float xv[4], uv[4];
    int64_t idx[4];
    int n = 0;
    float num = 0.f, den = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (trs[i] < 0) continue;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (tcs[j] < 0) continue;
        const TileDesc& td = G.tiles[trs[i] * G.n_tc + tcs[j]];
        const int lr = R - td.xr0, lc = C - td.xc0;
        const int64_t id = td.xoff + (int64_t)lr * td.xpitch + lc;
        const float xa = x[id], ua = u[id];
        const float al = gamma * G.omr[td.omr_off + lr] * G.omc[td.omc_off + lc];
        num += al * (2.f * xa - ua);
        den += al;
        xv[n] = xa;
        uv[n] = ua;
        idx[n] = id;
        ++n;
      }
    }
    const float z = num / den;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k < n) {
        u[idx[k]] = uv[k] + rho * (z - xv[k]);
        const double e = (double)xv[k] - (double)z;
        pp += e * e;
      }
    }
    if (zg) {
      const int64_t gi = (int64_t)R * G.nxc + C;
      const double e = (double)z - (double)zg[gi];
      dd += e * e;
      zg[gi] = z;
    }
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
__global__ void __launch_bounds__(NB) assemble_kernel(const GridArgs G, const float* __restrict__ x,
                                                      float* __restrict__ out) {
  const int R = blockIdx.y;
  const int C = blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= G.nxc) return;
  const int2 rc = G.rowcov[R], cc = G.colcov[C];
  const int trs[2] = {rc.x, rc.y}, tcs[2] = {cc.x, cc.y};
  float num = 0.f, den = 0.f;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    if (trs[i] < 0) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (tcs[j] < 0) continue;
      const TileDesc& td = G.tiles[trs[i] * G.n_tc + tcs[j]];
      const int lr = R - td.xr0, lc = C - td.xc0;
      const float om = G.omr[td.omr_off + lr] * G.omc[td.omc_off + lc];
      num += om * x[td.xoff + (int64_t)lr * td.xpitch + lc];
      den += om;
    }
  }
  out[(int64_t)R * G.nxc + C] = num / den;
}

// FP64 block partials of sum_l hub(|grad x(l)|) over every tile of the stack
// (forward differences, zero on each tile's last row / column).
__global__ void __launch_bounds__(NB) huber_value_kernel(const TileDesc* __restrict__ tiles,
                                                         const float* __restrict__ x, double delta,
                                                         double* __restrict__ partials) {
  __shared__ double red[NB / 32];
  const TileDesc td = tiles[blockIdx.z];
  const int R = blockIdx.y;
  double acc = 0.0;
  if (R < td.nxr) {
    for (int C = blockIdx.x * blockDim.x + threadIdx.x; C < td.nxc; C += gridDim.x * blockDim.x) {
      const int64_t idx = td.xoff + (int64_t)R * td.xpitch + C;
      const double c0 = x[idx];
      const double dr = (R + 1 < td.nxr) ? (double)x[idx + td.xpitch] - c0 : 0.0;
      const double dc = (C + 1 < td.nxc) ? (double)x[idx + 1] - c0 : 0.0;
      const double s = sqrt(dr * dr + dc * dc);
      acc += (s <= delta) ? 0.5 * s * s : delta * (s - 0.5 * delta);
    }
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0)
    partials[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
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

cudaError_t launch_consensus(const GridArgs& g, const float* x, float* u, float gamma, float rho,
                             float* zbuf, double* partials, cudaStream_t s, int* n_blocks_out) {
  dim3 grid(cdiv(g.nxc, NB), g.nxr);
  if (n_blocks_out) *n_blocks_out = grid.x * grid.y;
  consensus_kernel<<<grid, NB, 0, s>>>(g, x, u, gamma, rho, zbuf, partials);
  return cudaGetLastError();
}

int consensus_blocks(int nxr, int nxc) { return cdiv(nxc, NB) * nxr; }

cudaError_t launch_assemble(const GridArgs& g, const float* x, float* out, cudaStream_t s) {
  dim3 grid(cdiv(g.nxc, NB), g.nxr);
  assemble_kernel<<<grid, NB, 0, s>>>(g, x, out);
  return cudaGetLastError();
}

int huber_blocks(int n_tiles, int max_nxr, int max_nxc) {
  return cdiv(max_nxc, NB) * max_nxr * n_tiles;
}

cudaError_t launch_huber_value(const TileDesc* tiles, int n_tiles, int max_nxr, int max_nxc,
                               const float* x, double delta, double* partials, cudaStream_t s) {
  dim3 grid(cdiv(max_nxc, NB), max_nxr, n_tiles);
  huber_value_kernel<<<grid, NB, 0, s>>>(tiles, x, delta, partials);
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
