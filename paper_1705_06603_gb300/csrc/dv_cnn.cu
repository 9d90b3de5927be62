// Learned warm start of Algorithm 1: a small convolutional network that maps
// the observed image and PSF descriptor maps to a correction of the start
// image, x0 = max(0, y_pad + net(features)).  Hand-written kernels:
//   - the forward pass, in training and inference alike (the solve's warm
//     start, dv_cnn_forward), as implicit GEMMs on the tensor cores (tcgen05,
//     BF16 weights and activations, FP32 accumulators in tensor memory);
//   - backward data (a 3x3 convolution on CUDA cores with the flipped,
//     transposed weights and the ReLU mask of the layer input fused in),
//     backward weights (per-tile partial sums reduced in a fixed order),
//     mean-squared-error loss, Adam.
// Architecture: 5 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1 channels, ReLU between
// layers, none after the last.  The first layer's 5 input channels are padded
// to 8 with zeros.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>

#include "dv_internal.cuh"
#include "dv_tcgen05.cuh"

namespace dv {
namespace {

using bf16 = __nv_bfloat16;

constexpr int TS = 16;             // output tile side
constexpr int HALO = TS + 2;
constexpr int NTH = 128;           // threads per conv CTA: 16 columns x 8 row pairs
constexpr int WID = 32;            // hidden width
constexpr int CIN0 = 8;            // padded input channels
constexpr int NLAYER = 6;
constexpr int NB = 256;

__host__ __device__ constexpr int layer_cin(int l) { return l == 0 ? CIN0 : WID; }
__host__ __device__ constexpr int layer_cout(int l) { return l == NLAYER - 1 ? 1 : WID; }
constexpr int layer_cin_logical(int l) { return l == 0 ? DV_CNN_IN_CH : WID; }

__device__ __forceinline__ float tof(const bf16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float tof(const float v) { return v; }
__device__ __forceinline__ void store(float* p, float v) { *p = v; }

size_t conv_smem(int cin, int cout) {
  return sizeof(float) * ((size_t)cin * HALO * HALO + (size_t)9 * cin * cout + cout);
}

// out[n,y,x,o] = act(b[o] + sum_{dy,dx,i} w[dy*3+dx][i][o] in[n, y+dy-1, x+dx-1, i])
// optionally multiplied by (mask[n,y,x,o] > 0).  Each thread computes the
// COUT outputs of two vertically adjacent pixels of a 16x16 tile.
template <int CIN, int COUT, typename TIN, typename TOUT, bool RELU, bool MASK>
__global__ void __launch_bounds__(NTH) conv_kernel(const TIN* __restrict__ in,
                                                   const float* __restrict__ w,
                                                   const float* __restrict__ bias,
                                                   const bf16* __restrict__ mask,
                                                   TOUT* __restrict__ out, int H, int W) {
  extern __shared__ __align__(16) float smem[];
  float* sx = smem;                          // [CIN][HALO*HALO], channel-major
  float* sw = sx + CIN * HALO * HALO;        // [9][CIN][COUT]
  float* sb = sw + 9 * CIN * COUT;
  const int n = blockIdx.z, y0 = blockIdx.y * TS, x0 = blockIdx.x * TS;
  const int tid = threadIdx.x;
  for (int e = tid; e < 9 * CIN * COUT; e += NTH) sw[e] = w[e];
  for (int e = tid; e < COUT; e += NTH) sb[e] = bias ? bias[e] : 0.f;
  for (int e = tid; e < HALO * HALO * CIN; e += NTH) {
    const int pix = e / CIN, ci = e - pix * CIN;
    const int yy = y0 - 1 + pix / HALO, xx = x0 - 1 + pix % HALO;
    float v = 0.f;
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = tof(in[(((int64_t)n * H + yy) * W + xx) * CIN + ci]);
    sx[ci * HALO * HALO + pix] = v;
  }
  __syncthreads();
  const int tx = tid & (TS - 1), ty = (tid >> 4) * 2;
  float acc0[COUT], acc1[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc0[o] = acc1[o] = sb[o];
#pragma unroll 1
  for (int tap = 0; tap < 9; ++tap) {
    const int dy = tap / 3, dx = tap - dy * 3;
    const float* xr = sx + (ty + dy) * HALO + tx + dx;
#pragma unroll 4
    for (int ci = 0; ci < CIN; ++ci) {
      const float v0 = xr[ci * HALO * HALO], v1 = xr[ci * HALO * HALO + HALO];
      const float* wr = sw + (tap * CIN + ci) * COUT;
      if constexpr (COUT % 4 == 0) {
#pragma unroll
        for (int o = 0; o < COUT; o += 4) {
          const float4 q = *reinterpret_cast<const float4*>(wr + o);
          acc0[o] = fmaf(q.x, v0, acc0[o]);
          acc0[o + 1] = fmaf(q.y, v0, acc0[o + 1]);
          acc0[o + 2] = fmaf(q.z, v0, acc0[o + 2]);
          acc0[o + 3] = fmaf(q.w, v0, acc0[o + 3]);
          acc1[o] = fmaf(q.x, v1, acc1[o]);
          acc1[o + 1] = fmaf(q.y, v1, acc1[o + 1]);
          acc1[o + 2] = fmaf(q.z, v1, acc1[o + 2]);
          acc1[o + 3] = fmaf(q.w, v1, acc1[o + 3]);
        }
      } else {
#pragma unroll
        for (int o = 0; o < COUT; ++o) {
          acc0[o] = fmaf(wr[o], v0, acc0[o]);
          acc1[o] = fmaf(wr[o], v1, acc1[o]);
        }
      }
    }
  }
  const int xx = x0 + tx;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int yy = y0 + ty + r;
    if (yy >= H || xx >= W) continue;
    const int64_t base = (((int64_t)n * H + yy) * W + xx) * COUT;
#pragma unroll
    for (int o = 0; o < COUT; ++o) {
      float v = r == 0 ? acc0[o] : acc1[o];
      if (RELU) v = fmaxf(v, 0.f);
      if (MASK && !(tof(mask[base + o]) > 0.f)) v = 0.f;
      store(out + base + o, v);
    }
  }
}

// Per 16x16 tile: partial dW[tap][i][o] = sum_p in[p + off(tap)][i] dz[p][o]
// and partial db[o] = sum_p dz[p][o].  Thread t < 9*CIN owns (tap, i).
template <int CIN, int COUT>
__global__ void __launch_bounds__(NB) wgrad_kernel(const bf16* __restrict__ in,
                                                   const float* __restrict__ dz,
                                                   float* __restrict__ part, int H, int W) {
  extern __shared__ __align__(16) float smem[];
  float* sx = smem;                        // [CIN][HALO*HALO]
  float* sd = sx + CIN * HALO * HALO;      // [TS*TS][COUT]
  const int n = blockIdx.z, y0 = blockIdx.y * TS, x0 = blockIdx.x * TS;
  const int tid = threadIdx.x;
  for (int e = tid; e < HALO * HALO * CIN; e += NB) {
    const int pix = e / CIN, ci = e - pix * CIN;
    const int yy = y0 - 1 + pix / HALO, xx = x0 - 1 + pix % HALO;
    float v = 0.f;
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = tof(in[(((int64_t)n * H + yy) * W + xx) * CIN + ci]);
    sx[ci * HALO * HALO + pix] = v;
  }
  for (int e = tid; e < TS * TS * COUT; e += NB) {
    const int pix = e / COUT, o = e - pix * COUT;
    const int yy = y0 + pix / TS, xx = x0 + pix % TS;
    sd[e] = (yy < H && xx < W) ? dz[(((int64_t)n * H + yy) * W + xx) * COUT + o] : 0.f;
  }
  __syncthreads();
  const int nblk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  float* out = part + (int64_t)nblk * (9 * CIN * COUT + COUT);
  for (int t = tid; t < 9 * CIN; t += NB) {
    const int tap = t / CIN, ci = t - tap * CIN;
    const int dy = tap / 3, dx = tap - dy * 3;
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = 0.f;
    const float* xr = sx + ci * HALO * HALO + dy * HALO + dx;
#pragma unroll 2
    for (int p = 0; p < TS * TS; ++p) {
      const float v = xr[(p / TS) * HALO + (p % TS)];
      const float* d = sd + p * COUT;
#pragma unroll
      for (int o = 0; o < COUT; ++o) acc[o] = fmaf(v, d[o], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < COUT; ++o) out[(tap * CIN + ci) * COUT + o] = acc[o];
  }
  for (int o = tid; o < COUT; o += NB) {
    float s = 0.f;
    for (int p = 0; p < TS * TS; ++p) s += sd[p * COUT + o];
    out[9 * CIN * COUT + o] = s;
  }
}

// grad[k] = sum_{b < nblk} part[b][k] in a fixed order.
__global__ void reduce_cols_kernel(const float* __restrict__ part, int nblk, int ncol,
                                   float* __restrict__ grad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ncol) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * ncol + k];
  grad[k] = s;
}

// dz = (out - target) / npix; FP64 block partials of (out - target)^2.
__global__ void __launch_bounds__(NB) mse_kernel(const float* __restrict__ out,
                                                 const float* __restrict__ target, int64_t n,
                                                 float* __restrict__ dz, double* __restrict__ part) {
  __shared__ double red[NB / 32];
  double acc = 0.0;
  const float inv = 1.0f / (float)n;
  for (int64_t i = blockIdx.x * (int64_t)NB + threadIdx.x; i < n; i += (int64_t)gridDim.x * NB) {
    const float d = out[i] - target[i];
    dz[i] = d * inv;
    acc += (double)d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < NB / 32; ++i) s += red[i];
    part[blockIdx.x] = s;
  }
}

// *out = sum of the n partials (one block of NB threads, fixed order).
__global__ void __launch_bounds__(NB) sum_kernel(const double* __restrict__ part, int n,
                                                 double* __restrict__ out) {
  __shared__ double red[NB];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += NB) t += part[i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int w = NB / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Adam on the FP32 master parameters (bias-corrected; t counts from 1).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Compute copies of one layer's weights, rounded to bfloat16:
//   wf[tap][i][o]  (forward, i padded to cin_p)
//   wt[tap][o][i]  (backward data: taps flipped, channels transposed)
__global__ void pack_kernel(const float* __restrict__ wl, int cin, int cin_p, int cout,
                            float* __restrict__ wf, float* __restrict__ wt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 9 * cin_p * cout) return;
  const int tap = e / (cin_p * cout), r = e - tap * cin_p * cout;
  const int i = r / cout, o = r - i * cout;
  const float v = i < cin ? __bfloat162float(__float2bfloat16_rn(wl[(tap * cin + i) * cout + o])) : 0.f;
  wf[e] = v;
  if (wt) wt[((8 - tap) * cout + o) * cin_p + i] = v;
}

// FP32 input (n, 5 channels) -> bfloat16 (n, 8 channels, zeros beyond 5).
__global__ void input_kernel(const float* __restrict__ in, int64_t npix, bf16* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npix * CIN0) return;
  const int64_t p = i / CIN0;
  const int c = (int)(i - p * CIN0);
  out[i] = __float2bfloat16_rn(c < DV_CNN_IN_CH ? in[p * DV_CNN_IN_CH + c] : 0.f);
}

// One training batch from a crop table: xb [b][r][c][5] and tb [b][r][c] =
// the crop x crop window at (r0, c0) of pair crops[b] = {pair, r0, c0}.
__global__ void gather_crops_kernel(const float* __restrict__ feats, const float* __restrict__ targets,
                                    int H, int W, const int* __restrict__ crops, int batch, int crop,
                                    float* __restrict__ xb, float* __restrict__ tb) {
  const int64_t n = (int64_t)batch * crop * crop;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = (int)(i / ((int64_t)crop * crop));
  const int rem = (int)(i - (int64_t)b * crop * crop), r = rem / crop, c = rem - r * crop;
  const int* cb = crops + 3 * b;
  const int64_t src = ((int64_t)cb[0] * H + cb[1] + r) * W + cb[2] + c;
  tb[i] = targets[src];
#pragma unroll
  for (int ch = 0; ch < DV_CNN_IN_CH; ++ch) xb[i * DV_CNN_IN_CH + ch] = feats[src * DV_CNN_IN_CH + ch];
}

// Warm-start features of the global x grid (reading of the inputs in the
// header): [y edge-replicated, 3 interpolated PSF descriptors, 100 sigma].
__global__ void features_kernel(const float* __restrict__ y, int hy, int wy, int rad,
                                const WTab* __restrict__ wrow, const WTab* __restrict__ wcol,
                                const float* __restrict__ desc, int Gr, int Gc, float sig100,
                                int nxr, int nxc, float* __restrict__ f) {
  const int C = blockIdx.x * blockDim.x + threadIdx.x, R = blockIdx.y;
  if (C >= nxc) return;
  const int64_t o = ((int64_t)R * nxc + C) * DV_CNN_IN_CH;
  const int ry = min(max(R - rad, 0), hy - 1), rx = min(max(C - rad, 0), wy - 1);
  f[o] = y[(int64_t)ry * wy + rx];
  const WTab tr = wrow[R], tc = wcol[C];
  float m[3] = {0.f, 0.f, 0.f};
  for (int da = 0; da < 2; ++da) {
    const int a = tr.a0 + da;
    if (a >= Gr) continue;
    const float wa = da ? tr.w1 : tr.w0;
    for (int db = 0; db < 2; ++db) {
      const int b = tc.a0 + db;
      if (b >= Gc) continue;
      const float wgt = wa * (db ? tc.w1 : tc.w0);
      for (int k = 0; k < 3; ++k) m[k] = fmaf(wgt, desc[(a * Gc + b) * 3 + k], m[k]);
    }
  }
  f[o + 1] = m[0];
  f[o + 2] = m[1];
  f[o + 3] = m[2];
  f[o + 4] = sig100;
}

// x0 = max(0, f[., 0] + d) on the global x grid
__global__ void apply_warm_kernel(const float* __restrict__ f, const float* __restrict__ d,
                                  int64_t n, float* __restrict__ x0) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x0[i] = fmaxf(0.f, f[i * DV_CNN_IN_CH] + d[i]);
}

// ---------------------------------------------------------------------------
// Tensor-core 3x3 convolution (inference).  A CTA owns 4 image rows x 128
// pixels; per output row r, tap (dy, dx) and 16-channel k-step, one
// tcgen05.mma (M = 128 pixels, N = NP output channels, K = 16 channels):
//   A = staged input pixels of row r + dy starting at column dx, K-major, no
//       swizzle: the 6 x 130 staged pixels of each 8-channel chunk form a
//       panel with pixels 16 bytes apart, so (r + dy, dx) is a start offset;
//   B = the layer's weights of that tap and k-step, NP rows x 16 channels,
//       resident in shared memory for the whole CTA.
// Accumulator row r lives in tensor-memory columns [r NP, r NP + NP); lane =
// pixel.  Thread 0 issues the MMAs; the 4 warps stage and run the epilogue
// (bias, ReLU, BF16 or FP32 NHWC store).
constexpr int TCR = 4;              // output rows per CTA
constexpr int TCW = 128;            // output pixels per row (MMA M)
constexpr int TCSP = (TCR + 2) * (TCW + 2);   // staged pixels
constexpr int TCTH = 128;

template <int CINP, int NP>
struct ConvTC {
  static constexpr int NPAN = CINP / 8;                 // 8-channel panels of A
  static constexpr int APANEL = TCSP * 16 + 16;
  static constexpr int KS = CINP / 16;                  // k-steps per tap
  static constexpr int BSTEP = 2 * NP * 16;             // bytes of B per (tap, k-step)
  static constexpr int BBYTES = 9 * KS * BSTEP;
  // padded so that at most 4 CTAs (128 tensor-memory columns at most each)
  // share an SM and tcgen05.alloc never waits
  static constexpr int SMEM0 = 64 + NPAN * APANEL + BBYTES + NP * 4;
  static constexpr int SMEM = SMEM0 > 58 * 1024 ? SMEM0 : 58 * 1024;
  static constexpr int TMEM = TCR * NP <= 32 ? 32 : (TCR * NP <= 64 ? 64 : 128);
};

// B images of one layer: [tap][k-step][panel][o < NP][8 channels] BF16 from
// the BF16-rounded forward weights wf[tap][i < cin_p][o < cout] (zero beyond).
__global__ void pack_tc_kernel(const float* __restrict__ wf, int cin_p, int cout, int cinp_tc, int np,
                               bf16* __restrict__ out) {
  const int ks_n = cinp_tc / 16;
  const int n = 9 * ks_n * 2 * np * 8;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int ch = e % 8, o = (e / 8) % np, pn = (e / (8 * np)) % 2, ks = (e / (16 * np)) % ks_n,
            tap = e / (16 * np * ks_n);
  const int i = 16 * ks + 8 * pn + ch;
  out[e] = __float2bfloat16_rn(i < cin_p && o < cout ? wf[(tap * cin_p + i) * cout + o] : 0.f);
}

template <int CINP, int NP, int COUT, bool RELU, bool OUTF32>
__global__ void __launch_bounds__(TCTH) tconv_kernel(const bf16* __restrict__ in, int cin,
                                                     const bf16* __restrict__ wtc,
                                                     const float* __restrict__ bias,
                                                     void* __restrict__ out, int H, int W,
                                                     int* err) {
  using G = ConvTC<CINP, NP>;
  using namespace tcg;
  extern __shared__ __align__(1024) unsigned char tsm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(tsm);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tsm + 8);
  int* abort_flag = reinterpret_cast<int*>(tsm + 16);
  unsigned char* sA = tsm + 64;
  unsigned char* sB = sA + G::NPAN * G::APANEL;
  float* sBias = reinterpret_cast<float*>(sB + G::BBYTES);
  const int n = blockIdx.z, y0 = blockIdx.y * TCR, x0 = blockIdx.x * TCW;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, G::TMEM);
  // weights and bias
  for (int e = tid; e < G::BBYTES / 16; e += TCTH)
    reinterpret_cast<uint4*>(sB)[e] = reinterpret_cast<const uint4*>(wtc)[e];
  for (int e = tid; e < NP; e += TCTH) sBias[e] = e < COUT ? bias[e] : 0.f;
  // input pixels (rows y0 - 1 .. y0 + TCR, columns x0 - 1 .. x0 + TCW), 8 channels per panel
  for (int e = tid; e < TCSP * G::NPAN; e += TCTH) {
    const int p = e / G::NPAN, q = e - p * G::NPAN;
    const int yy = y0 - 1 + p / (TCW + 2), xx = x0 - 1 + p % (TCW + 2);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (yy >= 0 && yy < H && xx >= 0 && xx < W && 8 * q < cin)
      v = *reinterpret_cast<const uint4*>(in + (((int64_t)n * H + yy) * W + xx) * cin + 8 * q);
    *reinterpret_cast<uint4*>(sA + (size_t)q * G::APANEL + p * 16) = v;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  if (tid == 0) {
    const uint32_t id = idesc(1, TCW, NP);
    const uint64_t a0 = sdesc(saddr(sA), G::APANEL);
    const uint64_t b0 = sdesc(saddr(sB), NP * 16);
    for (int r = 0; r < TCR; ++r) {
      bool first = true;
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap - 3 * dy;
#pragma unroll
        for (int ks = 0; ks < G::KS; ++ks) {
          const uint64_t ad = a0 + (uint64_t)(2 * ks * (G::APANEL >> 4) + (r + dy) * (TCW + 2) + dx);
          const uint64_t bd = b0 + (uint64_t)((tap * G::KS + ks) * (G::BSTEP >> 4));
          mma_bf16(tbase + (uint32_t)(r * NP), ad, bd, id, first ? 0u : 1u);
          first = false;
        }
      }
    }
    tc_commit(bar);
  }
  __syncwarp();
  const bool ok = wait_bar(bar, 0, abort_flag, err);
  tc_fence_after();
  const int xx = x0 + 32 * warp + lane;
  const uint32_t lanes = (uint32_t)(32 * warp) << 16;
  for (int r = 0; r < TCR && ok; ++r) {
    float v[NP];
    if constexpr (NP == 32) {
      float t[32];
      tmem_ld32(tbase + lanes + (uint32_t)(r * NP), t);
#pragma unroll
      for (int o = 0; o < 32; ++o) v[o] = t[o];
    } else {
      uint32_t t[16];
      tmem_ld16_nowait(tbase + lanes + (uint32_t)(r * NP), t);
      tmem_wait_ld();
#pragma unroll
      for (int o = 0; o < 16; ++o) v[o] = __uint_as_float(t[o]);
    }
    const int yy = y0 + r;
    if (yy >= H || xx >= W) continue;
    const int64_t pix = ((int64_t)n * H + yy) * W + xx;
    if constexpr (OUTF32) {
      float* o = reinterpret_cast<float*>(out) + pix * COUT;
#pragma unroll
      for (int c = 0; c < COUT; ++c) o[c] = RELU ? fmaxf(v[c] + sBias[c], 0.f) : v[c] + sBias[c];
    } else {
      static_assert(COUT % 8 == 0, "BF16 output in 16-byte groups");
      uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(out) + pix * COUT);
#pragma unroll
      for (int g = 0; g < COUT / 8; ++g) {
        uint32_t wv[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          float a = v[8 * g + 2 * h] + sBias[8 * g + 2 * h];
          float b = v[8 * g + 2 * h + 1] + sBias[8 * g + 2 * h + 1];
          if (RELU) {
            a = fmaxf(a, 0.f);
            b = fmaxf(b, 0.f);
          }
          const __nv_bfloat162 hb = __floats2bfloat162_rn(a, b);
          wv[h] = *reinterpret_cast<const uint32_t*>(&hb);
        }
        o[g] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_free(tbase, G::TMEM);
  }
}

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace
}  // namespace dv

struct dv_cnn {
  int64_t nparam = 0;
  int64_t off_w[dv::NLAYER], off_b[dv::NLAYER];
  float* d_p = nullptr;       // FP32 master parameters (logical layout)
  float* d_g = nullptr;       // gradients
  float* d_m = nullptr;       // Adam moments
  float* d_v = nullptr;
  float* d_wf[dv::NLAYER] = {};  // bfloat16-rounded compute weights
  float* d_wt[dv::NLAYER] = {};
  dv::bf16* d_wtc[dv::NLAYER] = {};   // tensor-core B images (inference)
  int* d_err = nullptr;               // bounded-wait error word of the tensor-core kernels
  int64_t step = 0;
  // activation buffers (grown on demand)
  int64_t cap_pix = 0;
  dv::bf16* d_act[dv::NLAYER] = {};  // layer inputs: [0] 8 channels, others 32
  float* d_out = nullptr;
  float* d_dz[2] = {nullptr, nullptr};
  float* d_part = nullptr;
  int64_t cap_part = 0;
  double* d_lpart = nullptr;
  double* d_loss = nullptr;
  double* h_loss = nullptr;
  bool packed = false;
};

namespace dv {
namespace {

template <int CIN, int COUT, typename TIN, typename TOUT, bool RELU, bool MASK>
cudaError_t conv_launch(const TIN* in, const float* w, const float* b, const bf16* mask, TOUT* out,
                        int N, int H, int W, cudaStream_t s) {
  const size_t smem = conv_smem(CIN, COUT);
  cudaError_t e = cudaFuncSetAttribute(conv_kernel<CIN, COUT, TIN, TOUT, RELU, MASK>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(cdiv(W, TS), cdiv(H, TS), N);
  conv_kernel<CIN, COUT, TIN, TOUT, RELU, MASK><<<grid, NTH, smem, s>>>(in, w, b, mask, out, H, W);
  return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t wgrad_launch(const bf16* in, const float* dz, float* part, float* grad_w, float* grad_b,
                         int N, int H, int W, cudaStream_t s) {
  const size_t smem = sizeof(float) * ((size_t)CIN * HALO * HALO + (size_t)TS * TS * COUT);
  cudaError_t e = cudaFuncSetAttribute(wgrad_kernel<CIN, COUT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(cdiv(W, TS), cdiv(H, TS), N);
  wgrad_kernel<CIN, COUT><<<grid, NB, smem, s>>>(in, dz, part, H, W);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nblk = grid.x * grid.y * grid.z, ncol = 9 * CIN * COUT + COUT;
  // columns of the padded layout map to the logical layout: only i < cin is kept
  (void)grad_w;
  (void)grad_b;
  reduce_cols_kernel<<<cdiv(ncol, NB), NB, 0, s>>>(part, nblk, ncol, part + (int64_t)nblk * ncol);
  return cudaGetLastError();
}

// Copies a reduced padded-layout gradient (9*cin_p*cout + cout) to the logical layout.
__global__ void unpad_grad_kernel(const float* __restrict__ src, int cin, int cin_p, int cout,
                                  float* __restrict__ gw, float* __restrict__ gb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 9 * cin * cout) {
    const int tap = e / (cin * cout), r = e - tap * cin * cout;
    const int i = r / cout, o = r - i * cout;
    gw[e] = src[(tap * cin_p + i) * cout + o];
  } else if (e < 9 * cin * cout + cout) {
    gb[e - 9 * cin * cout] = src[9 * cin_p * cout + (e - 9 * cin * cout)];
  }
}

dv_status ensure_capacity(dv_cnn* c, int64_t npix, int64_t nblk) {
  if (npix > c->cap_pix) {
    for (int l = 0; l < NLAYER; ++l)
      if (c->d_act[l]) cudaFree(c->d_act[l]);
    for (float* p : {c->d_out, c->d_dz[0], c->d_dz[1]})
      if (p) cudaFree(p);
    for (int l = 0; l < NLAYER; ++l)
      DV_TRY_CUDA(cudaMalloc(&c->d_act[l], (size_t)npix * layer_cin(l) * sizeof(bf16)));
    DV_TRY_CUDA(cudaMalloc(&c->d_out, (size_t)npix * sizeof(float)));
    DV_TRY_CUDA(cudaMalloc(&c->d_dz[0], (size_t)npix * WID * sizeof(float)));
    DV_TRY_CUDA(cudaMalloc(&c->d_dz[1], (size_t)npix * WID * sizeof(float)));
    c->cap_pix = npix;
  }
  const int64_t need = nblk * (9 * WID * WID + WID) + (9 * WID * WID + WID);
  if (need > c->cap_part) {
    if (c->d_part) cudaFree(c->d_part);
    DV_TRY_CUDA(cudaMalloc(&c->d_part, (size_t)need * sizeof(float)));
    c->cap_part = need;
  }
  return DV_OK;
}

__host__ __device__ constexpr int tc_cinp(int l) { return l == 0 ? 16 : WID; }
__host__ __device__ constexpr int tc_np(int l) { return l == NLAYER - 1 ? 16 : WID; }

dv_status pack(dv_cnn* c, cudaStream_t s) {
  for (int l = 0; l < NLAYER; ++l) {
    const int n = 9 * layer_cin(l) * layer_cout(l);
    pack_kernel<<<cdiv(n, NB), NB, 0, s>>>(c->d_p + c->off_w[l], layer_cin_logical(l), layer_cin(l),
                                           layer_cout(l), c->d_wf[l], c->d_wt[l]);
    DV_TRY_CUDA(cudaGetLastError());
    const int nt = 9 * tc_cinp(l) * tc_np(l);
    pack_tc_kernel<<<cdiv(nt, NB), NB, 0, s>>>(c->d_wf[l], layer_cin(l), layer_cout(l), tc_cinp(l),
                                               tc_np(l), c->d_wtc[l]);
    DV_TRY_CUDA(cudaGetLastError());
  }
  c->packed = true;
  return DV_OK;
}

template <int CINP, int NP, int COUT, bool RELU, bool OUTF32>
cudaError_t tconv_launch(const bf16* in, int cin, const bf16* wtc, const float* b, void* out, int N,
                         int H, int W, int* err, cudaStream_t s) {
  using G = ConvTC<CINP, NP>;
  cudaError_t e = cudaFuncSetAttribute(tconv_kernel<CINP, NP, COUT, RELU, OUTF32>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(cdiv(W, TCW), cdiv(H, TCR), N);
  tconv_kernel<CINP, NP, COUT, RELU, OUTF32><<<grid, TCTH, G::SMEM, s>>>(in, cin, wtc, b, out, H, W, err);
  return cudaGetLastError();
}

// Inference pass on tensor cores (same layers; activations in the training
// buffers, not kept consistent with the backward pass).
dv_status forward_tc(dv_cnn* c, const float* in, int N, int H, int W, float* out, int* err,
                     cudaStream_t s) {
  const int64_t npix = (int64_t)N * H * W;
  DV_TRY(ensure_capacity(c, npix, (int64_t)N * cdiv(H, TS) * cdiv(W, TS)));
  if (!c->packed) DV_TRY(pack(c, s));
  input_kernel<<<cdiv(npix * CIN0, NB), NB, 0, s>>>(in, npix, c->d_act[0]);
  DV_TRY_CUDA(cudaGetLastError());
  DV_TRY_CUDA((tconv_launch<16, WID, WID, true, false>(c->d_act[0], CIN0, c->d_wtc[0],
                                                      c->d_p + c->off_b[0], c->d_act[1], N, H, W,
                                                      err, s)));
  for (int l = 1; l < NLAYER - 1; ++l)
    DV_TRY_CUDA((tconv_launch<WID, WID, WID, true, false>(c->d_act[l], WID, c->d_wtc[l],
                                                         c->d_p + c->off_b[l], c->d_act[l + 1], N,
                                                         H, W, err, s)));
  DV_TRY_CUDA((tconv_launch<WID, 16, 1, false, true>(c->d_act[NLAYER - 1], WID, c->d_wtc[NLAYER - 1],
                                                    c->d_p + c->off_b[NLAYER - 1],
                                                    out ? out : c->d_out, N, H, W, err, s)));
  return DV_OK;
}

// Loss and gradients (into d_g) for the last forward pass.
dv_status backward(dv_cnn* c, const float* target, int N, int H, int W, cudaStream_t s) {
  const int64_t npix = (int64_t)N * H * W;
  const int grid = std::min(cdiv(npix, NB), 1024);
  mse_kernel<<<grid, NB, 0, s>>>(c->d_out, target, npix, c->d_dz[0], c->d_lpart);
  DV_TRY_CUDA(cudaGetLastError());
  sum_kernel<<<1, NB, 0, s>>>(c->d_lpart, grid, c->d_loss);
  DV_TRY_CUDA(cudaGetLastError());
  const int nblk = N * cdiv(H, TS) * cdiv(W, TS);
  int cur = 0;   // d_dz[cur] holds dL/dz of layer l
  for (int l = NLAYER - 1; l >= 0; --l) {
    const int cin = layer_cin(l), cout = layer_cout(l), ncol = 9 * cin * cout + cout;
    if (l == NLAYER - 1)
      DV_TRY_CUDA((wgrad_launch<WID, 1>(c->d_act[l], c->d_dz[cur], c->d_part, nullptr, nullptr, N, H, W, s)));
    else if (l == 0)
      DV_TRY_CUDA((wgrad_launch<CIN0, WID>(c->d_act[l], c->d_dz[cur], c->d_part, nullptr, nullptr, N, H, W, s)));
    else
      DV_TRY_CUDA((wgrad_launch<WID, WID>(c->d_act[l], c->d_dz[cur], c->d_part, nullptr, nullptr, N, H, W, s)));
    unpad_grad_kernel<<<cdiv(ncol, NB), NB, 0, s>>>(c->d_part + (int64_t)nblk * ncol,
                                                    layer_cin_logical(l), cin, cout,
                                                    c->d_g + c->off_w[l], c->d_g + c->off_b[l]);
    DV_TRY_CUDA(cudaGetLastError());
    if (l == 0) break;
    // dL/dz_{l-1} = (W_l^T dz_l) masked by relu'(z_{l-1}) = (act_l > 0)
    if (l == NLAYER - 1)
      DV_TRY_CUDA((conv_launch<1, WID, float, float, false, true>(
          c->d_dz[cur], c->d_wt[l], nullptr, c->d_act[l], c->d_dz[cur ^ 1], N, H, W, s)));
    else
      DV_TRY_CUDA((conv_launch<WID, WID, float, float, false, true>(
          c->d_dz[cur], c->d_wt[l], nullptr, c->d_act[l], c->d_dz[cur ^ 1], N, H, W, s)));
    cur ^= 1;
  }
  return DV_OK;
}

dv_status check_shape(int N, int H, int W) {
  if (N < 1 || H < 1 || W < 1 || H > 65535 * TS || N > 65535)
    return fail(DV_ERR_INVALID_ARG, "bad network input shape %d x %d x %d", N, H, W);
  return DV_OK;
}

}  // namespace

// Forward pass of the whole global x grid in row strips (halo of NLAYER rows,
// so every kept row is exact); writes x0 = max(0, y_pad + net(features)).
dv_status warmstart_x0(dv_plan* P, cudaStream_t s, float* x0) {
  Range range("dv warm start");
  dv_cnn* c = P->cnn;
  const int nxr = P->nxr, nxc = P->nxc;
  const int64_t n = (int64_t)nxr * nxc;
  if (!P->d_feat) {
    DV_TRY_CUDA(cudaMalloc(&P->d_feat, (size_t)n * DV_CNN_IN_CH * sizeof(float)));
    DV_TRY_CUDA(cudaMalloc(&P->d_wsd, (size_t)n * sizeof(float)));
    P->device_bytes += n * (DV_CNN_IN_CH + 1) * sizeof(float);
  }
  dim3 grid(cdiv(nxc, NB), nxr);
  features_kernel<<<grid, NB, 0, s>>>(P->d_y, P->hy, P->wy, P->rad, P->d_wrow, P->d_wcol, P->d_desc,
                                      P->Gr, P->Gc, (float)(100.0 * P->prob.noise_sigma), nxr, nxc,
                                      P->d_feat);
  DV_TRY_CUDA(cudaGetLastError());
  const int strip = std::max(64, (int)std::min<int64_t>(nxr, (1 << 22) / std::max(nxc, 1)));
  for (int r0 = 0; r0 < nxr; r0 += strip) {
    const int r1 = std::min(nxr, r0 + strip);
    const int a = std::max(0, r0 - NLAYER), b = std::min(nxr, r1 + NLAYER);
    DV_TRY(forward_tc(c, P->d_feat + (int64_t)a * nxc * DV_CNN_IN_CH, 1, b - a, nxc, nullptr,
                      P->d_err, s));
    DV_TRY_CUDA(cudaMemcpyAsync(P->d_wsd + (int64_t)r0 * nxc, c->d_out + (int64_t)(r0 - a) * nxc,
                                (size_t)(r1 - r0) * nxc * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  apply_warm_kernel<<<cdiv(n, NB), NB, 0, s>>>(P->d_feat, P->d_wsd, n, x0);
  DV_TRY_CUDA(cudaGetLastError());
  P->launches += 2 + 7 * cdiv(nxr, strip);
  return DV_OK;
}

// Per-PSF descriptors of the warm-start features: RMS radius / 8, 10 x peak,
// fraction of |h| beyond radius 3 (|h| normalised to unit sum).
void psf_descriptors(const float* psfs, int G, int K, std::vector<float>& out) {
  out.assign((size_t)G * 3, 0.f);
  const int c = K / 2;
  for (int g = 0; g < G; ++g) {
    const float* h = psfs + (size_t)g * K * K;
    double s = 0.0;
    for (int k = 0; k < K * K; ++k) s += std::fabs((double)h[k]);
    if (!(s > 0.0)) continue;
    double m2 = 0.0, pk = 0.0, wing = 0.0;
    for (int i = 0; i < K; ++i)
      for (int j = 0; j < K; ++j) {
        const double v = std::fabs((double)h[i * K + j]) / s;
        const int r2 = (i - c) * (i - c) + (j - c) * (j - c);
        m2 += v * r2;
        pk = std::max(pk, v);
        if (r2 > 9) wing += v;
      }
    out[(size_t)g * 3 + 0] = (float)(std::sqrt(m2) / 8.0);
    out[(size_t)g * 3 + 1] = (float)(10.0 * pk);
    out[(size_t)g * 3 + 2] = (float)wing;
  }
}

}  // namespace dv

using namespace dv;

namespace dv {
namespace {
void free_cnn(dv_cnn* c) {
  if (!c) return;
  for (float* p : {c->d_p, c->d_g, c->d_m, c->d_v, c->d_out, c->d_dz[0], c->d_dz[1], c->d_part})
    if (p) cudaFree(p);
  for (int l = 0; l < NLAYER; ++l) {
    if (c->d_wf[l]) cudaFree(c->d_wf[l]);
    if (c->d_wt[l]) cudaFree(c->d_wt[l]);
    if (c->d_wtc[l]) cudaFree(c->d_wtc[l]);
    if (c->d_act[l]) cudaFree(c->d_act[l]);
  }
  if (c->d_err) cudaFree(c->d_err);
  if (c->d_lpart) cudaFree(c->d_lpart);
  if (c->d_loss) cudaFree(c->d_loss);
  if (c->h_loss) cudaFreeHost(c->h_loss);
  delete c;
}
}  // namespace
}  // namespace dv

extern "C" dv_status dv_cnn_create(int32_t width, int32_t depth, uint64_t seed, void* stream,
                                   dv_cnn** out) {
  clear_error();
  if (!out) return fail(DV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (width != WID || depth != NLAYER)
    return fail(DV_ERR_UNSUPPORTED, "the library implements width %d and depth %d only", WID, NLAYER);
  dv_cnn* c = new (std::nothrow) dv_cnn();
  if (!c) return fail(DV_ERR_OOM, "host allocation failed");
  int64_t off = 0;
  for (int l = 0; l < NLAYER; ++l) {
    c->off_w[l] = off;
    off += 9LL * layer_cin_logical(l) * layer_cout(l);
    c->off_b[l] = off;
    off += layer_cout(l);
  }
  c->nparam = off;
  // He-normal initialisation (seeded), biases zero
  std::vector<float> p((size_t)off, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < NLAYER; ++l) {
    const double sd = std::sqrt(2.0 / (9.0 * layer_cin_logical(l))) * (l == NLAYER - 1 ? 0.1 : 1.0);
    std::normal_distribution<double> nd(0.0, sd);
    for (int64_t k = 0; k < 9LL * layer_cin_logical(l) * layer_cout(l); ++k) p[c->off_w[l] + k] = (float)nd(rng);
  }
  auto cleanup = [&](dv_status st) {
    free_cnn(c);
    return st;
  };
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  for (float** q : {&c->d_p, &c->d_g, &c->d_m, &c->d_v})
    if ((e = cudaMalloc(q, (size_t)off * sizeof(float))) != cudaSuccess)
      return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
  for (int l = 0; l < NLAYER; ++l) {
    const size_t n = (size_t)9 * layer_cin(l) * layer_cout(l);
    const size_t nt = (size_t)9 * tc_cinp(l) * tc_np(l);
    if ((e = cudaMalloc(&c->d_wf[l], n * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_wt[l], n * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_wtc[l], nt * sizeof(bf16))) != cudaSuccess)
      return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
  }
  if ((e = cudaMalloc(&c->d_err, sizeof(int))) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_err, 0, sizeof(int), s)) != cudaSuccess)
    return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
  if ((e = cudaMalloc(&c->d_lpart, 1024 * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&c->d_loss, sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost(&c->h_loss, sizeof(double))) != cudaSuccess)
    return cleanup(cuda_fail(e, "allocation", __FILE__, __LINE__));
  if ((e = cudaMemcpyAsync(c->d_p, p.data(), (size_t)off * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_m, 0, (size_t)off * sizeof(float), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_v, 0, (size_t)off * sizeof(float), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_g, 0, (size_t)off * sizeof(float), s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cleanup(cuda_fail(e, "upload", __FILE__, __LINE__));
  *out = c;
  return DV_OK;
}

extern "C" int64_t dv_cnn_param_count(const dv_cnn* c) { return c ? c->nparam : 0; }

extern "C" dv_status dv_cnn_get_params(const dv_cnn* c, float* host, int64_t n, int64_t* step) {
  clear_error();
  if (!c || !host || n != c->nparam) return fail(DV_ERR_INVALID_ARG, "need the cnn and %lld floats",
                                                 (long long)(c ? c->nparam : 0));
  DV_TRY_CUDA(cudaMemcpy(host, c->d_p, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost));
  if (step) *step = c->step;
  return DV_OK;
}

extern "C" dv_status dv_cnn_set_params(dv_cnn* c, const float* host, int64_t n, void* stream) {
  clear_error();
  if (!c || !host || n != c->nparam) return fail(DV_ERR_INVALID_ARG, "need the cnn and %lld floats",
                                                 (long long)(c ? c->nparam : 0));
  cudaStream_t s = (cudaStream_t)stream;
  DV_TRY_CUDA(cudaMemcpyAsync(c->d_p, host, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, s));
  DV_TRY_CUDA(cudaMemsetAsync(c->d_m, 0, (size_t)n * sizeof(float), s));
  DV_TRY_CUDA(cudaMemsetAsync(c->d_v, 0, (size_t)n * sizeof(float), s));
  c->step = 0;
  DV_TRY(pack(c, s));
  DV_TRY_CUDA(cudaStreamSynchronize(s));
  return DV_OK;
}

extern "C" dv_status dv_cnn_forward(dv_cnn* c, const float* in_dev, int32_t N, int32_t H, int32_t W,
                                    float* out_dev, void* stream) {
  clear_error();
  if (!c || !in_dev || !out_dev) return fail(DV_ERR_INVALID_ARG, "NULL argument");
  DV_TRY(check_shape(N, H, W));
  return forward_tc(c, in_dev, N, H, W, out_dev, c->d_err, (cudaStream_t)stream);
}

extern "C" dv_status dv_cnn_gradients(dv_cnn* c, const float* in_dev, const float* target_dev,
                                      int32_t N, int32_t H, int32_t W, float* grad_host,
                                      double* loss_host, void* stream) {
  clear_error();
  if (!c || !in_dev || !target_dev) return fail(DV_ERR_INVALID_ARG, "NULL argument");
  DV_TRY(check_shape(N, H, W));
  cudaStream_t s = (cudaStream_t)stream;
  DV_TRY(forward_tc(c, in_dev, N, H, W, nullptr, c->d_err, s));
  DV_TRY(backward(c, target_dev, N, H, W, s));
  DV_TRY_CUDA(cudaMemcpyAsync(c->h_loss, c->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (grad_host)
    DV_TRY_CUDA(cudaMemcpyAsync(grad_host, c->d_g, (size_t)c->nparam * sizeof(float),
                                cudaMemcpyDeviceToHost, s));
  DV_TRY_CUDA(cudaStreamSynchronize(s));
  if (loss_host) *loss_host = 0.5 * *c->h_loss / ((double)N * H * W);
  return DV_OK;
}

extern "C" dv_status dv_cnn_train_step(dv_cnn* c, const float* in_dev, const float* target_dev,
                                       int32_t N, int32_t H, int32_t W, float lr,
                                       double* loss_host, void* stream) {
  clear_error();
  if (!c || !in_dev || !target_dev || !(lr > 0.f)) return fail(DV_ERR_INVALID_ARG, "bad argument");
  DV_TRY(check_shape(N, H, W));
  cudaStream_t s = (cudaStream_t)stream;
  DV_TRY(forward_tc(c, in_dev, N, H, W, nullptr, c->d_err, s));
  DV_TRY(backward(c, target_dev, N, H, W, s));
  c->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - (float)std::pow((double)b1, (double)c->step);
  const float c2 = 1.f - (float)std::pow((double)b2, (double)c->step);
  adam_kernel<<<cdiv(c->nparam, NB), NB, 0, s>>>(c->d_p, c->d_g, c->d_m, c->d_v, c->nparam, lr, b1, b2,
                                                 1e-8f, c1, c2);
  DV_TRY_CUDA(cudaGetLastError());
  DV_TRY(pack(c, s));
  if (loss_host) {
    DV_TRY_CUDA(cudaMemcpyAsync(c->h_loss, c->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    DV_TRY_CUDA(cudaStreamSynchronize(s));
    *loss_host = 0.5 * *c->h_loss / ((double)N * H * W);
  }
  return DV_OK;
}

extern "C" dv_status dv_cnn_train_crops(dv_cnn* c, const float* feats_dev, const float* targets_dev,
                                       int32_t n_pairs, int32_t H, int32_t W, const int32_t* crops_host,
                                       int32_t n_steps, int32_t batch, int32_t crop,
                                       const float* lr_host, double* losses_host, void* stream) {
  Range range("dv cnn training");
  clear_error();
  if (!c || !feats_dev || !targets_dev || !crops_host || !lr_host)
    return fail(DV_ERR_INVALID_ARG, "NULL argument");
  if (n_pairs < 1 || H < 1 || W < 1 || n_steps < 0 || batch < 1 || crop < 1 || crop > H || crop > W)
    return fail(DV_ERR_INVALID_ARG, "bad pair stack %d x %d x %d or crop %d x %d", n_pairs, H, W,
                batch, crop);
  DV_TRY(check_shape(batch, crop, crop));
  for (int64_t k = 0; k < (int64_t)n_steps * batch; ++k) {
    const int32_t* cb = crops_host + 3 * k;
    if (cb[0] < 0 || cb[0] >= n_pairs || cb[1] < 0 || cb[1] > H - crop || cb[2] < 0 || cb[2] > W - crop)
      return fail(DV_ERR_INVALID_ARG, "crop %lld = {%d, %d, %d} outside the pairs", (long long)k,
                  cb[0], cb[1], cb[2]);
  }
  for (int t = 0; t < n_steps; ++t)
    if (!(lr_host[t] > 0.f)) return fail(DV_ERR_INVALID_ARG, "learning rate of step %d is not positive", t);
  if (n_steps == 0) return DV_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t npix = (int64_t)batch * crop * crop;
  int* d_crops = nullptr;
  float* d_xb = nullptr;
  double* d_losses = nullptr;
  auto done = [&](dv_status st) {
    if (st == DV_OK) {
      const cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    } else {
      cudaStreamSynchronize(s);
    }
    cudaFree(d_crops);
    cudaFree(d_xb);
    cudaFree(d_losses);
    return st;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&d_crops, (size_t)n_steps * batch * 3 * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&d_xb, (size_t)npix * (DV_CNN_IN_CH + 1) * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&d_losses, (size_t)n_steps * sizeof(double))) != cudaSuccess)
    return done(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
  float* d_tb = d_xb + npix * DV_CNN_IN_CH;
  if ((e = cudaMemcpyAsync(d_crops, crops_host, (size_t)n_steps * batch * 3 * sizeof(int),
                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return done(cuda_fail(e, "upload", __FILE__, __LINE__));
  const float b1 = 0.9f, b2 = 0.999f;
  for (int t = 0; t < n_steps; ++t) {
    gather_crops_kernel<<<cdiv(npix, NB), NB, 0, s>>>(feats_dev, targets_dev, H, W,
                                                      d_crops + (int64_t)t * batch * 3, batch, crop,
                                                      d_xb, d_tb);
    if ((e = cudaGetLastError()) != cudaSuccess) return done(cuda_fail(e, "gather", __FILE__, __LINE__));
    dv_status st = forward_tc(c, d_xb, batch, crop, crop, nullptr, c->d_err, s);
    if (st == DV_OK) st = backward(c, d_tb, batch, crop, crop, s);
    if (st != DV_OK) return done(st);
    if ((e = cudaMemcpyAsync(d_losses + t, c->d_loss, sizeof(double), cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
      return done(cuda_fail(e, "loss copy", __FILE__, __LINE__));
    c->step += 1;
    const float c1 = 1.f - (float)std::pow((double)b1, (double)c->step);
    const float c2 = 1.f - (float)std::pow((double)b2, (double)c->step);
    adam_kernel<<<cdiv(c->nparam, NB), NB, 0, s>>>(c->d_p, c->d_g, c->d_m, c->d_v, c->nparam, lr_host[t],
                                                   b1, b2, 1e-8f, c1, c2);
    if ((e = cudaGetLastError()) != cudaSuccess) return done(cuda_fail(e, "adam", __FILE__, __LINE__));
    if ((st = pack(c, s)) != DV_OK) return done(st);
  }
  if (losses_host) {
    if ((e = cudaMemcpyAsync(losses_host, d_losses, (size_t)n_steps * sizeof(double),
                             cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return done(cuda_fail(e, "loss download", __FILE__, __LINE__));
  }
  int h_err = 0;
  if ((e = cudaMemcpyAsync(&h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return done(cuda_fail(e, "error word", __FILE__, __LINE__));
  const dv_status st = done(DV_OK);
  if (st == DV_OK && h_err)
    return fail(DV_ERR_TIMEOUT, "a tensor-core wait of the training forward pass gave up (%d)", h_err);
  if (st == DV_OK && losses_host)
    for (int t = 0; t < n_steps; ++t) losses_host[t] *= 0.5 / (double)npix;
  return st;
}

extern "C" dv_status dv_cnn_destroy(dv_cnn* c) {
  clear_error();
  free_cnn(c);
  return DV_OK;
}

extern "C" dv_status dv_plan_set_warmstart(dv_plan* P, dv_cnn* c) {
  clear_error();
  if (!P) return fail(DV_ERR_INVALID_ARG, "plan is NULL");
  P->cnn = c;
  return DV_OK;
}

extern "C" dv_status dv_warmstart_features(dv_plan* P, const float* y_dev, float* feat_dev,
                                           void* stream) {
  clear_error();
  if (!P || !y_dev || !feat_dev) return fail(DV_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  dim3 grid(cdiv(P->nxc, NB), P->nxr);
  features_kernel<<<grid, NB, 0, s>>>(y_dev, P->hy, P->wy, P->rad, P->d_wrow, P->d_wcol, P->d_desc,
                                      P->Gr, P->Gc, (float)(100.0 * P->prob.noise_sigma), P->nxr,
                                      P->nxc, feat_dev);
  DV_TRY_CUDA(cudaGetLastError());
  P->launches += 1;
  return DV_OK;
}
