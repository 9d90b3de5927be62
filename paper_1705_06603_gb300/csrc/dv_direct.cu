// Direct (spatial-domain) FP32 kernels of the shift-variant operator of
// Sec. II-B and its adjoint, batched over all tiles in one launch.
//
//   H:    y(i,j) = sum_p sum_{a,b} hflip_p(a,b) (w_p . x)(i + a, j + b)
//   H^T:  g(R,C) = sum_p w_p(R,C) sum_{a,b} h_p(a,b) r(R - (K-1) + a, C - (K-1) + b)
//
// Both are correlations of a staged input region with a K x K filter.  One CTA
// owns a TM x TN output block of one tile (a WorkItem); each thread keeps an
// RT x CT register block of accumulators and slides a CT + K - 1 wide window of
// the input row through registers, so every shared-memory load feeds many FMAs.
// For H the weighted copy w_p . x is staged per active PSF p (at most the
// PSFs whose weights touch the block); for H^T the residual is staged once and
// each PSF's correlation is weighted by w_p at the output.  Epilogues: the
// residual W (H x - y) (or an FP64 partial of its weighted square) for H, and
// the projected-gradient step of the Local-Solver for H^T.
#include <algorithm>
#include <cstdio>

#include "dv_internal.cuh"

namespace dv {
namespace {

constexpr int TM = 64, TN = 64;     // output block
constexpr int RT = 4, CT = 8;       // register block per thread
constexpr int NTX = TN / CT;        // 8 threads across
constexpr int NTY = TM / RT;        // 16 threads down
constexpr int NT = NTX * NTY;       // 128 threads

__host__ __device__ constexpr int round4(int v) { return (v + 3) & ~3; }
__host__ __device__ constexpr int imax(int a, int b) { return a > b ? a : b; }
// Row pitch of the staged input region: TN + K - 1 columns, plus the float4
// over-read of the last thread's window.
__host__ __device__ constexpr int in_pitch(int K) {
  return imax(round4(TN + K - 1), TN - CT + 4 * ((CT + K - 1 + 3) / 4));
}

// Floats of the staged input region; also holds the (TM+2) x (TN+2) halo block
// of the iterate used by the fused step of H^T.
__host__ __device__ constexpr int in_elems(int K) {
  return imax((TM + K - 1) * in_pitch(K), (TM + 2) * (TN + 2));
}
constexpr int SPW = TN + 2;         // row pitch of the halo block

size_t smem_bytes(int K) {
  const int rows = TM + K - 1, sp = in_pitch(K);
  return sizeof(float) * ((size_t)in_elems(K) + (size_t)K * round4(K) + rows + sp);
}

// acc[q][c] += sum_{a,b} f(a,b) in(row0 + q + a, col0 + c + b), compile-time K.
template <int K>
__device__ __forceinline__ void corr_accum(const float* __restrict__ sIn,
                                           const float* __restrict__ sF,
                                           float (&acc)[RT][CT], int row0, int col0) {
  constexpr int SP = in_pitch(K);
  constexpr int KP = round4(K);
  constexpr int XW4 = (CT + K - 1 + 3) / 4;
#pragma unroll 1
  for (int t = 0; t < RT + K - 1; ++t) {
    float xv[XW4 * 4];
    const float4* src = reinterpret_cast<const float4*>(sIn + (row0 + t) * SP + col0);
#pragma unroll
    for (int v = 0; v < XW4; ++v) {
      const float4 q4 = src[v];
      xv[4 * v + 0] = q4.x;
      xv[4 * v + 1] = q4.y;
      xv[4 * v + 2] = q4.z;
      xv[4 * v + 3] = q4.w;
    }
#pragma unroll
    for (int q = 0; q < RT; ++q) {
      const int a = t - q;
      if (a >= 0 && a < K) {
        const float4* fr = reinterpret_cast<const float4*>(sF + a * KP);
#pragma unroll
        for (int b4 = 0; b4 < KP / 4; ++b4) {
          const float4 f4 = fr[b4];
          const float fv[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (4 * b4 + e < K) {
#pragma unroll
              for (int c = 0; c < CT; ++c) acc[q][c] = fmaf(fv[e], xv[c + 4 * b4 + e], acc[q][c]);
            }
          }
        }
      }
    }
  }
}

// Same sum for a run-time K (any odd K the plan accepts).
__device__ __forceinline__ void corr_accum_rt(const float* __restrict__ sIn,
                                              const float* __restrict__ sF, int K, int SP,
                                              float (&acc)[RT][CT], int row0, int col0) {
  const int KP = round4(K);
  for (int a = 0; a < K; ++a) {
    for (int b = 0; b < K; ++b) {
      const float f = sF[a * KP + b];
#pragma unroll
      for (int q = 0; q < RT; ++q) {
        const float* row = sIn + (row0 + q + a) * SP + col0 + b;
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[q][c] = fmaf(f, row[c], acc[q][c]);
      }
    }
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;
}

// ---------------------------------------------------------------------------
// H: output y-block block (r0, c0) of a tile; input x rows r0 .. r0 + TM + K - 2
// ---------------------------------------------------------------------------
template <int KC>
__global__ void __launch_bounds__(NT) direct_H_kernel(const OpArgs A) {
  extern __shared__ __align__(16) float smem[];
  __shared__ double red[NT / 32];
  const int K = KC > 0 ? KC : A.K;
  const int SP = in_pitch(K);
  const int KP = round4(K);
  const int ROWS = TM + K - 1;
  float* sIn = smem;
  float* sF = sIn + in_elems(K);
  float* sWr = sF + K * KP;
  float* sWc = sWr + ROWS;

  const WorkItem wi = A.work[blockIdx.x];
  const TileDesc td = A.tiles[wi.tile];
  const int tid = threadIdx.x, tx = tid % NTX, ty = tid / NTX;

  float acc[RT][CT];
#pragma unroll
  for (int q = 0; q < RT; ++q)
#pragma unroll
    for (int c = 0; c < CT; ++c) acc[q][c] = 0.f;

  for (int a = wi.a_lo; a <= wi.a_hi; ++a) {
    for (int b = wi.b_lo; b <= wi.b_hi; ++b) {
      __syncthreads();
      for (int e = tid; e < ROWS; e += NT) {
        const int R = wi.r0 + e;
        sWr[e] = R < td.nxr ? wsel(A.wrow[td.wr0 + R], a) : 0.f;
      }
      for (int e = tid; e < SP; e += NT) {
        const int C = wi.c0 + e;
        sWc[e] = (e < TN + K - 1 && C < td.nxc) ? wsel(A.wcol[td.wc0 + C], b) : 0.f;
      }
      const float* f = A.psf + (size_t)(a * A.Gc + b) * K * KP;
      for (int e = tid; e < K * KP; e += NT) sF[e] = f[e];
      __syncthreads();
      for (int e = tid; e < ROWS * SP; e += NT) {
        const int ir = e / SP, ic = e - ir * SP;
        const float wgt = sWr[ir] * sWc[ic];
        float v = 0.f;
        if (wgt != 0.f)
          v = wgt * A.in[td.xoff + (int64_t)(wi.r0 + ir) * td.xpitch + (wi.c0 + ic)];
        sIn[e] = v;
      }
      __syncthreads();
      if constexpr (KC > 0)
        corr_accum<KC>(sIn, sF, acc, ty * RT, tx * CT);
      else
        corr_accum_rt(sIn, sF, K, SP, acc, ty * RT, tx * CT);
    }
  }

  const int i0 = wi.r0 + ty * RT, j0 = wi.c0 + tx * CT;
  double part = 0.0;
#pragma unroll
  for (int q = 0; q < RT; ++q) {
    const int i = i0 + q;
    if (i >= td.nyr) continue;
#pragma unroll
    for (int c = 0; c < CT; ++c) {
      const int j = j0 + c;
      if (j >= td.nyc) continue;
      const float v = acc[q][c];
      if (A.mode == OP_PLAIN) {
        A.out[td.yoff + (int64_t)i * td.ypitch + j] = v;
      } else {
        const int64_t gi = (int64_t)(td.xr0 + i) * A.wy + (td.xc0 + j);
        const float wt = A.W ? A.W[gi] : 1.f;
        const float d = v - A.y[gi];
        if (A.mode == OP_RESID)
          A.out[td.yoff + (int64_t)i * td.ypitch + j] = wt * d;
        else
          part += (double)wt * (double)d * (double)d;
      }
    }
  }
  if (A.mode == OP_OBJ) {
    const double s = block_sum(part, red);
    if (tid == 0) A.partials[blockIdx.x] = s;
  }
}

// p = kappa (dr, dc) of the Huber prior at tile pixel (R, C), read from the
// staged iterate at smem position (li, lj); zero above / left of the tile.
__device__ __forceinline__ void huber_p(const float* sW, int SPW, int li, int lj, int R, int C,
                                        int nxr, int nxc, float delta, float& pr, float& pc) {
  if (R < 0 || C < 0) {
    pr = pc = 0.f;
    return;
  }
  const float c0 = sW[li * SPW + lj];
  const float dr = (R + 1 < nxr) ? sW[(li + 1) * SPW + lj] - c0 : 0.f;
  const float dc = (C + 1 < nxc) ? sW[li * SPW + lj + 1] - c0 : 0.f;
  const float s2 = dr * dr + dc * dc;
  const float k = (s2 <= delta * delta) ? 1.f : delta * rsqrtf(s2);
  pr = k * dr;
  pc = k * dc;
}

// ---------------------------------------------------------------------------
// H^T: output x block (R0, C0) of a tile; input r rows R0 - (K-1) .. R0 + TM - 1
// ---------------------------------------------------------------------------
template <int KC>
__global__ void __launch_bounds__(NT) direct_Ht_kernel(const OpArgs A) {
  extern __shared__ __align__(16) float smem[];
  const int K = KC > 0 ? KC : A.K;
  const int SP = in_pitch(K);
  const int KP = round4(K);
  const int ROWS = TM + K - 1;
  float* sIn = smem;
  float* sF = sIn + in_elems(K);

  const WorkItem wi = A.work[blockIdx.x];
  const TileDesc td = A.tiles[wi.tile];
  const int tid = threadIdx.x, tx = tid % NTX, ty = tid / NTX;

  for (int e = tid; e < ROWS * SP; e += NT) {
    const int ir = e / SP, ic = e - ir * SP;
    const int ry = wi.r0 - (K - 1) + ir, rx = wi.c0 - (K - 1) + ic;
    float v = 0.f;
    if (ic < TN + K - 1 && ry >= 0 && ry < td.nyr && rx >= 0 && rx < td.nyc)
      v = A.in[td.yoff + (int64_t)ry * td.ypitch + rx];
    sIn[e] = v;
  }

  const int R0 = wi.r0 + ty * RT, C0 = wi.c0 + tx * CT;
  float g[RT][CT];
#pragma unroll
  for (int q = 0; q < RT; ++q)
#pragma unroll
    for (int c = 0; c < CT; ++c) g[q][c] = 0.f;

  for (int a = wi.a_lo; a <= wi.a_hi; ++a) {
    for (int b = wi.b_lo; b <= wi.b_hi; ++b) {
      __syncthreads();
      const float* f = A.psf + (size_t)(a * A.Gc + b) * K * KP;
      for (int e = tid; e < K * KP; e += NT) sF[e] = f[e];
      __syncthreads();
      float acc[RT][CT];
#pragma unroll
      for (int q = 0; q < RT; ++q)
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[q][c] = 0.f;
      if constexpr (KC > 0)
        corr_accum<KC>(sIn, sF, acc, ty * RT, tx * CT);
      else
        corr_accum_rt(sIn, sF, K, SP, acc, ty * RT, tx * CT);
      float wr[RT], wc[CT];
#pragma unroll
      for (int q = 0; q < RT; ++q)
        wr[q] = (R0 + q < td.nxr) ? wsel(A.wrow[td.wr0 + R0 + q], a) : 0.f;
#pragma unroll
      for (int c = 0; c < CT; ++c)
        wc[c] = (C0 + c < td.nxc) ? wsel(A.wcol[td.wc0 + C0 + c], b) : 0.f;
#pragma unroll
      for (int q = 0; q < RT; ++q)
#pragma unroll
        for (int c = 0; c < CT; ++c) g[q][c] = fmaf(wr[q] * wc[c], acc[q][c], g[q][c]);
    }
  }

  if (A.mode == OP_PLAIN) {
#pragma unroll
    for (int q = 0; q < RT; ++q) {
      if (R0 + q >= td.nxr) continue;
#pragma unroll
      for (int c = 0; c < CT; ++c)
        if (C0 + c < td.nxc) A.out[td.xoff + (int64_t)(R0 + q) * td.xpitch + C0 + c] = g[q][c];
    }
    return;
  }

  // OP_STEP: grad = g + lambda D^T psi(D w) + alpha (w - u); w_next = max(0, w - tau grad)
  __syncthreads();
  float* sW = sIn;               // (TM + 2) x (TN + 2) halo block of w, pitch SPW
  for (int e = tid; e < (TM + 2) * SPW; e += NT) {
    const int ir = e / SPW, ic = e - ir * SPW;
    const int R = wi.r0 - 1 + ir, C = wi.c0 - 1 + ic;
    float v = 0.f;
    if (R >= 0 && R < td.nxr && C >= 0 && C < td.nxc)
      v = A.w[td.xoff + (int64_t)R * td.xpitch + C];
    sW[e] = v;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < RT; ++q) {
    const int R = R0 + q;
    if (R >= td.nxr) continue;
    const float om_r = A.omr[td.omr_off + R];
#pragma unroll
    for (int c = 0; c < CT; ++c) {
      const int C = C0 + c;
      if (C >= td.nxc) continue;
      const int li = ty * RT + q + 1, lj = tx * CT + c + 1;
      float pr, pc, pru, pcu, prl, pcl;
      huber_p(sW, SPW, li, lj, R, C, td.nxr, td.nxc, A.delta, pr, pc);
      huber_p(sW, SPW, li - 1, lj, R - 1, C, td.nxr, td.nxc, A.delta, pru, pcu);
      huber_p(sW, SPW, li, lj - 1, R, C - 1, td.nxr, td.nxc, A.delta, prl, pcl);
      const float hub = pru - pr + pcl - pc;
      const float wv = sW[li * SPW + lj];
      const float alpha = A.gamma * om_r * A.omc[td.omc_off + C];
      const int64_t idx = td.xoff + (int64_t)R * td.xpitch + C;
      const float grad = g[q][c] + A.lambda * hub + alpha * (wv - A.u[idx]);
      A.out[idx] = fmaxf(0.f, wv - td.tau * grad);
    }
  }
}

template <int KC>
cudaError_t launch_H_t(const OpArgs& a, cudaStream_t s) {
  direct_H_kernel<KC><<<a.n_work, NT, smem_bytes(a.K), s>>>(a);
  return cudaGetLastError();
}

template <int KC>
cudaError_t launch_Ht_t(const OpArgs& a, cudaStream_t s) {
  direct_Ht_kernel<KC><<<a.n_work, NT, smem_bytes(a.K), s>>>(a);
  return cudaGetLastError();
}

template <int KC>
cudaError_t prepare_t(int K) {
  const int smem = (int)smem_bytes(KC > 0 ? KC : K);
  cudaError_t e = cudaFuncSetAttribute(direct_H_kernel<KC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(direct_Ht_kernel<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem);
}

}  // namespace

int direct_tile_m() { return TM; }
int direct_tile_n() { return TN; }

cudaError_t launch_direct_H(const OpArgs& a, cudaStream_t s) {
  if (a.n_work <= 0) return cudaSuccess;
  switch (a.K) {
    case 3: return launch_H_t<3>(a, s);
    case 5: return launch_H_t<5>(a, s);
    case 7: return launch_H_t<7>(a, s);
    case 9: return launch_H_t<9>(a, s);
    case 15: return launch_H_t<15>(a, s);
    case 31: return launch_H_t<31>(a, s);
    case 63: return launch_H_t<63>(a, s);
    default: return launch_H_t<0>(a, s);
  }
}

cudaError_t launch_direct_Ht(const OpArgs& a, cudaStream_t s) {
  if (a.n_work <= 0) return cudaSuccess;
  switch (a.K) {
    case 3: return launch_Ht_t<3>(a, s);
    case 5: return launch_Ht_t<5>(a, s);
    case 7: return launch_Ht_t<7>(a, s);
    case 9: return launch_Ht_t<9>(a, s);
    case 15: return launch_Ht_t<15>(a, s);
    case 31: return launch_Ht_t<31>(a, s);
    case 63: return launch_Ht_t<63>(a, s);
    default: return launch_Ht_t<0>(a, s);
  }
}

size_t direct_smem_bytes(int K) { return smem_bytes(K); }

// Sets the dynamic shared-memory limit of the direct kernels used for K on the
// current device.  Called at plan creation, never during stream capture.  The
// run-time-K kernel keeps the largest limit requested so far.
cudaError_t direct_prepare(int K) {
  static int rt_max = 0;
  switch (K) {
    case 3: return prepare_t<3>(K);
    case 5: return prepare_t<5>(K);
    case 7: return prepare_t<7>(K);
    case 9: return prepare_t<9>(K);
    case 15: return prepare_t<15>(K);
    case 31: return prepare_t<31>(K);
    case 63: return prepare_t<63>(K);
    default:
      rt_max = std::max(rt_max, K);
      return prepare_t<0>(rt_max);
  }
}

}  // namespace dv
