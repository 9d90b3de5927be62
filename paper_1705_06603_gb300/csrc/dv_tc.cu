// BF16 tensor-core kernels of the shift-variant operator of Sec. II-B and its
// adjoint (FP32 accumulation), on the direct path's 64x64 output blocks.
//
// For one PSF and one filter row a, a correlation is a banded-Toeplitz
// product:  Y[i][j] += sum_c S[i + a][c] T_a[c][j],  T_a[c][j] = f(a, c - j)
// for 0 <= c - j < K, with S the staged input block and f the (flipped for H)
// PSF.  Each warp owns 16 output rows x 64 columns = 8 tiles of the
// m16n8k16 BF16 MMA; for tap row a and k-step ks, tile nt reads the 16
// columns [8 nt + 16 ks, +16) of rows shifted by a.  A operands come from
// shared memory with ldmatrix (any row shift is just another row address;
// 8-column chunk q = nt + 2 ks is shared by several tiles), B fragments depend
// only on (PSF, a, ks) and are precomputed on the host in bfloat16.
//   H:   S = bf16(w_p . x); all PSFs accumulate into the same fragments.
//   H^T: S = bf16(r) staged once; each PSF's correlation is weighted by w_p at
//        the output (FP32) and summed.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "dv_internal.cuh"

namespace dv {
namespace {

constexpr int TM = 64, TN = 64, NW = 4, NT = 32 * NW;
constexpr int NTILE = TN / 8;     // 8 MMA tiles across a warp's 64 columns

__host__ __device__ constexpr int ksteps(int K) { return (8 + K - 1 + 15) / 16; }
// staged width (bf16 elements): chunks 0 .. 7 + 2 KS - 1, 8 columns each
__host__ __device__ constexpr int swidth(int K) { return 8 * (NTILE + 2 * ksteps(K) - 1); }

// Shared memory: [S (bf16) | B fragments of one PSF] at 0, reused by the
// (TM+2) x (TN+2) fp32 halo of the step epilogue; the fp32 output staging
// block after both.
__host__ __device__ constexpr size_t tc_off_out(int K) {
  return (((size_t)(TM + K - 1) * swidth(K) * 2 + (size_t)K * ksteps(K) * 32 * 8 >
                   (size_t)(TM + 2) * (TN + 2) * 4
               ? (size_t)(TM + K - 1) * swidth(K) * 2 + (size_t)K * ksteps(K) * 32 * 8
               : (size_t)(TM + 2) * (TN + 2) * 4) +
          15) / 16 * 16;
}
size_t tc_smem(int K) { return tc_off_out(K) + (size_t)TM * (TN + 4) * 4; }

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x2(uint32_t& r0, uint32_t& r1, const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(a));
}

// acc[nt][.] += sum_a sum_ks  A(rows + a, chunk nt + 2 ks) B(a, ks)
template <int K>
__device__ __forceinline__ void tc_corr(const __nv_bfloat16* sS, const uint2* sB, int row0,
                                        float (&acc)[NTILE][4]) {
  constexpr int KS = ksteps(K);
  constexpr int W = swidth(K);
  constexpr int NCH = NTILE + 2 * KS;   // chunks read per tap row
  const int lane = threadIdx.x & 31;
  const __nv_bfloat16* rowp = sS + (row0 + (lane & 15)) * W;
#pragma unroll 1
  for (int a = 0; a < K; ++a) {
    uint32_t r0[NCH], r1[NCH];
#pragma unroll
    for (int q = 0; q < NCH - 1; ++q) ldsm_x2(r0[q], r1[q], rowp + a * W + 8 * q);
    r0[NCH - 1] = r1[NCH - 1] = 0u;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const uint2 b = sB[(a * KS + ks) * 32 + lane];
#pragma unroll
      for (int nt = 0; nt < NTILE; ++nt) {
        const int q = nt + 2 * ks;
        mma_bf16(acc[nt], r0[q], r1[q], r0[q + 1], r1[q + 1], b.x, b.y);
      }
    }
  }
}

// Accumulator element (tile nt, slot e) -> (row, col) in the warp's 16 x 64 band
__device__ __forceinline__ void frag_pos(int nt, int e, int& r, int& c) {
  const int lane = threadIdx.x & 31;
  r = (lane >> 2) + (e >= 2 ? 8 : 0);
  c = 8 * nt + 2 * (lane & 3) + (e & 1);
}

template <int K>
__global__ void __launch_bounds__(NT) tc_H_kernel(const OpArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int KS = ksteps(K), W = swidth(K), ROWS = TM + K - 1;
  __nv_bfloat16* sS = reinterpret_cast<__nv_bfloat16*>(smem);
  uint2* sB = reinterpret_cast<uint2*>(smem + (size_t)ROWS * W * 2);
  float* sO = reinterpret_cast<float*>(smem + tc_off_out(K));
  __shared__ float sWr[ROWS], sWc[W];
  __shared__ double red[NW];
  const WorkItem wi = A.work[blockIdx.x];
  const TileDesc td = A.tiles[wi.tile];
  const int tid = threadIdx.x, warp = tid >> 5;
  float acc[NTILE][4];
#pragma unroll
  for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;

  for (int a = wi.a_lo; a <= wi.a_hi; ++a) {
    for (int b = wi.b_lo; b <= wi.b_hi; ++b) {
      __syncthreads();
      for (int e = tid; e < ROWS; e += NT) {
        const int R = wi.r0 + e;
        sWr[e] = R < td.nxr ? wsel(A.wrow[td.xr0 + R], a) : 0.f;
      }
      for (int e = tid; e < W; e += NT) {
        const int C = wi.c0 + e;
        sWc[e] = (e < TN + K - 1 && C < td.nxc) ? wsel(A.wcol[td.xc0 + C], b) : 0.f;
      }
      const uint2* bsrc = A.bfrag + (size_t)(a * A.Gc + b) * K * KS * 32;
      for (int e = tid; e < K * KS * 32; e += NT) sB[e] = bsrc[e];
      __syncthreads();
      for (int e = tid; e < ROWS * W; e += NT) {
        const int ir = e / W, ic = e - ir * W;
        const float wgt = sWr[ir] * sWc[ic];
        float v = 0.f;
        if (wgt != 0.f) v = wgt * A.in[td.xoff + (int64_t)(wi.r0 + ir) * td.xpitch + (wi.c0 + ic)];
        sS[e] = __float2bfloat16_rn(v);
      }
      __syncthreads();
      tc_corr<K>(sS, sB, 16 * warp, acc);
    }
  }
  __syncthreads();
#pragma unroll
  for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int r, c;
      frag_pos(nt, e, r, c);
      sO[(16 * warp + r) * (TN + 4) + c] = acc[nt][e];
    }
  __syncthreads();
  double part = 0.0;
  for (int e = tid; e < TM * TN; e += NT) {
    const int il = e / TN, jl = e - il * TN;
    const int i = wi.r0 + il, j = wi.c0 + jl;
    if (i >= td.nyr || j >= td.nyc) continue;
    const float v = sO[il * (TN + 4) + jl];
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
  if (A.mode == OP_OBJ) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[warp] = part;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int i = 0; i < NW; ++i) s += red[i];
      A.partials[blockIdx.x] = s;
    }
  }
}

// p = kappa (dr, dc) of the Huber prior at tile pixel (R, C) from the staged
// iterate (smem (li, lj), pitch SPW); zero above / left of the tile.
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

template <int K>
__global__ void __launch_bounds__(NT) tc_Ht_kernel(const OpArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int KS = ksteps(K), W = swidth(K), ROWS = TM + K - 1;
  __nv_bfloat16* sS = reinterpret_cast<__nv_bfloat16*>(smem);
  uint2* sB = reinterpret_cast<uint2*>(smem + (size_t)ROWS * W * 2);
  float* sO = reinterpret_cast<float*>(smem + tc_off_out(K));
  const WorkItem wi = A.work[blockIdx.x];
  const TileDesc td = A.tiles[wi.tile];
  const int tid = threadIdx.x, warp = tid >> 5;
  // residual block, rows R0 - (K-1) .., columns C0 - (K-1) .., zero outside the y-block
  for (int e = tid; e < ROWS * W; e += NT) {
    const int ir = e / W, ic = e - ir * W;
    const int ry = wi.r0 - (K - 1) + ir, rx = wi.c0 - (K - 1) + ic;
    float v = 0.f;
    if (ic < TN + K - 1 && ry >= 0 && ry < td.nyr && rx >= 0 && rx < td.nyc)
      v = A.in[td.yoff + (int64_t)ry * td.ypitch + rx];
    sS[e] = __float2bfloat16_rn(v);
  }
  float g[NTILE][4];
#pragma unroll
  for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) g[nt][e] = 0.f;
  // output weights of this thread's fragment rows / columns are looked up per PSF
  for (int a = wi.a_lo; a <= wi.a_hi; ++a) {
    for (int b = wi.b_lo; b <= wi.b_hi; ++b) {
      __syncthreads();
      const uint2* bsrc = A.bfrag + (size_t)(a * A.Gc + b) * K * KS * 32;
      for (int e = tid; e < K * KS * 32; e += NT) sB[e] = bsrc[e];
      __syncthreads();
      float acc[NTILE][4];
#pragma unroll
      for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
      tc_corr<K>(sS, sB, 16 * warp, acc);
      const int lane = tid & 31;
      float wr[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int R = wi.r0 + 16 * warp + (lane >> 2) + 8 * h;
        wr[h] = R < td.nxr ? wsel(A.wrow[td.xr0 + R], a) : 0.f;
      }
#pragma unroll
      for (int nt = 0; nt < NTILE; ++nt) {
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          const int C = wi.c0 + 8 * nt + 2 * (lane & 3) + e2;
          const float wc = C < td.nxc ? wsel(A.wcol[td.xc0 + C], b) : 0.f;
          g[nt][e2] = fmaf(wr[0] * wc, acc[nt][e2], g[nt][e2]);
          g[nt][e2 + 2] = fmaf(wr[1] * wc, acc[nt][e2 + 2], g[nt][e2 + 2]);
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int nt = 0; nt < NTILE; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int r, c;
      frag_pos(nt, e, r, c);
      sO[(16 * warp + r) * (TN + 4) + c] = g[nt][e];
    }
  __syncthreads();
  if (A.mode == OP_PLAIN) {
    for (int e = tid; e < TM * TN; e += NT) {
      const int il = e / TN, jl = e - il * TN;
      const int R = wi.r0 + il, C = wi.c0 + jl;
      if (R < td.nxr && C < td.nxc)
        A.out[td.xoff + (int64_t)R * td.xpitch + C] = sO[il * (TN + 4) + jl];
    }
    return;
  }
  // OP_STEP: grad = g + lambda D^T psi(D w) + alpha (w - u); w_next = max(0, w - tau grad)
  float* sW = reinterpret_cast<float*>(smem);   // (TM+2) x (TN+2) halo of w (reuses S and B)
  constexpr int SPW = TN + 2;
  for (int e = tid; e < (TM + 2) * SPW; e += NT) {
    const int ir = e / SPW, ic = e - ir * SPW;
    const int R = wi.r0 - 1 + ir, C = wi.c0 - 1 + ic;
    float v = 0.f;
    if (R >= 0 && R < td.nxr && C >= 0 && C < td.nxc) v = A.w[td.xoff + (int64_t)R * td.xpitch + C];
    sW[e] = v;
  }
  __syncthreads();
  for (int e = tid; e < TM * TN; e += NT) {
    const int il = e / TN, jl = e - il * TN;
    const int R = wi.r0 + il, C = wi.c0 + jl;
    if (R >= td.nxr || C >= td.nxc) continue;
    const int li = il + 1, lj = jl + 1;
    float pr, pc, pru, pcu, prl, pcl;
    huber_p(sW, SPW, li, lj, R, C, td.nxr, td.nxc, A.delta, pr, pc);
    huber_p(sW, SPW, li - 1, lj, R - 1, C, td.nxr, td.nxc, A.delta, pru, pcu);
    huber_p(sW, SPW, li, lj - 1, R, C - 1, td.nxr, td.nxc, A.delta, prl, pcl);
    const float hub = pru - pr + pcl - pc;
    const float wv = sW[li * SPW + lj];
    const float alpha = A.gamma * A.omr[td.omr_off + R] * A.omc[td.omc_off + C];
    const int64_t idx = td.xoff + (int64_t)R * td.xpitch + C;
    const float grad = sO[il * (TN + 4) + jl] + A.lambda * hub + alpha * (wv - A.u[idx]);
    A.out[idx] = fmaxf(0.f, wv - td.tau * grad);
  }
}

template <int K>
cudaError_t prep_t() {
  const int smem = (int)tc_smem(K);
  cudaError_t e = cudaFuncSetAttribute(tc_H_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tc_Ht_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

uint16_t to_bf16(float f) {
  // round to nearest even on the IEEE single-precision bit pattern
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);   // inf / nan
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

}  // namespace

bool tc_supported(int K) { return K == 9 || K == 15 || K == 31 || K == 63; }

cudaError_t tc_prepare(int K) {
  switch (K) {
    case 9: return prep_t<9>();
    case 15: return prep_t<15>();
    case 31: return prep_t<31>();
    case 63: return prep_t<63>();
    default: return cudaErrorInvalidValue;
  }
}

// B fragments of the m16n8k16 MMA for every PSF, filter row and k-step:
// T[k][n] = f(a, k - n) for 0 <= k - n < K (f = flipped PSF for H, PSF for H^T);
// lane l holds (T[2t + 16 ks][g], T[2t + 1 + 16 ks][g]) and the same for k + 8,
// g = l / 4, t = l % 4, as bf16 pairs (lower k in the low half).
void tc_fragments(const float* psfs, int G, int K, bool flip, std::vector<uint2>& out) {
  const int KS = ksteps(K);
  out.assign((size_t)G * K * KS * 32, make_uint2(0u, 0u));
  for (int p = 0; p < G; ++p) {
    const float* h = psfs + (size_t)p * K * K;
    for (int a = 0; a < K; ++a)
      for (int ks = 0; ks < KS; ++ks)
        for (int l = 0; l < 32; ++l) {
          const int gq = l >> 2, t = l & 3;
          auto T = [&](int k) -> float {
            const int d = k - gq;
            if (d < 0 || d >= K) return 0.f;
            return flip ? h[(K - 1 - a) * K + (K - 1 - d)] : h[a * K + d];
          };
          const int k0 = 2 * t + 16 * ks;
          const uint32_t x = (uint32_t)to_bf16(T(k0)) | ((uint32_t)to_bf16(T(k0 + 1)) << 16);
          const uint32_t y = (uint32_t)to_bf16(T(k0 + 8)) | ((uint32_t)to_bf16(T(k0 + 9)) << 16);
          out[(((size_t)p * K + a) * KS + ks) * 32 + l] = make_uint2(x, y);
        }
  }
}

template <int K>
cudaError_t launch_H_tc(const OpArgs& a, cudaStream_t s) {
  tc_H_kernel<K><<<a.n_work, NT, tc_smem(K), s>>>(a);
  return cudaGetLastError();
}
template <int K>
cudaError_t launch_Ht_tc(const OpArgs& a, cudaStream_t s) {
  tc_Ht_kernel<K><<<a.n_work, NT, tc_smem(K), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tc_H(const OpArgs& a, cudaStream_t s) {
  if (a.n_work <= 0) return cudaSuccess;
  switch (a.K) {
    case 9: return launch_H_tc<9>(a, s);
    case 15: return launch_H_tc<15>(a, s);
    case 31: return launch_H_tc<31>(a, s);
    case 63: return launch_H_tc<63>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tc_Ht(const OpArgs& a, cudaStream_t s) {
  if (a.n_work <= 0) return cudaSuccess;
  switch (a.K) {
    case 9: return launch_Ht_tc<9>(a, s);
    case 15: return launch_Ht_tc<15>(a, s);
    case 31: return launch_Ht_tc<31>(a, s);
    case 63: return launch_Ht_tc<63>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dv
