// Block-FFT (overlap-save) kernels of the shift-variant operator of Sec. II-B
// and its adjoint.  Each CTA owns b x b output blocks (b = S - K + 1, S = 128)
// of the tiles and computes them with 128 x 128 complex FFTs held in shared
// memory -- the non-circulant local blur of Sec. II-B (circular convolution
// of size S followed by a crop to the valid part).
//
// Two PSFs are packed into one complex transform:
//   H:   y = Re IFFT( FFT(w_p1 x + i w_p2 x) . (Hh_p1 - i Hh_p2) )
//          = h_p1 * (w_p1 x) + h_p2 * (w_p2 x)          (valid part)
//   H^T: c_p1 + i c_p2 = IFFT( FFT(r) . (conj Hh_p1 + i conj Hh_p2) )
//        g += w_p1 c_p1 + w_p2 c_p2                     (first b x b outputs)
// where Hh_p is the S x S spectrum of the zero-padded PSF (computed on the host
// in FP64 at plan time, scaled by 1/S^2).
//
// A 128-point transform is done "four-step": n = n1 + 16 n2, k = k2 + 8 k1;
// 8-point DFTs over n2, twiddle W_128^{n1 k2}, 16-point DFTs over n1.  The
// per-thread DFTs run in registers; the exchange between the two steps goes
// through shared memory with rows/columns padded (position k2*17 + n1) so the
// accesses are free of bank conflicts.  The spectral product is applied
// between the forward and the inverse 16-point step of the column pass, so
// the column spectrum never leaves registers and no digit reversal is needed.
// Twiddles are exp(-2 pi i k / 128) computed on the host in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dv_internal.cuh"

namespace dv {
namespace {

constexpr int S = 128;             // FFT size
constexpr int P = 136;             // row pitch (complex) of the 128-row buffer
constexpr int NT = 512;            // threads per CTA
constexpr int BMAX = S;            // largest valid block side (K = 1)

__constant__ float2 c_w128[S];     // exp(-2 pi i k / 128)

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// W_128^k (conjugated for the inverse transform)
template <bool INV>
__device__ __forceinline__ float2 tw(int k) {
  const float2 w = c_w128[k & (S - 1)];
  return INV ? make_float2(w.x, -w.y) : w;
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// In-register DFT of length N (power of two), natural order in and out:
// X[k] = sum_n v[n] W_N^{+-nk}.  Radix-2 decimation in time.
template <int N, bool INV>
__device__ __forceinline__ void dft(float2 (&v)[N]) {
  constexpr int LB = ilog2(N);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int j = bitrev(i, LB);
    if (j > i) {
      const float2 t = v[i];
      v[i] = v[j];
      v[j] = t;
    }
  }
#pragma unroll
  for (int len = 2; len <= N; len <<= 1) {
    const int half = len / 2;
#pragma unroll
    for (int i = 0; i < N; i += len) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const float2 a = v[i + k];
        float2 b = v[i + k + half];
        if (k != 0) {
          if (4 * k == len) {           // W_len^{len/4} = -i (forward) or +i (inverse)
            b = INV ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
          } else {
            b = cmul(b, tw<INV>(k * (S / len)));
          }
        }
        v[i + k] = cadd(a, b);
        v[i + k + half] = csub(a, b);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Buffer layout.  A holds 128 rows of P = 136 complex values.  Spatial rows
// are stored "padded natural": element n of a row sits at position
// pos(n) = n + n/16, so the 16 n1-phases of a row land in distinct banks.
// After the forward row transform, frequency k = k2 + 8 k1 of a row sits at
// position k1 + 17 k2 (digit-permuted); columns are transformed in that
// order and the PSF spectra are stored permuted the same way on the host.
// Every step works in place on the positions its own task reads, so a step
// needs no barrier between its loads and stores.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pos(int n) { return n + (n >> 4); }

// Forward 128-point transforms of all 128 rows (padded natural -> permuted).
__device__ __forceinline__ void row_fwd(float2* A, const float2* sTw) {
  // step 1: tasks (row, n1): 8-point DFT over n2, twiddle W^{n1 k2}
#pragma unroll 1
  for (int r = 0; r < 4; ++r) {
    const int n1 = threadIdx.x & 15;
    float2* row = A + ((threadIdx.x >> 4) + 32 * r) * P;
    float2 v[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) v[n2] = row[n1 + 17 * n2];
    dft<8, false>(v);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) row[n1 + 17 * k2] = k2 ? cmul(v[k2], sTw[n1 * k2]) : v[k2];
  }
  __syncthreads();
  // step 2: tasks (row, k2): 16-point DFT over n1 -> X[k2 + 8 k1] at k1 + 17 k2
#pragma unroll 1
  for (int r = 0; r < 2; ++r) {
    const int k2 = threadIdx.x & 7;
    float2* row = A + ((threadIdx.x >> 3) + 64 * r) * P;
    float2 u[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) u[n1] = row[n1 + 17 * k2];
    dft<16, false>(u);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) row[k1 + 17 * k2] = u[k1];
  }
  __syncthreads();
}

// Inverse transforms of rows [row_lo, row_lo + nrows) (permuted -> padded natural).
__device__ __forceinline__ void row_inv(float2* A, const float2* sTw, int row_lo, int nrows) {
  for (int base = 0; base < nrows; base += NT / 8) {
    const int rl = base + (threadIdx.x >> 3);
    if (rl < nrows) {
      const int k2 = threadIdx.x & 7;
      float2* row = A + (row_lo + rl) * P;
      float2 u[16];
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) u[k1] = row[k1 + 17 * k2];
      dft<16, true>(u);
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) {
        const float2 w = sTw[n1 * k2];
        row[n1 + 17 * k2] = cmul(u[n1], make_float2(w.x, -w.y));
      }
    }
  }
  __syncthreads();
  for (int base = 0; base < nrows; base += NT / 16) {
    const int rl = base + (threadIdx.x >> 4);
    if (rl < nrows) {
      const int n1 = threadIdx.x & 15;
      float2* row = A + (row_lo + rl) * P;
      float2 v[8];
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) v[k2] = row[n1 + 17 * k2];
      dft<8, true>(v);
#pragma unroll
      for (int n2 = 0; n2 < 8; ++n2) row[n1 + 17 * n2] = v[n2];
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Column pass: forward 128-point transforms of the 128 column positions,
// spectral product, inverse transforms; rows stay in natural order (n1 + 16 n2).
// Split in three steps so that spectra can be kept across PSF pairs in a
// per-CTA scratch spectrum (scr, [kr][c] layout, written and read back by the
// same thread only):
//   col_fwd1: 8-point DFTs over n2 and twiddles (tasks (c, n1)).
//   col_mid:  16-point DFT over n1 (or the stored spectrum), product with
//             F(kr, c) built from the pair's permuted spectra h1, h2, optional
//             accumulation through scr, inverse 16-point DFT (tasks (c, k2)).
//   col_inv3: inverse 8-point DFTs over k2 back to natural rows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void col_fwd1(float2* A, const float2* sTw) {
  const int c = threadIdx.x & (S - 1);
  const int p = (c & 15) + 17 * (c >> 4);
  const int t0 = threadIdx.x >> 7;   // 0..3, uniform in a warp
#pragma unroll 1
  for (int j = 0; j < 4; ++j) {
    const int n1 = t0 + 4 * j;
    float2 v[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) v[n2] = A[(n1 + 16 * n2) * P + p];
    dft<8, false>(v);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) A[(n1 + 16 * k2) * P + p] = k2 ? cmul(v[k2], sTw[n1 * k2]) : v[k2];
  }
  __syncthreads();
}

// load_spec:  take the column spectrum from scr instead of transforming A
// store_spec: save the column spectrum to scr before the product
// accum_in:   add the spectrum accumulated in scr to the product
// final:      run the inverse transform into A; otherwise save the product
//             (plus accumulation) to scr and stop
template <bool ADJ>
__device__ __forceinline__ void col_mid(float2* A, const float2* sTw, const float2* __restrict__ h1,
                                        const float2* __restrict__ h2, float2* __restrict__ scr,
                                        bool load_spec, bool store_spec, bool accum_in,
                                        bool final) {
  const int c = threadIdx.x & (S - 1);
  const int p = (c & 15) + 17 * (c >> 4);
  const int t0 = threadIdx.x >> 7;
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    const int k2 = t0 + 4 * j;
    float2 u[16];
    if (load_spec) {
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) u[k1] = scr[(k2 + 8 * k1) * S + c];
    } else {
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) u[n1] = A[(n1 + 16 * k2) * P + p];
      dft<16, false>(u);
      if (store_spec) {
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) scr[(k2 + 8 * k1) * S + c] = u[k1];
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
      const int kr = k2 + 8 * k1;
      const float2 a = h1[kr * S + c];
      const float2 b = h2 ? h2[kr * S + c] : make_float2(0.f, 0.f);
      // H:   F = Hh1 - i Hh2          H^T: F = conj(Hh1) + i conj(Hh2)
      const float2 f = ADJ ? make_float2(a.x + b.y, b.x - a.y) : make_float2(a.x + b.y, a.y - b.x);
      u[k1] = cmul(u[k1], f);
      if (accum_in) u[k1] = cadd(u[k1], scr[kr * S + c]);
    }
    if (!final) {
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) scr[(k2 + 8 * k1) * S + c] = u[k1];
      continue;
    }
    dft<16, true>(u);
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) {
      const float2 w = sTw[n1 * k2];
      A[(n1 + 16 * k2) * P + p] = cmul(u[n1], make_float2(w.x, -w.y));
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void col_inv3(float2* A) {
  const int c = threadIdx.x & (S - 1);
  const int p = (c & 15) + 17 * (c >> 4);
  const int t0 = threadIdx.x >> 7;
#pragma unroll 1
  for (int j = 0; j < 4; ++j) {
    const int n1 = t0 + 4 * j;
    float2 v[8];
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) v[k2] = A[(n1 + 16 * k2) * P + p];
    dft<8, true>(v);
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) A[(n1 + 16 * n2) * P + p] = v[n2];
  }
  __syncthreads();
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

struct PairSched {
  int np, nb;       // active PSFs, active grid columns
  __device__ void psf(const WorkItem& w, int j, int& a, int& b) const {
    a = w.a_lo + j / nb;
    b = w.b_lo + j % nb;
  }
};

// ---------------------------------------------------------------------------
// H: output y-block block (r0, c0) of size b; input x rows r0 .. r0 + S - 1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT, 1) fft_H_kernel(const OpArgs A) {
  extern __shared__ __align__(16) float2 buf[];
  float2* scr = A.scratch + (size_t)blockIdx.x * S * S;  // this CTA's spectrum accumulator
  __shared__ float sw[4][S];
  __shared__ float2 sTw[S];
  __shared__ double red[NT / 32];
  for (int e = threadIdx.x; e < S; e += NT) sTw[e] = c_w128[e];
  const int K = A.K, b = S - K + 1;
  const float2* spec = A.spec;

  __shared__ WorkItem wi;
  __shared__ TileDesc td;
  __shared__ int s_item;
  for (;;) {
    // dynamic scheduling: items are sorted heaviest first; each is computed
    // whole by one CTA, so the result does not depend on the assignment
    __syncthreads();
    if (threadIdx.x == 0) {
      s_item = atomicAdd(A.counter, 1);
      if (s_item < A.n_work) {
        wi = A.work[s_item];
        td = A.tiles[wi.tile];
      }
    }
    __syncthreads();
    const int item = s_item;
    if (item >= A.n_work) break;
    const int nb = wi.b_hi - wi.b_lo + 1;
    const int np = (wi.a_hi - wi.a_lo + 1) * nb;
    const PairSched ps{np, nb};
    if (np == 0) {   // no PSF touches the block: the output is zero
      for (int e = threadIdx.x; e < S * P; e += NT) buf[e] = make_float2(0.f, 0.f);
      __syncthreads();
    }

    for (int j = 0; j < np; j += 2) {
      int a1, b1, a2 = -1, b2 = -1;
      ps.psf(wi, j, a1, b1);
      const bool two = j + 1 < np;
      const bool last = j + 2 >= np;
      if (two) ps.psf(wi, j + 1, a2, b2);
      __syncthreads();
      for (int e = threadIdx.x; e < S; e += NT) {
        const int R = wi.r0 + e, C = wi.c0 + e;
        const bool rin = R < td.nxr, cin = C < td.nxc;
        const WTab tr = rin ? A.wrow[td.wr0 + R] : WTab{0, 0.f, 0.f, 0};
        const WTab tc = cin ? A.wcol[td.wc0 + C] : WTab{0, 0.f, 0.f, 0};
        sw[0][e] = rin ? wsel(tr, a1) : 0.f;
        sw[1][e] = cin ? wsel(tc, b1) : 0.f;
        sw[2][e] = (rin && two) ? wsel(tr, a2) : 0.f;
        sw[3][e] = (cin && two) ? wsel(tc, b2) : 0.f;
      }
      __syncthreads();
      {
        // thread -> column n, rows m = m0 + 4 k
        const int n = threadIdx.x & (S - 1), m0 = threadIdx.x >> 7;
        const float wc1 = sw[1][n], wc2 = sw[3][n];
        const bool cin = wc1 != 0.f || wc2 != 0.f;
        const float* src = A.in + td.xoff + (int64_t)(wi.r0 + m0) * td.xpitch + (wi.c0 + n);
        const int64_t step = 4 * (int64_t)td.xpitch;
        float2* dst = buf + m0 * P + pos(n);
#pragma unroll 4
        for (int m = m0; m < S; m += 4, src += step, dst += 4 * P) {
          const float w1 = sw[0][m] * wc1, w2 = sw[2][m] * wc2;
          float v = 0.f;
          if (cin && (w1 != 0.f || w2 != 0.f)) v = *src;
          *dst = make_float2(w1 * v, w2 * v);
        }
      }
      __syncthreads();
      row_fwd(buf, sTw);
      col_fwd1(buf, sTw);
      // sum over pairs of FFT(w1 x + i w2 x) (Hh1 - i Hh2) in scr; one inverse at the end
      col_mid<false>(buf, sTw, spec + (size_t)(a1 * A.Gc + b1) * S * S,
                     two ? spec + (size_t)(a2 * A.Gc + b2) * S * S : nullptr, scr, false, false,
                     j > 0, last);
      if (last) {
        col_inv3(buf);
        row_inv(buf, sTw, K - 1, b);
      }
    }

    // epilogue: residual, plain output or objective partial (one per work item)
    double part = 0.0;
    {
      const int jl = threadIdx.x & (S - 1), i0 = threadIdx.x >> 7;
      const int jj = wi.c0 + jl;
      if (jl < b && jj < td.nyc) {
        for (int il = i0; il < b; il += 4) {
          const int i = wi.r0 + il;
          if (i >= td.nyr) break;
          const float v = buf[(il + K - 1) * P + pos(jl + K - 1)].x;
          if (A.mode == OP_PLAIN) {
            A.out[td.yoff + (int64_t)i * td.ypitch + jj] = v;
          } else {
            const int64_t gi = (int64_t)(td.xr0 + i) * A.wy + (td.xc0 + jj);
            const float wt = A.W ? A.W[gi] : 1.f;
            const float d = v - A.y[gi];
            if (A.mode == OP_RESID)
              A.out[td.yoff + (int64_t)i * td.ypitch + jj] = wt * d;
            else
              part += (double)wt * (double)d * (double)d;
          }
        }
      }
    }
    if (A.mode == OP_OBJ) {
      const double t = block_sum(part, red);
      if (threadIdx.x == 0) A.partials[item] = t;
    }
  }
}

// p = kappa (dr, dc) of the Huber prior at tile pixel (R, C) from the staged
// iterate (smem position (li, lj), pitch SPW); zero above / left of the tile.
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
// H^T: output x block (R0, C0) of size b; input r rows R0 - (K-1) .. R0 - K + S.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT, 1) fft_Ht_kernel(const OpArgs A) {
  extern __shared__ __align__(16) float2 buf[];
  float* g = reinterpret_cast<float*>(buf + S * P);     // b x b outputs, thread-owned slots
  float2* scr = A.scratch + (size_t)blockIdx.x * S * S;  // this CTA's spectrum of r
  __shared__ float2 sTw[S];
  __shared__ float sw[4][S];
  const int K = A.K, b = S - K + 1;
  const float2* spec = A.spec;
  for (int e = threadIdx.x; e < S; e += NT) sTw[e] = c_w128[e];

  __shared__ WorkItem wi;
  __shared__ TileDesc td;
  __shared__ int s_item;
  for (;;) {
    // dynamic scheduling: items are sorted heaviest first; each is computed
    // whole by one CTA, so the result does not depend on the assignment
    __syncthreads();
    if (threadIdx.x == 0) {
      s_item = atomicAdd(A.counter, 1);
      if (s_item < A.n_work) {
        wi = A.work[s_item];
        td = A.tiles[wi.tile];
      }
    }
    __syncthreads();
    const int item = s_item;
    if (item >= A.n_work) break;
    const int nb = wi.b_hi - wi.b_lo + 1;
    const int np = (wi.a_hi - wi.a_lo + 1) * nb;
    const PairSched ps{np, nb};
    for (int e = threadIdx.x; e < b * b; e += NT) g[e] = 0.f;
    __syncthreads();

    for (int j = 0; j < np; j += 2) {
      int a1, b1, a2 = -1, b2 = -1;
      ps.psf(wi, j, a1, b1);
      const bool two = j + 1 < np;
      if (two) ps.psf(wi, j + 1, a2, b2);
      __syncthreads();
      // output weights of the pair (rows / columns of the b x b output block)
      for (int e = threadIdx.x; e < S; e += NT) {
        const int R = wi.r0 + e, C = wi.c0 + e;
        const bool rin = e < b && R < td.nxr, cin = e < b && C < td.nxc;
        const WTab tr = rin ? A.wrow[td.wr0 + R] : WTab{0, 0.f, 0.f, 0};
        const WTab tc = cin ? A.wcol[td.wc0 + C] : WTab{0, 0.f, 0.f, 0};
        sw[0][e] = rin ? wsel(tr, a1) : 0.f;
        sw[1][e] = cin ? wsel(tc, b1) : 0.f;
        sw[2][e] = (rin && two) ? wsel(tr, a2) : 0.f;
        sw[3][e] = (cin && two) ? wsel(tc, b2) : 0.f;
      }
      const float2* h1 = spec + (size_t)(a1 * A.Gc + b1) * S * S;
      const float2* h2 = two ? spec + (size_t)(a2 * A.Gc + b2) * S * S : nullptr;
      if (j == 0) {
        // thread -> column n, rows m = m0 + 4 k of the residual region
        const int n = threadIdx.x & (S - 1), m0 = threadIdx.x >> 7;
        const int rx = wi.c0 - (K - 1) + n;
        const bool cin = rx >= 0 && rx < td.nyc;
        const int ry0 = wi.r0 - (K - 1) + m0;
        const float* src = A.in + td.yoff + (int64_t)ry0 * td.ypitch + rx;
        const int64_t step = 4 * (int64_t)td.ypitch;
        float2* dst = buf + m0 * P + pos(n);
#pragma unroll 4
        for (int m = m0; m < S; m += 4, src += step, dst += 4 * P) {
          const int ry = ry0 + (m - m0);
          float v = 0.f;
          if (cin && ry >= 0 && ry < td.nyr) v = *src;
          *dst = make_float2(v, 0.f);
        }
        __syncthreads();
        row_fwd(buf, sTw);
        col_fwd1(buf, sTw);
        col_mid<true>(buf, sTw, h1, h2, scr, false, np > 2, false, true);
      } else {
        // FFT(r) of this block was kept in scr by the first pair
        col_mid<true>(buf, sTw, h1, h2, scr, true, false, false, true);
      }
      col_inv3(buf);
      row_inv(buf, sTw, 0, b);
      {
        const int jj = threadIdx.x & (S - 1), i0 = threadIdx.x >> 7;
        if (jj < b) {
          const float wc1 = sw[1][jj], wc2 = sw[3][jj];
          const float2* srcp = buf + i0 * P + pos(jj);
          float* a = g + i0 * b + jj;
          for (int i = i0; i < b; i += 4, srcp += 4 * P, a += 4 * b) {
            const float2 cv = *srcp;
            *a = fmaf(sw[2][i] * wc2, cv.y, fmaf(sw[0][i] * wc1, cv.x, *a));
          }
        }
      }
    }

    if (A.mode == OP_PLAIN) {
      for (int e = threadIdx.x; e < b * b; e += NT) {
        const int R = wi.r0 + e / b, C = wi.c0 + e % b;
        if (R < td.nxr && C < td.nxc) A.out[td.xoff + (int64_t)R * td.xpitch + C] = g[e];
      }
      continue;
    }

    // OP_STEP: grad = g + lambda D^T psi(D w) + alpha (w - u); w_next = max(0, w - tau grad)
    __syncthreads();
    float* sW = reinterpret_cast<float*>(buf);
    const int SPW = b + 2;
    for (int e = threadIdx.x; e < SPW * SPW; e += NT) {
      const int ir = e / SPW, ic = e - ir * SPW;
      const int R = wi.r0 - 1 + ir, C = wi.c0 - 1 + ic;
      float v = 0.f;
      if (R >= 0 && R < td.nxr && C >= 0 && C < td.nxc)
        v = A.w[td.xoff + (int64_t)R * td.xpitch + C];
      sW[e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += NT) {
      const int i = e / b, jj = e % b;
      const int R = wi.r0 + i, C = wi.c0 + jj;
      if (R >= td.nxr || C >= td.nxc) continue;
      const int li = i + 1, lj = jj + 1;
      float pr, pc, pru, pcu, prl, pcl;
      huber_p(sW, SPW, li, lj, R, C, td.nxr, td.nxc, A.delta, pr, pc);
      huber_p(sW, SPW, li - 1, lj, R - 1, C, td.nxr, td.nxc, A.delta, pru, pcu);
      huber_p(sW, SPW, li, lj - 1, R, C - 1, td.nxr, td.nxc, A.delta, prl, pcl);
      const float hub = pru - pr + pcl - pc;
      const float wv = sW[li * SPW + lj];
      const float alpha = A.gamma * A.omr[td.omr_off + R] * A.omc[td.omc_off + C];
      const int64_t idx = td.xoff + (int64_t)R * td.xpitch + C;
      const float grad = g[e] + A.lambda * hub + alpha * (wv - A.u[idx]);
      A.out[idx] = fmaxf(0.f, wv - td.tau * grad);
    }
  }
}

constexpr size_t kSmemH = sizeof(float2) * (size_t)S * P;
constexpr size_t kSmem = sizeof(float2) * (size_t)S * P + sizeof(float) * (size_t)BMAX * BMAX;

}  // namespace

int fft_size() { return S; }

int fft_block(int K) { return S - K + 1; }

bool fft_supported(int K) { return K >= 1 && S - K + 1 >= 32; }

// Uploads the twiddle table and sets the kernels' shared-memory limit on the
// current device (plan creation; never during stream capture).
cudaError_t fft_prepare() {
  float2 w[S];
  for (int k = 0; k < S; ++k) {
    const double a = -2.0 * 3.14159265358979323846 * k / S;
    w[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  cudaError_t e = cudaMemcpyToSymbol(c_w128, w, sizeof w);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fft_H_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemH);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fft_Ht_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSmem);
}

// Spectra of the zero-padded PSFs on the S x S grid, in FP64 on the host:
// Hh(kr, kc) = sum_{m,n < K} h(m, n) exp(-2 pi i (kr m + kc n) / S) / S^2,
// row kr natural, column frequency kc stored at the column position the
// kernels' row transform leaves it in.
void fft_spectra(const float* psfs, int G, int K, std::vector<float2>& out) {
  std::vector<double> cr(S), ci(S);
  for (int j = 0; j < S; ++j) {
    const double a = -2.0 * 3.14159265358979323846 * j / S;
    cr[j] = std::cos(a);
    ci[j] = std::sin(a);
  }
  out.assign((size_t)G * S * S, make_float2(0.f, 0.f));
  std::vector<double> tr((size_t)K * S), ti((size_t)K * S);
  const double scale = 1.0 / ((double)S * S);
  for (int g = 0; g < G; ++g) {
    const float* h = psfs + (size_t)g * K * K;
    for (int m = 0; m < K; ++m)
      for (int kc = 0; kc < S; ++kc) {
        double sr = 0.0, si = 0.0;
        for (int n = 0; n < K; ++n) {
          const int j = (kc * n) % S;
          sr += h[m * K + n] * cr[j];
          si += h[m * K + n] * ci[j];
        }
        tr[(size_t)m * S + kc] = sr;
        ti[(size_t)m * S + kc] = si;
      }
    for (int kr = 0; kr < S; ++kr)
      for (int kc = 0; kc < S; ++kc) {
        double sr = 0.0, si = 0.0;
        for (int m = 0; m < K; ++m) {
          const int j = (kr * m) % S;
          const double ar = tr[(size_t)m * S + kc], ai = ti[(size_t)m * S + kc];
          sr += ar * cr[j] - ai * ci[j];
          si += ar * ci[j] + ai * cr[j];
        }
        // stored at the column position c of frequency kc = (c >> 4) + 8 (c & 15)
        const int c = (kc >> 3) + 16 * (kc & 7);
        out[((size_t)g * S + kr) * S + c] = make_float2((float)(sr * scale), (float)(si * scale));
      }
  }
}

cudaError_t launch_fft_H(const OpArgs& a, cudaStream_t s, int grid) {
  if (a.n_work <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  fft_H_kernel<<<std::min(grid, a.n_work), NT, kSmemH, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fft_Ht(const OpArgs& a, cudaStream_t s, int grid) {
  if (a.n_work <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  fft_Ht_kernel<<<std::min(grid, a.n_work), NT, kSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dv
