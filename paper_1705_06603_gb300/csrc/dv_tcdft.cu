// Block-DFT form of the shift-variant operator H of Sec. II-B on the tensor
// cores (tcgen05, FP16 operands, FP32 accumulation in tensor memory).
//
// Overlap-save on 128 x 128 blocks, as the FP32 block-FFT path: a CTA owns a
// b x b block of H's output (b = 129 - K) and reads the 128 x 128 x window
// below it.  For every PSF p active on the block, X_p = w_p . x (zero outside
// the tile) is transformed by two dense DFT stages, Z_p = F X_p F with
// F[k][n] = exp(-2 pi i k n / 128), multiplied by the PSF's spectrum, and the
// products are summed; one inverse transform of the sum, cropped to rows and
// columns K - 1 .. 127, is the block of H x (the non-circulant local blur of
// Sec. II-B: circular convolution of size 128, then the valid part).
//
// Each DFT stage is a GEMM on the tensor cores with the constant matrices
// [Fr; Fi] (cos and -sin, FP16) in shared memory:
//   stage 1  Y^T[c][kr]  = sum_r X[r][c] F[kr][r]          (M = c, N = re|im kr)
//   stage 2  Z^T[kc][kr] = sum_c F[kc][c] Y[kr][c]          (M = kc, N = re|im kr)
//            as Fr [Yr | Yi] + Fi [-Yi | Yr] over one buffer [-Yi | Yr | Yi]
//   inverse  T^T[c][kr]  = sum_kc conj F[c][kc] Z[kr][kc]   (Fr [Zr | Zi] + Fi [Zi | -Zr])
//            x[r][c]     = Re sum_kr conj F[r][kr] T[kr][c]  (Fr Tr + Fi Ti)
// Operands are K-major, no swizzle: a matrix of R rows and K columns is stored
// as K / 8 panels of R 16-byte rows (a panel stride padded by 16 bytes), so a
// 16-wide k-step is two consecutive panels (LBO = panel stride, SBO = 128).
// Between stages the staging warps read the accumulators (each warp owns 32
// tensor-memory lanes and half of the columns), round to FP16 and write the
// next operand; the spectral products accumulate in FP32 in tensor memory.
// Scaling keeps the FP16 values in range: the spectra carry 1 / 128 and the
// first inverse stage's result another 1 / 128 (the inverse DFT's 1 / 128^2).
//
// Warps 0-7 stage operands and run the epilogue, one lane of warp 8 allocates
// tensor memory and issues the MMAs.  The grid is persistent (one CTA per SM,
// items from an atomic counter, heaviest first).  Every wait is bounded.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dv_internal.cuh"
#include "dv_tcgen05.cuh"

namespace dv {
namespace {

using namespace tcg;

constexpr int S = 128;                      // transform size
constexpr int NWS = 8;                      // staging / epilogue warps
constexpr int NTS = 32 * NWS;
constexpr int NTH = NTS + 32;               // + the MMA warp
constexpr int CROWS = 2 * S;                // [Fr; Fi]
constexpr int CPAN = CROWS * 16 + 16;       // panel stride (bytes) of the constants
constexpr int CBYTES = (S / 8) * CPAN;
constexpr int XPAN = S * 16 + 16;           // 128-row operand
constexpr int XBYTES = (S / 8) * XPAN;
constexpr int YROWS = 3 * S;                // [-Yi | Yr | Yi] or [Zr | Zi | -Zr]
constexpr int YPAN = YROWS * 16 + 16;
constexpr int YBYTES = (S / 8) * YPAN;
constexpr int kHdrD = 1024;
constexpr int SMEM_D = kHdrD + CBYTES + XBYTES + YBYTES + 2 * S * 4;
constexpr uint32_t TMEM_COLS = 512;         // D [0, 256), Z sum [256, 512)
static_assert(SMEM_D <= 227 * 1024, "shared memory");
static_assert(YBYTES >= 2 * XBYTES, "T operands fit in the Y buffer");
static_assert(CPAN % 16 == 0 && XPAN % 16 == 0 && YPAN % 16 == 0, "alignment");

struct BarsD {
  uint64_t bx, by, bd, fin;
  uint32_t tmem;
  int abort;
  int item;
};
static_assert(sizeof(BarsD) <= 256, "barrier header");

__device__ __forceinline__ void sync_st() { named_sync<NTS>(); }
__device__ __forceinline__ bool all_st(bool v) { return named_all<NTS>(v); }

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ void st_h(unsigned char* base, int off, float v) {
  *reinterpret_cast<__half*>(base + off) = __float2half_rn(v);
}

// Byte offset of element (row, k) in a panel layout with panel stride pan.
__device__ __forceinline__ int el(int row, int k, int pan) { return (k >> 3) * pan + 16 * row + 2 * (k & 7); }

// One GEMM chain of 8 k-steps (K = 128): D (+)= A B^T, A rows from a0, B rows
// from b0 (shared-memory addresses of row 0 of panel 0).
__device__ __forceinline__ void chain(uint32_t d, uint32_t a0, uint32_t apan, uint32_t b0,
                                      uint32_t bpan, uint32_t id, bool acc) {
  const uint64_t ad = sdesc(a0, apan), bd = sdesc(b0, bpan);
#pragma unroll
  for (int j = 0; j < 8; ++j)
    mma_bf16(d, ad + (uint64_t)(j * 2 * (apan >> 4)), bd + (uint64_t)(j * 2 * (bpan >> 4)), id,
            (acc || j > 0) ? 1u : 0u);
}

__global__ void __launch_bounds__(NTH, 1) dft_H_kernel(const OpArgs A) {
  extern __shared__ __align__(1024) unsigned char smem[];
  BarsD* H = reinterpret_cast<BarsD*>(smem);
  unsigned char* sC = smem + kHdrD;
  unsigned char* sX = sC + CBYTES;
  unsigned char* sY = sX + XBYTES;
  float* sWr = reinterpret_cast<float*>(sY + YBYTES);
  float* sWc = sWr + S;
  __shared__ WorkItem wi;
  __shared__ TileDesc td;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = A.K, b = S - K + 1;
  if (tid == 0) {
    mbar_init(&H->bx, NTS);
    mbar_init(&H->by, NTS);
    mbar_init(&H->bd, 1);
    mbar_init(&H->fin, 1);
    H->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == NWS) tmem_alloc(&H->tmem, TMEM_COLS);
  // constants [Fr; Fi] (the plan's byte image of the panels)
  for (int e = tid; e < CBYTES / 16; e += NTH)
    reinterpret_cast<uint4*>(sC)[e] = __ldg(reinterpret_cast<const uint4*>(A.tcop) + e);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = H->tmem;
  const uint32_t aC = saddr(sC), aX = saddr(sX), aY = saddr(sY);
  const uint32_t id256 = idesc(0, 128, 256), id128 = idesc(0, 128, 128);
  // phase counters (uses of each barrier so far)
  uint32_t nx = 0, ny = 0, nd = 0;
  const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
  const int h = warp >> 2;          // column half of the staging warp
  const int L = 32 * (warp & 3) + lane;   // its tensor-memory lane
  bool ok = true;

  for (;;) {
    // the previous item's tensor-memory reads are ordered before the next
    // item's MMAs
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      const int it = atomicAdd(A.counter, 1);
      H->item = it;
      if (it < A.n_work) {
        wi = A.work[it];
        td = A.tiles[wi.tile];
      }
    }
    __syncthreads();
    tc_fence_after();
    if (H->item >= A.n_work || !ok || *(volatile int*)&H->abort) break;
    const int nb = wi.b_hi - wi.b_lo + 1;
    const int np = (wi.a_hi - wi.a_lo + 1) * nb;

    if (warp == NWS) {
      // ---------------------------------------------------------- MMA lane
      if (lane == 0) {
        for (int p = 0; p < np && ok; ++p) {
          ok = wait_bar(&H->bx, nx++ & 1, &H->abort, A.err, A.wait_ns ? A.wait_ns : kWaitNs);
          if (!ok) break;
          tc_fence_after();
          chain(tbase, aX, XPAN, aC, CPAN, id256, false);                  // Y^T
          tc_commit(&H->bd);
          ok = wait_bar(&H->by, ny++ & 1, &H->abort, A.err, A.wait_ns ? A.wait_ns : kWaitNs);
          if (!ok) break;
          tc_fence_after();
          chain(tbase, aC, CPAN, aY + 16 * S, YPAN, id256, false);         // Fr [Yr | Yi]
          chain(tbase, aC + 16 * S, CPAN, aY, YPAN, id256, true);          // Fi [-Yi | Yr]
          tc_commit(&H->bd);
        }
        if (ok && np > 0) {
          ok = wait_bar(&H->by, ny++ & 1, &H->abort, A.err, A.wait_ns ? A.wait_ns : kWaitNs);
          if (ok) {
            tc_fence_after();
            chain(tbase, aC, CPAN, aY, YPAN, id256, false);                // Fr [Zr | Zi]
            chain(tbase, aC + 16 * S, CPAN, aY + 16 * S, YPAN, id256, true);   // Fi [Zi | -Zr]
            tc_commit(&H->bd);
            ok = wait_bar(&H->by, ny++ & 1, &H->abort, A.err, A.wait_ns ? A.wait_ns : kWaitNs);
          }
          if (ok) {
            tc_fence_after();
            chain(tbase, aC, CPAN, aX, XPAN, id128, false);                // Fr Tr
            chain(tbase, aC + 16 * S, CPAN, aY, XPAN, id128, true);        // Fi Ti
            tc_commit(&H->bd);
          }
        }
        if (!ok) *(volatile int*)&H->abort = 1;
      }
      __syncwarp();
      continue;
    }

    // -------------------------------------------------- staging / epilogue
    const float* img = A.in + td.xoff;
    // X_p^T into sX: element (m = c, k = r) = w_p(r0 + r, c0 + c) x(r0 + r, c0 + c)
    auto stage_x = [&](int p) {
      const int ga = wi.a_lo + p / nb, gb = wi.b_lo + p % nb;
      for (int e = tid; e < S; e += NTS) {
        const int R = wi.r0 + e, C = wi.c0 + e;
        sWr[e] = R < td.nxr ? wsel(A.wrow[td.wr0 + R], ga) : 0.f;
        sWc[e] = C < td.nxc ? wsel(A.wcol[td.wc0 + C], gb) : 0.f;
      }
      sync_st();
      // item (c, q): column c, rows 8q .. 8q + 7; threads of a warp take
      // consecutive columns (coalesced loads)
      for (int e0 = tid; e0 < S * (S / 8); e0 += 2 * NTS) {
        float v[2][8];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int e = e0 + u * NTS;
          const int c = e & (S - 1), q = e >> 7;
          const int C = wi.c0 + c;
          const float wc = sWc[c];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int r = 8 * q + t, R = wi.r0 + r;
            const float w = sWr[r] * wc;
            v[u][t] = (w != 0.f && R < td.nxr && C < td.nxc)
                          ? w * __ldg(img + (int64_t)R * td.xpitch + C) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int e = e0 + u * NTS;
          const int c = e & (S - 1), q = e >> 7;
          *reinterpret_cast<uint4*>(sX + q * XPAN + 16 * c) =
              make_uint4(pack_h2(v[u][0], v[u][1]), pack_h2(v[u][2], v[u][3]),
                         pack_h2(v[u][4], v[u][5]), pack_h2(v[u][6], v[u][7]));
        }
      }
      fence_async_smem();
    };
    auto wait_d = [&]() {
      const bool w = wait_bar(&H->bd, nd++ & 1, &H->abort, A.err, A.wait_ns ? A.wait_ns : kWaitNs);
      ok = all_st(w);
      tc_fence_after();
      return ok;
    };
    auto arrive = [&](uint64_t* bar) {
      tc_fence_before();
      mbar_arrive(bar);
    };

    if (np > 0) {
      stage_x(0);
      arrive(&H->bx);
    }
    for (int p = 0; p < np && ok; ++p) {
      // Y^T (lane c): columns 0..127 = Yr[kr], 128..255 = Yi[kr]; this warp
      // takes half h -> rows of the buffer [-Yi | Yr | Yi]
      if (!wait_d()) break;
      for (int c0 = 0; c0 < S; c0 += 16) {
        uint32_t r[16];
        tmem_ld16_nowait(tbase + lanes + (uint32_t)(S * h + c0), r);
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const float v = __uint_as_float(r[t]);
          const int kr = c0 + t;
          if (h == 0) {
            st_h(sY, el(S + kr, L, YPAN), v);
          } else {
            st_h(sY, el(kr, L, YPAN), -v);
            st_h(sY, el(2 * S + kr, L, YPAN), v);
          }
        }
      }
      fence_async_smem();
      arrive(&H->by);
      // the next PSF's X (its MMAs wait until the product below has read D)
      if (p + 1 < np) stage_x(p + 1);
      if (!wait_d()) break;
      // Z^T (lane kc): columns kr (re) and S + kr (im); sum += Z . Hh_p over
      // kr in this warp's half
      const int ga = wi.a_lo + p / nb, gb = wi.b_lo + p % nb;
      const float2* hh = A.spec + (size_t)(ga * A.Gc + gb) * S * S;
      for (int k0 = 64 * h; k0 < 64 * h + 64; k0 += 16) {
        uint32_t zr[16], zi[16], ar[16], ai[16];
        float2 hv[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) hv[t] = __ldg(hh + (size_t)(k0 + t) * S + L);
        tmem_ld16_nowait(tbase + lanes + (uint32_t)k0, zr);
        tmem_ld16_nowait(tbase + lanes + (uint32_t)(S + k0), zi);
        if (p > 0) {
          tmem_ld16_nowait(tbase + lanes + (uint32_t)(2 * S + k0), ar);
          tmem_ld16_nowait(tbase + lanes + (uint32_t)(3 * S + k0), ai);
        }
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const float a = __uint_as_float(zr[t]), bb = __uint_as_float(zi[t]);
          const float re = a * hv[t].x - bb * hv[t].y, im = a * hv[t].y + bb * hv[t].x;
          ar[t] = __float_as_uint(p > 0 ? __uint_as_float(ar[t]) + re : re);
          ai[t] = __float_as_uint(p > 0 ? __uint_as_float(ai[t]) + im : im);
        }
        tmem_st16_nowait(tbase + lanes + (uint32_t)(2 * S + k0), ar);
        tmem_st16_nowait(tbase + lanes + (uint32_t)(3 * S + k0), ai);
      }
      tmem_wait_st();
      if (p + 1 < np) arrive(&H->bx);   // D read: the next PSF may overwrite it
    }
    float* out = A.out;
    if (np > 0 && ok) {
      // inverse, stage 1 operand: the sum (lane kc) -> [Zr | Zi | -Zr]
      for (int k0 = 64 * h; k0 < 64 * h + 64; k0 += 16) {
        uint32_t ar[16], ai[16];
        tmem_ld16_nowait(tbase + lanes + (uint32_t)(2 * S + k0), ar);
        tmem_ld16_nowait(tbase + lanes + (uint32_t)(3 * S + k0), ai);
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int kr = k0 + t;
          const float zr = __uint_as_float(ar[t]), zi = __uint_as_float(ai[t]);
          st_h(sY, el(kr, L, YPAN), zr);
          st_h(sY, el(S + kr, L, YPAN), zi);
          st_h(sY, el(2 * S + kr, L, YPAN), -zr);
        }
      }
      fence_async_smem();
      arrive(&H->by);
      // T^T (lane c): columns kr (re), S + kr (im), scaled by 1 / 128, into the
      // stage-2 operands Tr (sX) and Ti (sY), rows c, k = kr
      if (wait_d()) {
        for (int k0 = 0; k0 < S; k0 += 16) {
          uint32_t r[16];
          tmem_ld16_nowait(tbase + lanes + (uint32_t)(S * h + k0), r);
          tmem_wait_ld();
          unsigned char* dst = h == 0 ? sX : sY;
#pragma unroll
          for (int t = 0; t < 16; t += 8) {
            const float s = 1.f / S;
            *reinterpret_cast<uint4*>(dst + ((k0 + t) >> 3) * XPAN + 16 * L) = make_uint4(
                pack_h2(s * __uint_as_float(r[t]), s * __uint_as_float(r[t + 1])),
                pack_h2(s * __uint_as_float(r[t + 2]), s * __uint_as_float(r[t + 3])),
                pack_h2(s * __uint_as_float(r[t + 4]), s * __uint_as_float(r[t + 5])),
                pack_h2(s * __uint_as_float(r[t + 6]), s * __uint_as_float(r[t + 7])));
          }
        }
        fence_async_smem();
        arrive(&H->by);
      }
      // x (lane r, columns c): rows and columns K - 1 .. 127 are the block's
      // valid outputs
      if (ok && wait_d()) {
        const int r = L;
        const int i = wi.r0 + r - (K - 1);
        const bool rin = r >= K - 1 && i < td.nyr;
        for (int c0 = 64 * h; c0 < 64 * h + 64; c0 += 16) {
          uint32_t v[16];
          tmem_ld16_nowait(tbase + lanes + (uint32_t)c0, v);
          tmem_wait_ld();
          if (!rin) continue;
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int c = c0 + t, jj = wi.c0 + c - (K - 1);
            if (c < K - 1 || jj >= td.nyc || jj - wi.c0 >= b) continue;
            const float y = __uint_as_float(v[t]);
            if (A.mode == OP_PLAIN) {
              out[td.yoff + (int64_t)i * td.ypitch + jj] = y;
            } else {
              const int64_t gi = (int64_t)(td.xr0 + i) * A.wy + (td.xc0 + jj);
              const float wt = A.W ? A.W[gi] : 1.f;
              out[td.yoff + (int64_t)i * td.ypitch + jj] = wt * (y - A.y[gi]);
            }
          }
        }
      }
    } else if (np == 0 && ok) {
      // no PSF reaches the block: H x is zero there
      for (int e = tid; e < b * b; e += NTS) {
        const int i = wi.r0 + e / b, jj = wi.c0 + e % b;
        if (i >= td.nyr || jj >= td.nyc) continue;
        const int64_t gi = (int64_t)(td.xr0 + i) * A.wy + (td.xc0 + jj);
        const float wt = (A.mode != OP_PLAIN && A.W) ? A.W[gi] : 1.f;
        out[td.yoff + (int64_t)i * td.ypitch + jj] = A.mode == OP_PLAIN ? 0.f : -wt * A.y[gi];
      }
    }
    if (!ok) *(volatile int*)&H->abort = 1;
  }
  // teardown: every MMA this CTA issued has completed before tensor memory is freed
  if (warp == NWS && lane == 0) {
    tc_commit(&H->fin);
    drain_bar(&H->fin, 0, A.err);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == NWS) {
    tc_fence_after();
    tmem_free(tbase, TMEM_COLS);
  }
}

}  // namespace

bool dft_supported(int K) { return K >= 1 && S - K + 1 >= 32; }

cudaError_t dft_prepare() {
  return cudaFuncSetAttribute(dft_H_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_D);
}

// Byte image of the constant operand [Fr; Fi]: 16 panels of 256 16-byte rows
// (padded), row n < 128: cos(2 pi n k / 128), row 128 + n: -sin(2 pi n k / 128),
// k the column; FP16, from FP64 on the host.
void dft_constants(std::vector<uint8_t>& out) {
  out.assign(CBYTES, 0);
  for (int n = 0; n < CROWS; ++n)
    for (int k = 0; k < S; ++k) {
      const int nn = n & (S - 1);
      const double a = 2.0 * 3.14159265358979323846 * (double)((nn * k) % S) / S;
      const float v = n < S ? (float)std::cos(a) : (float)-std::sin(a);
      const __half hv = __float2half_rn(v);
      std::memcpy(out.data() + (k >> 3) * CPAN + 16 * n + 2 * (k & 7), &hv, 2);
    }
}

// Spectra of the zero-padded PSFs, natural order [kr][kc], scaled by 1 / 128:
// Hh(kr, kc) = sum_{m, n < K} h(m, n) exp(-2 pi i (kr m + kc n) / 128) / 128, FP64.
void dft_spectra(const float* psfs, int G, int K, std::vector<float2>& out) {
  std::vector<double> cr(S), ci(S);
  for (int j = 0; j < S; ++j) {
    const double a = -2.0 * 3.14159265358979323846 * j / S;
    cr[j] = std::cos(a);
    ci[j] = std::sin(a);
  }
  out.assign((size_t)G * S * S, make_float2(0.f, 0.f));
  std::vector<double> tr((size_t)K * S), ti((size_t)K * S);
  for (int g = 0; g < G; ++g) {
    const float* hp = psfs + (size_t)g * K * K;
    for (int m = 0; m < K; ++m)
      for (int kc = 0; kc < S; ++kc) {
        double sr = 0.0, si = 0.0;
        for (int n = 0; n < K; ++n) {
          const int j = (kc * n) % S;
          sr += hp[m * K + n] * cr[j];
          si += hp[m * K + n] * ci[j];
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
        out[((size_t)g * S + kr) * S + kc] = make_float2((float)(sr / S), (float)(si / S));
      }
  }
}

cudaError_t launch_dft_H(const OpArgs& a, cudaStream_t s, int grid) {
  if (a.n_work <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  dft_H_kernel<<<std::min(grid, a.n_work), NTH, SMEM_D, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dv
