// Block-DFT forms of the shift-variant operator H of Sec. II-B and of its
// adjoint on the tensor cores (tcgen05, FP16 operands, FP32 accumulation in
// tensor memory), and the Local-Solver step that follows the adjoint.
//
// Overlap-save on 128 x 128 blocks.  H: a work item is a b x b block of the
// output (b = 129 - K) and the 128 x 128 window of x below it.  For every PSF
// p = (a, b) active on the block (Eq. (2): first-order interpolation, weights
// w_p(r, c) = wr_a(r) wc_b(c)), X_p = w_p . x is transformed, multiplied by
// the PSF's spectrum, and the products are summed; one inverse transform of the
// sum, cropped to rows and columns K - 1 .. 127, is the block of H x (the
// valid part of a circular convolution of size 128 is the non-circulant
// local blur).  H^T: a work item is a b x b block of x and the 128 x 128
// window of r from K - 1 rows and columns above and left of it (zero outside
// the tile); the window is transformed once, multiplied by each PSF's
// conjugate spectrum (correlation), transformed back, and the PSF's weights
// applied to the valid rows and columns 0 .. b - 1.
//
// The input is real, so only half of every spectrum is formed (k = 0 .. 64
// along the first transformed axis; the other half is its conjugate mirror).
// With F[k][n] = exp(-2 pi i k n / 128) = Fr + i Fi, each stage is a GEMM on
// the tensor cores, ordered so that every tensor-memory lane (a thread) owns a
// row of the next stage's operand:
//   F1  Y'[j][c] = sum_r A1[j][r] v[r][c]   (H: v = wr_a x, once per PSF grid
//        row a; H^T: v = r, once per block).  A1 rows 2k = Fr(k), 2k + 1 =
//        Fi(k) (k < 64), row 1 = Fr(64): the packed real and imaginary parts
//        of Y(k) = F v along r (Y(0), Y(64) are real, Y(128 - k) = conj Y(k))
//   F2  P = Fr (wc_b Y')^T, Q = Fi (wc_b Y')^T   (M = kc, N = j; H^T: wc = 1)
//        Z(k)[kc] = P[2k] - Q[2k+1] + i (Q[2k] + P[2k+1])   (k = 0, 64 apart)
//   H: product  S(k)[kc] += Z(k)[kc] Hh_p(k, kc) over the PSFs (FP32, tensor
//        memory), then one inverse per block; H^T: per PSF T = Z conj(Hh_p)
//        and one inverse, the row weights wr_a applied to U (rows r) and
//        summed over a inside I2, the column weight wc_b to I2's result as it
//        is added to H^T r (tensor memory)
//   I1  U[r][kc] = sum_k alpha_k exp(+2 pi i r k / 128) S(k)[kc]   (alpha = 1 at
//        k = 0, 64, else 2: the mirror half folded in), as one N = 256 GEMM
//        [Ur | Ui] = Fr [aSr | aSi] + Fi [aSi | -aSr] over k = 0 .. 79
//   I2  x[r][c] = Re sum_kc exp(+2 pi i c kc / 128) U[r][kc] / 128 = Ur Fr + Ui Fi
// Operands are K-major, no swizzle: a matrix of R rows and K columns is stored
// as K / 8 panels of R 16-byte rows (panel stride padded by 16 bytes), so a
// 16-wide k-step is two consecutive panels (LBO = panel stride, SBO = 128).
// Scaling keeps the FP16 values in range: each window is staged times 2^-e
// (its largest magnitude f 2^e, f in [0.5, 1); the output times 2^e, both
// exact), the spectra carry 1 / 128 and the staged U (H^T: Z) another 1 / 128
// (the inverse DFT's 1 / 128^2).
//
// Roles: 8 staging warps (two per tensor-memory lane quarter, one per half of
// a stage's columns) stage operands, take the products and write the output;
// warp 8 issues the MMAs; warps 9 .. 11 claim work items, load the window
// (FP32 -> FP16, transposed) and the interpolation tables, and prefetch the
// next item's rows into L2.  A stage's operand is released to the MMA warp in
// two halves (one async-proxy fence each, one mbarrier per 16-wide K chunk),
// so the MMAs of the first half run while the second is staged.  The grid is
// persistent (one CTA per SM, items from an atomic counter, heaviest first).
// Every wait is bounded; the staging warps take every branch after a wait
// together, and so do the loader warps.
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
constexpr int NWK = 8;                      // staging warps
constexpr int NTW = 32 * NWK;
constexpr int NLW = 3;                      // loader warps
constexpr int WMMA = NWK, WLOAD = NWK + 1;  // MMA warp, first loader warp
constexpr int NT = 32 * (NWK + 1 + NLW);    // 12 warps, at most 3 per SM sub-partition
// half spectra: per PSF [9 groups of 8 k][2][kc][4] FP16 pairs, k = 8 g + 4 u + t
// (k = 0 .. 64 used), so that a warp's 16-byte loads of 4 k at its 32 kc are contiguous
constexpr int SPSF = 9 * 2 * S * 4;
constexpr int CPAN = 2 * S * 16 + 16;       // [Fr; Fi] (256 rows) panel stride
constexpr int CBYTES = (S / 8) * CPAN;
constexpr int XPAN = S * 16 + 16;           // 128-row operand panel stride
constexpr int XBYTES = (S / 8) * XPAN;
constexpr int IPAN = 3 * S * 16 + 16;       // I1 operand [aSr; aSi; -aSr] (384 rows)
constexpr int IPANELS = 10;                 // k = 0 .. 79 (zero beyond 64)
constexpr int kHdrD = 1024;
constexpr int OFF_C = kHdrD;                // [Fr; Fi]
constexpr int OFF_A1 = OFF_C + CBYTES;      // A1
constexpr int OFF_WIN = OFF_A1 + XBYTES;    // the window, x^T (rows c, K = r)
constexpr int OFF_X = OFF_WIN + XBYTES;     // (wr_a x)^T;  I1 operand, Ur, output tile
constexpr int OFF_Y = OFF_X + XBYTES;       // wc_b Y';     (I1 operand), Ui, (output tile)
constexpr int OFF_TAB = OFF_Y + XBYTES;     // [2 slots][rows | cols] interpolation tables
constexpr int OFF_WV = OFF_TAB + 2 * 2 * S * (int)sizeof(WTab);   // [2][wr] [2][wc]
constexpr int SMEM_D = OFF_WV + 4 * S * 4;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t TM_F1 = 0, TM_P = 128, TM_Q = 256, TM_SUM = 384;   // D columns
constexpr uint32_t TM_I1 = 128, TM_I2 = 384;
constexpr uint32_t TMT_I2 = 0, TMT_G = 384;   // H^T: I2 (summed over row weights), H^T r
static_assert(SMEM_D <= 227 * 1024, "shared memory");
static_assert(IPANELS * IPAN <= 2 * XBYTES, "I1 operand fits in the X and Y buffers");
static_assert(S * (S + 1) * 4 <= 2 * XBYTES, "output tile fits in the X and Y buffers");
static_assert(64 * 129 * 4 <= 2 * XBYTES, "H^T output band fits in the X and Y buffers");
static_assert(OFF_Y == OFF_X + XBYTES, "X and Y buffers are contiguous");
static_assert(CPAN % 16 == 0 && XPAN % 16 == 0 && IPAN % 16 == 0 && OFF_WV % 16 == 0, "alignment");

struct BarsD {
  uint64_t win_full, win_empty;           // loader <-> staging warps
  uint64_t f1_done, f2_done, i1_done, i2_done, fin;   // MMA completions
  uint64_t p_done;                        // product read P, Q (staging -> MMA)
  uint64_t xch[8], ych[8], sch[5], uch[8];  // operand chunks (staging -> MMA)
  uint32_t tmem;
  int abort;
  int mbox[2];                            // na, nb of the next block for the MMA warp (na < 0: stop)
  int item[2];                            // work item of a slot (-1: stop)
  int next_item;                          // the loaders' next claimed item
  uint32_t lmax[NLW];                     // the loader warps' largest |window value| (bits)
  float wscale[2];                        // 2^e: the output factor of a slot's window
  float sscale[2];                        // 2^-e or 1: the staging factor (1 if stored scaled)
};
static_assert(sizeof(BarsD) <= kHdrD, "barrier header");

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack_h2(uint32_t v) {
  return __half22float2(*reinterpret_cast<const __half2*>(&v));
}
// k-step i (16 wide) of a chain: D (+)= A B^T, A rows from a0, B rows from b0
__device__ __forceinline__ void kstep(uint32_t d, uint32_t a0, uint32_t apan, uint32_t b0,
                                      uint32_t bpan, uint32_t id, int i, bool acc) {
  mma_bf16(d, sdesc(a0 + 2 * i * apan, apan), sdesc(b0 + 2 * i * bpan, bpan), id, acc ? 1u : 0u);
}

// barrier 2 over the loader warps, as an AND-vote
__device__ __forceinline__ bool loader_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 2, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(32 * NLW)
      : "memory");
  return r != 0;
}

template <bool ADJ>
__global__ void __launch_bounds__(NT, 1) dft_kernel(const OpArgs A) {
  extern __shared__ __align__(1024) unsigned char smem[];
  BarsD* H = reinterpret_cast<BarsD*>(smem);
  unsigned char* sC = smem + OFF_C;
  unsigned char* sWin = smem + OFF_WIN;
  unsigned char* sX = smem + OFF_X;
  unsigned char* sY = smem + OFF_Y;
  WTab* sTab = reinterpret_cast<WTab*>(smem + OFF_TAB);
  float* sWr = reinterpret_cast<float*>(smem + OFF_WV);   // [2][S]
  float* sWc = sWr + 2 * S;                               // [2][S]
  __shared__ WorkItem wis[2];
  __shared__ TileDesc tds[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = A.K, b = S - K + 1;
  const uint64_t limit = A.wait_ns ? A.wait_ns : kWaitNs;
  if (tid == 0) {
    mbar_init(&H->win_full, NLW);
    mbar_init(&H->win_empty, NWK);
    mbar_init(&H->f1_done, 1);
    mbar_init(&H->f2_done, 1);
    mbar_init(&H->i1_done, 1);
    mbar_init(&H->i2_done, 1);
    mbar_init(&H->fin, 1);
    mbar_init(&H->p_done, NWK);
    for (int i = 0; i < 8; ++i) {
      mbar_init(&H->xch[i], NWK);
      mbar_init(&H->ych[i], NWK);
      mbar_init(&H->uch[i], NWK);
    }
    for (int i = 0; i < 5; ++i) mbar_init(&H->sch[i], NWK);
    H->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == WMMA) tmem_alloc(&H->tmem, TMEM_COLS);
  // constants [Fr; Fi] and A1 (the plan's byte image of the panels)
  for (int e = tid; e < (CBYTES + XBYTES) / 16; e += NT)
    reinterpret_cast<uint4*>(sC)[e] = __ldg(reinterpret_cast<const uint4*>(A.tcop) + e);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = H->tmem;
  bool ok = true;

  if (warp >= WLOAD) {
    // --------------------------------------------------------------- loaders
    // loader warp lw takes panels q = lw, lw + 3, .. of the window; warp 0
    // claims the items, warps 1 and 2 fetch the row / column tables.  The
    // window is H's x below the output block, or H^T's r from K - 1 rows and
    // columns above and left of it (zero outside the tile), in FP16 as loaded
    // while its largest magnitude m = f 2^e (f in [0.5, 1)) is found; the
    // staging warps multiply by 2^-e (exact) and the output by 2^e.  Outside
    // [2^-10, 2^15) a second pass stores the window times 2^-e instead.
    const int lw = warp - WLOAD;
    auto psfs = [](const WorkItem& w2) { return (w2.a_hi - w2.a_lo + 1) * (w2.b_hi - w2.b_lo + 1); };
    const int off = ADJ ? K - 1 : 0;
    int it = 0;
    if (lw == 0 && lane == 0) it = atomicAdd(A.counter, 1);
    for (uint32_t n = 0; !A.test_withhold; ++n) {
      const int slot = n & 1;
      bool w = n == 0 || wait_bar(&H->win_empty, (n - 1) & 1, &H->abort, A.err, limit);
      if (!(ok = loader_all(w && !*(volatile int*)&H->abort))) break;
      if (lw == 0 && lane == 0) {
        if (it < A.n_work) {
          const WorkItem w2 = A.work[it];
          wis[slot] = w2;
          tds[slot] = A.tiles[w2.tile];
          H->next_item = atomicAdd(A.counter, 1);
        }
        H->item[slot] = it < A.n_work ? it : -1;
      }
      loader_all(true);   // slot written
      if (H->item[slot] < 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&H->win_full);
        break;
      }
      const WorkItem& w2 = wis[slot];
      const TileDesc& t2 = tds[slot];
      if (psfs(w2) > 0) {
        if (lw > 0) {
          // interpolation table of the rows (lw = 1) or columns of the window
          // of H / the output block of H^T ({-2, 0, 0} outside the tile: no
          // grid index has a weight there)
          WTab* tab = sTab + slot * 2 * S + (lw - 1) * S;
          for (int e = lane; e < S; e += 32) {
            WTab v{-2, 0.f, 0.f, 0};
            if (lw == 1 && w2.r0 + e < t2.nxr) v = A.wrow[t2.wr0 + w2.r0 + e];
            if (lw == 2 && w2.c0 + e < t2.nxc) v = A.wcol[t2.wc0 + w2.c0 + e];
            tab[e] = v;
          }
        }
        // the window as (scaled) v^T in FP16: row c, 8 consecutive r per 16
        // bytes; two panels (64 loads) in flight a lane, 8-byte loads where
        // aligned
        const float* img = A.in + (ADJ ? t2.yoff : t2.xoff);
        const int64_t pitch = ADJ ? t2.ypitch : t2.xpitch;
        const int nrow = ADJ ? t2.nyr : t2.nxr, ncol = ADJ ? t2.nyc : t2.nxc;
        const int wr0 = w2.r0 - off, wc0 = w2.c0 - off;
        const bool al2 = ((reinterpret_cast<uintptr_t>(img + wc0) & 7) == 0) && (pitch % 2 == 0);
        float sc = 1.f;
        uint32_t mx = 0;   // bits of the largest magnitude (monotonic for |v|)
        int e = 0;
        for (int pass = 0; pass < 2; ++pass) {
          for (int q0 = lw; q0 < S / 8; q0 += 2 * NLW) {
            const bool two = q0 + NLW < S / 8;
            if (al2) {
              float2 v[2][2][8];
#pragma unroll
              for (int qq = 0; qq < 2; ++qq)
#pragma unroll
                for (int m = 0; m < 2; ++m)
#pragma unroll
                  for (int t = 0; t < 8; ++t) {
                    const int R = wr0 + 8 * (q0 + qq * NLW) + t, C = wc0 + 2 * lane + 64 * m;
                    const float* src = img + (int64_t)R * pitch + C;
                    float2 u = make_float2(0.f, 0.f);
                    if ((qq == 0 || two) && R >= 0 && R < nrow && C >= 0) {
                      if (C + 1 < ncol) u = __ldg(reinterpret_cast<const float2*>(src));
                      else if (C < ncol) u.x = __ldg(src);
                    }
                    v[qq][m][t] = u;
                  }
              if (pass == 0) {
#pragma unroll
                for (int qq = 0; qq < 2; ++qq)
#pragma unroll
                  for (int m = 0; m < 2; ++m)
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                      mx = max(mx, max(__float_as_uint(fabsf(v[qq][m][t].x)),
                                       __float_as_uint(fabsf(v[qq][m][t].y))));
              }
#pragma unroll
              for (int qq = 0; qq < 2; ++qq) {
                if (qq == 1 && !two) break;
                const int q = q0 + qq * NLW;
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                  const int c = 2 * lane + 64 * m;
                  const float2* f = v[qq][m];
                  *reinterpret_cast<uint4*>(sWin + q * XPAN + 16 * c) =
                      make_uint4(pack_h2(sc * f[0].x, sc * f[1].x), pack_h2(sc * f[2].x, sc * f[3].x),
                                 pack_h2(sc * f[4].x, sc * f[5].x), pack_h2(sc * f[6].x, sc * f[7].x));
                  *reinterpret_cast<uint4*>(sWin + q * XPAN + 16 * (c + 1)) =
                      make_uint4(pack_h2(sc * f[0].y, sc * f[1].y), pack_h2(sc * f[2].y, sc * f[3].y),
                                 pack_h2(sc * f[4].y, sc * f[5].y), pack_h2(sc * f[6].y, sc * f[7].y));
                }
              }
            } else {
              float v[2][4][8];
#pragma unroll
              for (int qq = 0; qq < 2; ++qq)
#pragma unroll
                for (int m = 0; m < 4; ++m)
#pragma unroll
                  for (int t = 0; t < 8; ++t) {
                    const int R = wr0 + 8 * (q0 + qq * NLW) + t, C = wc0 + lane + 32 * m;
                    v[qq][m][t] = ((qq == 0 || two) && R >= 0 && R < nrow && C >= 0 && C < ncol)
                                      ? __ldg(img + (int64_t)R * pitch + C)
                                      : 0.f;
                  }
              if (pass == 0) {
#pragma unroll
                for (int qq = 0; qq < 2; ++qq)
#pragma unroll
                  for (int m = 0; m < 4; ++m)
#pragma unroll
                    for (int t = 0; t < 8; ++t) mx = max(mx, __float_as_uint(fabsf(v[qq][m][t])));
              }
#pragma unroll
              for (int qq = 0; qq < 2; ++qq) {
                if (qq == 1 && !two) break;
                const int q = q0 + qq * NLW;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                  const float* f = v[qq][m];
                  *reinterpret_cast<uint4*>(sWin + q * XPAN + 16 * (lane + 32 * m)) =
                      make_uint4(pack_h2(sc * f[0], sc * f[1]), pack_h2(sc * f[2], sc * f[3]),
                                 pack_h2(sc * f[4], sc * f[5]), pack_h2(sc * f[6], sc * f[7]));
                }
              }
            }
          }
          if (pass == 0) {
            // the window's largest magnitude over the three loader warps
            mx = __reduce_max_sync(0xffffffffu, mx);
            if (lane == 0) H->lmax[lw] = mx;
            loader_all(true);
            mx = max(H->lmax[0], max(H->lmax[1], H->lmax[2]));
            if (mx > 0 && mx < 0x7f800000u) frexpf(__uint_as_float(mx), &e);
            const bool again = e < -9 || e > 15;
            if (lw == 0 && lane == 0) {
              H->wscale[slot] = ldexpf(1.f, e);
              H->sscale[slot] = again ? 1.f : ldexpf(1.f, -e);
            }
            if (!again) break;
            sc = ldexpf(1.f, -e);
          }
        }
      }
      fence_async_smem();   // the window is an MMA operand (H^T) / staged from (H)
      __syncwarp();
      if (lane == 0) mbar_arrive(&H->win_full);
      // the next item's window and output-block rows into L2 while this block runs
      const int it2 = H->next_item;
      if (lw == 0) it = it2;
      if (it2 < A.n_work) {
        const WorkItem w3 = A.work[it2];
        const TileDesc t3 = A.tiles[w3.tile];
        const float* img = A.in + (ADJ ? t3.yoff : t3.xoff);
        const int64_t pitch = ADJ ? t3.ypitch : t3.xpitch;
        const int nrow = ADJ ? t3.nyr : t3.nxr, ncol = ADJ ? t3.nyc : t3.nxc;
        const int wr0 = w3.r0 - off, wc0 = max(w3.c0 - off, 0);
        if (psfs(w3) > 0) {
          const int c_end = min(w3.c0 - off + S, ncol);
          for (int rr = 32 * lw + lane; rr < S; rr += 32 * NLW) {
            const int R = wr0 + rr;
            if (R < 0 || R >= nrow || wc0 >= c_end) continue;
            const float* row = img + (int64_t)R * pitch;
            for (int C = wc0; C < c_end; C += 32) prefetch_l2(row + C);
            prefetch_l2(row + c_end - 1);
          }
        }
        if (!ADJ && A.mode != OP_PLAIN) {
          const int j_end = min(w3.c0 + b, t3.nyc);
          for (int rr = 32 * lw + lane; rr < b; rr += 32 * NLW) {
            const int i = w3.r0 + rr;
            if (i >= t3.nyr || w3.c0 >= j_end) continue;
            const int64_t g0 = (int64_t)(t3.xr0 + i) * A.wy + t3.xc0;
            for (int j = w3.c0; j < j_end; j += 32) prefetch_l2(A.y + g0 + j);
            prefetch_l2(A.y + g0 + j_end - 1);
            if (A.W) {
              for (int j = w3.c0; j < j_end; j += 32) prefetch_l2(A.W + g0 + j);
              prefetch_l2(A.W + g0 + j_end - 1);
            }
          }
        }
        if (ADJ && A.mode != OP_PLAIN) {
          // the iterate's rows r0 - 1 .. r0 + b and the dual's rows r0 .. r0 + b - 1
          const int c0 = max(w3.c0 - 1, 0), j_end = min(w3.c0 + b + 1, t3.nxc);
          for (int rr = 32 * lw + lane; rr < b + 2; rr += 32 * NLW) {
            const int R = w3.r0 - 1 + rr;
            if (R < 0 || R >= t3.nxr || c0 >= j_end) continue;
            const int64_t g0 = t3.xoff + (int64_t)R * t3.xpitch;
            for (int j = c0; j < j_end; j += 32) {
              prefetch_l2(A.w + g0 + j);
              prefetch_l2(A.u + g0 + j);
            }
            prefetch_l2(A.w + g0 + j_end - 1);
            prefetch_l2(A.u + g0 + j_end - 1);
          }
        }
      }
    }
  } else if (warp == WMMA) {
    // ------------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t aC = saddr(sC), aA1 = saddr(smem + OFF_A1), aX = saddr(sX), aY = saddr(sY);
      const uint32_t id256 = idesc(0, 128, 256), id128 = idesc(0, 128, 128);
      uint32_t ph_x = 0, ph_y = 0, ph_p = 0, ph_b = 0;
      auto wt = [&](uint64_t* bar, uint32_t ph) {
        if (!wait_bar(bar, ph & 1, &H->abort, A.err, limit)) return false;
        tc_fence_after();
        return true;
      };
      if constexpr (ADJ) {
        const uint32_t aWin = saddr(sWin);
        uint32_t ph_s = 0, ph_u = 0;
        while (ok) {
          if (!(ok = wt(&H->xch[0], ph_x))) break;
          const int na = H->mbox[0], nb = H->mbox[1];
          if (na < 0) break;
          // F1 on the window as loaded, F2 into P, Q
          for (int i = 0; i < 8 && ok; ++i) {
            if (i > 0 && !(ok = wt(&H->xch[i], ph_x))) break;
            kstep(tbase + TM_F1, aA1, XPAN, aWin, XPAN, id128, i, i > 0);
          }
          ++ph_x;
          if (!ok) break;
          tc_commit(&H->f1_done);
          for (int i = 0; i < 8 && ok; ++i) {
            if (!(ok = wt(&H->ych[i], ph_y))) break;
            kstep(tbase + TM_P, aC, CPAN, aY, XPAN, id128, i, i > 0);
            kstep(tbase + TM_Q, aC + 16 * S, CPAN, aY, XPAN, id128, i, i > 0);
          }
          ++ph_y;
          if (!ok) break;
          tc_commit(&H->f2_done);
          // per PSF (column weight outer): I1, then I2 summed over the row weights
          for (int bi = 0; bi < nb && ok; ++bi)
            for (int ai = 0; ai < na && ok; ++ai) {
              for (int i = 0; i < 5 && ok; ++i) {
                if (!(ok = wt(&H->sch[i], ph_s))) break;
                kstep(tbase + TM_I1, aC, CPAN, aX, IPAN, id256, i, i > 0);
                kstep(tbase + TM_I1, aC + 16 * S, CPAN, aX + 16 * S, IPAN, id256, i, true);
              }
              ++ph_s;
              if (!ok) break;
              tc_commit(&H->i1_done);
              for (int i = 0; i < 8 && ok; ++i) {
                if (!(ok = wt(&H->uch[i], ph_u))) break;
                kstep(tbase + TMT_I2, aX, XPAN, aC, CPAN, id128, i, ai > 0 || i > 0);
                kstep(tbase + TMT_I2, aY, XPAN, aC + 16 * S, CPAN, id128, i, true);
              }
              ++ph_u;
              if (ok) tc_commit(&H->i2_done);
            }
        }
      } else {
      while (ok) {
        if (!(ok = wt(&H->xch[0], ph_x))) break;
        const int na = H->mbox[0], nb = H->mbox[1];
        if (na < 0) break;
        for (int ai = 0; ai < na && ok; ++ai) {
          // F1: Y' = A1 (wr_a x)
          for (int i = 0; i < 8 && ok; ++i) {
            if ((ai > 0 || i > 0) && !(ok = wt(&H->xch[i], ph_x))) break;
            kstep(tbase + TM_F1, aA1, XPAN, aX, XPAN, id128, i, i > 0);
          }
          ++ph_x;
          if (!ok) break;
          tc_commit(&H->f1_done);
          for (int bi = 0; bi < nb && ok; ++bi) {
            // F2 once the previous product has read P and Q
            if ((ai > 0 || bi > 0) && !(ok = wt(&H->p_done, ph_p++))) break;
            for (int i = 0; i < 8 && ok; ++i) {
              if (!(ok = wt(&H->ych[i], ph_y))) break;
              kstep(tbase + TM_P, aC, CPAN, aY, XPAN, id128, i, i > 0);
              kstep(tbase + TM_Q, aC + 16 * S, CPAN, aY, XPAN, id128, i, i > 0);
            }
            ++ph_y;
            if (ok) tc_commit(&H->f2_done);
          }
        }
        if (!ok || !(ok = wt(&H->p_done, ph_p++))) break;
        // I1: [Ur | Ui] = Fr [aSr | aSi] + Fi [aSi | -aSr]
        for (int i = 0; i < 5 && ok; ++i) {
          if (!(ok = wt(&H->sch[i], ph_b))) break;
          kstep(tbase + TM_I1, aC, CPAN, aX, IPAN, id256, i, i > 0);
          kstep(tbase + TM_I1, aC + 16 * S, CPAN, aX + 16 * S, IPAN, id256, i, true);
        }
        if (!ok) break;
        tc_commit(&H->i1_done);
        // I2: x = Ur Fr + Ui Fi
        for (int i = 0; i < 8 && ok; ++i) {
          if (!(ok = wt(&H->uch[i], ph_b))) break;
          kstep(tbase + TM_I2, aX, XPAN, aC, CPAN, id128, i, i > 0);
          kstep(tbase + TM_I2, aY, XPAN, aC + 16 * S, CPAN, id128, i, true);
        }
        if (!ok) break;
        tc_commit(&H->i2_done);
        ++ph_b;
      }
      }
    }
  } else {
    // --------------------------------------------------------- staging warps
    const int q4 = warp & 3, h = warp >> 2;
    const int L = 32 * q4 + lane;            // tensor-memory lane of this thread
    const uint32_t lanes = (uint32_t)(32 * q4) << 16;
    const unsigned int* spec = reinterpret_cast<const unsigned int*>(A.spec);
    uint32_t nblk = 0, ph_f1 = 0, ph_f2 = 0, ph_i = 0, nwr = 0, nwc = 0;
    auto arrive = [&](uint64_t* bar) {
      __syncwarp();
      if (lane == 0) mbar_arrive(bar);
    };
    auto wait_all = [&](uint64_t* bar, uint32_t ph) {
      const bool w = wait_bar(bar, ph & 1, &H->abort, A.err, limit);
      ok = named_all<NTW>(w && !*(volatile int*)&H->abort);
      tc_fence_after();
      return ok;
    };
    // the output block from an FP32 tile (pitch b + 1) or zero (tile null):
    // H x, or W (H x - y); warp w writes rows w, w + 8, .., lanes columns,
    // the observed image and weights of RB rows loaded before they are used
    auto write_out = [&](const WorkItem& wi, const TileDesc& td, const float* tile) {
      const int nr = min(b, td.nyr - wi.r0), nc = min(b, td.nyc - wi.c0);
      float* const out = A.out + td.yoff + (int64_t)wi.r0 * td.ypitch + wi.c0;
      const int64_t ypitch = td.ypitch;
      const bool resid = A.mode != OP_PLAIN;
      const float* const yb = A.y + (int64_t)(td.xr0 + wi.r0) * A.wy + td.xc0 + wi.c0;
      const float* const wb = A.W ? A.W + (yb - A.y) : nullptr;
      const int64_t wy = A.wy;
      constexpr int RB = 4, CB = S / 32;
      for (int il0 = warp; il0 < nr; il0 += RB * NWK) {
        float yo[RB][CB], wo[RB][CB];
        if (resid) {
#pragma unroll
          for (int u = 0; u < RB; ++u)
#pragma unroll
            for (int v = 0; v < CB; ++v) {
              const int il = il0 + u * NWK, jl = lane + 32 * v;
              yo[u][v] = 0.f;
              wo[u][v] = 1.f;
              if (il < nr && jl < nc) {
                yo[u][v] = __ldg(yb + il * wy + jl);
                if (wb) wo[u][v] = __ldg(wb + il * wy + jl);
              }
            }
        }
#pragma unroll
        for (int u = 0; u < RB; ++u)
#pragma unroll
          for (int v = 0; v < CB; ++v) {
            const int il = il0 + u * NWK, jl = lane + 32 * v;
            if (il >= nr || jl >= nc) continue;
            const float x = tile ? tile[il * (b + 1) + jl] : 0.f;
            out[il * ypitch + jl] = resid ? wo[u][v] * (x - yo[u][v]) : x;
          }
      }
    };

    if constexpr (ADJ) {
      uint32_t ph_i1 = 0, ph_i2 = 0;
      while (ok) {
        if (!wait_all(&H->win_full, nblk)) break;
        const int slot = nblk & 1;
        ++nblk;
        if (H->item[slot] < 0) {
          // stop: tell the MMA warp
          if (tid == 0) H->mbox[0] = -1;
          arrive(&H->xch[0]);
          break;
        }
        const WorkItem& wi = wis[slot];
        const TileDesc& td = tds[slot];
        const int na = wi.a_hi - wi.a_lo + 1, nb = wi.b_hi - wi.b_lo + 1;
        const WTab* tr = sTab + slot * 2 * S;
        const WTab* tc = tr + S;
        const bool any = na * nb > 0;
        if (any) {
          if (tid == 0) {
            H->mbox[0] = na;
            H->mbox[1] = nb;
          }
          // the window, as the loaders staged it, is F1's operand; F1's
          // result is scaled by the staging factor when Y' is staged
          const float sst = H->sscale[slot];
#pragma unroll
          for (int i = 0; i < 8; ++i) arrive(&H->xch[i]);
          if (!wait_all(&H->f1_done, ph_f1++)) break;
          arrive(&H->win_empty);
          // Y' into sY (rows j, K = c), released in two halves
#pragma unroll
          for (int i0 = 0; i0 < 8; i0 += 4) {
            uint32_t v[4][8];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) tmem_ld8_nowait(tbase + lanes + TM_F1 + 16 * (i0 + ii) + 8 * h, v[ii]);
            tmem_wait_ld();
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) {
              const float* f = reinterpret_cast<const float*>(v[ii]);
              *reinterpret_cast<uint4*>(sY + (2 * (i0 + ii) + h) * XPAN + 16 * L) =
                  make_uint4(pack_h2(sst * f[0], sst * f[1]), pack_h2(sst * f[2], sst * f[3]),
                             pack_h2(sst * f[4], sst * f[5]), pack_h2(sst * f[6], sst * f[7]));
            }
            fence_async_smem();
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) arrive(&H->ych[i0 + ii]);
          }
          tc_fence_before();
          if (!wait_all(&H->f2_done, ph_f2++)) break;
          // Z(k)[kc = L] / 128 from P and Q, kept as FP16 pairs: k = 16 i + 8 h + t
          // at index 8 i + t, and k = 64 (h == 0)
          uint32_t zh[32], z64 = 0;
#pragma unroll
          for (int i0 = 0; i0 < 4; i0 += 2) {
            uint32_t pv[2][16], qv[2][16];
#pragma unroll
            for (int ii = 0; ii < 2; ++ii) {
              tmem_ld16_nowait(tbase + lanes + TM_P + 32 * (i0 + ii) + 16 * h, pv[ii]);
              tmem_ld16_nowait(tbase + lanes + TM_Q + 32 * (i0 + ii) + 16 * h, qv[ii]);
            }
            tmem_wait_ld();
            const float is = 1.f / S;
            if (i0 == 0) z64 = pack_h2(is * __uint_as_float(pv[0][1]), is * __uint_as_float(qv[0][1]));
#pragma unroll
            for (int ii = 0; ii < 2; ++ii)
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                const float pr = __uint_as_float(pv[ii][2 * t]), pi = __uint_as_float(pv[ii][2 * t + 1]);
                const float qr = __uint_as_float(qv[ii][2 * t]), qi = __uint_as_float(qv[ii][2 * t + 1]);
                const bool k0 = i0 + ii == 0 && t == 0 && h == 0;   // Y(0) real; column 1 holds Y(64)
                zh[8 * (i0 + ii) + t] = pack_h2(is * (k0 ? pr : pr - qi), is * (k0 ? qr : qr + pi));
              }
          }
          tc_fence_before();   // P and Q have been read: I1 may overwrite them
          for (int bi = 0; bi < nb && ok; ++bi) {
            const int gb = wi.b_lo + bi;
            float* wc = sWc + (nwc++ & 1) * S;
            if (tid >= S) wc[tid - S] = wsel(tc[tid - S], gb);
            for (int ai = 0; ai < na && ok; ++ai) {
              const int ga = wi.a_lo + ai;
              float* wr = sWr + (nwr++ & 1) * S;
              if (tid < S) wr[tid] = wsel(tr[tid], ga);
              named_sync<NTW>();
              const unsigned int* hs = spec + (size_t)(ga * A.Gc + gb) * SPSF + 4 * L;
              uint32_t hv[33];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const int g = 2 * i + h;
                const uint4 u0 = __ldg(reinterpret_cast<const uint4*>(hs + (2 * g) * S * 4));
                const uint4 u1 = __ldg(reinterpret_cast<const uint4*>(hs + (2 * g + 1) * S * 4));
                hv[8 * i + 0] = u0.x; hv[8 * i + 1] = u0.y; hv[8 * i + 2] = u0.z; hv[8 * i + 3] = u0.w;
                hv[8 * i + 4] = u1.x; hv[8 * i + 5] = u1.y; hv[8 * i + 6] = u1.z; hv[8 * i + 7] = u1.w;
              }
              hv[32] = h == 0 ? __ldg(hs + 16 * S * 4) : 0u;
              // T = alpha Z conj(Hh) (correlation) into the I1 operand rows kc:
              // [aTr; aTi; -aTr], 5 chunks of 16 k (panel 2 i + h), two releases
#pragma unroll
              for (int i = 0; i < 5; ++i) {
                if (i == 2) {
                  fence_async_smem();
                  arrive(&H->sch[0]);
                  arrive(&H->sch[1]);
                }
                float ar[8], ai_[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                  float2 z, hf;
                  float al;
                  if (i < 4) {
                    z = unpack_h2(zh[8 * i + t]);
                    hf = unpack_h2(hv[8 * i + t]);
                    al = (i == 0 && t == 0 && h == 0) ? 1.f : 2.f;
                  } else {
                    const bool k64 = t == 0 && h == 0;
                    z = k64 ? unpack_h2(z64) : make_float2(0.f, 0.f);
                    hf = k64 ? unpack_h2(hv[32]) : make_float2(0.f, 0.f);
                    al = 1.f;
                  }
                  ar[t] = al * fmaf(z.x, hf.x, z.y * hf.y);
                  ai_[t] = al * fmaf(z.y, hf.x, -z.x * hf.y);
                }
                unsigned char* dst = sX + (2 * i + h) * IPAN + 16 * L;
                *reinterpret_cast<uint4*>(dst) =
                    make_uint4(pack_h2(ar[0], ar[1]), pack_h2(ar[2], ar[3]), pack_h2(ar[4], ar[5]),
                               pack_h2(ar[6], ar[7]));
                *reinterpret_cast<uint4*>(dst + 16 * S) =
                    make_uint4(pack_h2(ai_[0], ai_[1]), pack_h2(ai_[2], ai_[3]), pack_h2(ai_[4], ai_[5]),
                               pack_h2(ai_[6], ai_[7]));
                *reinterpret_cast<uint4*>(dst + 32 * S) =
                    make_uint4(pack_h2(-ar[0], -ar[1]), pack_h2(-ar[2], -ar[3]), pack_h2(-ar[4], -ar[5]),
                               pack_h2(-ar[6], -ar[7]));
              }
              fence_async_smem();
#pragma unroll
              for (int i = 2; i < 5; ++i) arrive(&H->sch[i]);
              if (!wait_all(&H->i1_done, ph_i1++)) break;
              // U (lane r) times wr_a(r) into the I2 operands Ur (sX) and Ui (sY)
              const float wrr = wr[L];
#pragma unroll
              for (int i0 = 0; i0 < 8; i0 += 4) {
                uint32_t ur[4][8], ui[4][8];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  tmem_ld8_nowait(tbase + lanes + TM_I1 + 16 * (i0 + i) + 8 * h, ur[i]);
                  tmem_ld8_nowait(tbase + lanes + TM_I1 + S + 16 * (i0 + i) + 8 * h, ui[i]);
                }
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  const float* fr = reinterpret_cast<const float*>(ur[i]);
                  const float* fi = reinterpret_cast<const float*>(ui[i]);
                  const int o = (2 * (i0 + i) + h) * XPAN + 16 * L;
                  *reinterpret_cast<uint4*>(sX + o) =
                      make_uint4(pack_h2(wrr * fr[0], wrr * fr[1]), pack_h2(wrr * fr[2], wrr * fr[3]),
                                 pack_h2(wrr * fr[4], wrr * fr[5]), pack_h2(wrr * fr[6], wrr * fr[7]));
                  *reinterpret_cast<uint4*>(sY + o) =
                      make_uint4(pack_h2(wrr * fi[0], wrr * fi[1]), pack_h2(wrr * fi[2], wrr * fi[3]),
                                 pack_h2(wrr * fi[4], wrr * fi[5]), pack_h2(wrr * fi[6], wrr * fi[7]));
                }
                fence_async_smem();
#pragma unroll
                for (int i = 0; i < 4; ++i) arrive(&H->uch[i0 + i]);
              }
              tc_fence_before();
              if (!wait_all(&H->i2_done, ph_i2++)) break;
              if (ai == na - 1) {
                // H^T r (+)= wc_b . sum_a (I2), columns c = 64 h + 16 i + t
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  uint32_t d[16], g[16];
                  tmem_ld16_nowait(tbase + lanes + TMT_I2 + 64 * h + 16 * i, d);
                  if (bi > 0) tmem_ld16_nowait(tbase + lanes + TMT_G + 64 * h + 16 * i, g);
                  tmem_wait_ld();
#pragma unroll
                  for (int t = 0; t < 16; ++t) {
                    const float v = wc[64 * h + 16 * i + t] * __uint_as_float(d[t]);
                    d[t] = __float_as_uint(bi > 0 ? __uint_as_float(g[t]) + v : v);
                  }
                  tmem_st16_nowait(tbase + lanes + TMT_G + 64 * h + 16 * i, d);
                }
                tmem_wait_st();
                tc_fence_before();
              }
            }
          }
          if (!ok) break;
        } else {
          arrive(&H->win_empty);
        }
        // H^T r (times the window's scale; zero without PSFs) from tensor
        // memory into an FP32 band of 64 output rows, then into the output
        // (warp w rows w, w + 8, .., lanes columns); the projected-gradient
        // step runs afterwards (dft_step_kernel)
        const float scale = any ? H->wscale[slot] : 0.f;
        constexpr int BH = 64, CB = S / 32;
        const int TP = b + 1;
        float* band = reinterpret_cast<float*>(sX);
        const int nr = min(b, td.nxr - wi.r0), nc = min(b, td.nxc - wi.c0);
        float* const out = A.out + td.xoff + (int64_t)wi.r0 * td.xpitch + wi.c0;
        const int64_t xpitch = td.xpitch;
        for (int i0 = 0; i0 < nr; i0 += BH) {
          if (any && (32 * q4 == i0 || 32 * q4 == i0 + 32)) {
            uint32_t v[4][16];
#pragma unroll
            for (int i = 0; i < 4; ++i) tmem_ld16_nowait(tbase + lanes + TMT_G + 64 * h + 16 * i, v[i]);
            tmem_wait_ld();
            const int rb = L - i0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int t = 0; t < 16; ++t) {
                const int c = 64 * h + 16 * i + t;
                if (c < b) band[rb * TP + c] = scale * __uint_as_float(v[i][t]);
              }
          } else if (!any) {
            for (int e = tid; e < BH * TP; e += NTW) band[e] = 0.f;
          }
          tc_fence_before();
          named_sync<NTW>();
          const int iend = min(i0 + BH, nr);
          for (int il = i0 + warp; il < iend; il += NWK)
#pragma unroll
            for (int v = 0; v < CB; ++v) {
              const int jl = lane + 32 * v;
              if (jl < nc) out[il * xpitch + jl] = band[(il - i0) * TP + jl];
            }
          named_sync<NTW>();   // the band is read before the next one is written
        }
      }
    } else {
    while (ok) {
      if (!wait_all(&H->win_full, nblk)) break;
      const int slot = nblk & 1;
      ++nblk;
      if (H->item[slot] < 0) {
        // stop: tell the MMA warp
        if (tid == 0) H->mbox[0] = -1;
        arrive(&H->xch[0]);
        break;
      }
      // (the loader rewrites this slot for the block after next, once this
      // block has finished)
      const WorkItem& wi = wis[slot];
      const TileDesc& td = tds[slot];
      const int na = wi.a_hi - wi.a_lo + 1, nb = wi.b_hi - wi.b_lo + 1;
      const WTab* tr = sTab + slot * 2 * S;
      const WTab* tc = tr + S;
      if (na * nb <= 0) {
        // no PSF reaches the block: H x is zero there
        arrive(&H->win_empty);
        write_out(wi, td, nullptr);
        continue;
      }
      if (tid == 0) {
        H->mbox[0] = na;
        H->mbox[1] = nb;
      }
      const float sst = H->sscale[slot];   // the window's staging factor
      // (wr_a x)^T into sX in 8 chunks of 16 r (panels 2i + half), a chunk
      // complete -> xch[i]
      auto stage_x = [&](int ga, bool last_use) {
        float* wr = sWr + (nwr++ & 1) * S;
        if (tid < S) wr[tid] = wsel(tr[tid], ga) * sst;
        named_sync<NTW>();
        const int c = tid & (S - 1), half = tid >> 7;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (i == 4) {   // first half complete: its k-steps can start
            fence_async_smem();
#pragma unroll
            for (int j = 0; j < 4; ++j) arrive(&H->xch[j]);
          }
          const int pan = 2 * i + half;
          const uint4 xv = *reinterpret_cast<const uint4*>(sWin + pan * XPAN + 16 * c);
          const float4 w0 = *reinterpret_cast<const float4*>(wr + 8 * pan);
          const float4 w1 = *reinterpret_cast<const float4*>(wr + 8 * pan + 4);
          const float2 x0 = unpack_h2(xv.x), x1 = unpack_h2(xv.y), x2 = unpack_h2(xv.z),
                       x3 = unpack_h2(xv.w);
          *reinterpret_cast<uint4*>(sX + pan * XPAN + 16 * c) =
              make_uint4(pack_h2(w0.x * x0.x, w0.y * x0.y), pack_h2(w0.z * x1.x, w0.w * x1.y),
                         pack_h2(w1.x * x2.x, w1.y * x2.y), pack_h2(w1.z * x3.x, w1.w * x3.y));
        }
        fence_async_smem();
#pragma unroll
        for (int i = 4; i < 8; ++i) arrive(&H->xch[i]);
        if (last_use) arrive(&H->win_empty);
      };
      stage_x(wi.a_lo, na == 1);
      float s64r = 0.f, s64i = 0.f;          // S(64) at this lane's kc (h == 0)
      for (int ai = 0; ai < na && ok; ++ai) {
        if (!wait_all(&H->f1_done, ph_f1++)) break;
        for (int bi = 0; bi < nb && ok; ++bi) {
          const bool first = ai == 0 && bi == 0;
          const int gb = wi.b_lo + bi;
          // wc_b Y' into sY: lane j, columns c = 16 i + 8 h + (0 .. 7) -> panel 2 i + h
          {
            float* wc = sWc + (nwc++ & 1) * S;
            if (tid >= S) wc[tid - S] = wsel(tc[tid - S], gb);
            named_sync<NTW>();
            uint32_t v[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i) tmem_ld8_nowait(tbase + lanes + TM_F1 + 16 * i + 8 * h, v[i]);
            tmem_wait_ld();
            tc_fence_before();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              if (i == 4) {
                fence_async_smem();
#pragma unroll
                for (int j = 0; j < 4; ++j) arrive(&H->ych[j]);
              }
              const int c0 = 16 * i + 8 * h;
              const float4 w0 = *reinterpret_cast<const float4*>(wc + c0);
              const float4 w1 = *reinterpret_cast<const float4*>(wc + c0 + 4);
              const float* f = reinterpret_cast<const float*>(v[i]);
              *reinterpret_cast<uint4*>(sY + (2 * i + h) * XPAN + 16 * L) =
                  make_uint4(pack_h2(w0.x * f[0], w0.y * f[1]), pack_h2(w0.z * f[2], w0.w * f[3]),
                             pack_h2(w1.x * f[4], w1.y * f[5]), pack_h2(w1.z * f[6], w1.w * f[7]));
            }
            fence_async_smem();
#pragma unroll
            for (int i = 4; i < 8; ++i) arrive(&H->ych[i]);
          }
          // the next row weight's X once F1 has been read for the last time
          if (bi == nb - 1 && ai + 1 < na) stage_x(wi.a_lo + ai + 1, ai + 2 == na);
          // this thread's spectrum values Hh_p(k, kc = L), k = 16 i + 8 h + t
          // (and k = 64 for h == 0), fetched while F2 runs
          const int ga = wi.a_lo + ai;
          const unsigned int* hs = spec + (size_t)(ga * A.Gc + gb) * SPSF + 4 * L;
          uint32_t hv[33];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int g = 2 * i + h;
            const uint4 u0 = __ldg(reinterpret_cast<const uint4*>(hs + (2 * g) * S * 4));
            const uint4 u1 = __ldg(reinterpret_cast<const uint4*>(hs + (2 * g + 1) * S * 4));
            hv[8 * i + 0] = u0.x; hv[8 * i + 1] = u0.y; hv[8 * i + 2] = u0.z; hv[8 * i + 3] = u0.w;
            hv[8 * i + 4] = u1.x; hv[8 * i + 5] = u1.y; hv[8 * i + 6] = u1.z; hv[8 * i + 7] = u1.w;
          }
          hv[32] = h == 0 ? __ldg(hs + 16 * S * 4) : 0u;
          if (!wait_all(&H->f2_done, ph_f2++)) break;
          // product: Z(k)[kc] from P, Q at columns 2k, 2k + 1, times Hh_p,
          // summed in tensor memory (columns 2k, 2k + 1 of the sum)
          float p1 = 0.f, q1 = 0.f;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint32_t col = 32 * i + 16 * h;
            uint32_t pv[16], qv[16], sv[16];
            tmem_ld16_nowait(tbase + lanes + TM_P + col, pv);
            tmem_ld16_nowait(tbase + lanes + TM_Q + col, qv);
            if (!first) tmem_ld16_nowait(tbase + lanes + TM_SUM + col, sv);
            tmem_wait_ld();
            if (i == 0) {
              p1 = __uint_as_float(pv[1]);
              q1 = __uint_as_float(qv[1]);
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const float pr = __uint_as_float(pv[2 * t]), pi = __uint_as_float(pv[2 * t + 1]);
              const float qr = __uint_as_float(qv[2 * t]), qi = __uint_as_float(qv[2 * t + 1]);
              // k = 0 (i, t, h = 0): Y(0) is real, column 1 holds Y(64)
              const bool k0 = i == 0 && t == 0 && h == 0;
              const float zr = k0 ? pr : pr - qi, zi = k0 ? qr : qr + pi;
              const float2 hf = unpack_h2(hv[8 * i + t]);
              float sr = first ? 0.f : __uint_as_float(sv[2 * t]);
              float si = first ? 0.f : __uint_as_float(sv[2 * t + 1]);
              sr = fmaf(zr, hf.x, fmaf(-zi, hf.y, sr));
              si = fmaf(zr, hf.y, fmaf(zi, hf.x, si));
              sv[2 * t] = __float_as_uint(sr);
              sv[2 * t + 1] = __float_as_uint(si);
            }
            tmem_st16_nowait(tbase + lanes + TM_SUM + col, sv);
          }
          if (h == 0) {
            // k = 64: Z = P[1] + i Q[1] (Y(64) is real)
            const float2 hf = unpack_h2(hv[32]);
            s64r = fmaf(p1, hf.x, fmaf(-q1, hf.y, first ? 0.f : s64r));
            s64i = fmaf(p1, hf.y, fmaf(q1, hf.x, first ? 0.f : s64i));
          }
          tmem_wait_st();
          tc_fence_before();
          arrive(&H->p_done);
        }
      }
      if (!ok) break;
      // I1 operand rows kc ([aSr; aSi; -aSr] at rows kc, S + kc, 2S + kc) in
      // 5 chunks of 16 k (panel 2 i + h, k = 16 i + 8 h + t), -> sch[i]
      {
        uint32_t sv[4][16];
#pragma unroll
        for (int i = 0; i < 4; ++i) tmem_ld16_nowait(tbase + lanes + TM_SUM + 32 * i + 16 * h, sv[i]);
        tmem_wait_ld();
        tc_fence_before();
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          float sr[8], si[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            if (i < 4) {
              const float al = (i == 0 && t == 0 && h == 0) ? 1.f : 2.f;
              sr[t] = al * __uint_as_float(sv[i][2 * t]);
              si[t] = al * __uint_as_float(sv[i][2 * t + 1]);
            } else {
              sr[t] = (t == 0 && h == 0) ? s64r : 0.f;
              si[t] = (t == 0 && h == 0) ? s64i : 0.f;
            }
          }
          unsigned char* dst = sX + (2 * i + h) * IPAN + 16 * L;
          *reinterpret_cast<uint4*>(dst) =
              make_uint4(pack_h2(sr[0], sr[1]), pack_h2(sr[2], sr[3]), pack_h2(sr[4], sr[5]),
                         pack_h2(sr[6], sr[7]));
          *reinterpret_cast<uint4*>(dst + 16 * S) =
              make_uint4(pack_h2(si[0], si[1]), pack_h2(si[2], si[3]), pack_h2(si[4], si[5]),
                         pack_h2(si[6], si[7]));
          *reinterpret_cast<uint4*>(dst + 32 * S) =
              make_uint4(pack_h2(-sr[0], -sr[1]), pack_h2(-sr[2], -sr[3]), pack_h2(-sr[4], -sr[5]),
                         pack_h2(-sr[6], -sr[7]));
        }
        fence_async_smem();
#pragma unroll
        for (int i = 0; i < 5; ++i) arrive(&H->sch[i]);
      }
      // U / 128 (lane r, columns kc = 16 i + 8 h + t) into the I2 operands Ur
      // (sX) and Ui (sY), panel 2 i + h, -> uch[i]
      if (!wait_all(&H->i1_done, ph_i)) break;
      for (int i0 = 0; i0 < 8; i0 += 4) {
        uint32_t ur[4][8], ui[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          tmem_ld8_nowait(tbase + lanes + TM_I1 + 16 * (i0 + i) + 8 * h, ur[i]);
          tmem_ld8_nowait(tbase + lanes + TM_I1 + S + 16 * (i0 + i) + 8 * h, ui[i]);
        }
        tmem_wait_ld();
        tc_fence_before();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float sc = 1.f / S;
          const float* fr = reinterpret_cast<const float*>(ur[i]);
          const float* fi = reinterpret_cast<const float*>(ui[i]);
          const int off = (2 * (i0 + i) + h) * XPAN + 16 * L;
          *reinterpret_cast<uint4*>(sX + off) =
              make_uint4(pack_h2(sc * fr[0], sc * fr[1]), pack_h2(sc * fr[2], sc * fr[3]),
                         pack_h2(sc * fr[4], sc * fr[5]), pack_h2(sc * fr[6], sc * fr[7]));
          *reinterpret_cast<uint4*>(sY + off) =
              make_uint4(pack_h2(sc * fi[0], sc * fi[1]), pack_h2(sc * fi[2], sc * fi[3]),
                         pack_h2(sc * fi[4], sc * fi[5]), pack_h2(sc * fi[6], sc * fi[7]));
        }
        fence_async_smem();
#pragma unroll
        for (int i = 0; i < 4; ++i) arrive(&H->uch[i0 + i]);
      }
      // x (lane r, columns c) -> the valid rows and columns K - 1 .. 127 of an
      // FP32 tile in the X and Y buffers, then the output block row by row
      if (!wait_all(&H->i2_done, ph_i++)) break;
      {
        float* tile = reinterpret_cast<float*>(sX);
        const int r = L - (K - 1);
        const float scale = H->wscale[slot];
        uint32_t v[4][16];
#pragma unroll
        for (int i = 0; i < 4; ++i) tmem_ld16_nowait(tbase + lanes + TM_I2 + 64 * h + 16 * i, v[i]);
        tmem_wait_ld();
        if (r >= 0) {
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const int cc = 64 * h + 16 * i + t - (K - 1);
              if (cc >= 0) tile[r * (b + 1) + cc] = scale * __uint_as_float(v[i][t]);
            }
        }
        tc_fence_before();
        named_sync<NTW>();
        write_out(wi, td, tile);
        named_sync<NTW>();   // the tile is read before the next block's X is staged
      }
    }
    }
  }

  if (!ok) *(volatile int*)&H->abort = 1;
  // teardown: every MMA this CTA issued has completed before tensor memory is freed
  if (warp == WMMA && lane == 0) {
    tc_commit(&H->fin);
    drain_bar(&H->fin, 0, A.err);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == WMMA) {
    tc_fence_after();
    tmem_free(tbase, TMEM_COLS);
  }
}

// The Local-Solver's projected-gradient step (the fused step of the other
// H^T kernels) after the block-DFT H^T has written g = H^T r into the output:
// w_next = max(0, w - tau (g + lambda D^T psi(D w) + alpha (w - u))), g read
// in place.  One CTA per H^T output block (b x b x-pixels, the same work
// items), the iterate's halo in shared memory; bound by HBM traffic.
__global__ void __launch_bounds__(256) dft_step_kernel(const OpArgs A) {
  extern __shared__ float sWs[];   // (b + 2)^2: iterate rows r0 - 1 .. r0 + b
  const WorkItem wi = A.work[blockIdx.x];
  const TileDesc td = A.tiles[wi.tile];
  const int b = S - A.K + 1, HW = b + 2;
  const int nr = min(b, td.nxr - wi.r0), nc = min(b, td.nxc - wi.c0);
  if (nr <= 0 || nc <= 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int hr = warp; hr < nr + 2; hr += 8)
    for (int hc = lane; hc < nc + 2; hc += 32) {
      const int R = wi.r0 - 1 + hr, C = wi.c0 - 1 + hc;
      sWs[hr * HW + hc] = (R >= 0 && R < td.nxr && C >= 0 && C < td.nxc)
                              ? __ldg(A.w + td.xoff + (int64_t)R * td.xpitch + C)
                              : 0.f;
    }
  __syncthreads();
  for (int il = warp; il < nr; il += 8) {
    const int R = wi.r0 + il;
    const float orr = A.gamma * A.omr[td.omr_off + R];
    for (int jl = lane; jl < nc; jl += 32) {
      const int C = wi.c0 + jl;
      const int64_t idx = td.xoff + (int64_t)R * td.xpitch + C;
      const int li = il + 1, lj = jl + 1;
      float pr, pc, pru, pcu, prl, pcl;
      huber_p(sWs, HW, li, lj, R, C, td.nxr, td.nxc, A.delta, pr, pc);
      huber_p(sWs, HW, li - 1, lj, R - 1, C, td.nxr, td.nxc, A.delta, pru, pcu);
      huber_p(sWs, HW, li, lj - 1, R, C - 1, td.nxr, td.nxc, A.delta, prl, pcl);
      const float hub = pru - pr + pcl - pc;
      const float wv = sWs[li * HW + lj];
      const float alpha = orr * A.omc[td.omc_off + C];
      const float grad = A.out[idx] + A.lambda * hub + alpha * (wv - A.u[idx]);
      A.out[idx] = fmaxf(0.f, wv - td.tau * grad);
    }
  }
}

}  // namespace

bool dft_supported(int K) { return K >= 1 && S - K + 1 >= 32; }

cudaError_t dft_prepare() {
  cudaError_t e = cudaFuncSetAttribute(dft_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_D);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(dft_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_D);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(dft_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (S + 2) * (S + 2) * (int)sizeof(float));
}

// Byte image of the constant operands, FP16 from FP64 on the host: [Fr; Fi]
// (16 panels of 256 16-byte rows, padded; row n < 128: cos(2 pi n k / 128),
// row 128 + n: -sin(2 pi n k / 128), k the column), then A1 (16 panels of 128
// rows; row 2m: cos(2 pi m k / 128), row 2m + 1: -sin(2 pi m k / 128) for
// m = 1 .. 63, row 1: cos(pi k) = Fr(64)).
void dft_constants(std::vector<uint8_t>& out) {
  out.assign(CBYTES + XBYTES, 0);
  auto put = [&](size_t off, double v) {
    const __half hv = __float2half_rn((float)v);
    std::memcpy(out.data() + off, &hv, 2);
  };
  auto ang = [](int n, int k) { return 2.0 * 3.14159265358979323846 * (double)((n * k) % S) / S; };
  for (int n = 0; n < 2 * S; ++n)
    for (int k = 0; k < S; ++k) {
      const int nn = n & (S - 1);
      put((size_t)(k >> 3) * CPAN + 16 * n + 2 * (k & 7), n < S ? std::cos(ang(nn, k)) : -std::sin(ang(nn, k)));
    }
  for (int j = 0; j < S; ++j)
    for (int k = 0; k < S; ++k) {
      const int m = j >> 1;
      const double v = j == 1 ? std::cos(ang(S / 2, k)) : (j & 1) ? -std::sin(ang(m, k)) : std::cos(ang(m, k));
      put(CBYTES + (size_t)(k >> 3) * XPAN + 16 * j + 2 * (k & 7), v);
    }
}

// Half spectra of the zero-padded PSFs, kr = 0 .. 64 in the layout of SPSF,
// scaled by 1 / 128:
// Hh(kr, kc) = sum_{m, n < K} h(m, n) exp(-2 pi i (kr m + kc n) / 128) / 128,
// summed in FP64 on the host and stored as FP16 (re, im) pairs.
void dft_spectra(const float* psfs, int G, int K, std::vector<uint32_t>& out) {
  std::vector<double> cr(S), ci(S);
  for (int j = 0; j < S; ++j) {
    const double a = -2.0 * 3.14159265358979323846 * j / S;
    cr[j] = std::cos(a);
    ci[j] = std::sin(a);
  }
  out.assign((size_t)G * SPSF, 0u);
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
    for (int kr = 0; kr <= S / 2; ++kr)
      for (int kc = 0; kc < S; ++kc) {
        double sr = 0.0, si = 0.0;
        for (int m = 0; m < K; ++m) {
          const int j = (kr * m) % S;
          const double ar = tr[(size_t)m * S + kc], ai = ti[(size_t)m * S + kc];
          sr += ar * cr[j] - ai * ci[j];
          si += ar * ci[j] + ai * cr[j];
        }
        const __half2 hv = __floats2half2_rn((float)(sr / S), (float)(si / S));
        const size_t e = (size_t)g * SPSF + ((size_t)(2 * (kr >> 3) + ((kr >> 2) & 1)) * S + kc) * 4 + (kr & 3);
        std::memcpy(&out[e], &hv, 4);
      }
  }
}

cudaError_t launch_dft_H(const OpArgs& a, cudaStream_t s, int grid) {
  if (a.n_work <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  dft_kernel<false><<<std::min(grid, a.n_work), NT, SMEM_D, s>>>(a);
  return cudaGetLastError();
}

// H^T r into the output, then (OP_STEP) the projected-gradient step in place
cudaError_t launch_dft_Ht(const OpArgs& a, cudaStream_t s, int grid) {
  if (a.n_work <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  OpArgs p = a;
  p.mode = OP_PLAIN;
  dft_kernel<true><<<std::min(grid, a.n_work), NT, SMEM_D, s>>>(p);
  if (a.mode == OP_PLAIN) return cudaGetLastError();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int b = S - a.K + 1;
  dft_step_kernel<<<a.n_work, 256, (size_t)(b + 2) * (b + 2) * sizeof(float), s>>>(a);
  return cudaGetLastError();
}

int dft_Ht_kernels(int mode) { return mode == OP_PLAIN ? 1 : 2; }

}  // namespace dv
