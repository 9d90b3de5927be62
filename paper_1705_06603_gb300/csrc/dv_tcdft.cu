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
// [Fr; Fi] (cos and -sin, FP16) in shared memory, ordered so that every
// tensor-memory lane (a thread) owns one row of the next stage's operand:
//   stage 1  Y[kr][c]    = sum_r F[kr][r] X[r][c]            (M = kr, N = c; Fr and Fi)
//   stage 2  Z^T[kc][kr] = sum_c F[kc][c] Y[kr][c]            (M = kc, N = re|im kr)
//            as Fr [Yr | Yi] + Fi [-Yi | Yr] over one buffer [-Yi | Yr | Yi]
//   inverse  U[r][kc]    = sum_kr conj F[r][kr] Z[kr][kc]     (Fr [Zr | Zi] + Fi [Zi | -Zr])
//            x[r][c]     = Re sum_kc U[r][kc] conj F[c][kc]   (Ur Fr + Ui Fi)
// Operands are K-major, no swizzle: a matrix of R rows and K columns is stored
// as K / 8 panels of R 16-byte rows (a panel stride padded by 16 bytes), so a
// 16-wide k-step is two consecutive panels (LBO = panel stride, SBO = 128).
// Between stages the staging warps read the accumulators (each warp owns 32
// tensor-memory lanes and half of the columns), round to FP16 and write the
// next operand; the spectral products accumulate in FP32 in tensor memory.
// Scaling keeps the FP16 values in range: the spectra carry 1 / 128 and the
// first inverse stage's result another 1 / 128 (the inverse DFT's 1 / 128^2).
//
// Eight warps stage operands, take the products and run the epilogue; thread
// 0 issues the MMAs.  The grid is persistent (one CTA per SM, items from an
// atomic counter, heaviest first).  Every wait is bounded.
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
constexpr int NWS = 8;                      // warps (two per tensor-memory lane quarter)
constexpr int NTS = 32 * NWS;
constexpr int CROWS = 2 * S;                // [Fr; Fi]
constexpr int CPAN = CROWS * 16 + 16;       // panel stride (bytes) of the constants
constexpr int CBYTES = (S / 8) * CPAN;
constexpr int XPAN = S * 16 + 16;           // 128-row operand
constexpr int XBYTES = (S / 8) * XPAN;
constexpr int YROWS = 3 * S;                // [-Yi | Yr | Yi] or [Zr | Zi | -Zr]
constexpr int YPAN = YROWS * 16 + 16;
constexpr int YBYTES = (S / 8) * YPAN;
constexpr int kHdrD = 1024;
constexpr int SMEM_D = kHdrD + CBYTES + XBYTES + YBYTES + 2 * S * (int)sizeof(WTab) + 4 * S * 4;
constexpr uint32_t TMEM_COLS = 512;         // D [0, 256), Z sum [256, 512)
static_assert(SMEM_D <= 227 * 1024, "shared memory");
static_assert(YBYTES >= 2 * XBYTES, "T operands fit in the Y buffer");
static_assert(YBYTES >= S * (S + 1) * 4, "output tile fits in the Y buffer");
static_assert(CPAN % 16 == 0 && XPAN % 16 == 0 && YPAN % 16 == 0, "alignment");

struct BarsD {
  uint64_t bd, fin;
  uint32_t tmem;
  int abort;
  int item[2];                // work items of the two slots (current, next)
};
static_assert(sizeof(BarsD) <= 256, "barrier header");

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

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

// All 8 warps stage operands, take the products and run the epilogue; thread
// 0 also issues each stage's MMAs once every warp has written the operand
// (a CTA barrier, then the MMAs run asynchronously and complete on bd).  8
// warps, two per SM sub-partition, may hold up to 255 registers a thread: the
// block's x window and a PSF's spectrum slice stay in registers.
__global__ void __launch_bounds__(NTS, 1) dft_H_kernel(const OpArgs A) {
  extern __shared__ __align__(1024) unsigned char smem[];
  BarsD* H = reinterpret_cast<BarsD*>(smem);
  unsigned char* sC = smem + kHdrD;
  unsigned char* sX = sC + CBYTES;
  unsigned char* sY = sX + XBYTES;
  WTab* sTr = reinterpret_cast<WTab*>(sY + YBYTES);   // interpolation weights of the
  WTab* sTc = sTr + S;                                  // window's rows and columns
  float* sWv = reinterpret_cast<float*>(sTc + S);       // [2][wr | wc] of a PSF
  __shared__ WorkItem wis[2];
  __shared__ TileDesc tds[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = A.K, b = S - K + 1;
  const uint64_t limit = A.wait_ns ? A.wait_ns : kWaitNs;
  // thread 0: the next work item into slot s
  auto fetch = [&](int slot) {
    const int it = atomicAdd(A.counter, 1);
    H->item[slot] = it;
    if (it < A.n_work) {
      wis[slot] = A.work[it];
      tds[slot] = A.tiles[wis[slot].tile];
    }
  };
  if (tid == 0) {
    mbar_init(&H->bd, 1);
    mbar_init(&H->fin, 1);
    H->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&H->tmem, TMEM_COLS);
  // constants [Fr; Fi] (the plan's byte image of the panels)
  for (int e = tid; e < CBYTES / 16; e += NTS)
    reinterpret_cast<uint4*>(sC)[e] = __ldg(reinterpret_cast<const uint4*>(A.tcop) + e);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = H->tmem;
  const uint32_t aC = saddr(sC), aX = saddr(sX), aY = saddr(sY);
  const uint32_t id256 = idesc(0, 128, 256), id128 = idesc(0, 128, 128);
  uint32_t nd = 0;                          // completions of bd waited for so far
  const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
  const int h = warp >> 2;                  // column half of the warp
  const int L = 32 * (warp & 3) + lane;     // its tensor-memory lane
  bool ok = true;

  // operands written by every thread -> visible to the MMAs, thread 0 issues
  auto publish = [&]() {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  };
  auto wait_d = [&]() {
    const bool w = wait_bar(&H->bd, nd++ & 1, &H->abort, A.err, limit);
    __syncthreads();
    ok = ok && w && !*(volatile int*)&H->abort;
    tc_fence_after();
    return ok;
  };

  // the 128 x 128 x window of a block, kept in registers (FP16) for all its
  // PSFs: item u of this thread = column c, rows 8q .. 8q + 7 (e = tid + 256 u);
  // loaded for the next block while the current block's inverse runs
  uint32_t xv[8][4];
  // every load of the window is issued before the first is used; threads
  // 0 .. 2S - 1 also fetch the weight table of one window row or column
  // (stored once the current block's last X_p has been staged)
  auto load_x = [&](const WorkItem& w2, const TileDesc& t2, WTab& tab) {
    const float* img2 = A.in + t2.xoff;
    const int C = w2.c0 + (tid & (S - 1));
    float v[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = (tid + u * NTS) >> 7;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int R = w2.r0 + 8 * q + t;
        v[u][t] = (R < t2.nxr && C < t2.nxc) ? __ldg(img2 + (int64_t)R * t2.xpitch + C) : 0.f;
      }
    }
    tab = WTab{-2, 0.f, 0.f, 0};
    if (tid < S) {
      const int R = w2.r0 + tid;
      if (R < t2.nxr) tab = A.wrow[t2.wr0 + R];
    } else {
      const int Cc = w2.c0 + tid - S;
      if (Cc < t2.nxc) tab = A.wcol[t2.wc0 + Cc];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int t = 0; t < 4; ++t) xv[u][t] = pack_h2(v[u][2 * t], v[u][2 * t + 1]);
  };
  static_assert(NTS == 2 * S, "one weight table entry per thread");
  auto store_tab = [&](const WTab& tab) { (tid < S ? sTr : sTc - S)[tid] = tab; };
  auto psfs_of = [](const WorkItem& w2) { return (w2.a_hi - w2.a_lo + 1) * (w2.b_hi - w2.b_lo + 1); };
  // the x window of the item in slot s and the observed image and weights of
  // its output block, prefetched into L2 a block ahead (one 128-byte line
  // per request, at an element inside the image)
  auto prefetch_next = [&](int slot) {
    if (H->item[slot] >= A.n_work) return;
    const WorkItem& w2 = wis[slot];
    const TileDesc& t2 = tds[slot];
    if (psfs_of(w2) == 0) return;
    const int rr = tid & (S - 1);
    const int R = w2.r0 + rr, c_end = min(w2.c0 + S, t2.nxc);
    if (R < t2.nxr) {
      const float* row = A.in + t2.xoff + (int64_t)R * t2.xpitch;
      for (int C = w2.c0 + 32 * (tid >> 7); C < c_end; C += 64) prefetch_l2(row + C);
      if ((tid >> 7) == 0) prefetch_l2(row + c_end - 1);
    }
    if (A.mode != OP_PLAIN) {
      const int bb = S - A.K + 1;
      const int i = w2.r0 + rr, j_end = min(w2.c0 + bb, t2.nyc);
      if (rr < bb && i < t2.nyr && w2.c0 < j_end) {
        const int64_t g0 = (int64_t)(t2.xr0 + i) * A.wy + t2.xc0;
        const float* src = (tid >> 7) == 0 ? A.y : A.W;
        if (src) {
          for (int j = w2.c0; j < j_end; j += 32) prefetch_l2(src + g0 + j);
          prefetch_l2(src + g0 + j_end - 1);
        }
      }
    }
  };
  if (tid == 0) fetch(0);
  int cur = 0;
  bool have_x = false;
  for (;;) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (H->item[cur] >= A.n_work || !ok || *(volatile int*)&H->abort) break;
    // the next item (slot cur ^ 1 is free: the previous block has finished),
    // published by the next barrier
    if (tid == 0) fetch(cur ^ 1);
    const WorkItem& wi = wis[cur];
    const TileDesc& td = tds[cur];
    const int nb = wi.b_hi - wi.b_lo + 1;
    const int np = psfs_of(wi);
    float* out = A.out;

    if (np == 0) {
      // no PSF reaches the block: H x is zero there
      for (int e = tid; e < b * b; e += NTS) {
        const int i = wi.r0 + e / b, jj = wi.c0 + e % b;
        if (i >= td.nyr || jj >= td.nyc) continue;
        const int64_t gi = (int64_t)(td.xr0 + i) * A.wy + (td.xc0 + jj);
        const float wt = (A.mode != OP_PLAIN && A.W) ? A.W[gi] : 1.f;
        out[td.yoff + (int64_t)i * td.ypitch + jj] = A.mode == OP_PLAIN ? 0.f : -wt * A.y[gi];
      }
      __syncthreads();
      if (tid == 0) fetch(cur ^ 1);
      cur ^= 1;
      have_x = false;
      continue;
    }
    if (!have_x) {
      WTab tab;
      load_x(wi, td, tab);
      store_tab(tab);
      __syncthreads();
    }

    // X_p^T into sX: element (m = c, k = r) = w_p(r0 + r, c0 + c) x(r0 + r, c0 + c)
    // (rows and columns outside the tile have the table {-2, 0, 0}); the
    // PSF's row and column weights go to buffer p & 1 of sWv, which stage
    // p - 2 last read, before the barriers of pair p - 2's stages
    auto stage_x = [&](int p) {
      const int ga = wi.a_lo + p / nb, gb = wi.b_lo + p % nb;
      float* wv = sWv + (p & 1) * 2 * S;
      wv[tid] = tid < S ? wsel(sTr[tid], ga) : wsel(sTc[tid - S], gb);
      __syncthreads();
      const int c = tid & (S - 1);
      const float wc = wv[S + c];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = (tid + u * NTS) >> 7;
        const float4 w0 = *reinterpret_cast<const float4*>(wv + 8 * q);
        const float4 w1 = *reinterpret_cast<const float4*>(wv + 8 * q + 4);
        const float wr[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        uint32_t o[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float2 fx = __half22float2(*reinterpret_cast<const __half2*>(&xv[u][t]));
          o[t] = pack_h2(wr[2 * t] * wc * fx.x, wr[2 * t + 1] * wc * fx.y);
        }
        *reinterpret_cast<uint4*>(sX + q * XPAN + 16 * c) = make_uint4(o[0], o[1], o[2], o[3]);
      }
    };

    stage_x(0);
    publish();
    if (tid == 0) {
      chain(tbase, aC, CPAN, aX, XPAN, id128, false);                    // Yr = Fr X
      chain(tbase + S, aC + 16 * S, CPAN, aX, XPAN, id128, false);       // Yi = Fi X
      tc_commit(&H->bd);
    }
    prefetch_next(cur ^ 1);
    for (int p = 0; p < np; ++p) {
      // Y (lane kr): columns 0..127 = Yr[kr][c], 128..255 = Yi[kr][c] into
      // rows S + kr (Yr), kr (-Yi) and 2S + kr (Yi) of the buffer [-Yi | Yr | Yi];
      // half h of the warps takes c in [64h, 64h + 64), 8 consecutive c per
      // 16-byte store
      if (!wait_d()) break;
      for (int c0 = 64 * h; c0 < 64 * h + 64; c0 += 16) {
        uint32_t yr[16], yi[16];
        tmem_ld16_nowait(tbase + lanes + (uint32_t)c0, yr);
        tmem_ld16_nowait(tbase + lanes + (uint32_t)(S + c0), yi);
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 16; t += 8) {
          const float* f = reinterpret_cast<const float*>(yr + t);
          const float* g = reinterpret_cast<const float*>(yi + t);
          const int off = ((c0 + t) >> 3) * YPAN + 16 * L;
          *reinterpret_cast<uint4*>(sY + off + 16 * S) = make_uint4(
              pack_h2(f[0], f[1]), pack_h2(f[2], f[3]), pack_h2(f[4], f[5]), pack_h2(f[6], f[7]));
          *reinterpret_cast<uint4*>(sY + off) = make_uint4(
              pack_h2(-g[0], -g[1]), pack_h2(-g[2], -g[3]), pack_h2(-g[4], -g[5]),
              pack_h2(-g[6], -g[7]));
          *reinterpret_cast<uint4*>(sY + off + 32 * S) = make_uint4(
              pack_h2(g[0], g[1]), pack_h2(g[2], g[3]), pack_h2(g[4], g[5]), pack_h2(g[6], g[7]));
        }
      }
      publish();
      if (tid == 0) {
        chain(tbase, aC, CPAN, aY + 16 * S, YPAN, id256, false);         // Fr [Yr | Yi]
        chain(tbase, aC + 16 * S, CPAN, aY, YPAN, id256, true);          // Fi [-Yi | Yr]
        tc_commit(&H->bd);
      }
      // the PSF's spectrum at this thread's column kc = L and rows kr of its
      // half, fetched while the stage-2 MMAs run
      const int ga = wi.a_lo + p / nb, gb = wi.b_lo + p % nb;
      const unsigned int* hh =
          reinterpret_cast<const unsigned int*>(A.spec) + (size_t)(ga * A.Gc + gb) * S * S;
      uint32_t hv[64];
#pragma unroll
      for (int t = 0; t < 64; ++t) hv[t] = __ldg(hh + (size_t)(64 * h + t) * S + L);
      // the next PSF's X (S1 of PSF p has completed: sX is free)
      if (p + 1 < np) stage_x(p + 1);
      if (!wait_d()) break;
      // Z^T (lane kc): columns kr (re) and S + kr (im); sum += Z . Hh_p over
      // kr in this warp's half
#pragma unroll
      for (int k8 = 0; k8 < 8; ++k8) {
        const int k0 = 64 * h + 8 * k8;
        uint32_t zr[8], zi[8], ar[8], ai[8];
        tmem_ld8_nowait(tbase + lanes + (uint32_t)k0, zr);
        tmem_ld8_nowait(tbase + lanes + (uint32_t)(S + k0), zi);
        if (p > 0) {
          tmem_ld8_nowait(tbase + lanes + (uint32_t)(2 * S + k0), ar);
          tmem_ld8_nowait(tbase + lanes + (uint32_t)(3 * S + k0), ai);
        }
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const float2 hf = __half22float2(*reinterpret_cast<const __half2*>(&hv[8 * k8 + t]));
          const float a = __uint_as_float(zr[t]), bb = __uint_as_float(zi[t]);
          const float re = a * hf.x - bb * hf.y, im = a * hf.y + bb * hf.x;
          ar[t] = __float_as_uint(p > 0 ? __uint_as_float(ar[t]) + re : re);
          ai[t] = __float_as_uint(p > 0 ? __uint_as_float(ai[t]) + im : im);
        }
        tmem_st8_nowait(tbase + lanes + (uint32_t)(2 * S + k0), ar);
        tmem_st8_nowait(tbase + lanes + (uint32_t)(3 * S + k0), ai);
      }
      tmem_wait_st();
      if (p + 1 < np) {
        publish();   // D read, X_{p+1} written
        if (tid == 0) {
          chain(tbase, aC, CPAN, aX, XPAN, id128, false);
          chain(tbase + S, aC + 16 * S, CPAN, aX, XPAN, id128, false);
          tc_commit(&H->bd);
        }
      }
    }
    if (!ok) break;
    // inverse, stage 1 operand: the sum (lane kc, columns kr) -> rows kc,
    // S + kc, 2S + kc of [Zr | Zi | -Zr], 8 consecutive kr per 16-byte store
    for (int k0 = 64 * h; k0 < 64 * h + 64; k0 += 16) {
      uint32_t ar[16], ai[16];
      tmem_ld16_nowait(tbase + lanes + (uint32_t)(2 * S + k0), ar);
      tmem_ld16_nowait(tbase + lanes + (uint32_t)(3 * S + k0), ai);
      tmem_wait_ld();
#pragma unroll
      for (int t = 0; t < 16; t += 8) {
        const float* zr = reinterpret_cast<const float*>(ar + t);
        const float* zi = reinterpret_cast<const float*>(ai + t);
        const int off = ((k0 + t) >> 3) * YPAN + 16 * L;
        *reinterpret_cast<uint4*>(sY + off) = make_uint4(
            pack_h2(zr[0], zr[1]), pack_h2(zr[2], zr[3]), pack_h2(zr[4], zr[5]), pack_h2(zr[6], zr[7]));
        *reinterpret_cast<uint4*>(sY + off + 16 * S) = make_uint4(
            pack_h2(zi[0], zi[1]), pack_h2(zi[2], zi[3]), pack_h2(zi[4], zi[5]), pack_h2(zi[6], zi[7]));
        *reinterpret_cast<uint4*>(sY + off + 32 * S) = make_uint4(
            pack_h2(-zr[0], -zr[1]), pack_h2(-zr[2], -zr[3]), pack_h2(-zr[4], -zr[5]),
            pack_h2(-zr[6], -zr[7]));
      }
    }
    publish();
    if (tid == 0) {
      chain(tbase, aC, CPAN, aY, YPAN, id256, false);                    // Fr [Zr | Zi]
      chain(tbase, aC + 16 * S, CPAN, aY + 16 * S, YPAN, id256, true);   // Fi [Zi | -Zr]
      tc_commit(&H->bd);
    }
    // the next block's x window, in flight while this block's inverse runs
    have_x = H->item[cur ^ 1] < A.n_work && psfs_of(wis[cur ^ 1]) > 0;
    if (have_x) {
      WTab tab;
      load_x(wis[cur ^ 1], tds[cur ^ 1], tab);
      store_tab(tab);   // this block's tables were last read by its last X_p
    }
    // U (lane r): columns kc (re), S + kc (im), scaled by 1 / 128, into the
    // last stage's operands Ur (sX) and Ui (sY), rows r, k = kc
    if (!wait_d()) break;
    for (int k0 = 0; k0 < S; k0 += 16) {
      uint32_t r[16];
      tmem_ld16_nowait(tbase + lanes + (uint32_t)(S * h + k0), r);
      tmem_wait_ld();
      unsigned char* dst = h == 0 ? sX : sY;
      const float sc = 1.f / S;
#pragma unroll
      for (int t = 0; t < 16; t += 8)
        *reinterpret_cast<uint4*>(dst + ((k0 + t) >> 3) * XPAN + 16 * L) = make_uint4(
            pack_h2(sc * __uint_as_float(r[t]), sc * __uint_as_float(r[t + 1])),
            pack_h2(sc * __uint_as_float(r[t + 2]), sc * __uint_as_float(r[t + 3])),
            pack_h2(sc * __uint_as_float(r[t + 4]), sc * __uint_as_float(r[t + 5])),
            pack_h2(sc * __uint_as_float(r[t + 6]), sc * __uint_as_float(r[t + 7])));
    }
    publish();
    if (tid == 0) {
      chain(tbase, aX, XPAN, aC, CPAN, id128, false);                    // Ur Fr
      chain(tbase, aY, XPAN, aC + 16 * S, CPAN, id128, true);            // Ui Fi
      tc_commit(&H->bd);
    }
    // x (lane r, columns c) -> an FP32 tile in the Y buffer (free once the
    // last MMAs have completed), then the valid rows and columns K - 1 .. 127
    // are written row by row (coalesced observed image, weights and output)
    if (!wait_d()) break;
    {
      float* tile = reinterpret_cast<float*>(sY);
      constexpr int TPT = S + 1;
      for (int c0 = 64 * h; c0 < 64 * h + 64; c0 += 16) {
        uint32_t v[16];
        tmem_ld16_nowait(tbase + lanes + (uint32_t)c0, v);
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 16; ++t) tile[L * TPT + c0 + t] = __uint_as_float(v[t]);
      }
      __syncthreads();
      const int nr = min(b, td.nyr - wi.r0), nc = min(b, td.nyc - wi.c0);
      // batches of EPB elements a thread: the observed image and weights of
      // a batch are loaded before any of its outputs is written
      constexpr int EPB = 18;
      for (int e0 = tid; e0 < nr * b; e0 += EPB * NTS) {
        float yo[EPB], wo[EPB];
#pragma unroll
        for (int u = 0; u < EPB; ++u) {
          const int e = e0 + u * NTS, il = e / b, jl = e - il * b;
          yo[u] = 0.f;
          wo[u] = 1.f;
          if (A.mode != OP_PLAIN && e < nr * b && jl < nc) {
            const int64_t gi = (int64_t)(td.xr0 + wi.r0 + il) * A.wy + (td.xc0 + wi.c0 + jl);
            yo[u] = __ldg(A.y + gi);
            if (A.W) wo[u] = __ldg(A.W + gi);
          }
        }
#pragma unroll
        for (int u = 0; u < EPB; ++u) {
          const int e = e0 + u * NTS, il = e / b, jl = e - il * b;
          if (e >= nr * b || jl >= nc) continue;
          const float y = tile[(il + K - 1) * TPT + jl + K - 1];
          out[td.yoff + (int64_t)(wi.r0 + il) * td.ypitch + wi.c0 + jl] =
              A.mode == OP_PLAIN ? y : wo[u] * (y - yo[u]);
        }
      }
    }
    cur ^= 1;
  }
  if (!ok) *(volatile int*)&H->abort = 1;
  // teardown: every MMA this CTA issued has completed before tensor memory is freed
  if (tid == 0) {
    tc_commit(&H->fin);
    drain_bar(&H->fin, 0, A.err);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
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
// Hh(kr, kc) = sum_{m, n < K} h(m, n) exp(-2 pi i (kr m + kc n) / 128) / 128,
// summed in FP64 on the host and stored as FP16 (re, im) pairs.
void dft_spectra(const float* psfs, int G, int K, std::vector<uint32_t>& out) {
  std::vector<double> cr(S), ci(S);
  for (int j = 0; j < S; ++j) {
    const double a = -2.0 * 3.14159265358979323846 * j / S;
    cr[j] = std::cos(a);
    ci[j] = std::sin(a);
  }
  out.assign((size_t)G * S * S, 0u);
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
        const __half2 hv = __floats2half2_rn((float)(sr / S), (float)(si / S));
        std::memcpy(&out[((size_t)g * S + kr) * S + kc], &hv, 4);
      }
  }
}

cudaError_t launch_dft_H(const OpArgs& a, cudaStream_t s, int grid) {
  if (a.n_work <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  dft_H_kernel<<<std::min(grid, a.n_work), NTS, SMEM_D, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dv
