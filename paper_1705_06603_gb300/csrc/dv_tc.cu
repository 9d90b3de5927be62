// Tensor-core (tcgen05) kernels of the shift-variant operator of Sec. II-B
// and its adjoint: BF16 or TF32 operands, FP32 accumulation in tensor memory.
//
// For one PSF and one filter row a, a correlation is a banded-Toeplitz
// product over the staged input block S:
//     D[i][j] += sum_c S[i + a][c] T_a[c][j],   T_a[c][j] = f(a, c - j), 0 <= c - j < K,
// with f the flipped PSF (H) or the PSF (H^T).  A CTA owns BM = 128 output
// rows x BN = 64 output columns; one tcgen05.mma (M = 128, N = 64, 32 bytes
// of K) covers the k-step ks of tap row a:
//   A = rows i + a of S, columns [KM ks, KM ks + KM): shared memory, K-major,
//       no swizzle, each 16-byte column chunk a panel of rows 16 bytes apart,
//       so the row shift a is the start address plus 16 a;
//   B = T_a on the same columns, N x KM, K-major: a 64-row window of one
//       "tall" matrix per tap row, Bt[n'][k] = f(a, k + KM (KS - 1) - n'),
//       two panels of (64 + KM (KS - 1)) x 16 bytes of which only K + CH - 1
//       rows per panel are nonzero.  Those windows are precomputed on the
//       host per PSF and tap row and streamed by cp.async.bulk into a ring of
//       stages (zero outside the windows) guarded by mbarriers.
// The FP32 input window (rows + K - 1, columns of all k-steps) is copied once
// per CTA into shared memory by cp.async (zero-filled outside the tile), then
// converted into the operand panels:
//   H:   S = w_p . x per PSF (double-buffered when it fits); all PSFs
//        accumulate into one 128 x 64 FP32 accumulator in tensor memory.
//   H^T: S = r once; PSF p accumulates into tensor-memory buffer p & 1 and the
//        epilogue warps add w_p . D_p into registers while the next PSF's
//        MMAs run; the projected-gradient step is fused.
// Warp roles: warps 0-3 stage operands and run the epilogue (warp w reads
// tensor-memory lanes 32w .. 32w + 31, i.e. output rows); warp 4 allocates
// tensor memory and one of its lanes issues every MMA; one lane of warp 5
// refills the B ring as soon as the MMAs of a stage have completed.  Every
// mbarrier wait gives up after about two seconds, records the timeout in the
// plan's error word and sends the whole CTA to its teardown, which waits (with
// its own bound) for the copies and MMAs it issued and frees tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "dv_internal.cuh"
#include "dv_tcgen05.cuh"

namespace dv {
namespace {

constexpr int BM = 128, BN = 64;
constexpr int NWE = 4;                    // staging / epilogue warps
constexpr int NTH = 32 * (NWE + 2);       // + the MMA warp and the bulk-copy warp
constexpr int OPITCH = BN + 1;            // fp32 output staging pitch (floats)

// PREC 0: BF16 (8 elements per 16-byte chunk, MMA K = 16); 1: TF32 (4, 8)
template <int PREC>
struct Elt {
  static constexpr int bytes = PREC == 0 ? 2 : 4;
  static constexpr int chunk = 16 / bytes;
  static constexpr int km = 32 / bytes;
};

constexpr int kSmemMax = 227 * 1024;      // dynamic shared memory per CTA
constexpr int kHdrBytes = 512;            // mbarrier header at the start of it
constexpr int kMaxWcol = 16;              // H^T: PSF grid columns whose output weights are staged
constexpr int kMaxWcolBytes = kMaxWcol * BN * 4;

template <int PREC, int K>
struct Geo {
  static constexpr int KM = Elt<PREC>::km;
  static constexpr int CH = Elt<PREC>::chunk;
  static constexpr int KS = (BN - 1 + K + KM - 1) / KM;   // MMAs per tap row
  static constexpr int COLS = KS * KM;                    // staged input columns
  static constexpr int NCH = COLS / CH;                   // 16-byte column panels
  static constexpr int ROWS = BM + K - 1;                 // staged input rows
  static constexpr int APANEL = ROWS * 16 + 16;           // + 16 spreads panels over banks
  static constexpr int ABYTES = NCH * APANEL;
  static constexpr int RB = BN + KM * (KS - 1);           // rows of the tall B operand
  static constexpr int BPANEL = RB * 16;
  static constexpr int BBYTES = 2 * BPANEL;               // one ring stage (one tap row)
  static constexpr int WR = K + CH - 1;                   // nonzero rows per panel
  static constexpr int S0 = KM * (KS - 1) - K + 1;        // first nonzero row of panel 0
  static constexpr int WBYTES_TX = 2 * WR * 16;           // bytes streamed per tap row
  static constexpr int XBYTES = ROWS * COLS * 4;          // FP32 input window
  // epilogue: fp32 output block, and for the H^T step the (BM + 2) x (BN + 2)
  // halo of the iterate
  static constexpr int OBYTES = BM * OPITCH * 4;
  static constexpr int HBYTES = (BM + 2) * (BN + 2) * 4;
  // H: [A buffers (also the output block) | x window | B ring | weights]
  static constexpr int WGT_H = 2 * (ROWS + COLS) * 4;
  static constexpr int sz_h(int na, int nst) {
    return kHdrBytes + (na * ABYTES > OBYTES ? na * ABYTES : OBYTES) + XBYTES + nst * BBYTES + WGT_H;
  }
  static constexpr int NA = sz_h(2, 8) <= kSmemMax ? 2 : 1;
  static constexpr int NST_H = sz_h(NA, 16) <= kSmemMax ? 16 : (sz_h(NA, 8) <= kSmemMax ? 8 : 4);
  static constexpr int AREG_H = NA * ABYTES > OBYTES ? NA * ABYTES : OBYTES;
  // H^T: [A | x window, later output block + halo | B ring | column weights]
  static constexpr int UREG_HT = XBYTES > OBYTES + HBYTES ? XBYTES : OBYTES + HBYTES;
  static constexpr int sz_ht(int nst) {
    return kHdrBytes + ABYTES + UREG_HT + nst * BBYTES + kMaxWcolBytes;
  }
  static constexpr int NST_HT = sz_ht(16) <= kSmemMax ? 16 : (sz_ht(8) <= kSmemMax ? 8 : 4);
  static_assert(S0 >= 0 && S0 + CH + WR <= RB, "Toeplitz windows inside the panels");
  static_assert(sz_h(NA, NST_H) <= kSmemMax && sz_ht(NST_HT) <= kSmemMax, "shared memory");
};

constexpr int NSTMAX = 16;
struct Bars {            // mbarriers etc., at the start of dynamic shared memory
  uint64_t bfull[NSTMAX], bempty[NSTMAX];
  uint64_t afull[2], aempty[2];
  uint64_t dfull[2], dempty[2];
  uint64_t fin;          // all MMAs of the CTA complete (teardown)
  uint32_t tmem;         // tensor-memory base written by tcgen05.alloc
  int abort;             // set by the first wait that gives up
};
static_assert(sizeof(Bars) <= kHdrBytes, "barrier header");
constexpr int kHdr = kHdrBytes;

template <int PREC, int K>
constexpr size_t smem_H() { return (size_t)Geo<PREC, K>::sz_h(Geo<PREC, K>::NA, Geo<PREC, K>::NST_H); }
template <int PREC, int K>
constexpr size_t smem_Ht() { return (size_t)Geo<PREC, K>::sz_ht(Geo<PREC, K>::NST_HT); }
// Requests are at least this large so that at most 3 CTAs (128 tensor-memory
// columns at most each) share an SM: their allocations stay within the 512
// columns, so tcgen05.alloc never has to wait for another CTA.
constexpr size_t kMinSmem = 58 * 1024;

using namespace tcg;

__device__ __forceinline__ void named_sync() { tcg::named_sync<32 * NWE>(); }
__device__ __forceinline__ bool named_all(bool v) { return tcg::named_all<32 * NWE>(v); }
template <int PREC>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  if constexpr (PREC == 0)
    mma_bf16(d, a, b, idesc(1, BM, BN), acc);
  else
    mma_tf32(d, a, b, idesc(2, BM, BN), acc);
}

template <int PREC, int K>
__device__ __forceinline__ void put_chunk(unsigned char* abuf, int ir, int q, const float* v) {
  using G = Geo<PREC, K>;
  *reinterpret_cast<uint4*>(abuf + (size_t)q * G::APANEL + ir * 16) = pack_chunk<PREC>(v);
}

// The MMAs of one tap row: KS k-steps accumulating into tensor-memory column
// d.  ad = descriptor of A at rows a .. (k-step 0), bd = descriptor of the B
// stage at the window of k-step 0; the start-address field counts 16-byte
// units and never carries out of its 14 bits (shared memory < 256 KB), so
// the k-step descriptors are plain constant offsets.
template <int PREC, int K>
__device__ __forceinline__ void issue_row(uint32_t d, uint64_t ad, uint64_t bd, bool first) {
  using G = Geo<PREC, K>;
  mma<PREC>(d, ad, bd, first ? 0u : 1u);
#pragma unroll
  for (int ks = 1; ks < G::KS; ++ks)
    mma<PREC>(d, ad + (uint64_t)(2 * ks * (G::APANEL >> 4)), bd - (uint64_t)(ks * G::KM), 1u);
}

// One lane of warp 5: streams the B tap rows of the PSFs (a_lo..a_hi) x
// (b_lo..b_hi), in the order the MMA lane consumes them, through the
// NST-stage ring; a stage is refilled once the MMAs that read it completed.
template <int PREC, int K, int NST>
__device__ void producer(const OpArgs& A, const WorkItem& wi, Bars* H, unsigned char* breg, int np) {
  using G = Geo<PREC, K>;
  const int nb = wi.b_hi - wi.b_lo + 1;
  const int total = np * K;
  int issued = 0;
  for (int it = 0; it < total; ++it) {
    const int s = it % NST;
    if (it >= NST && !wait_bar(&H->bempty[s], (uint32_t)((it / NST - 1) & 1), &H->abort, A.err)) break;
    const int p = it / K, a = it - p * K;
    const int ga = wi.a_lo + p / nb, gb = wi.b_lo + p % nb;
    const unsigned char* src = A.tcop + ((size_t)(ga * A.Gc + gb) * K + a) * G::WBYTES_TX;
    unsigned char* dst = breg + (size_t)s * G::BBYTES;
    mbar_expect_tx(&H->bfull[s], G::WBYTES_TX);
    bulk_g2s(dst + G::S0 * 16, src, G::WR * 16, &H->bfull[s]);
    bulk_g2s(dst + G::BPANEL + (G::S0 + G::CH) * 16, src + G::WR * 16, G::WR * 16, &H->bfull[s]);
    issued = it + 1;
  }
  // teardown: every copy issued must have landed before the CTA exits
  for (int it = (issued > NST ? issued - NST : 0); it < issued; ++it)
    if (!drain_bar(&H->bfull[it % NST], (uint32_t)((it / NST) & 1), A.err)) break;
}

// One lane of warp 4: issues the MMAs of every tap row as soon as its B
// stage has landed, and releases the stage with a commit (never waits for
// MMA completion except at buffer hand-overs).
// H (ADJ = false): PSF p reads A buffer p % NA and accumulates into d0.
// H^T (ADJ = true): PSF p reads the single A buffer and accumulates into
// d0 + 64 (p & 1) once the epilogue has released that buffer.
template <int PREC, int K, bool ADJ, int NST>
__device__ void issuer(const OpArgs& A, Bars* H, unsigned char* areg, unsigned char* breg,
                       uint32_t d0, int np) {
  using G = Geo<PREC, K>;
  // B descriptor of stage 0 at the window of k-step 0
  const uint64_t bd0 = sdesc(saddr(breg) + 16u * G::KM * (G::KS - 1), G::BPANEL);
  bool ok = true;
  for (int p = 0; p < np && ok; ++p) {
    uint32_t a_base, d;
    if constexpr (ADJ) {
      a_base = saddr(areg);
      d = d0 + 64u * (uint32_t)(p & 1);
      if (p == 0) ok = wait_bar(&H->afull[0], 0, &H->abort, A.err);
      if (ok && p >= 2) ok = wait_bar(&H->dempty[p & 1], (uint32_t)((p / 2 - 1) & 1), &H->abort, A.err);
    } else {
      const int ab = p % G::NA;
      a_base = saddr(areg + (size_t)ab * G::ABYTES);
      d = d0;
      ok = wait_bar(&H->afull[ab], (uint32_t)((p / G::NA) & 1), &H->abort, A.err);
    }
    if (!ok) break;
    tc_fence_after();
    const uint64_t ad0 = sdesc(a_base, G::APANEL);
    int s = (p * K) % NST;
    uint32_t ph = (uint32_t)(((p * K) / NST) & 1);
    for (int a = 0; a < K; ++a) {
      if (!wait_bar(&H->bfull[s], ph, &H->abort, A.err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      issue_row<PREC, K>(d, ad0 + (uint64_t)a, bd0 + (uint64_t)(s * (G::BBYTES >> 4)),
                         ADJ ? (a == 0) : (p == 0 && a == 0));
      tc_commit(&H->bempty[s]);
      if (++s == NST) {
        s = 0;
        ph ^= 1u;
      }
    }
    if (!ok) break;
    if constexpr (ADJ) {
      tc_commit(&H->dfull[p & 1]);
    } else {
      tc_commit(&H->aempty[p % G::NA]);
    }
  }
  if constexpr (!ADJ) {
    if (ok && np > 0) tc_commit(&H->dfull[0]);
  }
  // teardown: the MMAs this lane issued must be complete before tensor
  // memory is freed and the CTA exits
  tc_commit(&H->fin);
  drain_bar(&H->fin, 0, A.err);
}

// Zeroes the rows of the B ring outside the windows the bulk copies fill
// (the staging threads, once per CTA, before the first MMA may run).
template <int PREC, int K, int NST>
__device__ __forceinline__ void zero_ring(unsigned char* breg, int tid) {
  using G = Geo<PREC, K>;
  for (int e = tid; e < NST * 2 * G::RB; e += 32 * NWE) {
    const int s = e / (2 * G::RB), rem = e - s * 2 * G::RB, pn = rem / G::RB, n = rem - pn * G::RB;
    const int w0 = G::S0 + pn * G::CH;
    if (n < w0 || n >= w0 + G::WR)
      *reinterpret_cast<uint4*>(breg + (size_t)s * G::BBYTES + pn * G::BPANEL + n * 16) =
          make_uint4(0u, 0u, 0u, 0u);
  }
}

// FP32 window rows r0 .., columns c0 .. of a pitched image into sX
// [ROWS][COLS] by cp.async; elements outside [0, nr) x [0, nc) (and columns
// past `cmax` of the window) are zero-filled.
template <int PREC, int K>
__device__ __forceinline__ void load_window(float* sX, const float* img, int64_t pitch, int r0, int c0,
                                            int nr, int nc, int cmax, int tid) {
  using G = Geo<PREC, K>;
  for (int e = tid; e < G::ROWS * G::COLS; e += 32 * NWE) {
    const int ir = e / G::COLS, ic = e - ir * G::COLS;
    const int R = r0 + ir, C = c0 + ic;
    const bool in = R >= 0 && R < nr && C >= 0 && C < nc && ic < cmax;
    const float* src = in ? img + (int64_t)R * pitch + C : img;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(saddr(sX + e)), "l"(src),
                 "r"(in ? 4 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void init_bars(Bars* H) {
  for (int s = 0; s < NSTMAX; ++s) {
    mbar_init(&H->bfull[s], 1);
    mbar_init(&H->bempty[s], 1);
  }
  for (int b = 0; b < 2; ++b) {
    mbar_init(&H->afull[b], 32 * NWE);
    mbar_init(&H->aempty[b], 1);
    mbar_init(&H->dfull[b], 1);
    mbar_init(&H->dempty[b], 32 * NWE);
  }
  mbar_init(&H->fin, 1);
  H->abort = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// ------------------------------------------------------------------ H kernel
template <int PREC, int K>
__global__ void __launch_bounds__(NTH, 1) tc_H_kernel(const OpArgs A) {
  using G = Geo<PREC, K>;
  extern __shared__ __align__(1024) unsigned char smem[];
  Bars* H = reinterpret_cast<Bars*>(smem);
  constexpr int NST = G::NST_H;
  unsigned char* areg = smem + kHdr;
  float* sX = reinterpret_cast<float*>(areg + G::AREG_H);                  // [ROWS][COLS]
  unsigned char* breg = reinterpret_cast<unsigned char*>(sX) + G::XBYTES;
  float* sWr = reinterpret_cast<float*>(breg + (size_t)NST * G::BBYTES);   // [2][ROWS]
  float* sWc = sWr + 2 * G::ROWS;                                         // [2][COLS]
  __shared__ double red[NWE];
  const WorkItem wi = A.work[blockIdx.x];
  const TileDesc td = A.tiles[wi.tile];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) init_bars(H);
  if (warp == NWE) tmem_alloc(&H->tmem, 64);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = H->tmem;
  const int nb = wi.b_hi - wi.b_lo + 1;
  const int np = (wi.a_hi - wi.a_lo + 1) * nb;

  if (warp == NWE) {
    if (lane == 0) issuer<PREC, K, false, NST>(A, H, areg, breg, tbase, np);
    __syncwarp();
  } else if (warp == NWE + 1) {
    if (lane == 0) producer<PREC, K, NST>(A, wi, H, breg, np);
    __syncwarp();
  } else {
    // the x window (rows r0 .., columns c0 ..) once, then S_p = w_p . x per
    // PSF into A buffer p % NA
    zero_ring<PREC, K, NST>(breg, tid);
    if (np > 0)
      load_window<PREC, K>(sX, A.in + td.xoff, td.xpitch, wi.r0, wi.c0, td.nxr, td.nxc, G::COLS, tid);
    bool ok = true;
    for (int p = 0; p < np && ok; ++p) {
      const int ab = p % G::NA;
      if (p >= G::NA) {
        ok = named_all(wait_bar(&H->aempty[ab], (uint32_t)((p / G::NA - 1) & 1), &H->abort, A.err));
        if (!ok) break;
      }
      const int ga = wi.a_lo + p / nb, gb = wi.b_lo + p % nb;
      float* wr = sWr + ab * G::ROWS;
      float* wc = sWc + ab * G::COLS;
      for (int e = tid; e < G::ROWS; e += 32 * NWE) {
        const int R = wi.r0 + e;
        wr[e] = R < td.nxr ? wsel(A.wrow[td.wr0 + R], ga) : 0.f;
      }
      for (int e = tid; e < G::COLS; e += 32 * NWE) {
        const int C = wi.c0 + e;
        wc[e] = C < td.nxc ? wsel(A.wcol[td.wc0 + C], gb) : 0.f;
      }
      named_sync();
      unsigned char* abuf = areg + (size_t)ab * G::ABYTES;
      for (int e = tid; e < G::ROWS * G::NCH; e += 32 * NWE) {
        const int ir = e / G::NCH, q = e - ir * G::NCH;
        float v[G::CH];
        const float rw = wr[ir];
        const float4* src = reinterpret_cast<const float4*>(sX + ir * G::COLS + q * G::CH);
        const float4* wcs = reinterpret_cast<const float4*>(wc + q * G::CH);
#pragma unroll
        for (int i = 0; i < G::CH; i += 4) {
          const float4 t = src[i / 4], c = wcs[i / 4];
          v[i] = rw * c.x * t.x;
          v[i + 1] = rw * c.y * t.y;
          v[i + 2] = rw * c.z * t.z;
          v[i + 3] = rw * c.w * t.w;
        }
        put_chunk<PREC, K>(abuf, ir, q, v);
      }
      fence_async_smem();
      mbar_arrive(&H->afull[ab]);
    }
    // epilogue: accumulator row 32 warp + lane -> fp32 staging block
    float* sO = reinterpret_cast<float*>(areg);
    if (ok && np > 0) ok = named_all(wait_bar(&H->dfull[0], 0, &H->abort, A.err));
    tc_fence_after();
    named_sync();   // every staging thread is past its last A write
    {
      const int i = 32 * warp + lane;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v[32];
        if (ok && np > 0) {
          tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + 32u * h, v);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) sO[i * OPITCH + 32 * h + j] = v[j];
      }
    }
    tc_fence_before();
    named_sync();
    double part = 0.0;
    if (ok) {
      for (int e = tid; e < BM * BN; e += 32 * NWE) {
        const int il = e / BN, jl = e - il * BN;
        const int i = wi.r0 + il, j = wi.c0 + jl;
        if (i >= td.nyr || j >= td.nyc) continue;
        const float v = sO[il * OPITCH + jl];
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
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
      if (lane == 0) red[warp] = part;
      named_sync();
      if (tid == 0) A.partials[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == NWE) {
    tc_fence_after();
    tmem_free(tbase, 64);
  }
}

// ---------------------------------------------------------------- H^T kernel
template <int PREC, int K>
__global__ void __launch_bounds__(NTH, 2) tc_Ht_kernel(const OpArgs A) {
  using G = Geo<PREC, K>;
  extern __shared__ __align__(1024) unsigned char smem[];
  Bars* H = reinterpret_cast<Bars*>(smem);
  constexpr int NST = G::NST_HT;
  unsigned char* areg = smem + kHdr;
  unsigned char* ureg = areg + G::ABYTES;      // r window, later output block + halo
  unsigned char* breg = ureg + G::UREG_HT;
  float* sWcol = reinterpret_cast<float*>(breg + (size_t)NST * G::BBYTES);   // [kMaxWcol][BN]
  const WorkItem wi = A.work[blockIdx.x];
  const TileDesc td = A.tiles[wi.tile];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) init_bars(H);
  if (warp == NWE) tmem_alloc(&H->tmem, 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = H->tmem;
  const int nb = wi.b_hi - wi.b_lo + 1;
  const int np = (wi.a_hi - wi.a_lo + 1) * nb;

  if (warp == NWE) {
    if (lane == 0) issuer<PREC, K, true, NST>(A, H, areg, breg, tbase, np);
    __syncwarp();
  } else if (warp == NWE + 1) {
    if (lane == 0) producer<PREC, K, NST>(A, wi, H, breg, np);
    __syncwarp();
  } else {
    // residual block: rows R0 - (K-1) .., columns C0 - (K-1) .., zero
    // outside the y-block and beyond the BN + K - 1 columns a block reads
    zero_ring<PREC, K, NST>(breg, tid);
    float* sX = reinterpret_cast<float*>(ureg);
    load_window<PREC, K>(sX, A.in + td.yoff, td.ypitch, wi.r0 - (K - 1), wi.c0 - (K - 1), td.nyr,
                         td.nyc, BN + K - 1, tid);
    named_sync();
    for (int e = tid; e < G::ROWS * G::NCH; e += 32 * NWE) {
      const int ir = e / G::NCH, q = e - ir * G::NCH;
      float v[G::CH];
      const float4* src = reinterpret_cast<const float4*>(sX + ir * G::COLS + q * G::CH);
#pragma unroll
      for (int i = 0; i < G::CH; i += 4) {
        const float4 t = src[i / 4];
        v[i] = t.x;
        v[i + 1] = t.y;
        v[i + 2] = t.z;
        v[i + 3] = t.w;
      }
      put_chunk<PREC, K>(areg, ir, q, v);
    }
    fence_async_smem();
    mbar_arrive(&H->afull[0]);
    // output column weights of the block's PSF grid columns
    const bool wcol_staged = nb <= kMaxWcol;
    if (wcol_staged) {
      for (int e = tid; e < nb * BN; e += 32 * NWE) {
        const int bi = e / BN, j = e - bi * BN;
        const int C = wi.c0 + j;
        sWcol[e] = C < td.nxc ? wsel(A.wcol[td.wc0 + C], wi.b_lo + bi) : 0.f;
      }
    }
    named_sync();

    // g = sum_p w_p . D_p over this thread's output row, in registers
    const int i = 32 * warp + lane;
    const int R = wi.r0 + i;
    float g[BN];
#pragma unroll
    for (int j = 0; j < BN; ++j) g[j] = 0.f;
    bool ok = true;
    for (int p = 0; p < np; ++p) {
      const int db = p & 1;
      if (!named_all(wait_bar(&H->dfull[db], (uint32_t)((p / 2) & 1), &H->abort, A.err))) {
        ok = false;
        break;
      }
      tc_fence_after();
      const int ga = wi.a_lo + p / nb, gb = wi.b_lo + p % nb;
      const float wr = R < td.nxr ? wsel(A.wrow[td.wr0 + R], ga) : 0.f;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v[32];
        tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + 64u * db + 32u * h, v);
        const float* wcs = sWcol + (gb - wi.b_lo) * BN + 32 * h;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float wc;
          if (wcol_staged) {
            wc = wcs[j];
          } else {
            const int C = wi.c0 + 32 * h + j;
            wc = C < td.nxc ? wsel(A.wcol[td.wc0 + C], gb) : 0.f;
          }
          g[32 * h + j] = fmaf(wr * wc, v[j], g[32 * h + j]);
        }
      }
      tc_fence_before();
      mbar_arrive(&H->dempty[db]);
    }
    // the r window is dead once A was converted (every thread passed the
    // first D wait); the output block and the iterate halo reuse it
    float* sO = reinterpret_cast<float*>(ureg);
    float* sW = reinterpret_cast<float*>(ureg + G::OBYTES);
    named_sync();
    if (ok) {
#pragma unroll
      for (int j = 0; j < BN; ++j) sO[i * OPITCH + j] = g[j];
    }
    named_sync();
    if (ok && A.mode == OP_PLAIN) {
      for (int e = tid; e < BM * BN; e += 32 * NWE) {
        const int il = e / BN, jl = e - il * BN;
        const int Ro = wi.r0 + il, Co = wi.c0 + jl;
        if (Ro < td.nxr && Co < td.nxc)
          A.out[td.xoff + (int64_t)Ro * td.xpitch + Co] = sO[il * OPITCH + jl];
      }
    } else if (ok) {
      // OP_STEP: grad = g + lambda D^T psi(D w) + alpha (w - u); w_next = max(0, w - tau grad)
      constexpr int SPW = BN + 2;
      for (int e = tid; e < (BM + 2) * SPW; e += 32 * NWE) {
        const int ir = e / SPW, ic = e - ir * SPW;
        const int Rr = wi.r0 - 1 + ir, Cc = wi.c0 - 1 + ic;
        float v = 0.f;
        if (Rr >= 0 && Rr < td.nxr && Cc >= 0 && Cc < td.nxc)
          v = A.w[td.xoff + (int64_t)Rr * td.xpitch + Cc];
        sW[e] = v;
      }
      named_sync();
      for (int e = tid; e < BM * BN; e += 32 * NWE) {
        const int il = e / BN, jl = e - il * BN;
        const int Ro = wi.r0 + il, Co = wi.c0 + jl;
        if (Ro >= td.nxr || Co >= td.nxc) continue;
        const int li = il + 1, lj = jl + 1;
        float pr, pc, pru, pcu, prl, pcl;
        huber_p(sW, SPW, li, lj, Ro, Co, td.nxr, td.nxc, A.delta, pr, pc);
        huber_p(sW, SPW, li - 1, lj, Ro - 1, Co, td.nxr, td.nxc, A.delta, pru, pcu);
        huber_p(sW, SPW, li, lj - 1, Ro, Co - 1, td.nxr, td.nxc, A.delta, prl, pcl);
        const float hub = pru - pr + pcl - pc;
        const float wv = sW[li * SPW + lj];
        const float alpha = A.gamma * A.omr[td.omr_off + Ro] * A.omc[td.omc_off + Co];
        const int64_t idx = td.xoff + (int64_t)Ro * td.xpitch + Co;
        const float grad = sO[il * OPITCH + jl] + A.lambda * hub + alpha * (wv - A.u[idx]);
        A.out[idx] = fmaxf(0.f, wv - td.tau * grad);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == NWE) {
    tc_fence_after();
    tmem_free(tbase, 128);
  }
}

template <int PREC, int K>
size_t sm_H() { return std::max(smem_H<PREC, K>(), kMinSmem); }
template <int PREC, int K>
size_t sm_Ht() { return std::max(smem_Ht<PREC, K>(), kMinSmem); }

template <int PREC, int K>
cudaError_t prep_t() {
  cudaError_t e = cudaFuncSetAttribute(tc_H_kernel<PREC, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm_H<PREC, K>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tc_Ht_kernel<PREC, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sm_Ht<PREC, K>());
}

template <int PREC, int K>
cudaError_t launch_t(const OpArgs& a, cudaStream_t s, bool adjoint) {
  if (adjoint)
    tc_Ht_kernel<PREC, K><<<a.n_work, NTH, sm_Ht<PREC, K>(), s>>>(a);
  else
    tc_H_kernel<PREC, K><<<a.n_work, NTH, sm_H<PREC, K>(), s>>>(a);
  return cudaGetLastError();
}

template <int PREC>
cudaError_t dispatch(const OpArgs& a, cudaStream_t s, bool adjoint) {
  switch (a.K) {
    case 9: return launch_t<PREC, 9>(a, s, adjoint);
    case 15: return launch_t<PREC, 15>(a, s, adjoint);
    case 31: return launch_t<PREC, 31>(a, s, adjoint);
    case 63: return launch_t<PREC, 63>(a, s, adjoint);
    default: return cudaErrorInvalidValue;
  }
}

template <int PREC>
cudaError_t prep_prec(int K) {
  switch (K) {
    case 9: return prep_t<PREC, 9>();
    case 15: return prep_t<PREC, 15>();
    case 31: return prep_t<PREC, 31>();
    case 63: return prep_t<PREC, 63>();
    default: return cudaErrorInvalidValue;
  }
}

uint16_t to_bf16(float f) {
  // round to nearest even on the IEEE single-precision bit pattern
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);   // inf / nan
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

uint32_t to_tf32(float f) {
  // round to nearest, ties away from zero, keeping 10 mantissa bits
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return u & 0xffffe000u;
  u += 0x1000u;
  return u & 0xffffe000u;
}

}  // namespace

int tc_block_m() { return BM; }
int tc_block_n() { return BN; }
bool tc_supported(int K) { return K == 9 || K == 15 || K == 31 || K == 63; }

cudaError_t tc_prepare(int K, int prec) {
  return prec == DV_PREC_TF32 ? prep_prec<1>(K) : prep_prec<0>(K);
}

// B operands of every PSF and tap row a: the nonzero windows of the two
// panels (K chunks 0 and 1) of the tall matrix Bt[n'][k] = f(a, k + KM (KS - 1)
// - n') (f = flipped PSF for H, the PSF for H^T), rows S0 .. S0 + WR - 1 of
// panel 0 then rows S0 + CH .. S0 + CH + WR - 1 of panel 1, 16 bytes per row,
// exactly as the kernels copy them into their ring stages.
void tc_operands(const float* psfs, int G, int K, int prec, bool flip, std::vector<uint8_t>& out) {
  const bool tf = prec == DV_PREC_TF32;
  const int bytes = tf ? 4 : 2, km = 32 / bytes, ch = 16 / bytes;
  const int KS = (BN - 1 + K + km - 1) / km;
  const int WR = K + ch - 1, S0 = km * (KS - 1) - K + 1;
  const size_t per_row = (size_t)2 * WR * 16;
  out.assign((size_t)G * K * per_row, 0);
  for (int p = 0; p < G; ++p) {
    const float* h = psfs + (size_t)p * K * K;
    for (int a = 0; a < K; ++a) {
      uint8_t* dst = out.data() + ((size_t)p * K + a) * per_row;
      for (int pn = 0; pn < 2; ++pn)
        for (int r = 0; r < WR; ++r) {
          const int n = S0 + pn * ch + r;
          for (int kk = 0; kk < ch; ++kk) {
            const int k = pn * ch + kk;
            const int d = k + km * (KS - 1) - n;
            float v = 0.f;
            if (d >= 0 && d < K) v = flip ? h[(K - 1 - a) * K + (K - 1 - d)] : h[a * K + d];
            uint8_t* e = dst + (size_t)pn * WR * 16 + (size_t)r * 16 + (size_t)kk * bytes;
            if (tf) {
              const uint32_t t = to_tf32(v);
              std::memcpy(e, &t, 4);
            } else {
              const uint16_t t = to_bf16(v);
              std::memcpy(e, &t, 2);
            }
          }
        }
    }
  }
}

cudaError_t launch_tc_H(const OpArgs& a, cudaStream_t s) {
  if (a.n_work <= 0) return cudaSuccess;
  return a.prec == DV_PREC_TF32 ? dispatch<1>(a, s, false) : dispatch<0>(a, s, false);
}

cudaError_t launch_tc_Ht(const OpArgs& a, cudaStream_t s) {
  if (a.n_work <= 0) return cudaSuccess;
  return a.prec == DV_PREC_TF32 ? dispatch<1>(a, s, true) : dispatch<0>(a, s, true);
}

}  // namespace dv
