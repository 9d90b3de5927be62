// BF16 tensor-core (tcgen05) kernels of the shift-variant operator of
// Sec. II-B and its adjoint in the column-band layout: a CTA owns 128 output
// columns (the MMA M dimension, one tensor-memory lane each) and up to NR
// output rows (the MMA N dimension, up to 256).  One tcgen05.mma costs about
// the same time for every N up to 256 at M = 128, so the output rows ride on
// N and the banded Toeplitz factor, whose extent is set by M, is kept narrow:
//     D[j][i] += sum_c T_a[j][c] S[i + a][c],   T_a[j][c] = f(a, c - j), 0 <= c - j < K,
// for tap row a of PSF f (flipped for H), output column j, output row i, and
// S the staged input block.  Per tap row, KS = ceil((127 + K) / 16) k-steps:
//   A = T_a on columns [16 ks, 16 ks + 16): a 128-row window of one "tall"
//       matrix At[j'][k] = f(a, k + 16 (KS - 1) - j'), two 16-byte panels of
//       (128 + 16 (KS - 1)) rows of which K + 7 are nonzero; those windows are
//       precomputed per PSF and tap row and streamed by cp.async.bulk into a
//       ring of stages (zero elsewhere) guarded by mbarriers;
//   B = rows i + a of S, the same columns: shared memory, K-major, no
//       swizzle, rows 16 bytes apart in each column panel, so the row shift a
//       is the start address plus 16 a.
//   H:   S = bf16(w_p . x), built per PSF from x in global memory (L2) into
//        one of two S buffers while the MMAs of the previous PSF read the
//        other; all PSFs accumulate into one accumulator in tensor memory.
//   H^T: S = bf16(r) staged once; PSF p accumulates into D, and the epilogue
//        warps add w_p . D into a second tensor-memory region G; the
//        projected-gradient step is fused into the write-out.
// Warps 0-7 stage operands and run the epilogue (warp w owns output columns
// 32 (w % 4) .. + 31 = its tensor-memory lanes, and rows 16 (w / 4) .. + 15 of
// every 32-row chunk of the accumulator), warp 8 allocates tensor memory and
// one of its lanes issues the MMAs, one lane of warp 9 refills the ring.
// Every wait is bounded (see dv_tcgen05.cuh), by OpArgs.wait_ns when set.
#include <algorithm>
#include <climits>
#include <cstring>

#include "dv_internal.cuh"
#include "dv_tcgen05.cuh"

namespace dv {
namespace {

using namespace tcg;

constexpr int MC = 128;                   // output columns per CTA (MMA M)
constexpr int KM = 16, CH = 8;            // BF16: K per MMA, elements per 16-byte chunk
constexpr int NWE = 8;                    // staging / epilogue warps
constexpr int NT = 32 * NWE;
constexpr int NTH = 32 * (NWE + 2);       // + the MMA warp and the bulk-copy warp
constexpr int kMaxNST = 8;                // ring stages (one tap row each), at most
constexpr int TP = MC + 1;                // fp32 transposition tile pitch (floats)
constexpr int HW = MC + 2;                // halo tile pitch (floats)
constexpr int kHdr = 512;
constexpr int kMaxB = kTcMaxB;            // PSF grid columns with a k-step range of their own
constexpr int kSmemMax = 227 * 1024;

template <int K>
struct GeoT {
  static constexpr int NST = 4;                           // ring stages (one tap row each)
  static constexpr int KS = (MC - 1 + K + KM - 1) / KM;   // MMAs per tap row
  static constexpr int COLS = KS * KM;                    // staged input columns
  static constexpr int NCH = COLS / CH;                   // 16-byte column panels of S
  // output rows per CTA: the MMA N dimension at its maximum, 256 (an MMA with
  // N = 128 takes about as long as one with N = 256)
  static constexpr int NR = 256;
  static constexpr int ROWS = NR + K - 1;                 // staged input rows
  static constexpr int SPANEL = ROWS * 16 + 16;
  static constexpr int SBYTES = NCH * SPANEL;
  // H: S buffers.  Two let the next PSF's S be built while the current PSF's
  // MMAs run; for K = 63 two buffers of 256 + 62 rows do not fit next to the
  // ring, so one buffer is rebuilt after each PSF's MMAs
  static constexpr int DBUF = K <= 31 ? 2 : 1;
  static constexpr int RA = MC + KM * (KS - 1);           // rows of the tall Toeplitz operand
  static constexpr int APANEL = RA * 16;
  static constexpr int ABYTES = 2 * APANEL;               // one ring stage
  static constexpr int WR = K + CH - 1;                   // nonzero rows per panel
  static constexpr int S0 = KM * (KS - 1) - K + 1;        // first nonzero row of panel 0
  static constexpr int WTX = 2 * WR * 16;                 // bytes streamed per tap row
  // H^T: fp32 staging / epilogue tiles
  static constexpr int UBYTES = K <= 31 ? 64 * 1024 : 48 * 1024;
  static constexpr int WCOFF = (ROWS + 3) / 4 * 4;        // H: sWc after sWr, 16-byte aligned
  static constexpr int SMEM_H = kHdr + DBUF * SBYTES + NST * ABYTES + (WCOFF + COLS) * 4;
  // H^T: [... | row weights of two PSF grid rows [2][NR] | omega rows [NR] | omega columns [MC]]
  static constexpr int SMEM_HT = kHdr + SBYTES + UBYTES + NST * ABYTES + 2 * NR * 4 +
                                 (NR + MC) * 4;
  // H epilogue with one S buffer: transposition tile, then the observed image
  // and noise weights of two 32-row chunks
  static constexpr int TOFF = (32 * TP * 4 + 15) / 16 * 16;
  static constexpr int TMEM_H = NR;
  static constexpr int TMEM_HT = 2 * NR;                  // accumulator D and sum G
  static_assert(S0 >= 0 && S0 + CH + WR <= RA, "Toeplitz windows inside the panels");
  static_assert(NST <= kMaxNST, "ring barriers");
  static_assert(SMEM_H <= kSmemMax && SMEM_HT <= kSmemMax, "shared memory");
  static_assert(SBYTES >= 32 * TP * 4 && UBYTES >= 32 * TP * 4 + 34 * HW * 4, "epilogue tiles");
  static_assert(UBYTES >= (COLS + 4) * 4 && SBYTES >= (COLS + 4) * 4, "staging chunk");
  static_assert(SBYTES >= 4 * 32 * MC * 4 + (DBUF == 1 ? TOFF : 0),
                "H epilogue prefetch buffers in an S buffer");
  // 16-byte alignment of every region accessed with 16-byte vectors or bulk copies
  static_assert(SPANEL % 16 == 0 && SBYTES % 16 == 0 && APANEL % 16 == 0 &&
                    (COLS * 2) % 16 == 0 && (COLS * 4) % 16 == 0 && (WCOFF * 4) % 16 == 0 &&
                    (S0 * 16) % 16 == 0 && UBYTES % 16 == 0 && kHdr % 16 == 0,
                "alignment");
};

struct Bars {
  uint64_t rfull[kMaxNST], rempty[kMaxNST];
  uint64_t sfull[2], sempty[2];  // S buffer staged / consumed (H: per PSF, H^T: buffer 0 once)
  uint64_t dfull[2], dempty[2];  // accumulator buffer complete / read (H: buffer 0 only)
  uint64_t fin;
  uint64_t wait_ns;           // bound of every pipeline wait of this launch
  uint32_t tmem;
  int abort;
  int ksr[kMaxB];             // k-step range of PSF grid column b_lo + b: lo | hi << 8
};
static_assert(sizeof(Bars) <= kHdr, "barrier header");

__device__ __forceinline__ void sync_stage() { named_sync<NT>(); }
__device__ __forceinline__ bool all_stage(bool v) { return named_all<NT>(v); }

__device__ __forceinline__ void init_bars(Bars* H, uint64_t wait_ns) {
  for (int s = 0; s < kMaxNST; ++s) {
    mbar_init(&H->rfull[s], 1);
    mbar_init(&H->rempty[s], 1);
  }
  for (int b = 0; b < 2; ++b) {
    mbar_init(&H->sfull[b], NT);
    mbar_init(&H->sempty[b], 1);
  }
  for (int b = 0; b < 2; ++b) {
    mbar_init(&H->dfull[b], 1);
    mbar_init(&H->dempty[b], NT);
  }
  mbar_init(&H->fin, 1);
  H->abort = 0;
  H->wait_ns = wait_ns ? wait_ns : kWaitNs;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bulk-copy lane: the Toeplitz windows of every (PSF, tap row) of the block,
// in the order the MMA lane consumes them.
template <int K>
__device__ void producer(const OpArgs& A, const WorkItem& wi, Bars* H, unsigned char* ring, int np) {
  using G = GeoT<K>;
  // test of the bounded waits (dv_plan_set_test_fault): no copy is issued, so
  // the MMA lane's first wait on the ring runs out with nothing in flight
  if (A.test_withhold) return;
  const int nb = wi.b_hi - wi.b_lo + 1;
  const int total = np * K;
  int issued = 0;
  for (int it = 0; it < total; ++it) {
    const int s = it % G::NST;
    if (it >= G::NST &&
        !wait_bar(&H->rempty[s], (uint32_t)((it / G::NST - 1) & 1), &H->abort, A.err, H->wait_ns))
      break;
    const int p = it / K, a = it - p * K;
    const int ga = wi.a_lo + p / nb, gb = wi.b_lo + p % nb;
    const unsigned char* src = A.tcop + ((size_t)(ga * A.Gc + gb) * K + a) * G::WTX;
    unsigned char* dst = ring + (size_t)s * G::ABYTES;
    mbar_expect_tx(&H->rfull[s], G::WTX);
    bulk_g2s(dst + G::S0 * 16, src, G::WR * 16, &H->rfull[s]);
    bulk_g2s(dst + G::APANEL + (G::S0 + CH) * 16, src + G::WR * 16, G::WR * 16, &H->rfull[s]);
    issued = it + 1;
  }
  for (int it = (issued > G::NST ? issued - G::NST : 0); it < issued; ++it)
    if (!drain_bar(&H->rfull[it % G::NST], (uint32_t)((it / G::NST) & 1), A.err)) break;
}

// K-step ranges of the block's PSF grid columns (computed on the host by
// tcT_kstep_ranges), copied into the barrier header by warp NWE.
__device__ __forceinline__ void load_ranges(const OpArgs& A, Bars* H, int lane) {
  if (lane < kMaxB) H->ksr[lane] = A.ksr[(size_t)blockIdx.x * kMaxB + lane];
  __syncwarp();
}

// One tap row: N k-steps from the start descriptors, as a straight run of
// MMAs with constant descriptor offsets (a runtime loop or a branch per MMA
// issues noticeably slower than the tensor pipe retires them).
template <int N, int SB>
__device__ __forceinline__ void issue_row(uint32_t d, uint64_t ad, uint64_t bd, uint32_t id,
                                          uint32_t acc) {
  mma_bf16(d, ad, bd, id, acc);
#pragma unroll
  for (int i = 1; i < N; ++i) mma_bf16(d, ad - (uint64_t)(i * KM), bd + (uint64_t)(i * SB), id, 1u);
}

template <int N, int SB>
__device__ __forceinline__ void issue_n(int n, uint32_t d, uint64_t ad, uint64_t bd, uint32_t id,
                                        uint32_t acc) {
  if (n == N) {
    issue_row<N, SB>(d, ad, bd, id, acc);
  } else if constexpr (N > 1) {
    issue_n<N - 1, SB>(n, d, ad, bd, id, acc);
  }
}

// MMA lane.  H (ADJ = false): every PSF accumulates into D once its S is
// staged, and S is released after its MMAs.  H^T: S is staged once; PSF p
// overwrites D once the epilogue has folded PSF p - 1 into G.
template <int K, bool ADJ>
__device__ void issuer(const OpArgs& A, const WorkItem& wi, Bars* H, unsigned char* sS,
                       unsigned char* ring, uint32_t d, int np, int nrow) {
  using G = GeoT<K>;
  const uint32_t id = idesc(1, MC, nrow);
  const uint64_t ad0 = sdesc(saddr(ring) + 16u * KM * (G::KS - 1), G::APANEL);
  const int nb = wi.b_hi - wi.b_lo + 1;
  int s = 0;
  uint32_t ph = 0;
  bool ok = true;
  bool fresh = true;   // the next MMA overwrites the accumulator
  for (int p = 0; p < np && ok; ++p) {
    if (ADJ) {
      ok = p == 0 ? wait_bar(&H->sfull[0], 0, &H->abort, A.err, H->wait_ns)
                  : wait_bar(&H->dempty[0], (uint32_t)((p - 1) & 1), &H->abort, A.err, H->wait_ns);
    } else if (G::DBUF == 2) {
      ok = wait_bar(&H->sfull[p & 1], (uint32_t)((p >> 1) & 1), &H->abort, A.err, H->wait_ns);
    } else {
      ok = wait_bar(&H->sfull[0], (uint32_t)(p & 1), &H->abort, A.err, H->wait_ns);
    }
    if (!ok) break;
    tc_fence_after();
    const uint32_t dp = d;
    const int b = p % nb;
    const int kr = b < kMaxB ? H->ksr[b] : (G::KS - 1) << 8;
    const int klo = kr & 0xff, nks = (kr >> 8) - klo + 1;
    const uint64_t adk = ad0 - (uint64_t)(klo * KM);
    const int sb = (ADJ || G::DBUF == 1) ? 0 : (p & 1);
    const uint64_t bdk = sdesc(saddr(sS + sb * G::SBYTES), G::SPANEL) +
                         (uint64_t)(2 * klo * (G::SPANEL >> 4));
    if (ADJ) fresh = true;
    for (int a = 0; a < K; ++a) {
      if (!wait_bar(&H->rfull[s], ph, &H->abort, A.err, H->wait_ns)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint64_t ad = adk + (uint64_t)(s * (G::ABYTES >> 4));
      const uint64_t bd = bdk + (uint64_t)a;
      issue_n<G::KS, 2 * (G::SPANEL >> 4)>(nks, dp, ad, bd, id, fresh ? 0u : 1u);
      fresh = false;
      tc_commit(&H->rempty[s]);
      if (++s == G::NST) {
        s = 0;
        ph ^= 1u;
      }
    }
    if (!ok) break;
    tc_commit(ADJ ? &H->dfull[0] : &H->sempty[sb]);
  }
  if (!ADJ && ok && np > 0) tc_commit(&H->dfull[0]);
  tc_commit(&H->fin);
  drain_bar(&H->fin, 0, A.err);
}

// Zeroes the rows of the ring stages outside the windows the copies fill.
template <int K>
__device__ __forceinline__ void zero_ring(unsigned char* ring, int tid) {
  using G = GeoT<K>;
  for (int e = tid; e < G::NST * 2 * G::RA; e += NT) {
    const int st = e / (2 * G::RA), rem = e - st * 2 * G::RA, pn = rem / G::RA, n = rem - pn * G::RA;
    const int w0 = G::S0 + pn * CH;
    if (n < w0 || n >= w0 + G::WR)
      *reinterpret_cast<uint4*>(ring + (size_t)st * G::ABYTES + pn * G::APANEL + n * 16) =
          make_uint4(0u, 0u, 0u, 0u);
  }
}

// Rows [r0, r0 + ROWS) x columns [c0, c0 + COLS) of a pitched FP32 image,
// zero outside [0, nr) x [0, nc) and at window columns >= cmax, in passes of
// `rows_per` rows through the FP32 staging buffer `stg` (row pitch COLS + 4).
// Each row is fetched from column c0 - sh, sh = c0 mod 4, in 16-byte copies
// where a copy lies inside the image (and the image rows are 16-byte
// aligned), element copies with zero fill elsewhere.  `sink(ir, ic, v8)`
// receives 8 consecutive values of window row ir starting at column ic.
template <int K, class Sink>
__device__ __forceinline__ void stream_window(float* stg, int rows_per, const float* img,
                                              int64_t pitch, int r0, int c0, int nr, int nc,
                                              int cmax, int tid, Sink sink) {
  using G = GeoT<K>;
  constexpr int SP = G::COLS + 4;
  constexpr int NQ = SP / 4;                     // 16-byte slots per staged row
  const bool al = (pitch & 3) == 0 && (reinterpret_cast<uintptr_t>(img) & 15) == 0;
  const int sh = al ? (c0 & 3) : 0;
  const int cs = c0 - sh;                        // global column of staged column 0
  for (int rb = 0; rb < G::ROWS; rb += rows_per) {
    const int nrows = min(rows_per, G::ROWS - rb);
    for (int e = tid; e < nrows * NQ; e += NT) {
      const int ir = e / NQ, m = e - ir * NQ;
      const int R = r0 + rb + ir, C = cs + 4 * m;
      float* dst = stg + ir * SP + 4 * m;
      const bool row_in = R >= 0 && R < nr;
      if (al && row_in && C >= 0 && C + 4 <= nc) {
        cp_async16(dst, img + (int64_t)R * pitch + C);
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const bool in = row_in && C + t >= 0 && C + t < nc;
          cp_async4(dst + t, in ? img + (int64_t)R * pitch + C + t : img, in);
        }
      }
    }
    cp_async_wait_all();
    sync_stage();
    for (int e = tid; e < nrows * G::NCH; e += NT) {
      const int ir = e / G::NCH, q = e - ir * G::NCH;
      const float* src = stg + ir * SP + q * CH + sh;
      float vals[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) vals[t] = (q * CH + t < cmax) ? src[t] : 0.f;
      sink(rb + ir, q * CH, vals);
    }
    sync_stage();
  }
}

template <int K>
__device__ __forceinline__ void put_s(unsigned char* sS, int ir, int q, const float* v) {
  using G = GeoT<K>;
  *reinterpret_cast<uint4*>(sS + (size_t)q * G::SPANEL + ir * 16) = pack_chunk<0>(v);
}

// H: S = bf16((w_r w_c) x) on window rows [0, ROWS) and the 8-column chunks
// [qlo, qlo + nq) the PSF's k-steps read, straight from the FP32 x tile
// (zero outside [0, nr) x [0, nc) and on rows of zero weight).  Loads are
// issued U items at a time (16-byte loads where the rows are aligned).
template <int K>
__device__ __forceinline__ void restage_h(unsigned char* sb, const float* __restrict__ img,
                                          int64_t pitch, bool al, int r0, int c0, int nr, int nc,
                                          const float* sWr, const float* sWc, int qlo, int nq,
                                          int tid) {
  using G = GeoT<K>;
  constexpr int U = 8;   // items (8 values each) in flight per thread
  const int total = G::ROWS * nq;
  for (int e0 = tid; e0 < total; e0 += U * NT) {
    float v[U][CH];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * NT;
#pragma unroll
      for (int t = 0; t < CH; ++t) v[u][t] = 0.f;
      if (e < total) {
        const int ir = e / nq, q = qlo + (e - ir * nq);
        const int R = r0 + ir, C = c0 + q * CH;
        if (R < nr && sWr[ir] != 0.f) {
          const float* src = img + (int64_t)R * pitch + C;
          if (al && C + CH <= nc) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(src));
            const float4 b = __ldg(reinterpret_cast<const float4*>(src) + 1);
            v[u][0] = a.x; v[u][1] = a.y; v[u][2] = a.z; v[u][3] = a.w;
            v[u][4] = b.x; v[u][5] = b.y; v[u][6] = b.z; v[u][7] = b.w;
          } else {
#pragma unroll
            for (int t = 0; t < CH; ++t)
              if (C + t < nc) v[u][t] = __ldg(src + t);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * NT;
      if (e < total) {
        const int ir = e / nq, q = qlo + (e - ir * nq);
        const float rw = sWr[ir];
        const float4 w0 = *reinterpret_cast<const float4*>(sWc + q * CH);
        const float4 w1 = *reinterpret_cast<const float4*>(sWc + q * CH + 4);
        const float cw[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        float o[8];
#pragma unroll
        for (int t = 0; t < CH; ++t) o[t] = rw * cw[t] * v[u][t];
        put_s<K>(sb, ir, q, o);
      }
    }
  }
}

// ------------------------------------------------------------------ H kernel
template <int K>
__global__ void __launch_bounds__(NTH, 1) tcT_H_kernel(const OpArgs A) {
  using G = GeoT<K>;
  extern __shared__ __align__(1024) unsigned char smem[];
  Bars* H = reinterpret_cast<Bars*>(smem);
  unsigned char* sS = smem + kHdr;                                        // [DBUF][SBYTES]
  unsigned char* ring = sS + G::DBUF * G::SBYTES;
  float* sWr = reinterpret_cast<float*>(ring + (size_t)G::NST * G::ABYTES);   // [ROWS]
  float* sWc = sWr + G::WCOFF;                                            // [COLS]
  __shared__ double red[NWE];
  const WorkItem wi = A.work[blockIdx.x];
  const TileDesc td = A.tiles[wi.tile];
  const int nrow = wi.pad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) init_bars(H, A.wait_ns);
  if (warp == NWE) {
    tmem_alloc(&H->tmem, G::TMEM_H);
    load_ranges(A, H, lane);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = H->tmem;
  const int nb = wi.b_hi - wi.b_lo + 1;
  const int np = (wi.a_hi - wi.a_lo + 1) * nb;

  if (warp == NWE) {
    if (lane == 0) issuer<K, false>(A, wi, H, sS, ring, tbase, np, nrow);
    __syncwarp();
  } else if (warp == NWE + 1) {
    if (lane == 0) producer<K>(A, wi, H, ring, np);
    __syncwarp();
  } else {
    zero_ring<K>(ring, tid);
    const float* img = A.in + td.xoff;
    const bool al = (td.xpitch & 3) == 0 && (reinterpret_cast<uintptr_t>(img) & 15) == 0;
    bool ok = true;
    for (int p = 0; p < np && ok; ++p) {
      const int ga = wi.a_lo + p / nb, b = p % nb, gb = wi.b_lo + b;
      const int kr = b < kMaxB ? H->ksr[b] : (G::KS - 1) << 8;
      const int qlo = 2 * (kr & 0xff), nq = 2 * ((kr >> 8) - (kr & 0xff) + 1);
      sync_stage();   // the previous PSF's weights are no longer read
      for (int e = tid; e < G::ROWS; e += NT) {
        const int R = wi.r0 + e;
        sWr[e] = R < td.nxr ? wsel(A.wrow[td.wr0 + R], ga) : 0.f;
      }
      for (int e = tid; e < G::COLS; e += NT) {
        const int C = wi.c0 + e;
        sWc[e] = C < td.nxc ? wsel(A.wcol[td.wc0 + C], gb) : 0.f;
      }
      sync_stage();
      // two buffers: S buffer p & 1 was last read by PSF p - 2; one buffer:
      // by PSF p - 1
      const int sb = G::DBUF == 2 ? (p & 1) : 0;
      if (G::DBUF == 2 && p >= 2) {
        ok = all_stage(wait_bar(&H->sempty[sb], (uint32_t)(((p >> 1) - 1) & 1), &H->abort, A.err,
                                H->wait_ns));
        if (!ok) break;
      } else if (G::DBUF == 1 && p >= 1) {
        ok = all_stage(wait_bar(&H->sempty[0], (uint32_t)((p - 1) & 1), &H->abort, A.err,
                                H->wait_ns));
        if (!ok) break;
      }
      restage_h<K>(sS + sb * G::SBYTES, img, td.xpitch, al, wi.r0, wi.c0, td.nxr, td.nxc, sWr,
                   sWc, qlo, nq, tid);
      fence_async_smem();
      mbar_arrive(&H->sfull[sb]);
    }
    // epilogue: 32-row chunks of the accumulator, transposed through the S
    // buffer of the last PSF (free once every MMA has completed).  The
    // observed image (and noise weights) of chunk c + 1 are copied into the
    // other S buffer by cp.async while chunk c is written; chunk 0's copy
    // overlaps the last PSF's MMAs.
    constexpr int PER = 32 * MC / NT;    // outputs per thread and chunk
    const bool obs = A.mode != OP_PLAIN;
    if (G::DBUF == 2 && ok && np >= 2)   // the other buffer was last read by PSF np - 2
      ok = all_stage(wait_bar(&H->sempty[np & 1], (uint32_t)(((np - 2) >> 1) & 1), &H->abort,
                              A.err, H->wait_ns));
    // two buffers: the prefetch goes to the buffer the last PSF did not read
    // and the transposition to the other; one buffer: both share it, after
    // every MMA has completed
    float* sYb = reinterpret_cast<float*>(G::DBUF == 2 ? sS + (np & 1) * G::SBYTES
                                                       : sS + G::TOFF);   // [2][32 * MC] observed image
    float* sWb = sYb + 2 * 32 * MC;                      // [2][32 * MC] noise weights
    auto prefetch = [&](int i0, int buf) {
      if (obs) {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int e = tid + u * NT, il = e / MC, jl = e - il * MC;
          const int i = wi.r0 + i0 + il, jj = wi.c0 + jl;
          const bool in = i0 + il < nrow && i < td.nyr && jj < td.nyc;
          const int64_t gi = (int64_t)(td.xr0 + i) * A.wy + (td.xc0 + jj);
          cp_async4(sYb + buf * 32 * MC + e, in ? A.y + gi : A.y, in);
          if (A.W) cp_async4(sWb + buf * 32 * MC + e, in ? A.W + gi : A.W, in);
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (G::DBUF == 2 && ok && np > 0) prefetch(0, 0);
    if (ok && np > 0) ok = all_stage(wait_bar(&H->dfull[0], 0, &H->abort, A.err, H->wait_ns));
    if (ok && (np == 0 || G::DBUF == 1)) prefetch(0, 0);
    tc_fence_after();
    sync_stage();
    float* sT = reinterpret_cast<float*>(G::DBUF == 2 ? sS + ((np + 1) & 1) * G::SBYTES : sS);
    const int j = 32 * (warp & 3) + lane, hf = warp >> 2;
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    double part = 0.0;
    for (int i0 = 0, c = 0; i0 < nrow && ok; i0 += 32, ++c) {
      if (i0 + 32 < nrow) prefetch(i0 + 32, (c + 1) & 1);
      else asm volatile("cp.async.commit_group;" ::: "memory");
      uint32_t v[16];
      if (np > 0) {
        tmem_ld16_nowait(tbase + lanes + (uint32_t)(i0 + 16 * hf), v);
        tmem_wait_ld();
      } else {
#pragma unroll
        for (int t = 0; t < 16; ++t) v[t] = 0u;
      }
#pragma unroll
      for (int t = 0; t < 16; ++t) sT[(16 * hf + t) * TP + j] = __uint_as_float(v[t]);
      asm volatile("cp.async.wait_group 1;" ::: "memory");   // chunk c has landed
      sync_stage();
      const float* yb = sYb + (c & 1) * 32 * MC;
      const float* wb = sWb + (c & 1) * 32 * MC;
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + u * NT, il = e / MC, jl = e - il * MC;
        const int i = wi.r0 + i0 + il, jj = wi.c0 + jl;
        if (i0 + il >= nrow || i >= td.nyr || jj >= td.nyc) continue;
        const float y = sT[il * TP + jl];
        if (!obs) {
          A.out[td.yoff + (int64_t)i * td.ypitch + jj] = y;
        } else {
          const float dd = y - yb[e];
          const float wt = A.W ? wb[e] : 1.f;
          if (A.mode == OP_RESID)
            A.out[td.yoff + (int64_t)i * td.ypitch + jj] = wt * dd;
          else
            part += (double)wt * (double)dd * (double)dd;
        }
      }
      sync_stage();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (A.mode == OP_OBJ) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
      if (lane == 0) red[warp] = part;
      sync_stage();
      if (tid == 0) {
        double t = 0.0;
        for (int w2 = 0; w2 < NWE; ++w2) t += red[w2];
        A.partials[blockIdx.x] = t;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == NWE) {
    tc_fence_after();
    tmem_free(tbase, G::TMEM_H);
  }
}

// ---------------------------------------------------------------- H^T kernel
template <int K>
__global__ void __launch_bounds__(NTH, 1) tcT_Ht_kernel(const OpArgs A) {
  using G = GeoT<K>;
  extern __shared__ __align__(1024) unsigned char smem[];
  Bars* H = reinterpret_cast<Bars*>(smem);
  unsigned char* sS = smem + kHdr;
  float* sU = reinterpret_cast<float*>(sS + G::SBYTES);                 // staging / epilogue
  unsigned char* ring = reinterpret_cast<unsigned char*>(sU) + G::UBYTES;
  float* sWr = reinterpret_cast<float*>(ring + (size_t)G::NST * G::ABYTES); // [2][NR]
  float* sOr = sWr + 2 * G::NR;                                          // gamma omega rows [NR]
  float* sOc = sOr + G::NR;                                              // omega columns [MC]
  const WorkItem wi = A.work[blockIdx.x];
  const TileDesc td = A.tiles[wi.tile];
  const int nrow = wi.pad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) init_bars(H, A.wait_ns);
  if (warp == NWE) {
    tmem_alloc(&H->tmem, G::TMEM_HT);
    load_ranges(A, H, lane);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = H->tmem;
  const int nb = wi.b_hi - wi.b_lo + 1;
  const int na = wi.a_hi - wi.a_lo + 1;
  const int np = na * nb;

  if (warp == NWE) {
    if (lane == 0) issuer<K, true>(A, wi, H, sS, ring, tbase, np, nrow);
    __syncwarp();
  } else if (warp == NWE + 1) {
    if (lane == 0) producer<K>(A, wi, H, ring, np);
    __syncwarp();
  } else {
    zero_ring<K>(ring, tid);
    // residual rows R0 - (K-1) .., columns C0 - (K-1) ..: zero outside the
    // y-block and past the 127 + K columns a block reads
    stream_window<K>(sU, G::UBYTES / ((G::COLS + 4) * 4), A.in + td.yoff, td.ypitch, wi.r0 - (K - 1),
                     wi.c0 - (K - 1), td.nyr, td.nyc, MC - 1 + K, tid,
                     [&](int ir, int ic, const float* v) { put_s<K>(sS, ir, ic / CH, v); });
    if (A.mode != OP_PLAIN) {   // consensus profiles of the step epilogue
      for (int e = tid; e < G::NR; e += NT) {
        const int R = wi.r0 + e;
        sOr[e] = R < td.nxr ? A.gamma * A.omr[td.omr_off + R] : 0.f;
      }
      for (int e = tid; e < MC; e += NT) {
        const int Cc = wi.c0 + e;
        sOc[e] = Cc < td.nxc ? A.omc[td.omc_off + Cc] : 0.f;
      }
    }
    fence_async_smem();
    mbar_arrive(&H->sfull[0]);
    sync_stage();

    float* sT = sU;                      // [32][TP]
    float* sH = sU + 32 * TP;            // [34][HW] halo of the iterate
    constexpr int PER = 32 * MC / NT;    // outputs per thread and chunk
    const bool step = A.mode != OP_PLAIN;
    // OP_STEP splits w_next = max(0, w - tau (g + lambda D^T psi(D w) + alpha (w - u)))
    // into q = w - tau (lambda D^T psi(D w) + alpha (w - u)), which does not
    // need g and is computed into the output while the MMAs run, and the
    // final max(0, q - tau g).
    auto q_chunk = [&](int i0) {
      for (int e = tid; e < 34 * HW; e += NT) {
        const int ir = e / HW, ic = e - ir * HW;
        const int Rr = wi.r0 + i0 - 1 + ir, Cc = wi.c0 - 1 + ic;
        const bool in = Rr >= 0 && Rr < td.nxr && Cc >= 0 && Cc < td.nxc;
        cp_async4(sH + e, in ? A.w + td.xoff + (int64_t)Rr * td.xpitch + Cc : A.w, in);
      }
      float uv[PER];
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + u * NT, il = e / MC, jl = e - il * MC;
        const int Ro = wi.r0 + i0 + il, Co = wi.c0 + jl;
        uv[u] = (i0 + il < nrow && Ro < td.nxr && Co < td.nxc)
                    ? __ldg(A.u + td.xoff + (int64_t)Ro * td.xpitch + Co)
                    : 0.f;
      }
      cp_async_wait_all();
      sync_stage();
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + u * NT, il = e / MC, jl = e - il * MC;
        const int Ro = wi.r0 + i0 + il, Co = wi.c0 + jl;
        if (i0 + il >= nrow || Ro >= td.nxr || Co >= td.nxc) continue;
        const int li = il + 1, lj = jl + 1;
        float pr, pc, pru, pcu, prl, pcl;
        huber_p(sH, HW, li, lj, Ro, Co, td.nxr, td.nxc, A.delta, pr, pc);
        huber_p(sH, HW, li - 1, lj, Ro - 1, Co, td.nxr, td.nxc, A.delta, pru, pcu);
        huber_p(sH, HW, li, lj - 1, Ro, Co - 1, td.nxr, td.nxc, A.delta, prl, pcl);
        const float hub = pru - pr + pcl - pc;
        const float wv = sH[li * HW + lj];
        const float alpha = sOr[i0 + il] * sOc[jl];
        A.out[td.xoff + (int64_t)Ro * td.xpitch + Co] =
            wv - td.tau * (A.lambda * hub + alpha * (wv - uv[u]));
      }
      sync_stage();
    };
    const int nck = (nrow + 31) / 32;
    const int qper = np > 0 ? (nck + np - 1) / np : nck;   // q chunks per PSF interval
    int qc = 0;

    // G (tensor-memory columns NR ..) = sum_p w_p . D_p; each warp covers 16
    // rows of every 32-row chunk for its 32 columns, D and G loaded together
    const int j = 32 * (warp & 3) + lane, hf = warp >> 2;
    const int C = wi.c0 + j;
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    bool ok = true;
    for (int p = 0; p < np; ++p) {
      const int ai = p / nb, gb = wi.b_lo + p % nb;
      // column weight of the PSF and, for the first PSF of a grid row, the
      // row weights (buffer ai & 1: the fold of the previous grid row reads
      // the other one), fetched while its MMAs run
      const float wc = C < td.nxc ? wsel(A.wcol[td.wc0 + C], gb) : 0.f;
      float* wrow = sWr + (ai & 1) * G::NR;
      if (p % nb == 0)
        for (int e = tid; e < G::NR; e += NT) {
          const int R = wi.r0 + e;
          wrow[e] = R < td.nxr ? wsel(A.wrow[td.wr0 + R], wi.a_lo + ai) : 0.f;
        }
      if (step)
        for (int k = 0; k < qper && qc < nck; ++k) q_chunk(32 * qc++);
      if (!all_stage(wait_bar(&H->dfull[0], (uint32_t)(p & 1), &H->abort, A.err, H->wait_ns))) {
        ok = false;
        break;
      }
      tc_fence_after();
      // software-pipelined: the loads of the next 16 rows are issued before
      // the sums of the current ones are stored
      uint32_t dv[16], gv[16];
      if (16 * hf < nrow) {
        tmem_ld16_nowait(tbase + lanes + (uint32_t)(16 * hf), dv);
        if (p > 0) tmem_ld16_nowait(tbase + lanes + (uint32_t)(G::NR + 16 * hf), gv);
      }
      for (int i0 = 16 * hf; i0 < nrow; i0 += 32) {
        tmem_wait_ld();
        uint32_t ov[16];
        float wr[16];
#pragma unroll
        for (int t = 0; t < 16; t += 4) {
          const float4 w4 = *reinterpret_cast<const float4*>(wrow + i0 + t);
          wr[t] = w4.x;
          wr[t + 1] = w4.y;
          wr[t + 2] = w4.z;
          wr[t + 3] = w4.w;
        }
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const float dd = __uint_as_float(dv[t]);
          ov[t] = __float_as_uint(p > 0 ? fmaf(wr[t] * wc, dd, __uint_as_float(gv[t])) : wr[t] * wc * dd);
        }
        if (i0 + 32 < nrow) {
          tmem_ld16_nowait(tbase + lanes + (uint32_t)(i0 + 32), dv);
          if (p > 0) tmem_ld16_nowait(tbase + lanes + (uint32_t)(G::NR + i0 + 32), gv);
        }
        tmem_st16_nowait(tbase + lanes + (uint32_t)(G::NR + i0), ov);
      }
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&H->dempty[0]);
    }
    if (step && ok)
      while (qc < nck) q_chunk(32 * qc++);
    // final pass: g out of tensor memory (transposed through shared memory)
    for (int i0 = 0; i0 < nrow && ok; i0 += 32) {
      uint32_t gv[16];
      if (np > 0) {
        tmem_ld16_nowait(tbase + lanes + (uint32_t)(G::NR + i0 + 16 * hf), gv);
        tmem_wait_ld();
      } else {
#pragma unroll
        for (int t = 0; t < 16; ++t) gv[t] = 0u;
      }
#pragma unroll
      for (int t = 0; t < 16; ++t) sT[(16 * hf + t) * TP + j] = __uint_as_float(gv[t]);
      sync_stage();
      if (!step) {
        for (int e = tid; e < 32 * MC; e += NT) {
          const int il = e / MC, jl = e - il * MC;
          const int Ro = wi.r0 + i0 + il, Co = wi.c0 + jl;
          if (i0 + il < nrow && Ro < td.nxr && Co < td.nxc)
            A.out[td.xoff + (int64_t)Ro * td.xpitch + Co] = sT[il * TP + jl];
        }
      } else {
        float qv[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int e = tid + u * NT, il = e / MC, jl = e - il * MC;
          const int Ro = wi.r0 + i0 + il, Co = wi.c0 + jl;
          qv[u] = (i0 + il < nrow && Ro < td.nxr && Co < td.nxc)
                      ? A.out[td.xoff + (int64_t)Ro * td.xpitch + Co]
                      : 0.f;
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int e = tid + u * NT, il = e / MC, jl = e - il * MC;
          const int Ro = wi.r0 + i0 + il, Co = wi.c0 + jl;
          if (i0 + il < nrow && Ro < td.nxr && Co < td.nxc)
            A.out[td.xoff + (int64_t)Ro * td.xpitch + Co] =
                fmaxf(0.f, qv[u] - td.tau * sT[il * TP + jl]);
        }
      }
      sync_stage();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == NWE) {
    tc_fence_after();
    tmem_free(tbase, G::TMEM_HT);
  }
}

template <int K>
cudaError_t prep_t() {
  cudaError_t e = cudaFuncSetAttribute(tcT_H_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       GeoT<K>::SMEM_H);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tcT_Ht_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              GeoT<K>::SMEM_HT);
}

template <int K>
cudaError_t launch_t(const OpArgs& a, cudaStream_t s, bool adjoint) {
  if (adjoint)
    tcT_Ht_kernel<K><<<a.n_work, NTH, GeoT<K>::SMEM_HT, s>>>(a);
  else
    tcT_H_kernel<K><<<a.n_work, NTH, GeoT<K>::SMEM_H, s>>>(a);
  return cudaGetLastError();
}

cudaError_t dispatch(const OpArgs& a, cudaStream_t s, bool adjoint) {
  switch (a.K) {
    case 9: return launch_t<9>(a, s, adjoint);
    case 15: return launch_t<15>(a, s, adjoint);
    case 31: return launch_t<31>(a, s, adjoint);
    case 63: return launch_t<63>(a, s, adjoint);
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

}  // namespace

int tcT_block_cols() { return MC; }
int tcT_max_rows(int K) { return K > 0 ? 256 : 0; }

// A k-step covers staged columns [16 ks, 16 ks + 16) and so reaches output
// columns 16 ks - K + 1 .. 16 ks + 15 of the block.  H: S = w_p . x is zero
// where the PSF's column weight is zero, so steps outside its support add
// zeros, and steps reaching no valid output column are not needed.  H^T: the
// weight multiplies the output, so only steps reaching an output column of
// nonzero weight count, and steps whose staged residual columns are all zero
// (outside the y tile) add nothing.  An empty range falls back to every step.
int64_t tcT_kstep_ranges(const std::vector<TileDesc>& tiles, const std::vector<WorkItem>& items,
                         const std::vector<WTab>& wcol, int K, bool adjoint,
                         std::vector<uint16_t>& out) {
  const int KS = (MC - 1 + K + KM - 1) / KM, COLS = KS * KM;
  out.assign(items.size() * kMaxB, (uint16_t)((KS - 1) << 8));
  int64_t steps = 0;
  for (size_t it = 0; it < items.size(); ++it) {
    const WorkItem& wi = items[it];
    const TileDesc& td = tiles[wi.tile];
    const int nb = wi.b_hi - wi.b_lo + 1, na = wi.a_hi - wi.a_lo + 1;
    const int ncv = std::min(MC, (adjoint ? td.nxc : td.nyc) - wi.c0);
    const int span = adjoint ? ncv : std::min(COLS, std::min(ncv + K - 1, td.nxc - wi.c0));
    for (int b = 0; b < nb; ++b) {
      int klo = 0, khi = KS - 1;
      if (b < kMaxB) {
        const int gb = wi.b_lo + b;
        int lo = INT_MAX, hi = -1;
        for (int c = 0; c < span; ++c)
          if (wsel(wcol[td.wc0 + wi.c0 + c], gb) != 0.f) {
            lo = std::min(lo, c);
            hi = std::max(hi, c);
          }
        if (hi >= 0) {
          if (adjoint) {
            // staged residual column c holds y column c0 - (K - 1) + c
            const int slo = std::max(0, K - 1 - wi.c0);
            const int shi = std::min(MC - 2 + K, td.nyc - 1 - wi.c0 + K - 1);
            const int wlo = lo / KM, whi = std::min(KS - 1, (hi + K - 1) / KM);
            const int l2 = std::max(wlo, slo / KM), h2 = std::min(whi, shi / KM);
            klo = l2 <= h2 ? l2 : wlo;
            khi = l2 <= h2 ? h2 : whi;
          } else {
            klo = lo / KM;
            khi = std::min(KS - 1, hi / KM);
          }
        }
        out[it * kMaxB + b] = (uint16_t)(klo | (khi << 8));
      }
      steps += (int64_t)na * (khi - klo + 1);
    }
  }
  return steps;
}

cudaError_t tcT_prepare(int K) {
  switch (K) {
    case 9: return prep_t<9>();
    case 15: return prep_t<15>();
    case 31: return prep_t<31>();
    case 63: return prep_t<63>();
    default: return cudaErrorInvalidValue;
  }
}

// Toeplitz operands of every PSF and tap row a: the nonzero windows of the
// two panels (K chunks 0 and 1) of At[j'][k] = f(a, k + 16 (KS - 1) - j')
// (f = flipped PSF for H, the PSF for H^T), rows S0 .. S0 + K + 6 of panel 0
// then rows S0 + 8 .. S0 + K + 14 of panel 1, 16 bytes (8 BF16) per row, as
// the kernels copy them into their ring stages.
void tcT_operands(const float* psfs, int G, int K, bool flip, std::vector<uint8_t>& out) {
  const int KS = (MC - 1 + K + KM - 1) / KM;
  const int WR = K + CH - 1, S0 = KM * (KS - 1) - K + 1;
  const size_t per_row = (size_t)2 * WR * 16;
  out.assign((size_t)G * K * per_row, 0);
  for (int p = 0; p < G; ++p) {
    const float* h = psfs + (size_t)p * K * K;
    for (int a = 0; a < K; ++a) {
      uint8_t* dst = out.data() + ((size_t)p * K + a) * per_row;
      for (int pn = 0; pn < 2; ++pn)
        for (int r = 0; r < WR; ++r) {
          const int n = S0 + pn * CH + r;
          for (int kk = 0; kk < CH; ++kk) {
            const int k = pn * CH + kk;
            const int d = k + KM * (KS - 1) - n;
            float v = 0.f;
            if (d >= 0 && d < K) v = flip ? h[(K - 1 - a) * K + (K - 1 - d)] : h[a * K + d];
            const uint16_t t = to_bf16(v);
            std::memcpy(dst + (size_t)pn * WR * 16 + (size_t)r * 16 + (size_t)kk * 2, &t, 2);
          }
        }
    }
  }
}

cudaError_t launch_tcT_H(const OpArgs& a, cudaStream_t s) {
  if (a.n_work <= 0) return cudaSuccess;
  return dispatch(a, s, false);
}

cudaError_t launch_tcT_Ht(const OpArgs& a, cudaStream_t s) {
  if (a.n_work <= 0) return cudaSuccess;
  return dispatch(a, s, true);
}

}  // namespace dv
