// Image quality against a reference, the measures of the paper's evaluation
// (Sec. IV-C): SNR = 10 log10(sum ref^2 / sum (x - ref)^2) over all pixels and
// the mean structural similarity (Wang, Bovik, Sheikh, Simoncelli 2004) over
// every 11 x 11 window inside the image:
//   SSIM = (2 mu_x mu_r + C1)(2 s_xr + C2) / ((mu_x^2 + mu_r^2 + C1)(s_x^2 + s_r^2 + C2)),
// local moments under the separable, unit-sum Gaussian window of standard
// deviation 1.5, C1 = (0.01 L)^2, C2 = (0.03 L)^2, L the dynamic range.
// One CTA per 16 x 32 block of window centres: the block's halo of both
// images in shared memory, the horizontal 11-tap pass of the five moments
// (x, r, x^2, r^2, x r) into shared memory, then the vertical pass and the
// SSIM per centre; FP64 partial sums per CTA, summed in a fixed order.
#include <cmath>

#include "dv_internal.cuh"

namespace dv {
namespace {

constexpr int QW = 32, QH = 16;            // window centres per CTA (columns, rows)
constexpr int QR = 5, QT = 2 * QR + 1;     // window radius and side
constexpr int HR = QH + 2 * QR, HC = QW + 2 * QR;
constexpr int QNT = 256;

struct QGauss {
  float g[QT];
};

__global__ void __launch_bounds__(QNT) quality_kernel(const float* __restrict__ x,
                                                      const float* __restrict__ ref, int rows,
                                                      int cols, QGauss G, float c1, float c2,
                                                      double* __restrict__ part) {
  __shared__ float sx[HR][HC + 1], sr[HR][HC + 1];
  __shared__ float sm[5][HR][QW + 1];
  __shared__ double red[3][QNT / 32];
  const int r0 = blockIdx.y * QH, c0 = blockIdx.x * QW;
  const int tid = threadIdx.x;
  double sig = 0.0, err = 0.0, ss = 0.0;
  for (int e = tid; e < HR * HC; e += QNT) {
    const int ir = e / HC, ic = e - ir * HC;
    const int R = r0 - QR + ir, C = c0 - QR + ic;
    const bool in = R >= 0 && R < rows && C >= 0 && C < cols;
    const float a = in ? x[(int64_t)R * cols + C] : 0.f;
    const float b = in ? ref[(int64_t)R * cols + C] : 0.f;
    sx[ir][ic] = a;
    sr[ir][ic] = b;
    // SNR sums over the pixels this CTA owns
    if (in && ir >= QR && ir < QR + QH && ic >= QR && ic < QR + QW) {
      const double d = (double)a - (double)b;
      sig += (double)b * (double)b;
      err += d * d;
    }
  }
  __syncthreads();
  for (int e = tid; e < HR * QW; e += QNT) {
    const int ir = e / QW, ic = e - ir * QW;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
    for (int k = 0; k < QT; ++k) {
      const float g = G.g[k], a = sx[ir][ic + k], b = sr[ir][ic + k];
      m0 = fmaf(g, a, m0);
      m1 = fmaf(g, b, m1);
      m2 = fmaf(g * a, a, m2);
      m3 = fmaf(g * b, b, m3);
      m4 = fmaf(g * a, b, m4);
    }
    sm[0][ir][ic] = m0;
    sm[1][ir][ic] = m1;
    sm[2][ir][ic] = m2;
    sm[3][ir][ic] = m3;
    sm[4][ir][ic] = m4;
  }
  __syncthreads();
  for (int e = tid; e < QH * QW; e += QNT) {
    const int il = e / QW, ic = e - il * QW;
    const int R = r0 + il, C = c0 + ic;
    if (R < QR || R >= rows - QR || C < QR || C >= cols - QR) continue;
    float mx = 0.f, mr = 0.f, exx = 0.f, err2 = 0.f, exr = 0.f;
#pragma unroll
    for (int k = 0; k < QT; ++k) {
      const float g = G.g[k];
      mx = fmaf(g, sm[0][il + k][ic], mx);
      mr = fmaf(g, sm[1][il + k][ic], mr);
      exx = fmaf(g, sm[2][il + k][ic], exx);
      err2 = fmaf(g, sm[3][il + k][ic], err2);
      exr = fmaf(g, sm[4][il + k][ic], exr);
    }
    const float vx = exx - mx * mx, vr = err2 - mr * mr, cxr = exr - mx * mr;
    ss += (double)(((2.f * mx * mr + c1) * (2.f * cxr + c2)) /
                   ((mx * mx + mr * mr + c1) * (vx + vr + c2)));
  }
  // block sums
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_down_sync(0xffffffffu, ss, o);
    sig += __shfl_down_sync(0xffffffffu, sig, o);
    err += __shfl_down_sync(0xffffffffu, err, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = ss;
    red[1][tid >> 5] = sig;
    red[2][tid >> 5] = err;
  }
  __syncthreads();
  if (tid < 3) {
    double t = 0.0;
    for (int w = 0; w < QNT / 32; ++w) t += red[tid][w];
    part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 3 + tid] = t;
  }
}

// Sums the n partials of each component in a fixed order; out[0] = SNR (dB),
// out[1] = mean SSIM over the nwin windows.
__global__ void __launch_bounds__(QNT) quality_sum_kernel(const double* __restrict__ part,
                                                          int64_t n, double nwin,
                                                          double* __restrict__ out) {
  __shared__ double red[3][QNT];
  double t[3] = {0.0, 0.0, 0.0};
  for (int64_t i = threadIdx.x; i < n; i += QNT)
    for (int q = 0; q < 3; ++q) t[q] += part[i * 3 + q];
  for (int q = 0; q < 3; ++q) red[q][threadIdx.x] = t[q];
  __syncthreads();
  for (int s = QNT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[2][0] > 0.0 ? 10.0 * log10(red[1][0] / red[2][0]) : (double)INFINITY;
    out[1] = red[0][0] / nwin;
  }
}

}  // namespace
}  // namespace dv

using namespace dv;

extern "C" int64_t dv_image_quality_workspace(int32_t rows, int32_t cols) {
  if (rows < 1 || cols < 1) return 0;
  return (int64_t)((cols + QW - 1) / QW) * ((rows + QH - 1) / QH) * 3;
}

extern "C" dv_status dv_image_quality(const float* x_dev, const float* ref_dev, int32_t rows,
                                      int32_t cols, double dynamic_range, double* work_dev,
                                      double* out_dev, void* stream) {
  clear_error();
  if (!x_dev || !ref_dev || !work_dev || !out_dev) return fail(DV_ERR_INVALID_ARG, "NULL argument");
  if (rows < QT || cols < QT || rows > 65535 * QH)
    return fail(DV_ERR_INVALID_ARG, "image of %d x %d: need at least %d x %d and at most %d rows",
                rows, cols, QT, QT, 65535 * QH);
  if (!(dynamic_range > 0.0) || !std::isfinite(dynamic_range))
    return fail(DV_ERR_INVALID_ARG, "dynamic range must be finite and > 0");
  QGauss G;
  {
    double w[QT], s = 0.0;
    for (int k = 0; k < QT; ++k) s += (w[k] = std::exp(-0.5 * (k - QR) * (k - QR) / (1.5 * 1.5)));
    for (int k = 0; k < QT; ++k) G.g[k] = (float)(w[k] / s);
  }
  const float c1 = (float)((0.01 * dynamic_range) * (0.01 * dynamic_range));
  const float c2 = (float)((0.03 * dynamic_range) * (0.03 * dynamic_range));
  const dim3 grid((unsigned)((cols + QW - 1) / QW), (unsigned)((rows + QH - 1) / QH));
  const int64_t n = (int64_t)grid.x * grid.y;
  cudaStream_t s = (cudaStream_t)stream;
  quality_kernel<<<grid, QNT, 0, s>>>(x_dev, ref_dev, rows, cols, G, c1, c2, work_dev);
  DV_TRY_CUDA(cudaGetLastError());
  quality_sum_kernel<<<1, QNT, 0, s>>>(work_dev, n,
                                       (double)(rows - 2 * QR) * (double)(cols - 2 * QR), out_dev);
  DV_TRY_CUDA(cudaGetLastError());
  return DV_OK;
}
