// Allocation-free evaluation of the Huber prior value of one image.
//
// Some callers cannot call cudaMalloc: code that runs as a plug-in inside a
// host framework which reserves all device memory up front and forbids driver
// allocations, or real-time loops where an allocation (which may synchronise
// the device and take milliseconds) is not allowed.  For them this file offers
// dv_prior_value_noalloc: the same per-block FP64 partial sums as the solver's
// prior reduction, but with the partials kept in a fixed-size array that lives
// in the library's own device memory (every GPU that loads the library holds
// it until the process exits), so the call allocates nothing.
#include <mutex>

#include "dv_internal.cuh"

namespace dv {
namespace {

constexpr int NB = 256;                       // threads per block = pixels per block-row chunk
constexpr int kMaxDevices = 64;

// Per-block partial sums shared by every call (see the header for the limit).
static __device__ __align__(256) double g_prior_partials[DV_NOALLOC_MAX_BLOCKS];

std::mutex g_setup_mutex;
double* g_partials_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NB / 32; ++i) s += red[i];
  return s;
}

// One block per (row, 256-column chunk): partial of sum hub(|grad x|) with
// forward differences set to zero on the last row / column.
__global__ void __launch_bounds__(NB) prior_partials_kernel(const float* __restrict__ x, int rows,
                                                            int cols, double delta,
                                                            double* __restrict__ partials) {
  __shared__ double red[NB / 32];
  const int R = blockIdx.y;
  const int C = blockIdx.x * NB + threadIdx.x;
  double acc = 0.0;
  if (C < cols) {
    const int64_t idx = (int64_t)R * cols + C;
    const double c0 = x[idx];
    const double dr = (R + 1 < rows) ? (double)x[idx + cols] - c0 : 0.0;
    const double dc = (C + 1 < cols) ? (double)x[idx + 1] - c0 : 0.0;
    const double s = sqrt(dr * dr + dc * dc);
    acc = (s <= delta) ? 0.5 * s * s : delta * (s - 0.5 * delta);
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// Sums the first n partials in a fixed order and writes (not adds) the result.
__global__ void __launch_bounds__(NB) prior_finish_kernel(const double* __restrict__ partials,
                                                          int n, double* __restrict__ out) {
  __shared__ double red[NB / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += NB) s += partials[i];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) *out = t;
}

// Device address of the static partials array for the current device, looked
// up once per device.
dv_status partials_for_current_device(double** out) {
  int dev = 0;
  DV_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(DV_ERR_UNSUPPORTED, "device ordinal %d is beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    DV_TRY_CUDA(cudaGetSymbolAddress(&p, g_prior_partials));
    g_partials_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_ptr[dev];
  return DV_OK;
}

}  // namespace
}  // namespace dv

using namespace dv;

extern "C" dv_status dv_prior_value_noalloc(const float* x_dev, int32_t rows, int32_t cols,
                                            double delta, double* value_dev, void* stream) {
  clear_error();
  if (!x_dev || !value_dev) return fail(DV_ERR_INVALID_ARG, "x_dev and value_dev must not be NULL");
  if (rows < 1 || cols < 1) return fail(DV_ERR_INVALID_ARG, "rows and cols must be >= 1");
  if (!(delta > 0.0)) return fail(DV_ERR_INVALID_ARG, "delta must be > 0");
  const int64_t chunks = (cols + NB - 1) / NB;
  const int64_t nblk = chunks * rows;
  if (nblk > DV_NOALLOC_MAX_BLOCKS || rows > 65535)
    return fail(DV_ERR_INVALID_ARG,
                "image of %d x %d needs %lld partial sums (one per row and 256 columns) and "
                "%d rows; the allocation-free scratch holds %d partials and the grid at most "
                "65535 rows",
                rows, cols, (long long)nblk, rows, DV_NOALLOC_MAX_BLOCKS);
  double* partials = nullptr;
  DV_TRY(partials_for_current_device(&partials));
  cudaStream_t s = (cudaStream_t)stream;
  prior_partials_kernel<<<dim3((unsigned)chunks, (unsigned)rows), NB, 0, s>>>(x_dev, rows, cols,
                                                                             delta, partials);
  DV_TRY_CUDA(cudaGetLastError());
  prior_finish_kernel<<<1, NB, 0, s>>>(partials, (int)nblk, value_dev);
  DV_TRY_CUDA(cudaGetLastError());
  return DV_OK;
}
