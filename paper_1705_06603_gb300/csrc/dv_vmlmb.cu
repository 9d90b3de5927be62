// VMLM-B Local-Solver (Sec. IV-B: the paper's local solver is VMLM-B, a
// limited-memory variable-metric method with bound constraints), batched over
// every tile of the plan.  Per tile i it minimises
//   Phi_i(w) = 1/2 ||H_i w - y_i||^2_W + lambda phi(D w) + 1/2 ||w - u_i||^2_alpha,  w >= 0,
// warm-started from the current x_i, with a memory of m pairs (s, y) that is
// reset at the start of every local solve:
//   free set F = {w > 0 or g < 0}; q = g on F, 0 elsewhere;
//   two-loop recursion on q with the stored pairs (full-vector products),
//   H0 = (s'y / y'y) I of the newest pair; d = -q on F, 0 elsewhere;
//   without pairs, or if g'd >= 0 (memory reset), d = -tau_i q (the
//   projected-gradient step of the plain Local-Solver);
//   Armijo along the projection arc w(a) = max(0, w + a d):
//   Phi(w(a)) <= Phi(w) + c1 g'(w(a) - w), c1 = 1e-4, a = 1, 1/2, ... (at most
//   20 trials; a tile that accepts none stays put and resets its memory);
//   the pair (w(a) - w, g(w(a)) - g) is kept if s'y > 0.
// The operator applies are the plan's tile-mode H / H^T launches; the per-tile
// scalars (products, objective terms) are FP64 partial sums per (tile, row
// chunk) that the host adds in a fixed order and turns into the next step's
// per-tile coefficients.  The kernels here are plain streaming kernels over
// the tile stacks.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dv_internal.cuh"

namespace dv {
namespace {

constexpr int VT = 256;            // threads per block
constexpr int VROWS = 16;          // tile rows per block of the streaming kernels

__device__ __forceinline__ double vblock_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < VT / 32; ++w) t += red[w];
  __syncthreads();
  return t;
}

// Per (tile, row chunk) FP64 partial of
//   mode 0: sum a b;   mode 1: sum a (b - c);   mode 2: sum alpha (b - c)^2
// over the tile's x pixels (alpha = gamma omega_r omega_c).
__global__ void __launch_bounds__(VT) vm_dot_kernel(const TileDesc* __restrict__ tiles,
                                                    const float* __restrict__ a,
                                                    const float* __restrict__ b,
                                                    const float* __restrict__ c,
                                                    const float* __restrict__ omr,
                                                    const float* __restrict__ omc, float gamma,
                                                    int mode, double* __restrict__ part) {
  __shared__ double red[VT / 32];
  const TileDesc td = tiles[blockIdx.y];
  const int r0 = blockIdx.x * VROWS, r1 = min(r0 + VROWS, td.nxr);
  double acc = 0.0;
  for (int R = r0; R < r1; ++R) {
    const int64_t base = td.xoff + (int64_t)R * td.xpitch;
    float racc = 0.f;
    for (int C = threadIdx.x; C < td.nxc; C += VT) {
      const int64_t i = base + C;
      float v;
      if (mode == 0) {
        v = a[i] * b[i];
      } else if (mode == 1) {
        v = a[i] * (b[i] - c[i]);
      } else {
        const float d = b[i] - c[i];
        v = gamma * omr[td.omr_off + R] * omc[td.omc_off + C] * d * d;
      }
      racc += v;
    }
    acc += (double)racc;
  }
  const double t = vblock_sum(acc, red);
  if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// y <- y + coef[tile] x over the tile's x pixels (mode 0); mode 1: y = coef y.
// (y and x may be the same buffer, so neither is declared restrict.)
__global__ void __launch_bounds__(VT) vm_axpy_kernel(const TileDesc* __restrict__ tiles, float* y,
                                                     const float* x,
                                                     const float* __restrict__ coef, int mode) {
  const TileDesc td = tiles[blockIdx.y];
  const float k = coef[blockIdx.y];
  const int r0 = blockIdx.x * VROWS, r1 = min(r0 + VROWS, td.nxr);
  for (int R = r0; R < r1; ++R) {
    const int64_t base = td.xoff + (int64_t)R * td.xpitch;
    for (int C = threadIdx.x; C < td.nxc; C += VT) {
      const int64_t i = base + C;
      y[i] = mode == 0 ? fmaf(k, x[i], y[i]) : k * y[i];
    }
  }
}

// q = g on the free set {w > 0 or g < 0}, 0 elsewhere (mode 0);
// d = -coef[tile] q on the free set, 0 elsewhere (mode 1, in place on q).
__global__ void __launch_bounds__(VT) vm_free_kernel(const TileDesc* __restrict__ tiles,
                                                     const float* __restrict__ w,
                                                     const float* __restrict__ g,
                                                     float* __restrict__ q,
                                                     const float* __restrict__ coef, int mode) {
  const TileDesc td = tiles[blockIdx.y];
  const float k = mode == 1 ? coef[blockIdx.y] : 0.f;
  const int r0 = blockIdx.x * VROWS, r1 = min(r0 + VROWS, td.nxr);
  for (int R = r0; R < r1; ++R) {
    const int64_t base = td.xoff + (int64_t)R * td.xpitch;
    for (int C = threadIdx.x; C < td.nxc; C += VT) {
      const int64_t i = base + C;
      const bool fr = w[i] > 0.f || g[i] < 0.f;
      q[i] = mode == 0 ? (fr ? g[i] : 0.f) : (fr ? -k * q[i] : 0.f);
    }
  }
}

// Trial point of the projection arc: wt = max(0, w + alpha[tile] d).
__global__ void __launch_bounds__(VT) vm_trial_kernel(const TileDesc* __restrict__ tiles,
                                                      const float* __restrict__ w,
                                                      const float* __restrict__ d,
                                                      const float* __restrict__ alpha,
                                                      float* __restrict__ wt) {
  const TileDesc td = tiles[blockIdx.y];
  const float a = alpha[blockIdx.y];
  const int r0 = blockIdx.x * VROWS, r1 = min(r0 + VROWS, td.nxr);
  for (int R = r0; R < r1; ++R) {
    const int64_t base = td.xoff + (int64_t)R * td.xpitch;
    for (int C = threadIdx.x; C < td.nxc; C += VT) {
      const int64_t i = base + C;
      wt[i] = fmaxf(0.f, fmaf(a, d[i], w[i]));
    }
  }
}

// psi(D w) at (R, C) of a tile (forward differences, zero on the tile's last
// row / column; psi(v) = v for |v| <= delta, delta v / |v| otherwise).
__device__ __forceinline__ void vm_psi(const float* __restrict__ w, const TileDesc& td, int R, int C,
                                       float delta, float& pr, float& pc) {
  if (R < 0 || C < 0) {
    pr = pc = 0.f;
    return;
  }
  const int64_t i = td.xoff + (int64_t)R * td.xpitch + C;
  const float c0 = w[i];
  const float dr = (R + 1 < td.nxr) ? w[i + td.xpitch] - c0 : 0.f;
  const float dc = (C + 1 < td.nxc) ? w[i + 1] - c0 : 0.f;
  const float s2 = dr * dr + dc * dc;
  const float k = (s2 <= delta * delta) ? 1.f : delta * rsqrtf(s2);
  pr = k * dr;
  pc = k * dc;
}

// g = ht + lambda D^T psi(D w) + alpha (w - u), ht = H_i^T r.
__global__ void __launch_bounds__(VT) vm_grad_kernel(const TileDesc* __restrict__ tiles,
                                                     const float* __restrict__ ht,
                                                     const float* __restrict__ w,
                                                     const float* __restrict__ u,
                                                     const float* __restrict__ omr,
                                                     const float* __restrict__ omc, float gamma,
                                                     float lambda, float delta,
                                                     float* __restrict__ g) {
  const TileDesc td = tiles[blockIdx.y];
  const int r0 = blockIdx.x * VROWS, r1 = min(r0 + VROWS, td.nxr);
  for (int R = r0; R < r1; ++R) {
    const int64_t base = td.xoff + (int64_t)R * td.xpitch;
    for (int C = threadIdx.x; C < td.nxc; C += VT) {
      const int64_t i = base + C;
      float pr, pc, pru, pcu, prl, pcl;
      vm_psi(w, td, R, C, delta, pr, pc);
      vm_psi(w, td, R - 1, C, delta, pru, pcu);
      vm_psi(w, td, R, C - 1, delta, prl, pcl);
      const float hub = pru - pr + pcl - pc;
      const float alpha = gamma * omr[td.omr_off + R] * omc[td.omc_off + C];
      g[i] = ht[i] + lambda * hub + alpha * (w[i] - u[i]);
    }
  }
}

int vm_chunks(const dv_plan* P) { return (P->max_nxr + VROWS - 1) / VROWS; }

dim3 vm_grid(const dv_plan* P) { return dim3((unsigned)vm_chunks(P), (unsigned)P->T); }

constexpr int VRING = 64;          // coefficient slots staged ahead of the kernels

// Host side of one local solve: per-tile sums of device partials (fixed
// order) and per-tile coefficients for the next kernel.  Coefficients go
// through a ring of pinned slots and matching device slots with stream-ordered
// copies (a slot is rewritten only after a synchronisation that follows its
// copy); device partials are downloaded into distinct segments of a pinned
// landing buffer and summed after one synchronisation per batch.
struct VmState {
  dv_plan* P;
  cudaStream_t s;
  int T, nch;
  int slot = 0, since_sync = 0;
  int64_t used = 0;                    // doubles of the landing buffer queued

  dv_status wait() {
    DV_TRY_CUDA(cudaStreamSynchronize(s));
    since_sync = 0;
    return DV_OK;
  }

  // Queues the download of T * per partials; returns their landing offset.
  dv_status enqueue(const double* dptr, int64_t count, int64_t& off) {
    if (used + count > P->h_vpart_cap) return fail(DV_ERR_UNSUPPORTED, "VMLM-B partials exceed the landing buffer");
    off = used;
    DV_TRY_CUDA(cudaMemcpyAsync(P->h_vpart + used, dptr, count * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
    used += count;
    return DV_OK;
  }
  // Per-tile sums of a landed download (after wait()), k-th partial in order.
  void sum(int64_t off, int per, std::vector<double>& out) const {
    const double* h = P->h_vpart + off;
    out.assign(T, 0.0);
    for (int t = 0; t < T; ++t)
      for (int k = 0; k < per; ++k) out[t] += h[(size_t)t * per + k];
  }
  dv_status land() {
    DV_TRY(wait());
    used = 0;
    return DV_OK;
  }

  // One vm_dot launch with its partials queued for download.
  dv_status dot_async(const float* a, const float* b, const float* c, int mode, int64_t& off) {
    vm_dot_kernel<<<vm_grid(P), VT, 0, s>>>(P->d_tiles, a, b, c, P->d_omr, P->d_omc,
                                            (float)P->prob.gamma, mode, P->d_vpart);
    DV_TRY_CUDA(cudaGetLastError());
    P->launches += 1;
    return enqueue(P->d_vpart, (int64_t)T * nch, off);
  }
  // Per-tile sums of one vm_dot launch; synchronises the stream.
  dv_status dot(const float* a, const float* b, const float* c, int mode, std::vector<double>& out) {
    int64_t off;
    DV_TRY(dot_async(a, b, c, mode, off));
    DV_TRY(land());
    sum(off, nch, out);
    return DV_OK;
  }

  // Stages per-tile coefficients; returns the device slot the next kernel reads.
  dv_status set_coef(const std::vector<double>& c, const float*& dev) {
    if (since_sync == VRING) DV_TRY(wait());
    float* h = P->h_vcoef + (size_t)slot * T;
    float* d = P->d_vcoef + (size_t)slot * T;
    for (int t = 0; t < T; ++t) h[t] = (float)c[t];
    DV_TRY_CUDA(cudaMemcpyAsync(d, h, T * sizeof(float), cudaMemcpyHostToDevice, s));
    slot = (slot + 1) % VRING;
    since_sync += 1;
    dev = d;
    return DV_OK;
  }

  dv_status axpy(float* y, const float* x, const std::vector<double>& c, int mode) {
    const float* cd;
    DV_TRY(set_coef(c, cd));
    vm_axpy_kernel<<<vm_grid(P), VT, 0, s>>>(P->d_tiles, y, x, cd, mode);
    DV_TRY_CUDA(cudaGetLastError());
    P->launches += 1;
    return DV_OK;
  }

  dv_status free_set(const float* w, const float* g, float* q, const std::vector<double>* c) {
    const float* cd = P->d_vcoef;
    if (c) DV_TRY(set_coef(*c, cd));
    vm_free_kernel<<<vm_grid(P), VT, 0, s>>>(P->d_tiles, w, g, q, cd, c ? 1 : 0);
    DV_TRY_CUDA(cudaGetLastError());
    P->launches += 1;
    return DV_OK;
  }

  dv_status trial(const float* w, const float* d, const std::vector<double>& a, float* wt) {
    const float* cd;
    DV_TRY(set_coef(a, cd));
    vm_trial_kernel<<<vm_grid(P), VT, 0, s>>>(P->d_tiles, w, d, cd, wt);
    DV_TRY_CUDA(cudaGetLastError());
    P->launches += 1;
    return DV_OK;
  }

  // Phi_i at wq for every tile: data term from the H launch's per-item
  // partials, prior from the Huber partials, proximity term from vm_dot.
  // objective_async queues the launches and downloads; objective_sum reads
  // them after land().
  struct ObjParts {
    int64_t data, prior, prox;
  };
  dv_status objective_async(const float* wq, ObjParts& o) {
    const OpTables& tb = P->tab[tab_index_of(P->path)];
    DV_TRY_CUDA(launch_op_H(P, P->path, op_args_H(P, P->path, OP_OBJ, wq, nullptr, false), s));
    P->launches += 1;
    DV_TRY(enqueue(P->d_part, tb.nH, o.data));
    DV_TRY_CUDA(launch_huber_value(P->d_tiles, T, P->max_nxr, P->max_nxc, wq, P->prob.delta,
                                   P->d_vhub, s));
    P->launches += 1;
    DV_TRY(enqueue(P->d_vhub, huber_blocks(T, P->max_nxr, P->max_nxc), o.prior));
    return dot_async(nullptr, wq, P->d_u, 2, o.prox);
  }
  void objective_sum(const ObjParts& o, std::vector<double>& phi) const {
    const OpTables& tb = P->tab[tab_index_of(P->path)];
    std::vector<double> data(T, 0.0), prior, prox;
    const double* itemp = P->h_vpart + o.data;
    for (int i = 0; i < tb.nH; ++i) data[tb.tileH[i]] += itemp[i];
    sum(o.prior, huber_blocks(T, P->max_nxr, P->max_nxc) / T, prior);
    sum(o.prox, nch, prox);
    phi.assign(T, 0.0);
    for (int t = 0; t < T; ++t)
      phi[t] = 0.5 * data[t] + P->prob.lambda * prior[t] + 0.5 * prox[t];
  }
  dv_status objective(const float* wq, std::vector<double>& phi) {
    ObjParts o;
    DV_TRY(objective_async(wq, o));
    DV_TRY(land());
    objective_sum(o, phi);
    return DV_OK;
  }

  // Gradient of Phi_i at wq into gq: r = W(H wq - y), H^T r, prior, proximity.
  dv_status gradient(const float* wq, float* gq) {
    DV_TRY_CUDA(launch_op_H(P, P->path, op_args_H(P, P->path, OP_RESID, wq, P->d_r, false), s));
    DV_TRY_CUDA(launch_op_Ht(P, P->path,
                             op_args_Ht(P, P->path, OP_PLAIN, P->d_r, P->d_vht, false, wq, P->d_u),
                             s));
    vm_grad_kernel<<<vm_grid(P), VT, 0, s>>>(P->d_tiles, P->d_vht, wq, P->d_u, P->d_omr, P->d_omc,
                                             (float)P->prob.gamma, (float)P->prob.lambda,
                                             (float)P->prob.delta, gq);
    DV_TRY_CUDA(cudaGetLastError());
    P->launches += 3;
    return DV_OK;
  }
};

}  // namespace

// Device and pinned-host state of the VMLM-B solver (allocated on the first call).
dv_status vmlmb_alloc(dv_plan* P) {
  if (P->h_vpart) return DV_OK;          // allocated last: everything is in place
  const int m = P->vm_m;
  const size_t n = (size_t)P->xstack;
  const size_t np = (size_t)P->T * vm_chunks(P);
  const size_t nh = (size_t)huber_blocks(P->T, P->max_nxr, P->max_nxc);
  // a buffer left by an earlier call that failed part-way is kept
  auto dev = [&](void** b, size_t bytes) -> dv_status {
    if (*b) return DV_OK;
    DV_TRY_CUDA(cudaMalloc(b, bytes));
    P->device_bytes += (int64_t)bytes;
    return DV_OK;
  };
  float** bufs[] = {&P->d_vg, &P->d_vgt, &P->d_vd, &P->d_vq, &P->d_vht};
  for (float** b : bufs) DV_TRY(dev((void**)b, n * sizeof(float)));
  DV_TRY(dev((void**)&P->d_vs, (size_t)m * n * sizeof(float)));
  DV_TRY(dev((void**)&P->d_vy, (size_t)m * n * sizeof(float)));
  DV_TRY(dev((void**)&P->d_vpart, np * sizeof(double)));
  DV_TRY(dev((void**)&P->d_vhub, nh * sizeof(double)));
  DV_TRY(dev((void**)&P->d_vcoef, (size_t)VRING * P->T * sizeof(float)));
  // landing: the largest batch is one objective (H items, Huber blocks, one
  // vm_dot) plus one vm_dot
  int64_t nitems = 0;
  for (const OpTables& tb : P->tab) nitems = std::max<int64_t>(nitems, tb.nH);
  const int64_t cap = nitems + (int64_t)nh + 2 * (int64_t)np;
  if (!P->h_vcoef &&
      cudaHostAlloc((void**)&P->h_vcoef, (size_t)VRING * P->T * sizeof(float),
                    cudaHostAllocDefault) != cudaSuccess) {
    P->h_vcoef = nullptr;
    cudaGetLastError();
    return fail(DV_ERR_OOM, "pinned coefficient ring of the VMLM-B solver");
  }
  if (cudaHostAlloc((void**)&P->h_vpart, (size_t)cap * sizeof(double), cudaHostAllocDefault) !=
      cudaSuccess) {
    P->h_vpart = nullptr;
    cudaGetLastError();
    return fail(DV_ERR_OOM, "pinned landing buffer of the VMLM-B solver");
  }
  P->h_vpart_cap = cap;
  return DV_OK;
}

// n_iter VMLM-B iterations on every tile from the iterate in d_w[cur]; the
// result ends in d_w[cur ^ (n_iter & 1)], like the projected-gradient solver.
// Pair k of the local solve occupies slot k mod m for every tile; rho[slot][t]
// = 1 / s'y while the pair belongs to tile t's memory, 0 otherwise (a pair
// with rho 0 leaves the recursion unchanged).  A tile's memory is cleared
// when its direction is not a descent direction, when no trial is accepted
// and when a pair has s'y <= 0; so its valid pairs are always the last (at
// most m) pairs since its last reset.
dv_status vmlmb_local_solve(dv_plan* P, int n_iter, cudaStream_t s) {
  if (n_iter <= 0) return DV_OK;
  DV_TRY(vmlmb_alloc(P));
  VmState V{P, s, P->T, vm_chunks(P)};
  const int T = V.T, m = P->vm_m;
  const size_t n = (size_t)P->xstack;
  int par = P->cur;
  std::vector<double> phi, gd, lin, sy, yy;
  std::vector<double> rho((size_t)m * T, 0.0), gamma0(T, 1.0), tau(T);
  std::vector<int> npair(T, 0);
  // frozen[t]: tile t ended this local solve under the vm_stop_rel test
  std::vector<int> frozen(T, 0);
  const double stop_rel = P->prob.vm_stop_rel;
  for (int t = 0; t < T; ++t) tau[t] = P->tau[t];
  auto clear = [&](int t) {
    npair[t] = 0;
    for (int k = 0; k < m; ++k) rho[(size_t)k * T + t] = 0.0;
  };
  DV_TRY(V.objective(P->d_w[par], phi));
  DV_TRY(V.gradient(P->d_w[par], P->d_vg));
  int it_run = 0;
  for (int it = 0; it < n_iter; ++it) {
    float* w = P->d_w[par];
    float* wt = P->d_w[par ^ 1];
    const int nfill = std::min(it, m);                 // slots written so far
    auto slot_of = [&](int j) { return (it - 1 - j) % m; };   // j-th newest
    // q = projected gradient; first loop, newest pair first
    DV_TRY(V.free_set(w, P->d_vg, P->d_vq, nullptr));
    std::vector<std::vector<double>> a(nfill, std::vector<double>(T, 0.0));
    for (int j = 0; j < nfill; ++j) {
      const int sl = slot_of(j);
      std::vector<double> dots;
      DV_TRY(V.dot(P->d_vs + (size_t)sl * n, P->d_vq, nullptr, 0, dots));
      std::vector<double> c(T);
      for (int t = 0; t < T; ++t) {
        a[j][t] = rho[(size_t)sl * T + t] * dots[t];
        c[t] = -a[j][t];
      }
      DV_TRY(V.axpy(P->d_vq, P->d_vy + (size_t)sl * n, c, 0));
    }
    {
      std::vector<double> c(T);
      for (int t = 0; t < T; ++t) c[t] = npair[t] > 0 ? gamma0[t] : 1.0;
      DV_TRY(V.axpy(P->d_vq, P->d_vq, c, 1));
    }
    for (int j = nfill - 1; j >= 0; --j) {     // oldest pair first
      const int sl = slot_of(j);
      std::vector<double> dots;
      DV_TRY(V.dot(P->d_vy + (size_t)sl * n, P->d_vq, nullptr, 0, dots));
      std::vector<double> c(T);
      for (int t = 0; t < T; ++t) c[t] = a[j][t] - rho[(size_t)sl * T + t] * dots[t];
      DV_TRY(V.axpy(P->d_vq, P->d_vs + (size_t)sl * n, c, 0));
    }
    // d = -q on the free set (tiles without pairs: -tau q, the plain step)
    {
      std::vector<double> c(T);
      for (int t = 0; t < T; ++t) c[t] = npair[t] > 0 ? 1.0 : tau[t];
      DV_TRY_CUDA(cudaMemcpyAsync(P->d_vd, P->d_vq, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
      DV_TRY(V.free_set(w, P->d_vg, P->d_vd, &c));
    }
    DV_TRY(V.dot(P->d_vg, P->d_vd, nullptr, 0, gd));
    // not a descent direction: clear the tile's memory, take the plain step
    std::vector<double> keep(T, 1.0), step(T, 0.0);
    bool any_reset = false;
    for (int t = 0; t < T; ++t)
      if (!(gd[t] < 0.0)) {
        clear(t);
        keep[t] = 0.0;
        step[t] = -tau[t];
        any_reset = true;
      }
    if (any_reset) {
      DV_TRY(V.free_set(w, P->d_vg, P->d_vq, nullptr));   // q = projected gradient
      DV_TRY(V.axpy(P->d_vd, P->d_vd, keep, 1));
      DV_TRY(V.axpy(P->d_vd, P->d_vq, step, 0));
      DV_TRY(V.dot(P->d_vg, P->d_vd, nullptr, 0, gd));
    }
    // a tile whose full step promises a decrease below the resolution of its
    // objective ends its local solve: it keeps its iterate from here on
    int active = 0;
    for (int t = 0; t < T; ++t) {
      if (!frozen[t] && stop_rel > 0.0 && -gd[t] <= stop_rel * std::fabs(phi[t])) {
        frozen[t] = 1;
        P->vm_stops += 1;
      }
      active += !frozen[t];
    }
    if (active == 0) break;
    // Armijo along the projection arc, alpha = 1, 1/2, ...
    std::vector<double> alpha(T, 1.0), acc(T, 0.0), phit, phinew(phi);
    std::vector<int> done(frozen), tries(T, 0);
    int trials_run = 0;
    for (int trial = 0; trial < 20; ++trial) {
      std::vector<double> at(T);
      bool any = false;
      for (int t = 0; t < T; ++t) {
        at[t] = done[t] ? acc[t] : alpha[t];
        any = any || !done[t];
      }
      if (!any) break;
      trials_run = trial + 1;
      DV_TRY(V.trial(w, P->d_vd, at, wt));
      VmState::ObjParts o;
      int64_t olin;
      DV_TRY(V.objective_async(wt, o));
      DV_TRY(V.dot_async(P->d_vg, wt, w, 1, olin));
      DV_TRY(V.land());
      V.objective_sum(o, phit);
      V.sum(olin, V.nch, lin);
      for (int t = 0; t < T; ++t) {
        if (done[t]) continue;
        tries[t] = trial + 1;
        if (phit[t] <= phi[t] + 1e-4 * lin[t]) {
          done[t] = 1;
          acc[t] = alpha[t];
          phinew[t] = phit[t];
        } else {
          alpha[t] *= 0.5;
        }
      }
    }
    bool failed = false;
    for (int t = 0; t < T; ++t)
      if (!done[t]) {
        clear(t);
        failed = true;
      }
    if (failed) DV_TRY(V.trial(w, P->d_vd, acc, wt));   // unaccepted tiles stay put
    phi = phinew;
    P->vm_iters += 1;
    P->vm_trials += trials_run;
    P->vm_trials_max = std::max(P->vm_trials_max, trials_run);
    for (int t = 0; t < T; ++t)
      if (!frozen[t]) {
        P->vm_tile_iters += 1;
        P->vm_tile_trials += tries[t];
      }
    // gradient at the new iterate and the pair (s, y) = (wt - w, gt - g)
    DV_TRY(V.gradient(wt, P->d_vgt));
    const int sl = it % m;
    float* sv = P->d_vs + (size_t)sl * n;
    float* yv = P->d_vy + (size_t)sl * n;
    DV_TRY_CUDA(cudaMemcpyAsync(sv, wt, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    DV_TRY_CUDA(cudaMemcpyAsync(yv, P->d_vgt, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    const std::vector<double> minus(T, -1.0);
    DV_TRY(V.axpy(sv, w, minus, 0));
    DV_TRY(V.axpy(yv, P->d_vg, minus, 0));
    {
      int64_t osy, oyy;
      DV_TRY(V.dot_async(sv, yv, nullptr, 0, osy));
      DV_TRY(V.dot_async(yv, yv, nullptr, 0, oyy));
      DV_TRY(V.land());
      V.sum(osy, V.nch, sy);
      V.sum(oyy, V.nch, yy);
    }
    std::swap(P->d_vg, P->d_vgt);
    for (int t = 0; t < T; ++t) {
      if (sy[t] > 0.0 && yy[t] > 0.0) {
        rho[(size_t)sl * T + t] = 1.0 / sy[t];
        gamma0[t] = sy[t] / yy[t];
        npair[t] = std::min(npair[t] + 1, m);
      } else {
        clear(t);
      }
    }
    par ^= 1;
    it_run = it + 1;
  }
  // every tile stopped early: the result is in d_w[par]; the caller expects it
  // where n_iter iterations would leave it
  if ((it_run & 1) != (n_iter & 1))
    DV_TRY_CUDA(cudaMemcpyAsync(P->d_w[P->cur ^ (n_iter & 1)], P->d_w[par], n * sizeof(float),
                                cudaMemcpyDeviceToDevice, s));
  return DV_OK;
}

}  // namespace dv
