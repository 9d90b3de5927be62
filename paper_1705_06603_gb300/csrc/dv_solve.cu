// Entry points of libdv that run work: the global operator and its adjoint
// (Sec. II-B), Algorithm 1 (Sec. III-B) with the local solves replayed as CUDA
// graphs, the FP64 objective / residual reductions, host-buffer solves,
// checkpoint / resume of the D-R state, and per-kernel event timing.
#include <algorithm>
#include <cmath>

#include "dv_internal.cuh"

namespace dv {
namespace {

enum Kind { KIND_H = 0, KIND_HT = 1, KIND_CONS = 2, KIND_LOCAL = 3 };

// Whether the captured local solve runs the tile groups concurrently.
bool grouped(const dv_plan* P) { return P->ngrp > 1 && P->path == DV_PATH_TENSOR; }

int nhub(const dv_plan* P) { return huber_blocks(P->T, P->max_nxr, P->max_nxc); }
int ncons(const dv_plan* P) { return consensus_blocks(P->n_citems); }
double* part_data(dv_plan* P) { return P->d_part; }
int npart_data(const dv_plan* P) {
  return std::max(std::max(P->tab[0].nH, P->tab[1].nH), P->tab[2].nH);
}
double* part_hub(dv_plan* P) { return P->d_part + npart_data(P); }
double* part_cons(dv_plan* P) { return P->d_part + npart_data(P) + nhub(P); }

dv_status pool_event(dv_plan* P, int* idx) {
  KernelTimer& T = P->timer;
  if (T.next == T.pool.size()) {
    cudaEvent_t e;
    DV_TRY_CUDA(cudaEventCreate(&e));
    T.pool.push_back(e);
  }
  *idx = (int)T.next++;
  return DV_OK;
}

// Collects the durations of every pending timed launch (synchronising on them).
dv_status harvest(dv_plan* P) {
  KernelTimer& T = P->timer;
  for (const Pending& q : T.pending) {
    DV_TRY_CUDA(cudaEventSynchronize(T.pool[q.ev1]));
    float ms = 0.f;
    DV_TRY_CUDA(cudaEventElapsedTime(&ms, T.pool[q.ev0], T.pool[q.ev1]));
    T.total_ms[q.kind] += ms;
    T.count[q.kind] += 1;
  }
  T.pending.clear();
  T.next = 0;
  return DV_OK;
}

// Launches one kernel through fn, bracketed by pool events when timing is on.
template <class F>
dv_status timed_launch(dv_plan* P, int kind, cudaStream_t s, F fn) {
  int e0 = -1, e1 = -1;
  if (P->timing) {
    DV_TRY(pool_event(P, &e0));
    DV_TRY(pool_event(P, &e1));
    DV_TRY_CUDA(cudaEventRecord(P->timer.pool[e0], s));
  }
  DV_TRY_CUDA(fn(s));
  P->launches += 1;
  if (P->timing) {
    DV_TRY_CUDA(cudaEventRecord(P->timer.pool[e1], s));
    P->timer.pending.push_back(Pending{kind, e0, e1});
  }
  return DV_OK;
}

// kernels one inner-iteration H^T launch runs (the block DFT adds its step kernel)
static int ht_kernels(const dv_plan* P) {
  return P->path == DV_PATH_TENSOR && P->dft_Ht ? dft_Ht_kernels(OP_STEP) : 1;
}

cudaError_t launch_inner_H(dv_plan* P, int par, cudaStream_t s) {
  return launch_op_H(P, P->path, op_args_H(P, P->path, OP_RESID, P->d_w[par], P->d_r, false), s);
}

cudaError_t launch_inner_Ht(dv_plan* P, int par, cudaStream_t s) {
  return launch_op_Ht(P, P->path,
                      op_args_Ht(P, P->path, OP_STEP, P->d_r, P->d_w[par ^ 1], false, P->d_w[par],
                                 P->d_u),
                      s);
}

// Tile group g of the inner iterations: the same kernels on the group's items.
cudaError_t launch_group_H(dv_plan* P, int par, int g, cudaStream_t s) {
  return launch_op_H(P, P->path,
                     group_args(P, P->path, op_args_H(P, P->path, OP_RESID, P->d_w[par], P->d_r, false),
                                false, g),
                     s);
}

cudaError_t launch_group_Ht(dv_plan* P, int par, int g, cudaStream_t s) {
  return launch_op_Ht(P, P->path,
                      group_args(P, P->path,
                                 op_args_Ht(P, P->path, OP_STEP, P->d_r, P->d_w[par ^ 1], false,
                                            P->d_w[par], P->d_u),
                                 true, g),
                      s);
}

// Captures the n_inner iterations of every tile group on a stream of its own
// (fork from and join back into the capture stream).
dv_status capture_groups(dv_plan* P, cudaStream_t cs, int par, int n_inner) {
  DV_TRY_CUDA(cudaEventRecord(P->grp_fork, cs));
  for (int g = 0; g < P->ngrp; ++g) DV_TRY_CUDA(cudaStreamWaitEvent(P->grp_stream[g], P->grp_fork, 0));
  for (int g = 0; g < P->ngrp; ++g) {
    int pg = par;
    for (int i = 0; i < n_inner; ++i) {
      DV_TRY_CUDA(launch_group_H(P, pg, g, P->grp_stream[g]));
      DV_TRY_CUDA(launch_group_Ht(P, pg, g, P->grp_stream[g]));
      pg ^= 1;
    }
    DV_TRY_CUDA(cudaEventRecord(P->grp_join[g], P->grp_stream[g]));
    DV_TRY_CUDA(cudaStreamWaitEvent(cs, P->grp_join[g], 0));
  }
  return DV_OK;
}

dv_status capture_node(cudaStream_t cs, cudaGraphNode_t* node) {
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  DV_TRY_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &deps, nullptr, &nd));
  if (st != cudaStreamCaptureStatusActive || nd != 1 || !deps)
    return fail(DV_ERR_CUDA, "unexpected capture state while recording a timing node");
  *node = deps[0];
  return DV_OK;
}

// Objective reduction of eval_objective, enqueued only: x_hat, its tile
// restrictions, the FP32 operator's data-term partials, the prior partials,
// the fixed-order FP64 sums and their read-back (with the device error word)
// into pinned memory.
dv_status enqueue_objective(dv_plan* P, bool residuals, cudaStream_t s) {
  const GridArgs g = grid_args(P);
  float* tmp = P->d_w[P->cur ^ 1];
  DV_TRY_CUDA(launch_assemble(g, P->d_w[P->cur], P->d_xg, s));
  DV_TRY_CUDA(launch_scatter(g, P->T, P->max_nxr, P->max_nxc, P->d_xg, nullptr, P->hy, P->wy,
                             P->rad, tmp, nullptr, s, nullptr));
  DV_TRY_CUDA(launch_op_H(P, P->fpath, op_args_H(P, P->fpath, OP_OBJ, tmp, nullptr, false), s));
  DV_TRY_CUDA(launch_huber_value(P->d_tiles, P->T, P->max_nxr, P->max_nxc, tmp, P->prob.delta,
                                 part_hub(P), s));
  const double* parts[4] = {part_data(P), part_hub(P), part_cons(P), part_cons(P) + ncons(P)};
  const int counts[4] = {obj_parts(P), nhub(P), ncons(P), ncons(P)};
  DV_TRY_CUDA(launch_reduce(parts, counts, residuals ? 4 : 2, P->d_scal, s));
  DV_TRY_CUDA(cudaMemcpyAsync(P->h_scal, P->d_scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  int* h_err = reinterpret_cast<int*>(P->h_scal + 6);
  DV_TRY_CUDA(cudaMemcpyAsync(h_err, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  return DV_OK;
}
constexpr int kObjLaunches = 5;

// Waits for an enqueued objective reduction and checks the error word.
dv_status read_objective(dv_plan* P, bool residuals, cudaStream_t s) {
  DV_TRY_CUDA(cudaStreamSynchronize(s));
  const int* h_err = reinterpret_cast<const int*>(P->h_scal + 6);
  if (*h_err != 0)
    return fail(DV_ERR_TIMEOUT, "a tensor-core operator kernel gave up waiting on its pipeline");
  if (!residuals) P->h_scal[2] = P->h_scal[3] = NAN;
  return DV_OK;
}

cudaError_t launch_cons(dv_plan* P, int cur, bool track_z, bool residuals, cudaStream_t s) {
  return launch_consensus(grid_args(P), P->d_w[cur], P->d_u, (float)P->prob.gamma,
                          (float)P->prob.rho, track_z ? P->d_z : nullptr,
                          residuals ? part_cons(P) : nullptr, s, nullptr);
}

// Records an external event-record node on the capture stream (timed graphs).
dv_status timing_node(dv_plan* P, cudaStream_t cs, int which, cudaGraphNode_t* node) {
  const cudaError_t e = cudaEventRecordWithFlags(P->timer.placeholders[which], cs,
                                                 cudaEventRecordExternal);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord", __FILE__, __LINE__);
  return capture_node(cs, node);
}

// Captures one outer iteration: the local solve (tile groups on their own
// streams, or one launch per operator), then, with g.cons, the consensus and
// dual update on the resulting iterate and, with bit 3, the objective reduction.
dv_status capture_outer(dv_plan* P, GraphEntry& g) {
  cudaStream_t cs = P->cap_stream;
  if (g.timed && P->timer.placeholders.empty()) {
    cudaEvent_t a, b;
    DV_TRY_CUDA(cudaEventCreate(&a));
    DV_TRY_CUDA(cudaEventCreate(&b));
    P->timer.placeholders = {a, b};
  }
  DV_TRY_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  dv_status st = DV_OK;
  int par = g.parity;
  const bool grp = grouped(P);
  auto bracket = [&](int kind, auto&& body) -> dv_status {
    cudaGraphNode_t n0 = nullptr, n1 = nullptr;
    if (g.timed) DV_TRY(timing_node(P, cs, 0, &n0));
    DV_TRY(body());
    if (g.timed) {
      DV_TRY(timing_node(P, cs, 1, &n1));
      g.ev_start.push_back(n0);
      g.ev_end.push_back(n1);
      g.kinds.push_back(kind);
    }
    return DV_OK;
  };
  if (grp) {
    // the tile groups run concurrently: the local solve is timed as a whole
    st = bracket(KIND_LOCAL, [&]() { return capture_groups(P, cs, par, g.n_inner); });
    par ^= (g.n_inner & 1);
  } else {
    for (int i = 0; i < g.n_inner && st == DV_OK; ++i) {
      for (int k = 0; k < 2 && st == DV_OK; ++k)
        st = bracket(k == 0 ? KIND_H : KIND_HT, [&]() -> dv_status {
          const cudaError_t e = k == 0 ? launch_inner_H(P, par, cs) : launch_inner_Ht(P, par, cs);
          return e == cudaSuccess ? DV_OK : cuda_fail(e, "kernel launch during capture", __FILE__, __LINE__);
        });
      par ^= 1;
    }
  }
  if (st == DV_OK && (g.cons & 1))
    st = bracket(KIND_CONS, [&]() -> dv_status {
      const cudaError_t e = launch_cons(P, par, (g.cons & 2) != 0, (g.cons & 4) != 0, cs);
      return e == cudaSuccess ? DV_OK : cuda_fail(e, "kernel launch during capture", __FILE__, __LINE__);
    });
  if (st == DV_OK && (g.cons & 8)) {
    const int keep = P->cur;
    P->cur = par;                       // the objective reads the iterate the graph leaves
    st = enqueue_objective(P, (g.cons & 4) != 0, cs);
    P->cur = keep;
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
  if (st != DV_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture", __FILE__, __LINE__);
  g.graph = graph;
  DV_TRY_CUDA(cudaGraphInstantiate(&g.exec, graph, 0));
  return DV_OK;
}

dv_status get_graph(dv_plan* P, int n_inner, int par, int cons, GraphEntry** out) {
  for (GraphEntry& g : P->graphs)
    if (g.n_inner == n_inner && g.parity == par && g.timed == P->timing && g.cons == cons) {
      *out = &g;
      return DV_OK;
    }
  GraphEntry g;
  g.n_inner = n_inner;
  g.parity = par;
  g.timed = P->timing;
  g.cons = cons;
  DV_TRY(capture_outer(P, g));
  P->graphs.push_back(g);
  *out = &P->graphs.back();
  return DV_OK;
}

// Launches a captured outer iteration (or local solve), swapping pool events
// into its timing nodes.
dv_status launch_graph(dv_plan* P, GraphEntry* g, cudaStream_t s) {
  if (g->timed) {
    for (size_t j = 0; j < g->kinds.size(); ++j) {
      int e0, e1;
      DV_TRY(pool_event(P, &e0));
      DV_TRY(pool_event(P, &e1));
      DV_TRY_CUDA(cudaGraphExecEventRecordNodeSetEvent(g->exec, g->ev_start[j], P->timer.pool[e0]));
      DV_TRY_CUDA(cudaGraphExecEventRecordNodeSetEvent(g->exec, g->ev_end[j], P->timer.pool[e1]));
      P->timer.pending.push_back(Pending{g->kinds[j], e0, e1});
    }
  }
  DV_TRY_CUDA(cudaGraphLaunch(g->exec, s));
  P->launches += (1 + ht_kernels(P)) * g->n_inner * (grouped(P) ? P->ngrp : 1) + ((g->cons & 1) ? 1 : 0) +
                 ((g->cons & 8) ? kObjLaunches : 0);
  return DV_OK;
}

// The Local-Solver of Algorithm 1 on every tile: n_inner x {r = W (H_i w - y_i);
// w <- max(0, w - tau (H_i^T r + lambda D^T psi(D w) + alpha (w - u)))}.
// Eager (no graphs) or VMLM-B; the captured form runs in run_outer.
dv_status local_solve(dv_plan* P, int n_inner, cudaStream_t s) {
  Range range("dv local solve");
  if (n_inner <= 0) return DV_OK;
  if (P->prob.local_solver == DV_SOLVER_VMLMB) {
    DV_TRY(vmlmb_local_solve(P, n_inner, s));
    P->cur ^= (n_inner & 1);
    return DV_OK;
  }
  if (P->prob.use_graphs) {
    GraphEntry* g = nullptr;
    DV_TRY(get_graph(P, n_inner, P->cur, 0, &g));
    DV_TRY(launch_graph(P, g, s));
  } else {
    int par = P->cur;
    for (int i = 0; i < n_inner; ++i) {
      DV_TRY(timed_launch(P, KIND_H, s, [&](cudaStream_t st) { return launch_inner_H(P, par, st); }));
      DV_TRY(timed_launch(P, KIND_HT, s, [&](cudaStream_t st) { return launch_inner_Ht(P, par, st); }));
      P->launches += ht_kernels(P) - 1;
      par ^= 1;
    }
  }
  P->cur ^= (n_inner & 1);
  return DV_OK;
}

dv_status consensus_step(dv_plan* P, bool track_z, bool residuals, cudaStream_t s) {
  Range range("dv consensus");
  return timed_launch(P, KIND_CONS, s, [&](cudaStream_t st) {
    return launch_cons(P, P->cur, track_z, residuals, st);
  });
}

// Terms of F(x_hat) = sum_i [1/2 ||y_i - H_i C_i x_hat||^2_W + lambda phi(D C_i x_hat)]
// reduced in FP64: h_scal[0] = sum_i ||y_i - H_i C_i x_hat||^2_W (without the 1/2),
// h_scal[1] = sum_i phi(D C_i x_hat), and (when the last consensus step wrote
// them) h_scal[2..3] = the squared primal / dual residuals.  Synchronises the stream.
dv_status eval_objective(dv_plan* P, bool residuals, cudaStream_t s) {
  Range range("dv objective");
  DV_TRY(enqueue_objective(P, residuals, s));
  P->launches += kObjLaunches;
  return read_objective(P, residuals, s);
}

struct RunResult {
  int inner_done = 0;
  bool have_resid = false;
  bool have_obj = false;
};

// n outer iterations of Algorithm 1 from the plan's current state.  With CUDA
// graphs (projected gradient) one graph launch covers an outer iteration:
// local solve, consensus and dual update and, when due, the objective
// reduction, whose read-back is the only host synchronisation.
dv_status run_outer(dv_plan* P, int n, bool want_stats, cudaStream_t s, RunResult& rr) {
  const dv_problem& pr = P->prob;
  const bool track_z = want_stats || pr.check_every > 0;
  const bool captured = pr.use_graphs && pr.local_solver == DV_SOLVER_PG;
  const bool target = pr.check_every > 0 && pr.target_objective > 0.0;
  int next_check = pr.check_every;   // outer iterations of this call before the next check
  int k_prev = -1;
  double F_prev = 0.0;
  for (int k = 0; k < n; ++k) {
    const int ni = pr.n_inner + P->outer_done * pr.inner_increment;
    const bool check = pr.check_every > 0 && k + 1 == next_check;
    const bool last = k + 1 == n;
    const bool resid = track_z && (check || last);
    if (captured && ni > 0) {
      Range range("dv outer iteration");
      const int cons = 1 | (track_z ? 2 : 0) | (resid ? 4 : 0) | (check ? 8 : 0);
      GraphEntry* g = nullptr;
      DV_TRY(get_graph(P, ni, P->cur, cons, &g));
      DV_TRY(launch_graph(P, g, s));
      P->cur ^= (ni & 1);
      if (check) {
        Range robj("dv objective");
        DV_TRY(read_objective(P, true, s));
      }
    } else {
      DV_TRY(local_solve(P, ni, s));
      DV_TRY(consensus_step(P, track_z, resid, s));
      if (check) DV_TRY(eval_objective(P, true, s));
    }
    rr.inner_done += ni;
    P->outer_done += 1;
    rr.have_resid = resid;
    rr.have_obj = false;
    if (check) {
      rr.have_obj = true;
      const double F = 0.5 * P->h_scal[0] + pr.lambda * P->h_scal[1];
      if (target && F <= pr.target_objective) break;
      // next check: with a target, where the decrease per outer iteration
      // since the last check would reach it (0.9 of that, between 1 and
      // 2 check_every iterations; the decrease slows, so this errs early);
      // otherwise every check_every iterations
      int gap = pr.check_every;
      if (target && k_prev >= 0 && F_prev > F) {
        const double rate = (F_prev - F) / (double)(k - k_prev);
        const double need = (F - pr.target_objective) / rate;
        gap = (int)std::min<double>(2.0 * pr.check_every, std::max(1.0, std::ceil(0.9 * need)));
      }
      k_prev = k;
      F_prev = F;
      next_check = k + 1 + gap;
    }
  }
  return DV_OK;
}

dv_status finish(dv_plan* P, float* x_out, dv_stats* st, const RunResult& rr, int64_t l0,
                 cudaStream_t s) {
  DV_TRY_CUDA(launch_assemble(grid_args(P), P->d_w[P->cur], P->d_xg, s));
  P->launches += 1;
  if (x_out && x_out != P->d_xg)
    DV_TRY_CUDA(cudaMemcpyAsync(x_out, P->d_xg, (size_t)P->nxr * P->nxc * sizeof(float),
                                cudaMemcpyDeviceToDevice, s));
  DV_TRY_CUDA(cudaEventRecord(P->ev1, s));
  if (st) {
    if (!rr.have_obj) DV_TRY(eval_objective(P, rr.have_resid, s));
    st->data_term = 0.5 * P->h_scal[0];
    st->prior_term = P->h_scal[1];
    st->objective = 0.5 * P->h_scal[0] + P->prob.lambda * P->h_scal[1];
    st->primal_res = std::sqrt(P->h_scal[2]);
    st->dual_res = std::sqrt(P->h_scal[3]);
    st->outer_done = P->outer_done;
    st->inner_done = rr.inner_done;
    float ms = 0.f;
    DV_TRY_CUDA(cudaEventSynchronize(P->ev1));
    DV_TRY_CUDA(cudaEventElapsedTime(&ms, P->ev0, P->ev1));
    st->ms_total = ms;
    st->kernel_launches = P->launches - l0;
    st->vm_trials_per_iter = P->vm_iters > 0 ? (double)P->vm_trials / (double)P->vm_iters : 0.0;
    st->vm_tile_trials =
        P->vm_tile_iters > 0 ? (double)P->vm_tile_trials / (double)P->vm_tile_iters : 0.0;
    st->vm_trials_max = P->vm_trials_max;
    st->vm_stops = P->vm_stops;
  }
  return DV_OK;
}

// Clears the per-call Armijo counters of the VMLM-B Local-Solver.
void reset_call_counters(dv_plan* P) {
  P->vm_iters = P->vm_trials = P->vm_tile_iters = P->vm_tile_trials = 0;
  P->vm_trials_max = P->vm_stops = 0;
}

dv_status check_plan(const dv_plan* P) {
  if (!P) return fail(DV_ERR_INVALID_ARG, "plan is NULL");
  return DV_OK;
}

// Algorithm 1 from the start image; y is already in P->d_y.
dv_status solve_internal(dv_plan* P, const float* x0, float* x_out, dv_stats* st, cudaStream_t s,
                         int64_t l0) {
  Range range("dv solve");
  reset_call_counters(P);
  const GridArgs g = grid_args(P);
  const bool track_z = st || P->prob.check_every > 0;
  if (!x0 && P->prob.use_warmstart) {
    if (!P->cnn) return fail(DV_ERR_INVALID_ARG, "use_warmstart is set but no network is attached");
    DV_TRY(warmstart_x0(P, s, P->d_xg));
    x0 = P->d_xg;
  }
  DV_TRY_CUDA(launch_scatter(g, P->T, P->max_nxr, P->max_nxc, x0, P->d_y, P->hy, P->wy, P->rad,
                             P->d_w[0], P->d_u, s, track_z ? P->d_z : nullptr));
  P->launches += 1;
  P->cur = 0;
  P->outer_done = 0;
  RunResult rr;
  DV_TRY(run_outer(P, P->prob.n_outer, st != nullptr, s, rr));
  return finish(P, x_out, st, rr, l0, s);
}

}  // namespace
}  // namespace dv

using namespace dv;

extern "C" dv_status dv_apply_H(dv_plan* P, const float* x_dev, float* y_dev, void* stream) {
  clear_error();
  DV_TRY(check_plan(P));
  if (!x_dev || !y_dev) return fail(DV_ERR_INVALID_ARG, "x_dev and y_dev must not be NULL");
  DV_TRY_CUDA(launch_op_H(P, P->path, op_args_H(P, P->path, OP_PLAIN, x_dev, y_dev, true),
                          (cudaStream_t)stream));
  P->launches += 1;
  return DV_OK;
}

extern "C" dv_status dv_apply_Ht(dv_plan* P, const float* r_dev, float* g_dev, void* stream) {
  clear_error();
  DV_TRY(check_plan(P));
  if (!r_dev || !g_dev) return fail(DV_ERR_INVALID_ARG, "r_dev and g_dev must not be NULL");
  DV_TRY_CUDA(launch_op_Ht(P, P->path,
                           op_args_Ht(P, P->path, OP_PLAIN, r_dev, g_dev, true, nullptr, nullptr),
                            (cudaStream_t)stream));
  P->launches += 1;
  return DV_OK;
}

extern "C" dv_status dv_consensus_solve(dv_plan* P, const float* y_dev, const float* x0_dev,
                                        float* x_out_dev, dv_stats* stats, void* stream) {
  clear_error();
  DV_TRY(check_plan(P));
  if (!y_dev || !x_out_dev) return fail(DV_ERR_INVALID_ARG, "y_dev and x_out_dev must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t l0 = P->launches;
  DV_TRY_CUDA(cudaEventRecord(P->ev0, s));
  DV_TRY_CUDA(cudaMemcpyAsync(P->d_y, y_dev, (size_t)P->hy * P->wy * sizeof(float),
                              cudaMemcpyDeviceToDevice, s));
  return solve_internal(P, x0_dev, x_out_dev, stats, s, l0);
}

extern "C" dv_status dv_consensus_solve_host(dv_plan* P, const float* y_host, const float* x0_host,
                                             float* x_out_host, dv_stats* stats, void* stream) {
  clear_error();
  DV_TRY(check_plan(P));
  if (!y_host || !x_out_host)
    return fail(DV_ERR_INVALID_ARG, "y_host and x_out_host must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nx = (size_t)P->nxr * P->nxc;
  if (x0_host && !P->d_hx0) {
    DV_TRY_CUDA(cudaMalloc((void**)&P->d_hx0, nx * sizeof(float)));
    P->device_bytes += nx * sizeof(float);
  }
  const int64_t l0 = P->launches;
  DV_TRY_CUDA(cudaEventRecord(P->ev0, s));
  DV_TRY_CUDA(cudaMemcpyAsync(P->d_y, y_host, (size_t)P->hy * P->wy * sizeof(float),
                              cudaMemcpyHostToDevice, s));
  if (x0_host)
    DV_TRY_CUDA(cudaMemcpyAsync(P->d_hx0, x0_host, nx * sizeof(float), cudaMemcpyHostToDevice, s));
  DV_TRY(solve_internal(P, x0_host ? P->d_hx0 : nullptr, P->d_xg, stats, s, l0));
  DV_TRY_CUDA(cudaMemcpyAsync(x_out_host, P->d_xg, nx * sizeof(float), cudaMemcpyDeviceToHost, s));
  int* h_err = reinterpret_cast<int*>(P->h_scal + 6);
  DV_TRY_CUDA(cudaMemcpyAsync(h_err, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  DV_TRY_CUDA(cudaStreamSynchronize(s));
  if (*h_err != 0)
    return fail(DV_ERR_TIMEOUT, "a tensor-core operator kernel gave up waiting on its pipeline");
  return DV_OK;
}

extern "C" dv_status dv_consensus_continue(dv_plan* P, const float* y_dev, int32_t n_outer,
                                           float* x_out_dev, dv_stats* stats, void* stream) {
  clear_error();
  DV_TRY(check_plan(P));
  if (!y_dev || !x_out_dev || n_outer < 0)
    return fail(DV_ERR_INVALID_ARG, "need y_dev, x_out_dev and n_outer >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t l0 = P->launches;
  DV_TRY_CUDA(cudaEventRecord(P->ev0, s));
  DV_TRY_CUDA(cudaMemcpyAsync(P->d_y, y_dev, (size_t)P->hy * P->wy * sizeof(float),
                              cudaMemcpyDeviceToDevice, s));
  RunResult rr;
  reset_call_counters(P);
  if ((stats || P->prob.check_every > 0) && n_outer > 0) {
    // the dual residual needs the previous zbar: rebuild it from the current state
    DV_TRY_CUDA(launch_assemble(grid_args(P), P->d_w[P->cur], P->d_z, s));
    P->launches += 1;
  }
  DV_TRY(run_outer(P, n_outer, stats != nullptr, s, rr));
  return finish(P, x_out_dev, stats, rr, l0, s);
}

extern "C" dv_status dv_state_export(dv_plan* P, float* x_stack_dev, float* u_stack_dev,
                                     int32_t* outer_done, void* stream) {
  clear_error();
  DV_TRY(check_plan(P));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b = (size_t)P->xstack * sizeof(float);
  if (x_stack_dev) DV_TRY_CUDA(cudaMemcpyAsync(x_stack_dev, P->d_w[P->cur], b, cudaMemcpyDeviceToDevice, s));
  if (u_stack_dev) DV_TRY_CUDA(cudaMemcpyAsync(u_stack_dev, P->d_u, b, cudaMemcpyDeviceToDevice, s));
  if (outer_done) *outer_done = P->outer_done;
  return DV_OK;
}

extern "C" dv_status dv_state_import(dv_plan* P, const float* x_stack_dev, const float* u_stack_dev,
                                     int32_t outer_done, void* stream) {
  clear_error();
  DV_TRY(check_plan(P));
  if (!x_stack_dev || !u_stack_dev || outer_done < 0)
    return fail(DV_ERR_INVALID_ARG, "need both stacks and outer_done >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b = (size_t)P->xstack * sizeof(float);
  DV_TRY_CUDA(cudaMemcpyAsync(P->d_w[0], x_stack_dev, b, cudaMemcpyDeviceToDevice, s));
  DV_TRY_CUDA(cudaMemcpyAsync(P->d_u, u_stack_dev, b, cudaMemcpyDeviceToDevice, s));
  P->cur = 0;
  P->outer_done = outer_done;
  return DV_OK;
}

namespace dv {
namespace {
// Destroys the captured local solves (they hold the kernel arguments of the
// time of capture); they are captured again on their next use.
dv_status drop_graphs(dv_plan* P) {
  DV_TRY_CUDA(cudaDeviceSynchronize());
  for (GraphEntry& g : P->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  P->graphs.clear();
  return DV_OK;
}
}  // namespace
}  // namespace dv

extern "C" dv_status dv_plan_set_wait_limit(dv_plan* P, double seconds) {
  clear_error();
  DV_TRY(check_plan(P));
  if (!(seconds >= 0.0 && seconds <= 60.0))
    return fail(DV_ERR_INVALID_ARG, "the wait limit must be in [0, 60] seconds");
  DV_TRY(drop_graphs(P));
  P->wait_ns = (uint64_t)(seconds * 1e9);
  return DV_OK;
}

extern "C" dv_status dv_plan_set_wait_test(dv_plan* P, int32_t withhold) {
  clear_error();
  DV_TRY(check_plan(P));
  if (withhold != 0 && withhold != 1) return fail(DV_ERR_INVALID_ARG, "withhold must be 0 or 1");
  DV_TRY(drop_graphs(P));
  P->test_fault = withhold;
  return DV_OK;
}

extern "C" dv_status dv_plan_set_timing(dv_plan* P, int32_t enable) {
  clear_error();
  DV_TRY(check_plan(P));
  DV_TRY(harvest(P));
  P->timing = enable != 0;
  for (int k = 0; k < 4; ++k) {
    P->timer.total_ms[k] = 0.0;
    P->timer.count[k] = 0;
  }
  return DV_OK;
}

extern "C" dv_status dv_plan_kernel_time(dv_plan* P, int32_t kind, double* total_ms,
                                         int64_t* launches) {
  clear_error();
  DV_TRY(check_plan(P));
  if (kind < 0 || kind > 3) return fail(DV_ERR_INVALID_ARG, "kind must be 0, 1, 2 or 3");
  DV_TRY(harvest(P));
  if (total_ms) *total_ms = P->timer.total_ms[kind];
  if (launches) *launches = P->timer.count[kind];
  return DV_OK;
}
