// Restarted (F)GMRES of Sec. 5 as a resumable state machine.
//
// A run alternates "enqueue" steps (work put on the problem's stream, ending
// with an asynchronous copy of the device scalars to pinned host memory) and
// "after" steps (host decisions on those scalars once the stream has
// drained).  A single solve drives one run and waits after every enqueue; a
// batch drives many runs in rounds and waits once per round for all of
// them.  Host work is orchestration only: every arithmetic step is a kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "bec_internal.h"

namespace bec {

namespace {
constexpr int S_REF = 0, S_BETA = 1, S_W = 2, S_RES = 3, S_TRUE = 4, S_WB = 6, S_ONE = 15;

#define BEC_TRY(expr)            \
  do {                           \
    bec_status _s = (expr);      \
    if (_s != BEC_OK) return _s; \
  } while (0)

bec_status enqueue_scalar_read(bec_problem* p) {
  BEC_TRY(launch_publish_scalars(p));
  return BEC_OK;
}
}  // namespace

// z = P_eps^{-1} (s y), s = *scale_dev (1 if null)
bec_status apply_pinv(bec_problem* p, const double* y, double* z, const double* scale_dev) {
  NvtxRange range("bec P_eps^-1");
  const int fp64 = p->desc.precision == BEC_PC_FP64;
  if (p->desc.route == BEC_ROUTE_MG || p->desc.route == BEC_ROUTE_LEARNED) {
    // the learned route's step alpha is fixed (and the correction judged) by
    // a calibration apply whenever the weights, eps or the judge setting
    // changed; a rejected correction is skipped
    const bool learned = p->desc.route == BEC_ROUTE_LEARNED && !net_bypassed(p);
    if (learned && !net_calibrated(p)) BEC_TRY(net_calibrate(p));
    BEC_TRY(launch_time_fwd(p, y, p->mg.lv[0].b, fp64, scale_dev));
    BEC_TRY(mg_vcycle(p));
    if (learned && !net_rejected(p)) BEC_TRY(net_correct(p));
    return launch_time_inv(p, p->mg.lv[0].x, z, fp64);
  }
  const double n = (double)(p->m + 1);
  const double per_axis = (2.0 / n) / 16.0;   // (orthonormal / raw)^2 for one forward+inverse pair
  double scale = 0.5 / p->N;
  for (int d = 0; d < p->dim; ++d) scale *= per_axis;
  const long long rows = p->J / p->m * p->N;    // lines along x
  if (fp64) {
    BEC_TRY(launch_dst_rows(p, y, 1, z, 1, rows, 1));
    if (p->dim >= 2) BEC_TRY(launch_dst_cols(p, z, 1));
    BEC_TRY(launch_time_pass(p, z, 1, scale, scale_dev));
    if (p->dim >= 2) BEC_TRY(launch_dst_cols(p, z, 1));
    BEC_TRY(launch_dst_rows(p, z, 1, z, 1, rows, 1));
  } else {
    void* s = p->pc_scratch;
    BEC_TRY(launch_dst_rows(p, y, 1, s, 0, rows, 0));
    if (p->dim >= 2) BEC_TRY(launch_dst_cols(p, s, 0));
    BEC_TRY(launch_time_pass(p, s, 0, scale, scale_dev));
    if (p->dim >= 2) BEC_TRY(launch_dst_cols(p, s, 0));
    BEC_TRY(launch_dst_rows(p, s, 0, z, 1, rows, 0));
  }
  return BEC_OK;
}

void gmres_run_init(GmresRun& r, bec_problem* p, const double* f, double* u,
                    const bec_gmres_opts& o, bool use_graphs) {
  r = GmresRun();
  r.p = p;
  r.f = f;
  r.u = u;
  r.o = o;
  r.use_graphs = use_graphs;
  r.x_nonzero = o.use_x0 != 0;
  const int R = o.restart;
  r.Vp.resize(R + 1);
  r.Zp.resize(R);
  for (int i = 0; i <= R; ++i) r.Vp[i] = p->V + (long long)i * p->U;
  for (int i = 0; i < R && o.flexible; ++i) r.Zp[i] = p->Z + (long long)i * p->U;
  r.state = GmresRun::BEGIN;
}

namespace {

// The body of one Arnoldi iteration j, ending with the scalar read.
bec_status iteration_body(GmresRun& r) {
  bec_problem* p = r.p;
  const int j = r.j;
  double* sigma = p->sigma;
  double* h1 = p->hcol;
  double* h2 = p->hcol + (p->max_restart + 2);
  double* vnext = p->V + (long long)(j + 1) * p->U;
  if (r.o.left_pc) {
    BEC_TRY(launch_apply_L(p, r.Vp[j], p->t, 0.0, sigma + j));
    BEC_TRY(apply_pinv(p, p->t, p->w, nullptr));
    BEC_TRY(launch_dots(p, p->w, r.Vp.data(), j + 1, sigma, h1));
    // classical Gram-Schmidt, second pass fused with the first update
    BEC_TRY(launch_update_dots(p, p->w, r.Vp.data(), j + 1, sigma, h1, h2));
    BEC_TRY(launch_combine(p, vnext, p->w, r.Vp.data(), j + 1, sigma, h2, -1.0, S_W));
    BEC_TRY(launch_hessenberg(p, j, h1, h2, S_W, S_RES));
    return enqueue_scalar_read(p);
  }
  // Right preconditioning: Arnoldi on A - I with A = L P^{-1} (same Krylov
  // space, H(A) = H(A - I) + I).  w = L z_j - v_j no longer carries the
  // dominant v_j component of a near-identity A, so one classical
  // Gram-Schmidt pass is kept unless the test of Daniel, Gragg, Kaufman and
  // Stewart (||w after|| < ||w before|| / sqrt 2) asks for a second one; that
  // decision is taken on the device.
  double* z = r.o.flexible ? p->Z + (long long)j * p->U : p->t;
  if (!r.ext_pinv) BEC_TRY(apply_pinv(p, r.Vp[j], z, sigma + j));
  BEC_TRY(launch_stencil_dots(p, z, p->w, r.Vp.data(), j + 1, sigma, h1, r.Vp[j], sigma + j, S_WB));
  BEC_TRY(launch_combine(p, vnext, p->w, r.Vp.data(), j + 1, sigma, h1, -1.0, S_W));
  BEC_TRY(launch_reorth_flag(p, S_WB, S_W));
  BEC_TRY(launch_dots(p, vnext, r.Vp.data(), j + 1, sigma, h2, p->flag));
  BEC_TRY(launch_combine(p, vnext, vnext, r.Vp.data(), j + 1, sigma, h2, -1.0, S_W, p->flag));
  BEC_TRY(launch_hessenberg(p, j, h1, h2, S_W, S_RES, 1.0));
  return enqueue_scalar_read(p);
}

// Enqueue iteration j, from the problem's graph cache when graphs are used.
bec_status enqueue_iteration(GmresRun& r) {
  NvtxRange range("bec Arnoldi iteration");
  bec_problem* p = r.p;
  if (!r.use_graphs) return iteration_body(r);
  const int mode = (r.o.left_pc ? 1 : 0) | (r.o.flexible ? 2 : 0) | (r.ext_pinv ? 4 : 0);
  if (p->graph_mode != mode || (int)p->graphs.size() < r.o.restart) {
    for (auto& g : p->graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    p->graphs.assign(p->max_restart, IterGraph());
    p->graph_mode = mode;
  }
  IterGraph& g = p->graphs[r.j];
  if (g.exec == nullptr) {
    if (!g.warm) {   // first use runs eagerly (one-time attribute setting, lazy loading)
      g.warm = true;
      return iteration_body(r);
    }
    const long long before = p->launches;
    const bool prof = p->prof.on;
    p->prof.on = false;
    BEC_CUDA_TRY(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    const bec_status s = iteration_body(r);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->stream, &graph);
    p->prof.on = prof;
    if (s != BEC_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      g.exec = nullptr;
      return cuda_fail(ei, "cudaGraphInstantiate");
    }
    g.kernels = p->launches - before;
    p->launches = before;
  }
  BEC_CUDA_TRY(cudaGraphLaunch(g.exec, p->stream));
  p->launches += g.kernels;
  return BEC_OK;
}

}  // namespace

// Advance one step.  `enqueued` tells the caller that work ending in a
// scalar read was put on the stream and the next call must come after the
// stream has drained.
bec_status gmres_run_step(GmresRun& r, bool* enqueued) {
  bec_problem* p = r.p;
  *enqueued = false;
  switch (r.state) {
    case GmresRun::BEGIN: {   // reference norm: ||f|| (right) or ||P^{-1} f|| (left)
      if (r.o.left_pc) {
        BEC_TRY(apply_pinv(p, r.f, p->t, nullptr));
        BEC_TRY(launch_norm(p, p->t, S_REF));
      } else {
        BEC_TRY(launch_norm(p, r.f, S_REF));
      }
      if (!r.o.use_x0) BEC_TRY(launch_zero(p, r.u));
      BEC_TRY(enqueue_scalar_read(p));
      r.state = GmresRun::AFTER_BEGIN;
      *enqueued = true;
      return BEC_OK;
    }
    case GmresRun::AFTER_BEGIN: {
      r.ref = p->host_scal[S_REF];
      if (!std::isfinite(r.ref)) {
        set_error("right-hand side contains NaN or Inf");
        r.state = GmresRun::DONE;
        return r.status = BEC_ENUMERIC;
      }
      if (r.ref == 0.0) {
        BEC_TRY(launch_zero(p, r.u));
        r.converged = true;
        r.zero_rhs = true;
        r.state = GmresRun::DONE;
        return BEC_OK;
      }
      r.state = GmresRun::CYCLE;
      return BEC_OK;
    }
    case GmresRun::CYCLE: {   // r0, stored unnormalised in V_0
      r.beta_slot = S_BETA;
      if (r.x_nonzero) {
        BEC_TRY(launch_residual(p, r.f, r.u, p->V));
        r.Vp[0] = p->V;
      } else if (!r.o.left_pc && !r.use_graphs) {
        r.Vp[0] = r.f;            // alias the caller's f (read only)
        r.beta_slot = S_REF;
      } else {
        if (!r.o.left_pc) BEC_TRY(launch_copy(p, r.f, p->V));
        r.Vp[0] = p->V;
      }
      if (r.o.left_pc) BEC_TRY(apply_pinv(p, r.x_nonzero ? p->V : r.f, p->V, nullptr));
      if (r.beta_slot == S_BETA) {
        BEC_TRY(launch_norm(p, r.Vp[0], S_BETA));
        BEC_TRY(enqueue_scalar_read(p));
        *enqueued = true;
      }
      r.state = GmresRun::AFTER_CYCLE;
      return BEC_OK;
    }
    case GmresRun::AFTER_CYCLE: {
      const double beta = r.beta_slot == S_BETA ? p->host_scal[S_BETA] : r.ref;
      if (!std::isfinite(beta)) {
        set_error("NaN or Inf in the GMRES residual");
        r.state = GmresRun::DONE;
        return r.status = BEC_ENUMERIC;
      }
      r.monitored = beta / r.ref;
      if (beta <= r.o.rtol * r.ref) {
        r.converged = true;
        r.state = GmresRun::FINISH;
        return BEC_OK;
      }
      if (r.iters >= r.o.maxit) {
        r.state = GmresRun::FINISH;
        return BEC_OK;
      }
      BEC_TRY(launch_gmres_start(p, r.beta_slot));
      r.j = 0;
      r.k = 0;
      r.state = GmresRun::ITER;
      return BEC_OK;
    }
    case GmresRun::ITER: {
      BEC_TRY(enqueue_iteration(r));
      r.state = GmresRun::AFTER_ITER;
      *enqueued = true;
      return BEC_OK;
    }
    case GmresRun::AFTER_ITER: {
      const double res = p->host_scal[S_RES];
      ++r.iters;
      r.k = r.j + 1;
      if (!std::isfinite(res)) {
        set_error("NaN or Inf in the GMRES recurrences");
        r.state = GmresRun::DONE;
        return r.status = BEC_ENUMERIC;
      }
      r.monitored = res / r.ref;
      if (res <= r.o.rtol * r.ref) r.converged = true;
      const bool stop = r.converged || r.iters >= r.o.maxit;
      if (!stop && r.j + 1 < r.o.restart) {
        ++r.j;
        r.state = GmresRun::ITER;
        return BEC_OK;
      }
      // end of the cycle: least squares and the solution update
      BEC_TRY(launch_least_squares(p, r.k));
      double* sigma = p->sigma;
      if (r.o.left_pc) {
        BEC_TRY(launch_combine(p, r.u, r.u, r.Vp.data(), r.k, sigma, p->ycoef, 1.0, -1));
      } else if (r.o.flexible) {
        BEC_TRY(launch_combine(p, r.u, r.u, r.Zp.data(), r.k, nullptr, p->ycoef, 1.0, -1));
      } else {
        BEC_TRY(launch_combine(p, p->t, nullptr, r.Vp.data(), r.k, sigma, p->ycoef, 1.0, -1));
        BEC_TRY(apply_pinv(p, p->t, p->w, nullptr));
        const double* wl[1] = {p->w};
        BEC_TRY(launch_combine(p, r.u, r.u, wl, 1, nullptr, p->scal + S_ONE, 1.0, -1));
      }
      r.x_nonzero = true;
      if (stop) {
        r.state = GmresRun::FINISH;
      } else {
        ++r.restarts;
        r.state = GmresRun::CYCLE;
      }
      return BEC_OK;
    }
    case GmresRun::FINISH: {
      BEC_TRY(launch_residual_norms(p, r.f, r.u, S_TRUE));
      BEC_TRY(enqueue_scalar_read(p));
      r.state = GmresRun::AFTER_FINISH;
      *enqueued = true;
      return BEC_OK;
    }
    case GmresRun::AFTER_FINISH: {
      r.true_relres = p->host_scal[S_TRUE] / p->host_scal[S_TRUE + 1];
      r.state = GmresRun::DONE;
      return BEC_OK;
    }
    case GmresRun::DONE:
      return r.status;
  }
  return BEC_OK;
}

void gmres_run_pinv_operands(const GmresRun& r, const double** y, double** z,
                             const double** scale_dev) {
  bec_problem* p = r.p;
  *y = r.Vp[r.j];
  *z = r.o.flexible ? p->Z + (long long)r.j * p->U : p->t;
  *scale_dev = p->sigma + r.j;
}

void gmres_run_info(const GmresRun& r, bec_gmres_info* info) {
  if (info == nullptr) return;
  std::memset(info, 0, sizeof(*info));
  info->iters = r.iters;
  info->restarts = r.restarts;
  info->converged = r.converged ? 1 : 0;
  info->prec_relres = r.zero_rhs ? 0.0 : r.monitored;
  info->true_relres = r.zero_rhs ? 0.0 : r.true_relres;
}

bec_status gmres_run_result(const GmresRun& r) {
  if (r.status != BEC_OK) return r.status;
  return r.converged ? BEC_OK : BEC_ENOTCONV;
}

bec_status gmres_solve_one(bec_problem* p, const double* f, double* u, const bec_gmres_opts* o,
                           bec_gmres_info* info) {
  BEC_TRY(net_prepare(p));
  GmresRun r;
  gmres_run_init(r, p, f, u, *o, false);
  while (r.state != GmresRun::DONE) {
    bool enq = false;
    const bec_status s = gmres_run_step(r, &enq);
    if (s != BEC_OK) return s;
    if (enq) BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  }
  gmres_run_info(r, info);
  if (p->net) BEC_TRY(net_check(p));
  BEC_TRY(pc_check(p));
  return gmres_run_result(r);
}

}  // namespace bec
