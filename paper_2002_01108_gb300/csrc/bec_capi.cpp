// C ABI of libbec: problem set-up, the preconditioner apply of Sec. 4, the
// all-at-once operator of Sec. 2 and restarted (F)GMRES of Sec. 5.  Host code
// only: every arithmetic step runs in the kernels of the other units.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bec_internal.h"

namespace bec {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

bec_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return BEC_ECUDA;
}

void prof_begin(bec_problem* p) {
  Profiler& f = p->prof;
  if (!f.on) return;
  if ((size_t)(2 * f.used + 2) > f.ev.size()) {
    f.overflow++;
    f.pending = -1;
    return;
  }
  cudaEventRecord(f.ev[2 * f.used], p->stream);
  f.pending = f.used;
}

void prof_end(bec_problem* p, const char* name) {
  Profiler& f = p->prof;
  if (!f.on || f.pending < 0) return;
  cudaEventRecord(f.ev[2 * f.pending + 1], p->stream);
  f.names[f.pending] = name;
  f.used++;
  f.pending = -1;
}

namespace {

constexpr double kPi = 3.14159265358979323846;

// device scalar slots
constexpr int S_REF = 0, S_BETA = 1, S_W = 2, S_RES = 3, S_TRUE = 4, S_ONE = 15;

bool is_pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2(long long x) {
  int l = 0;
  while ((1LL << l) < x) ++l;
  return l;
}

bec_status einval(const char* msg) {
  set_error(msg);
  return BEC_EINVAL;
}

template <typename T>
bec_status dmalloc(T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) return BEC_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return BEC_ENOMEM;
  }
  return BEC_OK;
}

template <typename T>
bec_status upload(T* dst, const std::vector<T>& src, cudaStream_t s) {
  BEC_CUDA_TRY(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return BEC_OK;
}

void destroy_profiler(bec_problem* p) {
  for (cudaEvent_t e : p->prof.ev) cudaEventDestroy(e);
  p->prof.ev.clear();
  p->prof.names.clear();
  p->prof.used = 0;
  p->prof.pending = -1;
  p->prof.on = false;
}

void free_all(bec_problem* p) {
  destroy_profiler(p);
  net_free(p);
  mg_free(p);
  for (auto& g : p->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  p->graphs.clear();
  PcTables& t = p->tab;
  void* ptrs[] = {t.space.tw64, t.space.tw32, t.time.tw64, t.time.tw32, t.sin2_64, t.sin2_32,
                  t.mu64, t.mu32, t.mum64, t.mum32, t.es64, t.eis64, t.es32, t.eis32,
                  t.lamf64, t.lamf32, t.rinv64, p->pc_scratch, p->pc_err, p->V, p->Z, p->w, p->t, p->partials, p->hcol, p->H, p->cs,
                  p->sn, p->g, p->ycoef, p->sigma, p->flag, p->scal, p->io_f, p->io_u,
                  p->io_f2, p->io_u2};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->host_scal) cudaFreeHost(p->host_scal);
  for (cudaEvent_t& e : p->io_ev)
    if (e) cudaEventDestroy(e);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
}

// e^{-2 pi i j / n}, j < n
void twiddles(int n, std::vector<double2>& t64, std::vector<float2>& t32) {
  t64.resize(n);
  t32.resize(n);
  for (int j = 0; j < n; ++j) {
    const double a = -2.0 * kPi * j / n;
    t64[j] = make_double2(std::cos(a), std::sin(a));
    t32[j] = make_float2((float)t64[j].x, (float)t64[j].y);
  }
}

bec_status read_scalars(bec_problem* p) {
  const bec_status s = launch_publish_scalars(p);
  if (s != BEC_OK) return s;
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return BEC_OK;
}

#define BEC_TRY(expr)                  \
  do {                                 \
    bec_status _s = (expr);            \
    if (_s != BEC_OK) return _s;       \
  } while (0)

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }
bool aligned8(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 7u) == 0; }

bec_status check_vec(const void* q) {
  if (q == nullptr) return einval("null vector pointer");
  if (!aligned8(q)) return einval("vector pointer not 8-byte aligned");
  return BEC_OK;
}

bool overlap(const bec_problem* p, const double* a, const double* b) {
  return a < b + p->U && b < a + p->U;
}

}  // namespace

bec_status check_gmres_opts(const bec_problem* p, const bec_gmres_opts* o) {
  if (o == nullptr) return einval("null options");
  if (o->restart < 1 || o->restart > p->max_restart)
    return einval("restart must be in [1, max_restart]");
  if (o->maxit < 1) return einval("maxit must be >= 1");
  if (!(o->rtol >= 0.0) || !std::isfinite(o->rtol)) return einval("rtol must be finite and >= 0");
  if (o->flexible && p->Z == nullptr) return einval("flexible GMRES needs desc.flexible");
  if (o->flexible && o->left_pc) return einval("flexible GMRES is right-preconditioned");
  if (p->desc.precision == BEC_PC_FP32 && !o->flexible)
    return einval("the FP32 preconditioner is inexact: use flexible GMRES");
  if (p->eps <= 0.0) return einval("call bec_set_eps first");
  return BEC_OK;
}

}  // namespace bec

using namespace bec;

extern "C" {

bec_status bec_allocate_problem(const bec_problem_desc* d, void* stream, bec_problem** out) {
  if (d == nullptr || out == nullptr) return einval("null argument");
  *out = nullptr;
  if (d->dim < 1 || d->dim > 3) return einval("dim must be 1, 2 or 3");
  if (!is_pow2((long long)d->nx + 1) || d->nx + 1 < 4 || d->nx + 1 > 1024)
    return einval("nx + 1 must be a power of two in [4, 1024]");
  if (d->dim >= 2 && d->ny != d->nx) return einval("dim 2 and 3 need ny == nx");
  if (!is_pow2(d->N) || d->N < 2 || d->N > 1024)
    return einval("N must be a power of two in [2, 1024]");
  if (!(d->T > 0.0) || !std::isfinite(d->T)) return einval("T must be finite and > 0");
  if (!(d->a > 0.0) || !std::isfinite(d->a)) return einval("a must be finite and > 0");
  if (d->route != BEC_ROUTE_FST && d->route != BEC_ROUTE_MG && d->route != BEC_ROUTE_LEARNED)
    return einval("route must be BEC_ROUTE_FST, BEC_ROUTE_MG or BEC_ROUTE_LEARNED");
  const bool mgroute = d->route == BEC_ROUTE_MG || d->route == BEC_ROUTE_LEARNED;
  if (d->route == BEC_ROUTE_FST && d->a_nodes != nullptr)
    return einval("a variable coefficient (a_nodes) needs BEC_ROUTE_MG or BEC_ROUTE_LEARNED");
  if (mgroute && d->dim != 2) return einval("the multigrid route is 2D");
  if (mgroute && d->N > 512) return einval("the multigrid route needs N <= 512");
  if (d->route == BEC_ROUTE_LEARNED) {
    if (d->precision != BEC_PC_FP32) return einval("the learned route needs BEC_PC_FP32");
    if (d->nx < 31) return einval("the learned route needs nx >= 31");
    if (d->net_channels != 0 && d->net_channels != 4 && d->net_channels != 32)
      return einval("net_channels must be 0, 4 or 32");
  }
  if (d->mg_pre < 0 || d->mg_post < 0 || d->mg_pre > 8 || d->mg_post > 8)
    return einval("mg_pre and mg_post must lie in [0, 8]");
  if (!(d->mg_omega >= 0.0) || d->mg_omega >= 2.0) return einval("mg_omega must lie in [0, 2)");
  if (d->precision != BEC_PC_FP64 && d->precision != BEC_PC_FP32)
    return einval("precision must be BEC_PC_FP64 or BEC_PC_FP32");
  if (d->max_restart < 0 || d->max_restart > kMaxRestart)
    return einval("max_restart must be in [0, 60]");
  if (d->space != BEC_SPACE_FD && d->space != BEC_SPACE_Q1)
    return einval("space must be BEC_SPACE_FD or BEC_SPACE_Q1");
  if (d->space == BEC_SPACE_Q1 && d->route != BEC_ROUTE_FST)
    return einval("Q1 elements need BEC_ROUTE_FST");
  if (d->space == BEC_SPACE_Q1 && d->dim == 3) return einval("Q1 elements are 1D or 2D");
  if (d->route != BEC_ROUTE_MG && (d->wind != nullptr || (d->side != 0.0 && d->side != 1.0)))
    return einval("wind and side need BEC_ROUTE_MG");
  if (!(d->side >= 0.0) || !std::isfinite(d->side)) return einval("side must be finite and >= 0");
  if (d->mg_smoother != BEC_MG_JACOBI && d->mg_smoother != BEC_MG_ILU)
    return einval("mg_smoother must be BEC_MG_JACOBI or BEC_MG_ILU");
  if (d->mg_smoother == BEC_MG_ILU && d->route != BEC_ROUTE_MG)
    return einval("the ILU smoother needs BEC_ROUTE_MG");
  if (d->mg_smoother == BEC_MG_ILU && d->precision == BEC_PC_FP64 && d->nx > 511)
    return einval("the FP64 ILU smoother needs nx <= 511 (its shared-memory staging)");
  if (d->time_scheme != BEC_TIME_BDF1 && d->time_scheme != BEC_TIME_BDF2)
    return einval("time_scheme must be BEC_TIME_BDF1 or BEC_TIME_BDF2");
  if (d->time_scheme == BEC_TIME_BDF2 && (d->route != BEC_ROUTE_FST || d->dim == 3 || d->N < 4))
    return einval("BDF2 needs BEC_ROUTE_FST, dim 1 or 2 and N >= 4");

  bec_problem* p = new (std::nothrow) bec_problem();
  if (p == nullptr) return BEC_ENOMEM;
  p->desc = *d;
  p->dim = d->dim;
  p->m = d->nx;
  p->N = d->N;
  p->J = d->nx;
  for (int k = 1; k < d->dim; ++k) p->J *= d->nx;
  p->U = p->J * d->N;
  p->tau = d->T / d->N;
  p->h = 1.0 / (d->nx + 1);
  p->a = d->a;
  p->stream = static_cast<cudaStream_t>(stream);
  p->max_restart = d->max_restart == 0 ? 30 : d->max_restart;
  cudaGetDevice(&p->device);

  const int n = p->m + 1, N = p->N, R = p->max_restart;
  PcTables& t = p->tab;
  t.space.n = n;
  t.space.logn = ilog2(n);
  t.time.n = N;
  t.time.logn = ilog2(N);
  const long long U = p->U;
  const long long parts = std::max<long long>(
      std::max<long long>((long long)kMaxVec * kReduceBlocks, (long long)kMaxVec * kStencilDotBlocks),
      2 * stencil_blocks(p));
  bec_status s = BEC_OK;
  auto chain = [&](bec_status r) {
    if (s == BEC_OK) s = r;
  };
  chain(dmalloc(&t.space.tw64, n));
  chain(dmalloc(&t.space.tw32, n));
  chain(dmalloc(&t.time.tw64, N));
  chain(dmalloc(&t.time.tw32, N));
  chain(dmalloc(&t.sin2_64, n));
  chain(dmalloc(&t.sin2_32, n));
  chain(dmalloc(&t.mu64, p->m));
  chain(dmalloc(&t.mu32, p->m));
  if (d->space == BEC_SPACE_Q1) {
    chain(dmalloc(&t.mum64, p->m));
    chain(dmalloc(&t.mum32, p->m));
  }
  chain(dmalloc(&t.es64, N));
  chain(dmalloc(&t.eis64, N));
  chain(dmalloc(&t.es32, N));
  chain(dmalloc(&t.eis32, N));
  chain(dmalloc(&t.lamf64, N / 2 + 1));
  chain(dmalloc(&t.lamf32, N / 2 + 1));
  if (d->precision == BEC_PC_FP64 && d->route == BEC_ROUTE_FST)
    chain(dmalloc(&t.rinv64, (size_t)p->J * (N / 2 + 1)));
  if (mgroute && s == BEC_OK) {
    p->mg.pre = d->mg_pre == 0 ? 1 : d->mg_pre;
    p->mg.post = (d->mg_pre == 0 && d->mg_post == 0) ? 1 : d->mg_post;
    p->mg.omega = d->mg_omega == 0.0 ? 0.8 : d->mg_omega;
    p->mg.ilu = d->mg_smoother == BEC_MG_ILU;
    chain(mg_setup(p, d->a_nodes, d->wind));
    if (d->route == BEC_ROUTE_LEARNED && s == BEC_OK)
      // inference runs all N/2 + 1 frequencies in one batch up to 160 of them
      // (training batches stay at most 32); each frequency takes two network
      // samples (r and i r)
      chain(net_setup(p, d->a_nodes, d->net_channels == 0 ? 32 : d->net_channels, d->net_fp32,
                      2 * std::max(32, std::min(p->N / 2 + 1, 160))));
  }
  p->desc.a_nodes = nullptr;   // copied by mg_setup; the caller keeps its array
  p->desc.wind = nullptr;
  p->ld = p->m;
  p->Jp = p->J;
  if (d->precision == BEC_PC_FP32 && d->route == BEC_ROUTE_FST) {
    // rows of m + 1 slots (the last one zero): 16-byte aligned rows and time
    // slices for the TMA tiles of the time pass
    p->ld = p->m + 1;
    p->Jp = p->J / p->m * p->ld;
    float* sc = nullptr;
    chain(dmalloc(&sc, (size_t)N * p->Jp));
    p->pc_scratch = sc;
    chain(dmalloc(&p->pc_err, (size_t)1));
    if (s == BEC_OK) {
      const cudaError_t e = cudaMemset(p->pc_err, 0, sizeof(int));
      if (e != cudaSuccess) s = cuda_fail(e, "cudaMemset");
    }
    // the TMA time pass moves tiles of 32 points of a slice; thinner slices
    // keep the kernel whose threads load the tile
    if (s == BEC_OK && p->Jp >= 32) s = time16_make_map(p);
    if (s == BEC_OK) s = cols16_make_map(p);
  }
  chain(dmalloc(&p->V, (size_t)(R + 1) * U));
  if (d->flexible) chain(dmalloc(&p->Z, (size_t)R * U));
  chain(dmalloc(&p->w, (size_t)U));
  chain(dmalloc(&p->t, (size_t)U));
  chain(dmalloc(&p->partials, (size_t)parts));
  chain(dmalloc(&p->hcol, (size_t)2 * (R + 2)));
  chain(dmalloc(&p->H, (size_t)(R + 1) * R));
  chain(dmalloc(&p->cs, (size_t)R));
  chain(dmalloc(&p->sn, (size_t)R));
  chain(dmalloc(&p->g, (size_t)R + 1));
  chain(dmalloc(&p->ycoef, (size_t)R));
  chain(dmalloc(&p->sigma, (size_t)R + 1));
  chain(dmalloc(&p->flag, (size_t)1));
  chain(dmalloc(&p->scal, (size_t)kScalSlots));
  if (d->host_io) {
    chain(dmalloc(&p->io_f, (size_t)U));
    chain(dmalloc(&p->io_u, (size_t)U));
    chain(dmalloc(&p->io_f2, (size_t)U));
    chain(dmalloc(&p->io_u2, (size_t)U));
    if (s == BEC_OK) {
      cudaError_t e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking);
      for (int i = 0; i < 4 && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&p->io_ev[i], cudaEventDisableTiming);
      if (e != cudaSuccess) s = cuda_fail(e, "copy stream / events");
    }
  }
  if (s == BEC_OK) {
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&p->host_scal),
                                  kScalSlots * sizeof(double), cudaHostAllocMapped);
    if (e == cudaSuccess)
      e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&p->host_scal_dev), p->host_scal, 0);
    if (e != cudaSuccess) {
      if (p->host_scal) cudaFreeHost(p->host_scal);
      cudaGetLastError();
      p->host_scal = nullptr;
      set_error("cudaHostAlloc of the scalar mirror failed");
      s = BEC_ENOMEM;
    }
  }
  if (s != BEC_OK) {
    free_all(p);
    delete p;
    return s;
  }

  // tables that do not depend on eps
  std::vector<double2> tw64;
  std::vector<float2> tw32;
  twiddles(n, tw64, tw32);
  chain(upload(t.space.tw64, tw64, p->stream));
  chain(upload(t.space.tw32, tw32, p->stream));
  std::vector<double2> ttw64;
  std::vector<float2> ttw32;
  twiddles(N, ttw64, ttw32);
  chain(upload(t.time.tw64, ttw64, p->stream));
  chain(upload(t.time.tw32, ttw32, p->stream));
  std::vector<double> s64(n), mu64(p->m);
  std::vector<float> s32(n), mu32(p->m);
  for (int j = 0; j < n; ++j) {
    s64[j] = 2.0 * std::sin(j * kPi / n);
    s32[j] = (float)s64[j];
  }
  // 1D eigenvalues on the sine basis, k = 1..m: FD stiffness (4a/h^2)
  // sin^2(k pi h / 2); Q1 stiffness a (4/h) sin^2(k pi h / 2) and mass
  // (h/3)(2 + cos(k pi h)) (the tridiagonal Toeplitz K1 and M1)
  const bool q1 = d->space == BEC_SPACE_Q1;
  std::vector<double> mum64(p->m);
  std::vector<float> mum32(p->m);
  for (int k = 1; k <= p->m; ++k) {
    const double sk = std::sin(k * kPi * p->h / 2.0);
    mu64[k - 1] = (q1 ? 4.0 * p->a / p->h : 4.0 * p->a / (p->h * p->h)) * sk * sk;
    mu32[k - 1] = (float)mu64[k - 1];
    mum64[k - 1] = p->h / 3.0 * (2.0 + std::cos(k * kPi * p->h));
    mum32[k - 1] = (float)mum64[k - 1];
  }
  chain(upload(t.sin2_64, s64, p->stream));
  chain(upload(t.sin2_32, s32, p->stream));
  chain(upload(t.mu64, mu64, p->stream));
  chain(upload(t.mu32, mu32, p->stream));
  if (q1) {
    chain(upload(t.mum64, mum64, p->stream));
    chain(upload(t.mum32, mum32, p->stream));
  }
  std::vector<double> scal0(kScalSlots, 0.0);
  scal0[S_ONE] = 1.0;
  chain(upload(p->scal, scal0, p->stream));
  if (s == BEC_OK) {
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaStreamSynchronize");
  }
  if (s != BEC_OK) {
    free_all(p);
    delete p;
    return s;
  }
  *out = p;
  return BEC_OK;
}

bec_status bec_set_eps(bec_problem* p, double eps) {
  if (p == nullptr) return einval("null problem");
  if (!(eps > 0.0 && eps <= 1.0)) return einval("eps must lie in (0, 1]");
  net_invalidate(p);   // the learned route's steps depend on lambda'_k
  const int N = p->N;
  std::vector<double> es(N), eis(N);
  std::vector<float> es32(N), eis32(N);
  const double le = std::log(eps);
  for (int j = 0; j < N; ++j) {
    es[j] = std::exp(le * j / N);
    eis[j] = std::exp(-le * j / N);
    es32[j] = (float)es[j];
    eis32[j] = (float)eis[j];
  }
  // lambda'_k = sum_j r_j eps^{j/N} e^{-2 pi i j k / N}, the eigenvalue that
  // pairs with the forward-sign FFT (lambda_{N-k} of eq. repsdiagform):
  // 1 - eps^{1/N} e^{-2 pi i k/N} for BDF1 (r = (1, -1)), and for BDF2
  // (r = (3/2, -2, 1/2)) the same sum over j = 0, 1, 2
  const double e1 = std::exp(le / N);
  const bool bdf2 = p->desc.time_scheme == BEC_TIME_BDF2;
  std::vector<double2> lam(N / 2 + 1);
  std::vector<float2> lam32(N / 2 + 1);
  for (int k = 0; k <= N / 2; ++k) {
    const double a = 2.0 * kPi * k / N;
    double re, im;
    if (!bdf2) {
      re = 1.0 - e1 * std::cos(a);
      im = e1 * std::sin(a);
      if (k == 0) re = 1.0 - e1, im = 0.0;
      if (2 * k == N) re = 1.0 + e1, im = 0.0;
    } else {
      const double e2 = std::exp(2.0 * le / N);
      re = 1.5 - 2.0 * e1 * std::cos(a) + 0.5 * e2 * std::cos(2.0 * a);
      im = 2.0 * e1 * std::sin(a) - 0.5 * e2 * std::sin(2.0 * a);
      if (k == 0) re = 1.5 - 2.0 * e1 + 0.5 * e2, im = 0.0;
      if (2 * k == N) re = 1.5 + 2.0 * e1 + 0.5 * e2, im = 0.0;
    }
    lam[k] = make_double2(re, im);
    lam32[k] = make_float2((float)re, (float)im);
  }
  const PcTables& t = p->tab;
  BEC_TRY(upload(t.es64, es, p->stream));
  BEC_TRY(upload(t.eis64, eis, p->stream));
  BEC_TRY(upload(t.es32, es32, p->stream));
  BEC_TRY(upload(t.eis32, eis32, p->stream));
  BEC_TRY(upload(t.lamf64, lam, p->stream));
  BEC_TRY(upload(t.lamf32, lam32, p->stream));
  if (t.rinv64) BEC_TRY(launch_rinv_table(p));
  if (p->mg.ilu) BEC_TRY(mg_ilu_setup(p));
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  p->eps = eps;
  return BEC_OK;
}

bec_status bec_apply_A(bec_problem* p, const double* v, double* y) {
  if (p == nullptr) return einval("null problem");
  BEC_TRY(check_vec(v));
  BEC_TRY(check_vec(y));
  if (overlap(p, v, y)) return einval("v and y must not overlap");
  return launch_apply_L(p, v, y, 0.0);
}

bec_status bec_apply_P(bec_problem* p, const double* v, double* y) {
  if (p == nullptr) return einval("null problem");
  if (p->eps <= 0.0) return einval("call bec_set_eps first");
  BEC_TRY(check_vec(v));
  BEC_TRY(check_vec(y));
  if (overlap(p, v, y)) return einval("v and y must not overlap");
  return launch_apply_L(p, v, y, p->eps);
}

bec_status bec_apply_Pinv(bec_problem* p, const double* y, double* z) {
  if (p == nullptr) return einval("null problem");
  if (p->eps <= 0.0) return einval("call bec_set_eps first");
  BEC_TRY(check_vec(y));
  BEC_TRY(check_vec(z));
  if (y != z && overlap(p, y, z)) return einval("y and z must be equal or disjoint");
  return apply_pinv(p, y, z, nullptr);
}

bec_status bec_build_rhs(bec_problem* p, const double* u0, const double* fsrc, double* f) {
  if (p == nullptr) return einval("null problem");
  BEC_TRY(check_vec(u0));
  BEC_TRY(check_vec(fsrc));
  BEC_TRY(check_vec(f));
  return launch_build_rhs(p, u0, fsrc, f);
}

bec_status bec_build_rhs_dirichlet(bec_problem* p, const double* u0, const double* fsrc,
                                   const double* g, double* f) {
  if (p == nullptr) return einval("null problem");
  if (p->bcoef == nullptr) return einval("bec_build_rhs_dirichlet needs BEC_ROUTE_MG");
  BEC_TRY(check_vec(u0));
  BEC_TRY(check_vec(fsrc));
  BEC_TRY(check_vec(g));
  BEC_TRY(check_vec(f));
  return launch_build_rhs_dirichlet(p, u0, fsrc, g, f);
}

bec_status bec_gmres_solve(bec_problem* p, const double* f, double* u, const bec_gmres_opts* opts,
                           bec_gmres_info* info) {
  if (p == nullptr) return einval("null problem");
  BEC_TRY(check_gmres_opts(p, opts));
  if (f == nullptr || u == nullptr) return einval("null vector pointer");
  if (!aligned16(f) || !aligned16(u)) return einval("f and u must be 16-byte aligned");
  if (overlap(p, f, u)) return einval("f and u must not overlap");
  return gmres_solve_one(p, f, u, opts, info);
}

bec_status bec_gmres_solve_host(bec_problem* p, const double* f_host, double* u_host,
                                const bec_gmres_opts* opts, bec_gmres_info* info) {
  if (p == nullptr) return einval("null problem");
  if (p->io_f == nullptr) return einval("bec_gmres_solve_host needs desc.host_io");
  BEC_TRY(check_gmres_opts(p, opts));
  if (f_host == nullptr || u_host == nullptr) return einval("null host pointer");
  const size_t bytes = (size_t)p->U * sizeof(double);
  BEC_CUDA_TRY(cudaMemcpyAsync(p->io_f, f_host, bytes, cudaMemcpyHostToDevice, p->stream));
  if (opts->use_x0)
    BEC_CUDA_TRY(cudaMemcpyAsync(p->io_u, u_host, bytes, cudaMemcpyHostToDevice, p->stream));
  const bec_status s = gmres_solve_one(p, p->io_f, p->io_u, opts, info);
  if (s != BEC_OK && s != BEC_ENOTCONV) return s;
  BEC_CUDA_TRY(cudaMemcpyAsync(u_host, p->io_u, bytes, cudaMemcpyDeviceToHost, p->stream));
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return s;
}

bec_status bec_gmres_solve_host_many(bec_problem* p, const double* const* f_host,
                                     double* const* u_host, int count, const bec_gmres_opts* opts,
                                     bec_gmres_info* infos) {
  if (p == nullptr) return einval("null problem");
  if (p->io_f2 == nullptr) return einval("bec_gmres_solve_host_many needs desc.host_io");
  BEC_TRY(check_gmres_opts(p, opts));
  if (opts->use_x0) return einval("bec_gmres_solve_host_many starts every solve from zero");
  if (count < 1 || f_host == nullptr || u_host == nullptr) return einval("bad right-hand side list");
  for (int i = 0; i < count; ++i)
    if (f_host[i] == nullptr || u_host[i] == nullptr) return einval("null host pointer");
  const size_t bytes = (size_t)p->U * sizeof(double);
  double* F[2] = {p->io_f, p->io_f2};
  double* Ub[2] = {p->io_u, p->io_u2};
  cudaEvent_t* loaded = p->io_ev;
  cudaEvent_t* solved = p->io_ev + 2;
  cudaStream_t cs = p->copy_stream;
  // Solve i uses buffer pair i % 2.  The copy stream loads f of solve i + 1
  // while solve i runs, and reads u of solve i back while solve i + 1 runs.
  for (int i = 0; i < count && i < 2; ++i) {
    BEC_CUDA_TRY(cudaMemcpyAsync(F[i], f_host[i], bytes, cudaMemcpyHostToDevice, cs));
    BEC_CUDA_TRY(cudaEventRecord(loaded[i], cs));
  }
  bec_status worst = BEC_OK;
  for (int i = 0; i < count; ++i) {
    const int b = i & 1;
    BEC_CUDA_TRY(cudaStreamWaitEvent(p->stream, loaded[b], 0));
    bec_gmres_info local;
    const bec_status s = gmres_solve_one(p, F[b], Ub[b], opts, infos ? &infos[i] : &local);
    if (s != BEC_OK && s != BEC_ENOTCONV) {
      cudaStreamSynchronize(cs);
      return s;
    }
    if (s == BEC_ENOTCONV) worst = s;
    BEC_CUDA_TRY(cudaEventRecord(solved[b], p->stream));
    BEC_CUDA_TRY(cudaStreamWaitEvent(cs, solved[b], 0));
    BEC_CUDA_TRY(cudaMemcpyAsync(u_host[i], Ub[b], bytes, cudaMemcpyDeviceToHost, cs));
    if (i + 2 < count) {
      BEC_CUDA_TRY(cudaMemcpyAsync(F[b], f_host[i + 2], bytes, cudaMemcpyHostToDevice, cs));
      BEC_CUDA_TRY(cudaEventRecord(loaded[b], cs));
    }
  }
  BEC_CUDA_TRY(cudaStreamSynchronize(cs));
  return worst;
}

bec_status bec_true_relres(bec_problem* p, const double* f, const double* u, double* out) {
  if (p == nullptr || out == nullptr) return einval("null argument");
  BEC_TRY(check_vec(f));
  BEC_TRY(check_vec(u));
  BEC_TRY(launch_residual_norms(p, f, u, S_TRUE));
  BEC_TRY(read_scalars(p));
  *out = p->host_scal[S_TRUE] / p->host_scal[S_TRUE + 1];
  return BEC_OK;
}

bec_status bec_free_problem(bec_problem* p) {
  if (p == nullptr) return BEC_OK;
  cudaStreamSynchronize(p->stream);
  free_all(p);
  delete p;
  return BEC_OK;
}

long long bec_problem_size(const bec_problem* p) { return p ? p->U : 0; }

long long bec_kernel_launches(const bec_problem* p) { return p ? p->launches : 0; }

bec_status bec_profile_start(bec_problem* p, int capacity) {
  if (p == nullptr || capacity < 1) return einval("null problem or capacity < 1");
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  destroy_profiler(p);
  p->prof.ev.resize((size_t)2 * capacity);
  for (auto& e : p->prof.ev) {
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) {
      e = nullptr;
      p->prof.ev.clear();
      return cuda_fail(err, "cudaEventCreate");
    }
  }
  p->prof.names.assign((size_t)capacity, nullptr);
  p->prof.overflow = 0;
  p->prof.on = true;
  return BEC_OK;
}

bec_status bec_profile_stop(bec_problem* p, bec_kernel_time* out, int cap, int* count) {
  if (p == nullptr || count == nullptr || (out == nullptr && cap > 0))
    return einval("null argument");
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  std::vector<bec_kernel_time> agg;
  for (int i = 0; i < p->prof.used; ++i) {
    float ms = 0.f;
    BEC_CUDA_TRY(cudaEventElapsedTime(&ms, p->prof.ev[2 * i], p->prof.ev[2 * i + 1]));
    const char* nm = p->prof.names[i];
    auto it = std::find_if(agg.begin(), agg.end(),
                           [nm](const bec_kernel_time& k) { return std::strcmp(k.name, nm) == 0; });
    if (it == agg.end()) {
      agg.push_back(bec_kernel_time{nm, 1, (double)ms});
    } else {
      it->launches++;
      it->ms += ms;
    }
  }
  destroy_profiler(p);
  *count = (int)agg.size();
  for (int i = 0; i < (int)agg.size() && i < cap; ++i) out[i] = agg[i];
  return BEC_OK;
}

long long bec_learned_num_weights(const bec_problem* p) { return p ? net_num_weights(p) : 0; }

static bec_status need_net(const bec_problem* p) {
  if (p == nullptr || p->net == nullptr) return einval("not a BEC_ROUTE_LEARNED problem");
  return BEC_OK;
}

bec_status bec_learned_get_weights(bec_problem* p, float* host) {
  BEC_TRY(need_net(p));
  if (host == nullptr) return einval("null host pointer");
  return net_get_weights(p, host);
}

bec_status bec_learned_set_weights(bec_problem* p, const float* host) {
  BEC_TRY(need_net(p));
  if (host == nullptr) return einval("null host pointer");
  return net_set_weights(p, host);
}

bec_status bec_learned_train(bec_problem* p, int steps, int batch, double lr,
                             unsigned long long seed, double* loss_history) {
  BEC_TRY(need_net(p));
  if (steps < 0 || batch < 1 || batch > 32 || !(lr > 0.0)) return einval("bad training arguments");
  if (p->eps <= 0.0) return einval("call bec_set_eps first");
  return net_train(p, steps, batch, (float)lr, seed, loss_history);
}

bec_status bec_learned_loss_grad(bec_problem* p, int B, const int* lam_idx, const double* r,
                                 const double* e_target, double* loss, float* grad) {
  BEC_TRY(need_net(p));
  if (lam_idx == nullptr || r == nullptr || e_target == nullptr || loss == nullptr)
    return einval("null argument");
  if (B < 1 || B > 32) return einval("B must lie in [1, 32]");
  for (int b = 0; b < B; ++b)
    if (lam_idx[b] < 0 || lam_idx[b] > p->N / 2) return einval("frequency index out of range");
  if (p->eps <= 0.0) return einval("call bec_set_eps first");
  return net_loss_grad(p, B, lam_idx, r, e_target, loss, grad);
}

long long bec_learned_fallbacks(bec_problem* p) {
  if (p == nullptr || p->net == nullptr) return -1;
  return net_fallbacks(p);
}

bec_status bec_learned_set_judge(bec_problem* p, int on) {
  BEC_TRY(need_net(p));
  net_set_judge(p, on != 0);
  return BEC_OK;
}

bec_status bec_learned_judge_radii(bec_problem* p, double* host) {
  BEC_TRY(need_net(p));
  if (host == nullptr) return einval("null host pointer");
  return net_judge_radii(p, host);
}

bec_status bec_learned_residual_ratios(bec_problem* p, double* host) {
  BEC_TRY(need_net(p));
  if (host == nullptr) return einval("null host pointer");
  return net_residual_ratios(p, host);
}

bec_status bec_inject_fault(int kind) {
  if (kind == BEC_FAULT_NONE) return BEC_OK;
  if (kind == BEC_FAULT_TC_WITHHOLD_LOADS) {
    tc_withhold_next_loads();
    return BEC_OK;
  }
  if (kind == BEC_FAULT_PERSIST_WITHHOLD) {
    persist_withhold_next();
    return BEC_OK;
  }
  if (kind == BEC_FAULT_TMA_WITHHOLD_LOADS) {
    tma_withhold_next();
    return BEC_OK;
  }
  return einval("unknown fault kind");
}

bec_status bec_autotune(bec_problem* p, int force, bec_tune_report* report) {
  if (p == nullptr) return einval("null problem");
  return autotune(p, force, report);
}

bec_status bec_set_tiles(bec_problem* p, int rows_warps, int cols_warps, int time_warps) {
  if (p == nullptr) return einval("null problem");
  return set_tiles(p, rows_warps, cols_warps, time_warps);
}

bec_status bec_convert_to_float(const double* x, float* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (x == nullptr || y == nullptr))) return einval("bad conversion arguments");
  const cudaError_t e = launch_convert(x, y, n, 1, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? BEC_OK : cuda_fail(e, "convert_kernel_f32");
}

bec_status bec_convert_to_double(const float* x, double* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (x == nullptr || y == nullptr))) return einval("bad conversion arguments");
  const cudaError_t e = launch_convert(x, y, n, 0, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? BEC_OK : cuda_fail(e, "convert_kernel_f64");
}

bec_status bec_reciprocal_fp64(const double* x, double* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (x == nullptr || y == nullptr))) return einval("bad reciprocal arguments");
  const cudaError_t e = launch_rcp64(x, y, n, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? BEC_OK : cuda_fail(e, "rcp64_kernel");
}

const char* bec_status_string(bec_status s) {
  switch (s) {
    case BEC_OK: return "BEC_OK";
    case BEC_EINVAL: return "BEC_EINVAL";
    case BEC_ENOMEM: return "BEC_ENOMEM";
    case BEC_ECUDA: return "BEC_ECUDA";
    case BEC_ENOTCONV: return "BEC_ENOTCONV";
    case BEC_ENUMERIC: return "BEC_ENUMERIC";
    case BEC_ETIMEOUT: return "BEC_ETIMEOUT";
    case BEC_EUNSUPPORTED: return "BEC_EUNSUPPORTED";
  }
  return "BEC_UNKNOWN";
}

const char* bec_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
