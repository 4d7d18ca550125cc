// Internal declarations shared by the translation units of libbec.
#pragma once

#include <cuda_bf16.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "bec.h"
#include <nvtx3/nvToolsExt.h>

namespace bec {

// NVTX range for the duration of a scope (host thread; visible in Nsight
// timelines, a no-op without a tool attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Tables for one transform length n: twiddles e^{-2 pi i j / n}, j < n.
struct FftTables {
  int n = 0, logn = 0;
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
};

// Block widths (warps per block) of the P_eps^{-1} passes: the defaults, and
// a problem's tuned choice (0 = the default; see bec_autotune).
constexpr int kRowsWarps = 8;
constexpr int default_cols_warps(int tsize) { return tsize == 8 ? 8 : 16; }
constexpr int default_time_warps(int tsize) { return tsize == 8 ? 8 : 16; }
struct TileChoice {
  int rows = 0, cols = 0, time = 0;
};

// Everything the preconditioner kernels read besides the vectors.
struct PcTables {
  FftTables space;           // n = nx + 1
  FftTables time;            // n = N
  double* sin2_64 = nullptr; // 2 sin(j pi / n), j < n   (DST-I pre-pass)
  float* sin2_32 = nullptr;
  double* mu64 = nullptr;    // 1D stiffness eigenvalues mu_i, i = 1..m (times a)
  float* mu32 = nullptr;
  double* mum64 = nullptr;   // 1D mass eigenvalues (Q1 elements only; null: M = I)
  float* mum32 = nullptr;
  double* es64 = nullptr;    // eps^{j/N}, j < N
  double* eis64 = nullptr;   // eps^{-j/N}
  float* es32 = nullptr;
  float* eis32 = nullptr;
  double2* lamf64 = nullptr; // 1 - eps^{1/N} e^{-2 pi i k / N}, k = 0..N/2
  float2* lamf32 = nullptr;
  // [J][N/2+1]: 1 / |lambda'_k + tau mu_q|^2, FP64 sine-transform route only
  // (replaces a division per mode and frequency in the ALU-bound time pass)
  double* rinv64 = nullptr;
};

// Event pairs around kernel launches (bec_profile_start / bec_profile_stop).
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;       // 2 per record
  std::vector<const char*> names;    // 1 per record
  int used = 0;                      // records completed
  int pending = -1;                  // record whose start event is in flight
  long long overflow = 0;
};

// One multigrid level: real Galerkin stencils and complex work arrays for
// all N/2+1 frequencies, in the preconditioner's precision.
struct MgLevel {
  int m = 0;
  long long J = 0;
  void* SM = nullptr;   // [9][J] mass stencil (level 0: identity)
  void* SK = nullptr;   // [9][J] stiffness stencil
  void* x = nullptr;    // [K][J] complex
  void* b = nullptr;
  void* r = nullptr;
  void* dinv = nullptr; // [K][J] complex: 1 / D of the ILU smoother (BEC_MG_ILU)
  void* ilu_nb = nullptr;   // [2][J][8] real: the M and K entries towards the lower
                            // (W, S, SE, SW) and upper (E, N, NW, NE) neighbours
};

struct MgState {
  int pre = 1, post = 1;
  double omega = 0.8;
  int ilu = 0;          // smoother: 0 damped Jacobi, 1 ILU
  int K = 0;            // N/2 + 1 frequencies
  std::vector<MgLevel> lv;
};

struct NetState;   // learned correction (bec_net.cu)

// One Arnoldi iteration captured as a CUDA graph (batched solves).
struct IterGraph {
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;   // kernel launches inside the graph
  bool warm = false;       // ran eagerly once
};

}  // namespace bec

struct bec_problem {
  bec_problem_desc desc;
  int dim = 0, m = 0, N = 0;
  long long J = 0, U = 0;
  double tau = 0.0, h = 0.0, a = 1.0;
  double eps = -1.0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int max_restart = 30;
  long long launches = 0;

  bec::PcTables tab;
  bec::TileChoice tile;         // block widths of the P_eps^{-1} passes
  void* pc_scratch = nullptr;   // N x Jp elements of the preconditioner's type
  // Row length and points per time slice of pc_scratch: in FP32 every row
  // of m values gets one zero pad slot (ld = m + 1), so that rows and time
  // slices start on 16-byte boundaries (tensor-memory-access tiles); else
  // ld = m, Jp = J.
  int ld = 0;
  long long Jp = 0;
  int* pc_err = nullptr;        // device word: a bounded wait of the time pass ran out
  bool time_map_ok = false;     // time_map describes pc_scratch for the N = 256 time pass
  CUtensorMap time_map;
  bool cols_map_ok = false;     // cols_map describes pc_scratch for the n = 256 column pass
  CUtensorMap cols_map;

  // Krylov workspace (FP64)
  double* V = nullptr;          // (max_restart + 1) x U
  double* Z = nullptr;          // max_restart x U (flexible only)
  double* w = nullptr;          // U
  double* t = nullptr;          // U
  double* partials = nullptr;   // reduction partials
  double* hcol = nullptr;       // two Gram-Schmidt coefficient columns, 2 x (max_restart + 2)
  double* H = nullptr;          // (max_restart + 1) x max_restart, column-major
  double* cs = nullptr;         // Givens cosines
  double* sn = nullptr;         // Givens sines
  double* g = nullptr;          // rotated right-hand side (max_restart + 1)
  double* ycoef = nullptr;      // least-squares solution (max_restart)
  double* sigma = nullptr;      // 1 / ||stored V_i||: V_i is kept unnormalised (max_restart + 1)
  int* flag = nullptr;          // device flag: second Gram-Schmidt pass needed
  double* scal = nullptr;       // device scalars (norms, residual estimate)
  double* host_scal = nullptr;  // mapped pinned mirror of scal (host address)
  double* host_scal_dev = nullptr;   // its device address
  double* io_f = nullptr;       // host_io staging
  double* io_u = nullptr;
  double* io_f2 = nullptr;      // second staging pair (bec_gmres_solve_host_many)
  double* io_u2 = nullptr;
  cudaStream_t copy_stream = nullptr;   // host <-> device copies of the pipelined solves
  cudaEvent_t io_ev[4] = {nullptr, nullptr, nullptr, nullptr};   // loaded[2], solved[2]
  bec::Profiler prof;
  double* kcoef = nullptr;      // variable a: tau K row [centre, W, E, S, N] x J
  double* bcoef = nullptr;      // multigrid route: -tau x the couplings of each point to
                                // its W, E, S, N boundary nodes, [4][J] (0 if interior)
  bec::MgState mg;              // BEC_ROUTE_MG hierarchy
  bec::NetState* net = nullptr;  // BEC_ROUTE_LEARNED network
  std::vector<bec::IterGraph> graphs;   // per Arnoldi index j (batched solves)
  int graph_mode = -1;          // left / flexible flags the graphs were captured with
};

namespace bec {

// Restarted (F)GMRES as a resumable state machine (bec_gmres.cpp).
struct GmresRun {
  enum State { BEGIN, AFTER_BEGIN, CYCLE, AFTER_CYCLE, ITER, AFTER_ITER, FINISH, AFTER_FINISH, DONE };
  bec_problem* p = nullptr;
  const double* f = nullptr;
  double* u = nullptr;
  bec_gmres_opts o{};
  bool use_graphs = false;
  // the P_eps^{-1} of each Arnoldi step is enqueued by the caller (a batch's
  // persistent launch for all instances), not by the iteration itself
  bool ext_pinv = false;
  State state = BEGIN;
  bec_status status = BEC_OK;
  double ref = 0.0, monitored = 1.0, true_relres = 0.0;
  int iters = 0, restarts = 0, j = 0, k = 0, beta_slot = 1;
  bool converged = false, x_nonzero = false, zero_rhs = false;
  std::vector<const double*> Vp, Zp;
};
void gmres_run_init(GmresRun& r, bec_problem* p, const double* f, double* u,
                    const bec_gmres_opts& o, bool use_graphs);
bec_status gmres_run_step(GmresRun& r, bool* enqueued);
// Operands of the P_eps^{-1} of the coming Arnoldi step (state ITER, right
// preconditioning): z = P^{-1} (s y) with s = *scale_dev.
void gmres_run_pinv_operands(const GmresRun& r, const double** y, double** z,
                             const double** scale_dev);
void gmres_run_info(const GmresRun& r, bec_gmres_info* info);
bec_status gmres_run_result(const GmresRun& r);
bec_status gmres_solve_one(bec_problem* p, const double* f, double* u,
                           const bec_gmres_opts* o, bec_gmres_info* info);
bec_status check_gmres_opts(const bec_problem* p, const bec_gmres_opts* o);
// z = P_eps^{-1} (s y), s = *scale_dev (1 if null)
bec_status apply_pinv(bec_problem* p, const double* y, double* z, const double* scale_dev);

}  // namespace bec

namespace bec {

constexpr int kReduceBlocks = 608;   // 4 x 152 SMs: fixed => deterministic sums
constexpr int kStencilDotBlocks = 1216;  // 8 x 152: fused stencil + dots grid
constexpr int kScalSlots = 16;
constexpr int kMaxRestart = 60;
constexpr int kMaxVec = 32;          // vectors one fused Krylov launch handles

// Krylov basis vectors handed to a kernel by value.
struct VecList {
  const double* v[kMaxVec];
};

// ---- error plumbing
void set_error(const std::string& msg);
bec_status cuda_fail(cudaError_t e, const char* where);
#define BEC_CUDA_TRY(expr)                                            \
  do {                                                                \
    cudaError_t _e = (expr);                                          \
    if (_e != cudaSuccess) return ::bec::cuda_fail(_e, #expr);        \
  } while (0)
void prof_begin(bec_problem* p);
void prof_end(bec_problem* p, const char* name);
// Call BEC_LAUNCH_BEGIN(p) right before a kernel launch and
// BEC_LAUNCH_CHECK(p, name) right after it.
#define BEC_LAUNCH_BEGIN(p) ::bec::prof_begin(p)
#define BEC_LAUNCH_CHECK(p, where)                                    \
  do {                                                                \
    (p)->launches++;                                                  \
    cudaError_t _e = cudaGetLastError();                              \
    if (_e != cudaSuccess) return ::bec::cuda_fail(_e, where);        \
    ::bec::prof_end(p, where);                                        \
  } while (0)

// ---- preconditioner passes (bec_dst.cu, bec_time.cu)
// Each pass runs with the problem's tuned block width (p->tile); the _w
// variants take an explicit width (4, 8 or 16 warps; 0 = the default).
// DST-I (unnormalised, times 4) along x of `rows` contiguous rows of length m.
bec_status launch_dst_rows(bec_problem* p, const void* in, int in_fp64,
                           void* out, int out_fp64, long long rows, int fp64);
bec_status launch_dst_rows_w(bec_problem* p, const void* in, int in_fp64, void* out,
                             int out_fp64, long long rows, int fp64, int w);
// DST-I (same scaling) along y of every [ny][nx] slice, in place.
bec_status launch_dst_cols(bec_problem* p, void* data, int fp64);
bec_status launch_dst_cols_w(bec_problem* p, void* data, int fp64, int w);
// Time pass: scale, FFT over N, divide by the shifted eigenvalues, inverse
// FFT, unscale, for every spatial mode, in place.  The divide is multiplied by
// `scale` and, when scale_dev is not null, by the device scalar *scale_dev.
// true when the FP32 time pass runs as the four-step N = 256 kernel (no
// tunable block width)
bool time16_applies(const bec_problem* p);
// describes pc_scratch to the TMA unit for that kernel (at allocation;
// leaves time_map_ok false when the layout or the driver does not allow it)
bec_status time16_make_map(bec_problem* p);
// the same for the FP32 2D column pass with n = 256 (dst_cols16_tma_kernel)
bec_status cols16_make_map(bec_problem* p);
bool cols16_applies(const bec_problem* p);
// BEC_ETIMEOUT (and clears the word) when a bounded wait of the time pass
// ran out since the last check; synchronises the problem's stream
bec_status pc_check(bec_problem* p);
bec_status launch_time_pass(bec_problem* p, void* data, int fp64, double scale,
                            const double* scale_dev);
bec_status launch_time_pass_w(bec_problem* p, void* data, int fp64, double scale,
                              const double* scale_dev, int w);
// rinv64[q][k] = 1 / |lambda'_k + tau mu_q|^2 from the current lambda' table
bec_status launch_rinv_table(bec_problem* p);
// y = x converted between FP64 and FP32 (to_float: double -> float) by the
// integer conversions of the FP32 passes
// y = 1/x by the FP64 reciprocal of the multigrid smoother (rcp64)
cudaError_t launch_rcp64(const double* x, double* y, long long n, cudaStream_t st);
cudaError_t launch_convert(const void* x, void* y, long long n, int to_float, cudaStream_t st);
// the shared memory pass `which` (0 x-DST, 1 y-DST, 2 time pass) needs at
// block width w (0 = the default)
size_t pass_smem_bytes(int which, int logn, int fp64, int w);
// bec_autotune / bec_set_tiles (bec_tune.cu)
bec_status autotune(bec_problem* p, int force, bec_tune_report* rep);
bec_status set_tiles(bec_problem* p, int rows, int cols, int time);

// ---- multigrid route (bec_mg.cu, bec_time.cu)
// Builds the coefficient rows, the Galerkin hierarchy and its buffers.
bec_status mg_setup(bec_problem* p, const double* a_nodes, const double* wind);
// the ILU smoother's 1 / D for every level and frequency (after the eps tables)
bec_status mg_ilu_setup(bec_problem* p);
// f = tau (fsrc - K_b g) + u0 in slice 1 (multigrid route)
bec_status launch_build_rhs_dirichlet(bec_problem* p, const double* u0, const double* fsrc,
                                      const double* g, double* f);
void mg_free(bec_problem* p);
// One V-cycle for every frequency: level-0 b -> level-0 x.
bec_status mg_vcycle(bec_problem* p);
// The same from level l0 (level-l0 b -> level-l0 x); l0 below the coarsest.
bec_status mg_vcycle_from(bec_problem* p, int l0);
// r = b - B x on level l for every frequency ([K][J_l] complex arrays)
bec_status mg_residual_level(bec_problem* p, int l, void* r, const void* x, const void* b);
// bc = R rf from level lf to level lf + 1, every frequency
bec_status mg_restrict_to(bec_problem* p, int lf, void* bc, const void* rf);
// r = b - B x on the finest level for every frequency ([K][J] complex arrays)
bec_status mg_residual_level0(bec_problem* p, void* r, const void* x, const void* b);
// xo = x + omega D^{-1} (b - B x) on the finest grid, every frequency (xo != x)
bec_status mg_smooth_level0(bec_problem* p, void* xo, const void* x, const void* b);
// spec[k][q] = sum_j e^{-2 pi i jk/N} eps^{j/N} (s y)[j][q], k <= N/2 (s = *scale_dev or 1)
bec_status launch_time_fwd(bec_problem* p, const double* y, void* spec, int fp64,
                           const double* scale_dev);
// z[j][q] = eps^{-j/N} N^{-1} sum_k spec_k e^{2 pi i jk/N} (Hermitian extension)
bec_status launch_time_inv(bec_problem* p, const void* spec, double* z, int fp64);

// ---- persistent batched P_eps^{-1} (bec_persist.cu)
constexpr int kPersistMaxJobs = 64;
// One instance's FP32 sine-transform P_eps^{-1} of one round: z = P^{-1} (s y).
struct PersistJob {
  const double* y;
  double* z;
  float* s;                    // the instance's FP32 scratch (N Jp floats, rows of ld)
  const double* scale_dev;     // s (null: 1)
  const float* sin2;
  const float2* tws;           // spatial FFT twiddles
  const float2* twt;           // time FFT twiddles
  const float* es;
  const float* eis;
  const float2* lamf;
  const float* mu;
  long long J;                 // points per time slice of s (the problem's Jp)
  float tau, scale_h;
  int m, ld, N, logn, logt;
  int tiles[5];                // tiles (queue items) of the five passes, 8 warps each
};
// The work queue of one launch, passed by value.
struct PersistQueue {
  int njobs, total;
  int pass_start[6];                          // first item of each pass
  int job_start[5 * (kPersistMaxJobs + 1)];   // first item of (pass p, job i) at p (njobs + 1) + i
  int target[5 * kPersistMaxJobs];            // tiles a pass must report before the next starts
};
// FP32, sine transform, 2D, finite differences, backward Euler, sides 31..255, N 4..512
bool persist_supported(const bec_problem* p);
void persist_make_job(const bec_problem* p, const double* y, double* z, const double* scale_dev,
                      PersistJob* j);
// Enqueues on `st`: the copy of the jobs to jobs_dev, the reset of the
// counters ctr_dev (4 + 5 njobs ints; ctr_dev[1] is the error word) and one
// persistent launch.  withhold != 0: a test of the bounded waits (instance
// 0's first pass never completes, so the launch ends with the error word set).
bec_status persist_launch(const PersistJob* jobs_host, PersistJob* jobs_dev, int njobs,
                          PersistQueue* q, int* ctr_dev, int withhold, cudaStream_t st);
// test hook (bec_inject_fault): the next launch withholds instance 0's first
// pass; persist_take_withhold returns and clears the request
void persist_withhold_next();
int persist_take_withhold();

// ---- learned correction (bec_net.cu)
bec_status net_setup(bec_problem* p, const double* a_nodes, int channels, int fp32_acts, int bmax);
void net_free(bec_problem* p);
bec_status net_correct(bec_problem* p);   // after the V-cycle: x += alpha (corrected - x)
// the calibration apply that fixes alpha and judges the correction (it uses
// the level-0 multigrid arrays: call it before an apply's Step 1);
// net_calibrated: alpha matches the weights, eps and the judge setting;
// net_invalidate: they changed
bec_status net_calibrate(bec_problem* p);
bool net_calibrated(const bec_problem* p);
void net_invalidate(bec_problem* p);
// the route acts as the multigrid route alone (during the training's recording solve)
bool net_bypassed(const bec_problem* p);
bec_status net_train(bec_problem* p, int steps, int batch, float lr, unsigned long long seed,
                     double* loss_hist);
long long net_num_weights(const bec_problem* p);
bec_status net_get_weights(bec_problem* p, float* host);
bec_status net_set_weights(bec_problem* p, const float* host);
bec_status net_loss_grad(bec_problem* p, int B, const int* lams, const double* r, const double* et,
                         double* loss_out, float* grad_host);
long long net_fallbacks(bec_problem* p);
// BEC_ETIMEOUT (and clears the flag) when a bounded device wait of the
// network's kernels ran out since the last check; synchronises.
bec_status net_check(bec_problem* p);

// ---- tensor-core convolutions (bec_conv_tc.cu): every layer of the network,
// BF16 NHWC activations, tcgen05 MMA with TMA-staged halo tiles
bool tc_conv_supported();
// test hook: the next tensor-core convolution withholds its tile loads
void tc_withhold_next_loads();
// the next TMA-staged FP32 pass (time or column) issues no tile load (test
// hook, one-shot); tma_take_withhold returns and clears the request
void tma_withhold_next();
int tma_take_withhold();
// BF16 elements of the converted weights of all 9 layers
int tc_weights_elems();
// the operand layout of every layer from the FP32 master weights W (layer l
// at W + woff[l], [tap][c_in][c_out]); host array woff of 9 offsets
bec_status tc_convert_weights(bec_problem* p, const float* W, const long long* woff,
                              __nv_bfloat16* wt);
// output channels of the learned correction's network: one real plane per pole
constexpr int kNetOut = 8;
// out = conv3x3(in) of layer l (no activation), times the layer's gate
// (channel-major, [32][m^2]) when gate is not null (layers 0..7): l = 0 reads the 16-channel
// padded input planes, l = 8 stores its kNetOut output channels
bec_status tc_conv3x3(bec_problem* p, int layer, const __nv_bfloat16* in, const __nv_bfloat16* wt,
                      __nv_bfloat16* out, const float* gate, int m, int B, int bmax, int* err);
bec_status net_residual_ratios(bec_problem* p, double* host);
// the calibration's spectral-radius test on (default) or off; recalibrates
void net_set_judge(bec_problem* p, bool on);
// the last calibration fell back to the V-cycle's iterates (alpha = 0)
bool net_rejected(const bec_problem* p);
// calibrates the learned route now when it is due (before a solve starts,
// outside any graph capture); a no-op for other routes
bec_status net_prepare(bec_problem* p);
// per-frequency radii (V-cycle, corrected) and their maxima, 2K + 2 doubles
bec_status net_judge_radii(bec_problem* p, double* host);

// ---- stencils (bec_stencil.cu)
// number of blocks (partial sums) the residual-norm kernel writes
long long stencil_blocks(const bec_problem* p);
// y = L v; with corner != 0, y = P_eps v (adds -corner * v^N to slice 1);
// with out_scale != null the result is multiplied by the device scalar.
bec_status launch_apply_L(bec_problem* p, const double* v, double* y,
                          double corner, const double* out_scale = nullptr);
// w = L z - s vshift (s = *sshift; no shift if vshift is null) and
// hout[i] = sigma_i <V_i, w> for i < nv in one pass over z, w, V; with
// norm_slot >= 0 also scal[norm_slot] = ||w||.
bec_status launch_stencil_dots(bec_problem* p, const double* z, double* w,
                               const double* const* V, int nv,
                               const double* sigma, double* hout,
                               const double* vshift = nullptr,
                               const double* sshift = nullptr, int norm_slot = -1);
bec_status launch_build_rhs(bec_problem* p, const double* u0,
                            const double* fsrc, double* f);
// partials[b] = sum over block b of (f - L u)^2, partials[B + b] = sum f^2;
// then scal[slot] = sqrt(sum r^2), scal[slot+1] = sqrt(sum f^2).
bec_status launch_residual_norms(bec_problem* p, const double* f,
                                 const double* u, int slot);
// r = f - L u (u may be null: r = f)
bec_status launch_residual(bec_problem* p, const double* f, const double* u,
                           double* r);

// ---- Krylov BLAS (bec_krylov.cu).  V is a host array of nv device
// pointers; sigma (device, may be null = all ones) scales V_i.
// hout[i] = sigma_i <V_i, w>; with flag != null and *flag == 0 on the
// device, nothing is computed and hout = 0 (a skipped reorthogonalisation).
bec_status launch_dots(bec_problem* p, const double* w, const double* const* V,
                       int nv, const double* sigma, double* hout,
                       const int* flag = nullptr);
// scal[slot] = sqrt(sum of nb partials) (skipped when flag && !*flag)
bec_status launch_finish_sqrt(bec_problem* p, const double* parts, int nb, int slot,
                              const int* flag);
// *flag = (scal[after] < scal[before] / sqrt(2)): the second Gram-Schmidt pass
// is needed (the test of Daniel, Gragg, Kaufman and Stewart)
bec_status launch_reorth_flag(bec_problem* p, int before_slot, int after_slot);
// w -= sum_i coef_i sigma_i V_i, then hout[i] = sigma_i <V_i, w>
bec_status launch_update_dots(bec_problem* p, double* w,
                              const double* const* V, int nv,
                              const double* sigma, const double* coef,
                              double* hout);
// out = w + sign sum_i coef_i sigma_i V_i (w may be null = 0, out may be w);
// if norm_slot >= 0 also scal[norm_slot] = ||out||.
bec_status launch_combine(bec_problem* p, double* out, const double* w,
                          const double* const* V, int nv, const double* sigma,
                          const double* coef, double sign, int norm_slot,
                          const int* flag = nullptr);
// dots of a finished partial array: hout[i] = sigma_i sum_b partials[i nb + b]
bec_status launch_finish_dots(bec_problem* p, int nv, int nb,
                              const double* sigma, double* hout,
                              const int* flag = nullptr);
// scal[slot] = ||x||
bec_status launch_norm(bec_problem* p, const double* x, int slot);
// Hessenberg column j: H(0:j, j) = h1 + h2 (the two Gram-Schmidt passes),
// H(j+1, j) = scal[norm_slot] and sigma[j+1] = 1 / H(j+1, j); applies the
// previous rotations, makes rotation j, updates g and writes |g[j+1]| to
// scal[res_slot].
bec_status launch_hessenberg(bec_problem* p, int j, const double* h1,
                             const double* h2, int norm_slot, int res_slot,
                             double shift = 0.0);
// g = (scal[slot], 0, ...), sigma[0] = 1 / scal[slot].
bec_status launch_gmres_start(bec_problem* p, int slot);
// ycoef = H(0:k,0:k)^{-1} g(0:k)
bec_status launch_least_squares(bec_problem* p, int k);
bec_status launch_copy(bec_problem* p, const double* x, double* y);
// copies the kScalSlots scalars to the mapped host mirror with a kernel, so
// that the read never queues behind a large copy on a copy engine
bec_status launch_publish_scalars(bec_problem* p);
bec_status launch_zero(bec_problem* p, double* x);

}  // namespace bec
