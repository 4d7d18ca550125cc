/*
 * bec.h -- C ABI of the GB300 (sm_103a) library for the block epsilon-circulant
 * (BEC) all-at-once preconditioner of Lin & Ng, "An all-at-once preconditioner
 * for evolutionary partial differential equations" (arXiv 2002.01108).
 *
 * Problem (Sec. 2, eqs. heateq/stepsystem/allatoncesystem): the heat equation
 * u_t = div(a grad u) + f on (0,1)^dim, zero Dirichlet data, backward Euler with
 * tau = T/N, finite differences in space (M = I, K = FD Laplacian times a), gives
 *     L u = f,   L = block lower-bidiagonal(A_0 = I + tau K on the diagonal,
 *                                          -I below it),
 *     u = (u^1; ...; u^N),  f = (tau f^1 + u^0; tau f^2; ...; tau f^N).
 * The preconditioner (start of Sec. 3) is P_eps = L - eps E_1 E_N^T, i.e. L with
 * -eps I in block (1, N), eps in (0, 1] (Theorem pinvertibility).
 *
 * Layout of every space-time vector: N slices of J = nx * ny doubles, slice n
 * (n = 1..N) at offset (n-1) J, and inside a slice x fastest ([N][ny][nx]).
 * For dim = 1, J = nx.
 *
 * Conventions for every entry point:
 *  - Vector arguments are DEVICE pointers owned by the caller (except where
 *    marked host), 8-byte aligned, holding U = N * J doubles, on the device
 *    the problem was allocated on.  The library never frees them.
 *  - Work is enqueued on the problem's CUDA stream and is asynchronous, except
 *    bec_gmres_solve / bec_gmres_solve_host / bec_true_relres, which
 *    synchronise that stream to return scalars.
 *  - The apply and solve paths allocate nothing; all workspace is made by
 *    bec_allocate_problem and released by bec_free_problem.
 *  - Invalid arguments return BEC_EINVAL and enqueue nothing.  A CUDA failure
 *    returns BEC_ECUDA; bec_last_error() then describes it.
 *  - A problem object must not be used from two host threads at once.
 */
#ifndef BEC_H
#define BEC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bec_problem bec_problem;

typedef enum {
  BEC_OK = 0,
  BEC_EINVAL = 1,      /* bad argument (size, pointer, eps outside (0,1], ...) */
  BEC_ENOMEM = 2,      /* device or host allocation failed */
  BEC_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  BEC_ENOTCONV = 4,    /* GMRES hit maxit; u and info still hold the best iterate */
  BEC_ENUMERIC = 5,    /* NaN or Inf met in the Krylov recurrences */
  BEC_ETIMEOUT = 6,    /* a bounded device wait ran out */
  BEC_EUNSUPPORTED = 7 /* valid request that the library does not implement */
} bec_status;

/* How P_eps^{-1} solves the shifted spatial systems B_k z = y (Sec. 4, Step 2). */
enum {
  BEC_ROUTE_FST = 0,   /* 2D/1D sine transform: exact for constant a (Sec. 4) */
  BEC_ROUTE_LEARNED = 2, /* BEC_ROUTE_MG plus a learned correction of what each
                          V-cycle leaves, on the grid of spacing 2h:
                          ec_k = sum_j sigma_j / (lambda'_k + sigma_j) Nc_j,
                          8 fixed poles sigma_j > 0, the residue maps Nc_j
                          real operators (the outputs of one 4-level
                          convolutional network of one real plane, applied
                          to the real and imaginary parts; BF16 activations,
                          FP32 accumulation) whose layers are gated by
                          functions of log a only.  So the correction is
                          linear in the residual and analytic in lambda'_k:
                          a dependence on conj(lambda'_k) would come back
                          from Step 3 amplified by up to 1/eps.  Trained on
                          the GPU by bec_learned_train on pairs the
                          multigrid generates; the corrected iterate gets one
                          damped-Jacobi sweep and the step from the V-cycle's
                          iterate towards it is scaled by one alpha for all
                          frequencies, the minimal-residual step of a
                          calibration apply on a fixed right-hand side
                          (alpha = 0: the V-cycle is the fallback).  So
                          P_eps^{-1} stays a fixed linear operator.  Needs
                          BEC_PC_FP32 and nx >= 31. */
  BEC_ROUTE_MG = 1     /* one geometric multigrid V-cycle per shifted system,
                          any positive a (Sec. 4; Example 2 of Sec. 5): bilinear
                          prolongation, full-weighting restriction, Galerkin
                          coarse operators, damped Jacobi smoothing; 2D only.
                          An inexact preconditioner: use flexible GMRES or
                          accept that GMRES sees a fixed linear operator. */
};

/* Arithmetic of the preconditioner apply.  The operator L, the Krylov vectors,
 * the Gram-Schmidt dots and the Hessenberg least squares are always FP64. */
enum {
  BEC_PC_FP64 = 0,     /* transforms and divide in double */
  BEC_PC_FP32 = 1      /* transforms and divide in float / complex64; input and
                          output stay double (an inexact preconditioner, use
                          flexible GMRES) */
};

typedef struct {
  int dim;             /* 1, 2 or 3 (the unit interval, square or cube) */
  int nx, ny;          /* interior points per side (h = 1/(nx+1)); ny must
                          equal nx for dim 2 and 3 (the cube has nx points
                          along z too) and is ignored for dim 1.
                          nx + 1 must be a power of two in [4, 1024]. */
  int N;               /* time steps; a power of two in [2, 1024] */
  double T;            /* final time, tau = T / N */
  double a;            /* constant diffusion coefficient a > 0 */
  int route;           /* BEC_ROUTE_FST */
  int precision;       /* BEC_PC_FP64 or BEC_PC_FP32 */
  int max_restart;     /* largest GMRES restart length a solve may ask for
                          (0 selects 30); sizes the Krylov basis */
  int flexible;        /* nonzero: also allocate the FGMRES basis Z */
  int host_io;         /* nonzero: also allocate the staging vectors used by
                          bec_gmres_solve_host */
  const double* a_nodes; /* HOST array of (nx+2)*(nx+2) values of a(x) > 0 on
                          all grid nodes, boundary included, [iy][ix]; copied.
                          NULL: a is the constant `a`.  The face coefficient
                          between two nodes is the mean of their values
                          (conservative 5-point scheme).  Needs BEC_ROUTE_MG. */
  int mg_pre, mg_post;   /* damped-Jacobi sweeps before / after the coarse
                          correction (0, 0 select 1, 1: the paper's counts) */
  double mg_omega;       /* Jacobi damping (0 selects 0.8) */
  int net_channels;      /* BEC_ROUTE_LEARNED: channels (4 or 32; 0 selects 32) */
  int net_fp32;          /* BEC_ROUTE_LEARNED: nonzero keeps activations in FP32
                            (used to check gradients); default BF16 */
  int space;             /* spatial discretisation: BEC_SPACE_FD (0, M = I and
                            the 3- or 5-point K) or BEC_SPACE_Q1 (linear / bilinear
                            finite elements on the uniform mesh, Sec. 5 Example
                            1: M = M1 (x) M1, K = a (M1 (x) K1 + K1 (x) M1) in 2D,
                            M1 = h/6 tridiag(1, 4, 1), K1 = 1/h tridiag(-1, 2, -1);
                            needs BEC_ROUTE_FST) */
  int time_scheme;       /* BEC_TIME_BDF1 (0, backward Euler, Sec. 2) or
                            BEC_TIME_BDF2 (the two-step backward difference
                            r = (3/2, -2, 1/2) of Sec. 4 eq. pstepscheme and
                            Sec. 5; needs BEC_ROUTE_FST, dim 1 or 2, N >= 4) */
  const double* wind;    /* HOST array of 2*(nx+2)*(nx+2) values, the velocity
                            (w_x then w_y, each [iy][ix] on all nodes), copied;
                            NULL: no convection.  Adds w . grad u to K with
                            first-order upwind differences (Example 3 of Sec. 5
                            with the upwind stencil in place of SUPG elements).
                            Needs BEC_ROUTE_MG. */
  double side;           /* side length of the square domain (0 selects 1);
                            h = side / (nx + 1).  Needs BEC_ROUTE_MG. */
  int mg_smoother;       /* BEC_MG_JACOBI (0, damped Jacobi) or BEC_MG_ILU (the
                            incomplete factorisation (D + L) D^{-1} (D + U) of
                            each shifted system, diag kept, ILU(0) on the
                            5-point finest grid: the ILU smoothing of Examples 2
                            and 3 of Sec. 5).  BEC_MG_ILU needs BEC_ROUTE_MG,
                            and nx <= 511 with BEC_PC_FP64. */
} bec_problem_desc;

enum { BEC_MG_JACOBI = 0, BEC_MG_ILU = 1 };

enum { BEC_SPACE_FD = 0, BEC_SPACE_Q1 = 1 };
enum { BEC_TIME_BDF1 = 0, BEC_TIME_BDF2 = 1 };

/* Validates desc, allocates the workspace (Krylov basis (max_restart+1) x U
 * doubles, Z when flexible, one U-vector of preconditioner scratch, tables)
 * and returns a problem bound to `stream` (a cudaStream_t; NULL = the legacy
 * default stream) on the current device.  eps starts unset. */
bec_status bec_allocate_problem(const bec_problem_desc* desc, void* stream,
                                bec_problem** out);

/* Sets eps in (0, 1] (Theorem pinvertibility) and recomputes the tables of
 * Sec. 4: D_eps = diag(eps^{(k-1)/N}) and lambda_k = sum_j r_j eps^{j/N}
 * theta^{jk} (eq. repsdiagform): 1 - eps^{1/N} theta^k for BDF1, and
 * 3/2 - 2 eps^{1/N} theta^k + 1/2 eps^{2/N} theta^{2k} for BDF2 (the
 * eigenvalues of R_eps of eq. pstepbecpreconditioner).  eps = 1 is the block
 * circulant preconditioner of McDonald, Pestana and Wathen.  Else
 * BEC_EINVAL. */
bec_status bec_set_eps(bec_problem* p, double eps);

/* y = L v (Sec. 2, eq. allatoncesystem): y^n = (I + tau K) v^n - v^{n-1},
 * with no v^0 term.  With BEC_TIME_BDF2 it is L = R (x) M + tau I (x) K of
 * eq. pstepscheme: y^n = (3/2 M + tau K) v^n - 2 M v^{n-1} + 1/2 M v^{n-2},
 * terms before v^1 absent.  v and y must not overlap. */
bec_status bec_apply_A(bec_problem* p, const double* v, double* y);

/* y = P_eps v (start of Sec. 3); as bec_apply_A plus -eps v^N into slice 1
 * (BDF2: the wrapped terms eps r_j M v^{N+n-j} of eq. pstepbecpreconditioner
 * in slices 1 and 2).  A check of bec_apply_Pinv, not part of the solve.
 * v, y must not overlap. */
bec_status bec_apply_P(bec_problem* p, const double* v, double* y);

/* z = P_eps^{-1} y by the three steps of Sec. 4 (eqs. ytild, blockdiaginv,
 * zcompt): scale slice k by eps^{(k-1)/N}, FFT along time, solve the N shifted
 * systems (lambda_k I + tau K) z~ = y~, of which only ceil((N+1)/2) are
 * distinct (half-spectrum remark of Sec. 4), inverse FFT and unscale.  The
 * shifted systems are solved exactly by the 2D sine transform
 * (BEC_ROUTE_FST), or approximately by one multigrid V-cycle each
 * (BEC_ROUTE_MG).  y == z (in place) is allowed; partial overlap is not.
 * Needs bec_set_eps first (else BEC_EINVAL). */
bec_status bec_apply_Pinv(bec_problem* p, const double* y, double* z);

/* f = (tau f^1 + M u^0; tau f^2; ...; tau f^N) (Sec. 2; M = I for finite
 * differences).  u0: J doubles, fsrc: U doubles (the source at t_1..t_N, taken
 * as given: with Q1 elements pass the load vector), f: U doubles.  BDF2: the
 * known terms of the first two block rows move to the right, with the value
 * before u^0 taken equal to u^0 (the paper does not state it):
 * f^1 = tau f^1 + 3/2 M u^0, f^2 = tau f^2 - 1/2 M u^0. */
bec_status bec_build_rhs(bec_problem* p, const double* u0, const double* fsrc,
                         double* f);

/* As bec_build_rhs, with Dirichlet values on the boundary (Example 3 of
 * Sec. 5: the hot wall): f^n = tau (fsrc^n - K_b g^n) (+ u^0 in slice 1),
 * K_b the couplings of the boundary-adjacent points to the boundary nodes.
 * g: device array of N * (nx+2)^2 doubles, the node values at t_1..t_N
 * ([n][iy][ix]; only the boundary nodes are read).  Needs BEC_ROUTE_MG
 * (finite differences with M = I, 2D); else BEC_EINVAL. */
bec_status bec_build_rhs_dirichlet(bec_problem* p, const double* u0, const double* fsrc,
                                   const double* g, double* f);

typedef struct {
  int restart;         /* GMRES(restart); 1 <= restart <= max_restart */
  int maxit;           /* cap on total inner iterations */
  double rtol;         /* stop when the monitored residual <= rtol * reference */
  int flexible;        /* right preconditioning with stored Z (FGMRES); needs
                          desc.flexible.  Required for BEC_PC_FP32. */
  int left_pc;         /* left preconditioning as in Sec. 5 (monitors the
                          preconditioned residual, reference ||P^{-1} f||).
                          0 = right preconditioning (monitors ||f - L u||,
                          reference ||f||). */
  int use_x0;          /* nonzero: u holds the initial guess; else x0 = 0 */
} bec_gmres_opts;

typedef struct {
  int iters;           /* total inner iterations */
  int restarts;        /* completed restart cycles beyond the first */
  int converged;       /* 1 if the monitored residual met rtol */
  double prec_relres;  /* final monitored residual / reference */
  double true_relres;  /* RES = ||f - L u|| / ||f|| (Sec. 5), recomputed */
} bec_gmres_info;

/* Solves L u = f by restarted GMRES preconditioned with P_eps (Sec. 5:
 * zero initial guess unless use_x0, modified stopping rule rtol).  The Arnoldi
 * basis is built with classical Gram-Schmidt applied twice, the least squares
 * by Givens rotations, all in FP64 on the device; the host reads one scalar
 * per iteration.  f and u are device vectors that must not overlap.  Returns
 * BEC_ENOTCONV when maxit is reached (u and info are still written). */
bec_status bec_gmres_solve(bec_problem* p, const double* f, double* u,
                           const bec_gmres_opts* opts, bec_gmres_info* info);

/* As bec_gmres_solve, but f and u are HOST pointers (pinned memory gives the
 * fastest copies); copies in, solves, copies out, synchronises.  Needs
 * desc.host_io. */
bec_status bec_gmres_solve_host(bec_problem* p, const double* f_host,
                                double* u_host, const bec_gmres_opts* opts,
                                bec_gmres_info* info);

/* Solves `count` systems with the same problem, one after another, from host
 * buffers (f_host[i] -> u_host[i], U doubles each; pinned memory gives the
 * fastest copies).  Not a construct of the paper: a serving form.  Two
 * device buffer pairs and a copy stream (allocated with desc.host_io) let
 * the host-to-device copy of f for solve i + 1 and the device-to-host copy
 * of u from solve i - 1 run while solve i computes.  Every solve starts from
 * zero (opts->use_x0 must be 0); infos (may be NULL) receives count records.
 * Returns BEC_ENOTCONV if any solve did not converge (all results are still
 * written), or the first hard error.  Synchronises. */
bec_status bec_gmres_solve_host_many(bec_problem* p, const double* const* f_host,
                                     double* const* u_host, int count,
                                     const bec_gmres_opts* opts, bec_gmres_info* infos);

/* RES = ||f - L u||_2 / ||f||_2 (Sec. 5) computed on the device; writes the
 * value to *out (host) after synchronising the stream. */
bec_status bec_true_relres(bec_problem* p, const double* f, const double* u,
                           double* out);

/* RES = ||f - L u||_2 / ||f||_2 (Sec. 5), WITHOUT allocating anything and
 * without a problem object.  The paper has no counterpart: this exists for
 * callers that cannot allocate device memory at the point where they check a
 * solution -- device memory owned by another allocator (a framework's caching
 * pool), a memory budget fixed at start-up, a no-allocation-after-
 * initialisation policy, or a device that is nearly full.
 *  - Operator covered: only the finite-difference backward-Euler L of
 *    bec_allocate_problem with BEC_SPACE_FD, BEC_TIME_BDF1, a constant
 *    coefficient `a` (no a_nodes, no wind) and the unit side, in dim 1 or 2:
 *    y^n = (I + tau K) u^n - u^{n-1}, tau = T / N, K the 3- or 5-point
 *    Laplacian times a with h = 1 / (nx + 1).  For a problem set up with Q1
 *    elements, BDF2, a variable coefficient, convection, another side or
 *    dim 3 it would compute the residual of a different operator; use
 *    bec_true_relres there.  dim 3 is rejected (BEC_EINVAL).
 *  - f, u: device vectors of U = N * J doubles ([N][ny][nx]); res_out: one
 *    device double that receives RES.  All owned by the caller; the result
 *    is written asynchronously on `stream` (a cudaStream_t, NULL = legacy
 *    default stream), so synchronise before reading it.
 *  - Scratch: the block partial sums live in a file-scope device array of
 *    16384 pairs of doubles (256 KiB) that every GPU which loads the library
 *    holds until the process exits.  Sizes with ceil(J/256) * ceil(N/8) >
 *    16384 (about 33.5M unknowns) are rejected with BEC_EINVAL and a message
 *    in bec_last_error(); so are the size rules of bec_allocate_problem.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  No cudaMalloc, cudaFree or allocating
 *    library routine is called.
 *  - Every call shares the array and leaves its partial sums there; each
 *    call writes every slot it reads, so nothing needs clearing, but calls
 *    that overlap on the GPU (e.g. on two streams at once) race on it. */
bec_status bec_relres_noalloc(int dim, int nx, int N, double T, double a,
                              const double* f, const double* u, double* res_out,
                              void* stream);

/* Releases the workspace; p may be NULL. */
bec_status bec_free_problem(bec_problem* p);

/* ---- Learned correction (BEC_ROUTE_LEARNED) -------------------------------
 * The network's weights, FP32, concatenated in this order (C channels):
 *  - the 9 convolutions of the residual path, layer i an array
 *    [3][3][c_in][c_out] (1 -> C, C -> C x 7, C -> 8);
 *  - the a-gates' first convolutions A1_0..A1_7, [3][3][1][8] each;
 *  - their second convolutions A2_0..A2_7, [3][3][8][C] each.
 * Gated layer i's output is multiplied point by point by
 * 1 + tanh(conv(relu(conv(log a, A1_i)), A2_i)), log a centred on the
 * layer's grid.  The network maps one real plane to 8 (output channel j:
 * residue j) and runs on the real and on the imaginary part of x = the
 * restricted residual / sigma_0: Nc_j(x) = N_j(Re x) + i N_j(Im x), real
 * operators, as the exact inverse's symmetry ec(conj lambda, conj r) =
 * conj ec(lambda, r) requires.  The poles are sigma_j = sigma_0 rho^j with
 * sigma_0 = tau a_mean 2 pi^2 and sigma_7 = 2 tau a_mean (nx + 1)^2.  The
 * initial weights (a fixed seeded sequence) give a small correction (last
 * layer std 0.01 sqrt(1 / (9 C))) and gates of 1. */
long long bec_learned_num_weights(const bec_problem* p);
bec_status bec_learned_get_weights(bec_problem* p, float* host);
bec_status bec_learned_set_weights(bec_problem* p, const float* host);

/* Trains the network on the GPU: every ceil((N/2+1)/batch) steps a fresh set
 * of pairs is made for all frequencies: first a recording solve (FGMRES on a
 * seeded random right-hand side, preconditioned by the multigrid alone, to
 * RES 1e-10 within one restart cycle) keeps its Krylov vectors; the sets of
 * pairs take as right-hand sides, alternately, the time spectrum of the next
 * of them (the inputs its V-cycles were given) and a seeded Gaussian field
 * per frequency; r = what one V-cycle leaves of it, and the target the
 * coarse-grid correction B_{k,1}^{-1} R_0 r on the grid of spacing 2h, by 12
 * defect-correction V-cycles from level 1.  Each step draws `batch`
 * frequencies (1..32), runs the forward and backward kernels on the
 * relative error ||ec - ec*||^2 / ||ec*||^2 and takes one Adam step, the
 * learning rate ramped up linearly to lr over the first 100 steps, then
 * decayed along a cosine to lr / 10 at the last step.  loss_history (host, `steps` doubles, may be NULL)
 * receives the mean batch loss of every step.  The next apply recalibrates
 * the step alpha.  Synchronises. */
bec_status bec_learned_train(bec_problem* p, int steps, int batch, double lr,
                             unsigned long long seed, double* loss_history);

/* Loss and weight gradient for B given samples (a check of the kernels):
 * lam_idx (host, B ints) the frequency index k of each sample, r DEVICE
 * complex128 fine-grid residuals [B][ny][nx][2], e_target DEVICE complex128
 * coarse targets [B][mc][mc][2], mc = (nx - 1) / 2.  loss (host) receives the
 * mean relative error, grad (host, may be NULL) the gradient of every weight.
 * Synchronises. */
bec_status bec_learned_loss_grad(bec_problem* p, int B, const int* lam_idx,
                                 const double* r, const double* e_target,
                                 double* loss, float* grad);

/* 1 when the last calibration kept the V-cycle's iterates (alpha = 0: the
 * minimal-residual sums vanish or are not finite, or the judge rejected the
 * correction), else 0; -1: not learned.  Synchronises. */
long long bec_learned_fallbacks(bec_problem* p);

/* The judge (on by default; on = 0 turns it off, as for checking the
 * correction's arithmetic against a reference): after the calibrated step is
 * found, 10 power iterations per frequency on the error operator
 * E_k = I - M_k B_k of one apply, from the calibration right-hand side
 * normalised per frequency, once with M_k the V-cycle alone and once with
 * the corrected preconditioner.  The last ||E_k v|| (||v|| = 1) estimates
 * E_k's spectral radius.  The correction is kept only when its largest
 * estimate over k is below the V-cycle's; otherwise alpha = 0 for all
 * frequencies and P_eps^{-1} is the multigrid route's.  The multigrid's
 * work per calibration grows by 20 V-cycles and 10 network applies.
 * Changing the setting recalibrates at the next apply. */
bec_status bec_learned_set_judge(bec_problem* p, int on);

/* The judge's estimates of the last calibration, host array of
 * 2 (N/2+1) + 2 doubles: the V-cycle's radius per frequency k = 0..N/2, the
 * corrected preconditioner's per frequency, then the two maxima.  NaN when
 * the judge is off or no calibration ran since the weights, eps or the
 * setting changed.  Synchronises. */
bec_status bec_learned_judge_radii(bec_problem* p, double* host);

/* ||b_k - B_k x_k|| after the calibrated step divided by the V-cycle's
 * ||b_k - B_k x_k||, for every frequency k = 0..N/2, on the calibration's
 * fixed right-hand side (host array of N/2+1 doubles; 1 means the correction
 * gained nothing there).  The calibration runs at the first apply after the
 * weights or eps change.  Synchronises. */
bec_status bec_learned_residual_ratios(bec_problem* p, double* host);

/* ---- Failure detection (test hook) ---------------------------------------
 * Not a construct of the paper.  Every device wait of the library's kernels
 * is bounded; one that runs out sets an error word and the kernel returns
 * (freeing what it holds), and the next synchronising call on the problem
 * (bec_gmres_solve, the learned-route calls) returns BEC_ETIMEOUT.
 * bec_inject_fault(BEC_FAULT_PERSIST_WITHHOLD) makes the next persistent batch
 * launch (BEC_BATCH_PERSISTENT) never report instance 0's first pass done, so
 * the blocks that wait for it run out after about 0.2 s and bec_batch_solve
 * returns BEC_ETIMEOUT.
 * bec_inject_fault(BEC_FAULT_TC_WITHHOLD_LOADS) makes the next tensor-core
 * convolution withhold its tile loads, so that its waits run out (about
 * 0.2 s): a host-side injection that faults, traps and hangs nothing.
 * bec_inject_fault(BEC_FAULT_TMA_WITHHOLD_LOADS) does the same to the next
 * TMA-staged FP32 preconditioner pass (the N = 256 time pass or the n = 256
 * column pass): it issues no tile load, its blocks' waits run out and they
 * return without writing, and bec_gmres_solve returns BEC_ETIMEOUT.  Each
 * injection is one-shot; BEC_FAULT_NONE does nothing. */
enum { BEC_FAULT_NONE = 0, BEC_FAULT_TC_WITHHOLD_LOADS = 1, BEC_FAULT_PERSIST_WITHHOLD = 2,
       BEC_FAULT_TMA_WITHHOLD_LOADS = 3 };
bec_status bec_inject_fault(int kind);

/* ---- Tile shapes of the P_eps^{-1} passes --------------------------------
 * Not a construct of the paper.  The x-DST, y-DST and time passes group
 * their lines into blocks of 4, 8 or 16 warps (one line pair per warp).
 * bec_autotune times each width on this GPU with the problem's own
 * workspace (it overwrites the Krylov basis and scratch, so it must not
 * overlap a solve on the same problem), keeps the fastest per pass, and
 * caches the choice for the process per (precision, dim, nx, N); force = 1
 * re-times a cached shape.  The width only regroups lines, so every choice
 * gives the same result bit for bit.  Transforms shorter than 32 and the
 * multigrid and learned routes have nothing to tune (the report is zero).
 * bec_batch_create tunes each instance.  When the environment variable
 * BEC_TUNE_CACHE names a file, choices are also read from and appended to
 * it, so that later processes skip the timing.  Synchronises. */
typedef struct {
  int rows_warps, cols_warps, time_warps; /* chosen widths (warps per block) */
  float rows_ms[3], cols_ms[3], time_ms[3]; /* ms per launch at 4, 8, 16 warps; 0 = not tried */
  int cached;                              /* 1: taken from an earlier tuning of the shape */
} bec_tune_report;
bec_status bec_autotune(bec_problem* p, int force, bec_tune_report* report /* may be NULL */);
/* Sets the widths by hand: 0 (the default), 4, 8 or 16 warps per pass.
 * BEC_EINVAL for other values, for a non-zero width of a transform shorter
 * than 32, or for a width whose shared memory does not fit a block. */
bec_status bec_set_tiles(bec_problem* p, int rows_warps, int cols_warps, int time_warps);

/* ---- Precision conversions ---------------------------------------------
 * Not a construct of the paper.  The conversions the FP32 preconditioner
 * applies where it reads y and writes z: n doubles to floats (IEEE round to
 * nearest, ties to even) and n floats to doubles (exact).  They are done in
 * integer arithmetic, because the hardware conversion runs on the FP64 pipe,
 * and they agree with the hardware conversion bit for bit.  x and y are device
 * arrays that must not overlap; the calls are asynchronous on `stream` (a
 * cudaStream_t, NULL = the default stream).  BEC_EINVAL for n < 0 or a null
 * pointer with n > 0. */
bec_status bec_convert_to_float(const double* x, float* y, long long n, void* stream);
bec_status bec_convert_to_double(const float* x, double* y, long long n, void* stream);

/* y = 1/x for n doubles, by the reciprocal the FP64 multigrid smoother uses
 * in place of a division (a float reciprocal refined by two Newton-Raphson
 * steps; within one unit in the last place; |x| outside [2^-120, 2^120],
 * zero, infinities and NaN take the IEEE division).  Not a construct of the
 * paper; exported so that it can be checked.  Same conventions as the
 * conversions above. */
bec_status bec_reciprocal_fp64(const double* x, double* y, long long n, void* stream);

/* ---- Batches of independent problems of uneven size ---------------------
 * Not a construct of the paper: many independent instances (different grid,
 * N and eps) solved together.  Each instance is a bec_problem (own
 * workspace, own tables) bound to one of `nstreams` CUDA streams the batch
 * creates.  bec_batch_solve runs every instance's restarted GMRES in rounds:
 * one Arnoldi iteration of every active instance is enqueued, then the host
 * waits once per stream and every instance reads its residual.  Work of
 * instances on different streams overlaps on the GPU.  The mode:
 *  - BEC_BATCH_STREAMS: each iteration's kernels are launched one by one on
 *    the instance's stream;
 *  - BEC_BATCH_GRAPHS: each iteration is replayed from a per-iteration CUDA
 *    graph of the instance;
 *  - BEC_BATCH_PERSISTENT: per stream, the P_eps^{-1} (Sec. 4, Steps 1-3)
 *    of every instance of the stream that takes an Arnoldi step in the
 *    round runs in ONE launch (up to 64 instances per launch): a device work
 *    queue hands out the items (pass, instance, tile) of the five passes in
 *    order, one per block, and a block waits (bounded, about 0.2 s; then
 *    BEC_ETIMEOUT) until the previous pass of its instance is complete; the
 *    rest of each step is replayed from the instance's graph after that
 *    launch, on the same stream.  Needs FP32
 *    sine-transform instances in 2D (finite differences, backward Euler)
 *    with sides 31..255 and N in 4..512, and right preconditioning.  The
 *    results equal the other modes' bit for bit (the tiles compute exactly
 *    what the per-instance passes compute). */
typedef struct bec_batch bec_batch;
enum { BEC_BATCH_STREAMS = 0, BEC_BATCH_GRAPHS = 1, BEC_BATCH_PERSISTENT = 2 };

/* descs[i] and eps[i] for i < count as in bec_allocate_problem/bec_set_eps;
 * nstreams in [1, 64]; use_graphs is the mode (BEC_BATCH_*; any other value
 * is BEC_EINVAL).  On failure nothing stays allocated and bec_last_error()
 * names the failing instance. */
bec_status bec_batch_create(const bec_problem_desc* descs, const double* eps,
                            int count, int nstreams, int use_graphs,
                            bec_batch** out);

/* The problem object of instance i (for bec_build_rhs, bec_apply_*, ...);
 * owned by the batch. */
bec_status bec_batch_problem(bec_batch* b, int i, bec_problem** out);

/* Solves every instance: f[i], u[i] are device vectors of instance i
 * (16-byte aligned), opts apply to all, infos[i] (may be NULL) receives each
 * instance's result.  Synchronises.  Returns the first error met, else
 * BEC_ENOTCONV if some instance missed rtol within maxit, else BEC_OK. */
bec_status bec_batch_solve(bec_batch* b, const double* const* f,
                           double* const* u, const bec_gmres_opts* opts,
                           bec_gmres_info* infos);

/* Total space-time unknowns of the batch; kernels launched by all instances
 * (in BEC_BATCH_PERSISTENT mode each shared P_eps^{-1} launch counts once). */
long long bec_batch_unknowns(const bec_batch* b);
long long bec_batch_kernel_launches(const bec_batch* b);

/* Releases every instance and the streams; b may be NULL. */
bec_status bec_batch_free(bec_batch* b);

/* Number of space-time unknowns U = N * J of the problem (0 if p is NULL). */
long long bec_problem_size(const bec_problem* p);

/* Number of kernels the library launched on this problem since allocation. */
long long bec_kernel_launches(const bec_problem* p);

/* Per-kernel timing (not part of the method): while profiling is on, every
 * kernel launch of this problem is bracketed by two CUDA events on the
 * problem's stream.  bec_profile_start creates `capacity` event pairs and
 * clears earlier records (launches beyond capacity are counted but not
 * timed); bec_profile_stop synchronises the stream, sums the event intervals
 * per kernel name into out[0 .. *count-1] (at most `cap` entries, names are
 * static strings owned by the library), destroys the events and turns
 * profiling off. */
typedef struct {
  const char* name;
  long long launches;    /* launches recorded with timing */
  double ms;             /* summed event time of those launches */
} bec_kernel_time;
bec_status bec_profile_start(bec_problem* p, int capacity);
bec_status bec_profile_stop(bec_problem* p, bec_kernel_time* out, int cap,
                            int* count);

const char* bec_status_string(bec_status s);

/* Text of the last error met by the calling thread ("" if none). */
const char* bec_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BEC_H */
