/*
 * lbtr.h -- C ABI of the GB300 IMEX trust-region library for the discretised
 * Landau-Brazovskii (LB) model (arXiv 2603.03933).
 *
 * Problem (paper §2): on a periodic box with lattice A = diag(L_x, L_y[, L_z]) and a
 * grid of N = M^d points, minimise
 *     E(phi) = 1/2 sum_k Lambda_k |phi_hat_k|^2 + (1/N) sum_x F(phi(x)),
 *     Lambda_k = xi^2 (1 - |Bk|^2)^2,  B = 2 pi A^{-T},
 *     F(u) = tau/2 u^2 - gamma/6 u^3 + u^4/24,
 * over zero-mean real fields (the mass constraint, removed by P = [0, I] in §3).
 * phi_hat is the paper's normalised transform (1/N) sum_x phi(x) e^{-i(Bk).x}.
 *
 * Conventions shared by every call:
 *  - A field is a contiguous array of N real values in row-major order with x
 *    fastest: [y][x] in 2D, [z][y][x] in 3D.
 *  - Inner products and norms are the paper's <u,v>_N = (1/N) sum_x u v, which by
 *    Parseval is the Euclidean metric on the N-1 free Fourier coefficients.
 *  - Field pointers are DEVICE pointers owned by the caller.  Their element type is
 *    the context's working type: double for LB_FP64, float for LB_MIXED (except
 *    lb_imex_tr_solve, whose iterate is always double).  Base addresses must be
 *    16-byte aligned.
 *  - Scalar outputs (double*, info structs) are HOST pointers.  Calls that return
 *    scalars synchronise the given stream before writing them; lb_hessvec only
 *    enqueues work on the stream and returns.
 *  - The context owns all scratch memory (allocated in lb_create).  A context is
 *    not thread-safe: calls on one context must not overlap.
 *  - No C++ exception crosses this boundary; every call returns an lb_status and
 *    lb_last_error() describes the last failure of that context.
 */
#ifndef LBTR_H
#define LBTR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *lb_stream; /* same type as cudaStream_t; NULL = legacy default stream */

typedef enum {
    LB_OK = 0,
    LB_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment or parameter */
    LB_ERR_NOT_ZERO_MEAN = 2, /* an input field violates the mass constraint */
    LB_ERR_NONFINITE = 3,     /* NaN or Inf met in an input or a reduction */
    LB_ERR_NOCONV = 4,        /* iteration cap reached; outputs hold the last iterate */
    LB_ERR_TIMEOUT = 5,       /* a device-side grid barrier gave up waiting */
    LB_ERR_CUDA = 6,          /* a CUDA runtime call failed */
    LB_ERR_OOM = 7,           /* device allocation failed */
    LB_ERR_UNSUPPORTED = 8    /* grid size or dimension outside what the kernels cover */
} lb_status;

typedef enum { LB_FP64 = 0, LB_MIXED = 1 } lb_precision;
/* LB_FP64: every step in double.  LB_MIXED: FFTs, diagonals and the pointwise
 * updates in float; dot products, norms, the secular equation, the
 * actual/predicted-reduction ratio and the Lanczos tridiagonal step in double. */

typedef struct {
    int dim;          /* 2 or 3 */
    int n;            /* M, points per axis: a power of two, 8..512 (2D) or 8..256 (3D) */
    double box[3];    /* L_x, L_y, L_z: box lengths (A = diag(box)); box[2] unused in 2D */
    double xi;        /* Lambda_k = xi^2 (1 - |Bk|^2)^2; xi = 1 is the paper's model */
    double tau;       /* reduced temperature (eq. lb_energy) */
    double gamma;     /* three-body coefficient (eq. lb_energy) */
} lb_problem;

typedef struct lb_ctx lb_ctx;

/* Create a context on the current CUDA device for `prob` in precision `prec`.
 * Allocates the scratch memory of every call below (a few field-sized buffers).
 * Errors: LB_ERR_INVALID_ARG (null pointers, non-positive box or n),
 * LB_ERR_UNSUPPORTED (n not a power of two in range, dim not 2/3), LB_ERR_OOM. */
lb_status lb_create(const lb_problem *prob, lb_precision prec, lb_ctx **out);

/* Release a context and its scratch memory.  NULL is accepted. */
lb_status lb_destroy(lb_ctx *ctx);

/* Text of the last error of `ctx` (static storage of the context; never NULL). */
const char *lb_last_error(const lb_ctx *ctx);

/* Bytes of device scratch memory owned by the context. */
size_t lb_workspace_bytes(const lb_ctx *ctx);

/* Change the model parameters (tau, gamma, xi) of an existing context without
 * reallocating.  Grid and box are fixed at creation. */
lb_status lb_set_params(lb_ctx *ctx, double xi, double tau, double gamma);

/*
 * Energy and gradient (paper §2: eq. interaction_bulk_energy and the gradient
 * formulas grad G = Lambda Psi_hat, grad F = F_N Gamma F_N^{-1} Psi_hat after it).
 *   phi    [in]  device field, zero mean.
 *   energy [out] host double: E(phi) = G + F.
 *   grad   [out] device field or NULL: g = P[F^{-1} Lambda F phi + F'(phi)].
 *   gmax   [out] host double or NULL: max_x |g(x)|.
 * Errors: LB_ERR_NOT_ZERO_MEAN if |mean(phi)| > 1e-10 max(1, rms(phi)) (FP64) or
 * 1e-5 max(1, rms) (MIXED); LB_ERR_NONFINITE.
 */
lb_status lb_energy_grad(lb_ctx *ctx, const void *phi, double *energy, void *grad,
                         double *gmax, lb_stream stream);

/*
 * Energy and its derivatives with respect to the model parameters and the cell, for
 * parameter fits and cell optimisation (the paper has no such entry point; the energy is
 * that of §2, eq. interaction_bulk_energy, with Lambda_k = xi^2 (1 - |Bk|^2)^2 and
 * B = diag(2 pi / L_a)).  The grid values of phi are held fixed, so the field stretches
 * with the box:
 *   out[0] = E,
 *   out[1] = dE/dtau   = <phi^2 / 2>_N,
 *   out[2] = dE/dgamma = -<phi^3 / 6>_N,
 *   out[3 + a] = dE/dL_a = sum_k 1/2 |phi_hat_k|^2 4 xi^2 (1 - |Bk|^2) (Bk)_a^2 / L_a,
 *                a = x, y, z (out[5] = 0 in 2D); the bulk term does not depend on L.
 *   phi  [in]  device field, zero mean (checked as in lb_energy_grad).
 *   out  [out] host array of 6 doubles.
 *   grad [out] device field or NULL: g as in lb_energy_grad; the derivative of E with
 *              respect to the grid values of phi, restricted to zero-mean fields, is g / N.
 * Errors: those of lb_energy_grad; LB_ERR_NONFINITE.  Synchronises the stream.
 */
lb_status lb_energy_derivs(lb_ctx *ctx, const void *phi, double *out, void *grad, lb_stream stream);

/*
 * Hessian-vector product (paper §2, grad^2 G = Lambda and grad^2 F = F_N Gamma' F_N^{-1};
 * §3.2, H = D + T and the remark on computing T d by FFT):
 *   Hv = P[F^{-1}(Lambda F v) + F''(phi) v],  F''(u) = tau - gamma u + u^2/2.
 *   phi, v [in]  device fields (v must have zero mean; it is not checked here).
 *   hv     [out] device field; may not alias phi or v.
 * Asynchronous: enqueues kernels on `stream` and returns.
 */
lb_status lb_hessvec(lb_ctx *ctx, const void *phi, const void *v, void *hv, lb_stream stream);

/*
 * The same product for fields in HOST memory: count products H v_i at one phi (the way the
 * Lanczos step and the inner iteration use H), with the copies in and out overlapped with the
 * products.  The library keeps device staging with the context (phi and three (v, Hv) slots,
 * allocated on the first call) and two copy streams of its own; the products run on `stream`.
 *   phi   [in]  host field (copied once per call).
 *   count [in]  number of products (0: nothing is done).
 *   v     [in]  host array of `count` host fields (zero mean, not checked).
 *   hv    [out] host array of `count` host fields; none may alias phi or its v.
 * Fields are of the context's grid and precision (float for LB_MIXED, double for LB_FP64).
 * Page-locked host memory lets the copies overlap the products; pageable memory is accepted
 * and copied synchronously.  Synchronises `stream`: the results are in hv on return.
 * Errors: LB_ERR_INVALID_ARG (null pointers, negative count, aliasing); LB_ERR_CUDA.
 */
lb_status lb_hessvec_host(lb_ctx *ctx, const void *phi, int count, const void *const *v, void *const *hv,
                          lb_stream stream);

typedef struct {
    double eta;        /* IMEX step size (paper §4: 0.1) */
    double eps_sub;    /* stop when ||g + (H + lambda I) d|| < eps_sub (paper §4: 1e-13) */
    double rel_tol;    /* also stop when that residual < rel_tol * ||g||; 0 disables */
    int max_iter;      /* cap on IMEX iterations */
    int check_every;   /* iterations between host reads of the convergence flag */
} lb_sub_opts;

typedef struct {
    int iterations;        /* IMEX iterations performed */
    int converged;         /* 1 if the residual test of Algorithm 3 (eps_sub or rel_tol) passed */
    double residual;       /* ||g + (H + lambda I) d|| of the returned d */
    double lambda;         /* Lagrange multiplier of the returned d */
    double dnorm;          /* ||d|| */
    double model_value;    /* f(d) = <g,d> + <d,Hd>/2 (eq. tr_subproblem) */
    long long newton_steps;/* Newton steps spent on the secular equation, summed */
    double rel_residual;   /* residual / ||g|| */
    int stalled;           /* 1 if the LB_MIXED iteration ended because its residual stopped
                              falling (512 checked iterations without a 2 % drop of the squared
                              residual) before reaching the tolerance; converged is then 0 */
} lb_sub_info;

/* Fill `o` with the paper's values (eta 0.1, eps_sub 1e-13) and max_iter 20000. */
void lb_default_sub_opts(lb_sub_opts *o);

/*
 * Trust-region subproblem min_{||d|| <= r} <g,d> + <d,Hd>/2 (eq. tr_subproblem) by
 * the adaptive implicit-explicit iteration, Algorithm 3 of §3.2:
 *   b_k = d_k - eta (g + T d_k),
 *   lambda_{k+1} = 0 if phi_k(0) <= r^2 else the root of phi_k(lambda) = r^2 by Newton
 *   (eq. lambda_update_rule), d_{k+1} = (I + eta (D + lambda_{k+1} I))^{-1} b_k.
 *   phi [in] device field; g [in] device field (zero mean); r > 0.
 *   d0  [in] device field or NULL: initial point (NULL: d0 = -r g / ||g||, the
 *       deterministic start of the global-optimality theorem; non-NULL: e.g. the
 *       randomised start of the hard-case remark, which must satisfy ||d0|| <= r).
 *   d   [out] device field: the returned d_{k+1}.
 *   info[out] host struct (may be NULL).
 * Returns LB_ERR_NOCONV (with d holding the last iterate) if max_iter is reached, and in
 * LB_MIXED also when the float iteration stalls above the tolerance (info->stalled = 1;
 * info->residual and info->rel_residual give the residual reached).
 */
lb_status lb_tr_subproblem(lb_ctx *ctx, const void *phi, const void *g, double r,
                           const void *d0, const lb_sub_opts *opts, void *d,
                           lb_sub_info *info, lb_stream stream);

typedef struct {
    int max_steps;     /* Lanczos steps cap, 2..600 (basis vectors kept: max_steps + 1) */
    double tol;        /* stop when the Ritz residual ||H u - theta u|| <= tol */
    double sigma;      /* shift of the congruence M = Lambda + sigma; <= 0 picks
                          max(1e-2, max_x |F''(phi(x))|) */
    int check_every;   /* Lanczos steps between Rayleigh-Ritz checks */
    uint64_t seed;     /* seed of the start vector (counter-based Philox4x32-10) */
} lb_eig_opts;

typedef struct {
    double lambda_min; /* Rayleigh-Ritz estimate of the smallest eigenvalue of H */
    double kappa_min;  /* smallest Ritz value of M^{-1/2} H M^{-1/2}: same sign */
    double residual;   /* ||H u - lambda_min u|| for the unit Ritz vector u */
    int steps;         /* Lanczos steps taken */
    int converged;
} lb_eig_info;

void lb_default_eig_opts(lb_eig_opts *o);

/*
 * Smallest eigenvalue of the Hessian on zero-mean fields (the SP-II test of the
 * paper's §1 definition; the eigenvalue diagnostics of §4.1 and §4.3).  The paper
 * does not state its eigenvalue method; this is Lanczos with full
 * re-orthogonalisation on K = M^{-1/2} H M^{-1/2}, M = Lambda + sigma (diagonal in
 * reciprocal space), followed by Rayleigh-Ritz for H on V = M^{-1/2} Q.
 *   phi [in] device field.   vec [out] device field or NULL: the unit Ritz vector.
 * Returns LB_ERR_NOCONV if max_steps is reached before tol (results still filled).
 */
lb_status lb_lambda_min(lb_ctx *ctx, const void *phi, const lb_eig_opts *opts, void *vec,
                        lb_eig_info *info, lb_stream stream);

typedef struct {
    /* Algorithm 1/2 parameters; defaults are the paper's §4 values */
    double gamma_c, gamma_e, gamma_lam, theta, mu_lo, mu_hi, mu0, r0, nu0;
    double eps;          /* stop when max_x |g(x)| < eps (paper: 1e-10) */
    int max_outer;       /* cap on outer iterations */
    int second_order;    /* 1: also require lambda_min >= -tol2 before returning */
    double tol2;         /* second-order tolerance */
    lb_sub_opts sub;     /* inner solver (Algorithm 3) options */
    lb_eig_opts eig;     /* lambda_min options for the second-order test */
    int pcg_max_iter;    /* cap on CG iterations of each CONTRACT linear solve */
    double pcg_rtol;     /* relative tolerance of those solves */
    /* Nearly hard subproblems (§4.4 and the remark on the hard case after the global-
     * optimality theorem): if hard_tol > 0, every outer iteration computes lambda_min(H)
     * and its Ritz vector u (Lanczos, options `eig`); when lambda_min < 0 and
     * |<g, u>_N| <= hard_tol (the component g^(1) of g along u), the subproblem starts
     * from a random point of the trust region instead of -r g / ||g||.  0: off. */
    double hard_tol;
    /* Checkpoint / resume (no counterpart in the paper).  If checkpoint_path is non-NULL
     * and checkpoint_every > 0, the state carried between outer iterations (the iterate
     * and the scalars of Algorithm 1) is written to <checkpoint_path>.npy and .json after
     * every checkpoint_every-th outer iteration.  If resume != 0, the solve starts from
     * that checkpoint instead of phi_inout and repeats the remaining iterations exactly;
     * max_outer still counts from the first iteration of the original solve.  The path
     * is borrowed for the duration of the call.  The files also record the grid, the box
     * lengths, xi, tau, gamma, the precision and the subproblem step eta; a resume refuses a
     * checkpoint whose values differ from the context's and the options'.  Errors:
     * LB_ERR_INVALID_ARG when a file cannot be written or read, or belongs to another
     * problem. */
    const char *checkpoint_path;
    int checkpoint_every;
    int resume;
} lb_tr_opts;

typedef struct {
    int outer;           /* outer iterations performed */
    long long inner;     /* IMEX iterations summed over all subproblems */
    int accepted, contracted, shrunk;
    double energy;       /* E at the returned iterate */
    double gmax;         /* max_x |g| at the returned iterate */
    double lambda_min;   /* last second-order test value (NaN if never run) */
    int status;          /* lb_status of the solve */
    int randomized;      /* subproblems started from a random point of the ball */
    double g1_min;       /* smallest |g^(1)| seen by the nearly-hard test (NaN if never run) */
    int sub_stalled;     /* subproblems that ended stalled above their tolerance (LB_MIXED) */
    int sub_capped;      /* subproblems that ended at the iteration cap */
    double sub_worst_rel_res; /* largest residual / ||g|| among those (0 if none) */
} lb_tr_info;

void lb_default_tr_opts(lb_tr_opts *o);

/*
 * IMEX-TR: Algorithm 1 of §3.1 (TRACE outer loop) with CONTRACT (Algorithm 2) and the
 * subproblem solver above.  phi_inout is a DEVICE array of N doubles in both
 * precisions (the outer iterate, gradient and ratio test are kept in FP64); in
 * LB_MIXED the inner iterations run in float.
 * Returns LB_ERR_NOCONV if max_outer is reached (phi_inout holds the last iterate).
 * With the environment variable LBTR_TRACE=1, every outer iteration prints one JSON line
 * on stderr: j, E, max|g|, r, nu, mu, lambda, ||s||, rho, inner iterations, the
 * subproblem's status and the accepted / contracted / shrunk counts.
 */
lb_status lb_imex_tr_solve(lb_ctx *ctx, double *phi_inout, const lb_tr_opts *opts,
                           lb_tr_info *info, lb_stream stream);

/*
 * First-order gradient flow: the semi-implicit scheme (SIS) among the gradient-flow
 * methods §4 compares with, and the source of the first-order trajectories that §4
 * "Robustness to initial conditions" starts IMEX-TR from (initial, intermediate and
 * converged states).  The paper does not print the scheme; each step here treats the
 * reciprocal diagonal D = Lambda implicitly and F'(phi) explicitly, as the IMEX
 * subproblem solver of §3.2 does:
 *     phi <- phi - dt (I + dt D)^{-1} g(phi),
 * with the k = 0 coefficient held at zero, so that its fixed points are the zeros of g.
 * Computed in FP64 in both precisions.
 *   phi_inout [in/out] DEVICE array of N doubles, zero mean, 16-byte aligned.
 *   opts      NULL for the defaults (dt 1, eps 1e-8, max_steps 10000, check_every 10).
 *   info      [out] may be NULL.
 * max_x |g| is tested before the first step, every check_every steps and after the last
 * one; the solve stops when it is below eps.  Returns LB_ERR_NOCONV after max_steps steps
 * without that (phi_inout holds the last iterate), LB_ERR_INVALID_ARG for dt <= 0 or
 * max_steps < 0, LB_ERR_NOT_ZERO_MEAN / LB_ERR_NONFINITE as lb_energy_grad.
 */
typedef struct {
    double dt;           /* time step */
    double eps;          /* stop when max_x |g(x)| < eps */
    int max_steps;       /* cap on steps */
    int check_every;     /* steps between tests of max |g| (each test synchronises) */
} lb_sis_opts;

typedef struct {
    int steps;           /* steps taken */
    double energy;       /* E at the last test */
    double gmax;         /* max_x |g| at the last test */
    int status;          /* lb_status of the solve */
} lb_sis_info;

void lb_default_sis_opts(lb_sis_opts *o);
lb_status lb_sis_solve(lb_ctx *ctx, double *phi_inout, const lb_sis_opts *opts, lb_sis_info *info,
                       lb_stream stream);

/*
 * Hessian-vector product that allocates nothing (no counterpart in the paper; an
 * interface for callers that cannot call cudaMalloc, e.g. plug-ins whose host
 * framework owns all device memory, or loops that cannot afford the implicit device
 * synchronisation of cudaMalloc/cudaFree).  Same operator as lb_hessvec, without a
 * context: the problem is passed directly and the scratch is a fixed 3 MiB device
 * array inside the library, held on every device that loads it until the process
 * exits.  Limits: N = n^dim <= 2^18 points (up to 64^3 or 512^2); larger grids return
 * LB_ERR_UNSUPPORTED.  Fields are double for LB_FP64 and float for LB_MIXED.
 * The first call on each device resolves the scratch address and sets kernel
 * attributes (once per device, with that device current).  Every call shares the one
 * scratch array: calls that
 * overlap on the GPU (other streams, other host threads) race and must be serialised
 * by the caller.  Asynchronous on `stream`: each call writes its tables into the scratch
 * with a small kernel and enqueues the transform kernels; it neither copies from the host
 * nor synchronises.
 */
lb_status lb_hessvec_noalloc(const lb_problem *prob, lb_precision prec, const void *phi, const void *v,
                             void *hv, lb_stream stream);

/* Profiling aid.  Kernel classes of the library's launches: */
typedef enum {
    LB_K_XFWD = 0,     /* forward x-row real transform with its pointwise preprocessing */
    LB_K_XINV = 1,     /* inverse x-row real transform with its pointwise postprocessing */
    LB_K_XMID = 2,     /* fused inverse -> pointwise -> forward x-row transform */
    LB_K_COLY = 3,     /* column transform along y (non-innermost in 3D) */
    LB_K_COLI = 4,     /* innermost column transform with the reciprocal-space diagonal */
    LB_K_SECULAR = 5,  /* cooperative secular-equation Newton solve */
    LB_K_REDUCE = 6,   /* physical-space reductions and elementwise kernels */
    LB_K_COUNT = 7
} lb_kernel_class;

/* enable != 0: from now on every kernel the context launches is bracketed by CUDA
 * events on its stream, and the totals below are reset; enable == 0 stops that. */
lb_status lb_profile_enable(lb_ctx *ctx, int enable);

/* Synchronise the recorded events and return, for kernel class `kclass`, the summed
 * device time in ms, the number of launches and the summed algorithmic bytes (the
 * arrays each launch must read and write once: inputs, outputs and the spectra it
 * transforms, counted at the context's working precision). */
lb_status lb_profile_read(lb_ctx *ctx, int kclass, double *total_ms, long long *launches,
                          double *alg_bytes);

/*
 * Batches of independent problems, for parameter sweeps (phase-diagram sweeps over
 * (tau, gamma, M); the paper solves one problem at a time and has no batch
 * interface).  A batch owns one context per problem; the problems may differ in grid
 * size, dimension, box and parameters, and share the precision.
 *   probs [in]  `count` problem descriptions (copied).
 *   out   [out] the batch; destroy with lb_batch_destroy.
 * Errors: those of lb_create; LB_ERR_INVALID_ARG for count <= 0.
 */
typedef struct lb_batch lb_batch;
lb_status lb_batch_create(const lb_problem *probs, int count, lb_precision prec, lb_batch **out);
void lb_batch_destroy(lb_batch *batch);
const char *lb_batch_last_error(const lb_batch *batch);
int lb_batch_size(const lb_batch *batch);

/*
 * hv[i] = H_i v[i] for every problem i of the batch (each as lb_hessvec).  phi, v, hv:
 * host arrays of lb_batch_size() device pointers, fields laid out as in lb_hessvec.
 * The first call with a given set of pointers records the products of all problems as
 * one CUDA graph: the 2D problems as grouped launches or one persistent launch (see
 * lb_batch_set_launch below), the others as independent branches on up to 16 internal
 * streams, largest problems first on the least-loaded stream; later calls with the same pointers replay it, and a call with other
 * pointers records anew.  The graph is launched on `stream`; the call is
 * asynchronous.  Calls on the same batch must not overlap on the GPU (the problems'
 * contexts hold the scratch spectra).
 * Errors: LB_ERR_INVALID_ARG (null, misaligned or aliased fields), LB_ERR_CUDA.
 */
lb_status lb_batch_hessvec(lb_batch *batch, const void *const *phi, const void *const *v, void *const *hv,
                           lb_stream stream);

/*
 * Launch strategy of a batch's 2D problems (grids of 16..512 points per axis):
 *  strategy 0 (default): the problems of each grid size run as three grouped launches (rows
 *    forward, y lines with Lambda, rows inverse) whose blockIdx.y selects a problem;
 *  strategy 1: ONE persistent cooperative launch for all of them: the three passes of every
 *    product as three phases separated by grid barriers, each CTA taking the next (problem,
 *    task) pair from a device-side queue of the phase, largest grids first.  Its parameters:
 *    min_blocks, the register allocation (4 or 5 resident CTAs of 128 threads per SM);
 *    ctas_per_sm, the CTAs launched per SM (0: as many as fit); group, row blocks per row task.
 * lb_batch_set_launch sets them; lb_batch_tune chooses them by timing: it records and replays
 * the batch's graph `replays` times on `stream` for the grouped launches and for each
 * candidate of the persistent one (CUDA events), keeps the fastest and returns the table.
 * Both leave the graph to be recorded anew by the next lb_batch_hessvec call; tuning runs
 * products on the given fields and blocks until the timing is done.
 * Errors: LB_ERR_INVALID_ARG (bad arguments or fields), LB_ERR_TIMEOUT, LB_ERR_CUDA.
 */
typedef struct {
    int count;             /* candidates timed */
    int strategy[12];      /* 0 grouped launches, 1 persistent launch */
    int min_blocks[12];    /* register allocation of the persistent kernel (CTAs per SM) */
    int ctas_per_sm[12];   /* CTAs per SM of the persistent launch (0 for the grouped one) */
    int group[12];         /* row blocks per row task */
    double us[12];         /* mean device time of one product call (graph replay), microseconds */
    int chosen;            /* the candidate now in use */
} lb_batch_tuning;
lb_status lb_batch_set_launch(lb_batch *batch, int strategy, int min_blocks, int ctas_per_sm, int group);
lb_status lb_batch_tune(lb_batch *batch, const void *const *phi, const void *const *v, void *const *hv,
                        int replays, lb_batch_tuning *out, lb_stream stream);

/*
 * Algorithm 1 (as lb_imex_tr_solve) for every problem of the batch, several at a time: a
 * pool of host threads, each with its own internal stream, takes the problems from a
 * shared queue, largest first, so that the GPU works on several problems while each
 * driver waits for its scalars.  The solves start after the work already queued on
 * `stream` and the call returns when all have ended (later work on `stream` is ordered
 * after them).
 *   phi      [in/out] host array of lb_batch_size() DEVICE pointers, each N doubles as in
 *            lb_imex_tr_solve, distinct and 16-byte aligned.
 *   opts     options shared by all problems (NULL: the defaults); problem i checkpoints
 *            to (and resumes from) <checkpoint_path>.<i>.
 *   info     [out] host array of lb_batch_size() results, or NULL.
 *   nthreads host threads (<= 0: 8); at most the batch size and 16.
 * Returns LB_OK if every solve returned LB_OK, else the status of the first problem (in
 * batch order) that did not, whose message lb_batch_last_error then holds; every problem
 * is solved either way and info[i].status holds each one's status.  Blocks the calling
 * thread; other calls on the same batch must not run meanwhile (they share its streams
 * and contexts).
 */
lb_status lb_batch_tr_solve(lb_batch *batch, double *const *phi, const lb_tr_opts *opts, lb_tr_info *info,
                            int nthreads, lb_stream stream);

/* Profiling aid: the FP64 fused-multiply-add throughput of the current device, measured
 * with CUDA events on `stream` (8 independent FMA chains per thread, 8 blocks of 256
 * threads per SM; best of three timed runs after a warm-up), in TFLOP/s (2 flops per
 * FMA).  It is the bound of the FP64 path, whose transforms run on the FP64 pipe.
 * Synchronises the stream. */
lb_status lb_measure_fp64_rate(double *tflops, lb_stream stream);

/* Inner loop of lb_tr_subproblem (and of the subproblems of lb_imex_tr_solve) on 3D
 * 128^3 grids in LB_MIXED precision (Algorithm 3, §3.2): with `enable` != 0 (the default)
 * the whole solve -- b_0, every iteration with its stop test and multiplier rule, and the
 * returned iterate -- runs as ONE cooperative launch whose CTAs take the same decisions
 * from the same grid-wide sums; with 0, each iteration is two launches and the host polls
 * the device state between chunks of iterations.  Both follow the same tests and give the
 * same iterates up to summation order.  Other grids and precisions always take the
 * per-iteration launches.  lb_persistent_subproblem_available sets *available to 1 when the
 * context's grid and device admit the one-launch form and it is enabled. */
lb_status lb_set_persistent_subproblem(lb_ctx *ctx, int enable);
lb_status lb_persistent_subproblem_available(lb_ctx *ctx, int *available);

/* Test hook: cap on the device-side spin of grid barriers, in SM clock cycles
 * (0 restores the default of about two seconds).  Lets tests exercise the
 * LB_ERR_TIMEOUT path without a hang. */
lb_status lb_set_barrier_budget(lb_ctx *ctx, long long cycles);

#ifdef __cplusplus
}
#endif

#endif /* LBTR_H */
