/*
 * liblyap: trace(E X(v)) for sequences of parametrized Lyapunov equations on
 * one NVIDIA GB300 (sm_103a).
 *
 * Problem (Palitta, Tomljanovic, Nakic, Saak, "Efficient solution of
 * sequences of parametrized Lyapunov equations with applications", §1,
 * eqs. (Ljap jdba 1) and (formA), written in the transposed convention):
 *
 *     A(v) = A0 - U diag(v) V^T,     A(v)^T X + X A(v) = -G G^T,
 *     f(v) = trace(E X(v)),          v in (R \ {0})^k.
 *
 * The paper states the same family as A_p X + X A_p^T = -Q with
 * A_p = A0^T, B_l = V, B_r = U, Q = G G^T; X and f are the same.
 *
 * Method (§2.1): A0 is diagonalised once in FP64 (A0^T = Qp Lambda Qp^{-1});
 * the Sherman-Morrison-Woodbury formula (eq. (deltaX_SMW2)) turns each new v
 * into a capacitance system with D(v)^{-1} - N^T L0^{-1} M (eq.
 * (SMW_linearsystem)), solved by a recycled Krylov method (GCRO-DR) across
 * the sequence; every matvec applies L0^{-1}, i.e. the Cauchy matrix
 * Lc_ij = 1/(lambda_i + lambda_j) (eq. (Z(v))). f(v) follows from the
 * additive form of eq. (Xsmalllastline).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are column-major float64 (Fortran order), leading dimension
 *    equal to the row count.
 *  - mem_kind: LYAP_MEM_HOST means pointer arguments are host memory (the
 *    call copies them); LYAP_MEM_DEVICE means device memory on the context's
 *    GPU, read and written only by work queued on opts->stream (no copy
 *    through the host; device parameters are validated by a kernel and an
 *    invalid one is reported at the call's next synchronisation); the
 *    caller keeps ownership and must keep the buffers alive until the call
 *    returns. The solve calls drive the Krylov iteration from the host and
 *    return once their results are complete.
 *  - Handles (ctx, seed, server) are owned by the library and freed with the
 *    matching destroy/free call. Output arrays are caller-allocated.
 *  - Every function returns LYAP_OK (0) or a negative error code; nothing
 *    aborts, exits or throws across this boundary. Per-result problems
 *    (no convergence, breakdown, non-finite values) are reported in
 *    lyap_result_info.status while the call itself returns LYAP_OK.
 *  - Calls on one context are not thread-safe; use one context per thread.
 */
#ifndef LYAP_H
#define LYAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define LYAP_OK 0
#define LYAP_PENDING 1           /* serve_poll: request not finished yet       */
#define LYAP_EINVAL (-1)         /* bad shape/pointer, v_i == 0 (§1), NaN/Inf   */
#define LYAP_ENOMEM (-2)         /* device allocation failed or over budget    */
#define LYAP_EUNSTABLE_SEED (-3) /* max Re(lambda) >= 0 or lambda_i+lambda_j ~ 0 */
#define LYAP_ECUDA (-4)          /* CUDA runtime error                          */
#define LYAP_ESOLVER (-5)        /* cuSOLVER/cuBLAS failure in the seed factor  */
#define LYAP_ENOCONV (-6)        /* (per result) maxit reached                  */
#define LYAP_EBREAKDOWN (-7)     /* (per result) Krylov breakdown               */
#define LYAP_EDEVICE_TIMEOUT (-8)/* a bounded device-side wait expired          */
#define LYAP_ENOTFOUND (-9)      /* unknown seed id or ticket                   */
#define LYAP_ENONFINITE (-10)    /* (per result) NaN/Inf appeared in the solve  */
#define LYAP_ECANCELLED (-11)    /* request cancelled (serving)                 */

#define LYAP_MEM_HOST 0
#define LYAP_MEM_DEVICE 1

/* Precision of the capacitance solve.
 *  LYAP_FP64:    every Krylov step in FP64 (plain path).
 *  LYAP_BF16_IR: inner Krylov solves in FP32 with the Cauchy-matrix GEMM on
 *                tcgen05 tensor cores (operands split into two BF16 terms,
 *                three products, FP32 accumulation), wrapped in iterative
 *                refinement on the FP64 capacitance residual; the residual,
 *                the solution update and the trace stay in FP64. */
#define LYAP_FP64 0
#define LYAP_BF16_IR 2

/* Arithmetic of the mixed path's refinement residual (lyap_opts.residual).
 * All evaluate P - T(v) W with an error of the order of FP64 rounding:
 * FF pairs two FP32 values per number (about 48 significant bits, exact
 * products by FMA) and runs on the FP32 pipes; FP64 uses the FP64 pipes;
 * TC (the default) splits both operands into 8 exact 6-bit integer digits
 * (48 bits, scaled per row/column) whose products the BF16 tensor cores sum
 * without rounding; above 2n = 2046 the K dimension runs in chunks whose
 * exact sums are added in float-float. */
#define LYAP_RESID_FF 0
#define LYAP_RESID_FP64 1
#define LYAP_RESID_TC 2

/* Fault-injection bits for lyap_opts.inject (tests; none faults the GPU).
 *  ALLOC_FAIL:  the call fails as if a workspace allocation had failed.
 *  FORCE_MAXIT: every Krylov solve stops after one iteration (ENOCONV).
 *  DEVICE_WAIT: in the mixed path the tensor-core GEMM issues no copy, so
 *               its bounded mbarrier wait runs out (after about 50 us);
 *               the kernel records the expiry, frees its TMEM and returns,
 *               and the call returns LYAP_EDEVICE_TIMEOUT at its next
 *               synchronisation. The context stays usable. */
#define LYAP_INJECT_ALLOC_FAIL 0x1u
#define LYAP_INJECT_FORCE_MAXIT 0x2u
#define LYAP_INJECT_DEVICE_WAIT 0x4u

typedef struct lyap_ctx lyap_ctx;
typedef struct lyap_seed lyap_seed;
typedef struct lyap_server lyap_server;

/* Solver options. lyap_opts_default() fills the defaults, which follow the
 * paper's settings for its first example (§4, Ex. 1): relative residual
 * threshold 1e-10 tightened to 1e-12 for the FP64 path (the trace is a
 * linear functional of the capacitance solution and is wanted to 1e-10),
 * at most 300 iterations, s = 10 recycled vectors. The cycle length m is
 * not given in the paper; the default 40 is the fastest of 24..60 for both
 * paths on the 800-state benchmark. The TSVD rank defaults to 50, the
 * paper's Ex. 1 value (it uses 5 in Ex. 3); on the 800-state benchmark 50 is
 * within 2% of the fastest rank (64). The mixed path's inner tolerance
 * defaults to 1e-3: the tensor-core operator is accurate to about 1e-5, so a
 * tighter inner solve does not save refinement steps, and with the
 * residual on the tensor cores a refinement step is cheap; 1e-3 (about 4
 * steps) minimised the time. */
typedef struct {
  double tol;        /* FP64 path: stop when ||r|| <= tol ||b||               */
  double refine_tol; /* mixed path: outer stop on the FP64 residual           */
  double inner_tol;  /* mixed path: inner (FP32) relative residual target     */
  int maxit;         /* max Krylov iterations per solve                       */
  int m;             /* cycle length (Arnoldi steps + recycled vectors)       */
  int s;             /* recycled vectors (harmonic Ritz, smallest |theta|)    */
  int pbar;          /* rank of the truncated SVD of the off-diagonal coupling
                        kept in the preconditioner (eq. (prec)); 0 = block
                        diagonal only; at most 64; default 50            */
  int batch;         /* systems solved in lockstep (0 = library's choice)    */
  int precision;     /* LYAP_FP64 or LYAP_BF16_IR                              */
  int max_refine;    /* mixed path: max refinement steps                      */
  size_t hbm_budget; /* serving: admission budget in bytes (0 = 80% of free)  */
  void* stream;      /* cudaStream_t to run on (NULL = the context's stream)  */
  unsigned inject;   /* LYAP_INJECT_* bits (tests only)                       */
  int residual;      /* mixed path: LYAP_RESID_TC (default), _FF or _FP64      */
} lyap_opts;

/* Per-result report. */
typedef struct {
  int iters;          /* Krylov iterations (inner iterations summed)          */
  int refine_steps;   /* FP64 residual evaluations (mixed path)               */
  int status;         /* LYAP_OK, LYAP_ENOCONV, LYAP_EBREAKDOWN, ...          */
  double rel_resid;   /* final ||b - T(v) w|| / ||b||, evaluated in FP64      */
  double err_est;     /* estimate of |f - f_exact| / |f| (see lyap_trace_EX)  */
} lyap_result_info;

/* Seed facts, for reporting. */
typedef struct {
  int n, k, g;
  int real_path;        /* 1 when every eigenvalue is real                    */
  double cond_Q;        /* ||Qp||_F ||Qp^{-1}||_F                             */
  double f0;            /* trace(E X0), the seed's own value                 */
  double max_re_lambda; /* < 0 for an accepted seed                          */
  double min_abs_lambda_sum; /* min |lambda_i + lambda_j|                     */
  size_t resident_bytes;/* device bytes held by the seed                      */
} lyap_seed_stats;

/* Fill *opts with the defaults described above. */
void lyap_opts_default(lyap_opts* opts);

/* Human-readable name of a status code (static storage). */
const char* lyap_strerror(int code);

/* Detail of the last error raised on the calling thread (valid until the
 * thread's next failing call). */
const char* lyap_last_error(void);

/* Create a context on CUDA device `device` (its own stream and library
 * handles). Errors: LYAP_EINVAL (bad device), LYAP_ECUDA, LYAP_ESOLVER. */
int lyap_ctx_create(int device, lyap_ctx** out);
void lyap_ctx_destroy(lyap_ctx* ctx);

/* Offline seed factorisation and precomputation (§2.1 and its Table 1,
 * offline column): eig(A0^T) = Qp Lambda Qp^{-1} in FP64, Qp^{-1}, the seed
 * solution in eigen-coordinates (eqs. (seedLE), (Z(v))), the projected data
 * Ub = Qp^{-1} V, Vb = Qp^T U, the diagonal blocks of N^T L0^{-1} M
 * (eq. (N1M1)), the capacitance right-hand side, the trace vectors and
 * trace(E X0), and (pbar > 0) a truncated SVD of the off-diagonal coupling
 * for the preconditioner (eq. (prec)).
 *   A0: n x n; U, V: n x k; G: n x g; E: n x n symmetric, or NULL for I.
 *   1 <= k <= 8 (the per-row k x k blocks of the operator and of the
 *   preconditioner are held in registers), 1 <= n, k <= n, 1 <= g.
 * On success *out holds a device-resident seed; *cond_Q_out (may be NULL)
 * receives ||Qp||_F ||Qp^{-1}||_F.
 * Errors: LYAP_EINVAL, LYAP_EUNSTABLE_SEED (max Re lambda >= 0, or
 * min |lambda_i + lambda_j| below 1e-12 max |lambda|, where X is not unique),
 * LYAP_ENOMEM, LYAP_ESOLVER, LYAP_ECUDA. */
int lyap_seed_factor(lyap_ctx* ctx, int n, int k, int g, const double* A0, const double* U,
                     const double* V, const double* G, const double* E, int mem_kind,
                     const lyap_opts* opts, lyap_seed** out, double* cond_Q_out);

int lyap_seed_stats_get(const lyap_seed* seed, lyap_seed_stats* out);

/* Release a seed (device memory included). */
int lyap_seed_free(lyap_seed* seed);

/* Solve the capacitance systems of eq. (SMW_linearsystem) for nv parameter
 * vectors (v: nv x k, row i = v for system i, row-major, i.e. v[i*k + t]).
 * Systems are solved in the given order, in lockstep batches, recycling the
 * Krylov subspace across the sequence (§2.1). If w_out is not NULL it
 * receives, for each v, the shifted capacitance solution W' = W + P D(v) as
 * n x k complex128 (interleaved re, im; column-major), nv*n*k*2 doubles, in
 * mem_kind memory. info (may be NULL) receives nv reports (host memory).
 * Errors: LYAP_EINVAL (v_i == 0 or not finite, bad sizes; outputs are then
 * undefined), LYAP_ENOMEM, LYAP_ECUDA, LYAP_EDEVICE_TIMEOUT. */
int lyap_param_solve(lyap_seed* seed, int nv, const double* v, int mem_kind, const lyap_opts* opts,
                     double* w_out, lyap_result_info* info);

/* f(v) = trace(E X(v)) for nv parameter vectors (eq. (Xsmalllastline) and
 * the trace formula after it). trace_out: nv doubles in mem_kind memory.
 * info (may be NULL, host) gets per-result iterations, refinement steps, the
 * FP64 relative residual and err_est = |h^T r| / |f| with r the final FP64
 * capacitance residual and h the trace vector (a first-order estimate of the
 * relative trace error). Errors as lyap_param_solve. */
int lyap_trace_EX(lyap_seed* seed, int nv, const double* v, int mem_kind, const lyap_opts* opts,
                  double* trace_out, lyap_result_info* info);

/* f(v) and df/dv_i for nv parameter vectors: one adjoint capacitance solve
 * with T(v)^T per v (the transpose swaps Ub and Vb), then
 * df/dv_i = v_i^{-2} sum_s Z[s,i] W'[s,i] (derived from eq.
 * (SMW_linearsystem) with a v-independent right-hand side).
 * trace_out: nv doubles; grad_out: nv x k row-major; both in mem_kind
 * memory. Errors as lyap_param_solve. */
int lyap_grad(lyap_seed* seed, int nv, const double* v, int mem_kind, const lyap_opts* opts,
              double* trace_out, double* grad_out, lyap_result_info* info);

/* ----------------------------------------------------------------- serving
 * A continuous-batching server (an addition; the paper solves one
 * sweep at a time). Requests (one seed, nv parameter vectors) enter a FIFO
 * and are admitted while the registered seeds' resident bytes plus the
 * workspace estimate of all admitted, unfinished requests stay within
 * opts->hbm_budget (0: 80% of the free device memory at creation). Every
 * registered seed has its own CUDA stream and worker thread; whenever a
 * worker finishes a batch it takes every request admitted for its seed in
 * the meantime as its next lockstep batch, so requests arriving while
 * others run join at the next batch boundary of their seed, and batches of
 * different seeds overlap on the device. Factors and recycled Krylov spaces
 * stay resident in the seeds. A registered seed must not be used directly
 * while the server runs. All calls are host calls; pointers are host
 * memory; the server is safe to call from several host threads. */
int lyap_serve_create(lyap_ctx* ctx, const lyap_opts* opts, lyap_server** out);
/* Register a seed (the server does not take ownership). */
int lyap_serve_register_seed(lyap_server* srv, lyap_seed* seed, int* seed_id);
/* Device bytes that admission charges for a request of nv vectors on a
 * registered seed (the estimate lyap_serve_submit compares with the budget).
 * Errors: LYAP_EINVAL, LYAP_ENOTFOUND (seed id). */
int lyap_serve_estimate(lyap_server* srv, int seed_id, int nv, int want_grad, size_t* bytes);
/* Enqueue nv parameter vectors (nv x k row-major, copied); returns a ticket.
 * Errors: LYAP_EINVAL (v_i = 0 or not finite), LYAP_ENOTFOUND (seed id),
 * LYAP_ENOMEM (the request alone exceeds the budget). */
int lyap_serve_submit(lyap_server* srv, int seed_id, int nv, const double* v, int want_grad,
                      uint64_t* ticket);
/* Wait until every submitted request is finished (max_ms <= 0) or at most
 * max_ms milliseconds; the workers make progress on their own, this call
 * only waits. *busy (may be NULL) is set to 1 if work remains. */
int lyap_serve_run(lyap_server* srv, int max_ms, int* busy);
/* LYAP_PENDING until the request is done; then copies nv traces (and
 * nv x k gradients if requested), nv infos (each may be NULL) and the
 * submit-to-completion latency in seconds, returns the request's status
 * and forgets the ticket. A cancelled request returns LYAP_ECANCELLED. */
int lyap_serve_poll(lyap_server* srv, uint64_t ticket, double* trace_out, double* grad_out,
                    lyap_result_info* info, double* latency_s);
/* Cancel a request that has not been admitted yet (LYAP_EINVAL once it runs). */
int lyap_serve_cancel(lyap_server* srv, uint64_t ticket);
/* Finish running batches, stop the workers and free the server. */
void lyap_serve_destroy(lyap_server* srv);

/* --------------------------------------------- independent explicit check
 * Verification of given solutions through the explicit Lyapunov solution
 * (O(n^3) per vector, FP64): for nv parameter vectors v (nv x k row-major)
 * and their shifted capacitance solutions w (nv x n x k complex128, as
 * written by lyap_param_solve), forms
 *   X(v) = X0 + Qp (Lc o (W' Ub^T + Ub W'^T)) Qp^T
 * (§2.1, eqs. (splitXv), (seedLE), (Xsmalllastline)) and evaluates the true
 * residual of the equation, R = A(v)^T X + X A(v) + G G^T, from the
 * caller's A0 (n x n), U, V (n x k), G (n x g) and E (n x n symmetric or
 * NULL for I). backward_err_out[b] = ||R||_F / (2 ||A(v)||_F ||X||_F +
 * ||G G^T||_F) (the form of §2.2's backward error proposition) and
 * trace_out[b] = trace(E X(v)), both host arrays. All other pointers are
 * in mem_kind memory. Synchronises. Errors: LYAP_EINVAL, LYAP_ENOMEM,
 * LYAP_ECUDA, LYAP_ESOLVER. */
int lyap_check_explicit(lyap_seed* seed, int nv, const double* v, const double* w, const double* A0, const double* U,
                        const double* V, const double* G, int g, const double* E, int mem_kind,
                        double* backward_err_out, double* trace_out);

/* --------------------------------------------------- projection framework
 * The large-scale method of §2.2 (eqs. (EK_def), (param_projected), the
 * backward error proposition, Algorithm 1). One extended Krylov space
 * EK_m(A0^T, P), P = [X0 U, V] (eq. (rhs_newexpression) in this header's
 * convention), is built from the LU factors of A0 and serves every v; the
 * projected equation of each m is solved by the small-scale path above for
 * all remaining v in one batch, and v is accepted once its backward error
 * Delta_{m,v} <= eps.
 *
 * lyap_proj_create: A0 n x n, U, V n x k, E n x n symmetric or NULL (= I),
 *   column-major FP64 in mem_kind memory (copied). XBr (n x k) = X0 U, the
 *   seed solution times U, with fX0 = trace(E X0), as Assumption 2 of the
 *   paper supposes them available; when XBr is NULL both come from a
 *   one-off FP64 eigen-factorisation of A0 with G (n x g), which is then
 *   released. 1 <= k <= 8, 2k <= n. Errors: LYAP_EINVAL, LYAP_EUNSTABLE_SEED
 *   (A0 singular or, without XBr, not stable), LYAP_ENOMEM, LYAP_ESOLVER,
 *   LYAP_ECUDA.
 * lyap_proj_trace_EX: f(v) for nv parameter vectors (nv x k row-major, in
 *   mem_kind memory; outputs in the same kind). Algorithm 1 with the
 *   remaining vectors taken as one batch per m (every v whose Delta meets
 *   eps leaves, the others wait for the next block) while m < m_max; the
 *   space is kept and grown across calls. delta_out (may be NULL, host)
 *   receives Delta_{m,v}, blocks_out (may be NULL, host) the m used; info
 *   (may be NULL, host) reports LYAP_ENOCONV for a v whose Delta never met
 *   eps (its trace is then the last one computed). opts->precision selects
 *   the path of the projected solves. The call synchronises.
 * lyap_proj_dims: blocks built so far and the basis dimension.
 */
typedef struct lyap_proj lyap_proj;
int lyap_proj_create(lyap_ctx* ctx, int n, int k, int g, const double* A0, const double* U, const double* V,
                     const double* G, const double* E, const double* XBr, double fX0, int mem_kind,
                     const lyap_opts* opts, lyap_proj** out);
int lyap_proj_trace_EX(lyap_proj* proj, int nv, const double* v, int mem_kind, const lyap_opts* opts, double eps,
                       int m_max, double* trace_out, double* delta_out, int* blocks_out, lyap_result_info* info);
int lyap_proj_dims(const lyap_proj* proj, int* blocks, int* dim);
int lyap_proj_free(lyap_proj* proj);

/* ------------------------------------------------- allocation-free check
 * The paper has no counterpart to this call. It is for callers that cannot
 * allocate device memory while they run: hosts that reserve all of their
 * device memory once at start-up in their own pool and must not let it
 * grow, and plug-ins that live inside another framework's allocator and
 * may not go around it. For nv parameter vectors v (device, nv x k
 * row-major) and the caller's capacitance solutions w (device,
 * nv x n x k complex128 as written by lyap_param_solve), it writes
 * trace_out[b] = f(v_b) and resid_out[b] = ||P - T(v_b) W'_b|| / ||P|| in
 * FP64 (device, nv doubles each), in order on `stream` (NULL = default
 * stream), without synchronising.
 * It calls no allocation routine: intermediates live in one static device
 * array of LYAP_NOALLOC_MAX_ENTRIES complex doubles (33 MiB, 34,603,008
 * bytes, held by every GPU that loads the library until the process exits);
 * a call needs nv*n*k + ceil(nv*k/2) entries and returns LYAP_EINVAL when
 * that exceeds the limit. All calls share the array and it keeps the last
 * call's contents; every entry a call reads was written earlier in the same
 * call, so nothing needs clearing. Calls that overlap on the GPU (other
 * streams, or host threads without ordering) race on the array. The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress) once; make that first call before any stream
 * capture. A zero or non-finite v_i yields NaN in that system's residual
 * (its trace does not involve v). */
#define LYAP_NOALLOC_MAX_ENTRIES ((1u << 21) + (1u << 16))
int lyap_check_solution_noalloc(lyap_seed* seed, int nv, const double* v, const double* w, double* trace_out,
                                double* resid_out, void* stream);

/* ------------------------------------------------------- kernel accounting
 * For measurement only. lyap_prof_enable(1) clears the records and starts
 * timing selected kernels with CUDA events on their launch stream, together
 * with the algorithmic work of each launch (flops/bytes the method needs per
 * unit times the units, e.g. system-matvecs, the launch processed);
 * lyap_prof_enable(0) stops. lyap_prof_read synchronises the device and
 * returns one entry per kernel that ran, plus (launches != NULL) the number
 * of library kernel launches since the last enable. */
typedef struct {
  char name[32];
  long long launches;
  double total_ms;
  double units;
  double flops;
  double bytes;
} lyap_prof_kernel;

int lyap_prof_enable(int on);
int lyap_prof_read(lyap_prof_kernel* out, int max, int* count, long long* launches);

#ifdef __cplusplus
}
#endif

#endif /* LYAP_H */
