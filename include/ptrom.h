/*
 * ptrom.h -- C ABI of libptrom.so, the GB300 (sm_103a) implementation of the
 * projection-tree reduced-order model's hot path (arXiv 2103.01983).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - State layout (Sec. 2, Eq. 3): a state of n bodies is a length-2n FP64
 *    array x = [chi_1..chi_n, psi_1..psi_n]; velocities f use the same layout.
 *  - Circulations Gamma (length n, FP64) are the paper's Gamma_j; the factor
 *    1/(2 pi) of Eq. 2 is applied inside the library.
 *  - Unless a parameter says "host", every pointer is a DEVICE pointer
 *    allocated and owned by the caller; the library keeps no reference to it
 *    after the call returns.  Device buffers must be 8-byte aligned.
 *  - Every call is enqueued on the caller's CUDA stream `stream` (0 = the
 *    legacy default stream) and returns without synchronising, unless its
 *    comment says it synchronises (solvers that must read a convergence flag).
 *  - Every function returns a status: 0 (PTROM_OK) or a negative code below.
 *    On error nothing has been enqueued unless the code is PTROM_ECUDA (a CUDA
 *    error was reported while enqueuing or synchronising).  ptrom_last_error()
 *    returns a one-line description of the calling thread's last error.
 *  - Precision `prec`: PTROM_FP32C computes pair terms in FP32 and accumulates
 *    them with compensated (TwoSum) sums; inputs/outputs stay FP64.
 *    PTROM_FP64 computes everything in FP64 (slow on GB300; for checking).
 *    PTROM_TF32X3 (bs_jphi only; other calls reject it): the contraction
 *    runs on the tensor cores with each FP32 factor split into TF32 hi + lo
 *    parts and three products per term (hi*hi + hi*lo + lo*hi); the hi*hi
 *    sums run in tensor memory for at most 64 MMA steps, then fold into
 *    compensated totals.  PTROM_F16X3 (bs_jphi only): the same with FP16
 *    hi + lo parts (TF32's significand width, twice the K per MMA), the
 *    factors scaled by powers of two into FP16's range; delta = 0 falls
 *    back to PTROM_TF32X3.
 *  - A pair (i, j) whose positions coincide exactly is skipped in every sum:
 *    that is the j != i restriction of Eq. 1 (and a coincident body).
 */
#ifndef PTROM_H
#define PTROM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ptrom_stream_t; /* same type as cudaStream_t */

enum ptrom_status {
    PTROM_OK = 0,
    PTROM_EINVAL = -1,   /* bad argument (size, pointer, option)           */
    PTROM_ECUDA = -2,    /* a CUDA runtime call failed                     */
    PTROM_ENOCONV = -3,  /* iteration limit reached before the tolerance   */
    PTROM_ENAN = -4,     /* a NaN/Inf appeared in a residual               */
    PTROM_ETIMEOUT = -5, /* a device-side bounded wait gave up             */
    PTROM_ENOMEM = -6    /* a workspace was too small or allocation failed */
};

enum ptrom_prec { PTROM_FP32C = 0, PTROM_FP64 = 1, PTROM_TF32X3 = 2, PTROM_F16X3 = 3 };

/* Copies the calling thread's last error message into buf (NUL-terminated,
 * truncated to len) and returns the status it came with. */
int ptrom_last_error(char *buf, size_t len);

/* Library version (major*10000 + minor*100 + patch). */
int ptrom_version(void);

/* Tuning overrides for the all-pairs kernels (process-wide; results are
 * identical up to FP rounding for every choice, and each choice is
 * deterministic run to run).
 * ptrom_set_source_split(S): split every launch's sources over S CTAs per
 *   block of 64 targets (1 <= S <= 16; at most 8 with the cluster combine), or
 *   S = 0 to restore the automatic choice (the default).  Returns PTROM_EINVAL
 *   for S outside [0, 16]; a launch whose combine cannot take the forced S
 *   returns PTROM_EINVAL.
 * ptrom_set_split_mode(mode): how the S partial sums of a target block are
 *   added, both in a fixed split order:
 *     0  automatic (the default): global, unless a caller-supplied scratch
 *        holds the packed sources only (then cluster);
 *     1  cluster: the S CTAs form a thread-block cluster and add their
 *        partials through distributed shared memory (no scratch, S <= 8);
 *     2  global: each CTA writes its partial to scratch and the last to
 *        arrive adds them (S <= 16; PTROM_ENOMEM if a caller's scratch is too
 *        small).
 *   Returns PTROM_EINVAL for mode outside [0, 2]. */
int ptrom_set_source_split(int S);
int ptrom_set_split_mode(int mode);

/* Autotuning of the all-pairs source split S (with the global combine; a
 * forced S or the cluster combine bypasses it).
 * ptrom_tune_pairs(n, prec, delta, stream): times every S in 1..16 that
 *   leaves each warp at least 32 sources, for each all-pairs kernel the
 *   FOM step uses at n targets x n sources (velocity, velocity with self
 *   blocks, J v, J^T w with and without (df/dGamma)^T w) on synthetic
 *   bodies, and caches the fastest per (kernel, device, n, n); later launches
 *   of those shapes take it.  Synchronises the stream; allocates scratch from
 *   the library pool.  PTROM_EINVAL as bs_velocity.
 * ptrom_set_autotune(on): on = 1 tunes, the first time, any launch shape
 *   without a cached split (on the caller's data; not while the stream is
 *   being captured, and not for launches behind a device skip flag); that
 *   launch then synchronises its stream.  0 (the default) uses the cached
 *   split when there is one, else S = 4.  PTROM_EINVAL for on outside [0, 1].
 * ptrom_autotune_reset(): forgets every cached split. */
int ptrom_tune_pairs(int n, int prec, double delta, ptrom_stream_t stream);
int ptrom_set_autotune(int on);
int ptrom_autotune_reset(void);

/* Test hook for the tensor-core J Phi's failure path: with on = 1 the next
 * bs_jphi call with PTROM_TF32X3 or PTROM_F16X3 withholds its tile copies, so every pipeline
 * wait in every CTA runs out at its 1 s bound; each CTA then waits (bounded)
 * for its work in flight, frees its tensor memory and flags the status, and
 * the call returns PTROM_ETIMEOUT with the stream still usable.  The hook
 * clears itself after that one call.  PTROM_EINVAL for on outside [0, 1]. */
int ptrom_test_withhold_jphi_tc(int on);

/* Instrumentation (host-side, process-wide).
 * ptrom_launch_count: number of CUDA kernels the library has launched so far.
 * ptrom_timing_enable(on): on = 0 stops recording; on = 1 brackets every
 *   timed launch of any kind below with two CUDA events recorded on the
 *   launch's own stream (up to 65536 launches; later ones are not timed);
 *   any other positive `on` is a bit mask (bit k = kind k) of the kinds to
 *   time, so a caller can time the all-pairs kernels alone (the events of
 *   the small kinds add launch gaps of their own); bit 30 is ignored, so
 *   (1 << 30) | 1 times kind 0 alone.
 * ptrom_timing_read: synchronises the recorded events and returns, for each
 *   kernel kind k < nkinds (enum ptrom_kernel_kind), the summed device time in
 *   milliseconds (ms[k]) and the number of timed launches (count[k]); then
 *   forgets them.  Returns PTROM_EINVAL for NULL arrays or nkinds < 1. */
enum ptrom_kernel_kind {
    PTROM_K_VELOCITY = 0,      /* bs_velocity without self blocks */
    PTROM_K_VELOCITY_D = 1,    /* bs_velocity with self blocks    */
    PTROM_K_JVP = 2,
    PTROM_K_VJP = 3,
    PTROM_K_JPHI = 4,
    PTROM_K_PTROM_STEP = 5,
    PTROM_K_PACK = 6,          /* source packing before an all-pairs launch     */
    PTROM_K_FOM_VEC = 7,       /* FOM vector kernels: residual, normalise +
                                  precondition, GMRES correction, updates      */
    PTROM_K_FOM_ORTH = 8,      /* FOM CGS2 orthogonalisation + least squares    */
    PTROM_K_NKINDS = 9
};
long long ptrom_launch_count(void);
int ptrom_timing_enable(int on);
int ptrom_timing_read(double *ms, long long *count, int nkinds);

/*
 * bs_velocity -- regularised Biot-Savart velocity (Sec. 2, Eq. 1-2):
 *     f_i = sum_{j != i} Gamma_j/(2 pi) e3 x (t_i - s_j) / (|t_i - s_j|^2 + delta)
 * for nt targets t (xt, length 2*nt) and ns sources s (xs, length 2*ns,
 * strengths Gamma, length ns).  Targets may be the sources themselves
 * (xt == xs, nt == ns) or any other points (e.g. grid vertices, Sec. 6.1).
 *   f_out        [2*nt]  velocity at the targets.
 *   selfjac_out  [3*nt]  optional (NULL to skip): the per-target 2x2 block
 *                d f_i / d t_i = sum_j gamma_j A(t_i - s_j), the "diagonal
 *                block entries" of the inexact kernel Jacobian (Sec. 2, last
 *                paragraph), stored as [D00 (nt) | D01 (nt) | D10 (nt)];
 *                D11 = -D00 (the block is trace-free).
 * Errors: nt < 1 or ns < 1, delta < 0, NULL arrays, bad prec -> PTROM_EINVAL.
 */
int bs_velocity(int nt, const double *xt, int ns, const double *xs,
                const double *Gamma, double delta, double *f_out,
                double *selfjac_out, int prec, ptrom_stream_t stream);

/*
 * bs_velocity_noalloc -- bs_velocity for callers that must not allocate device
 * memory while they run.  The paper has no counterpart; this is a library
 * service.  bs_velocity takes a scratch buffer for its packed sources from a
 * stream-ordered memory pool on every call; a control or serving loop whose
 * memory policy forbids device allocation after start-up (an allocation can
 * block, fail under memory pressure or change the footprint mid-run), or a
 * process whose device memory belongs to another framework's allocator, cannot
 * accept that.  This variant keeps the scratch in one fixed device array
 * inside the library instead: PTROM_NOALLOC_MAX_SOURCES sources (3 MiB), held
 * by every GPU that loads the library until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 * Arguments, outputs and precision are those of bs_velocity.
 * Errors: as bs_velocity, plus PTROM_EINVAL when ns > PTROM_NOALLOC_MAX_SOURCES.
 * Notes: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  All calls share the one array and it keeps the last
 * call's contents (every record a call reads, and every arrival counter of its
 * source split's combine, is rewritten by that call first, so nothing needs
 * clearing); calls that overlap on the GPU -- on different
 * streams, or from different host threads -- race on it and must be ordered
 * by the caller.
 */
#define PTROM_NOALLOC_MAX_SOURCES 65536
int bs_velocity_noalloc(int nt, const double *xt, int ns, const double *xs,
                        const double *Gamma, double delta, double *f_out,
                        double *selfjac_out, int prec, ptrom_stream_t stream);

/*
 * bs_jvp -- Jacobian-vector product of the kernel, jv = (d f / d x) v, with
 * all blocks (the exact Jacobian whose product the Gauss-Newton/LSPG step of
 * Sec. 3.2 and a Jacobian-free Newton solve of Eq. linKstep need):
 *     (J v)_i = sum_{j != i} gamma_j A(x_i - x_j) (v_i - v_j),  gamma = Gamma/(2 pi).
 * x, v, jv: [2n]; Gamma: [n].  Errors as bs_velocity (n < 2 -> PTROM_EINVAL).
 */
int bs_jvp(int n, const double *x, const double *Gamma, double delta,
           const double *v, double *jv, int prec, ptrom_stream_t stream);

/*
 * bs_vjp -- transposed products (adjoint of Sec. 2's kernel):
 *     gx = (d f / d x)^T w,     (J^T w)_k = sum_j A(x_k - x_j)^T (gamma_j w_k - gamma_k w_j)
 *     gGamma = (d f / d Gamma)^T w,   gGamma_k = sum_i w_i . e3 x (x_i - x_k) / (2 pi s_ik)
 * Either output may be NULL (not computed).  x, w, gx: [2n]; Gamma, gGamma: [n].
 */
int bs_vjp(int n, const double *x, const double *Gamma, double delta,
           const double *w, double *gx_out, double *gGamma_out, int prec,
           ptrom_stream_t stream);

/*
 * bs_jphi -- the kernel Jacobian applied to every column of a basis,
 *     out = (d f / d x) Phi,   (J Phi)_i = sum_{j != i} gamma_j A(x_i - x_j) (Phi_i - Phi_j),
 * the J Phi of the LSPG Gauss-Newton least squares (Sec. 3.2, Eq.
 * GNLinearLeastSquares) with the exact kernel Jacobian.
 *   phi, out  [2n x M], column-major (column m is a state-layout vector at
 *             phi + m*2n).  x [2n], Gamma [n].
 *   prec      PTROM_FP32C (FP32 pipes), PTROM_FP64, or PTROM_TF32X3 /
 *             PTROM_F16X3: the sum over sources as S_i Phi_i - sum_j K_ij
 *             Phi_j (K_ij the pair block, S_i = sum_j K_ij), the second term
 *             a tensor-core contraction whose pair blocks are generated in
 *             shared memory; these precisions synchronise the stream (they
 *             read a status).
 * Errors: n < 2, M < 1, delta < 0, NULL arrays, bad prec -> PTROM_EINVAL;
 * PTROM_TF32X3 / PTROM_F16X3 only: PTROM_ETIMEOUT if a bounded pipeline wait
 * gave up.
 */
int bs_jphi(int n, const double *x, const double *Gamma, double delta,
            const double *phi, int M, double *out, int prec, ptrom_stream_t stream);

/* ------------------------------------------------------------------------
 * Full-order model (FOM): one implicit trapezoid step (Sec. 2, Eq. linKstep
 * with k=1, alpha0=1, alpha1=-1, beta0=beta1=1/2):
 *     r(xi) = xi - x^{n-1} - dt/2 (f(xi) + f(x^{n-1})) = 0,
 * solved by Newton from xi = x^{n-1}; each iteration solves
 * (I - dt/2 J) d = -r and sets xi += d, with J chosen by jac_mode:
 *   PTROM_JAC_BLOCKDIAG  only the per-body 2x2 self blocks d f_i/d x_i: the
 *                        paper's inexact kernel Jacobian (Sec. 2);
 *   PTROM_JAC_DENSE      the full 2n x 2n Jacobian, assembled in FP64 and
 *                        LU-factorised with partial pivoting (n <= 4096);
 *   PTROM_JAC_JFNK       the full Jacobian applied matrix-free through the
 *                        J v kernel inside restarted GMRES, right-
 *                        preconditioned by the block-diagonal Jacobian.
 * The Jacobian (self blocks / dense factors) is refreshed every p_it Newton
 * iterations.  Convergence: ||r||_2 <= tol * max(1, ||xi||_2), checked after
 * each evaluation of f(xi) (so the returned f is f at the returned state).
 * Optional superimposed inflow u (Sec. 6.3: a constant velocity per body,
 * dx/dt = f(x) + u): the residual becomes
 *     r(xi) = xi - x^{n-1} - dt/2 (f(xi) + f(x^{n-1})) - dt u,
 * the Jacobian is unchanged, and f (in/out) stays the pair sum of Eq. 2.
 * ------------------------------------------------------------------------ */
enum ptrom_jac_mode { PTROM_JAC_BLOCKDIAG = 0, PTROM_JAC_DENSE = 1, PTROM_JAC_JFNK = 2 };

typedef struct ptrom_fom_params {
    double dt;          /* time step (> 0)                                   */
    double delta;       /* de-singularisation constant delta_k of Eq. 2     */
    double tol;         /* Newton tolerance (see above)                     */
    int max_iter;       /* Newton iteration cap (the paper uses 100)         */
    int jac_mode;       /* enum ptrom_jac_mode                               */
    int p_it;           /* Jacobian refresh period in Newton iterations >= 1 */
    int prec;           /* pair-sum precision, enum ptrom_prec               */
    int gmres_restart;  /* JFNK: Krylov vectors per cycle, 1..64             */
    int gmres_max_iter; /* JFNK: Krylov iterations per Newton step           */
    double gmres_rtol;  /* JFNK: relative linear tolerance                   */
    const double *u_inf; /* superimposed inflow: DEVICE [2n] ([u_chi..., u_psi...])
                            or NULL for none; fom_step_batched requires NULL,
                            fom_adjoint_step ignores it (u does not depend on
                            x or Gamma)                                      */
} ptrom_fom_params;

typedef struct ptrom_fom_stats {
    int newton_iters;   /* Newton iterations taken (solves performed)        */
    int linear_iters;   /* total GMRES iterations (JFNK)                     */
    int velocity_evals; /* all-pairs velocity launches                       */
    int jvp_evals;      /* all-pairs J v launches                            */
    double res_norm;    /* ||r||_2 at the returned state                     */
    double res_norm0;   /* ||r||_2 at xi = x^{n-1}                           */
} ptrom_fom_stats;

/* Device workspace (bytes) fom_step needs for these parameters and n. */
size_t fom_workspace_bytes(const ptrom_fom_params *p, int n);

/*
 * fom_step -- advance one implicit trapezoid step.
 *   p      host pointer to the parameters.
 *   Gamma  [n] circulations.
 *   x      [2n] in: x^{n-1}; out: x^n (the last Newton iterate).
 *   f      [2n] in: f(x^{n-1}); out: f(x^n).
 *   work   device workspace of at least fom_workspace_bytes(p, n) bytes,
 *          256-byte aligned, owned by the caller; its contents on entry do not
 *          matter.  Calls that share one workspace must not overlap in time.
 *   stats  optional host pointer (NULL to skip).
 * Synchronises `stream` once per Newton iteration (to read ||r||) and once
 * per GMRES iteration.  Returns PTROM_ENOCONV if max_iter iterations did not
 * reach tol (x, f then hold the last iterate), PTROM_ENAN on a non-finite
 * residual, PTROM_EINVAL for bad parameters (n < 2, dt <= 0, delta < 0,
 * dense mode with n > 4096, work too small).
 */
int fom_step(const ptrom_fom_params *p, int n, const double *Gamma, double *x,
             double *f, void *work, size_t work_bytes, ptrom_fom_stats *stats,
             ptrom_stream_t stream);

/*
 * fom_steps -- nsteps implicit trapezoid steps (as fom_step, block-diagonal
 * Newton, p->jac_mode = PTROM_JAC_BLOCKDIAG only) with each step replayed
 * from one CUDA graph: the step's kernels (per Newton iteration the velocity
 * and self blocks, then the residual, Newton test and update) are captured
 * once for `iters` iterations, every kernel after the converged iteration
 * skips itself through a device flag, and the host reads the steps' status
 * once at the end instead of once per iteration.  iters: Newton iterations
 * captured per step (1 .. max_iter + 1), or 0: the first step runs as
 * fom_step and iters = its velocity evaluations + 2.  A step that does not
 * converge within iters stops the rollout there (later steps do nothing):
 * PTROM_ENOCONV with x at that step's last iterate (PTROM_ENAN for a
 * non-finite residual); *steps_done (optional) counts the converged steps.
 * stats (optional) sums the steps' counts.  Falls back to step-by-step
 * fom_step calls where the cooperative Newton kernel does not fit the GPU
 * and while ptrom_timing_enable is on.  Synchronises the stream at the end.
 * Errors: as fom_step, plus PTROM_EINVAL for another jac_mode, nsteps < 1
 * or iters outside [0, max_iter + 1].
 */
int fom_steps(const ptrom_fom_params *p, int n, const double *Gamma, double *x, double *f,
              void *work, size_t work_bytes, int nsteps, int iters, ptrom_fom_stats *stats,
              int *steps_done, ptrom_stream_t stream);

/*
 * Batched FOM over B independent instances of uneven size (parameter sweeps):
 * bs_velocity_batched evaluates Eq. 2 (optionally with the self blocks) for
 * every instance in ONE pack launch and ONE all-pairs launch (a flattened
 * work list of 64-target blocks).  fom_step_batched advances every instance
 * by one trapezoid step with the paper's inexact block-diagonal Newton; each
 * Newton iteration is one batched launch for the instances not yet converged.
 * n, x, Gamma, f, selfjac_out, work, work_bytes: HOST arrays of length B
 * holding per-instance sizes / DEVICE pointers / byte counts
 * (work[b]: fom_workspace_bytes(p, n[b]) bytes, 256-byte aligned);
 * delta: host array of per-instance constants (velocity); stats: optional
 * host array of B.  fom_step_batched synchronises once per Newton iteration
 * and requires p->jac_mode == PTROM_JAC_BLOCKDIAG.
 */
int bs_velocity_batched(int B, const int *n, const double *const *x,
                        const double *const *Gamma, const double *delta,
                        double *const *f_out, double *const *selfjac_out, int prec,
                        ptrom_stream_t stream);
int fom_step_batched(const ptrom_fom_params *p, int B, const int *n,
                     const double *const *Gamma, double *const *x, double *const *f,
                     void *const *work, const size_t *work_bytes,
                     ptrom_fom_stats *stats, ptrom_stream_t stream);

/*
 * fom_adjoint_step -- reverse-mode derivative of one fom_step (implicit
 * function theorem on the trapezoid residual r(x^n, x^{n-1}, Gamma) = 0 of
 * Eq. linKstep).  Given lambda = dL/dx^n:
 *     mu            = (I - dt/2 J(x^n))^{-T} lambda   (GMRES on the J^T w kernel,
 *                      right-preconditioned by the transposed self blocks)
 *     lambda  <-      mu + dt/2 J(x^{n-1})^T mu       (= dL/dx^{n-1})
 *     gGamma  +=      dt/2 (F(x^n) + F(x^{n-1}))^T mu,  F = d f / d Gamma.
 * x_n, x_prev [2n]: the step's end and start states (as fom_step produced
 * them); lambda [2n] in/out; gGamma [n] accumulated.  p's gmres_* fields and
 * prec are used (jac_mode is ignored).  work: fom_adjoint_workspace_bytes.
 */
size_t fom_adjoint_workspace_bytes(const ptrom_fom_params *p, int n);
int fom_adjoint_step(const ptrom_fom_params *p, int n, const double *Gamma,
                     const double *x_n, const double *x_prev, double *lambda,
                     double *gGamma, void *work, size_t work_bytes,
                     ptrom_fom_stats *stats, ptrom_stream_t stream);

/* ------------------------------------------------------------------------
 * Projection-tree ROM (PTROM): online Gauss-Newton (Alg. 4) over the hyper-
 * reduced pairwise interaction (Alg. 5), at the sampled bodies against the
 * clustered sources (Sec. 5.2).
 *
 * A model holds, for n_s sampled bodies (n_d = 2 n_s dofs, order
 * [chi_1..chi_ns, psi_1..psi_ns]), M POD modes, M_r residual modes and N_c
 * source clusters:
 *   phi_s   [n_d x M]   row-major: the sampled rows of Phi (Phi bar)
 *   x0_s    [n_d]       sampled rows of x^0(mu)
 *   phi_c   [2 N_c x M] row-major: cluster POD surrogates Phi~ (rows
 *                       [chi of every cluster; psi of every cluster])
 *   x0_c    [2 N_c]     cluster reference positions x^0_QT(mu)
 *   gamma_c [N_c]       cluster circulations Gamma~(mu)
 *   off     [n_s + 1], idx [off[n_s]]: CSR lists, sampled body i interacts
 *                       with clusters idx[off[i] .. off[i+1])
 *   A       [M_r x n_d] row-major: the gappy operator [P Phi_r]^+
 * Limits: M <= 128, M_r <= 256, n_s <= 512, N_c <= 1048576.  The clusters'
 * current positions x^QT live in the instance's shared memory while they fit
 * beside the rest (N_c up to several thousand), else in the instance's state
 * buffer, which ptrom_state_bytes then sizes to hold them.  The rest of the
 * working set -- [A C | A r] (8 M_r (M + 1) bytes with the FP64 least
 * squares, 4 M_r (M + 1) with FP32) and the per-sampled-body arrays -- must
 * fit one CTA's 220 KB of shared memory: M = 128 with M_r = 256 needs the
 * FP32 least squares (the FP64 one fits up to M_r ~ 160 at M = 128);
 * otherwise PTROM_EINVAL.
 * ------------------------------------------------------------------------ */
typedef struct ptrom_model ptrom_model;

typedef struct ptrom_model_desc {
    int n_s, M, M_r, N_c;
    double dt, delta;
    double tol;     /* Gauss-Newton tolerance on eps (Alg. 4)               */
    int max_gn;     /* Gauss-Newton iteration cap (the paper uses 100)      */
    int qr_prec;    /* PTROM_FP64 (FP64 Householder QR) or PTROM_FP32C (FP32) */
    /* HOST arrays, copied into the model */
    const double *phi_s, *x0_s, *phi_c, *x0_c, *gamma_c, *A;
    const int *off, *idx;
    const double *u_s;  /* [n_d] superimposed inflow at the sampled dofs (Sec. 6.3),
                           or NULL for none: the residual gains -dt u_s        */
} ptrom_model_desc;

typedef struct ptrom_stats {
    long long gn_iters;   /* Gauss-Newton iterations over all steps/instances */
    long long steps;      /* time steps taken (all instances)                */
    int noconv;           /* steps that hit max_gn                           */
    int max_iters;        /* largest iteration count of one step             */
} ptrom_stats;

/* Create a model on the current device from host arrays (copied).  The
 * model is immutable afterwards except through ptrom_set_param.
 * Errors: sizes out of the limits, NULL arrays, CSR indices out of range. */
int ptrom_model_create(const ptrom_model_desc *desc, ptrom_model **out);
void ptrom_free(ptrom_model *m);

/* Replace the parameter-dependent arrays (Sec. 5.2: reload the clustered
 * circulation for a new mu) -- x0_s, phi_c, x0_c, gamma_c (HOST, same sizes;
 * any may be NULL to keep the current one). */
int ptrom_set_param(ptrom_model *m, const double *x0_s, const double *phi_c,
                    const double *x0_c, const double *gamma_c);

/* Replace the superimposed inflow at the sampled dofs (HOST [n_d], or NULL
 * to remove it).  Like the circulation, the inflow is a parameter that
 * needs no retraining (Sec. 5.2). */
int ptrom_set_inflow(ptrom_model *m, const double *u_s);

/* Device bytes of per-instance online state for a model (xhat, the carried
 * velocity at the sampled dofs, flags). */
size_t ptrom_state_bytes(const ptrom_model *m);

/*
 * ptrom_step -- advance `batch` independent instances of one or more models
 * by `nsteps` time steps in ONE launch (one CTA per instance).
 *   models  [batch] host array of model handles (may repeat one model)
 *   state   [batch] host array of device pointers, each ptrom_state_bytes
 *           bytes, 256-byte aligned; zero-filled state means xhat = 0 and
 *           "carried velocity not yet computed" (computed at xhat as R11)
 *   xhat    [batch] host array of device pointers to M doubles: on return
 *           the reduced coordinates after the last step (also in the state)
 *   hist    optional [batch] host array of device pointers to nsteps x M
 *           doubles receiving xhat after every step (NULL to skip)
 *   stats   optional host pointer; filling it synchronises the stream.
 * Errors: PTROM_EINVAL for bad arguments.  Non-convergence of one step is
 * counted in stats (the step keeps its last iterate, as Alg. 4 does at
 * k = max_gn), not an error.
 */
int ptrom_step(ptrom_model *const *models, int batch, void *const *state,
               double *const *xhat, double *const *hist, int nsteps,
               ptrom_stats *stats, ptrom_stream_t stream);

/* ------------------------------------------------------------------------
 * ptrom_build -- the offline training of Sec. 5.1 for one or more training
 * parameters mu_p (circulations Gamma_p, initial states x0_p):
 *   Stage 1  FOM snapshots: the states x^n(mu_p), n = 1..steps (fom_step
 *            with the given FOM parameters), as Sec. 3.1 defines them, or
 *            the caller's (p->snapshots);
 *   Stage 2  POD Phi (M modes, Sec. 3.1) of all snapshots (exact: the
 *            eigenvectors of the smaller of S^T S and S S^T; randomized range
 *            finder with power iterations when min(2n, snapshots) exceeds
 *            ptrom_set_pod_exact_max's bound, default 2048); the quadtree of
 *            the weighted POD space W = Phi sigma (Sec. 4.1.1) and the source
 *            clusters of every body (Alg. 2 with Alg. 3: Barnes-Hut theta or
 *            neighbour p_c);
 *   Stage 3  Tier-II LSPG (Eq. GNLinearLeastSquares) over all bodies with the
 *            clustered sources, the inexact block-diagonal Jacobian and
 *            alpha = 1, run once per training parameter (its x0_p and its
 *            cluster values), collecting the residual at every Gauss-Newton
 *            iterate;
 *            residual POD Phi_r (M_r modes);
 *   Stage 4  greedy sampling of n_s bodies (Alg. 1), A = [P Phi_r]^+.
 * The returned online model is set to the first training parameter; use
 * ptrom_set_param_full (and ptrom_set_inflow_full) for any other mu.
 * All input arrays are DEVICE arrays: x0s [n_params][2n], gammas
 * [n_params][n], and p->u_infs [n_params][2n] (per-parameter superimposed
 * inflow, or NULL; p->fom.u_inf is ignored).  Limits of this build: n_params * steps <= 65536 snapshots
 * of at most 64 GB in all, n <= 131072; the residual snapshots keep up to 10
 * Gauss-Newton iterates per step (up to 24 GB), later ones are dropped.
 * Synchronises the stream (the host runs the tree and the small dense
 * algebra).
 * ------------------------------------------------------------------------ */
enum ptrom_criterion { PTROM_BARNES_HUT = 0, PTROM_NEIGHBOR = 1 };

typedef struct ptrom_build_params {
    int M, M_r, n_s;       /* POD rank, residual rank, sampled bodies        */
    int criterion;         /* enum ptrom_criterion                           */
    double theta, p_c;     /* Barnes-Hut opening ratio / neighbour factor    */
    int steps;             /* training time steps per parameter              */
    double tol;            /* Gauss-Newton tolerance (Tier II and online)    */
    int max_gn;            /* Gauss-Newton cap (Tier II and online)          */
    int qr_prec;           /* online least-squares precision                 */
    ptrom_fom_params fom;  /* Stage 1 FOM (dt and delta are the model's)     */
    const double *u_infs;  /* DEVICE [n_params][2n] inflow per parameter, or NULL */
    const double *snapshots; /* DEVICE [n_params * steps][2n]: the caller's Stage 1
                              states x^1..x^steps of each parameter in turn (read
                              only), or NULL to run the FOM                    */
} ptrom_build_params;

typedef struct ptrom_build_info {
    int n_snapshots, n_res_snapshots;  /* Stage 1 / Stage 3 columns          */
    int N_c;                           /* unique clusters of the sampled bodies */
    int N_c_all;                       /* unique clusters over all bodies    */
    double mean_list;                  /* mean clusters per sampled body     */
    double mean_list_all;              /* mean clusters per body (Tier II)   */
    double sigma_ratio;                /* sigma_M / sigma_1                   */
    double seconds_fom, seconds_pod, seconds_tree, seconds_tier2, seconds_sample;
} ptrom_build_info;

int ptrom_build(const ptrom_build_params *p, int n, int n_params, const double *x0s,
                const double *gammas, ptrom_model **out, ptrom_build_info *info,
                ptrom_stream_t stream);

/* POD method switch: exact eigensolve while min(2n, snapshots) <= n_max,
 * randomized above (default 2048).  Process-wide.  PTROM_EINVAL for n < 1. */
int ptrom_set_pod_exact_max(int n_max);

/* Reload a built model for a new parameter from the full per-body arrays
 * (DEVICE, [2n] and [n]): cluster circulations, POD surrogates and reference
 * positions are recomputed from the stored memberships (Sec. 5.2), without
 * retraining.  PTROM_EINVAL for models not made by ptrom_build. */
int ptrom_set_param_full(ptrom_model *m, const double *x0, const double *Gamma,
                         ptrom_stream_t stream);

/* Set a built model's superimposed inflow from the full per-body array
 * (DEVICE [2n]; NULL removes it): its sampled rows become the model's u_s. */
int ptrom_set_inflow_full(ptrom_model *m, const double *u, ptrom_stream_t stream);

/* x = x^0 + Phi xhat on the listed bodies (Sec. 5.3): rows [nrows] (DEVICE
 * int body indices), out [2 nrows] ([chi..., psi...]), xhat [M] (DEVICE).
 * Only for models made by ptrom_build (they keep Phi and x^0). */
int ptrom_reconstruct(const ptrom_model *m, const double *xhat, const int *rows,
                      int nrows, double *out, ptrom_stream_t stream);

/* Training data of a model made by ptrom_build in this process (a model
 * read by ptrom_load has none), for inspection and tests; any pointer may be
 * NULL.  M_r, n_params, steps: the residual basis size, the training
 * parameters and the time steps of each.  phi_r [2n x M_r] (HOST, row-major):
 * the residual POD basis of Stage 3b, on which Alg. 1 sampled.  tier2_xhat
 * [n_params x (steps + 1) x M] (HOST): the Tier-II LSPG reduced trajectory of
 * every training parameter (Stage 3), from xhat = 0.  PTROM_EINVAL for other
 * models. */
int ptrom_model_query_training(const ptrom_model *m, int *M_r, int *n_params, int *steps,
                               double *phi_r, double *tier2_xhat);

/* The online model's clusters, for inspection and tests; any pointer may be
 * NULL, and a first call with only the sizes tells how large the arrays are.
 * N_c clusters; list_off [n_s + 1], list_idx [n_list] (HOST): sampled body s
 * interacts with clusters list_idx[list_off[s] .. list_off[s+1]-1]; mem_off
 * [N_c + 1], mem [n_members] (HOST): cluster c's member bodies (models made by
 * ptrom_build or read by ptrom_load from one; PTROM_EINVAL otherwise);
 * phi_c [2 N_c x M] (row-major, chi rows then psi rows), x0_c [2 N_c],
 * gamma_c [N_c] (HOST): the clusters' POD surrogates, reference positions and
 * circulations (Def. 1) for the model's current parameter. */
int ptrom_model_query_clusters(const ptrom_model *m, int *N_c, int *n_list, int *n_members,
                               int *list_off, int *list_idx, int *mem_off, int *mem,
                               double *phi_c, double *x0_c, double *gamma_c);

/* Alg. 1 greedy sampling of bodies, on the host (no CUDA call).
 * phi_r [2n x M_r] (HOST, row-major: rows chi_1..chi_n, psi_1..psi_n), the
 * residual basis; sampled [n_s] (HOST, out): body ids in the order chosen.
 * Readings of the garbled counters: n_c = min(M_r, 2 n_s), n_it = min(n_c,
 * n_s), iteration i takes n_ci = floor(n_c/n_it) + [i <= n_c mod n_it] more
 * columns and n_ai = floor(n_s/n_it) + [i <= n_s mod n_it] bodies; from i = 2
 * on, the new columns minus their minimum-norm gappy fit by the earlier
 * columns on the chosen bodies' dofs; a body's error is the squared norm of
 * its two rows; ties go to the lowest body id.  ptrom_build runs the same
 * code.  PTROM_EINVAL for n < 1, M_r < 1, n_s outside [1, n] or NULL arrays. */
int ptrom_greedy_sample(int n, int M_r, const double *phi_r, int n_s, int *sampled);

/* The gappy operator A = [P Phi_r]^+ (Eq. gappySolution; the Moore-Penrose
 * inverse, so the minimum-norm right inverse when 2 n_s < M_r), on the host
 * (no CUDA call): phi_r as above, sampled [n_s] (HOST), A [M_r x 2 n_s]
 * (HOST, out, row-major; columns chi of the sampled bodies, then psi).
 * PTROM_EINVAL for bad sizes, NULL arrays or a body id outside [0, n). */
int ptrom_gappy_operator(int n, int M_r, const double *phi_r, int n_s, const int *sampled, double *A);

/* Host copies of a built model's offline data, for inspection and tests:
 * any pointer may be NULL.  phi [2n x M] row-major, sigma [M],
 * sampled [n_s] (body ids in Alg. 1 order), A [M_r x 2 n_s] row-major. */
int ptrom_model_query(const ptrom_model *m, int *n, int *M, int *M_r, int *n_s,
                      int *N_c, double *phi, double *sigma, int *sampled, double *A);

/* ------------------------------------------------------------------------
 * ptrom_save / ptrom_load -- a model as one binary file, so the offline
 * stages of Sec. 5.1 run once and the online model of Sec. 5.2-5.3 is
 * reloaded without retraining.
 *   ptrom_save  writes every array the model was created or last
 *               reparametrised with (FP64 host copies, not the FP32 device
 *               forms), plus, for models made by ptrom_build, the basis,
 *               singular values, sampled bodies, cluster memberships and the
 *               current x^0; the file ends with a 64-bit FNV-1a hash.
 *   ptrom_load  reads such a file and creates the model on the current
 *               device (as ptrom_model_create would); the caller owns *out
 *               and releases it with ptrom_free.  A loaded model steps,
 *               reparametrises and reconstructs exactly as the saved one.
 * Errors: PTROM_EINVAL for NULL arguments, files that cannot be opened or
 * written, a wrong tag, byte order or format version, a failed hash, array
 * lengths that disagree with the sizes, or out-of-range indices; PTROM_ECUDA
 * / PTROM_ENOMEM from the device upload.  On error *out is NULL.
 * ------------------------------------------------------------------------ */
int ptrom_save(const ptrom_model *m, const char *path);
int ptrom_load(const char *path, ptrom_model **out);

#ifdef __cplusplus
}
#endif
#endif /* PTROM_H */
