/* psr.h -- C ABI of libpsr, a batched steady-state perfectly-stirred-reactor (PSR)
 * solver for NVIDIA GB300 (sm_103a).
 *
 * Method (Adhikari, Sayre & Chandy, "Towards using GPGPU units for accelerating the
 * batched perfectly stirred reactor (PSR) calculations"): every reactor of a batch
 * solves the steady form of the mass, species and energy balances of Sec. 2,
 * Eqs. (1)-(3), with the net production rates of Sec. 3, Eqs. (4)-(9), by the hybrid
 * Newton / pseudo-transient scheme of Sec. 3 (Newton iteration on the error vector
 * with an LU-factored Jacobian; when Newton fails the estimate is conditioned by time
 * integration and Newton is tried again). The batch is the paper's "n independent
 * PSRs solved simultaneously" (Sec. 6).
 *
 * Conventions
 *  - Every function returns an int status: PSR_OK (0) or a negative PSR_E_* code;
 *    psr_last_error() returns a thread-local message for the last failure. No C++
 *    exception crosses this interface.
 *  - Units are CGS: mass fractions, K, s, dyn/cm^2, mol/cm^3.
 *  - Batch arrays are row-major: [B][K] for species arrays (one contiguous row per
 *    reactor), [B] for per-reactor scalars, [B][K+1][K+1] for Jacobians.
 *  - Unless a function says otherwise, pointers are DEVICE pointers owned by the
 *    caller, and the work is queued on the given CUDA stream (NULL = legacy default
 *    stream) without synchronising; results are valid once the stream reaches them.
 *  - Per-reactor outcomes (convergence failures) are reported in status[], never as a
 *    call error. Call errors are argument errors, CUDA errors and allocation failures.
 */
#ifndef PSR_H
#define PSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* call status */
#define PSR_OK 0
#define PSR_E_ARG (-1)      /* invalid argument (null pointer, size, option value) */
#define PSR_E_IO (-2)       /* mechanism file cannot be read */
#define PSR_E_FORMAT (-3)   /* mechanism text malformed */
#define PSR_E_CUDA (-4)     /* CUDA runtime error (message in psr_last_error) */
#define PSR_E_OOM (-5)      /* device or host allocation failed */
#define PSR_E_UNSUPPORTED (-6) /* valid input this build does not handle (e.g. too many species) */

/* per-reactor status written to status[] */
#define PSR_CONVERGED 0     /* ||F||_inf <= ftol and the last Newton step met the polish tolerance */
#define PSR_MAX_ITER 1      /* max_newton Newton iterations used */
#define PSR_NONFINITE 2     /* the residual at the initial guess is not finite */
#define PSR_TS_EXHAUSTED 4  /* max_ts_rounds time-stepping rounds, or dt collapsed */
#define PSR_REFINE_FALLBACK 5 /* PSR_MIXED: converged (same criterion) after the FP32-Jacobian
                                 launch left it unconverged and the FP64 re-solve succeeded */
#define PSR_BAD_INPUT 7     /* psr_batch_solve_multi: mechanism id out of range, not solved */

/* Jacobian of the Newton iteration (options.jacobian) */
#define PSR_JAC_ANALYTIC 0
#define PSR_JAC_FD 1        /* central differences, as the paper builds it (Sec. 1) */

/* precision of the Jacobian and its LU factors (the residual is always FP64) */
#define PSR_FP64 0
#define PSR_MIXED 1         /* FP32 Jacobian, FP32 LU; FP64 residual and Newton update */

/* energy equation */
#define PSR_ADIABATIC 0     /* Eq. (3) with Q = 0, dP/dt = 0 */
#define PSR_FIXED_T 1       /* reactor temperature fixed at T0 (the paper's runs, Secs. 5-6) */

typedef struct psr_mech psr_mech; /* opaque; owns host and device copies of the tables */

typedef struct {
    int32_t K;              /* species */
    int32_t I;              /* reactions */
    int32_t n_elements;
    int32_t n_third_body;   /* reactions with a [M] factor */
    int32_t n_falloff;      /* Troe falloff reactions */
    int32_t has_soot;       /* the mechanism carries MOMIC soot constants */
} psr_mech_info;

/* Load a `.psrmech` text mechanism (format in the generator's documentation) from a
 * file, or from `nbytes` bytes of text in host memory. On success *out owns host and
 * device tables on the current CUDA device; free with psr_mech_free. Errors:
 * PSR_E_IO, PSR_E_FORMAT (message names the offending record), PSR_E_CUDA, PSR_E_OOM. */
int psr_mech_load(const char *path, psr_mech **out);
int psr_mech_load_mem(const char *text, size_t nbytes, psr_mech **out);
int psr_mech_info_get(const psr_mech *m, psr_mech_info *out);
/* Host copies: species molecular weights W [K] (g/mol) and element counts [K][n_elements]. */
int psr_mech_weights(const psr_mech *m, double *W_out);
void psr_mech_free(psr_mech *m); /* NULL-safe */

/* Solver controls. psr_options_default fills the defaults noted here. */
typedef struct {
    double ftol;            /* 1e-8: ||F||_inf target (F_k dimensionless, F_T = N/(c_p T)) */
    double step_rtol;       /* 1e-10: polish: |dx_j| <= step_rtol |x_j| + atol_j on the last step */
    double step_atol_y;     /* 1e-14 */
    double step_atol_t;     /* 1e-10 K */
    double ts_rtol;         /* 1e-4: a pseudo-time step is solved when |dx_j| <= ts_rtol |x_j| + ts_atol_j */
    double ts_atol_y;       /* 1e-10 (temperature uses ts_rtol) */
    double dt0_over_tau;    /* 1e-6: first pseudo-time step / tau */
    double dt_shrink;       /* 0.25: dt factor after a failed pseudo-time step */
    double y_floor;         /* 1e-10: iterates keep Y_k >= -y_floor */
    double t_min, t_max;    /* 200 K, 5000 K: temperature bounds of the iterates */
    int32_t max_newton;     /* 500: Newton iterations (steady and inside pseudo-time steps) */
    int32_t max_damp;       /* 8: halvings of the damping factor */
    int32_t max_ts_rounds;  /* 100: Newton attempts followed by time stepping */
    int32_t ts_steps;       /* 12: pseudo-time steps per round */
    int32_t ts_newton;      /* 8: Newton iterations per pseudo-time step */
    int32_t precision;      /* PSR_FP64 (default) or PSR_MIXED */
    int32_t energy;         /* PSR_ADIABATIC (default) or PSR_FIXED_T */
    int32_t warps_per_block;/* 0 = default (2); at most 4 */
    int32_t blocks_per_sm;  /* 0 = as many as fit */
    int32_t mixed_fallback; /* PSR_MIXED: what the FP32-Jacobian launch leaves unconverged is
                               solved again with the FP64 Jacobian: 2 (default) the reactors it
                               stopped at its iteration cap first continued from its final
                               iterate, then everything left restarted from the initial guess;
                               1 restart only; 0 none */
    int32_t jacobian;       /* PSR_JAC_ANALYTIC (default) or PSR_JAC_FD: central differences
                               as the paper builds it (Sec. 1), K + 1 <= 64 gas mechanisms */
    int32_t mixed_max_newton; /* -1 (default: 300 for gas mechanisms, 200 with soot moments):
                               Newton cap of the FP32-Jacobian launch when the FP64 re-solve
                               follows (0 = max_newton); reactors it leaves are re-solved in
                               FP64 with max_newton per pass */
    int32_t jac_age;        /* 1 (default): a fresh Jacobian and LU every Newton iteration;
                               A > 1: the factors serve up to A iterations while undamped steps
                               keep shrinking (any failure retries with fresh factors) */
    int32_t ts_linear;      /* 150: while a reactor has used fewer Newton iterations than this,
                               each pseudo-time step is one linearised Newton iteration
                               (pseudo-transient continuation; dt grown by 2 x the ||F|| ratio
                               clipped to [0.1, 8]); later steps, and all steps when 0, are
                               solved by damped Newton (<= ts_newton iterations, to ts_rtol) */
    int32_t path;           /* PSR_PATH_AUTO (default): one warp per reactor when K + 1 <= 64,
                               else one thread block (block_threads); PSR_PATH_WARP / PSR_PATH_BLOCK force
                               one (PSR_E_UNSUPPORTED where the mechanism does not fit it) */
    int32_t handoff;        /* -1 (default: 75 for PSR_FP64, 90 for PSR_MIXED) or 0..100. One warp
                               per reactor only: once this percentage of the launch's working
                               warps found its work queue empty, the reactors still running stop
                               at their next Newton iteration and a second launch continues them
                               from their iterates with one thread block each, in the same
                               precision (PSR_MIXED: then the FP64 re-solve takes what is left).
                               0 = off. Gas mechanisms, analytic Jacobian. Which reactors are
                               handed over depends on timing, so results are reproducible to the
                               solver's tolerance, not bit for bit; 0 gives bit-identical runs. */
    int32_t lu_tensor;      /* PSR_LU_CUDA_CORES (default), PSR_LU_TF32 or PSR_LU_3XTF32: with
                               PSR_MIXED on the block solver (K + 1 >= 96), the LU's trailing
                               update A22 -= L21 U12 runs on the fifth-generation tensor cores
                               (tcgen05, TF32 operands, FP32 accumulation in tensor memory);
                               3XTF32 splits each operand into two TF32 parts (three products)
                               for FP32-like accuracy. Other solves ignore it. */
    int32_t block_threads;  /* threads per reactor on the block solver: 512, or 256 for
                               mechanisms with K + 1 <= 256 (more resident blocks when the
                               Jacobian sits in global memory, cheaper barriers); 0 (default)
                               = 256 where K + 1 <= 256, else 512 */
    int32_t persistent;     /* psr_batch_solve_multi: 0 (default) = one launch sequence per
                               mechanism on library streams forked from the caller's; 1 = one
                               persistent launch over all mechanisms (256-thread blocks take
                               block-solver reactors, largest K first, then their warps take
                               warp-solver reactors; PSR_MIXED re-solves in FP64 in the same
                               launch) where the batch allows it: analytic Jacobian, CUDA-core
                               LU, K + 1 <= 256 for every mechanism on the block solver (and for
                               all with PSR_MIXED and mixed_fallback > 0), else the per-mechanism
                               layout. block_threads, warps_per_block, blocks_per_sm and handoff
                               do not apply to the persistent launch. */
    int32_t reserved0;      /* 0 */
    int64_t spin_limit;     /* 0 (default: 2^25) or > 0: polls (about 1 us apart) a block of the
                               persistent launch waits for first-pass reactors still running
                               before it gives up on the FP64 re-solve it claimed (that reactor
                               then keeps the FP32 pass's failure status) */
} psr_options;

/* LU trailing update (psr_options.lu_tensor) */
#define PSR_LU_CUDA_CORES 0
#define PSR_LU_TF32 1
#define PSR_LU_3XTF32 3

/* threads per reactor (psr_options.path) */
#define PSR_PATH_AUTO 0
#define PSR_PATH_WARP 1     /* one warp per reactor, K + 1 <= 64 (gas, or gas + soot with K + 7 <= 64) */
#define PSR_PATH_BLOCK 2    /* one thread block per reactor, gas mechanisms with K + 1 <= 512 */

void psr_options_default(psr_options *o);

/* Solve B independent steady PSRs (Sec. 2 Eqs. (1)-(3), Sec. 3 Eqs. (4)-(9); hybrid
 * Newton / pseudo-transient iteration of Sec. 3).
 *   Y_in [B][K], T_in [B], tau [B] (s, > 0), P [B] (dyn/cm^2, > 0): inlets.
 *   Y0 [B][K], T0 [B]: initial guesses (T0 is the fixed temperature in PSR_FIXED_T).
 *   rate_mult [I] or NULL: multiplier applied to every rate of progress q_i (all ones
 *     when NULL); the sensitivity parameter of the adjoint is ln(rate_mult_i).
 *   Y_out [B][K], T_out [B]: final iterates (the root for PSR_CONVERGED reactors).
 *   iters [B], ts_steps [B], status [B], fnorm [B] (||F||_inf at the output state),
 *   nfev [B] (residual evaluations, the reactor's share of the FP64 work): each may be NULL.
 * One persistent kernel launch; reactors are taken from a work queue by warps. With
 * PSR_MIXED and mixed_fallback = 1 or 2 further launches re-solve with the FP64 Jacobian
 * the reactors the first left unconverged (the lists are built on the device; no host
 * synchronisation): mixed_fallback = 2 continues them from the first launch's final
 * iterate, then restarts from Y0/T0 those the continuation leaves; 1 restarts them from
 * Y0/T0. Their counters add up and a success reports PSR_REFINE_FALLBACK. If Y0/T0 alias
 * Y_out/T_out, a restart starts from the first launch's final iterate.
 * Mechanisms with K + 1 <= 64 run one warp per reactor; larger ones (K + 1 <= 512) one
 * thread block per reactor with the same method.
 * Device memory: a few scratch integers (B + 4 for the fallback, B more when status is
 * NULL) are allocated and freed on the stream.
 * Errors: PSR_E_ARG (including B > 2^31 - 2^22, the work queue's limit, checked before
 * the mechanism), PSR_E_UNSUPPORTED (K + 1 > 512; the finite-difference Jacobian with
 * K + 1 > 64), PSR_E_CUDA, PSR_E_OOM. */
int psr_batch_solve(const psr_mech *m, int64_t B,
                    const double *Y_in, const double *T_in, const double *tau, const double *P,
                    const double *Y0, const double *T0, const double *rate_mult,
                    double *Y_out, double *T_out,
                    int32_t *iters, int32_t *ts_steps, int32_t *status, double *fnorm,
                    int32_t *nfev, const psr_options *opt, void *cuda_stream);

/* psr_batch_solve for callers that cannot allocate device memory, e.g. code running
 * where the allocator is frozen after start-up or only pre-registered buffers may be
 * used. (The paper has no counterpart: this is a service of the library.) The call
 * allocates nothing (no cudaMalloc, cudaMallocAsync or cudaFree): the solver's only
 * scratch, its work-queue counter, sits in a static 256-byte device array that every
 * GPU loading the library keeps until exit. Arguments, outputs and results are those
 * of psr_batch_solve, with three differences: only mechanisms with K + 1 <= 64 (the
 * warp-per-reactor solver; larger ones need allocated Jacobian slots) are accepted,
 * PSR_E_UNSUPPORTED otherwise; PSR_MIXED runs the single FP32-Jacobian launch (no FP64
 * re-solve of unconverged reactors, mixed_fallback is ignored); and B must not exceed
 * 2^31 - 2^22 (PSR_E_ARG otherwise). Both Jacobian options are honoured. The first
 * call on each device looks up the array's device address (cudaGetSymbolAddress), so
 * make that first call before any stream capture. All calls share the array: it is
 * zeroed on the stream before each launch, and calls that overlap on the GPU (other
 * streams, other host threads) race on it and must be serialised by the caller. */
int psr_batch_solve_noalloc(const psr_mech *m, int64_t B,
                            const double *Y_in, const double *T_in, const double *tau, const double *P,
                            const double *Y0, const double *T0, const double *rate_mult,
                            double *Y_out, double *T_out,
                            int32_t *iters, int32_t *ts_steps, int32_t *status, double *fnorm,
                            int32_t *nfev, const psr_options *opt, void *cuda_stream);

/* Gas + MOMIC soot PSR (mechanisms with a soot record): the K + 1 gas balances plus six
 * moment balances F_r = (M_r - M_r,in - tau (R_r + W_r + G_r)) / (M_r + s_r) of the soot
 * moments M_0..M_5 (nucleation, surface growth and free-molecular coagulation of the
 * method of moments with interpolative closure that the paper couples to its PSR,
 * Abstract, Secs. 1, 5 and 7), solved for (Y, T, ln(M / s)).
 *   M_in [B][6] inlet moments (particles/cm^3 x carbon atoms^r, > 0), M0 [B][6] initial
 *   moments or NULL (then the nucleation-only steady state at the initial gas state),
 *   M_out [B][6] output moments; other arguments as psr_batch_solve. K + 7 <= 64. */
int psr_batch_solve_soot(const psr_mech *m, int64_t B,
                         const double *Y_in, const double *T_in, const double *tau, const double *P,
                         const double *M_in, const double *Y0, const double *T0, const double *M0,
                         const double *rate_mult, double *Y_out, double *T_out, double *M_out,
                         int32_t *iters, int32_t *ts_steps, int32_t *status, double *fnorm,
                         int32_t *nfev, const psr_options *opt, void *cuda_stream);

/* Residual [B][K+7] (gas rows as psr_eval_residual, then the six moment rows) and its
 * Jacobian [B][K+7][K+7] at states (Y, T, moments M [B][6]) of a sooting mechanism. The
 * soot-source columns of the Jacobian are central differences of the source function. */
int psr_eval_residual_soot(const psr_mech *m, int64_t B,
                           const double *Y_in, const double *T_in, const double *tau, const double *P,
                           const double *M_in, const double *Y, const double *T, const double *M,
                           const double *rate_mult, double *F_out, int32_t energy, void *cuda_stream);
int psr_eval_jacobian_soot(const psr_mech *m, int64_t B,
                           const double *Y_in, const double *T_in, const double *tau, const double *P,
                           const double *M_in, const double *Y, const double *T, const double *M,
                           const double *rate_mult, double *J_out, int32_t energy, int32_t precision,
                           void *cuda_stream);

/* Uneven batch: B reactors of up to 8 gas mechanisms (different K) in one call, e.g. a
 * mix of small and large mechanisms as a reacting-flow code hands them over (the paper's
 * batch of independent PSRs, Sec. 6). mech_id [B] (device, int32) picks mechs[mech_id[r]];
 * row_off [B] (device, int64) is the offset of reactor r's row in the packed arrays
 * Y_in, Y0 and Y_out (row r holds K of its mechanism); T_in, tau, P, T0, T_out and the
 * per-reactor outputs are [B] as in psr_batch_solve. No rate multipliers. A device
 * kernel buckets the reactors by mechanism; each mechanism's persistent solver (warp per
 * reactor for K + 1 <= 64, block per reactor above) then runs on its own library-owned
 * stream forked from and joined back to cuda_stream, largest K first, so the launches
 * overlap. The call can be captured into a CUDA graph (all work joins back into
 * cuda_stream); concurrent callers on one device serialise on a mutex while enqueueing.
 * A reactor whose mech_id is out of range gets status PSR_BAD_INPUT (status scratch is
 * allocated when status is NULL) and is otherwise untouched.
 * Device memory: scratch lists, 4 (8 + (n_mech + 1) B) bytes, allocated on the stream.
 * Errors: PSR_E_ARG (n_mech outside 1..8, NULL, soot mechanism), PSR_E_UNSUPPORTED,
 * PSR_E_CUDA. */
int psr_batch_solve_multi(const psr_mech *const *mechs, int32_t n_mech, int64_t B,
                          const int32_t *mech_id, const int64_t *row_off,
                          const double *Y_in, const double *T_in, const double *tau, const double *P,
                          const double *Y0, const double *T0, double *Y_out, double *T_out,
                          int32_t *iters, int32_t *ts_steps, int32_t *status, double *fnorm,
                          int32_t *nfev, const psr_options *opt, void *cuda_stream);

/* Jacobian by central differences, the paper's construction (Sec. 1): column j from
 * residuals at x +- h_j e_j, h_j = 1e-6 max(|x_j|, s_j) with s = 0.1 for mass fractions and
 * 1000 K for T; the mass-fraction columns reuse the state's rate constants (they depend
 * on T only, Sec. 3). Arguments and layout as psr_eval_jacobian (FP64). Gas mechanisms
 * with K + 1 <= 64; PSR_E_UNSUPPORTED otherwise. */
int psr_eval_jacobian_fd(const psr_mech *m, int64_t B,
                         const double *Y_in, const double *T_in, const double *tau, const double *P,
                         const double *Y, const double *T, const double *rate_mult, double *J_out,
                         int32_t energy, void *cuda_stream);

/* Autotuner for the launch shape (the paper has no counterpart; a service of the
 * library): solves the caller's sample batch (device arrays as psr_batch_solve, B >= 1,
 * ideally a few thousand reactors like the production batches) once per candidate shape
 * and writes the one with the most converged solves per second into opt->path,
 * opt->warps_per_block, opt->blocks_per_sm and opt->block_threads; every other field of
 * *opt is used as given. Candidates: threads per reactor (one warp for K + 1 <= 64, or a
 * thread block of 512 or, for K + 1 <= 256, 256 threads for gas mechanisms); on the warp
 * path 1..4 warps per block and 2-warp blocks capped at 2..4 blocks per SM; on the block
 * path (larger mechanisms) 0 (as many as fit), 1 or 2 blocks per SM. Synchronises
 * cuda_stream; allocates and frees output scratch on it. The roots do not depend on the
 * shape: within a path the arithmetic is the same, and the paths reach the same roots
 * within the solver's tolerance (the block path's Jacobian sums its contributions in
 * another order).
 * Errors: PSR_E_ARG (NULL, soot mechanism, B outside 1..2^24), PSR_E_CUDA, PSR_E_OOM. */
int psr_autotune(const psr_mech *m, int64_t B,
                 const double *Y_in, const double *T_in, const double *tau, const double *P,
                 const double *Y0, const double *T0, psr_options *opt, void *cuda_stream);

/* Rates at given states, the unit the paper times on its GPU (Secs. 4 and 6: forward
 * rate constants, Eq. (6); equilibrium constants and reverse rates, Eqs. (7)-(9); rates of
 * progress, Eq. (5); net production, Eq. (4)). Y [B][K], T [B] (K), P [B] (dyn/cm^2):
 * device arrays; rate_mult [I] or NULL as in psr_batch_solve. Outputs (device, each may
 * be NULL): kf_out, kr_out, q_out [B][I] in the mechanism file's reaction order, wdot_out
 * [B][K] (mol/cm^3/s). kf is the effective forward coefficient (times the Troe factor
 * P_r/(1+P_r) F for falloff reactions; the third-body [M] multiplies q, not kf); kr =
 * kf / K_c; q includes [M] and rate_mult. Gas mechanisms only.
 * Errors: PSR_E_ARG, PSR_E_UNSUPPORTED, PSR_E_CUDA. */
int psr_eval_rates(const psr_mech *m, int64_t B, const double *Y, const double *T, const double *P,
                   const double *rate_mult, double *kf_out, double *kr_out, double *q_out,
                   double *wdot_out, void *cuda_stream);

/* Same as psr_batch_solve with every array in HOST memory: the call copies the inputs
 * to the device, solves, copies the outputs back and synchronises the stream before
 * returning. Device buffers are allocated and freed inside the call. */
int psr_batch_solve_host(const psr_mech *m, int64_t B,
                         const double *Y_in, const double *T_in, const double *tau, const double *P,
                         const double *Y0, const double *T0, const double *rate_mult,
                         double *Y_out, double *T_out,
                         int32_t *iters, int32_t *ts_steps, int32_t *status, double *fnorm,
                         int32_t *nfev, const psr_options *opt, void *cuda_stream);

/* Steady residual F(x) (Sec. 2 Eqs. (2)-(3) at d/dt = 0 with Eqs. (4)-(9)) at B states
 * x = (Y [B][K], T [B]) for the given inlets: F_out [B][K+1], row b = (F_1..F_K, F_T)
 * with F_k = Y_k - Y_k,in - tau wdot_k W_k / rho and
 * F_T = [sum_k Y_k,in (h_k(T) - h_k(T_in)) + (tau/rho) sum_k h_k W_k wdot_k] / (c_p T)
 * (adiabatic) or T - T0 (fixed T, T0 taken from T). Errors: PSR_E_ARG, PSR_E_CUDA. */
int psr_eval_residual(const psr_mech *m, int64_t B,
                      const double *Y_in, const double *T_in, const double *tau, const double *P,
                      const double *Y, const double *T, const double *rate_mult,
                      double *F_out, int32_t energy, void *cuda_stream);

/* Analytic Jacobian dF/dx of psr_eval_residual at the same states, row-major
 * J_out [B][K+1][K+1] in FP64 (precision PSR_FP64) or FP64-stored values of the FP32
 * assembly (PSR_MIXED), exactly as the solver's Newton iteration uses them. */
int psr_eval_jacobian(const psr_mech *m, int64_t B,
                      const double *Y_in, const double *T_in, const double *tau, const double *P,
                      const double *Y, const double *T, const double *rate_mult,
                      double *J_out, int32_t energy, int32_t precision, void *cuda_stream);

/* Adjoint sensitivities of the steady state to the rate multipliers: for a loss L with
 * g = dL/dx at converged states x = (Y [B][K], T [B]) of the problem in psr_eval_residual,
 * grad_out [B][I] (reaction order of the mechanism file) receives
 *   dL/d ln m_i = g^T dx/d ln m_i = -lambda^T dF/d ln m_i,  J^T lambda = g,
 * by the implicit function theorem at F(x) = 0 (the steady balances of Sec. 2 with the
 * rates of Sec. 3; m_i multiplies q_i). J is the FP64 analytic Jacobian factored by the
 * solver's LU; lambda_out [B][K+1] (nullable) receives lambda, ok_out [B] (nullable)
 * 1 when J factored (0: gradient set to 0). g [B][K+1] rows are (dL/dY_1..dL/dY_K, dL/dT).
 * Errors: PSR_E_ARG, PSR_E_UNSUPPORTED (K + 1 > 64), PSR_E_CUDA. */
int psr_batch_adjoint(const psr_mech *m, int64_t B,
                      const double *Y_in, const double *T_in, const double *tau, const double *P,
                      const double *Y, const double *T, const double *rate_mult, const double *g,
                      double *grad_out, double *lambda_out, int32_t *ok_out, int32_t energy,
                      void *cuda_stream);

/* Batched dense solve A_b x_b = r_b by the solver's LU with partial pivoting
 * (Sec. 1, Sec. 3): A [B][n][n] row-major, r [B][n], x_out [B][n], ok_out [B]
 * (1 = factored, 0 = zero or non-finite pivot), n <= 64. PSR_MIXED factors in FP32. */
int psr_batch_lu_solve(int64_t B, int32_t n, const double *A, const double *r,
                       double *x_out, int32_t *ok_out, int32_t precision, void *cuda_stream);

/* psr_batch_lu_solve in FP32 with the LU's trailing update on the tensor cores (the
 * Sec. 1 / Sec. 3 LU of the mixed form's large-mechanism path): lu_tensor is PSR_LU_TF32
 * or PSR_LU_3XTF32 (PSR_LU_CUDA_CORES gives the FP32 CUDA-core LU). Sizes with n < 96 have
 * no trailing matrix large enough and use CUDA cores throughout. Arguments, layout and
 * errors as psr_batch_lu_solve. */
int psr_batch_lu_solve_tc(int64_t B, int32_t n, const double *A, const double *r, double *x_out, int32_t *ok_out,
                          int32_t lu_tensor, void *cuda_stream);

const char *psr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PSR_H */
