// Device-side pieces shared by the warp-per-reactor and block-per-reactor solvers:
// per-call parameter blocks, warp reductions, NASA-7 thermo and the Troe falloff form.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "psr_internal.h"

namespace psr {

constexpr unsigned kFull = 0xffffffffu;


constexpr double kZetaStep = 3.0;   // largest change of a log moment in one Newton step
constexpr double kLn10 = 2.302585092994045684;

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ double wmin(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Pivot keys: the IEEE bits of |a| (sign cleared) order like |a| for every non-NaN value
// and put NaN above infinity, so the pivot search runs on the integer pipe (GB300's FP64
// pipe is the scarce one) and a NaN column is picked and then rejected.
__device__ __forceinline__ uint32_t abs_key(float v) { return __float_as_uint(v) & 0x7fffffffu; }
__device__ __forceinline__ unsigned long long abs_key(double v) {
    return static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ bool key_is_finite_nonzero(uint32_t k) { return k != 0u && k < 0x7f800000u; }

// Warp arg-max of pivot keys with the hardware integer reductions: the largest key, ties
// to the smallest row (rows of lanes without a candidate are >= any real row).
__device__ __forceinline__ int warp_argmax_row(uint32_t key, int row) {
    const uint32_t m = __reduce_max_sync(kFull, key);
    return int(__reduce_min_sync(kFull, key == m ? uint32_t(row) : 0xffffffffu));
}
__device__ __forceinline__ int warp_argmax_row(unsigned long long key, int row) {
    const uint32_t hi = uint32_t(key >> 32), lo = uint32_t(key);
    const uint32_t mh = __reduce_max_sync(kFull, hi);
    const uint32_t ml = __reduce_max_sync(kFull, hi == mh ? lo : 0u);
    return int(__reduce_min_sync(kFull, (hi == mh && lo == ml) ? uint32_t(row) : 0xffffffffu));
}
__device__ __forceinline__ bool key_is_finite_nonzero(unsigned long long k) {
    return k != 0ull && k < 0x7ff0000000000000ull;
}


// ---------------------------------------------------------------- per-call parameters
struct Batch {
    int64_t B;
    const double *Y_in, *T_in, *tau, *P, *Y0, *T0, *rate_mult;
    double *Y_out, *T_out, *fnorm;
    int32_t *iters, *ts_steps, *status, *nfev;
    const double *M_in, *M0;   // [B][6] soot moments (sooting mechanisms); M0 may be NULL
    double *M_out;
    const int32_t *list;       // optional work list of reactor indices (device), length *list_len
    const int32_t *list_len;
    int fallback;              // second launch over a list: 1 = FP64 re-solve after a mixed launch
                               // (converged reactors report PSR_REFINE_FALLBACK), 2 = continuation
                               // in the same precision; counters add up, and reactors the first
                               // launch handed over (kStatusHandoff) start from Y_out / T_out
    const int64_t *row_off;    // optional [B] start of reactor r's row in Y_in / Y0 / Y_out (else r K)
};

// Outputs of the rate evaluation (the paper's timed unit): [B][I] in mechanism-file order
// and wdot [B][K]; any may be NULL.
struct RatesOut {
    double *kf, *kr, *q, *wdot;
};

// Start of reactor r's mass-fraction row.
__device__ __forceinline__ int64_t row_of(const Batch &bt, int64_t r, int K) {
    return bt.row_off ? bt.row_off[r] : r * K;
}

struct Opts {
    double ftol, step_rtol, step_atol_y, step_atol_t, ts_rtol, ts_atol_y, dt0_over_tau, dt_shrink,
        y_floor, t_min, t_max;
    int max_newton, max_damp, max_ts_rounds, ts_steps, ts_newton, energy;
    int jac_fd;   // Jacobian by central differences (the paper's method) instead of analytic
    int mixed_max_newton;   // Newton cap of the FP32-Jacobian launch when the FP64 re-solve follows
    int jac_age;            // iterations one Jacobian factorisation may serve (1 = fresh each time)
    int ts_linear;          // linearised pseudo-time steps while the iteration count is below this
    int handoff_pct;        // warp launch: once this percentage of its working warps found the work
                            // queue empty, running reactors stop and go to the block solver (0 = never)
    int lu_tc;              // block solver, FP32 Jacobian: LU trailing update on the tensor cores
                            // (0 = CUDA cores, 1 = TF32, 3 = 3xTF32)
    int mixed_fb;           // mixed form's FP64 re-solve: 0 off, 1 restart, 2 continue then restart
    int block_threads;      // block solver threads per reactor: 0 (= 512), 256 or 512
};

// Scalars of the last residual evaluation that the Jacobian reuses.
struct Mix {
    double T, lnT, invT, rho, Wbar, Ctot, lnPRT;
    double N, cp, sum_yin_cp, sum_y_dcp;     // energy row pieces
    double h_in;                             // sum_k Y_k,in h_k(T_in), per reactor
};

// Per-species 1/W and per-entry efficiency - 1 in the Jacobian's precision (FP32 copies
// avoid FP64-to-FP32 conversions, which run on the FP64 pipe, in the FP32 Jacobian).
template <class TJ>
__device__ __forceinline__ TJ inv_w(const DevMech &M, int j);
template <>
__device__ __forceinline__ double inv_w<double>(const DevMech &M, int j) { return __ldg(M.invW + j); }
template <>
__device__ __forceinline__ float inv_w<float>(const DevMech &M, int j) { return __ldg(M.invW_f + j); }
template <class TJ>
__device__ __forceinline__ TJ eff_v(const DevMech &M, int e);
template <>
__device__ __forceinline__ double eff_v<double>(const DevMech &M, int e) { return __ldg(M.eff_val + e); }
template <>
__device__ __forceinline__ float eff_v<float>(const DevMech &M, int e) { return __ldg(M.eff_val_f + e); }

// d/d[X_l] of one side's slot product given the products of the other two slots
// (d0 = [X_s1][X_s2], ...): the sum over the slots that species l fills (mask bits 0..2).
// The first slot is picked with selects (integer pipe); a species filling two slots adds
// one term and only the three-slot case a second.
__device__ __forceinline__ double slot_deriv(int m, double d0, double d1, double d2) {
    const double first = (m & 1) ? d0 : ((m & 2) ? d1 : ((m & 4) ? d2 : 0.0));
    const int rest = m & (m - 1);
    double v = first + ((rest & 2) ? d1 : ((rest & 4) ? d2 : 0.0));
    if (m == 7) v += d2;
    return v;
}

__device__ __forceinline__ float slot_deriv_f(int m, float d0, float d1, float d2) {
    const float first = (m & 1) ? d0 : ((m & 2) ? d1 : ((m & 4) ? d2 : 0.0f));
    const int rest = m & (m - 1);
    float v = first + ((rest & 2) ? d1 : ((rest & 4) ? d2 : 0.0f));
    if (m == 7) v += d2;
    return v;
}

// ---------------------------------------------------------------- thermo (NASA-7)
__device__ __forceinline__ void nasa7(const double *__restrict__ nasa, int k, double T, double lnT, double invT,
                                      double &cpR, double &hRT, double &sR, double &dcpR) {
    const double *c = nasa + size_t(k) * 16;
    const double tmid = __ldg(c);
    const double *a = c + (T < tmid ? 1 : 8);
    const double a1 = __ldg(a), a2 = __ldg(a + 1), a3 = __ldg(a + 2), a4 = __ldg(a + 3), a5 = __ldg(a + 4),
                 a6 = __ldg(a + 5), a7 = __ldg(a + 6);
    constexpr double k3 = 1.0 / 3.0, k5 = 1.0 / 5.0;
    cpR = a1 + T * (a2 + T * (a3 + T * (a4 + T * a5)));
    hRT = a1 + T * (0.5 * a2 + T * (k3 * a3 + T * (0.25 * a4 + T * (k5 * a5)))) + a6 * invT;
    sR = a1 * lnT + T * (a2 + T * (0.5 * a3 + T * (k3 * a4 + T * (0.25 * a5)))) + a7;
    dcpR = a2 + T * (2 * a3 + T * (3 * a4 + T * 4 * a5));
}

// ---------------------------------------------------------------- Troe falloff pieces
struct Troe {
    double fac;       // P_r / (1 + P_r) F
    double D;         // d ln(fac) / d ln P_r
    double dlnF_dT;   // d ln F / dT at fixed P_r
    double dlk0;      // d ln k0 / dT
};

// The value is FP64; the derivatives (for the Jacobian only) are evaluated in TD, FP32 for
// the FP32 Jacobian (they only steer Newton, and FP64 divisions are long, slow chains).
template <class TD = double>
__device__ __forceinline__ Troe troe_eval(const double *__restrict__ tp, double a_inf, double M, double T,
                                          double lnT, double invT, bool want_deriv) {
    Troe t;
    const double lnA0 = __ldg(tp), b0 = __ldg(tp + 1), th0 = __ldg(tp + 2), al = __ldg(tp + 3),
                 T3 = __ldg(tp + 4), T1 = __ldg(tp + 5), T2 = __ldg(tp + 6);
    const double Pr = exp(lnA0 + b0 * lnT - th0 * invT - a_inf) * M;     // k0 [M] / k_inf
    const double e3 = exp(-T / T3), e1 = exp(-T / T1);
    const double e2 = (T2 != 0.0) ? exp(-T2 * invT) : 0.0;
    const double Fc = (1.0 - al) * e3 + al * e1 + e2;
    const double L = log10(Fc);
    const double cc = -0.4 - 0.67 * L, nn = 0.75 - 1.27 * L;
    const double u = log10(Pr) + cc;
    const double den = nn - 0.14 * u;
    const double f1 = u / den;
    const double s = 1.0 + f1 * f1;
    const double lgF = L / s;
    const double F = exp(kLn10 * lgF);
    t.fac = Pr / (1.0 + Pr) * F;
    if (want_deriv) {
        const TD Ld = TD(L), f1d = TD(f1), sd = TD(s), nnd = TD(nn), dend = TD(den), ud = TD(u), Prd = TD(Pr);
        const TD iTd = TD(invT), ald = TD(al), one = TD(1);
        const TD dlgF_du = -Ld * TD(2) * f1d / (sd * sd) * nnd / (dend * dend);
        t.D = double(one / (one + Prd) + dlgF_du);
        const TD dFc = -(one - ald) / TD(T3) * TD(e3) - ald / TD(T1) * TD(e1) +
                       ((T2 != 0.0) ? TD(T2) * iTd * iTd * TD(e2) : TD(0));
        const TD dL_dT = dFc / (TD(Fc) * TD(kLn10));
        const TD df1_dL = (TD(-0.67) * nnd + TD(1.27) * ud) / (dend * dend);
        const TD dlgF_dL = one / sd - Ld * TD(2) * f1d / (sd * sd) * df1_dL;
        t.dlnF_dT = double(TD(kLn10) * dlgF_dL * dL_dT);
        t.dlk0 = double(TD(b0) * iTd + TD(th0) * iTd * iTd);
    } else {
        t.D = t.dlnF_dT = t.dlk0 = 0.0;
    }
    return t;
}

// Host launchers of the block-per-reactor solver (psr_block.cu, built with 512 and with
// 256 threads per block), for mechanisms whose K + 1 unknowns exceed one warp's 64.
#define PSR_BLOCK_DECLS                                                                                           \
    int block_check(const Mech &m);                                                                               \
    int block_resolve_list(const Mech &m, const Batch &bt, const Opts &o, int precision, cudaStream_t st,         \
                           int *queue);                                                                           \
    int block_solve(const Mech &m, const Batch &bt, const Opts &o, int precision, bool fallback, int bps_req,     \
                    cudaStream_t st);                                                                             \
    int block_eval(const Mech &m, const Batch &bt, int energy, int want_J, int precision, double *out,            \
                   cudaStream_t st, RatesOut ro = RatesOut{});                                                    \
    int block_adjoint(const Mech &m, const Batch &bt, int energy, const double *g, double *grad, double *lam_out, \
                      int32_t *ok, cudaStream_t st);                                                              \
    int block_lu(int64_t B, int n, const double *A, const double *r, double *x, int32_t *ok, int precision,     \
                 cudaStream_t st, int lu_tc = 0);
namespace bt512 {
PSR_BLOCK_DECLS
}
namespace bt256 {
PSR_BLOCK_DECLS
}
#undef PSR_BLOCK_DECLS

// One persistent launch over the mechanism classes of psr_batch_solve_multi (psr_multi.cu):
// ms[k] is the class in queue order k (classes [0, n_block) on the block solver, the rest on
// the warp solver, each group by decreasing K), class_of[k] the index of its bucketed list
// (lists + class_of[k] B, counts[class_of[k]] reactors). o1 = the first pass's options (the
// FP32 pass's Newton cap for PSR_MIXED), o = the FP64 re-solve's. PSR_E_UNSUPPORTED
// (nothing launched) where the batch needs what the persistent kernel leaves out.
#define PSR_MULTI_DECL(name)                                                                                  \
    int name(const Mech *const *ms, const int32_t *class_of, int n_cls, int n_block, const int32_t *counts,       \
             const int32_t *lists, const Batch &bt, const Opts &o, const Opts &o1, int fb_passes,                \
             long long spin_limit, cudaStream_t st);
PSR_MULTI_DECL(multi_persistent_f32)
PSR_MULTI_DECL(multi_persistent_f64)
#undef PSR_MULTI_DECL
inline int multi_persistent(const Mech *const *ms, const int32_t *class_of, int n_cls, int n_block,
                            const int32_t *counts, const int32_t *lists, const Batch &bt, const Opts &o,
                            const Opts &o1, int precision, int fb_passes, long long spin_limit, cudaStream_t st) {
    return precision == PSR_MIXED
               ? multi_persistent_f32(ms, class_of, n_cls, n_block, counts, lists, bt, o, o1, fb_passes, spin_limit, st)
               : multi_persistent_f64(ms, class_of, n_cls, n_block, counts, lists, bt, o, o1, fb_passes, spin_limit, st);
}

// Threads per reactor of the block solver: o.block_threads, 256 only where the K + 1
// unknowns fit; 0 = 256 where they fit, else 512 (at K = 200 the 256-thread solver is 7 %
// faster with the FP32 Jacobian, one block per SM either way, and 23 % with the FP64
// Jacobian in global memory, where two of its blocks fit on an SM).
inline bool block256(const Mech &m, const Opts &o) {
    return (o.block_threads == 256 || o.block_threads == 0) && m.K + 1 <= 256;
}
inline int block_check(const Mech &m) { return bt512::block_check(m); }
inline int block_resolve_list(const Mech &m, const Batch &bt, const Opts &o, int precision, cudaStream_t st,
                              int *queue) {
    return block256(m, o) ? bt256::block_resolve_list(m, bt, o, precision, st, queue)
                          : bt512::block_resolve_list(m, bt, o, precision, st, queue);
}
inline int block_solve(const Mech &m, const Batch &bt, const Opts &o, int precision, bool fallback, int bps_req,
                       cudaStream_t st) {
    return block256(m, o) ? bt256::block_solve(m, bt, o, precision, fallback, bps_req, st)
                          : bt512::block_solve(m, bt, o, precision, fallback, bps_req, st);
}
inline int block_eval(const Mech &m, const Batch &bt, int energy, int want_J, int precision, double *out,
                      cudaStream_t st, RatesOut ro = RatesOut{}) {
    return bt512::block_eval(m, bt, energy, want_J, precision, out, st, ro);
}
inline int block_adjoint(const Mech &m, const Batch &bt, int energy, const double *g, double *grad, double *lam_out,
                         int32_t *ok, cudaStream_t st) {
    return bt512::block_adjoint(m, bt, energy, g, grad, lam_out, ok, st);
}
inline int block_lu(int64_t B, int n, const double *A, const double *r, double *x, int32_t *ok, int precision,
                    cudaStream_t st, int lu_tc = 0) {
    return bt512::block_lu(B, n, A, r, x, ok, precision, st, lu_tc);
}

}  // namespace psr
