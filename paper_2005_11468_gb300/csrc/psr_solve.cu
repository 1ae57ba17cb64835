// Batched steady PSR solve on sm_103a: host launchers, the C entry points and the
// service kernels (residual, Jacobian, rates, adjoint, LU) of the warp-per-reactor path.
// The solver itself (device stages and solve_kernel) is in psr_warp.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "psr_device.cuh"
#include "psr_internal.h"
#include "psr_warp.cuh"

namespace psr {
namespace {

// Work list for a later launch of a solve (among in_list when given, else among all B):
// mode 0: every reactor not converged by the first launch (the mixed form's FP64 re-solve);
// mode 1: those it handed over unfinished (a continuation in the same precision); mode 2:
// those neither launch converged (the restart after a continuation).
__global__ void collect_unconverged(int64_t B, const int32_t *in_list, const int32_t *in_len, const int32_t *status,
                                    int32_t *list, int32_t *len, int mode) {
    const int64_t n = in_list ? int64_t(*in_len) : B;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = in_list ? int64_t(in_list[p]) : p;
        const int32_t s = status[r];
        const bool take = mode == 1 ? s == kStatusHandoff
                          : mode == 3 ? s == PSR_MAX_ITER
                                    : (s != PSR_CONVERGED && (mode == 0 || s != PSR_REFINE_FALLBACK));
        if (take) list[atomicAdd(len, 1)] = int32_t(r);
    }
}

// residual / Jacobian at given states: one warp per state
template <class TJ, bool SOOT>
__global__ void eval_kernel(DevMech M, Batch bt, int energy, int want_J, double *out, RatesOut ro, size_t ws_per_warp) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = int64_t(blockIdx.x) * (blockDim.x >> 5) + warp;
    if (r >= bt.B) return;
    constexpr int ns = SOOT ? kNMom : 0;
    WS<TJ> w = carve<TJ>(smem + warp * ws_per_warp, M.K, M.I, M.K + 1 + ns, M.n_troe, ns);
    Ctx cx;
    cx.M = M;
    cx.mult = bt.rate_mult;
    cx.K = M.K;
    cx.n = M.K + 1 + ns;
    cx.o.energy = energy;
    const int K = M.K, n = cx.n;
    cx.r.Yin = bt.Y_in + r * K;
    cx.r.Min = SOOT ? bt.M_in + r * kNMom : nullptr;
    cx.r.tau = bt.tau[r];
    cx.r.P = bt.P[r];
    cx.r.Tspec = bt.T0[r];
    {
        const double Tin = bt.T_in[r], lnTin = log(Tin);
        double s = 0.0;
        for (int h = 0; h < 2; ++h) {
            int j = lane + 32 * h;
            if (j < K) {
                double cpR, hRT, sR, dcpR;
                nasa7(M.nasa, j, Tin, lnTin, 1.0 / Tin, cpR, hRT, sR, dcpR);
                s += cx.r.Yin[j] * hRT * __ldg(M.invW + j);
            }
        }
        cx.mx.h_in = wsum(s) * kRu * Tin;
    }
    V2 y;
    y.a = (lane < K) ? bt.Y0[r * K + lane] : (lane == K ? bt.T0[r] : 0.0);
    y.b = (lane + 32 < K) ? bt.Y0[r * K + lane + 32] : (lane + 32 == K ? bt.T0[r] : 0.0);
    if constexpr (SOOT) init_moments(cx, bt, r, y);       // bt.M0 holds the state's moments
    const V2 zero{0.0, 0.0};
    V2 F, R;
    residual_R<TJ, SOOT>(cx, w, y, zero, y, F, R);
    if (want_J == 2) {   // rates of the residual just evaluated: effective kf, kr, q_i, wdot_k
        const int I = M.I;
        for (int i = lane; i < I; i += 32) {
            const int64_t o = r * I + __ldg(M.orig + i);
            if (ro.kf) ro.kf[o] = w.kf[i];
            if (ro.kr) ro.kr[o] = w.kr[i];
            if (ro.q) ro.q[o] = w.q[i];
        }
        if (ro.wdot)
            for (int j = lane; j < K; j += 32) ro.wdot[r * K + j] = w.v[j];
        return;
    }
    if (want_J == 3) {   // finite-difference Jacobian (gas mechanisms)
        if constexpr (!SOOT) {
            eval_J_fd<TJ>(M, w, y, zero, cx.mx, cx.sl, cx.r.Yin, cx.r.tau, cx.r.P, cx.r.Tspec, energy, cx.mult);
            for (int idx = lane; idx < n * n; idx += 32)
                out[r * n * n + idx] = double(w.J[size_t(idx / n) * w.P + idx % n]);
        }
        return;
    }
    if (!want_J) {
        if (lane < n) out[r * n + lane] = F.a;
        if (lane + 32 < n) out[r * n + lane + 32] = F.b;
        return;
    }
    eval_J<TJ, SOOT>(M, w, y, zero, cx.mx, cx.sl, cx.r.Yin, cx.r.Min, cx.r.tau, energy, cx.mult);
    for (int idx = lane; idx < n * n; idx += 32)
        out[r * n * n + idx] = double(w.J[size_t(idx / n) * w.P + idx % n]);
}

// Rates at given states, one warp per state (any K): NASA-7 Gibbs terms and
// concentrations per species, then per reaction k_f (Eq. (6)), K_c (Eqs. (8)-(9)),
// k_r (Eq. (7)), the third-body and falloff forms and q (Eq. (5)), written in the
// mechanism file's order; wdot (Eq. (4)) gathered per species from q kept in shared
// memory. Per warp: C and S/R - H/RT [K+1], q [I] (doubles).
__global__ void rates_kernel(DevMech M, int64_t B, const double *Y, const double *Tv, const double *Pv,
                             const double *__restrict__ mult, RatesOut ro) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int K = M.K, I = M.I;
    double *C = reinterpret_cast<double *>(smem) + size_t(warp) * (2 * (K + 1) + I);
    double *gS = C + (K + 1), *q = gS + (K + 1);
    for (int64_t r = int64_t(blockIdx.x) * wpb + warp; r < B; r += int64_t(gridDim.x) * wpb) {
        const double T = Tv[r], P = Pv[r];
        const double lnT = log(T), invT = 1.0 / T;
        const double *Yr = Y + r * K;
        double sYW = 0.0;
        for (int k = lane; k < K; k += 32) sYW += Yr[k] * __ldg(M.invW + k);
        sYW = wsum(sYW);
        const double rho = P / (sYW * kRu * T), Ctot = P / (kRu * T), lnPRT = log(kPatm / (kRu * T));
        for (int k = lane; k < K; k += 32) {
            double cpR, hRT, sR, dcpR;
            nasa7(M.nasa, k, T, lnT, invT, cpR, hRT, sR, dcpR);
            C[k] = rho * Yr[k] * __ldg(M.invW + k);
            gS[k] = sR - hRT;
        }
        if (lane == 0) {
            C[K] = 1.0;
            gS[K] = 0.0;
        }
        __syncwarp();
        for (int i = lane; i < I; i += 32) {
            const int16_t *sl6 = M.slots + size_t(i) * 6;
            const int s0 = __ldg(sl6), s1 = __ldg(sl6 + 1), s2 = __ldg(sl6 + 2), s3 = __ldg(sl6 + 3),
                      s4 = __ldg(sl6 + 4), s5 = __ldg(sl6 + 5);
            const double a = __ldg(M.lnA + i) + __ldg(M.beta + i) * lnT - __ldg(M.theta + i) * invT;
            const double lnKc = (gS[s3] + gS[s4] + gS[s5]) - (gS[s0] + gS[s1] + gS[s2]) + __ldg(M.dnu_d + i) * lnPRT;
            double kf = exp(a), kr = exp(a - lnKc);
            const int typ = __ldg(M.type + i);
            double Mc = 1.0;
            if (typ != kElem) {
                Mc = Ctot;
                for (int e = __ldg(M.eff_ptr + i); e < __ldg(M.eff_ptr + i + 1); ++e)
                    Mc += __ldg(M.eff_val + e) * C[__ldg(M.eff_sp + e)];
                if (typ == kTroe) {
                    const Troe t = troe_eval(M.troe + size_t(__ldg(M.troe_row + i)) * 8, a, Mc, T, lnT, invT, false);
                    kf *= t.fac;
                    kr *= t.fac;
                }
            }
            double qi = kf * (C[s0] * C[s1] * C[s2]) - kr * (C[s3] * C[s4] * C[s5]);
            if (typ == kThirdBody) qi *= Mc;
            if (mult) qi *= __ldg(mult + __ldg(M.orig + i));
            q[i] = qi;
            const int64_t o = r * I + __ldg(M.orig + i);
            if (ro.kf) ro.kf[o] = kf;
            if (ro.kr) ro.kr[o] = kr;
            if (ro.q) ro.q[o] = qi;
        }
        __syncwarp();
        if (ro.wdot) {
            for (int k = lane; k < K; k += 32) {
                double wd = 0.0;
                for (int e = __ldg(M.sp_ptr + k); e < __ldg(M.sp_ptr + k + 1); ++e)
                    wd += __ldg(M.sp_nu_d + e) * q[__ldg(M.sp_rxn + e)];
                ro.wdot[r * K + k] = wd;
            }
        }
        __syncwarp();
    }
}

// Adjoint sensitivities at given (converged) states, one warp per reactor: FP64
// Jacobian, transposed LU solve J^T lam = g, then per reaction
// dL/d ln m_i = -lam . dF/d ln m_i = (tau q_i / rho) [sum_k lam_k W_k nu_ki - lam_T dH_i / (c_p T)].
__global__ void adjoint_kernel(DevMech M, Batch bt, int energy, const double *g, double *grad, double *lam_out,
                               int32_t *ok, size_t ws_per_warp) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = int64_t(blockIdx.x) * (blockDim.x >> 5) + warp;
    if (r >= bt.B) return;
    WS<double> w = carve<double>(smem + warp * ws_per_warp, M.K, M.I, M.K + 1, M.n_troe);
    Ctx cx;
    cx.M = M;
    cx.mult = bt.rate_mult;
    cx.K = M.K;
    cx.n = M.K + 1;
    cx.o.energy = energy;
    const int K = M.K, n = K + 1, I = M.I;
    cx.r.Yin = bt.Y_in + r * K;
    cx.r.tau = bt.tau[r];
    cx.r.P = bt.P[r];
    cx.r.Tspec = bt.T0[r];
    {
        const double Tin = bt.T_in[r], lnTin = log(Tin);
        double s = 0.0;
        for (int h = 0; h < 2; ++h) {
            int j = lane + 32 * h;
            if (j < K) {
                double cpR, hRT, sR, dcpR;
                nasa7(M.nasa, j, Tin, lnTin, 1.0 / Tin, cpR, hRT, sR, dcpR);
                s += cx.r.Yin[j] * hRT * __ldg(M.invW + j);
            }
        }
        cx.mx.h_in = wsum(s) * kRu * Tin;
    }
    V2 y;
    y.a = (lane < K) ? bt.Y0[r * K + lane] : (lane == K ? bt.T0[r] : 0.0);
    y.b = (lane + 32 < K) ? bt.Y0[r * K + lane + 32] : (lane + 32 == K ? bt.T0[r] : 0.0);
    const V2 zero{0.0, 0.0};
    V2 F, R;
    residual_R<double, false>(cx, w, y, zero, y, F, R);
    cx.r.Min = nullptr;
    eval_J<double, false>(M, w, y, zero, cx.mx, cx.sl, cx.r.Yin, nullptr, cx.r.tau, energy, cx.mult);
    const bool good = lu_factor(w, n);
    V2 gv, lam{0.0, 0.0};
    gv.a = (lane < n) ? g[r * n + lane] : 0.0;
    gv.b = (lane + 32 < n) ? g[r * n + lane + 32] : 0.0;
    if (good) lu_solve_T(w, n, gv, lam);
    // the Jacobian pass replaced q_i: evaluate the residual once more to restore it
    residual_R<double, false>(cx, w, y, zero, y, F, R);
    if (lam_out) {
        if (lane < n) lam_out[r * n + lane] = lam.a;
        if (lane + 32 < n) lam_out[r * n + lane + 32] = lam.b;
    }
    // stage lam_k W_k (species) in v[] and lam_T in registers
    const double lamT = comp_get(lam, K);
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        if (j < K) w.v[j] = (h ? lam.b : lam.a) * __ldg(M.W + j);
    }
    __syncwarp();
    const double tau_rho = cx.r.tau / cx.mx.rho;
    const double eT = (energy == PSR_FIXED_T) ? 0.0 : lamT * kRu * cx.mx.T / (cx.mx.cp * cx.mx.T);
    for (int i = lane; i < I; i += 32) {
        const int16_t *pp = M.part + size_t(i) * 6;
        const int8_t *pn = M.part_nu + size_t(i) * 6;
        double lw = 0.0, dH = 0.0;
        for (int t = 0; t < 6; ++t) {
            const int l = __ldg(pp + t);
            if (l >= K) continue;
            const double nu = double(__ldg(pn + t));
            lw += nu * w.v[l];
            dH += nu * w.hRT[l];
        }
        const double gi = good ? tau_rho * w.q[i] * (lw - eT * dH) : 0.0;
        grad[r * I + __ldg(M.orig + i)] = gi;
    }
    if (ok && lane == 0) ok[r] = good ? 1 : 0;
}

template <class TJ>
__global__ void lu_kernel(int64_t B, int n, const double *A, const double *rhs, double *x, int32_t *ok,
                          size_t ws_per_warp) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = int64_t(blockIdx.x) * (blockDim.x >> 5) + warp;
    if (b >= B) return;
    WS<TJ> w = carve<TJ>(smem + warp * ws_per_warp, 0, 0, n, 0);
    for (int idx = lane; idx < n * n; idx += 32) w.J[size_t(idx / n) * w.P + idx % n] = TJ(A[b * n * n + idx]);
    __syncwarp();
    V2 r;
    r.a = (lane < n) ? rhs[b * n + lane] : 0.0;
    r.b = (lane + 32 < n) ? rhs[b * n + lane + 32] : 0.0;
    bool good = lu_factor(w, n);
    V2 xs{0.0, 0.0};
    if (good) {
        V2 nr{-r.a, -r.b};
        lu_solve_neg(w, n, nr, xs);
    }
    if (lane < n) x[b * n + lane] = xs.a;
    if (lane + 32 < n) x[b * n + lane + 32] = xs.b;
    if (lane == 0) ok[b] = good ? 1 : 0;
}

// ---------------------------------------------------------------- host side
Opts to_opts(const psr_options *po) {
    psr_options d;
    psr_options_default(&d);
    const psr_options &s = po ? *po : d;
    Opts o;
    o.ftol = s.ftol;
    o.step_rtol = s.step_rtol;
    o.step_atol_y = s.step_atol_y;
    o.step_atol_t = s.step_atol_t;
    o.ts_rtol = s.ts_rtol;
    o.ts_atol_y = s.ts_atol_y;
    o.dt0_over_tau = s.dt0_over_tau;
    o.dt_shrink = s.dt_shrink;
    o.y_floor = s.y_floor;
    o.t_min = s.t_min;
    o.t_max = s.t_max;
    o.max_newton = s.max_newton;
    o.max_damp = s.max_damp;
    o.max_ts_rounds = s.max_ts_rounds;
    o.ts_steps = s.ts_steps;
    o.ts_newton = s.ts_newton;
    o.jac_fd = s.jacobian;
    o.mixed_max_newton = s.mixed_max_newton;
    o.jac_age = s.jac_age < 1 ? 1 : s.jac_age;
    o.ts_linear = s.ts_linear;
    o.energy = s.energy;
    // handoff thresholds measured at K = 53 with the 256-thread block solver continuing (it
    // finishes a straggler ~1.6x sooner than a warp with the FP64 LU, ~1.3x with FP32): the
    // FP64 form at 75 %, the mixed form only at the very end of the launch, 90 %
    o.handoff_pct = s.handoff >= 0 ? s.handoff : (s.precision == PSR_FP64 ? 75 : 90);
    o.lu_tc = s.lu_tensor;
    o.mixed_fb = s.mixed_fallback;
    o.block_threads = s.block_threads;
    return o;
}

int check_opts(const psr_options *po) {
    if (!po) return PSR_OK;
    const psr_options &s = *po;
    if (!(s.ftol > 0) || !(s.step_rtol >= 0) || !(s.step_atol_y >= 0) || !(s.step_atol_t >= 0) ||
        !(s.ts_rtol > 0) || !(s.ts_atol_y >= 0) || !(s.dt0_over_tau > 0) || !(s.dt_shrink > 0 && s.dt_shrink < 1) ||
        !(s.y_floor >= 0) || !(s.t_min > 0 && s.t_max > s.t_min) || s.max_newton < 1 || s.max_damp < 1 ||
        s.max_ts_rounds < 0 || s.ts_steps < 1 || s.ts_newton < 1 ||
        (s.precision != PSR_FP64 && s.precision != PSR_MIXED) ||
        (s.energy != PSR_ADIABATIC && s.energy != PSR_FIXED_T) || s.warps_per_block < 0 || s.warps_per_block > 32 ||
        s.blocks_per_sm < 0 || s.mixed_fallback < 0 || s.mixed_fallback > 2 ||
        (s.jacobian != PSR_JAC_ANALYTIC && s.jacobian != PSR_JAC_FD) || s.mixed_max_newton < -1 || s.jac_age < 0 ||
        s.jac_age > 64 || s.ts_linear < 0 || s.path < PSR_PATH_AUTO || s.path > PSR_PATH_BLOCK || s.handoff < -1 ||
        s.handoff > 100 || (s.lu_tensor != PSR_LU_CUDA_CORES && s.lu_tensor != PSR_LU_TF32 && s.lu_tensor != PSR_LU_3XTF32) ||
        (s.block_threads != 0 && s.block_threads != 256 && s.block_threads != 512) || s.persistent < 0 ||
        s.persistent > 1 || s.reserved0 != 0 || s.spin_limit < 0)
        return set_error(PSR_E_ARG, "psr_options: value out of range");
    return PSR_OK;
}

// solve_kernel<TJ, SOOT, FDJ> is compiled in its own translation unit (psr_solve_inst.cu);
// the launchers reach it through its host address.
template <class TJ, bool SOOT, bool FDJ>
cudaError_t launch_solve_kernel(unsigned grid, int threads, size_t smem, cudaStream_t st, DevMech M, Batch bt,
                                Opts o, int *queue, size_t wsb) {
    void *args[] = {&M, &bt, &o, &queue, &wsb};
    cudaError_t e = cudaLaunchKernel(solve_kernel_entry<TJ, SOOT, FDJ>(), dim3(grid), dim3(threads), args, smem, st);
    const cudaError_t last = cudaGetLastError();
    return e != cudaSuccess ? e : last;
}

template <class TJ, bool SOOT, bool FDJ = false>
int launch_solve_qs(const Mech &m, const Batch &bt, const Opts &o, int wpb_req, int bps_req, cudaStream_t st,
                    int *queue) {
    const size_t wsb = ws_bytes<TJ>(m.K, m.I, m.K + 1 + m.dev.nsoot, m.n_troe, m.dev.nsoot);
    int dev = 0;
    cudaGetDevice(&dev);
    int max_smem = 0, nsm = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int wpb = std::min(wpb_req > 0 ? wpb_req : kDefaultSolveWarps, kMaxSolveWarps);
    while (wpb > 1 && size_t(wpb) * wsb > size_t(max_smem)) --wpb;
    const size_t smem = size_t(wpb) * wsb;
    if (smem > size_t(max_smem))
        return set_error(PSR_E_UNSUPPORTED, "mechanism too large for one warp's shared memory");
    const void *kern = solve_kernel_entry<TJ, SOOT, FDJ>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return cuda_error("cudaFuncSetAttribute", e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
    if (e != cudaSuccess) return cuda_error("occupancy", e);
    if (per_sm < 1) return set_error(PSR_E_UNSUPPORTED, "solver kernel does not fit on an SM");
    if (bps_req > 0 && bps_req < per_sm) per_sm = bps_req;
    int64_t want = (bt.B + wpb - 1) / wpb;
    int64_t grid = std::min<int64_t>(int64_t(per_sm) * nsm, want);
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(queue, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return cuda_error("cudaMemsetAsync(work queue)", e);
    e = launch_solve_kernel<TJ, SOOT, FDJ>(unsigned(grid), wpb * 32, smem, st, m.dev, bt, o, queue, wsb);
    if (e != cudaSuccess) return cuda_error("solve_kernel launch", e);
    return PSR_OK;
}

// The gas-only and the gas + soot solver are separate instantiations (the soot code
// would otherwise cost the gas kernel registers).
template <class TJ>
int launch_solve_q(const Mech &m, const Batch &bt, const Opts &o, int wpb_req, int bps_req, cudaStream_t st,
                   int *queue) {
    if (m.dev.nsoot) return launch_solve_qs<TJ, true>(m, bt, o, wpb_req, bps_req, st, queue);
    if (o.jac_fd) return launch_solve_qs<TJ, false, true>(m, bt, o, wpb_req, bps_req, st, queue);
    return launch_solve_qs<TJ, false>(m, bt, o, wpb_req, bps_req, st, queue);
}

// Reactors the warp launch hands over unfinished can continue on the block solver: gas
// mechanisms that fit it, with the analytic Jacobian (the block solver has no other).
bool can_hand_over(const Mech &m, const Opts &o) {
    return o.handoff_pct > 0 && !m.dev.nsoot && !o.jac_fd && block_check(m) == PSR_OK;
}

// One warp per reactor in the Jacobian precision TJ. With handoff enabled, the reactors
// the warp launch hands over once its queue has drained and most warps are idle continue
// from their iterates on the block solver in the same precision (a device-side list, no
// host synchronisation): the stragglers get a thread block each instead of one warp.
template <class TJ>
int launch_solve(const Mech &m, const Batch &bt, const Opts &o, int wpb_req, int bps_req, cudaStream_t st) {
    if (!can_hand_over(m, o)) {
        int *queue = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&queue), 2 * sizeof(int), st);
        if (e != cudaSuccess) return set_error(PSR_E_OOM, "work-queue allocation failed");
        Opts o1 = o;
        o1.handoff_pct = 0;
        const int rc = launch_solve_q<TJ>(m, bt, o1, wpb_req, bps_req, st, queue);
        cudaFreeAsync(queue, st);
        return rc;
    }
    const size_t B = size_t(bt.B);
    int32_t *scr = nullptr;
    // queues, list length, the list, and status / iteration counts when the caller passed none
    // (the second launch reads both)
    const size_t n_ints = 8 + B + (bt.status ? 0 : B) + (bt.iters ? 0 : B);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scr), n_ints * sizeof(int32_t), st);
    if (e != cudaSuccess) return set_error(PSR_E_OOM, "scratch allocation failed");
    int32_t *q0 = scr, *q1 = scr + 2, *len = scr + 4, *list = scr + 8, *extra = scr + 8 + B;
    Batch b1 = bt;
    if (!bt.status) {
        b1.status = extra;
        extra += B;
    }
    if (!bt.iters) b1.iters = extra;
    int rc = launch_solve_q<TJ>(m, b1, o, wpb_req, bps_req, st, q0);
    if (rc == PSR_OK) {
        cudaMemsetAsync(len, 0, sizeof(int32_t), st);
        collect_unconverged<<<unsigned((B + 255) / 256), 256, 0, st>>>(bt.B, bt.list, bt.list_len, b1.status, list,
                                                                       len, 1);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_error("collect_unconverged launch", e);
    }
    if (rc == PSR_OK) {
        Batch b2 = b1;
        b2.list = list;
        b2.list_len = len;
        b2.fallback = 2;
        rc = block_resolve_list(m, b2, o, sizeof(TJ) == 8 ? PSR_FP64 : PSR_MIXED, st, q1);
    }
    cudaFreeAsync(scr, st);
    return rc;
}

// The FP32-Jacobian launch of the mixed form with fallback stops a reactor at the
// mixed_max_newton cap, so reactors it would not converge reach the FP64 re-solve sooner.
// The default (-1) is 300 for gas mechanisms and 200 with soot moments, where the FP32 LU
// of the coupled Jacobian stalls sooner (measured: K = 53 gas batch fastest at 300, the
// sooting batch at 200).
Opts mixed_first(const Opts &o, bool soot) {
    Opts f = o;
    const int cap = o.mixed_max_newton >= 0 ? o.mixed_max_newton : (soot ? 200 : 300);
    if (cap > 0 && cap < o.max_newton) f.max_newton = cap;
    return f;
}

// Mixed form with per-reactor FP64 fallback: the FP32-Jacobian launch, then the reactors
// it left unconverged (a device-side list, no host synchronisation) solved again from
// their initial guesses with the FP64 Jacobian; those that converge get
// PSR_REFINE_FALLBACK and their iteration counts add up. Reactors the first launch handed
// over unfinished (handoff) are in the same list and continue from their iterates.
int launch_mixed(const Mech &m, const Batch &bt, const Opts &o, int wpb_req, int bps_req, bool fallback,
                 cudaStream_t st) {
    if (!fallback) return launch_solve<float>(m, bt, o, wpb_req, bps_req, st);
    const size_t B = size_t(bt.B);
    int32_t *scr = nullptr;
    // queues, list length, the list, and status / iteration counts when the caller passed none
    // (the second launch reads both)
    const size_t n_ints = 8 + B + (bt.status ? 0 : B) + (bt.iters ? 0 : B);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scr), n_ints * sizeof(int32_t), st);
    if (e != cudaSuccess) return set_error(PSR_E_OOM, "scratch allocation failed");
    int32_t *q0 = scr, *q1 = scr + 2, *len = scr + 4, *list = scr + 8, *extra = scr + 8 + B;
    Batch b1 = bt;
    if (!bt.status) {
        b1.status = extra;
        extra += B;
    }
    if (!bt.iters) b1.iters = extra;
    Opts o1 = mixed_first(o, m.dev.nsoot != 0);
    // the re-solve of gas-phase reactors runs on the block solver, which can also continue
    // the reactors the warp launch hands over
    const bool block_fb = !m.dev.nsoot && block_check(m) == PSR_OK;
    const bool hand = block_fb && can_hand_over(m, o);
    if (!hand) o1.handoff_pct = 0;
    int rc = launch_solve_q<float>(m, b1, o1, wpb_req, bps_req, st, q0);
    if (rc == PSR_OK && hand) {
        // handed-over reactors continue with the FP32 Jacobian on the block solver (same
        // cap as the warp launch); whatever that leaves unconverged joins the FP64 list
        cudaMemsetAsync(len, 0, sizeof(int32_t), st);
        collect_unconverged<<<unsigned((B + 255) / 256), 256, 0, st>>>(bt.B, bt.list, bt.list_len, b1.status, list,
                                                                       len, 1);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_error("collect_unconverged launch", e);
        if (rc == PSR_OK) {
            Batch bc = b1;
            bc.list = list;
            bc.list_len = len;
            bc.fallback = 2;
            rc = block_resolve_list(m, bc, o1, PSR_MIXED, st, q1);
        }
    }
    // FP64 re-solve of what the FP32 launch left unconverged: with mixed_fallback = 2 the
    // reactors it stopped at its iteration cap are first continued from its final iterate
    // (most converge in a few dozen iterations), then whatever is left, including the ones
    // that ended in exhausted pseudo-time stepping (whose iterate an FP64 continuation almost
    // never finishes), is restarted from the initial guess; with 1, only the restart
    const int passes = o.mixed_fb == 2 ? 2 : 1;
    for (int pass = 0; pass < passes && rc == PSR_OK; ++pass) {
        const bool from_iterate = passes == 2 && pass == 0;
        cudaMemsetAsync(len, 0, sizeof(int32_t), st);
        collect_unconverged<<<unsigned((B + 255) / 256), 256, 0, st>>>(bt.B, bt.list, bt.list_len, b1.status, list,
                                                                       len, pass == 0 ? (passes == 2 ? 3 : 0) : 2);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_error("collect_unconverged launch", e);
            break;
        }
        Batch b2 = b1;
        b2.list = list;
        b2.list_len = len;
        b2.fallback = 1;
        if (from_iterate) {
            b2.Y0 = b1.Y_out;
            if (o.energy != PSR_FIXED_T) b2.T0 = b1.T_out;   // T0 is the specified temperature otherwise
            if (m.dev.nsoot) b2.M0 = b1.M_out;
        }
        // the list is short: gas-phase reactors go to the block solver, one CTA each
        if (block_fb)
            rc = block_resolve_list(m, b2, o, PSR_FP64, st, q1);
        else
            rc = launch_solve_q<double>(m, b2, o, wpb_req, bps_req, st, q1);
    }
    cudaFreeAsync(scr, st);
    return rc;
}

template <class TJ, bool SOOT>
int launch_eval_s(const Mech &m, const Batch &bt, int energy, int want_J, double *out, cudaStream_t st,
                  RatesOut ro) {
    const size_t wsb = ws_bytes<TJ>(m.K, m.I, m.K + 1 + m.dev.nsoot, m.n_troe, m.dev.nsoot);
    const int wpb = 2;
    const size_t smem = wpb * wsb;
    cudaError_t e =
        cudaFuncSetAttribute(eval_kernel<TJ, SOOT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return cuda_error("cudaFuncSetAttribute", e);
    const int64_t grid = (bt.B + wpb - 1) / wpb;
    eval_kernel<TJ, SOOT><<<unsigned(grid), wpb * 32, smem, st>>>(m.dev, bt, energy, want_J, out, ro, wsb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error("eval_kernel launch", e);
    return PSR_OK;
}

template <class TJ>
int launch_eval(const Mech &m, const Batch &bt, int energy, int want_J, double *out, cudaStream_t st,
                RatesOut ro = RatesOut{}) {
    if (m.dev.nsoot) return launch_eval_s<TJ, true>(m, bt, energy, want_J, out, st, ro);
    return launch_eval_s<TJ, false>(m, bt, energy, want_J, out, st, ro);
}

// ---------------------------------------------------------------- allocation-free variant
// Callers that may not allocate device memory (for example code running under an
// allocator that is frozen after start-up, or a host that hands the library only
// pre-registered buffers) use psr_batch_solve_noalloc. The only scratch the solver
// kernel needs, its work-queue counter, then lives in this file-scope array, which
// every GPU that loads the library keeps until the process exits. All calls share it:
// it is zeroed on the stream before each launch, and calls that overlap on the GPU
// race on it.
constexpr int kNoAllocScratchInts = 64;                 // 256 bytes
static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocScratchInts];

constexpr int kMaxDevices = 64;
std::atomic<int32_t *> g_noalloc_addr[kMaxDevices];

// Device address of the scratch array on the current device: looked up once per device
// (host code cannot take the address of a __device__ symbol directly).
int noalloc_scratch(int32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error("cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return set_error(PSR_E_UNSUPPORTED, "device index too large");
    int32_t *addr = g_noalloc_addr[dev].load();
    if (!addr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error("cudaGetSymbolAddress(g_noalloc_scratch)", e);
        addr = static_cast<int32_t *>(p);
        g_noalloc_addr[dev].store(addr);
    }
    *out = addr;
    return PSR_OK;
}

// The persistent solver with its work-queue counter in the static array (the launcher
// zeroes it on the stream before the launch).
template <class TJ>
int launch_solve_noalloc(const Mech &m, const Batch &bt, const Opts &o, int wpb_req, int bps_req, cudaStream_t st) {
    int32_t *queue = nullptr;
    const int rc = noalloc_scratch(&queue);
    if (rc != PSR_OK) return rc;
    Opts o1 = o;
    o1.handoff_pct = 0;   // a continuation launch would need an allocated work list
    return launch_solve_q<TJ>(m, bt, o1, wpb_req, bps_req, st, queue);
}

// Mechanisms with at most 64 unknowns run on the warp-per-reactor kernels, larger gas
// mechanisms on the block-per-reactor kernels (psr_block.cu).
bool warp_path(const psr_mech *m) { return m->m.K + 1 + m->m.dev.nsoot <= kMaxWarpN; }

int check_mech(const psr_mech *m) {
    if (!m) return set_error(PSR_E_ARG, "mechanism is NULL");
    if (!warp_path(m)) {
        const int rc = block_check(m->m);
        if (rc) return rc;
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != m->m.device) return set_error(PSR_E_ARG, "mechanism was loaded on another CUDA device");
    return PSR_OK;
}

// ---------------------------------------------------------------- several mechanisms in one call
constexpr int kMaxMechs = 8;

// Reactor r goes to the work list of its mechanism; an out-of-range id is reported.
__global__ void bucket_by_mechanism(int64_t B, const int32_t *mech_id, int n_mech, int32_t *counts, int32_t *lists,
                                    int32_t *status) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < B; r += int64_t(gridDim.x) * blockDim.x) {
        const int c = mech_id[r];
        if (c < 0 || c >= n_mech) {
            status[r] = PSR_BAD_INPUT;
            continue;
        }
        lists[int64_t(c) * B + atomicAdd(counts + c, 1)] = int32_t(r);
    }
}

// Per device: one stream per mechanism class and the fork/join events, created on first
// use and kept until exit. The mutex serialises the (short) enqueue of concurrent callers.
struct ClassStreams {
    bool ready = false;
    cudaStream_t s[kMaxMechs];
    cudaEvent_t fork, join[kMaxMechs];
};
ClassStreams g_class[kMaxDevices];
std::mutex g_class_mu;

int class_streams(int dev, ClassStreams **out) {
    if (dev < 0 || dev >= kMaxDevices) return set_error(PSR_E_UNSUPPORTED, "device index too large");
    ClassStreams &c = g_class[dev];
    if (!c.ready) {
        cudaError_t e = cudaEventCreateWithFlags(&c.fork, cudaEventDisableTiming);
        for (int i = 0; i < kMaxMechs && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&c.s[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.join[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_error("class streams", e);
        c.ready = true;
    }
    *out = &c;
    return PSR_OK;
}

}  // namespace
}  // namespace psr

using namespace psr;

extern "C" {

int psr_batch_solve(const psr_mech *m, int64_t B, const double *Y_in, const double *T_in, const double *tau,
                    const double *P, const double *Y0, const double *T0, const double *rate_mult, double *Y_out,
                    double *T_out, int32_t *iters, int32_t *ts_steps, int32_t *status, double *fnorm,
                    int32_t *nfev, const psr_options *opt, void *cuda_stream) {
    if (B < 0) return set_error(PSR_E_ARG, "B < 0");
    if (B > kMaxBatch) return set_error(PSR_E_ARG, "B exceeds the work-queue limit of " + std::to_string(kMaxBatch));
    int rc = check_mech(m);
    if (rc) return rc;
    if (m->m.has_soot)
        return set_error(PSR_E_ARG, "mechanism carries soot: use the _soot entry points");
    if (B == 0) return PSR_OK;
    if (!Y_in || !T_in || !tau || !P || !Y0 || !T0 || !Y_out || !T_out)
        return set_error(PSR_E_ARG, "psr_batch_solve: required pointer is NULL");
    if ((rc = check_opts(opt))) return rc;
    Batch bt{B, Y_in, T_in, tau, P, Y0, T0, rate_mult, Y_out, T_out, fnorm, iters, ts_steps, status, nfev};
    const Opts o = to_opts(opt);
    psr_options d;
    psr_options_default(&d);
    const psr_options &po = opt ? *opt : d;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const bool block = po.path == PSR_PATH_BLOCK || !warp_path(m);
    if (po.path == PSR_PATH_WARP && !warp_path(m))
        return set_error(PSR_E_UNSUPPORTED, "PSR_PATH_WARP: K + 1 <= 64 only");
    if (po.jacobian == PSR_JAC_FD && block)
        return set_error(PSR_E_UNSUPPORTED, "finite-difference Jacobian: the warp path (K + 1 <= 64) only");
    if (block) {
        if ((rc = block_check(m->m))) return rc;
        return block_solve(m->m, bt, o, po.precision, po.mixed_fallback != 0, po.blocks_per_sm, st);
    }
    if (po.precision == PSR_MIXED)
        return launch_mixed(m->m, bt, o, po.warps_per_block, po.blocks_per_sm, po.mixed_fallback != 0, st);
    return launch_solve<double>(m->m, bt, o, po.warps_per_block, po.blocks_per_sm, st);
}

int psr_batch_solve_noalloc(const psr_mech *m, int64_t B, const double *Y_in, const double *T_in, const double *tau,
                            const double *P, const double *Y0, const double *T0, const double *rate_mult,
                            double *Y_out, double *T_out, int32_t *iters, int32_t *ts_steps, int32_t *status,
                            double *fnorm, int32_t *nfev, const psr_options *opt, void *cuda_stream) {
    if (B < 0) return set_error(PSR_E_ARG, "B < 0");
    if (B > kMaxBatch)
        return set_error(PSR_E_ARG, "psr_batch_solve_noalloc: B exceeds the static work-queue limit of " +
                                        std::to_string(kMaxBatch) + " reactors");
    int rc = check_mech(m);
    if (rc) return rc;
    if (m->m.has_soot)
        return set_error(PSR_E_ARG, "mechanism carries soot: use the _soot entry points");
    if (!warp_path(m) || (opt && opt->path == PSR_PATH_BLOCK))
        return set_error(PSR_E_UNSUPPORTED, "psr_batch_solve_noalloc: the warp path (K + 1 <= 64) only");
    if (B == 0) return PSR_OK;
    if (!Y_in || !T_in || !tau || !P || !Y0 || !T0 || !Y_out || !T_out)
        return set_error(PSR_E_ARG, "psr_batch_solve_noalloc: required pointer is NULL");
    if ((rc = check_opts(opt))) return rc;
    Batch bt{B, Y_in, T_in, tau, P, Y0, T0, rate_mult, Y_out, T_out, fnorm, iters, ts_steps, status, nfev};
    const Opts o = to_opts(opt);
    psr_options d;
    psr_options_default(&d);
    const psr_options &po = opt ? *opt : d;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (po.precision == PSR_MIXED)
        return launch_solve_noalloc<float>(m->m, bt, o, po.warps_per_block, po.blocks_per_sm, st);
    return launch_solve_noalloc<double>(m->m, bt, o, po.warps_per_block, po.blocks_per_sm, st);
}

int psr_batch_solve_soot(const psr_mech *m, int64_t B, const double *Y_in, const double *T_in, const double *tau,
                         const double *P, const double *M_in, const double *Y0, const double *T0, const double *M0,
                         const double *rate_mult, double *Y_out, double *T_out, double *M_out, int32_t *iters,
                         int32_t *ts_steps, int32_t *status, double *fnorm, int32_t *nfev, const psr_options *opt,
                         void *cuda_stream) {
    if (B < 0) return set_error(PSR_E_ARG, "B < 0");
    if (B > kMaxBatch) return set_error(PSR_E_ARG, "B exceeds the work-queue limit of " + std::to_string(kMaxBatch));
    int rc = check_mech(m);
    if (rc) return rc;
    if (!m->m.has_soot) return set_error(PSR_E_ARG, "mechanism has no soot record: use psr_batch_solve");
    if (opt && opt->path == PSR_PATH_BLOCK) return set_error(PSR_E_UNSUPPORTED, "soot: the warp path only");
    if (B == 0) return PSR_OK;
    if (!Y_in || !T_in || !tau || !P || !M_in || !Y0 || !T0 || !Y_out || !T_out || !M_out)
        return set_error(PSR_E_ARG, "psr_batch_solve_soot: required pointer is NULL");
    if ((rc = check_opts(opt))) return rc;
    Batch bt{B, Y_in, T_in, tau, P, Y0, T0, rate_mult, Y_out, T_out, fnorm, iters, ts_steps, status, nfev,
             M_in, M0, M_out};
    const Opts o = to_opts(opt);
    psr_options d;
    psr_options_default(&d);
    const psr_options &po = opt ? *opt : d;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (po.precision == PSR_MIXED)
        return launch_mixed(m->m, bt, o, po.warps_per_block, po.blocks_per_sm, po.mixed_fallback != 0, st);
    return launch_solve<double>(m->m, bt, o, po.warps_per_block, po.blocks_per_sm, st);
}

int psr_eval_residual_soot(const psr_mech *m, int64_t B, const double *Y_in, const double *T_in, const double *tau,
                           const double *P, const double *M_in, const double *Y, const double *T, const double *Mom,
                           const double *rate_mult, double *F_out, int32_t energy, void *cuda_stream) {
    int rc = check_mech(m);
    if (rc) return rc;
    if (!m->m.has_soot) return set_error(PSR_E_ARG, "mechanism has no soot record");
    if (B < 0 || B > kMaxBatch || (energy != PSR_ADIABATIC && energy != PSR_FIXED_T)) return set_error(PSR_E_ARG, "bad B or energy");
    if (B == 0) return PSR_OK;
    if (!Y_in || !T_in || !tau || !P || !M_in || !Y || !T || !Mom || !F_out) return set_error(PSR_E_ARG, "NULL pointer");
    Batch bt{B, Y_in, T_in, tau, P, Y, T, rate_mult, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
             M_in, Mom, nullptr};
    return launch_eval<double>(m->m, bt, energy, 0, F_out, static_cast<cudaStream_t>(cuda_stream));
}

int psr_eval_jacobian_soot(const psr_mech *m, int64_t B, const double *Y_in, const double *T_in, const double *tau,
                           const double *P, const double *M_in, const double *Y, const double *T, const double *Mom,
                           const double *rate_mult, double *J_out, int32_t energy, int32_t precision,
                           void *cuda_stream) {
    int rc = check_mech(m);
    if (rc) return rc;
    if (!m->m.has_soot) return set_error(PSR_E_ARG, "mechanism has no soot record");
    if (B < 0 || B > kMaxBatch || (energy != PSR_ADIABATIC && energy != PSR_FIXED_T) ||
        (precision != PSR_FP64 && precision != PSR_MIXED))
        return set_error(PSR_E_ARG, "bad B, energy or precision");
    if (B == 0) return PSR_OK;
    if (!Y_in || !T_in || !tau || !P || !M_in || !Y || !T || !Mom || !J_out) return set_error(PSR_E_ARG, "NULL pointer");
    Batch bt{B, Y_in, T_in, tau, P, Y, T, rate_mult, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
             M_in, Mom, nullptr};
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == PSR_MIXED) return launch_eval<float>(m->m, bt, energy, 1, J_out, st);
    return launch_eval<double>(m->m, bt, energy, 1, J_out, st);
}

int psr_batch_solve_host(const psr_mech *m, int64_t B, const double *Y_in, const double *T_in, const double *tau,
                         const double *P, const double *Y0, const double *T0, const double *rate_mult,
                         double *Y_out, double *T_out, int32_t *iters, int32_t *ts_steps, int32_t *status,
                         double *fnorm, int32_t *nfev, const psr_options *opt, void *cuda_stream) {
    int rc = check_mech(m);
    if (rc) return rc;
    if (B < 0 || B > kMaxBatch) return set_error(PSR_E_ARG, "B out of range");
    if (B == 0) return PSR_OK;
    if (!Y_in || !T_in || !tau || !P || !Y0 || !T0 || !Y_out || !T_out)
        return set_error(PSR_E_ARG, "psr_batch_solve_host: required pointer is NULL");
    const int K = m->m.K, I = m->m.I;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t nb = size_t(B);
    // one device buffer: inputs, outputs
    const size_t doubles = nb * K * 3 + nb * 6 + (rate_mult ? I : 0);
    const size_t ints = nb * 4;
    char *buf = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&buf), doubles * 8 + ints * 4 + 64, st);
    if (e != cudaSuccess) return set_error(PSR_E_OOM, "device buffers for psr_batch_solve_host");
    double *d = reinterpret_cast<double *>(buf);
    double *dYin = d, *dY0 = d + nb * K, *dYout = d + 2 * nb * K;
    double *dTin = d + 3 * nb * K, *dtau = dTin + nb, *dP = dtau + nb, *dT0 = dP + nb, *dTout = dT0 + nb,
           *dfn = dTout + nb;
    double *dmult = rate_mult ? dfn + nb : nullptr;
    int32_t *ip = reinterpret_cast<int32_t *>(buf + doubles * 8);
    int32_t *dit = ip, *dts = ip + nb, *dst = ip + 2 * nb, *dnf = ip + 3 * nb;
    cudaMemcpyAsync(dYin, Y_in, nb * K * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dY0, Y0, nb * K * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dTin, T_in, nb * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dtau, tau, nb * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dP, P, nb * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dT0, T0, nb * 8, cudaMemcpyHostToDevice, st);
    if (rate_mult) cudaMemcpyAsync(dmult, rate_mult, size_t(I) * 8, cudaMemcpyHostToDevice, st);
    rc = psr_batch_solve(m, B, dYin, dTin, dtau, dP, dY0, dT0, dmult, dYout, dTout, dit, dts, dst, dfn, dnf, opt,
                         st);
    if (rc == PSR_OK) {
        cudaMemcpyAsync(Y_out, dYout, nb * K * 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(T_out, dTout, nb * 8, cudaMemcpyDeviceToHost, st);
        if (fnorm) cudaMemcpyAsync(fnorm, dfn, nb * 8, cudaMemcpyDeviceToHost, st);
        if (iters) cudaMemcpyAsync(iters, dit, nb * 4, cudaMemcpyDeviceToHost, st);
        if (ts_steps) cudaMemcpyAsync(ts_steps, dts, nb * 4, cudaMemcpyDeviceToHost, st);
        if (status) cudaMemcpyAsync(status, dst, nb * 4, cudaMemcpyDeviceToHost, st);
        if (nfev) cudaMemcpyAsync(nfev, dnf, nb * 4, cudaMemcpyDeviceToHost, st);
    }
    cudaFreeAsync(buf, st);
    e = cudaStreamSynchronize(st);
    if (rc == PSR_OK && e != cudaSuccess) return cuda_error("psr_batch_solve_host", e);
    return rc;
}

int psr_eval_residual(const psr_mech *m, int64_t B, const double *Y_in, const double *T_in, const double *tau,
                      const double *P, const double *Y, const double *T, const double *rate_mult, double *F_out,
                      int32_t energy, void *cuda_stream) {
    int rc = check_mech(m);
    if (rc) return rc;
    if (m->m.has_soot)
        return set_error(PSR_E_ARG, "mechanism carries soot: use the _soot entry points");
    if (B < 0 || B > kMaxBatch || (energy != PSR_ADIABATIC && energy != PSR_FIXED_T)) return set_error(PSR_E_ARG, "bad B or energy");
    if (B == 0) return PSR_OK;
    if (!Y_in || !T_in || !tau || !P || !Y || !T || !F_out) return set_error(PSR_E_ARG, "NULL pointer");
    Batch bt{B, Y_in, T_in, tau, P, Y, T, rate_mult, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (!warp_path(m)) return block_eval(m->m, bt, energy, 0, PSR_FP64, F_out, static_cast<cudaStream_t>(cuda_stream));
    return launch_eval<double>(m->m, bt, energy, 0, F_out, static_cast<cudaStream_t>(cuda_stream));
}

int psr_eval_jacobian(const psr_mech *m, int64_t B, const double *Y_in, const double *T_in, const double *tau,
                      const double *P, const double *Y, const double *T, const double *rate_mult, double *J_out,
                      int32_t energy, int32_t precision, void *cuda_stream) {
    int rc = check_mech(m);
    if (rc) return rc;
    if (m->m.has_soot)
        return set_error(PSR_E_ARG, "mechanism carries soot: use the _soot entry points");
    if (B < 0 || B > kMaxBatch || (energy != PSR_ADIABATIC && energy != PSR_FIXED_T) ||
        (precision != PSR_FP64 && precision != PSR_MIXED))
        return set_error(PSR_E_ARG, "bad B, energy or precision");
    if (B == 0) return PSR_OK;
    if (!Y_in || !T_in || !tau || !P || !Y || !T || !J_out) return set_error(PSR_E_ARG, "NULL pointer");
    Batch bt{B, Y_in, T_in, tau, P, Y, T, rate_mult, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (!warp_path(m)) return block_eval(m->m, bt, energy, 1, precision, J_out, st);
    if (precision == PSR_MIXED) return launch_eval<float>(m->m, bt, energy, 1, J_out, st);
    return launch_eval<double>(m->m, bt, energy, 1, J_out, st);
}

int psr_batch_adjoint(const psr_mech *m, int64_t B, const double *Y_in, const double *T_in, const double *tau,
                      const double *P, const double *Y, const double *T, const double *rate_mult, const double *g,
                      double *grad_out, double *lambda_out, int32_t *ok_out, int32_t energy, void *cuda_stream) {
    int rc = check_mech(m);
    if (rc) return rc;
    if (m->m.has_soot)
        return set_error(PSR_E_ARG, "mechanism carries soot: use the _soot entry points");
    if (B < 0 || B > kMaxBatch || (energy != PSR_ADIABATIC && energy != PSR_FIXED_T)) return set_error(PSR_E_ARG, "bad B or energy");
    if (B == 0) return PSR_OK;
    if (!Y_in || !T_in || !tau || !P || !Y || !T || !g || !grad_out)
        return set_error(PSR_E_ARG, "psr_batch_adjoint: required pointer is NULL");
    Batch bt{B, Y_in, T_in, tau, P, Y, T, rate_mult, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (!warp_path(m))
        return block_adjoint(m->m, bt, energy, g, grad_out, lambda_out, ok_out, static_cast<cudaStream_t>(cuda_stream));
    const Mech &mm = m->m;
    const size_t wsb = ws_bytes<double>(mm.K, mm.I, mm.K + 1, mm.n_troe);
    const int wpb = 2;
    const size_t smem = wpb * wsb;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return cuda_error("cudaFuncSetAttribute", e);
    const int64_t grid = (B + wpb - 1) / wpb;
    adjoint_kernel<<<unsigned(grid), wpb * 32, smem, st>>>(mm.dev, bt, energy, g, grad_out, lambda_out, ok_out, wsb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error("adjoint_kernel launch", e);
    return PSR_OK;
}

int psr_batch_lu_solve(int64_t B, int32_t n, const double *A, const double *r, double *x_out, int32_t *ok_out,
                       int32_t precision, void *cuda_stream) {
    if (B < 0 || B > kMaxBatch || n < 1 || n > 512 || (precision != PSR_FP64 && precision != PSR_MIXED))
        return set_error(PSR_E_ARG, "psr_batch_lu_solve: bad B, n or precision");
    if (B == 0) return PSR_OK;
    if (!A || !r || !x_out || !ok_out) return set_error(PSR_E_ARG, "psr_batch_lu_solve: NULL pointer");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (n > kMaxWarpN) return block_lu(B, n, A, r, x_out, ok_out, precision, st);
    const int wpb = 4;
    const int64_t grid = (B + wpb - 1) / wpb;
    cudaError_t e;
    if (precision == PSR_MIXED) {
        const size_t wsb = ws_bytes<float>(0, 0, n, 0);
        e = cudaFuncSetAttribute(lu_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(wpb * wsb));
        if (e != cudaSuccess) return cuda_error("cudaFuncSetAttribute", e);
        lu_kernel<float><<<unsigned(grid), wpb * 32, wpb * wsb, st>>>(B, n, A, r, x_out, ok_out, wsb);
    } else {
        const size_t wsb = ws_bytes<double>(0, 0, n, 0);
        e = cudaFuncSetAttribute(lu_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(wpb * wsb));
        if (e != cudaSuccess) return cuda_error("cudaFuncSetAttribute", e);
        lu_kernel<double><<<unsigned(grid), wpb * 32, wpb * wsb, st>>>(B, n, A, r, x_out, ok_out, wsb);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error("lu_kernel launch", e);
    return PSR_OK;
}

int psr_batch_lu_solve_tc(int64_t B, int32_t n, const double *A, const double *r, double *x_out, int32_t *ok_out,
                          int32_t lu_tensor, void *cuda_stream) {
    if (lu_tensor != PSR_LU_CUDA_CORES && lu_tensor != PSR_LU_TF32 && lu_tensor != PSR_LU_3XTF32)
        return set_error(PSR_E_ARG, "psr_batch_lu_solve_tc: lu_tensor must be PSR_LU_CUDA_CORES, _TF32 or _3XTF32");
    if (n <= kMaxWarpN || lu_tensor == PSR_LU_CUDA_CORES)
        return psr_batch_lu_solve(B, n, A, r, x_out, ok_out, PSR_MIXED, cuda_stream);
    if (B < 0 || B > kMaxBatch || n > 512) return set_error(PSR_E_ARG, "psr_batch_lu_solve_tc: bad B or n");
    if (B == 0) return PSR_OK;
    if (!A || !r || !x_out || !ok_out) return set_error(PSR_E_ARG, "psr_batch_lu_solve_tc: NULL pointer");
    return block_lu(B, n, A, r, x_out, ok_out, PSR_MIXED, static_cast<cudaStream_t>(cuda_stream), lu_tensor);
}

int psr_batch_solve_multi(const psr_mech *const *mechs, int32_t n_mech, int64_t B, const int32_t *mech_id,
                          const int64_t *row_off, const double *Y_in, const double *T_in, const double *tau,
                          const double *P, const double *Y0, const double *T0, double *Y_out, double *T_out,
                          int32_t *iters, int32_t *ts_steps, int32_t *status, double *fnorm, int32_t *nfev,
                          const psr_options *opt, void *cuda_stream) {
    if (!mechs || n_mech < 1 || n_mech > kMaxMechs) return set_error(PSR_E_ARG, "n_mech must be 1..8");
    if (B < 0) return set_error(PSR_E_ARG, "B < 0");
    if (B > kMaxBatch) return set_error(PSR_E_ARG, "B exceeds the work-queue limit of " + std::to_string(kMaxBatch));
    for (int c = 0; c < n_mech; ++c) {
        const int rc = check_mech(mechs[c]);
        if (rc) return rc;
        if (mechs[c]->m.has_soot) return set_error(PSR_E_ARG, "psr_batch_solve_multi: gas mechanisms only");
    }
    if (B == 0) return PSR_OK;
    if (!mech_id || !row_off || !Y_in || !T_in || !tau || !P || !Y0 || !T0 || !Y_out || !T_out)
        return set_error(PSR_E_ARG, "psr_batch_solve_multi: required pointer is NULL");
    int rc = check_opts(opt);
    if (rc) return rc;
    int dev = 0;
    cudaGetDevice(&dev);
    ClassStreams *cs = nullptr;
    if ((rc = class_streams(dev, &cs))) return rc;
    const Opts o = to_opts(opt);
    psr_options d;
    psr_options_default(&d);
    const psr_options &po = opt ? *opt : d;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // scratch: per-class counts and lists, and a status array when the caller passed none
    const size_t nb = size_t(B);
    int32_t *scr = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scr),
                                    sizeof(int32_t) * (kMaxMechs + size_t(n_mech) * nb + (status ? 0 : nb)), st);
    if (e != cudaSuccess) return set_error(PSR_E_OOM, "scratch allocation failed");
    int32_t *counts = scr, *lists = scr + kMaxMechs;
    int32_t *stat = status ? status : lists + size_t(n_mech) * nb;
    cudaMemsetAsync(counts, 0, sizeof(int32_t) * kMaxMechs, st);
    bucket_by_mechanism<<<unsigned(std::min<int64_t>((B + 255) / 256, 4096)), 256, 0, st>>>(B, mech_id, n_mech,
                                                                                           counts, lists, stat);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFreeAsync(scr, st);
        return cuda_error("bucket_by_mechanism launch", e);
    }
    if (po.persistent && !o.jac_fd && !o.lu_tc) {
        // one persistent launch: block-solver classes first, then warp-solver classes, each
        // group by decreasing K
        int order[kMaxMechs], n_block = 0;
        const Mech *ms[kMaxMechs];
        bool fits = true;
        for (int c = 0; c < n_mech; ++c) order[c] = c;
        auto on_block = [&](int c) { return po.path == PSR_PATH_BLOCK || !warp_path(mechs[c]); };
        std::sort(order, order + n_mech, [&](int a, int b) {
            if (on_block(a) != on_block(b)) return on_block(a);
            return mechs[a]->m.K > mechs[b]->m.K;
        });
        const bool fb = po.precision == PSR_MIXED && po.mixed_fallback != 0;
        for (int k = 0; k < n_mech; ++k) {
            const Mech &mm = mechs[order[k]]->m;
            ms[k] = &mm;
            if (on_block(order[k])) ++n_block;
            if ((on_block(order[k]) || fb) && mm.K + 1 > 256) fits = false;
        }
        if (po.path == PSR_PATH_WARP && n_block > 0) {
            cudaFreeAsync(scr, st);
            return set_error(PSR_E_UNSUPPORTED, "PSR_PATH_WARP: K + 1 <= 64 only");
        }
        if (fits) {
            Batch bt{B, Y_in, T_in, tau, P, Y0, T0, nullptr, Y_out, T_out, fnorm, iters, ts_steps, stat, nfev};
            bt.row_off = row_off;
            Opts o1 = o;
            if (po.precision == PSR_MIXED && fb) o1 = mixed_first(o, false);
            o1.handoff_pct = 0;
            const long long spin = po.spin_limit > 0 ? po.spin_limit : (1ll << 25);
            rc = multi_persistent(ms, order, n_mech, n_block, counts, lists, bt, o, o1, po.precision,
                                  fb ? (po.mixed_fallback == 2 ? 2 : 1) : 0, spin, st);
            cudaFreeAsync(scr, st);
            return rc;
        }
    }
    // classes in order of decreasing size of the system, each on its own stream
    int order[kMaxMechs];
    for (int c = 0; c < n_mech; ++c) order[c] = c;
    std::sort(order, order + n_mech, [&](int a, int b) { return mechs[a]->m.K > mechs[b]->m.K; });
    std::lock_guard<std::mutex> lock(g_class_mu);
    cudaEventRecord(cs->fork, st);
    rc = PSR_OK;
    for (int k = 0; k < n_mech && rc == PSR_OK; ++k) {
        const int c = order[k];
        cudaStream_t sc = cs->s[k];
        cudaStreamWaitEvent(sc, cs->fork, 0);
        Batch bt{B, Y_in, T_in, tau, P, Y0, T0, nullptr, Y_out, T_out, fnorm, iters, ts_steps, stat, nfev};
        bt.list = lists + size_t(c) * nb;
        bt.list_len = counts + c;
        bt.row_off = row_off;
        const Mech &mm = mechs[c]->m;
        if (po.path == PSR_PATH_WARP && !warp_path(mechs[c]))
            rc = set_error(PSR_E_UNSUPPORTED, "PSR_PATH_WARP: K + 1 <= 64 only");
        else if (po.path == PSR_PATH_BLOCK || !warp_path(mechs[c]))
            rc = block_solve(mm, bt, o, po.precision, po.mixed_fallback != 0, po.blocks_per_sm, sc);
        else if (po.precision == PSR_MIXED)
            rc = launch_mixed(mm, bt, o, po.warps_per_block, po.blocks_per_sm, po.mixed_fallback != 0, sc);
        else
            rc = launch_solve<double>(mm, bt, o, po.warps_per_block, po.blocks_per_sm, sc);
        cudaEventRecord(cs->join[k], sc);
        cudaStreamWaitEvent(st, cs->join[k], 0);
    }
    cudaFreeAsync(scr, st);
    return rc;
}

int psr_autotune(const psr_mech *m, int64_t B, const double *Y_in, const double *T_in, const double *tau,
                 const double *P, const double *Y0, const double *T0, psr_options *opt, void *cuda_stream) {
    int rc = check_mech(m);
    if (rc) return rc;
    if (!opt) return set_error(PSR_E_ARG, "psr_autotune: opt is NULL");
    if ((rc = check_opts(opt))) return rc;
    if (m->m.has_soot) return set_error(PSR_E_ARG, "psr_autotune: gas mechanisms only");
    if (B < 1 || B > (int64_t(1) << 24)) return set_error(PSR_E_ARG, "psr_autotune: sample size out of 1..2^24");
    if (!Y_in || !T_in || !tau || !P || !Y0 || !T0) return set_error(PSR_E_ARG, "psr_autotune: NULL pointer");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t nb = size_t(B), K = size_t(m->m.K);
    char *buf = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&buf), nb * (K + 2) * 8 + nb * 4 * 4, st);
    if (e != cudaSuccess) return set_error(PSR_E_OOM, "psr_autotune: output buffers");
    double *Yo = reinterpret_cast<double *>(buf), *To = Yo + nb * K, *fn = To + nb;
    int32_t *it = reinterpret_cast<int32_t *>(fn + nb), *ts = it + nb, *stt = ts + nb, *nf = stt + nb;
    // candidates: warps per block x block cap on the warp path; the block path has one shape
    // candidates: threads per reactor (a warp, or a thread block of 512 or, where the
    // K + 1 unknowns fit, 256 threads for gas mechanisms), on the warp path warps per block
    // x block cap, on the block path a cap of 1-2 blocks per SM
    struct Cand {
        int wpb, bps, path, bt;
    };
    std::vector<Cand> cands;
    const bool fits256 = m->m.K + 1 <= 256;
    if (warp_path(m)) {
        for (int w : {1, 2, 3, 4}) cands.push_back({w, 0, PSR_PATH_WARP, 0});
        for (int b : {2, 3, 4}) cands.push_back({2, b, PSR_PATH_WARP, 0});
        if (!m->m.has_soot) {
            cands.push_back({0, 0, PSR_PATH_BLOCK, 512});
            cands.push_back({0, 0, PSR_PATH_BLOCK, 256});
        }
    } else {
        for (int bt : {512, 256}) {
            if (bt == 256 && !fits256) continue;
            for (int b : {0, 1, 2}) cands.push_back({0, b, PSR_PATH_BLOCK, bt});
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<int32_t> hs(nb);
    double best_score = -1.0;
    Cand best = cands[0];
    psr_options trial = *opt;
    rc = psr_batch_solve(m, B, Y_in, T_in, tau, P, Y0, T0, nullptr, Yo, To, it, ts, stt, fn, nf, &trial, st);
    for (size_t c = 0; c < cands.size() && rc == PSR_OK; ++c) {
        trial.warps_per_block = cands[c].wpb;
        trial.blocks_per_sm = cands[c].bps;
        trial.path = cands[c].path;
        trial.block_threads = cands[c].bt;
        cudaEventRecord(e0, st);
        rc = psr_batch_solve(m, B, Y_in, T_in, tau, P, Y0, T0, nullptr, Yo, To, it, ts, stt, fn, nf, &trial, st);
        cudaEventRecord(e1, st);
        if (rc) break;
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_error("psr_autotune", e);
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        e = cudaMemcpy(hs.data(), stt, nb * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            rc = cuda_error("psr_autotune status copy", e);
            break;
        }
        int64_t conv = 0;
        for (int32_t v : hs) conv += (v == PSR_CONVERGED || v == PSR_REFINE_FALLBACK);
        const double score = ms > 0.f ? double(conv) / ms : 0.0;   // converged solves per ms
        if (score > best_score) {
            best_score = score;
            best = cands[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(buf, st);
    if (rc == PSR_OK) {
        opt->warps_per_block = best.wpb;
        opt->blocks_per_sm = best.bps;
        opt->path = best.path;
        opt->block_threads = best.bt;
    }
    return rc;
}

int psr_eval_rates(const psr_mech *m, int64_t B, const double *Y, const double *T, const double *P,
                   const double *rate_mult, double *kf_out, double *kr_out, double *q_out, double *wdot_out,
                   void *cuda_stream) {
    int rc = check_mech(m);
    if (rc) return rc;
    if (m->m.has_soot) return set_error(PSR_E_ARG, "psr_eval_rates: gas mechanisms only");
    if (B < 0 || B > kMaxBatch) return set_error(PSR_E_ARG, "B out of range");
    if (B == 0) return PSR_OK;
    if (!Y || !T || !P) return set_error(PSR_E_ARG, "psr_eval_rates: NULL state pointer");
    RatesOut ro{kf_out, kr_out, q_out, wdot_out};
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const Mech &mm = m->m;
    const size_t per_warp = sizeof(double) * (2 * size_t(mm.K + 1) + size_t(mm.I));
    int dev = 0, max_smem = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int wpb = 8;
    while (wpb > 1 && size_t(wpb) * per_warp > size_t(max_smem)) --wpb;
    const size_t smem = size_t(wpb) * per_warp;
    if (smem > size_t(max_smem)) return set_error(PSR_E_UNSUPPORTED, "psr_eval_rates: mechanism too large");
    cudaError_t e = cudaFuncSetAttribute(rates_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return cuda_error("cudaFuncSetAttribute", e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rates_kernel, wpb * 32, smem);
    if (e != cudaSuccess) return cuda_error("occupancy", e);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(int64_t(std::max(per_sm, 1)) * nsm, (B + wpb - 1) / wpb));
    rates_kernel<<<unsigned(grid), wpb * 32, smem, st>>>(mm.dev, B, Y, T, P, rate_mult, ro);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error("rates_kernel launch", e);
    return PSR_OK;
}

int psr_eval_jacobian_fd(const psr_mech *m, int64_t B, const double *Y_in, const double *T_in, const double *tau,
                         const double *P, const double *Y, const double *T, const double *rate_mult, double *J_out,
                         int32_t energy, void *cuda_stream) {
    int rc = check_mech(m);
    if (rc) return rc;
    if (m->m.has_soot || !warp_path(m))
        return set_error(PSR_E_UNSUPPORTED, "finite-difference Jacobian: gas mechanisms with K + 1 <= 64");
    if (B < 0 || B > kMaxBatch || (energy != PSR_ADIABATIC && energy != PSR_FIXED_T)) return set_error(PSR_E_ARG, "bad B or energy");
    if (B == 0) return PSR_OK;
    if (!Y_in || !T_in || !tau || !P || !Y || !T || !J_out) return set_error(PSR_E_ARG, "NULL pointer");
    Batch bt{B, Y_in, T_in, tau, P, Y, T, rate_mult, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    return launch_eval<double>(m->m, bt, energy, 3, J_out, static_cast<cudaStream_t>(cuda_stream));
}

}  // extern "C"
