// Device side of the warp-per-reactor PSR solver: the per-reactor stages (thermo, rates,
// residual, Jacobian, LU, damped Newton, pseudo-time steps) and the persistent solve_kernel.
//
// Per reactor the warp runs the hybrid scheme of Sec. 3: damped Newton on the steady
// residual of Eqs. (2)-(3) (with Eqs. (4)-(9) for the rates), and, when Newton fails,
// backward-Euler pseudo-time steps of the transient balances (each solved by damped
// Newton) before Newton is tried again. State vectors live in registers (lane j owns
// components j and j + 32), species-indexed tables and the Jacobian in shared memory.
// The residual is always FP64; the Jacobian and its LU are FP64 (PSR_FP64) or FP32
// (PSR_MIXED), in which case Newton on the FP64 residual refines the FP32 solves.
//
// Everything here has internal linkage. psr_solve.cu includes it for the service kernels
// (residual, Jacobian, adjoint, LU); each solve_kernel instantiation is compiled in its
// own translation unit (psr_solve_inst.cu) so that the build runs in parallel, and the
// host launches it through solve_kernel_entry.
#pragma once
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "psr_device.cuh"
#include "psr_internal.h"

namespace psr {
// Host address of solve_kernel<TJ, SOOT, FDJ> (for cudaLaunchKernel and the function
// attribute and occupancy queries); each is defined in its own build of psr_solve_inst.cu.
template <class TJ, bool SOOT, bool FDJ>
const void *solve_kernel_entry();
template <> const void *solve_kernel_entry<float, false, false>();
template <> const void *solve_kernel_entry<double, false, false>();
template <> const void *solve_kernel_entry<float, false, true>();
template <> const void *solve_kernel_entry<double, false, true>();
template <> const void *solve_kernel_entry<float, true, false>();
template <> const void *solve_kernel_entry<double, true, false>();
}  // namespace psr

namespace psr {
namespace {

// Stage inlining (measured on GB300): the residual and Jacobian stay inlined where that was
// faster; PSR_STAGE_* override each stage's choice.
#ifndef PSR_STAGE
#define PSR_STAGE
#endif
#ifndef PSR_STAGE_F
#define PSR_STAGE_F PSR_STAGE
#endif
#ifndef PSR_STAGE_J
#define PSR_STAGE_J PSR_STAGE
#endif
// The LU is out of line by default: one copy instead of one per call site (measured at
// K = 53: 11 % faster for the FP32-Jacobian solver, 19 % for the FP64 one).
#ifndef PSR_STAGE_LU
#define PSR_STAGE_LU __noinline__
#endif
#ifndef PSR_STAGE_SOLVE
#define PSR_STAGE_SOLVE PSR_STAGE
#endif
#ifndef PSR_STAGE_RES
#define PSR_STAGE_RES
#endif
#ifndef PSR_STAGE_NEWTON
#define PSR_STAGE_NEWTON
#endif
#ifndef PSR_OUTLINE_F32
#define PSR_OUTLINE_F32 1
#endif
// A length-n vector distributed over the warp: lane l holds components l and l + 32.
struct V2 {
    double a, b;
};
__device__ __forceinline__ double comp_get(const V2 &v, int j) {
    double x = __shfl_sync(kFull, j < 32 ? v.a : v.b, j & 31);
    return x;
}

// Per-warp shared-memory workspace.
template <class TJ>
struct WS {
    double *C, *hRT, *gS;    // [K+1]: concentrations (C[K] = 1), H/RT, S/R - H/RT (sentinels 0)
    double *kf, *kr, *q;     // [I]: effective rate constants of the last residual, q_i (or Euler sums)
    double *v;               // [K] dense third-body column part of the concentration Jacobian
    double *tD, *tX;         // [n_troe] falloff d ln(kf)/d ln Pr and the extra d ln(kf)/dT term
    double *sfd;             // soot: [17][7] perturbed source evaluations, [7][8] derivatives
    TJ *J;                   // [n][P]
    TJ *rhs;                 // [n]
    int16_t *perm;           // [n] row order after pivoting
    int P;                   // row pitch of J (elements)
    // FP32 Jacobian only: FP32 copies of C and H/RT [K+1] and the dense third-body part [K]
    float *Cf, *hf, *vf;
};

constexpr int kSootFD = 17 * 7 + 7 * 8;   // doubles of the soot finite-difference scratch

template <class TJ>
__host__ __device__ inline size_t ws_bytes(int K, int I, int n, int nt, int ns = 0) {
    int P = n + 1;
    size_t b = sizeof(double) * (3 * (K + 1) + 3 * I + K + 2 * nt + (ns ? kSootFD : 0));
    b = (b + 15) & ~size_t(15);
    b += sizeof(TJ) * (size_t(n) * P + n);
    b = (b + 15) & ~size_t(15);
    b += sizeof(int16_t) * n;
    b = (b + 15) & ~size_t(15);
    if (sizeof(TJ) == 4) b += sizeof(float) * (3 * K + 2);
    return (b + 15) & ~size_t(15);
}

template <class TJ>
__device__ WS<TJ> carve(char *base, int K, int I, int n, int nt, int ns = 0) {
    WS<TJ> w;
    double *d = reinterpret_cast<double *>(base);
    w.C = d;
    w.hRT = d + (K + 1);
    w.gS = d + 2 * (K + 1);
    w.kf = d + 3 * (K + 1);
    w.kr = w.kf + I;
    w.q = w.kr + I;
    w.v = w.q + I;
    w.tD = w.v + K;
    w.tX = w.tD + nt;
    w.sfd = w.tX + nt;
    size_t off = sizeof(double) * (3 * (K + 1) + 3 * I + K + 2 * nt + (ns ? kSootFD : 0));
    off = (off + 15) & ~size_t(15);
    w.P = n + 1;
    w.J = reinterpret_cast<TJ *>(base + off);
    w.rhs = w.J + size_t(n) * w.P;
    off += sizeof(TJ) * (size_t(n) * w.P + n);
    off = (off + 15) & ~size_t(15);
    w.perm = reinterpret_cast<int16_t *>(base + off);
    off += sizeof(int16_t) * n;
    off = (off + 15) & ~size_t(15);
    if (sizeof(TJ) == 4) {
        w.Cf = reinterpret_cast<float *>(base + off);
        w.hf = w.Cf + (K + 1);
        w.vf = w.hf + (K + 1);
    } else {
        w.Cf = w.hf = w.vf = nullptr;
    }
    return w;
}

// Lane-owned species data of the last residual evaluation.
struct SpecLane {
    double cpR[2], dcpR[2];
};

// ---------------------------------------------------------------- MOMIC soot sources
// Moment sources S_r = R_r + W_r + G_r (r = 0..5) and the precursor sink (mol/cm^3/s) at
// log moments z_r = ln(M_r / s_r), precursor concentration CP and temperature T:
// nucleation R_r = J C_min^r, J = A_n exp(-theta_n/T) CP N_A; growth
// W_r = k_g CP chi_alpha pi d_C^2 M_0 sum_{l<r} C(r,l) mu_{l+2/3} 2^(r-l); free-molecular
// coagulation G_0 = -K_f M_0^2 f_{0,0}/2, G_1 = 0, G_r = K_f M_0^2/2 sum_k C(r,k) f_{k,r-k}
// with f = f(1/2) interpolated in log over the grid functions f(l), l = 0..3; fractional
// moments mu_p = exp(sum_r w_r(p) ln mu_r) with the loader's Lagrange weights.
__device__ __forceinline__ void soot_eval(const double *__restrict__ st, const double *z, double CP, double T,
                                          double *S, double &sink) {
    constexpr double kNA = 6.02214076e23;
    const double lnT = log(T), invT = 1.0 / T;
    const double lnM0 = __ldg(st + kSootLnScale) + z[0];
    const double M0 = exp(lnM0);
    double lnmu[kNMom];
#pragma unroll
    for (int r = 0; r < kNMom; ++r) lnmu[r] = __ldg(st + kSootLnScale + r) + z[r] - lnM0;
    double mu[kSootNFrac];
#pragma unroll
    for (int i = 0; i < kSootNFrac; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int r = 1; r < kNMom; ++r) acc += __ldg(st + kSootW + i * kNMom + r) * lnmu[r];
        mu[i] = exp(acc);
    }
    const double cmin = __ldg(st + kSootCmin);
    const double J = exp(__ldg(st + kSootNucLnA) - __ldg(st + kSootNucTheta) * invT) * CP * kNA;
    const double kg = exp(__ldg(st + kSootGrowLnA) + __ldg(st + kSootGrowBeta) * lnT - __ldg(st + kSootGrowTheta) * invT);
    const double pref = kg * CP * __ldg(st + kSootGrowPref) * M0;
    // growth: W_r = pref sum_{l<r} C(r, l) mu_{l+2/3} 2^(r-l)
    const double g0 = mu[24], g1 = mu[25], g2 = mu[26], g3 = mu[27], g4 = mu[28];
    double W[kNMom];
    W[0] = 0.0;
    W[1] = pref * (2.0 * g0);
    W[2] = pref * (4.0 * g0 + 2.0 * 2.0 * g1);
    W[3] = pref * (8.0 * g0 + 3.0 * 4.0 * g1 + 3.0 * 2.0 * g2);
    W[4] = pref * (16.0 * g0 + 4.0 * 8.0 * g1 + 6.0 * 4.0 * g2 + 4.0 * 2.0 * g3);
    W[5] = pref * (32.0 * g0 + 5.0 * 16.0 * g1 + 10.0 * 8.0 * g2 + 10.0 * 4.0 * g3 + 5.0 * 2.0 * g4);
    // coagulation: f(1/2) for the pairs (0,0) (1,1) (1,2) (1,3) (2,2) (1,4) (2,3)
    const double beta = __ldg(st + kSootKf) * sqrt(T) * M0 * M0;
    const int px[7] = {0, 1, 1, 1, 2, 1, 2}, py[7] = {0, 1, 2, 3, 2, 4, 3};
    const double binom[4][4] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 1, 0}, {1, 3, 3, 1}};
    double fh[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const int x = px[q], y = py[q];
        double lf = 0.0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            double f = 0.0;
#pragma unroll
            for (int k = 0; k <= l; ++k) {
                const int a = k + x, b = l - k + y;
                f += binom[l][k] * (mu[3 * a] * mu[3 * b + 2] + 2.0 * mu[3 * a + 1] * mu[3 * b + 1] + mu[3 * a + 2] * mu[3 * b]);
            }
            lf += __ldg(st + kSootWHalf + l) * log(f);
        }
        fh[q] = exp(lf);
    }
    double G[kNMom];
    G[0] = -0.5 * beta * fh[0];
    G[1] = 0.0;
    G[2] = 0.5 * beta * (2.0 * fh[1]);
    G[3] = 0.5 * beta * (6.0 * fh[2]);
    G[4] = 0.5 * beta * (8.0 * fh[3] + 6.0 * fh[4]);
    G[5] = 0.5 * beta * (10.0 * fh[5] + 20.0 * fh[6]);
    double cr = 1.0;
#pragma unroll
    for (int r = 0; r < kNMom; ++r) {
        S[r] = J * cr + W[r] + G[r];
        cr *= cmin;
    }
    sink = (J * cmin + W[1]) / (2.0 * kNA);
}

// ---------------------------------------------------------------- residual, Eqs. (2)-(9)
// Evaluates F at state y; leaves C, hRT, gS, kf, kr (effective) of this state in shared
// memory and the scalars/lane data in mx/sl for the Jacobian.
// FRZ: a perturbation of the mass fractions at the temperature of the previous (full)
// evaluation: thermo, k_f and k_r of elementary and third-body reactions are reused from
// the caches (rate constants depend on T only); falloff rows are recomputed ([M] moves).
template <class TJ, bool SOOT, bool FRZ = false>
__device__ PSR_STAGE_F void eval_F(const DevMech &M, const WS<TJ> &w, const V2 &y, V2 &F, Mix &mx, SpecLane &sl,
                       const double *Yin_row, const double *Min, double tau, double P, double Tspec, int energy,
                       const double *__restrict__ mult) {
    const int lane = threadIdx.x & 31;
    const int K = M.K, I = M.I;
    const double T = comp_get(y, K);
    const double lnT = log(T), invT = 1.0 / T;
    mx.T = T;
    mx.lnT = lnT;
    mx.invT = invT;
    // mixture: W_bar = 1 / sum Y/W, rho = P W_bar / (R T), [X_k] = rho Y_k / W_k
    double sYW = 0.0;
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        if (j < K) sYW += (h ? y.b : y.a) * __ldg(M.invW + j);
    }
    sYW = wsum(sYW);
    const double Wbar = 1.0 / sYW;
    const double rho = P * Wbar / (kRu * T);
    mx.Wbar = Wbar;
    mx.rho = rho;
    mx.Ctot = P / (kRu * T);
    mx.lnPRT = log(kPatm / (kRu * T));
    double s_yin_h = 0.0, s_cp = 0.0, s_yin_cp = 0.0, s_y_dcp = 0.0;
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        if (j < K) {
            double Yj = h ? y.b : y.a;
            double cpR, hRT, sR, dcpR;
            const double invW = __ldg(M.invW + j);
            w.C[j] = rho * Yj * invW;
            if constexpr (FRZ) {
                hRT = w.hRT[j];
                cpR = sl.cpR[h];
                dcpR = sl.dcpR[h];
            } else {
                nasa7(M.nasa, j, T, lnT, invT, cpR, hRT, sR, dcpR);
                w.hRT[j] = hRT;
                w.gS[j] = sR - hRT;
                sl.cpR[h] = cpR;
                sl.dcpR[h] = dcpR;
            }
            const double yin = Yin_row[j];
            s_yin_h += yin * hRT * invW;
            s_cp += Yj * cpR * invW;
            s_yin_cp += yin * cpR * invW;
            s_y_dcp += Yj * dcpR * invW;
        }
    }
    if (lane == 0) {
        w.C[K] = 1.0;
        w.hRT[K] = 0.0;
        w.gS[K] = 0.0;
    }
    __syncwarp();
    // rates of progress, Eqs. (5)-(9): elementary reactions [0, tb_first), two per lane
    // per pass so that each lane carries two independent exp chains
    const int nE = M.tb_first;
    for (int i0 = lane; i0 < nE; i0 += 64) {
        const int i1 = (i0 + 32 < nE) ? i0 + 32 : i0;
        const int16_t *p0 = M.slots + size_t(i0) * 6, *p1 = M.slots + size_t(i1) * 6;
        int a[6], b[6];
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            a[t] = __ldg(p0 + t);
            b[t] = __ldg(p1 + t);
        }
        const double A0 = __ldg(M.lnA + i0) + __ldg(M.beta + i0) * lnT - __ldg(M.theta + i0) * invT;
        const double A1 = __ldg(M.lnA + i1) + __ldg(M.beta + i1) * lnT - __ldg(M.theta + i1) * invT;
        const double K0 = (w.gS[a[3]] + w.gS[a[4]] + w.gS[a[5]]) - (w.gS[a[0]] + w.gS[a[1]] + w.gS[a[2]]) +
                          __ldg(M.dnu_d + i0) * mx.lnPRT;
        const double K1 = (w.gS[b[3]] + w.gS[b[4]] + w.gS[b[5]]) - (w.gS[b[0]] + w.gS[b[1]] + w.gS[b[2]]) +
                          __ldg(M.dnu_d + i1) * mx.lnPRT;
        const double Pf0 = w.C[a[0]] * w.C[a[1]] * w.C[a[2]], Pr0 = w.C[a[3]] * w.C[a[4]] * w.C[a[5]];
        const double Pf1 = w.C[b[0]] * w.C[b[1]] * w.C[b[2]], Pr1 = w.C[b[3]] * w.C[b[4]] * w.C[b[5]];
        double kf0, kf1, kr0, kr1;
        if constexpr (FRZ) {
            kf0 = w.kf[i0];
            kf1 = w.kf[i1];
            kr0 = w.kr[i0];
            kr1 = w.kr[i1];
        } else {
            kf0 = exp(A0);
            kf1 = exp(A1);
            kr0 = exp(A0 - K0);
            kr1 = exp(A1 - K1);
        }
        double q0 = kf0 * Pf0 - kr0 * Pr0, q1 = kf1 * Pf1 - kr1 * Pr1;
        if (mult) {
            q0 *= __ldg(mult + __ldg(M.orig + i0));
            q1 *= __ldg(mult + __ldg(M.orig + i1));
        }
        if constexpr (!FRZ) {
            w.kf[i0] = kf0;
            w.kr[i0] = kr0;
        }
        w.q[i0] = q0;
        if (i1 != i0) {
            if constexpr (!FRZ) {
                w.kf[i1] = kf1;
                w.kr[i1] = kr1;
            }
            w.q[i1] = q1;
        }
    }
    // third-body and falloff reactions [tb_first, I)
    for (int i = nE + lane; i < I; i += 32) {
        const int16_t *sl6 = M.slots + size_t(i) * 6;
        const int s0 = __ldg(sl6), s1 = __ldg(sl6 + 1), s2 = __ldg(sl6 + 2), s3 = __ldg(sl6 + 3),
                  s4 = __ldg(sl6 + 4), s5 = __ldg(sl6 + 5);
        const double a = __ldg(M.lnA + i) + __ldg(M.beta + i) * lnT - __ldg(M.theta + i) * invT;
        const double lnKc = (w.gS[s3] + w.gS[s4] + w.gS[s5]) - (w.gS[s0] + w.gS[s1] + w.gS[s2]) +
                            __ldg(M.dnu_d + i) * mx.lnPRT;
        const int typ = __ldg(M.type + i);
        double kf, kr;
        if (FRZ && typ == kThirdBody) {
            kf = w.kf[i];
            kr = w.kr[i];
        } else {
            kf = exp(a);
            kr = exp(a - lnKc);
        }
        double Mc = mx.Ctot;
        for (int e = __ldg(M.eff_ptr + i); e < __ldg(M.eff_ptr + i + 1); ++e)
            Mc += __ldg(M.eff_val + e) * w.C[__ldg(M.eff_sp + e)];
        if (typ == kTroe) {
            const int tr = __ldg(M.troe_row + i);
            using TD = typename std::conditional<sizeof(TJ) == 4, float, double>::type;
            Troe t = troe_eval<TD>(M.troe + size_t(tr) * 8, a, Mc, T, lnT, invT, !FRZ);
            kf *= t.fac;
            kr *= t.fac;
            if constexpr (!FRZ) {
                const TD iT = TD(invT);
                const TD dlkf = TD(__ldg(M.beta + i)) * iT + TD(__ldg(M.theta + i)) * iT * iT;
                w.tD[tr] = t.D;
                w.tX[tr] = double(TD(t.D) * (TD(t.dlk0) - dlkf) + TD(t.dlnF_dT));
            }
        }
        if constexpr (!FRZ) {
            w.kf[i] = kf;
            w.kr[i] = kr;
        }
        double q = kf * (w.C[s0] * w.C[s1] * w.C[s2]) - kr * (w.C[s3] * w.C[s4] * w.C[s5]);
        if (typ == kThirdBody) q *= Mc;
        if (mult) q *= __ldg(mult + __ldg(M.orig + i));
        w.q[i] = q;
    }
    __syncwarp();
    // MOMIC sources (every lane evaluates them; the warp pays for one evaluation)
    double Ssoot[kNMom], sink = 0.0, zs[kNMom];
    if constexpr (SOOT) {
#pragma unroll
        for (int r = 0; r < kNMom; ++r) zs[r] = comp_get(y, K + 1 + r);
        soot_eval(M.soot, zs, w.C[M.soot_P], T, Ssoot, sink);
    }
    // Eq. (4) (plus the soot sink on precursor and H2) and the species residuals of
    // Eq. (2); wdot_k is left in v[] for the Jacobian
    double s_hw = 0.0;
    const double tau_rho = tau / rho;
    F.a = 0.0;
    F.b = 0.0;
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        if (j < K) {
            double w0 = 0.0, w1 = 0.0;
            int e = __ldg(M.sp_ptr + j);
            const int e_end = __ldg(M.sp_ptr + j + 1);
            for (; e + 1 < e_end; e += 2) {
                w0 += __ldg(M.sp_nu_d + e) * w.q[__ldg(M.sp_rxn + e)];
                w1 += __ldg(M.sp_nu_d + e + 1) * w.q[__ldg(M.sp_rxn + e + 1)];
            }
            if (e < e_end) w0 += __ldg(M.sp_nu_d + e) * w.q[__ldg(M.sp_rxn + e)];
            double wd = w0 + w1;
            if constexpr (SOOT) wd += (j == M.soot_H2 ? sink : 0.0) - (j == M.soot_P ? sink : 0.0);
            const double Yj = h ? y.b : y.a;
            const double f = Yj - Yin_row[j] - tau_rho * __ldg(M.W + j) * wd;
            s_hw += w.hRT[j] * wd;
            if (h) F.b = f;
            else F.a = f;
            w.v[j] = wd;
        }
    }
    s_yin_h = wsum(s_yin_h);
    s_cp = wsum(s_cp);
    s_yin_cp = wsum(s_yin_cp);
    s_y_dcp = wsum(s_y_dcp);
    s_hw = wsum(s_hw);
    const double RT = kRu * T;
    const double cp = s_cp * kRu;                                  // c_p,mix, erg/(g K)
    const double N = s_yin_h * RT - mx.h_in + tau_rho * RT * s_hw;   // energy balance, erg/g
    mx.N = N;
    mx.cp = cp;
    mx.sum_yin_cp = s_yin_cp * kRu;
    mx.sum_y_dcp = s_y_dcp * kRu;
    const double FT = (energy == PSR_FIXED_T) ? (T - Tspec) : N / (cp * T);
    if (lane == (K & 31)) {
        if (K < 32) F.a = FT;
        else F.b = FT;
    }
    // moment balances F_r = (M_r - M_r,in - tau S_r) / (M_r + s_r)
    if constexpr (SOOT) {
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            if (j > K && j <= K + kNMom) {
                const int r = j - K - 1;
                const double sr = __ldg(M.soot + kSootScale + r);
                const double Mr = sr * exp(h ? y.b : y.a);
                double Sr = 0.0;
#pragma unroll
                for (int q = 0; q < kNMom; ++q) Sr = (q == r) ? Ssoot[q] : Sr;
                const double f = (Mr - Min[r] - tau * Sr) / (Mr + sr);
                if (h) F.b = f;
                else F.a = f;
            }
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------- Jacobian
// Per-reaction pieces of the concentration Jacobian, lanes over reactions, in the
// arithmetic type TA (FP64, or FP32 for the FP32 Jacobian, where the pieces only steer
// Newton and FP64 instructions are the scarce resource): d q_i / d[X_l] for each distinct
// participant l scattered as nu_ki d q_i / d[X_l] into J (shared-memory atomics in TJ),
// the third-body part d q_i / d[M] into the dense per-row vector vd (every column) and
// the efficiency corrections; q_i and kf_i are replaced by the reaction's Euler sum
// g_i = sum_l [X_l] d q_i / d[X_l] and its T-derivative d q_i / dT.
template <class TA>
__device__ __forceinline__ TA slot_deriv_t(int m, TA d0, TA d1, TA d2) {
    const TA first = (m & 1) ? d0 : ((m & 2) ? d1 : ((m & 4) ? d2 : TA(0)));
    const int rest = m & (m - 1);
    TA v = first + ((rest & 2) ? d1 : ((rest & 4) ? d2 : TA(0)));
    if (m == 7) v += d2;
    return v;
}
template <class TA>
__device__ __forceinline__ TA beta_v(const DevMech &M, int i);
template <>
__device__ __forceinline__ double beta_v<double>(const DevMech &M, int i) { return __ldg(M.beta + i); }
template <>
__device__ __forceinline__ float beta_v<float>(const DevMech &M, int i) { return __ldg(M.beta_f + i); }
template <class TA>
__device__ __forceinline__ TA theta_v(const DevMech &M, int i);
template <>
__device__ __forceinline__ double theta_v<double>(const DevMech &M, int i) { return __ldg(M.theta + i); }
template <>
__device__ __forceinline__ float theta_v<float>(const DevMech &M, int i) { return __ldg(M.theta_f + i); }
template <class TA>
__device__ __forceinline__ TA dnu_v(const DevMech &M, int i) {
    if constexpr (sizeof(TA) == 8) return __ldg(M.dnu_d + i);
    else return TA(__ldg(M.dnu + i));
}

template <class TJ, class TA>
__device__ __forceinline__ void jac_reactions(const DevMech &M, const WS<TJ> &w, const Mix &mx,
                                              const double *__restrict__ mult, const TA *C, const TA *hRT,
                                              TA *vd) {
    const int lane = threadIdx.x & 31;
    const int K = M.K, I = M.I, P = w.P;
    const TA invT = TA(mx.invT), Ctot = TA(mx.Ctot);
    for (int i = lane; i < I; i += 32) {
        const int16_t *sl6 = M.slots + size_t(i) * 6;
        int s[6];
        TA cs[6];
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            s[t] = __ldg(sl6 + t);
            cs[t] = C[s[t]];
        }
        const TA Pf = cs[0] * cs[1] * cs[2], Pr_ = cs[3] * cs[4] * cs[5];
        const TA d0 = cs[1] * cs[2], d1 = cs[0] * cs[2], d2 = cs[0] * cs[1];
        const TA d3 = cs[4] * cs[5], d4 = cs[3] * cs[5], d5 = cs[3] * cs[4];
        const TA kf = TA(w.kf[i]), kr = TA(w.kr[i]);
        const TA m = mult ? TA(__ldg(mult + __ldg(M.orig + i))) : TA(1);
        const int typ = __ldg(M.type + i);
        TA Mc = TA(1);
        if (typ != kElem) {
            Mc = Ctot;
            for (int e = __ldg(M.eff_ptr + i); e < __ldg(M.eff_ptr + i + 1); ++e)
                Mc += eff_v<TA>(M, e) * C[__ldg(M.eff_sp + e)];
        }
        const TA sM = (typ == kThirdBody) ? Mc : TA(1);
        const TA dlkf = beta_v<TA>(M, i) * invT + theta_v<TA>(M, i) * invT * invT;
        const TA dlKc = ((hRT[s[3]] + hRT[s[4]] + hRT[s[5]]) - (hRT[s[0]] + hRT[s[1]] + hRT[s[2]]) - dnu_v<TA>(M, i)) *
                        invT;
        TA dlkfe = dlkf, dqdM = TA(0);
        if (typ == kThirdBody) {
            dqdM = m * (kf * Pf - kr * Pr_);
        } else if (typ == kTroe) {
            const int tr = __ldg(M.troe_row + i);
            dlkfe = dlkf + TA(w.tX[tr]);
            dqdM = m * (kf * Pf - kr * Pr_) * TA(w.tD[tr]) / Mc;
        }
        const TA dlkre = dlkfe - dlKc;
        const TA Af = m * sM * kf, Ar = m * sM * kr;
        const int nf = (s[0] < K) + (s[1] < K) + (s[2] < K), nr = (s[3] < K) + (s[4] < K) + (s[5] < K);
        TA g = Af * TA(nf) * Pf - Ar * TA(nr) * Pr_;
        if (typ != kElem) g += dqdM * Mc;
        const TA dqdT = Af * Pf * dlkfe - Ar * Pr_ * dlkre;
        // d q / d[X_l] for each distinct participant from its slot masks
        const int16_t *pp = M.part + size_t(i) * 6;
        const int8_t *pn = M.part_nu + size_t(i) * 6;
        const int8_t *pfm = M.part_fm + size_t(i) * 6;
        const int8_t *prm = M.part_rm + size_t(i) * 6;
        int pl[6];
        TJ pnu[6], val[6];
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            pl[t] = __ldg(pp + t);
            pnu[t] = TJ(__ldg(pn + t));
            const int fm = __ldg(pfm + t), rm = __ldg(prm + t);
            const TA dfl = slot_deriv_t<TA>(fm, d0, d1, d2);
            const TA drl = slot_deriv_t<TA>(rm, d3, d4, d5);
            val[t] = TJ(Af * dfl - Ar * drl);
        }
        const TJ dqdM_t = TJ(dqdM);
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            if (pl[r] >= K || pnu[r] == TJ(0)) continue;
            TJ *row = w.J + size_t(pl[r]) * P;
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                if (pl[t] >= K) continue;
                atomicAdd(row + pl[t], pnu[r] * val[t]);
            }
            if (typ != kElem) {
                atomicAdd(vd + pl[r], TA(pnu[r]) * dqdM);
                for (int e = __ldg(M.eff_ptr + i); e < __ldg(M.eff_ptr + i + 1); ++e)
                    atomicAdd(row + __ldg(M.eff_sp + e), pnu[r] * dqdM_t * eff_v<TJ>(M, e));
            }
        }
        // per-reaction Euler sum and T-derivative replace q and kf (read by this lane only)
        w.q[i] = double(g);
        w.kf[i] = double(dqdT);
    }
}

// ---------------------------------------------------------------- Jacobian
// Analytic dF/dx at the state of the last eval_F (whose C, hRT, kf, kr, troe cache,
// v = wdot and mx/sl it reuses), plus diag(c), written into w.J (rows/cols 0..n-1).
// Chain: concentration Jacobian Jc = d wdot / d[X] (per-reaction sparse blocks, a dense
// third-body part v_k for every column, sparse efficiency corrections), its Euler sums
// s_k = sum_l Jc_kl [X_l] and T-derivatives wT_k, then the transform to (Y, T) through
// rho(Y, T) and the energy row of Eq. (3). Entries are accumulated in TJ.
template <class TJ, bool SOOT>
__device__ PSR_STAGE_J void eval_J(const DevMech &M, const WS<TJ> &w, const V2 &y, const V2 &c, const Mix &mx,
                                 const SpecLane &sl, const double *Yin_row, const double *Min, double tau,
                                 int energy, const double *__restrict__ mult) {
    const int lane = threadIdx.x & 31;
    const int K = M.K, I = M.I, n = K + 1 + (SOOT ? kNMom : 0), P = w.P;
    // wdot (left in v[] by eval_F) moves to registers; v[] becomes the dense part
    double wd[2];
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        wd[h] = (j < K) ? w.v[j] : 0.0;
    }
    __syncwarp();
    for (int idx = lane; idx < n * P; idx += 32) w.J[idx] = TJ(0);
    const double T = mx.T, invT = mx.invT;
    if constexpr (sizeof(TJ) == 4) {
        // FP32 Jacobian: FP32 copies of C and H/RT, the dense part accumulated in FP32
        for (int j = lane; j <= K; j += 32) {
            w.Cf[j] = float(w.C[j]);
            w.hf[j] = float(w.hRT[j]);
            if (j < K) w.vf[j] = 0.0f;
        }
        __syncwarp();
        jac_reactions<TJ, float>(M, w, mx, mult, w.Cf, w.hf, w.vf);
    } else {
        for (int j = lane; j < K; j += 32) w.v[j] = 0.0;
        __syncwarp();
        jac_reactions<TJ, double>(M, w, mx, mult, w.C, w.hRT, w.v);
    }
    __syncwarp();
    // species sums s_k = sum_i nu_ki g_i, wT_k = sum_i nu_ki dq_i/dT
    double sk[2] = {0.0, 0.0}, wT[2] = {0.0, 0.0}, vk[2] = {0.0, 0.0};
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        if (j < K) {
            double a = 0.0, b = 0.0;
            for (int e = __ldg(M.sp_ptr + j); e < __ldg(M.sp_ptr + j + 1); ++e) {
                const double nu = __ldg(M.sp_nu_d + e);
                const int r = __ldg(M.sp_rxn + e);
                a += nu * w.q[r];
                b += nu * w.kf[r];
            }
            sk[h] = a;
            wT[h] = b;
            if constexpr (sizeof(TJ) == 4) vk[h] = double(w.vf[j]);
            else vk[h] = w.v[j];
        }
    }
    const double rho = mx.rho, Wbar = mx.Wbar, RT = kRu * T;
    // energy row, Eq. (3): computed from the concentration Jacobian before the transform
    double eJ[2] = {0.0, 0.0};
    if (energy != PSR_FIXED_T) {
        // Q = sum H_k wdot_k, Sh = sum H_k s_k, Hv = sum H_k v_k, dN/dT pieces; H/RT staged
        // in the Jacobian's precision for the column sums
        for (int k = lane; k < K; k += 32) w.rhs[k] = TJ(w.hRT[k]);
        __syncwarp();
        double Q = 0.0, Sh = 0.0, Hv = 0.0, cw = 0.0, hwT = 0.0;
        for (int h = 0; h < 2; ++h) {
            int j = lane + 32 * h;
            if (j < K) {
                const double H = w.hRT[j] * RT;
                Q += H * wd[h];
                Sh += H * sk[h];
                Hv += H * vk[h];
                cw += sl.cpR[h] * kRu * wd[h];
                hwT += H * (wT[h] - sk[h] * invT);
            }
        }
        Q = wsum(Q);
        Sh = wsum(Sh);
        Hv = wsum(Hv);
        cw = wsum(cw);
        hwT = wsum(hwT);
        const double N = mx.N, cp = mx.cp;
        const double inv_cpT = 1.0 / (cp * T);
        for (int h = 0; h < 2; ++h) {
            int j = lane + 32 * h;
            if (j < K) {
                TJ colsum = TJ(0);
                for (int k = 0; k < K; ++k) colsum += w.rhs[k] * w.J[size_t(k) * P + j];
                const double cs = double(colsum) * RT + Hv;
                const double invWj = __ldg(M.invW + j);
                const double dN = tau * invWj * (cs + Wbar * (Q - Sh) / rho);
                const double cpj = sl.cpR[h] * kRu * invWj;
                eJ[h] = dN * inv_cpT - N * cpj * inv_cpT / cp;
            } else if (j == K) {
                const double dNdT = mx.sum_yin_cp + tau / rho * (cw + hwT) + tau * Q / (rho * T);
                eJ[h] = dNdT * inv_cpT - N * mx.sum_y_dcp * inv_cpT / cp - N * inv_cpT * invT;
            }
        }
    }
    __syncwarp();
    // species rows: dF_k/dY_j = delta_kj - tau W_k (Jc_kj + v_k)/W_j + tau W_k Wbar (s_k - wdot_k)/(rho W_j)
    //               dF_k/dT  = -(tau W_k / rho) (wT_k + (wdot_k - s_k)/T)
    for (int h = 0; h < 2; ++h) {
        int k = lane + 32 * h;
        if (k < K) {
            const double Wk = __ldg(M.W + k);
            const TJ ak = TJ(tau * Wk), bk = TJ(tau * Wk * Wbar * (sk[h] - wd[h]) / rho), vkt = TJ(vk[h]);
            TJ *row = w.J + size_t(k) * P;
            for (int j = 0; j < K; ++j) {
                const TJ invWj = inv_w<TJ>(M, j);
                row[j] = (bk - ak * (row[j] + vkt)) * invWj + ((j == k) ? TJ(1) : TJ(0));
            }
            row[K] = TJ(-(tau * Wk / rho) * (wT[h] + (wd[h] - sk[h]) * invT));
        }
    }
    __syncwarp();
    // energy row
    {
        TJ *row = w.J + size_t(K) * P;
        for (int h = 0; h < 2; ++h) {
            int j = lane + 32 * h;
            if (j < n) {
                double v;
                if (energy == PSR_FIXED_T) v = (j == K) ? 1.0 : 0.0;
                else v = eJ[h];
                row[j] = TJ(v);
            }
        }
    }
    __syncwarp();
    if constexpr (SOOT) {
        // soot couplings: central differences of the source function in (zeta_0..5, CP, T),
        // lanes 0..16 each evaluating one perturbed input, chained through CP(Y, T)
        const int Psp = M.soot_P, Hsp = M.soot_H2;
        const double CP = w.C[Psp];
        double z[kNMom];
#pragma unroll
        for (int r = 0; r < kNMom; ++r) z[r] = comp_get(y, K + 1 + r);
        const double hz = 1e-5, hC = 1e-3 * CP + 1e-9 * mx.Ctot, hT = 1e-5 * T;
        {
            double zi[kNMom];
#pragma unroll
            for (int r = 0; r < kNMom; ++r) zi[r] = z[r];
            double CPi = CP, Ti = T;
            const int t = lane < 17 ? lane : 0;
            const int inp = (t >= 1 && t <= 8) ? t - 1 : ((t >= 9) ? t - 9 : -1);
            const double sg = (t >= 9) ? -1.0 : 1.0;
#pragma unroll
            for (int r = 0; r < kNMom; ++r) zi[r] += (inp == r) ? sg * hz : 0.0;
            if (inp == 6) CPi += sg * hC;
            if (inp == 7) Ti += sg * hT;
            double Sx[kNMom], sx;
            soot_eval(M.soot, zi, CPi, Ti, Sx, sx);
            if (lane < 17) {
#pragma unroll
                for (int r = 0; r < kNMom; ++r) w.sfd[lane * 7 + r] = Sx[r];
                w.sfd[lane * 7 + 6] = sx;
            }
        }
        __syncwarp();
        double *D = w.sfd + 17 * 7;          // D[o][i]: o = S_0..S_5, sink; i = zeta_0..5, CP, T
        for (int idx = lane; idx < 56; idx += 32) {
            const int o = idx / 8, i = idx % 8;
            const double h = (i < 6) ? hz : (i == 6 ? hC : hT);
            D[idx] = (w.sfd[(1 + i) * 7 + o] - w.sfd[(9 + i) * 7 + o]) / (2.0 * h);
        }
        __syncwarp();
        const double invWP = __ldg(M.invW + Psp);
        const double RT = kRu * T;
        const double eco = (energy == PSR_FIXED_T) ? 0.0
                               : (tau / mx.rho) * (w.hRT[Hsp] - w.hRT[Psp]) * RT / (mx.cp * T);
        // rows: 0 precursor, 1 H2, 2 energy, 3..8 moments
        for (int idx = lane; idx < 9 * n; idx += 32) {
            const int rk = idx / n, j = idx % n;
            // d(input)/dx_j for the source inputs
            auto dsrc = [&](int o) {
                const double dCP = (j < K) ? ((j == Psp ? mx.rho * invWP : 0.0) - CP * mx.Wbar * __ldg(M.invW + j))
                                           : (j == K ? -CP * invT : 0.0);
                double v = D[o * 8 + 6] * dCP;
                if (j == K) v += D[o * 8 + 7];
                if (j > K) v += D[o * 8 + (j - K - 1)];
                return v;
            };
            double val;
            int row;
            if (rk == 0) {
                row = Psp;
                val = tau * __ldg(M.W + Psp) / mx.rho * dsrc(6);
            } else if (rk == 1) {
                row = Hsp;
                val = -tau * __ldg(M.W + Hsp) / mx.rho * dsrc(6);
            } else if (rk == 2) {
                row = K;
                val = eco * dsrc(6);
            } else {
                const int r = rk - 3;
                row = K + 1 + r;
                const double sr = __ldg(M.soot + kSootScale + r);
                const double Mr = sr * exp(z[r]);
                const double den = Mr + sr;
                const double num = Mr - Min[r] - tau * w.sfd[r];
                val = -tau * dsrc(r) / den;
                if (j == K + 1 + r) val += Mr / den - num * Mr / (den * den);
            }
            TJ *e = w.J + size_t(row) * P + j;
            *e = TJ(double(*e) + val);
        }
        __syncwarp();
    }
    // + diag(c)
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        if (j < n) w.J[size_t(j) * P + j] = TJ(double(w.J[size_t(j) * P + j]) + (h ? c.b : c.a));
    }
    __syncwarp();
}

// ---------------------------------------------------------------- finite-difference Jacobian
// The paper's Jacobian (Sec. 1): central differences of the residual, column j with
// h_j = 1e-6 max(|x_j|, s_j), s = 0.1 for mass fractions and 1000 K for T. The mass-
// fraction columns use the frozen-rate residual (the rate constants depend on T only,
// Sec. 3), so only the temperature column re-evaluates the exponentials; it comes last,
// after the base state's caches have served every other column. Gas mechanisms only.
template <class TJ>
__device__ void eval_J_fd(const DevMech &M, const WS<TJ> &w, const V2 &y, const V2 &c, Mix &mx, SpecLane &sl,
                          const double *Yin_row, double tau, double P, double Tspec, int energy,
                          const double *__restrict__ mult) {
    const int lane = threadIdx.x & 31;
    const int K = M.K, n = K + 1, Pp = w.P;
    V2 F0, Fp, Fm;
    eval_F<TJ, false, false>(M, w, y, F0, mx, sl, Yin_row, nullptr, tau, P, Tspec, energy, mult);
    for (int j = 0; j < n; ++j) {
        const double xj = comp_get(y, j);
        const double h = 1e-6 * fmax(fabs(xj), j < K ? 0.1 : 1000.0);
        V2 yp = y, ym = y;
        if (lane == (j & 31)) {
            if (j < 32) {
                yp.a += h;
                ym.a -= h;
            } else {
                yp.b += h;
                ym.b -= h;
            }
        }
        if (j < K) {
            eval_F<TJ, false, true>(M, w, yp, Fp, mx, sl, Yin_row, nullptr, tau, P, Tspec, energy, mult);
            eval_F<TJ, false, true>(M, w, ym, Fm, mx, sl, Yin_row, nullptr, tau, P, Tspec, energy, mult);
        } else {
            eval_F<TJ, false, false>(M, w, yp, Fp, mx, sl, Yin_row, nullptr, tau, P, Tspec, energy, mult);
            eval_F<TJ, false, false>(M, w, ym, Fm, mx, sl, Yin_row, nullptr, tau, P, Tspec, energy, mult);
        }
        const double inv2h = 0.5 / h;
        if (lane < n) w.J[size_t(lane) * Pp + j] = TJ((Fp.a - Fm.a) * inv2h);
        if (lane + 32 < n) w.J[size_t(lane + 32) * Pp + j] = TJ((Fp.b - Fm.b) * inv2h);
    }
    __syncwarp();
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        if (j < n) w.J[size_t(j) * Pp + j] = TJ(double(w.J[size_t(j) * Pp + j]) + (h ? c.b : c.a));
    }
    __syncwarp();
}

// ---------------------------------------------------------------- LU (partial pivoting)
// In-place LU of w.J (n x n) with row interchanges; perm holds the final row order.
// Returns false on a zero or non-finite pivot.
template <class TJ>
__device__ PSR_STAGE_LU bool lu_factor(const WS<TJ> &w, int n) {
    const int lane = threadIdx.x & 31;
    const int P = w.P;
    for (int j = lane; j < n; j += 32) w.perm[j] = int16_t(j);
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        // pivot: first row of largest |a_ik|, i >= k (integer keys of |a|)
        decltype(abs_key(TJ(0))) best = 0;
        int bi = n;
        for (int i = k + lane; i < n; i += 32) {
            const auto a = abs_key(w.J[size_t(i) * P + k]);
            if (a > best || (a == best && i < bi)) {
                best = a;
                bi = i;
            }
        }
        const int p = min(warp_argmax_row(best, bi), n);
        const TJ pv = (p < n) ? w.J[size_t(p) * P + k] : TJ(0);
        __syncwarp();   // every lane has read the pivot before the row swap overwrites it
        if (!key_is_finite_nonzero(abs_key(pv))) return false;
        if (p != k) {
            for (int j = lane; j < n; j += 32) {
                TJ t = w.J[size_t(k) * P + j];
                w.J[size_t(k) * P + j] = w.J[size_t(p) * P + j];
                w.J[size_t(p) * P + j] = t;
            }
            if (lane == 0) {
                int16_t t = w.perm[k];
                w.perm[k] = w.perm[p];
                w.perm[p] = t;
            }
        }
        __syncwarp();
        const TJ inv = TJ(1.0) / pv;
        // multipliers and trailing update: lanes over rows
        for (int i = k + 1 + lane; i < n; i += 32) {
            TJ *ri = w.J + size_t(i) * P;
            const TJ *rk = w.J + size_t(k) * P;
            const TJ l = ri[k] * inv;
            ri[k] = l;
            int j = k + 1;
            for (; j + 7 < n; j += 8) {   // loads batched ahead of the stores
                TJ a[8], b[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    a[u] = ri[j + u];
                    b[u] = rk[j + u];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) ri[j + u] = fma(-l, b[u], a[u]);
            }
            for (; j < n; ++j) ri[j] = fma(-l, rk[j], ri[j]);
        }
        __syncwarp();
    }
    return true;
}

// Blocked right-looking LU with partial pivoting (the LAPACK getrf order; the same pivots
// as lu_factor in exact arithmetic): panels of kLuNB columns are factored column by column
// (pivot search and full-row interchange as in lu_factor, the multipliers updating only the
// panel's columns), then U12 = L11^-1 A12 with one lane per column (L11 read by broadcast)
// and the trailing update A22 -= L21 U12 with one lane per row, the row's kLuNB
// multipliers in registers: ten shared-memory accesses per kLuNB FMAs instead of three per
// FMA, and one warp barrier per panel instead of one per column.
constexpr int kLuNB = 8;
template <class TJ>
__device__ PSR_STAGE_LU bool lu_factor_blocked(const WS<TJ> &w, int n) {
    const int lane = threadIdx.x & 31;
    const int P = w.P;
    TJ *J = w.J;
    for (int j = lane; j < n; j += 32) w.perm[j] = int16_t(j);
    __syncwarp();
    for (int k0 = 0; k0 < n; k0 += kLuNB) {
        const int kend = min(k0 + kLuNB, n);
        for (int k = k0; k < kend; ++k) {
            // pivot: first row of largest |a_ik|, i >= k (integer keys of |a|)
            decltype(abs_key(TJ(0))) best = 0;
            int bi = n;
            for (int i = k + lane; i < n; i += 32) {
                const auto a = abs_key(J[size_t(i) * P + k]);
                if (a > best || (a == best && i < bi)) {
                    best = a;
                    bi = i;
                }
            }
            const int p = min(warp_argmax_row(best, bi), n);
            const TJ pv = (p < n) ? J[size_t(p) * P + k] : TJ(0);
            __syncwarp();   // every lane has read the pivot before the row swap overwrites it
            if (!key_is_finite_nonzero(abs_key(pv))) return false;
            if (p != k) {
                for (int j = lane; j < n; j += 32) {
                    TJ t = J[size_t(k) * P + j];
                    J[size_t(k) * P + j] = J[size_t(p) * P + j];
                    J[size_t(p) * P + j] = t;
                }
                if (lane == 0) {
                    int16_t t = w.perm[k];
                    w.perm[k] = w.perm[p];
                    w.perm[p] = t;
                }
            }
            __syncwarp();
            const TJ inv = TJ(1.0) / pv;
            for (int i = k + 1 + lane; i < n; i += 32) {
                TJ *ri = J + size_t(i) * P;
                const TJ *rk = J + size_t(k) * P;
                const TJ l = ri[k] * inv;
                ri[k] = l;
                for (int c = k + 1; c < kend; ++c) ri[c] = fma(-l, rk[c], ri[c]);
            }
            __syncwarp();
        }
        if (kend >= n) break;   // the last panel may be narrower; every earlier one is kLuNB wide
        // U12 = L11^-1 A12 (unit lower L11): one lane per column
        for (int c = kend + lane; c < n; c += 32) {
            TJ u[kLuNB];
#pragma unroll
            for (int t = 0; t < kLuNB; ++t) u[t] = J[size_t(k0 + t) * P + c];
#pragma unroll
            for (int t = 1; t < kLuNB; ++t) {
                const TJ *Lt = J + size_t(k0 + t) * P + k0;
#pragma unroll
                for (int q = 0; q < t; ++q) u[t] = fma(-Lt[q], u[q], u[t]);
            }
#pragma unroll
            for (int t = 1; t < kLuNB; ++t) J[size_t(k0 + t) * P + c] = u[t];
        }
        __syncwarp();
        // A22 -= L21 U12: one lane per row, its multipliers in registers, U12 by broadcast
        for (int i = kend + lane; i < n; i += 32) {
            TJ *ri = J + size_t(i) * P;
            TJ l[kLuNB];
#pragma unroll
            for (int t = 0; t < kLuNB; ++t) l[t] = ri[k0 + t];
            for (int c = kend; c < n; ++c) {
                TJ a = ri[c];
#pragma unroll
                for (int t = 0; t < kLuNB; ++t) a = fma(-l[t], J[size_t(k0 + t) * P + c], a);
                ri[c] = a;
            }
        }
        __syncwarp();
    }
    return true;
}

// Solve (LU) x = -r with r distributed (V2), x returned as V2 (FP64 promote).
template <class TJ>
__device__ PSR_STAGE_SOLVE void lu_solve_neg(const WS<TJ> &w, int n, const V2 &r, V2 &x) {
    const int lane = threadIdx.x & 31;
    const int P = w.P;
    // rhs[k] = -r[perm[k]]: stage r in rhs via the permutation
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        if (j < n) w.rhs[j] = TJ(-(h ? r.b : r.a));
    }
    __syncwarp();
    TJ pr[2];
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        pr[h] = (j < n) ? w.rhs[w.perm[j]] : TJ(0);
    }
    __syncwarp();
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        if (j < n) w.rhs[j] = pr[h];
    }
    __syncwarp();
    // forward: unit lower
    for (int k = 0; k < n - 1; ++k) {
        const TJ bk = w.rhs[k];
        for (int i = k + 1 + lane; i < n; i += 32) w.rhs[i] = fma(-w.J[size_t(i) * P + k], bk, w.rhs[i]);
        __syncwarp();
    }
    // backward: upper
    for (int k = n - 1; k >= 0; --k) {
        const TJ xk = w.rhs[k] / w.J[size_t(k) * P + k];
        __syncwarp();
        for (int i = lane; i < k; i += 32) w.rhs[i] = fma(-w.J[size_t(i) * P + k], xk, w.rhs[i]);
        if (lane == 0) w.rhs[k] = xk;
        __syncwarp();
    }
    x.a = (lane < n) ? double(w.rhs[lane]) : 0.0;
    x.b = (lane + 32 < n) ? double(w.rhs[lane + 32]) : 0.0;
    __syncwarp();
}

// Solve J^T lam = g with the factors of P J = L U: U^T z = g (forward), L^T v = z
// (backward, unit diagonal), lam[perm[j]] = v[j]. g and lam are distributed (V2).
template <class TJ>
__device__ void lu_solve_T(const WS<TJ> &w, int n, const V2 &g, V2 &lam) {
    const int lane = threadIdx.x & 31;
    const int P = w.P;
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        if (j < n) w.rhs[j] = TJ(h ? g.b : g.a);
    }
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        const TJ zk = w.rhs[k] / w.J[size_t(k) * P + k];
        __syncwarp();
        for (int j = k + 1 + lane; j < n; j += 32) w.rhs[j] = fma(-w.J[size_t(k) * P + j], zk, w.rhs[j]);
        if (lane == 0) w.rhs[k] = zk;
        __syncwarp();
    }
    for (int k = n - 1; k >= 1; --k) {
        const TJ vk = w.rhs[k];
        for (int j = lane; j < k; j += 32) w.rhs[j] = fma(-w.J[size_t(k) * P + j], vk, w.rhs[j]);
        __syncwarp();
    }
    // lam_c = v_j for the j with perm[j] = c
    double out[2] = {0.0, 0.0};
    for (int j = 0; j < n; ++j) {
        const int c = w.perm[j];
        if (c == lane) out[0] = double(w.rhs[j]);
        if (c == lane + 32) out[1] = double(w.rhs[j]);
    }
    lam.a = out[0];
    lam.b = out[1];
    __syncwarp();
}

#ifndef PSR_LU_BLOCKED
#define PSR_LU_BLOCKED 1
#endif
// The solver's factorisation (the service kernels keep the unblocked one).
template <class TJ>
__device__ __forceinline__ bool lu_factor_solver(const WS<TJ> &w, int n) {
    if constexpr (PSR_LU_BLOCKED) return lu_factor_blocked(w, n);
    else return lu_factor(w, n);
}

// ---------------------------------------------------------------- solver pieces
struct Reactor {
    const double *Yin;
    const double *Min;   // [6] inlet soot moments (sooting mechanisms)
    double tau, P, Tspec;
};

__device__ __forceinline__ bool all_finite(const V2 &v) {
    return __all_sync(kFull, isfinite(v.a) && isfinite(v.b));
}

// mass fractions and log moments absolute, temperature relative
__device__ __forceinline__ double scaled_max(const V2 &dy, const V2 &y, int K, int n) {
    const int lane = threadIdx.x & 31;
    double m = 0.0;
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        if (j < n) {
            double d = fabs(h ? dy.b : dy.a);
            if (j == K) d /= fabs(h ? y.b : y.a);
            m = fmax(m, d);
        }
    }
    return wmax(m);
}

__device__ __forceinline__ bool in_bounds(const V2 &y, int K, const Opts &o) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        double v = h ? y.b : y.a;
        if (j < K) ok = ok && (v >= -o.y_floor);
        else if (j == K) ok = ok && (v >= o.t_min && v <= o.t_max);
    }
    return __all_sync(kFull, ok);
}

// Largest step fraction that keeps Y_k >= -y_floor and t_min <= T <= t_max, and moves no
// log moment by more than kZetaStep (moment sets stay in the range where the interpolative
// closure is defined).
__device__ __forceinline__ double max_in_bounds(const V2 &y, const V2 &dy, int K, int n, const Opts &o) {
    const int lane = threadIdx.x & 31;
    double lam = INFINITY;
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        const double x = h ? y.b : y.a, d = h ? dy.b : dy.a;
        if (j > K) {
            if (j < n && fabs(d) > kZetaStep) lam = fmin(lam, kZetaStep / fabs(d));
            continue;
        }
        const double lo = (j < K) ? -o.y_floor : o.t_min, hi = (j < K) ? INFINITY : o.t_max;
        if (d < 0 && x + d < lo) lam = fmin(lam, (lo - x) / d);
        else if (d > 0 && x + d > hi) lam = fmin(lam, (hi - x) / d);
    }
    return wmin(lam);
}

// |dx_j| <= rtol |x_j| + atol_j (species, temperature); |d zeta_r| <= atol_z (log moments)
__device__ __forceinline__ bool step_small(const V2 &dy, const V2 &y, int K, int n, double rtol, double atol_y,
                                           double atol_t, double atol_z) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int h = 0; h < 2; ++h) {
        int j = lane + 32 * h;
        if (j < n) {
            const double x = h ? y.b : y.a, d = h ? dy.b : dy.a;
            if (j <= K) ok = ok && (fabs(d) <= rtol * fabs(x) + ((j < K) ? atol_y : atol_t));
            else ok = ok && (fabs(d) <= atol_z);
        }
    }
    return __all_sync(kFull, ok);
}

__device__ __forceinline__ V2 axpy(const V2 &x, double a, const V2 &d) { return V2{x.a + a * d.a, x.b + a * d.b}; }

struct Ctx {
    DevMech M;
    Opts o;
    Reactor r;
    const double *mult;
    int nfev;
    Mix mx;
    SpecLane sl;
    int K, n;
    const int *idle;   // warps of this launch that found the work queue empty
    int handoff_at;    // idle count at which running reactors are handed over (0 = never)
    bool handoff;      // set once this reactor is to be handed to the block solver
};

// True once enough warps of the launch are idle that the reactor this warp is solving
// goes to the block solver (one thread block per reactor finishes a straggler far sooner
// than a lone warp): checked at each Newton iteration, one global load by lane 0.
__device__ __forceinline__ bool handoff_due(Ctx &cx) {
    if (cx.handoff_at <= 0) return false;
    int v = 0;
    if ((threadIdx.x & 31) == 0) v = *reinterpret_cast<const volatile int *>(cx.idle);
    v = __shfl_sync(kFull, v, 0);
    cx.handoff = v >= cx.handoff_at;
    return cx.handoff;
}

// One out-of-line copy of the residual for the FP32-Jacobian solver instead of one inlined
// copy per call site: with its Jacobian assembly in FP32 the solver is bound by instruction
// fetch more than by call overhead (measured at K = 53: 9 % faster out of line, while the
// FP64-Jacobian solver is 7 % faster with the copies inlined).
template <class TJ, bool SOOT>
__device__ __noinline__ void eval_F_outlined(const DevMech &M, const WS<TJ> &w, const V2 &y, V2 &F, Mix &mx,
                                             SpecLane &sl, const double *Yin_row, const double *Min, double tau,
                                             double P, double Tspec, int energy, const double *__restrict__ mult) {
    eval_F<TJ, SOOT>(M, w, y, F, mx, sl, Yin_row, Min, tau, P, Tspec, energy, mult);
}

template <class TJ, bool SOOT>
__device__ PSR_STAGE_RES void residual_R(Ctx &cx, const WS<TJ> &w, const V2 &y, const V2 &c, const V2 &xref, V2 &F,
                                         V2 &R) {
    ++cx.nfev;
    if constexpr (sizeof(TJ) == 4 && PSR_OUTLINE_F32)
        eval_F_outlined<TJ, SOOT>(cx.M, w, y, F, cx.mx, cx.sl, cx.r.Yin, cx.r.Min, cx.r.tau, cx.r.P, cx.r.Tspec,
                                  cx.o.energy, cx.mult);
    else
        eval_F<TJ, SOOT>(cx.M, w, y, F, cx.mx, cx.sl, cx.r.Yin, cx.r.Min, cx.r.tau, cx.r.P, cx.r.Tspec, cx.o.energy,
                         cx.mult);
    R.a = F.a + c.a * (y.a - xref.a);
    R.b = F.b + c.b * (y.b - xref.b);
}

// Damped Newton on R(y) = F(y) + c (y - xref) from y (see the oracle's description).
template <class TJ, bool SOOT, bool FDJ = false>
__device__ PSR_STAGE_NEWTON bool damped_newton(Ctx &cx, const WS<TJ> &w, V2 &y, const V2 &xref, const V2 &c, int max_it,
                              bool steady, int &counter, double *fnorm) {
    const int K = cx.K, n = cx.n;
    const Opts &o = cx.o;
    V2 F, R;
    residual_R<TJ, SOOT>(cx, w, y, c, xref, F, R);
    // ||F||_inf of the steady residual at the first and the last evaluated point
    if (fnorm) fnorm[0] = fnorm[1] = wmax(fmax(fabs(F.a), fabs(F.b)));
    double dn_prev = INFINITY;
    // Jacobian reuse (o.jac_age > 1): the LU factors serve up to jac_age iterations while
    // undamped steps keep shrinking; any failure with old factors retries with fresh ones
    bool have_lu = false, at_y = true;
    int age = 0;
    for (int it = 0; it < max_it; ++it) {
        if (counter >= o.max_newton || handoff_due(cx)) break;
        ++counter;
        bool fresh = false;
        if (!have_lu || age + 1 >= o.jac_age) {
            if (!at_y) {   // the last residual was a rejected trial: the Jacobian needs y's caches
                V2 Fy;
                residual_R<TJ, SOOT>(cx, w, y, c, xref, Fy, R);
                if (fnorm) fnorm[1] = wmax(fmax(fabs(Fy.a), fabs(Fy.b)));
                at_y = true;
            }
            if constexpr (FDJ)
                eval_J_fd<TJ>(cx.M, w, y, c, cx.mx, cx.sl, cx.r.Yin, cx.r.tau, cx.r.P, cx.r.Tspec, o.energy,
                              cx.mult);
            else
                eval_J<TJ, SOOT>(cx.M, w, y, c, cx.mx, cx.sl, cx.r.Yin, cx.r.Min, cx.r.tau, o.energy, cx.mult);
            if (!lu_factor_solver(w, n)) break;
            have_lu = true;
            age = 0;
            fresh = true;
        } else {
            ++age;
        }
        V2 dy;
        lu_solve_neg(w, n, R, dy);
        if (!all_finite(dy)) {
            if (!fresh) {
                have_lu = false;
                continue;
            }
            break;
        }
        if (steady) {
            const double rmax = wmax(fmax(fabs(R.a), fabs(R.b)));
            if (rmax <= o.ftol && step_small(dy, y, K, n, o.step_rtol, o.step_atol_y, o.step_atol_t, o.step_rtol)) {
                y = axpy(y, 1.0, dy);
                return true;
            }
        } else if (step_small(dy, y, K, n, o.ts_rtol, o.ts_atol_y, o.ts_rtol, o.ts_rtol)) {
            y = axpy(y, 1.0, dy);
            return true;
        }
        const double dn = scaled_max(dy, y, K, n);
        if (dn >= dn_prev) {
            if (!fresh) {
                have_lu = false;
                continue;
            }
            break;
        }
        double lam = fmin(1.0, max_in_bounds(y, dy, K, n, o));
        bool accepted = false;
        V2 yt, Rt;
        for (int d = 0; d < o.max_damp; ++d) {
            yt = axpy(y, lam, dy);
            if (in_bounds(yt, K, o)) {
                V2 Ft;
                residual_R<TJ, SOOT>(cx, w, yt, c, xref, Ft, Rt);
                at_y = false;
                if (fnorm) fnorm[1] = wmax(fmax(fabs(Ft.a), fabs(Ft.b)));
                if (all_finite(Rt)) {
                    V2 db;
                    lu_solve_neg(w, n, Rt, db);
                    if (scaled_max(db, y, K, n) < dn) {
                        accepted = true;
                        break;
                    }
                }
            }
            lam *= 0.5;
        }
        if (!accepted) {
            if (!fresh) {
                have_lu = false;
                continue;
            }
            break;
        }
        dn_prev = dn;
        y = yt;
        R = Rt;
        at_y = true;
        if (lam < 1.0) have_lu = false;   // a damped step: fresh factors next
    }
    return false;
}

// One linearised backward-Euler step of dx/dt = -D F / tau from x (pseudo-transient
// continuation): (J(x) + diag c) dx = -F(x), the full step taken when it stays in bounds
// and F stays finite. fx_valid: Fx holds F(x) and the rate caches are x's (true after an
// accepted step; the Jacobian consumes the caches). f_new = ||F||_inf at the new x.
template <class TJ, bool SOOT, bool FDJ = false>
__device__ bool linear_step(Ctx &cx, const WS<TJ> &w, V2 &x, V2 &Fx, bool &fx_valid, const V2 &c, int &counter,
                            double &f_new) {
    const int K = cx.K, n = cx.n;
    const Opts &o = cx.o;
    if (counter >= o.max_newton || handoff_due(cx)) return false;
    ++counter;
    const V2 zero{0.0, 0.0};
    if (!fx_valid) {
        V2 R;
        residual_R<TJ, SOOT>(cx, w, x, zero, x, Fx, R);
    }
    fx_valid = false;
    if constexpr (FDJ)
        eval_J_fd<TJ>(cx.M, w, x, c, cx.mx, cx.sl, cx.r.Yin, cx.r.tau, cx.r.P, cx.r.Tspec, o.energy, cx.mult);
    else
        eval_J<TJ, SOOT>(cx.M, w, x, c, cx.mx, cx.sl, cx.r.Yin, cx.r.Min, cx.r.tau, o.energy, cx.mult);
    if (!lu_factor_solver(w, n)) return false;
    V2 dx;
    lu_solve_neg(w, n, Fx, dx);
    if (!all_finite(dx) || max_in_bounds(x, dx, K, n, o) < 1.0) return false;
    const V2 xt = axpy(x, 1.0, dx);
    if (!in_bounds(xt, K, o)) return false;
    V2 Ft, R;
    residual_R<TJ, SOOT>(cx, w, xt, zero, xt, Ft, R);
    if (!all_finite(Ft)) return false;
    f_new = wmax(fmax(fabs(Ft.a), fabs(Ft.b)));
    x = xt;
    Fx = Ft;
    fx_valid = true;
    return true;
}

// Initial log moments: the given M0, or the nucleation-only steady state at the initial
// gas state, M_r = M_r,in + tau J C_min^r.
__device__ void init_moments(Ctx &cx, const Batch &bt, int64_t r, V2 &x) {
    const int lane = threadIdx.x & 31;
    const int K = cx.K;
    const double *st = cx.M.soot;
    double Mr[kNMom];
    if (bt.M0) {
#pragma unroll
        for (int q = 0; q < kNMom; ++q) Mr[q] = bt.M0[r * kNMom + q];
    } else {
        double sYW = 0.0;
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            if (j < K) sYW += (h ? x.b : x.a) * __ldg(cx.M.invW + j);
        }
        sYW = wsum(sYW);
        const double T0 = comp_get(x, K);
        const double YP = comp_get(x, cx.M.soot_P);
        const double rho = cx.r.P / (sYW * kRu * T0);
        const double CP = rho * YP * __ldg(cx.M.invW + cx.M.soot_P);
        const double J = exp(__ldg(st + kSootNucLnA) - __ldg(st + kSootNucTheta) / T0) * CP * 6.02214076e23;
        double cr = 1.0;
#pragma unroll
        for (int q = 0; q < kNMom; ++q) {
            Mr[q] = cx.r.Min[q] + cx.r.tau * J * cr;
            cr *= __ldg(st + kSootCmin);
        }
    }
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        if (j > K && j <= K + kNMom) {
            double m = 0.0;
#pragma unroll
            for (int q = 0; q < kNMom; ++q) m = (q == j - K - 1) ? Mr[q] : m;
            const double z = log(m / __ldg(st + kSootScale + (j - K - 1)));
            if (h) x.b = z;
            else x.a = z;
        }
    }
}

template <class TJ, bool SOOT, bool FDJ = false>
__device__ void solve_one(Ctx &cx, const WS<TJ> &w, const Batch &bt, int64_t r) {
    const int lane = threadIdx.x & 31;
    const int K = cx.K;
    const Opts &o = cx.o;
    const double tau = bt.tau[r];
    const int64_t row = row_of(bt, r, K);
    cx.r.Yin = bt.Y_in + row;
    cx.r.Min = (SOOT && bt.M_in) ? bt.M_in + r * kNMom : nullptr;
    cx.r.tau = tau;
    cx.r.P = bt.P[r];
    cx.r.Tspec = bt.T0[r];
    cx.nfev = 0;
    cx.handoff = false;
    // inlet enthalpy sum_k Y_k,in h_k(T_in)
    {
        const double Tin = bt.T_in[r], lnTin = log(Tin);
        double s = 0.0;
        for (int h = 0; h < 2; ++h) {
            int j = lane + 32 * h;
            if (j < K) {
                double cpR, hRT, sR, dcpR;
                nasa7(cx.M.nasa, j, Tin, lnTin, 1.0 / Tin, cpR, hRT, sR, dcpR);
                s += cx.r.Yin[j] * hRT * __ldg(cx.M.invW + j);
            }
        }
        cx.mx.h_in = wsum(s) * kRu * Tin;
    }
    V2 x;
    x.a = (lane < K) ? bt.Y0[row + lane] : (lane == K ? bt.T0[r] : 0.0);
    x.b = (lane + 32 < K) ? bt.Y0[row + lane + 32] : (lane + 32 == K ? bt.T0[r] : 0.0);
    if constexpr (SOOT) init_moments(cx, bt, r, x);
    const V2 zero{0.0, 0.0};
    V2 F, R;
    residual_R<TJ, SOOT>(cx, w, x, zero, x, F, R);
    int status, counter = 0, ts = 0, rounds = 0;
    V2 out = x;
    if (!all_finite(F)) {
        status = PSR_NONFINITE;
    } else {
        double dt = o.dt0_over_tau * tau;
        while (true) {
            V2 y = x;
            double fn[2];
            bool conv = damped_newton<TJ, SOOT, FDJ>(cx, w, y, x, zero, o.max_newton, true, counter, fn);
            if (conv) {
                status = PSR_CONVERGED;
                out = y;
                break;
            }
            if (cx.handoff) {   // the Newton iterate is no worse than x (monotone corrections)
                status = kStatusHandoff;
                out = y;
                break;
            }
            if (counter >= o.max_newton) {
                status = PSR_MAX_ITER;
                out = y;
                break;
            }
            ++rounds;
            if (rounds > o.max_ts_rounds) {
                status = PSR_TS_EXHAUSTED;
                out = x;
                break;
            }
            int taken = 0;
            bool done = false;
            double f_prev = fn[0];   // ||F(x)||_inf of the estimate being conditioned
            bool fx_valid = false;   // the steady attempt left the caches elsewhere
            V2 Fx = F;
            while (taken < o.ts_steps) {
                const double Tx = comp_get(x, K);
                const double s = tau / dt;
                V2 c;
                const double sT = (o.energy == PSR_FIXED_T) ? s : s / Tx;
                c.a = (lane < K) ? s : (lane == K ? sT : (lane < cx.n ? s : 0.0));
                c.b = (lane + 32 < K) ? s : (lane + 32 == K ? sT : (lane + 32 < cx.n ? s : 0.0));
                const int used0 = counter;
                V2 y = x;
                double f_new = 0.0;
                bool ok;
                const bool linear = counter < o.ts_linear;
                if (linear) {
                    ok = linear_step<TJ, SOOT, FDJ>(cx, w, y, Fx, fx_valid, c, counter, f_new);
                } else {
                    double fs[2];
                    ok = damped_newton<TJ, SOOT, FDJ>(cx, w, y, x, c, o.ts_newton, false, counter, fs);
                    f_new = fs[1];
                }
                const int used = counter - used0;
                if (cx.handoff) {   // the last accepted pseudo-time state
                    status = kStatusHandoff;
                    out = x;
                    done = true;
                    break;
                }
                if (counter >= o.max_newton) {
                    status = PSR_MAX_ITER;
                    out = x;
                    done = true;
                    break;
                }
                if (ok) {
                    x = y;
                    ++taken;
                    ++ts;
                    // switched evolution relaxation: dt follows the step's change of ||F||
                    double g;
                    if (linear) {
                        g = 2.0 * (f_new > 0.0 ? fmin(8.0, fmax(0.1, f_prev / f_new)) : 1.0);
                    } else {   // Newton-solved steps: also by how easily the step was solved
                        g = (used <= 3) ? 2.0 : (used == 4 ? 1.25 : 1.0);
                        if (f_new > 0.0) g *= fmin(4.0, fmax(1.0, f_prev / f_new));
                    }
                    f_prev = f_new;
                    dt = fmin(g * dt, 1e6 * tau);
                } else {
                    dt *= o.dt_shrink;
                    if (dt < 1e-16 * tau) {
                        status = PSR_TS_EXHAUSTED;
                        out = x;
                        done = true;
                        break;
                    }
                }
            }
            if (done) break;
        }
    }
    // report ||F||_inf at the output state
    residual_R<TJ, SOOT>(cx, w, out, zero, out, F, R);
    const double fn = wmax(fmax(fabs(F.a), fabs(F.b)));
    if (lane < K) bt.Y_out[row + lane] = out.a;
    if (lane + 32 < K) bt.Y_out[row + lane + 32] = out.b;
    const double Tout = comp_get(out, K);
    if (SOOT && bt.M_out) {
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            if (j > K && j <= K + kNMom)
                bt.M_out[r * kNMom + (j - K - 1)] = __ldg(cx.M.soot + kSootScale + (j - K - 1)) * exp(h ? out.b : out.a);
        }
    }
    if (lane == 0) {
        bt.T_out[r] = Tout;
        const bool fb = bt.fallback != 0;
        if (bt.status) bt.status[r] = (bt.fallback == 1 && status == PSR_CONVERGED) ? PSR_REFINE_FALLBACK : status;
        if (bt.iters) bt.iters[r] = counter + (fb ? bt.iters[r] : 0);
        if (bt.ts_steps) bt.ts_steps[r] = ts + (fb ? bt.ts_steps[r] : 0);
        if (bt.fnorm) bt.fnorm[r] = fn;
        if (bt.nfev) bt.nfev[r] = cx.nfev + (fb ? bt.nfev[r] : 0);
    }
}

// 3 resident 128-thread blocks per SM caps registers at 168 without spills (measured 5%
// faster than the uncapped 210-register build on GB300 at K = 53).
#ifndef PSR_MIN_BLOCKS
#define PSR_MIN_BLOCKS 3
#endif
constexpr int kMaxSolveWarps = 4;   // the solver kernel's block holds at most 4 warps (128 threads)
constexpr int kDefaultSolveWarps = 2;   // measured best at K = 53 for both forms (finer shared-memory packing)
template <class TJ, bool SOOT, bool FDJ = false>
// queue[0]: work-queue tickets; queue[1]: warps that found the queue empty (both zeroed
// by the launcher).
__global__ void __launch_bounds__(128, PSR_MIN_BLOCKS) solve_kernel(DevMech M, Batch bt, Opts o, int *queue,
                                                                   size_t ws_per_warp) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int ns = SOOT ? kNMom : 0;
    WS<TJ> w = carve<TJ>(smem + warp * ws_per_warp, M.K, M.I, M.K + 1 + ns, M.n_troe, ns);
    Ctx cx;
    cx.M = M;
    cx.o = o;
    cx.mult = bt.rate_mult;
    cx.K = M.K;
    cx.n = M.K + 1 + ns;
    cx.idle = queue + 1;
    const int64_t nwork = bt.list ? int64_t(*bt.list_len) : bt.B;
    // warps that never get a reactor go idle at once: the threshold counts working warps only;
    // a batch of fewer than two reactors per warp has no tail worth a second launch
    cx.handoff_at = 0;
    const int64_t W = int64_t(gridDim.x) * (blockDim.x >> 5);
    if (o.handoff_pct > 0 && nwork >= 2 * W) {
        const int64_t working = W < nwork ? W : nwork;
        cx.handoff_at = int((W - working) + (working * o.handoff_pct + 99) / 100);
    }
    while (true) {
        int p = 0;
        if (lane == 0) p = atomicAdd(queue, 1);
        p = __shfl_sync(kFull, p, 0);
        if (p >= nwork) {
            if (lane == 0) atomicAdd(queue + 1, 1);
            break;
        }
        const int64_t r = bt.list ? int64_t(bt.list[p]) : int64_t(p);
        solve_one<TJ, SOOT, FDJ>(cx, w, bt, r);
    }
}

}  // namespace
}  // namespace psr
