// Batched steady PSR solve for mechanisms too large for one warp (K + 1 > 64): one
// thread block per reactor, persistent over an atomic work queue.
//
// The method and its arithmetic are those of the warp solver: the hybrid damped Newton /
// pseudo-transient scheme of Sec. 3 on the residual of Eqs. (2)-(3) with the rates of
// Eqs. (4)-(9). Only the mapping differs. Thread j owns component j (n <= 512); state
// vectors, species and reaction tables sit in shared memory; the Jacobian [n][P] is in
// shared memory when it fits (the FP32 Jacobian of a K = 200 mechanism takes 162 KB) and
// otherwise in a per-block global slot that stays L2-resident (FP64 at K = 200: 323 KB
// per block, 49 MB for 152 blocks). Block-wide sums use a fixed reduction order, so every
// thread holds bit-identical scalars and all control flow is block-uniform.
//
// This header holds the solver's device code; psr_block.cu adds its kernels and host
// launchers, and the one-launch solver of a batch of several mechanisms includes it too.
#pragma once
#include <algorithm>
#include <string>

#include "psr_device.cuh"
#include "psr_internal.h"
#include "psr_tc.cuh"

// Built with 512 threads per block (every entry point of psr_block.cu), with 256 (its
// solver, the default for mechanisms with K + 1 <= 256: more resident blocks per SM when
// the Jacobian lives in global memory, cheaper block barriers) and, with 256 again, inside
// the persistent multi-mechanism kernel (psr_multi.cu); the code sits in namespace
// psr::bt512 or psr::bt256 of its translation unit.
#ifndef PSR_BLOCK_THREADS
#define PSR_BLOCK_THREADS 512
#endif
#if PSR_BLOCK_THREADS == 512
#define PSR_BLOCK_NS bt512
#elif PSR_BLOCK_THREADS == 256
#define PSR_BLOCK_NS bt256
#else
#error "PSR_BLOCK_THREADS must be 256 or 512"
#endif

namespace psr {
namespace PSR_BLOCK_NS {
namespace {

constexpr int kBT = PSR_BLOCK_THREADS;   // threads per block
constexpr int kBW = kBT / 32;     // warps per block
constexpr int kMaxBlockN = kBT;   // unknowns per reactor: thread j owns component j
constexpr int kRedSlots = 8;      // values reduced together

// Per-block workspace. Vectors [n]; species [K(+1)]; reactions [I]; Jacobian [n][P].
template <class TJ>
struct BWS {
    double *x, *y, *yt, *c, *F, *R, *Rt, *dy, *db;
    double *C, *hRT, *gS;     // [K+1] concentrations (C[K] = 1), H/RT, S/R - H/RT (sentinels 0)
    double *cpR, *dcpR;       // [K] c_p/R and its T-derivative of the last residual
    double *kf, *kr, *q;      // [I] effective rate constants, q_i (or Euler sums after the Jacobian)
    double *v, *ra, *rb;      // [K] wdot / dense third-body column part; row coefficients
    double *tD, *tX;          // [n_troe] falloff derivative caches
    double *red;              // [kRedSlots][kBW] reduction partials
    int *ired;                // [2][kBW] pivot-search partials (double-buffered), the work-queue
                              // slot, the tensor-core phase and failure flag
    TJ *J;                    // [n][P]
    TJ *rhs;                  // [n]
    int16_t *perm;            // [n]
    int P;
    // tensor-core trailing update (FP32 Jacobian only): mode 0 = off, 1 = TF32, 3 = 3xTF32
    int tc;
    uint64_t *bar;            // mbarrier of the MMA completions
    uint32_t *tmem_slot;      // tensor-memory base address of the accumulator
    char *stage;              // kStageBytes of operand tiles (128-byte aligned)
};

// Operand staging of the tensor-core update: hi and lo TF32 parts of a 128 x 16 L21 tile
// and of a 128 x 16 U12 tile (8 KB each). It reuses the rate arrays (kf, kr, q), which are
// dead between the Jacobian assembly and the next residual, when they are large enough.
constexpr int kStageBytes = 4 * 8192;
constexpr int kTcMinM = 64;      // smallest trailing matrix updated on the tensor cores
constexpr int kIred = 2 * kBW + 8;

__host__ __device__ inline bool stage_in_rates(int I) { return size_t(3) * I * 8 >= size_t(kStageBytes) + 128; }

__host__ __device__ inline int pitch_of(int n) { return (n & 1) ? n : n + 1; }

__host__ __device__ inline size_t bws_doubles(int K, int I, int nt, int n) {
    return size_t(9) * n + 3 * size_t(K + 1) + 2 * size_t(K) + 3 * size_t(I) + 3 * size_t(K) + 2 * size_t(nt) +
           size_t(kRedSlots) * kBW;
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Shared-memory bytes of one block: the vector/table part, rhs and perm, and the
// Jacobian itself when j_in_smem.
template <class TJ>
__host__ __device__ inline size_t bws_bytes(int K, int I, int nt, int n, bool j_in_smem, bool tc = false) {
    size_t b = align16(sizeof(double) * bws_doubles(K, I, nt, n));
    b = align16(b + sizeof(int) * kIred);
    b = align16(b + sizeof(TJ) * n);
    b = align16(b + sizeof(int16_t) * n);
    if (j_in_smem) b = align16(b + sizeof(TJ) * size_t(n) * pitch_of(n));
    if (tc && !stage_in_rates(I)) b = align16(b + kStageBytes + 128);
    return b;
}

template <class TJ>
__device__ BWS<TJ> bcarve(char *base, int K, int I, int nt, int n, TJ *Jglobal, int tc = 0) {
    BWS<TJ> w;
    double *d = reinterpret_cast<double *>(base);
    w.x = d;
    w.y = d + n;
    w.yt = d + 2 * n;
    w.c = d + 3 * n;
    w.F = d + 4 * n;
    w.R = d + 5 * n;
    w.Rt = d + 6 * n;
    w.dy = d + 7 * n;
    w.db = d + 8 * n;
    d += 9 * n;
    w.C = d;
    w.hRT = d + (K + 1);
    w.gS = d + 2 * (K + 1);
    d += 3 * (K + 1);
    w.cpR = d;
    w.dcpR = d + K;
    d += 2 * K;
    w.kf = d;
    w.kr = d + I;
    w.q = d + 2 * I;
    d += 3 * I;
    w.v = d;
    w.ra = d + K;
    w.rb = d + 2 * K;
    d += 3 * K;
    w.tD = d;
    w.tX = d + nt;
    d += 2 * nt;
    w.red = d;
    size_t off = align16(sizeof(double) * bws_doubles(K, I, nt, n));
    w.ired = reinterpret_cast<int *>(base + off);
    off = align16(off + sizeof(int) * kIred);
    w.rhs = reinterpret_cast<TJ *>(base + off);
    off = align16(off + sizeof(TJ) * n);
    w.perm = reinterpret_cast<int16_t *>(base + off);
    off = align16(off + sizeof(int16_t) * n);
    w.P = pitch_of(n);
    w.J = Jglobal ? Jglobal : reinterpret_cast<TJ *>(base + off);
    if (!Jglobal) off = align16(off + sizeof(TJ) * size_t(n) * w.P);
    w.tc = tc;
    w.bar = reinterpret_cast<uint64_t *>(w.ired + 2 * kBW + 4);     // 8-byte aligned (16-aligned base)
    w.tmem_slot = reinterpret_cast<uint32_t *>(w.ired + 2 * kBW + 6);
    char *st = stage_in_rates(I) ? reinterpret_cast<char *>(w.kf) : base + off;
    w.stage = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(st) + 127) & ~uintptr_t(127));
    return w;
}

// ---------------------------------------------------------------- tensor-core set-up
// Per block, when the tensor-core update is on: warp 0 allocates the accumulator's tensor
// memory, thread 0 initialises the mbarrier; the phase counter and the failure flag start
// at zero. tc_end frees the tensor memory (after a bounded wait for an update that failed
// to complete), before the block exits.
template <class TJ>
__device__ void tc_begin(const BWS<TJ> &w) {
    if (!w.tc) return;
    if (threadIdx.x < 32) tc::tmem_alloc(w.tmem_slot, tc::kTmemCols);
    if (threadIdx.x == 0) {
        tc::mbar_init(w.bar);
        w.ired[2 * kBW + 1] = 0;   // phase
        w.ired[2 * kBW + 2] = 0;   // failure
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

template <class TJ>
__device__ void tc_end(const BWS<TJ> &w) {
    if (!w.tc) return;
    __syncthreads();
    if (w.ired[2 * kBW + 2]) tc::mbar_wait(w.bar, uint32_t((w.ired[2 * kBW + 1] - 1) & 1));   // the timed-out MMAs
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(*w.tmem_slot, tc::kTmemCols);
}

// A22 -= L21 U12 on the tensor cores for the trailing matrix of a panel: rows and columns
// [r0, n), panel columns [k0, k0 + kb). Per 128-row tile and 128-column chunk, the K = kb
// panel width in rounds of 16: stage the TF32 tiles (hi, and lo for 3xTF32), one thread
// issues the MMAs into the tensor-memory accumulator, all wait on the mbarrier; then each
// warp reads its 32 accumulator lanes (rows) and subtracts them from the FP32 matrix.
// With 3xTF32 the product is A_hi B_hi + A_hi B_lo + A_lo B_hi (FP32-like accuracy).
// Returns false (block-uniform) when a wait timed out; the failure flag then turns the
// tensor cores off for the rest of the launch.
__device__ bool b_trailing_tc(const BWS<float> &w, int n, int r0, int k0, int kb) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int P = w.P, m = n - r0;
    float *J = w.J;
    const bool three = w.tc == 3;
    char *Ah = w.stage, *Al = w.stage + 8192, *Bh = w.stage + 16384, *Bl = w.stage + 24576;
    const uint32_t tbase = *w.tmem_slot;
    int phase = w.ired[2 * kBW + 1];
    bool ok = true;
    for (int rt = 0; rt < m && ok; rt += tc::kTileM) {
        for (int ct = 0; ct < m && ok; ct += tc::kTileM) {
            const int cols = min(tc::kTileM, m - ct);
            const int N = (cols + 15) & ~15;
            for (int kh = 0; kh < kb && ok; kh += tc::kTileK) {
                // stage L21 rows r0+rt.., panel columns k0+kh.. and U12 columns r0+ct.. (zero padded)
                for (int e = t; e < tc::kTileM * tc::kTileK; e += kBT) {
                    const int r = e >> 4, k = e & 15;
                    const int gr = rt + r, gk = kh + k;
                    const float a = (gr < m && gk < kb) ? J[size_t(r0 + gr) * P + k0 + gk] : 0.0f;
                    const int gc = ct + r;
                    const float b = (r < N && gc < m && gk < kb) ? J[size_t(k0 + gk) * P + r0 + gc] : 0.0f;
                    const uint32_t o = tc::tile_off(r, k);
                    const float ah = tc::to_tf32(a), bh = tc::to_tf32(b);
                    *reinterpret_cast<float *>(Ah + o) = ah;
                    *reinterpret_cast<float *>(Bh + o) = bh;
                    if (three) {
                        *reinterpret_cast<float *>(Al + o) = tc::to_tf32(a - ah);
                        *reinterpret_cast<float *>(Bl + o) = tc::to_tf32(b - bh);
                    }
                }
                tc::fence_async_smem();
                __syncthreads();
                if (t == 0) {
                    tc::fence_after_sync();
                    const uint32_t id = tc::idesc_tf32(tc::kTileM, N);
                    const uint32_t sAh = tc::smem_u32(Ah), sAl = tc::smem_u32(Al), sBh = tc::smem_u32(Bh),
                                   sBl = tc::smem_u32(Bl);
#pragma unroll
                    for (int s = 0; s < 2; ++s) {   // two K-steps of 8 per round
                        const uint32_t ko = 256u * s;
                        tc::mma_tf32(tbase, tc::smem_desc(sAh + ko), tc::smem_desc(sBh + ko), id, (kh > 0 || s > 0));
                        if (three) {
                            tc::mma_tf32(tbase, tc::smem_desc(sAh + ko), tc::smem_desc(sBl + ko), id, 1u);
                            tc::mma_tf32(tbase, tc::smem_desc(sAl + ko), tc::smem_desc(sBh + ko), id, 1u);
                        }
                    }
                    tc::commit(w.bar);
                }
                ok = __syncthreads_and(tc::mbar_wait(w.bar, uint32_t(phase & 1))) != 0;
                ++phase;
                tc::fence_after_sync();
            }
            if (ok) {
                // epilogue: warp w reads accumulator lanes 32 (w % 4).. (the lanes its SM
                // sub-partition may access), 16-column blocks (w / 4) * 16 + (kBW / 4) * 16 u
                const int q = wid & 3;
                const int row = rt + 32 * q + lane;
                for (int cb = (wid >> 2) * 16; cb < N; cb += (kBW / 4) * 16) {
                    float v[16];
                    tc::ld16(tbase + (uint32_t(32 * q) << 16) + uint32_t(cb), v);
                    if (row < m) {
                        float *Jr = J + size_t(r0 + row) * P + r0 + ct + cb;
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (ct + cb + i < m) Jr[i] -= v[i];
                    }
                }
            }
            tc::fence_before_sync();
            __syncthreads();
        }
    }
    if (t == 0) {
        w.ired[2 * kBW + 1] = phase;
        if (!ok) w.ired[2 * kBW + 2] = 1;
    }
    __syncthreads();
    return ok;
}

// ---------------------------------------------------------------- block reductions
// Sums of NV values over the block; every thread receives the same totals.
template <int NV>
__device__ __forceinline__ void bsum(double (&v)[NV], double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = wsum(v[k]);
    __syncthreads();   // the previous reduction's partials have been read
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) red[k * kBW + wid] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
#pragma unroll
        for (int u = 0; u < kBW; ++u) s += red[k * kBW + u];
        v[k] = s;
    }
}

__device__ __forceinline__ double bsum1(double x, double *red) {
    double v[1] = {x};
    bsum<1>(v, red);
    return v[0];
}

__device__ __forceinline__ double bmax(double x, double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    x = wmax(x);
    __syncthreads();
    if (lane == 0) red[wid] = x;
    __syncthreads();
    double m = red[0];
#pragma unroll
    for (int u = 1; u < kBW; ++u) m = fmax(m, red[u]);
    return m;
}

__device__ __forceinline__ double bmin(double x, double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    x = wmin(x);
    __syncthreads();
    if (lane == 0) red[wid] = x;
    __syncthreads();
    double m = red[0];
#pragma unroll
    for (int u = 1; u < kBW; ++u) m = fmin(m, red[u]);
    return m;
}

// ---------------------------------------------------------------- residual, Eqs. (2)-(9)
// F at state y (shared); leaves C, hRT, gS, cpR, dcpR, kf, kr, q, v = wdot and the falloff
// caches of this state in shared memory and the mixture scalars in mx (every thread).
template <class TJ>
__device__ void b_eval_F(const DevMech &M, const BWS<TJ> &w, const double *y, double *F, Mix &mx,
                         const double *Yin, double tau, double P, double Tspec, int energy,
                         const double *__restrict__ mult) {
    const int t = threadIdx.x;
    const int K = M.K, I = M.I;
    __syncthreads();   // y complete
    const double T = y[K];
    const double lnT = log(T), invT = 1.0 / T;
    mx.T = T;
    mx.lnT = lnT;
    mx.invT = invT;
    const double sYW = bsum1(t < K ? y[t] * __ldg(M.invW + t) : 0.0, w.red);
    const double Wbar = 1.0 / sYW;
    const double rho = P * Wbar / (kRu * T);
    mx.Wbar = Wbar;
    mx.rho = rho;
    mx.Ctot = P / (kRu * T);
    mx.lnPRT = log(kPatm / (kRu * T));
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // Y_in H/RT/W, Y c_p/R/W, Y_in c_p/R/W, Y dc_p/R/W, H/RT wdot
    if (t < K) {
        const double Yj = y[t];
        double cpR, hRT, sR, dcpR;
        nasa7(M.nasa, t, T, lnT, invT, cpR, hRT, sR, dcpR);
        const double invW = __ldg(M.invW + t);
        w.C[t] = rho * Yj * invW;
        w.hRT[t] = hRT;
        w.gS[t] = sR - hRT;
        w.cpR[t] = cpR;
        w.dcpR[t] = dcpR;
        const double yin = Yin[t];
        acc[0] = yin * hRT * invW;
        acc[1] = Yj * cpR * invW;
        acc[2] = yin * cpR * invW;
        acc[3] = Yj * dcpR * invW;
    } else if (t == K) {
        w.C[K] = 1.0;
        w.hRT[K] = 0.0;
        w.gS[K] = 0.0;
    }
    __syncthreads();
    // rates of progress, Eqs. (5)-(9): elementary reactions [0, tb_first)
    const int nE = M.tb_first;
    for (int i = t; i < nE; i += kBT) {
        const int16_t *sl6 = M.slots + size_t(i) * 6;
        const int s0 = __ldg(sl6), s1 = __ldg(sl6 + 1), s2 = __ldg(sl6 + 2), s3 = __ldg(sl6 + 3),
                  s4 = __ldg(sl6 + 4), s5 = __ldg(sl6 + 5);
        const double a = __ldg(M.lnA + i) + __ldg(M.beta + i) * lnT - __ldg(M.theta + i) * invT;
        const double lnKc = (w.gS[s3] + w.gS[s4] + w.gS[s5]) - (w.gS[s0] + w.gS[s1] + w.gS[s2]) +
                            __ldg(M.dnu_d + i) * mx.lnPRT;
        const double kf = exp(a), kr = exp(a - lnKc);
        double q = kf * (w.C[s0] * w.C[s1] * w.C[s2]) - kr * (w.C[s3] * w.C[s4] * w.C[s5]);
        if (mult) q *= __ldg(mult + __ldg(M.orig + i));
        w.kf[i] = kf;
        w.kr[i] = kr;
        w.q[i] = q;
    }
    // third-body and falloff reactions [tb_first, I)
    for (int i = nE + t; i < I; i += kBT) {
        const int16_t *sl6 = M.slots + size_t(i) * 6;
        const int s0 = __ldg(sl6), s1 = __ldg(sl6 + 1), s2 = __ldg(sl6 + 2), s3 = __ldg(sl6 + 3),
                  s4 = __ldg(sl6 + 4), s5 = __ldg(sl6 + 5);
        const double a = __ldg(M.lnA + i) + __ldg(M.beta + i) * lnT - __ldg(M.theta + i) * invT;
        const double lnKc = (w.gS[s3] + w.gS[s4] + w.gS[s5]) - (w.gS[s0] + w.gS[s1] + w.gS[s2]) +
                            __ldg(M.dnu_d + i) * mx.lnPRT;
        double kf = exp(a), kr = exp(a - lnKc);
        const int typ = __ldg(M.type + i);
        double Mc = mx.Ctot;
        for (int e = __ldg(M.eff_ptr + i); e < __ldg(M.eff_ptr + i + 1); ++e)
            Mc += __ldg(M.eff_val + e) * w.C[__ldg(M.eff_sp + e)];
        if (typ == kTroe) {
            const int tr = __ldg(M.troe_row + i);
            Troe tt = troe_eval(M.troe + size_t(tr) * 8, a, Mc, T, lnT, invT, true);
            kf *= tt.fac;
            kr *= tt.fac;
            const double dlkf = __ldg(M.beta + i) * invT + __ldg(M.theta + i) * invT * invT;
            w.tD[tr] = tt.D;
            w.tX[tr] = tt.D * (tt.dlk0 - dlkf) + tt.dlnF_dT;
        }
        w.kf[i] = kf;
        w.kr[i] = kr;
        double q = kf * (w.C[s0] * w.C[s1] * w.C[s2]) - kr * (w.C[s3] * w.C[s4] * w.C[s5]);
        if (typ == kThirdBody) q *= Mc;
        if (mult) q *= __ldg(mult + __ldg(M.orig + i));
        w.q[i] = q;
    }
    __syncthreads();
    // Eq. (4) and the species residuals of Eq. (2); wdot_k is left in v[] for the Jacobian
    const double tau_rho = tau / rho;
    if (t < K) {
        double w0 = 0.0, w1 = 0.0;
        int e = __ldg(M.sp_ptr + t);
        const int e_end = __ldg(M.sp_ptr + t + 1);
        for (; e + 1 < e_end; e += 2) {
            w0 += __ldg(M.sp_nu_d + e) * w.q[__ldg(M.sp_rxn + e)];
            w1 += __ldg(M.sp_nu_d + e + 1) * w.q[__ldg(M.sp_rxn + e + 1)];
        }
        if (e < e_end) w0 += __ldg(M.sp_nu_d + e) * w.q[__ldg(M.sp_rxn + e)];
        const double wd = w0 + w1;
        F[t] = y[t] - Yin[t] - tau_rho * __ldg(M.W + t) * wd;
        acc[4] = w.hRT[t] * wd;
        w.v[t] = wd;
    }
    bsum<5>(acc, w.red);
    const double RT = kRu * T;
    const double cp = acc[1] * kRu;
    const double N = acc[0] * RT - mx.h_in + tau_rho * RT * acc[4];
    mx.N = N;
    mx.cp = cp;
    mx.sum_yin_cp = acc[2] * kRu;
    mx.sum_y_dcp = acc[3] * kRu;
    if (t == K) F[K] = (energy == PSR_FIXED_T) ? (T - Tspec) : N / (cp * T);
    __syncthreads();
}

// ---------------------------------------------------------------- Jacobian
// Analytic dF/dx at the state of the last b_eval_F, plus diag(c), into w.J: per-reaction
// concentration-Jacobian blocks (shared-memory atomics), a dense third-body part per
// column, Euler sums and T-derivatives per species, the transform to (Y, T) and the
// energy row of Eq. (3). Same chain and precision as the warp solver's Jacobian.
// The per-reaction pass of the block Jacobian in FP64 (also the FP32 Jacobian's fallback
// where K + 1 exceeds the FP32 scratch, 2 kRedSlots kBW floats): see the warp solver's jac_reactions for the quantities.
template <class TJ>
__device__ void b_jac_reactions_f64(const DevMech &M, const BWS<TJ> &w, const Mix &mx,
                                    const double *__restrict__ mult) {
    const int t = threadIdx.x;
    const int K = M.K, I = M.I, P = w.P;
    const double invT = mx.invT;
    for (int i = t; i < I; i += kBT) {
        const int16_t *sl6 = M.slots + size_t(i) * 6;
        int s[6];
        double cs[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            s[u] = __ldg(sl6 + u);
            cs[u] = w.C[s[u]];
        }
        const double Pf = cs[0] * cs[1] * cs[2], Pr_ = cs[3] * cs[4] * cs[5];
        const double d0 = cs[1] * cs[2], d1 = cs[0] * cs[2], d2 = cs[0] * cs[1];
        const double d3 = cs[4] * cs[5], d4 = cs[3] * cs[5], d5 = cs[3] * cs[4];
        const double kf = w.kf[i], kr = w.kr[i];
        const double m = mult ? __ldg(mult + __ldg(M.orig + i)) : 1.0;
        const int typ = __ldg(M.type + i);
        double Mc = 1.0;
        if (typ != kElem) {
            Mc = mx.Ctot;
            for (int e = __ldg(M.eff_ptr + i); e < __ldg(M.eff_ptr + i + 1); ++e)
                Mc += __ldg(M.eff_val + e) * w.C[__ldg(M.eff_sp + e)];
        }
        const double sM = (typ == kThirdBody) ? Mc : 1.0;
        const double dlkf = __ldg(M.beta + i) * invT + __ldg(M.theta + i) * invT * invT;
        const double dlKc = ((w.hRT[s[3]] + w.hRT[s[4]] + w.hRT[s[5]]) - (w.hRT[s[0]] + w.hRT[s[1]] + w.hRT[s[2]]) -
                             __ldg(M.dnu_d + i)) * invT;
        double dlkfe = dlkf, dqdM = 0.0;
        if (typ == kThirdBody) {
            dqdM = m * (kf * Pf - kr * Pr_);
        } else if (typ == kTroe) {
            const int tr = __ldg(M.troe_row + i);
            dlkfe = dlkf + w.tX[tr];
            dqdM = m * (kf * Pf - kr * Pr_) * w.tD[tr] / Mc;
        }
        const double dlkre = dlkfe - dlKc;
        const double Af = m * sM * kf, Ar = m * sM * kr;
        const int nf = (s[0] < K) + (s[1] < K) + (s[2] < K), nr = (s[3] < K) + (s[4] < K) + (s[5] < K);
        double g = Af * nf * Pf - Ar * nr * Pr_;
        if (typ != kElem) g += dqdM * Mc;
        const double dqdT = Af * Pf * dlkfe - Ar * Pr_ * dlkre;
        const int16_t *pp = M.part + size_t(i) * 6;
        const int8_t *pn = M.part_nu + size_t(i) * 6;
        const int8_t *pfm = M.part_fm + size_t(i) * 6;
        const int8_t *prm = M.part_rm + size_t(i) * 6;
        int pl[6];
        TJ pnu[6], val[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            pl[u] = __ldg(pp + u);
            pnu[u] = TJ(__ldg(pn + u));
            const int fm = __ldg(pfm + u), rm = __ldg(prm + u);
            const double dfl = slot_deriv(fm, d0, d1, d2);
            const double drl = slot_deriv(rm, d3, d4, d5);
            val[u] = TJ(Af * dfl - Ar * drl);
        }
        const TJ dqdM_t = TJ(dqdM);
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            if (pl[r] >= K || pnu[r] == TJ(0)) continue;
            TJ *row = w.J + size_t(pl[r]) * P;
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                if (pl[u] >= K) continue;
                atomicAdd(row + pl[u], pnu[r] * val[u]);
            }
            if (typ != kElem) {
                atomicAdd(w.v + pl[r], double(pnu[r]) * dqdM);
                for (int e = __ldg(M.eff_ptr + i); e < __ldg(M.eff_ptr + i + 1); ++e)
                    atomicAdd(row + __ldg(M.eff_sp + e), pnu[r] * dqdM_t * eff_v<TJ>(M, e));
            }
        }
        w.q[i] = g;       // per-reaction Euler sum
        w.kf[i] = dqdT;   // and T-derivative replace q and kf
    }
}

// The same pass with FP32 arithmetic for the FP32 Jacobian (the pieces only steer Newton;
// FP64 instructions are the scarce resource): FP32 copies of the concentrations in the
// reduction scratch (free during the pass, K + 1 <= 2 kRedSlots kBW), the dense third-body part
// accumulated in FP32 in rhs (free until the energy row), ln K_c's T-derivative from the
// FP64 H/RT. g_i and d q_i / dT are stored in FP64 for the species sums.
template <class TJ>
__device__ void b_jac_reactions_f32(const DevMech &M, const BWS<TJ> &w, const Mix &mx,
                                    const double *__restrict__ mult) {
    const int t = threadIdx.x;
    const int K = M.K, I = M.I, P = w.P;
    float *Cf = reinterpret_cast<float *>(w.red);
    float *vf = reinterpret_cast<float *>(w.rhs);
    if (t <= K) Cf[t] = float(w.C[t]);
    if (t < K) vf[t] = 0.0f;
    __syncthreads();
    const double invT = mx.invT;
    const float invTf = float(invT), Ctot = float(mx.Ctot);
    for (int i = t; i < I; i += kBT) {
        const int16_t *sl6 = M.slots + size_t(i) * 6;
        int s[6];
        float cs[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            s[u] = __ldg(sl6 + u);
            cs[u] = Cf[s[u]];
        }
        const float Pf = cs[0] * cs[1] * cs[2], Pr_ = cs[3] * cs[4] * cs[5];
        const float d0 = cs[1] * cs[2], d1 = cs[0] * cs[2], d2 = cs[0] * cs[1];
        const float d3 = cs[4] * cs[5], d4 = cs[3] * cs[5], d5 = cs[3] * cs[4];
        const float kf = float(w.kf[i]), kr = float(w.kr[i]);
        const float m = mult ? float(__ldg(mult + __ldg(M.orig + i))) : 1.0f;
        const int typ = __ldg(M.type + i);
        float Mc = 1.0f;
        if (typ != kElem) {
            Mc = Ctot;
            for (int e = __ldg(M.eff_ptr + i); e < __ldg(M.eff_ptr + i + 1); ++e)
                Mc += __ldg(M.eff_val_f + e) * Cf[__ldg(M.eff_sp + e)];
        }
        const float sM = (typ == kThirdBody) ? Mc : 1.0f;
        const float dlkf = __ldg(M.beta_f + i) * invTf + __ldg(M.theta_f + i) * invTf * invTf;
        const float dlKc = float(((w.hRT[s[3]] + w.hRT[s[4]] + w.hRT[s[5]]) - (w.hRT[s[0]] + w.hRT[s[1]] + w.hRT[s[2]]) -
                                  __ldg(M.dnu_d + i)) * invT);
        float dlkfe = dlkf, dqdM = 0.0f;
        if (typ == kThirdBody) {
            dqdM = m * (kf * Pf - kr * Pr_);
        } else if (typ == kTroe) {
            const int tr = __ldg(M.troe_row + i);
            dlkfe = dlkf + float(w.tX[tr]);
            dqdM = m * (kf * Pf - kr * Pr_) * float(w.tD[tr]) / Mc;
        }
        const float dlkre = dlkfe - dlKc;
        const float Af = m * sM * kf, Ar = m * sM * kr;
        const int nf = (s[0] < K) + (s[1] < K) + (s[2] < K), nr = (s[3] < K) + (s[4] < K) + (s[5] < K);
        float g = Af * float(nf) * Pf - Ar * float(nr) * Pr_;
        if (typ != kElem) g += dqdM * Mc;
        const float dqdT = Af * Pf * dlkfe - Ar * Pr_ * dlkre;
        const int16_t *pp = M.part + size_t(i) * 6;
        const int8_t *pn = M.part_nu + size_t(i) * 6;
        const int8_t *pfm = M.part_fm + size_t(i) * 6;
        const int8_t *prm = M.part_rm + size_t(i) * 6;
        int pl[6];
        TJ pnu[6], val[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            pl[u] = __ldg(pp + u);
            pnu[u] = TJ(__ldg(pn + u));
            const int fm = __ldg(pfm + u), rm = __ldg(prm + u);
            const float dfl = slot_deriv_f(fm, d0, d1, d2);
            const float drl = slot_deriv_f(rm, d3, d4, d5);
            val[u] = TJ(Af * dfl - Ar * drl);
        }
        const TJ dqdM_t = TJ(dqdM);
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            if (pl[r] >= K || pnu[r] == TJ(0)) continue;
            TJ *row = w.J + size_t(pl[r]) * P;
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                if (pl[u] >= K) continue;
                atomicAdd(row + pl[u], pnu[r] * val[u]);
            }
            if (typ != kElem) {
                atomicAdd(vf + pl[r], float(pnu[r]) * dqdM);
                for (int e = __ldg(M.eff_ptr + i); e < __ldg(M.eff_ptr + i + 1); ++e)
                    atomicAdd(row + __ldg(M.eff_sp + e), pnu[r] * dqdM_t * eff_v<TJ>(M, e));
            }
        }
        w.q[i] = double(g);
        w.kf[i] = double(dqdT);
    }
}


template <class TJ>
__device__ void b_eval_J(const DevMech &M, const BWS<TJ> &w, const double *c, const Mix &mx, double tau,
                         int energy, const double *__restrict__ mult) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int K = M.K, I = M.I, n = K + 1, P = w.P;
    __syncthreads();
    const double wd = (t < K) ? w.v[t] : 0.0;
    __syncthreads();
    for (size_t idx = t; idx < size_t(n) * P; idx += kBT) w.J[idx] = TJ(0);
    if (t < K) w.v[t] = 0.0;
    __syncthreads();
    const double T = mx.T, invT = mx.invT;
    if constexpr (sizeof(TJ) == 4) {
        if (K + 1 <= kRedSlots * kBW * 2) {
            b_jac_reactions_f32(M, w, mx, mult);
        } else {
            b_jac_reactions_f64(M, w, mx, mult);
        }
    } else {
        b_jac_reactions_f64(M, w, mx, mult);
    }
    __syncthreads();
    double sk = 0.0, wT = 0.0, vk = 0.0;
    if (t < K) {
        for (int e = __ldg(M.sp_ptr + t); e < __ldg(M.sp_ptr + t + 1); ++e) {
            const double nu = __ldg(M.sp_nu_d + e);
            const int r = __ldg(M.sp_rxn + e);
            sk += nu * w.q[r];
            wT += nu * w.kf[r];
        }
        if constexpr (sizeof(TJ) == 4) {
            vk = (K + 1 <= kRedSlots * kBW * 2) ? double(reinterpret_cast<const float *>(w.rhs)[t]) : w.v[t];
        } else {
            vk = w.v[t];
        }
        w.v[t] = vk;   // the row transform below reads it per row (warps over rows)
    }
    const double rho = mx.rho, Wbar = mx.Wbar, RT = kRu * T;
    double eJ = 0.0;
    if (energy != PSR_FIXED_T) {
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // Q, Sh, Hv, cw, hwT
        if (t < K) w.rhs[t] = TJ(w.hRT[t]);          // H/RT in the Jacobian's precision (column sums)
        if (t < K) {
            const double H = w.hRT[t] * RT;
            acc[0] = H * wd;
            acc[1] = H * sk;
            acc[2] = H * vk;
            acc[3] = w.cpR[t] * kRu * wd;
            acc[4] = H * (wT - sk * invT);
        }
        bsum<5>(acc, w.red);
        const double Q = acc[0], Sh = acc[1], Hv = acc[2], cw = acc[3], hwT = acc[4];
        const double N = mx.N, cp = mx.cp;
        const double inv_cpT = 1.0 / (cp * T);
        if (t < K) {
            TJ colsum = TJ(0);
            for (int k = 0; k < K; ++k) colsum += w.rhs[k] * w.J[size_t(k) * P + t];
            const double cs = double(colsum) * RT + Hv;
            const double invWj = __ldg(M.invW + t);
            const double dN = tau * invWj * (cs + Wbar * (Q - Sh) / rho);
            const double cpj = w.cpR[t] * kRu * invWj;
            eJ = dN * inv_cpT - N * cpj * inv_cpT / cp;
        } else if (t == K) {
            const double dNdT = mx.sum_yin_cp + tau / rho * (cw + hwT) + tau * Q / (rho * T);
            eJ = dNdT * inv_cpT - N * mx.sum_y_dcp * inv_cpT / cp - N * inv_cpT * invT;
        }
    }
    if (t < K) {
        const double Wk = __ldg(M.W + t);
        w.ra[t] = tau * Wk;
        w.rb[t] = tau * Wk * Wbar * (sk - wd) / rho;
        // column K (untouched by the reaction pass) of species row t
        w.J[size_t(t) * P + K] = TJ(-(tau * Wk / rho) * (wT + (wd - sk) * invT));
    }
    __syncthreads();   // column sums read J before the transform rewrites it
    // species rows: dF_k/dY_j = delta_kj - tau W_k (Jc_kj + v_k)/W_j + tau W_k Wbar (s_k - wdot_k)/(rho W_j)
    for (int k = wid; k < K; k += kBW) {
        const TJ ak = TJ(w.ra[k]), bk = TJ(w.rb[k]), vkt = TJ(w.v[k]);
        TJ *row = w.J + size_t(k) * P;
        for (int j = lane; j < K; j += 32) {
            const TJ invWj = inv_w<TJ>(M, j);
            row[j] = (bk - ak * (row[j] + vkt)) * invWj + ((j == k) ? TJ(1) : TJ(0));
        }
    }
    if (t < n) {
        const double v = (energy == PSR_FIXED_T) ? ((t == K) ? 1.0 : 0.0) : eJ;
        w.J[size_t(K) * P + t] = TJ(v);
    }
    __syncthreads();
    if (t < n) w.J[size_t(t) * P + t] = TJ(double(w.J[size_t(t) * P + t]) + c[t]);
    __syncthreads();
}


// ---------------------------------------------------------------- LU (partial pivoting)
// Candidate for the next pivot: largest |a| by integer key, ties to the lower row (a NaN
// ranks first and then fails the factorisation).
template <class TJ>
__device__ __forceinline__ void pivot_candidate(TJ v, int row, unsigned long long &best, TJ &bv, int &bi) {
    const unsigned long long a = abs_key(v);
    if (a > best || (a == best && row < bi)) {
        best = a;
        bv = v;
        bi = row;
    }
}

template <class TJ>
__device__ __forceinline__ void warp_argmax(unsigned long long &best, TJ &bv, int &bi) {
    using Key = decltype(abs_key(TJ(0)));
    const int win = warp_argmax_row(Key(best), bi);               // hardware integer reductions
    const int src = __ffs(__ballot_sync(kFull, bi == win)) - 1;    // the lane holding that row
    best = __shfl_sync(kFull, best, src);
    bv = __shfl_sync(kFull, bv, src);
    bi = win;
}

constexpr int kNB = 32;                  // panel width of the blocked LU
constexpr int kTB = 4;                   // trailing-update tile per thread: rows w + kBW a (a < TA), columns l + 32 b
template <class TJ>
struct TileRows {
    static constexpr int value = sizeof(TJ) == 8 ? 4 : 8;
};

// Blocked right-looking LU with partial pivoting (the LAPACK getrf order: panel,
// row interchanges, triangular solve for the U block row, rank-32 trailing update), in
// place in w.J; perm = final row order. The panel is factored column by column with one
// thread per row (two block barriers per column: pivot offers, then the interchange);
// U12 = L11^-1 A12 takes one thread per column; A22 -= L21 U12 runs as a register-tiled
// product (8 x 4 outputs per thread, 12 shared loads per 32 FMAs). False on a zero or
// non-finite pivot (block-uniform).
template <class TJ>
__device__ __noinline__ bool b_lu(const BWS<TJ> &w, int n, bool tc_ok = true) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int P = w.P;
    TJ *J = w.J;
    unsigned long long *ckey = reinterpret_cast<unsigned long long *>(w.red);   // [2][kBW] pivot offers,
    TJ *cval = reinterpret_cast<TJ *>(w.red + 2 * kBW);                        // double-buffered
    int *crow = w.ired;
    if (t < n) w.perm[t] = int16_t(t);
    int buf = 0;
    for (int k0 = 0; k0 < n; k0 += kNB) {
        const int kb = min(kNB, n - k0);
        const int i = k0 + t;   // the panel row this thread owns
        {
            unsigned long long best = 0;
            TJ bv = TJ(0);
            int bi = n;
            if (i < n) pivot_candidate(J[size_t(i) * P + k0], i, best, bv, bi);
            warp_argmax(best, bv, bi);
            if (lane == 0) {
                ckey[buf + wid] = best;
                cval[buf + wid] = bv;
                crow[buf + wid] = bi;
            }
        }
        for (int c = 0; c < kb; ++c) {
            const int k = k0 + c;
            __syncthreads();   // offers for column k are written, the previous step's rows updated
            unsigned long long best = ckey[buf];
            TJ pv = cval[buf];
            int p = crow[buf];
#pragma unroll
            for (int u = 1; u < kBW; ++u) {
                const unsigned long long ob = ckey[buf + u];
                const int oi = crow[buf + u];
                if (ob > best || (ob == best && oi < p)) {
                    best = ob;
                    pv = cval[buf + u];
                    p = oi;
                }
            }
            if (!key_is_finite_nonzero(abs_key(pv)) || p >= n) return false;
            if (p != k) {
                for (int j = t; j < n; j += kBT) {
                    const TJ tmp = J[size_t(k) * P + j];
                    J[size_t(k) * P + j] = J[size_t(p) * P + j];
                    J[size_t(p) * P + j] = tmp;
                }
                if (t == 0) {
                    const int16_t tp = w.perm[k];
                    w.perm[k] = w.perm[p];
                    w.perm[p] = tp;
                }
            }
            __syncthreads();   // pivot row in place
            buf = kBW - buf;
            const TJ inv = TJ(1.0) / pv;
            unsigned long long nb_best = 0;
            TJ nb_v = TJ(0);
            int nb_i = n;
            if (i > k && i < n) {
                TJ *ri = J + size_t(i) * P;
                const TJ *rk = J + size_t(k) * P;
                const TJ l = ri[k] * inv;
                ri[k] = l;
                for (int cc = k + 1; cc < k0 + kb; ++cc) ri[cc] = fma(-l, rk[cc], ri[cc]);
                if (c + 1 < kb) pivot_candidate(ri[k + 1], i, nb_best, nb_v, nb_i);
            }
            if (c + 1 < kb) {
                warp_argmax(nb_best, nb_v, nb_i);
                if (lane == 0) {
                    ckey[buf + wid] = nb_best;
                    cval[buf + wid] = nb_v;
                    crow[buf + wid] = nb_i;
                }
            }
        }
        const int r0 = k0 + kb;   // first row / column of the trailing matrix
        if (r0 >= n) break;
        __syncthreads();   // panel factored
        // U12 = L11^-1 A12: one column per thread, forward substitution down the kb rows
        {
            const int j = r0 + t;
            if (j < n) {
                for (int r = 1; r < kb; ++r) {
                    const TJ *Lr = J + size_t(k0 + r) * P + k0;
                    TJ s0 = J[size_t(k0 + r) * P + j], s1 = TJ(0);
                    int c = 0;
                    for (; c + 1 < r; c += 2) {
                        s0 = fma(-Lr[c], J[size_t(k0 + c) * P + j], s0);
                        s1 = fma(-Lr[c + 1], J[size_t(k0 + c + 1) * P + j], s1);
                    }
                    if (c < r) s0 = fma(-Lr[c], J[size_t(k0 + c) * P + j], s0);
                    J[size_t(k0 + r) * P + j] = s0 + s1;
                }
            }
        }
        __syncthreads();
        const int m = n - r0;
        if constexpr (sizeof(TJ) == 4) {
            // A22 -= L21 U12 on the tensor cores (FP32 Jacobian, large trailing matrices)
            if (w.tc && tc_ok && m >= kTcMinM && !w.ired[2 * kBW + 2]) {
                if (!b_trailing_tc(w, n, r0, k0, kb)) return false;
                continue;
            }
        }
        // A22 -= L21 U12 in chunks of (kBW TA) x (32 TB): warp w takes rows w, w + kBW, ..
        constexpr int kTA = TileRows<TJ>::value;
        for (int rb = 0; rb < m; rb += kBW * kTA) {
            for (int cb = 0; cb < m; cb += 32 * kTB) {
                TJ acc[kTA][kTB];
#pragma unroll
                for (int a = 0; a < kTA; ++a)
#pragma unroll
                    for (int b = 0; b < kTB; ++b) acc[a][b] = TJ(0);
                const int row0 = r0 + rb + wid, col0 = r0 + cb + lane;
                for (int c = 0; c < kb; ++c) {
                    TJ lv[kTA], uv[kTB];
#pragma unroll
                    for (int a = 0; a < kTA; ++a) {
                        const int row = row0 + kBW * a;
                        lv[a] = (row < n) ? J[size_t(row) * P + k0 + c] : TJ(0);
                    }
#pragma unroll
                    for (int b = 0; b < kTB; ++b) {
                        const int col = col0 + 32 * b;
                        uv[b] = (col < n) ? J[size_t(k0 + c) * P + col] : TJ(0);
                    }
#pragma unroll
                    for (int a = 0; a < kTA; ++a)
#pragma unroll
                        for (int b = 0; b < kTB; ++b) acc[a][b] = fma(lv[a], uv[b], acc[a][b]);
                }
#pragma unroll
                for (int a = 0; a < kTA; ++a) {
                    const int row = row0 + kBW * a;
                    if (row < n) {
#pragma unroll
                        for (int b = 0; b < kTB; ++b) {
                            const int col = col0 + 32 * b;
                            if (col < n) J[size_t(row) * P + col] -= acc[a][b];
                        }
                    }
                }
            }
        }
        __syncthreads();   // trailing matrix updated before the next panel reads it
    }
    __syncthreads();
    return true;
}

// x = -(LU)^-1 r (r, x shared vectors of length n). Blocked substitutions: warp 0 solves
// each 32 x 32 diagonal block with the unknowns in registers (shuffles), then every thread
// updates one remaining row with that block's 32 unknowns.
template <class TJ>
__device__ void b_lu_solve_neg(const BWS<TJ> &w, int n, const double *r, double *x) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int P = w.P;
    __syncthreads();   // r complete
    if (t < n) w.rhs[t] = TJ(-r[w.perm[t]]);
    __syncthreads();
    const int nb = (n + 31) / 32;
    // forward: unit lower
    for (int b = 0; b < nb; ++b) {
        const int r0 = b * 32, r1 = min(n, r0 + 32);
        if (wid == 0) {
            const int i = r0 + lane;
            TJ xi = (i < r1) ? w.rhs[i] : TJ(0);
            for (int c = r0; c < r1 - 1; ++c) {
                const TJ xc = __shfl_sync(kFull, xi, c - r0);
                if (i > c && i < r1) xi = fma(-w.J[size_t(i) * P + c], xc, xi);
            }
            if (i < r1) w.rhs[i] = xi;
        }
        __syncthreads();
        for (int i = r1 + t; i < n; i += kBT) {
            const TJ *Li = w.J + size_t(i) * P;
            TJ s = w.rhs[i];
            for (int c = r0; c < r1; ++c) s = fma(-Li[c], w.rhs[c], s);
            w.rhs[i] = s;
        }
        __syncthreads();
    }
    // backward: upper
    for (int b = nb - 1; b >= 0; --b) {
        const int r0 = b * 32, r1 = min(n, r0 + 32);
        if (wid == 0) {
            const int i = r0 + lane;
            TJ xi = (i < r1) ? w.rhs[i] : TJ(0);
            for (int c = r1 - 1; c >= r0; --c) {
                const TJ own = (i == c) ? xi / w.J[size_t(c) * P + c] : xi;
                const TJ xc = __shfl_sync(kFull, own, c - r0);
                if (i == c) xi = xc;
                else if (i < c) xi = fma(-w.J[size_t(i) * P + c], xc, xi);
            }
            if (i < r1) w.rhs[i] = xi;
        }
        __syncthreads();
        for (int i = t; i < r0; i += kBT) {
            const TJ *Ui = w.J + size_t(i) * P;
            TJ s = w.rhs[i];
            for (int c = r0; c < r1; ++c) s = fma(-Ui[c], w.rhs[c], s);
            w.rhs[i] = s;
        }
        __syncthreads();
    }
    if (t < n) x[t] = double(w.rhs[t]);
    __syncthreads();
}

// J^T lam = g with the factors of P J = L U (U^T forward, L^T backward, lam[perm[j]] = v_j).
template <class TJ>
__device__ void b_lu_solve_T(const BWS<TJ> &w, int n, const double *g, double *lam) {
    const int t = threadIdx.x;
    const int P = w.P;
    __syncthreads();
    if (t < n) w.rhs[t] = TJ(g[t]);
    __syncthreads();
    if (t < 32) {
        const int lane = t;
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
    }
    __syncthreads();
    if (t < n) lam[w.perm[t]] = double(w.rhs[t]);
    __syncthreads();
}

// ---------------------------------------------------------------- solver pieces
struct BCtx {
    DevMech M;
    Opts o;
    const double *Yin;
    double tau, P, Tspec;
    const double *mult;
    int nfev;
    Mix mx;
    int K, n;
    double fn;   // ||F||_inf of the last residual (kept only with the tensor-core LU)
};

// With the TF32 tensor-core LU (one TF32 product, 2^-11 rounding) Newton converges only
// linearly near the root, and the polish test on the last step (which assumes fast
// convergence) would leave minor species a few 1e-6 off: the last iterations, from
// ||F||_inf <= kTcSwitchF on, factor on the CUDA cores in FP32.
constexpr double kTcSwitchF = 1e-6;

__device__ __forceinline__ bool b_all_finite(const double *v, int n) {
    const int t = threadIdx.x;
    return __syncthreads_and(t >= n || isfinite(v[t])) != 0;
}

// mass fractions absolute, temperature relative
__device__ __forceinline__ double b_scaled_max(const double *dy, const double *y, int K, int n, double *red) {
    const int t = threadIdx.x;
    double d = 0.0;
    if (t < n) {
        d = fabs(dy[t]);
        if (t == K) d /= fabs(y[t]);
    }
    return bmax(d, red);
}

__device__ __forceinline__ bool b_in_bounds(const double *y, int K, const Opts &o) {
    const int t = threadIdx.x;
    bool ok = true;
    if (t < K) ok = y[t] >= -o.y_floor;
    else if (t == K) ok = y[t] >= o.t_min && y[t] <= o.t_max;
    return __syncthreads_and(ok) != 0;
}

__device__ __forceinline__ double b_max_in_bounds(const double *y, const double *dy, int K, const Opts &o,
                                                  double *red) {
    const int t = threadIdx.x;
    double lam = INFINITY;
    if (t <= K) {
        const double x = y[t], d = dy[t];
        const double lo = (t < K) ? -o.y_floor : o.t_min, hi = (t < K) ? INFINITY : o.t_max;
        if (d < 0 && x + d < lo) lam = (lo - x) / d;
        else if (d > 0 && x + d > hi) lam = (hi - x) / d;
    }
    return bmin(lam, red);
}

// |dx_j| <= rtol |x_j| + atol_j (atol_y for species, atol_t for temperature)
__device__ __forceinline__ bool b_step_small(const double *dy, const double *y, int K, int n, double rtol,
                                             double atol_y, double atol_t) {
    const int t = threadIdx.x;
    bool ok = true;
    if (t < n) ok = fabs(dy[t]) <= rtol * fabs(y[t]) + ((t < K) ? atol_y : atol_t);
    return __syncthreads_and(ok) != 0;
}

template <class TJ>
__device__ void b_residual_R(BCtx &cx, const BWS<TJ> &w, const double *y, const double *c, const double *xref,
                             double *F, double *R) {
    ++cx.nfev;
    b_eval_F(cx.M, w, y, F, cx.mx, cx.Yin, cx.tau, cx.P, cx.Tspec, cx.o.energy, cx.mult);
    const int t = threadIdx.x;
    if (t < cx.n) R[t] = F[t] + c[t] * (y[t] - xref[t]);
    if (w.tc == 1) cx.fn = bmax(t < cx.n ? fabs(F[t]) : 0.0, w.red);
    __syncthreads();
}

// Damped Newton on R(y) = F(y) + c (y - xref) from y (y updated in place), the scheme of
// the warp solver: natural-monotonicity damping with the same LU factors, divergence
// stop, bounds; steady mode converges on ||R||_inf <= ftol plus a small last step.
template <class TJ>
__device__ bool b_damped_newton(BCtx &cx, const BWS<TJ> &w, double *y, const double *xref, const double *c,
                                int max_it, bool steady, int &counter, double *fnorm) {
    const int t = threadIdx.x;
    const int K = cx.K, n = cx.n;
    const Opts &o = cx.o;
    b_residual_R(cx, w, y, c, xref, w.F, w.R);
    // ||F||_inf of the steady residual at the first and the last evaluated point
    if (fnorm) fnorm[0] = fnorm[1] = bmax(t < n ? fabs(w.F[t]) : 0.0, w.red);
    double dn_prev = INFINITY;
    // Jacobian reuse (o.jac_age > 1), as in the warp solver
    bool have_lu = false, at_y = true;
    int age = 0;
    for (int it = 0; it < max_it; ++it) {
        if (counter >= o.max_newton) break;
        ++counter;
        bool fresh = false;
        if (!have_lu || age + 1 >= o.jac_age) {
            if (!at_y) {   // the last residual was a rejected trial: the Jacobian needs y's caches
                b_residual_R(cx, w, y, c, xref, w.F, w.R);
                if (fnorm) fnorm[1] = bmax(t < n ? fabs(w.F[t]) : 0.0, w.red);
                at_y = true;
            }
            b_eval_J(cx.M, w, c, cx.mx, cx.tau, o.energy, cx.mult);
            if (!b_lu(w, n, cx.fn > kTcSwitchF)) break;
            have_lu = true;
            age = 0;
            fresh = true;
        } else {
            ++age;
        }
        b_lu_solve_neg(w, n, w.R, w.dy);
        if (!b_all_finite(w.dy, n)) {
            if (!fresh) {
                have_lu = false;
                continue;
            }
            break;
        }
        bool done;
        if (steady) {
            const double rmax = bmax(t < n ? fabs(w.R[t]) : 0.0, w.red);
            done = rmax <= o.ftol && b_step_small(w.dy, y, K, n, o.step_rtol, o.step_atol_y, o.step_atol_t);
        } else {
            done = b_step_small(w.dy, y, K, n, o.ts_rtol, o.ts_atol_y, o.ts_rtol);
        }
        if (done) {
            if (t < n) y[t] += w.dy[t];
            __syncthreads();
            return true;
        }
        const double dn = b_scaled_max(w.dy, y, K, n, w.red);
        if (dn >= dn_prev) {
            if (!fresh) {
                have_lu = false;
                continue;
            }
            break;
        }
        double lam = fmin(1.0, b_max_in_bounds(y, w.dy, K, o, w.red));
        bool accepted = false;
        for (int d = 0; d < o.max_damp; ++d) {
            if (t < n) w.yt[t] = y[t] + lam * w.dy[t];
            __syncthreads();
            if (b_in_bounds(w.yt, K, o)) {
                b_residual_R(cx, w, w.yt, c, xref, w.F, w.Rt);
                at_y = false;
                if (fnorm) fnorm[1] = bmax(t < n ? fabs(w.F[t]) : 0.0, w.red);
                if (b_all_finite(w.Rt, n)) {
                    b_lu_solve_neg(w, n, w.Rt, w.db);
                    if (b_scaled_max(w.db, y, K, n, w.red) < dn) {
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
        if (t < n) {
            y[t] = w.yt[t];
            w.R[t] = w.Rt[t];
        }
        __syncthreads();
        at_y = true;
        if (lam < 1.0) have_lu = false;   // a damped step: fresh factors next
    }
    return false;
}
// One linearised backward-Euler step from x (w.x) with the diagonal shift in w.c, the
// warp solver's linear_step: (J(x) + diag c) dx = -F(x), the full step taken when it stays
// in bounds and F stays finite. fx_valid: w.F holds F(x) and the caches are x's.
template <class TJ>
__device__ bool b_linear_step(BCtx &cx, const BWS<TJ> &w, int &counter, bool &fx_valid, double &f_new) {
    const int t = threadIdx.x;
    const int K = cx.K, n = cx.n;
    const Opts &o = cx.o;
    if (counter >= o.max_newton) return false;
    ++counter;
    if (!fx_valid) b_residual_R(cx, w, w.x, w.c, w.x, w.F, w.R);
    fx_valid = false;   // the Jacobian consumes the rate caches
    b_eval_J(cx.M, w, w.c, cx.mx, cx.tau, o.energy, cx.mult);
    if (!b_lu(w, n, cx.fn > kTcSwitchF)) return false;
    b_lu_solve_neg(w, n, w.F, w.dy);
    if (!b_all_finite(w.dy, n)) return false;
    if (b_max_in_bounds(w.x, w.dy, K, o, w.red) < 1.0) return false;
    if (t < n) w.yt[t] = w.x[t] + w.dy[t];
    __syncthreads();
    if (!b_in_bounds(w.yt, K, o)) return false;
    b_residual_R(cx, w, w.yt, w.c, w.yt, w.Rt, w.db);
    if (!b_all_finite(w.Rt, n)) return false;
    f_new = bmax(t < n ? fabs(w.Rt[t]) : 0.0, w.red);
    if (t < n) {
        w.x[t] = w.yt[t];
        w.F[t] = w.Rt[t];
    }
    __syncthreads();
    fx_valid = true;
    return true;
}


__device__ void b_inlet_enthalpy(BCtx &cx, double Tin, double *red) {
    const int t = threadIdx.x;
    const double lnTin = log(Tin);
    double s = 0.0;
    if (t < cx.K) {
        double cpR, hRT, sR, dcpR;
        nasa7(cx.M.nasa, t, Tin, lnTin, 1.0 / Tin, cpR, hRT, sR, dcpR);
        s = cx.Yin[t] * hRT * __ldg(cx.M.invW + t);
    }
    cx.mx.h_in = bsum1(s, red) * kRu * Tin;
}

// Loads reactor r's inlet and starting point; returns true for a reactor a warp launch
// handed over unfinished (it continues from the iterate left in Y_out / T_out).
template <class TJ>
__device__ bool b_load_reactor(BCtx &cx, const BWS<TJ> &w, const Batch &bt, int64_t r) {
    const int t = threadIdx.x;
    const int K = cx.K;
    const int64_t row = row_of(bt, r, K);
    cx.Yin = bt.Y_in + row;
    cx.tau = bt.tau[r];
    cx.P = bt.P[r];
    cx.Tspec = bt.T0[r];
    cx.nfev = 0;
    b_inlet_enthalpy(cx, bt.T_in[r], w.red);
    // a reactor the warp launch handed over continues from the iterate it left in the outputs
    const bool cont = bt.fallback && bt.status && bt.status[r] == kStatusHandoff;
    const double *Ys = cont ? bt.Y_out : bt.Y0;
    const double *Ts = cont ? bt.T_out : bt.T0;
    if (t < cx.n) {
        w.x[t] = (t < K) ? Ys[row + t] : Ts[r];
        w.c[t] = 0.0;
    }
    __syncthreads();
    return cont;
}

template <class TJ>
__device__ void b_solve_one(BCtx &cx, const BWS<TJ> &w, const Batch &bt, int64_t r) {
    const int t = threadIdx.x;
    const int K = cx.K, n = cx.n;
    const Opts &o = cx.o;
    // a continued reactor keeps its counters (its Newton budget is the reactor's total)
    const bool cont = b_load_reactor(cx, w, bt, r);
    const double tau = cx.tau;
    if (cont && bt.nfev) cx.nfev = bt.nfev[r];
    b_residual_R(cx, w, w.x, w.c, w.x, w.F, w.R);
    int status, rounds = 0;
    int counter = (cont && bt.iters) ? bt.iters[r] : 0, ts = (cont && bt.ts_steps) ? bt.ts_steps[r] : 0;
    const double *out = w.x;
    if (!b_all_finite(w.F, n)) {
        status = PSR_NONFINITE;
    } else {
        double dt = o.dt0_over_tau * tau;
        while (true) {
            if (t < n) {
                w.y[t] = w.x[t];
                w.c[t] = 0.0;
            }
            __syncthreads();
            double fn[2];
            const bool conv = b_damped_newton(cx, w, w.y, w.x, w.c, o.max_newton, true, counter, fn);
            if (conv) {
                status = PSR_CONVERGED;
                out = w.y;
                break;
            }
            if (counter >= o.max_newton) {
                status = PSR_MAX_ITER;
                out = w.y;
                break;
            }
            ++rounds;
            if (rounds > o.max_ts_rounds) {
                status = PSR_TS_EXHAUSTED;
                out = w.x;
                break;
            }
            int taken = 0;
            bool done = false;
            double f_prev = fn[0];   // ||F(x)||_inf of the estimate being conditioned
            bool fx_valid = false;   // the steady attempt left the caches elsewhere
            while (taken < o.ts_steps) {
                const double Tx = w.x[K];
                const double s = tau / dt;
                const double sT = (o.energy == PSR_FIXED_T) ? s : s / Tx;
                __syncthreads();   // every thread has read x[K]
                if (t < n) {
                    w.c[t] = (t < K) ? s : sT;
                    w.y[t] = w.x[t];
                }
                __syncthreads();
                const int used0 = counter;
                double f_new = 0.0;
                bool ok;
                const bool linear = counter < o.ts_linear;
                if (linear) {
                    ok = b_linear_step(cx, w, counter, fx_valid, f_new);   // updates w.x itself
                } else {
                    double fs[2];
                    ok = b_damped_newton(cx, w, w.y, w.x, w.c, o.ts_newton, false, counter, fs);
                    f_new = fs[1];
                    if (ok) {
                        if (t < n) w.x[t] = w.y[t];
                        __syncthreads();
                    }
                }
                const int used = counter - used0;
                if (counter >= o.max_newton) {
                    status = PSR_MAX_ITER;
                    out = w.x;
                    done = true;
                    break;
                }
                if (ok) {
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
                        out = w.x;
                        done = true;
                        break;
                    }
                }
            }
            if (done) break;
        }
    }
    // report ||F||_inf at the output state
    if (t < n) w.c[t] = 0.0;
    __syncthreads();
    b_residual_R(cx, w, out, w.c, out, w.F, w.R);
    const double fn = bmax(t < n ? fabs(w.F[t]) : 0.0, w.red);
    if (t < K) bt.Y_out[row_of(bt, r, K) + t] = out[t];
    if (t == 0) {
        bt.T_out[r] = out[K];
        const bool add = bt.fallback != 0 && !cont;   // a restart adds its counters to the first launch's
        if (bt.status) bt.status[r] = (bt.fallback == 1 && status == PSR_CONVERGED) ? PSR_REFINE_FALLBACK : status;
        if (bt.iters) bt.iters[r] = counter + (add ? bt.iters[r] : 0);
        if (bt.ts_steps) bt.ts_steps[r] = ts + (add ? bt.ts_steps[r] : 0);
        if (bt.fnorm) bt.fnorm[r] = fn;
        if (bt.nfev) bt.nfev[r] = cx.nfev + (add ? bt.nfev[r] : 0);
    }
    __syncthreads();
}

}  // namespace
}  // namespace PSR_BLOCK_NS
}  // namespace psr
