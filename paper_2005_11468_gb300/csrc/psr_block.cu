// Kernels and host launchers of the block-per-reactor solver (device code in
// psr_block.cuh), built once per block size in the namespace psr_block.cuh selects.
#include "psr_block.cuh"

namespace psr {
namespace PSR_BLOCK_NS {
namespace {

// ---------------------------------------------------------------- kernels
template <class TJ>
__global__ void __launch_bounds__(kBT, 512 / kBT) block_solve_kernel(DevMech M, Batch bt, Opts o, int *queue, TJ *Jglob) {
    extern __shared__ __align__(128) char smem[];
    const int K = M.K, n = K + 1;
    const size_t slot = size_t(n) * pitch_of(n);
    const int tc = (sizeof(TJ) == 4 && n >= kTcMinM + kNB) ? o.lu_tc : 0;
    BWS<TJ> w = bcarve<TJ>(smem, K, M.I, M.n_troe, n, Jglob ? Jglob + blockIdx.x * slot : nullptr, tc);
    tc_begin(w);
    BCtx cx;
    cx.M = M;
    cx.o = o;
    cx.mult = bt.rate_mult;
    cx.K = K;
    cx.n = n;
    cx.fn = INFINITY;   // 3xTF32 (w.tc == 3) never switches
    const int64_t nwork = bt.list ? int64_t(*bt.list_len) : bt.B;
    while (true) {
        if (threadIdx.x == 0) w.ired[2 * kBW] = atomicAdd(queue, 1);
        __syncthreads();
        const int p = w.ired[2 * kBW];
        __syncthreads();
        if (p >= nwork) break;
        const int64_t r = bt.list ? int64_t(bt.list[p]) : int64_t(p);
        b_solve_one<TJ>(cx, w, bt, r);
    }
    tc_end(w);
}

__global__ void block_collect_unconverged(int64_t B, const int32_t *in_list, const int32_t *in_len,
                                          const int32_t *status, int32_t *list, int32_t *len) {
    const int64_t n = in_list ? int64_t(*in_len) : B;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = in_list ? int64_t(in_list[p]) : p;
        if (status[r] != PSR_CONVERGED) list[atomicAdd(len, 1)] = int32_t(r);
    }
}

// residual or Jacobian at given states, one block per state (grid-stride over states)
template <class TJ>
__global__ void __launch_bounds__(kBT, 512 / kBT) block_eval_kernel(DevMech M, Batch bt, int energy, int want_J,
                                                            double *out, RatesOut ro, TJ *Jglob) {
    extern __shared__ __align__(128) char smem[];
    const int K = M.K, n = K + 1;
    const size_t slot = size_t(n) * pitch_of(n);
    BWS<TJ> w = bcarve<TJ>(smem, K, M.I, M.n_troe, n, Jglob ? Jglob + blockIdx.x * slot : nullptr);
    BCtx cx;
    cx.M = M;
    cx.o.energy = energy;
    cx.mult = bt.rate_mult;
    cx.K = K;
    cx.n = n;
    const int t = threadIdx.x;
    for (int64_t r = blockIdx.x; r < bt.B; r += gridDim.x) {
        b_load_reactor(cx, w, bt, r);
        b_residual_R(cx, w, w.x, w.c, w.x, w.F, w.R);
        if (want_J == 2) {   // rates of the residual just evaluated: effective kf, kr, q_i, wdot_k
            for (int i = t; i < M.I; i += kBT) {
                const int64_t o = r * M.I + __ldg(M.orig + i);
                if (ro.kf) ro.kf[o] = w.kf[i];
                if (ro.kr) ro.kr[o] = w.kr[i];
                if (ro.q) ro.q[o] = w.q[i];
            }
            if (ro.wdot && t < K) ro.wdot[r * K + t] = w.v[t];
            __syncthreads();
            continue;
        }
        if (!want_J) {
            if (t < n) out[r * n + t] = w.F[t];
            continue;
        }
        b_eval_J(M, w, w.c, cx.mx, cx.tau, energy, cx.mult);
        for (int idx = t; idx < n * n; idx += kBT)
            out[r * n * n + idx] = double(w.J[size_t(idx / n) * w.P + idx % n]);
        __syncthreads();
    }
}

// Adjoint sensitivities at given (converged) states (the warp solver's formula):
// J^T lam = g with the FP64 factors, then
// dL/d ln m_i = (tau q_i / rho) [sum_k lam_k W_k nu_ki - lam_T dH_i / (c_p T)].
__global__ void __launch_bounds__(kBT, 512 / kBT) block_adjoint_kernel(DevMech M, Batch bt, int energy, const double *g,
                                                               double *grad, double *lam_out, int32_t *ok,
                                                               double *Jglob) {
    extern __shared__ __align__(128) char smem[];
    const int K = M.K, n = K + 1, I = M.I;
    const size_t slot = size_t(n) * pitch_of(n);
    BWS<double> w = bcarve<double>(smem, K, I, M.n_troe, n, Jglob ? Jglob + blockIdx.x * slot : nullptr);
    BCtx cx;
    cx.M = M;
    cx.o.energy = energy;
    cx.mult = bt.rate_mult;
    cx.K = K;
    cx.n = n;
    const int t = threadIdx.x;
    for (int64_t r = blockIdx.x; r < bt.B; r += gridDim.x) {
        b_load_reactor(cx, w, bt, r);
        b_residual_R(cx, w, w.x, w.c, w.x, w.F, w.R);
        b_eval_J(M, w, w.c, cx.mx, cx.tau, energy, cx.mult);
        const bool good = b_lu(w, n);
        if (t < n) {
            w.dy[t] = 0.0;
            w.db[t] = g[r * n + t];
        }
        __syncthreads();
        if (good) b_lu_solve_T(w, n, w.db, w.dy);   // lam in dy
        // the Jacobian pass replaced q_i: evaluate the residual once more to restore it
        b_residual_R(cx, w, w.x, w.c, w.x, w.F, w.R);
        if (lam_out && t < n) lam_out[r * n + t] = w.dy[t];
        const double lamT = w.dy[K];
        if (t < K) w.v[t] = w.dy[t] * __ldg(M.W + t);
        __syncthreads();
        const double tau_rho = cx.tau / cx.mx.rho;
        const double eT = (energy == PSR_FIXED_T) ? 0.0 : lamT * kRu * cx.mx.T / (cx.mx.cp * cx.mx.T);
        for (int i = t; i < I; i += kBT) {
            const int16_t *pp = M.part + size_t(i) * 6;
            const int8_t *pn = M.part_nu + size_t(i) * 6;
            double lw = 0.0, dH = 0.0;
            for (int u = 0; u < 6; ++u) {
                const int l = __ldg(pp + u);
                if (l >= K) continue;
                const double nu = double(__ldg(pn + u));
                lw += nu * w.v[l];
                dH += nu * w.hRT[l];
            }
            grad[r * I + __ldg(M.orig + i)] = good ? tau_rho * w.q[i] * (lw - eT * dH) : 0.0;
        }
        if (ok && t == 0) ok[r] = good ? 1 : 0;
        __syncthreads();
    }
}

template <class TJ>
__global__ void __launch_bounds__(kBT, 512 / kBT) block_lu_kernel(int64_t B, int n, const double *A, const double *rhs,
                                                          double *x, int32_t *ok, TJ *Jglob, int tc) {
    extern __shared__ __align__(128) char smem[];
    const size_t slot = size_t(n) * pitch_of(n);
    BWS<TJ> w = bcarve<TJ>(smem, 0, 0, 0, n, Jglob ? Jglob + blockIdx.x * slot : nullptr, tc);
    tc_begin(w);
    const int t = threadIdx.x;
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        for (int idx = t; idx < n * n; idx += kBT) w.J[size_t(idx / n) * w.P + idx % n] = TJ(A[b * n * n + idx]);
        if (t < n) w.R[t] = -rhs[b * n + t];
        __syncthreads();
        const bool good = b_lu(w, n);
        if (good) b_lu_solve_neg(w, n, w.R, w.dy);
        if (t < n) x[b * n + t] = good ? w.dy[t] : 0.0;
        if (t == 0) ok[b] = good ? 1 : 0;
        __syncthreads();
    }
    tc_end(w);
}

// ---------------------------------------------------------------- host side
struct Launch {
    size_t smem = 0;
    bool j_in_smem = false;
    int grid = 0;
};

// Shared-memory plan of one block for a kernel: the Jacobian in shared memory when the
// whole workspace fits, else in global slots (one per block).
template <class TJ, class KernelT>
int plan(KernelT kern, int K, int I, int nt, int n, int64_t units, int bps_req, Launch &L, bool tc = false) {
    int dev = 0, max_smem = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t with_j = bws_bytes<TJ>(K, I, nt, n, true, tc);
    L.j_in_smem = with_j <= size_t(max_smem);
    L.smem = L.j_in_smem ? with_j : bws_bytes<TJ>(K, I, nt, n, false, tc);
    if (L.smem > size_t(max_smem))
        return set_error(PSR_E_UNSUPPORTED, "mechanism tables exceed one block's shared memory");
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L.smem));
    if (e != cudaSuccess) return cuda_error("cudaFuncSetAttribute", e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBT, L.smem);
    if (e != cudaSuccess) return cuda_error("occupancy", e);
    if (per_sm < 1) return set_error(PSR_E_UNSUPPORTED, "block solver kernel does not fit on an SM");
    if (bps_req > 0 && bps_req < per_sm) per_sm = bps_req;
    L.grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(per_sm) * nsm, units)));
    return PSR_OK;
}

template <class TJ>
int launch_block(const Mech &m, const Batch &bt, const Opts &o, int bps_req, cudaStream_t st, int *queue) {
    const int K = m.K, n = K + 1;
    Launch L;
    const bool tc = sizeof(TJ) == 4 && n >= kTcMinM + kNB && o.lu_tc > 0;
    int rc = plan<TJ>(block_solve_kernel<TJ>, K, m.I, m.n_troe, n, bt.B, bps_req, L, tc);
    if (rc) return rc;
    TJ *Jg = nullptr;
    cudaError_t e;
    if (!L.j_in_smem) {
        e = cudaMallocAsync(reinterpret_cast<void **>(&Jg), sizeof(TJ) * size_t(n) * pitch_of(n) * L.grid, st);
        if (e != cudaSuccess) return set_error(PSR_E_OOM, "Jacobian slots for the block solver");
    }
    e = cudaMemsetAsync(queue, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        block_solve_kernel<TJ><<<L.grid, kBT, L.smem, st>>>(m.dev, bt, o, queue, Jg);
        e = cudaGetLastError();
    }
    if (Jg) cudaFreeAsync(Jg, st);
    if (e != cudaSuccess) return cuda_error("block_solve_kernel launch", e);
    return PSR_OK;
}

}  // namespace

// Second launch over the reactors a warp-solver launch listed (bt.list), one block per
// reactor, with the FP64 or the FP32 Jacobian: the mixed form's FP64 re-solve, or the
// continuation of reactors handed over unfinished. A short list would leave the GPU almost
// idle under the warp solver, where one reactor takes a warp for all of its iterations.
int block_resolve_list(const Mech &m, const Batch &bt, const Opts &o, int precision, cudaStream_t st, int *queue) {
    return precision == PSR_MIXED ? launch_block<float>(m, bt, o, 0, st, queue)
                                  : launch_block<double>(m, bt, o, 0, st, queue);
}

int block_check(const Mech &m) {
    if (m.dev.nsoot) return set_error(PSR_E_UNSUPPORTED, "soot moments need K + 7 <= 64 (warp solver)");
    if (m.K + 1 > kMaxBlockN)
        return set_error(PSR_E_UNSUPPORTED, "the block solver handles at most " + std::to_string(kMaxBlockN) + " unknowns");
    return PSR_OK;
}

int block_solve(const Mech &m, const Batch &bt, const Opts &o, int precision, bool fallback, int bps_req,
                cudaStream_t st) {
    const size_t B = size_t(bt.B);
    const bool mixed = precision == PSR_MIXED;
    const size_t n_ints = 4 + ((mixed && fallback) ? B + (bt.status ? 0 : B) : 0);
    int32_t *scr = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scr), n_ints * sizeof(int32_t), st);
    if (e != cudaSuccess) return set_error(PSR_E_OOM, "scratch allocation failed");
    int rc;
    if (!mixed) {
        rc = launch_block<double>(m, bt, o, bps_req, st, scr);
    } else if (!fallback) {
        rc = launch_block<float>(m, bt, o, bps_req, st, scr);
    } else {
        // FP32-Jacobian launch, then the reactors it left unconverged again in FP64
        int32_t *len = scr + 2, *list = scr + 4;
        Batch b1 = bt;
        if (!bt.status) b1.status = scr + 4 + B;
        Opts first = o;   // the FP32 launch stops at the mixed_max_newton cap (see the warp solver)
        const int cap = o.mixed_max_newton >= 0 ? o.mixed_max_newton : 300;   // the gas default
        if (cap > 0 && cap < o.max_newton) first.max_newton = cap;
        rc = launch_block<float>(m, b1, first, bps_req, st, scr);
        if (rc == PSR_OK) {
            cudaMemsetAsync(len, 0, sizeof(int32_t), st);
            block_collect_unconverged<<<unsigned((B + 255) / 256), 256, 0, st>>>(bt.B, bt.list, bt.list_len,
                                                                                 b1.status, list, len);
            e = cudaGetLastError();
            if (e != cudaSuccess) rc = cuda_error("block_collect_unconverged launch", e);
        }
        if (rc == PSR_OK) {
            Batch b2 = b1;
            b2.list = list;
            b2.list_len = len;
            b2.fallback = 1;
#if PSR_BLOCK_THREADS == 256
            // The list is a small part of the batch. When the whole batch holds at most 16
            // reactors per SM the list is likely shorter than one 512-thread block per SM, and
            // 512 threads per reactor finish each reactor sooner (K = 200, 2048 reactors: 1.23
            // -> 1.16 s per mixed step); larger batches and class lists keep two 256-thread
            // blocks per SM (the uneven batch's K = 200 class: 2.48 s, 2.56 s with 512 threads).
            int dev = 0, nsm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            if (!bt.list && B <= size_t(16) * size_t(nsm))
                rc = bt512::block_resolve_list(m, b2, o, PSR_FP64, st, scr + 1);
            else
                rc = launch_block<double>(m, b2, o, bps_req, st, scr + 1);
#else
            rc = launch_block<double>(m, b2, o, bps_req, st, scr + 1);
#endif
        }
    }
    cudaFreeAsync(scr, st);
    return rc;
}

template <class TJ>
static int block_eval_t(const Mech &m, const Batch &bt, int energy, int want_J, double *out, cudaStream_t st,
                        RatesOut ro) {
    const int K = m.K, n = K + 1;
    Launch L;
    int rc = plan<TJ>(block_eval_kernel<TJ>, K, m.I, m.n_troe, n, bt.B, 0, L);
    if (rc) return rc;
    TJ *Jg = nullptr;
    cudaError_t e;
    if (!L.j_in_smem) {
        e = cudaMallocAsync(reinterpret_cast<void **>(&Jg), sizeof(TJ) * size_t(n) * pitch_of(n) * L.grid, st);
        if (e != cudaSuccess) return set_error(PSR_E_OOM, "Jacobian slots for the block evaluator");
    }
    block_eval_kernel<TJ><<<L.grid, kBT, L.smem, st>>>(m.dev, bt, energy, want_J, out, ro, Jg);
    e = cudaGetLastError();
    if (Jg) cudaFreeAsync(Jg, st);
    if (e != cudaSuccess) return cuda_error("block_eval_kernel launch", e);
    return PSR_OK;
}

int block_eval(const Mech &m, const Batch &bt, int energy, int want_J, int precision, double *out, cudaStream_t st,
               RatesOut ro) {
    if (precision == PSR_MIXED && want_J == 1) return block_eval_t<float>(m, bt, energy, want_J, out, st, ro);
    return block_eval_t<double>(m, bt, energy, want_J, out, st, ro);
}

int block_adjoint(const Mech &m, const Batch &bt, int energy, const double *g, double *grad, double *lam_out,
                  int32_t *ok, cudaStream_t st) {
    const int K = m.K, n = K + 1;
    Launch L;
    int rc = plan<double>(block_adjoint_kernel, K, m.I, m.n_troe, n, bt.B, 0, L);
    if (rc) return rc;
    double *Jg = nullptr;
    cudaError_t e;
    if (!L.j_in_smem) {
        e = cudaMallocAsync(reinterpret_cast<void **>(&Jg), sizeof(double) * size_t(n) * pitch_of(n) * L.grid, st);
        if (e != cudaSuccess) return set_error(PSR_E_OOM, "Jacobian slots for the block adjoint");
    }
    block_adjoint_kernel<<<L.grid, kBT, L.smem, st>>>(m.dev, bt, energy, g, grad, lam_out, ok, Jg);
    e = cudaGetLastError();
    if (Jg) cudaFreeAsync(Jg, st);
    if (e != cudaSuccess) return cuda_error("block_adjoint_kernel launch", e);
    return PSR_OK;
}

template <class TJ>
static int block_lu_t(int64_t B, int n, const double *A, const double *r, double *x, int32_t *ok, cudaStream_t st,
                      int tc = 0) {
    Launch L;
    if (sizeof(TJ) != 4 || n < kTcMinM + kNB) tc = 0;
    int rc = plan<TJ>(block_lu_kernel<TJ>, 0, 0, 0, n, B, 0, L, tc > 0);
    if (rc) return rc;
    TJ *Jg = nullptr;
    cudaError_t e;
    if (!L.j_in_smem) {
        e = cudaMallocAsync(reinterpret_cast<void **>(&Jg), sizeof(TJ) * size_t(n) * pitch_of(n) * L.grid, st);
        if (e != cudaSuccess) return set_error(PSR_E_OOM, "matrix slots for the block LU");
    }
    block_lu_kernel<TJ><<<L.grid, kBT, L.smem, st>>>(B, n, A, r, x, ok, Jg, tc);
    e = cudaGetLastError();
    if (Jg) cudaFreeAsync(Jg, st);
    if (e != cudaSuccess) return cuda_error("block_lu_kernel launch", e);
    return PSR_OK;
}

// precision: PSR_FP64, PSR_MIXED (FP32), or PSR_MIXED with the tensor-core trailing update
// (lu_tc 1 = TF32, 3 = 3xTF32)
int block_lu(int64_t B, int n, const double *A, const double *r, double *x, int32_t *ok, int precision,
             cudaStream_t st, int lu_tc) {
    if (n > kMaxBlockN) return set_error(PSR_E_ARG, "psr_batch_lu_solve: n > 512");
    return precision == PSR_MIXED ? block_lu_t<float>(B, n, A, r, x, ok, st, lu_tc)
                                  : block_lu_t<double>(B, n, A, r, x, ok, st);
}

}  // namespace PSR_BLOCK_NS
}  // namespace psr
