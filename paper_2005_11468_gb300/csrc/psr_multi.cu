// One persistent launch for a batch of reactors of several gas mechanisms
// (psr_batch_solve_multi): every thread block takes reactors from class-ordered work
// queues until all are empty, so the classes share the GPU without a per-class launch.
//
// The method is the hybrid damped Newton / pseudo-transient scheme of Sec. 3 on the
// residual of Eqs. (2)-(3), as in the one-mechanism solvers; this file only schedules it.
// A block of kMT = 256 threads runs three phases:
//   1. block-solver classes (K + 1 > 64, or every class when the block path is forced), in
//      order of decreasing K: the whole block takes one reactor at a time from a single
//      atomic counter over the concatenated class lists, so the longest solves start first;
//      in the mixed form an FP64 re-solve already listed (below) is taken before the next
//      first-pass reactor;
//   2. warp-solver classes, again largest K first: each warp with a shared-memory slice
//      takes reactors from a second counter;
//   3. mixed form only: the FP64 re-solve of reactors the FP32-Jacobian passes left
//      unconverged (warp-solver classes continued from the FP32 iterate, then restarted from
//      the initial guess where that fails; block-solver classes restarted), one block per
//      reactor. Phases 1-2 append such reactors to a list as they finish, so blocks re-solve
//      them while others are still busy, instead of a second launch after the slowest
//      first-pass reactor.
//
// The wait in phase 3 (for a list entry, or for the end of the first pass) is bounded by
// psr_options.spin_limit polls about 1 us apart; a block that gives up sets the error word
// and leaves its entry unsolved (its status stays the FP32 pass's failure). Every producer
// it waits for is a reactor already being solved by a resident warp or block, so the wait
// ends when that reactor does.
//
// Built once per first-pass Jacobian precision: PSR_MULTI_TJ (float | double) and the name
// of the host entry, PSR_MULTI_ENTRY, come from the build.
#if !defined(PSR_MULTI_TJ) || !defined(PSR_MULTI_ENTRY)
#error "psr_multi.cu needs PSR_MULTI_TJ and PSR_MULTI_ENTRY"
#endif
#ifndef PSR_MULTI_MINB
#define PSR_MULTI_MINB 1   // resident blocks per SM the kernel is compiled for (register cap)
#endif
#define PSR_BLOCK_THREADS 256
#include "psr_block.cuh"
#include "psr_warp.cuh"

namespace psr {
namespace {

namespace blk = PSR_BLOCK_NS;
constexpr int kMT = blk::kBT;        // threads per block of the persistent kernel
constexpr int kMW = kMT / 32;        // warps per block
constexpr int kMaxClasses = 8;
constexpr int kMinB = PSR_MULTI_MINB;

// One class of the batch, in queue order.
struct MultiClass {
    DevMech M;
    int ci;            // index of the class's list in the bucketed lists
    int j_smem;        // first pass: the Jacobian in shared memory (block classes)
    int j_smem64;      // FP64 re-solve (mixed form): the FP64 Jacobian in shared memory
};

// Control words (zeroed before the launch) and the re-solve list (filled with -1).
enum : int { kQB = 0, kQW = 1, kQF = 2, kNF = 3, kDone = 4, kErr = 5, kCtlInts = 8 };

struct MultiArgs {
    MultiClass cls[kMaxClasses];
    int n_cls, n_block;                 // classes [0, n_block) run on the block solver
    const int32_t *counts, *lists;      // bucketed: class ci has counts[ci] reactors at lists + ci B
    int64_t B;
    int fb_passes;                      // mixed form: 2 continue then restart, 1 restart, 0 none
    long long spin_limit;               // polls of the phase-3 wait
    size_t ws_per_warp;                 // phase 2 shared-memory slice per warp
    int warps_active;                   // warps of a block with a slice
    char *jglob;                        // global Jacobian slots, jslot bytes per block
    size_t jslot;
    int *ctl;                           // kCtlInts control words
    unsigned long long *relist;         // [B] re-solve entries: (class << 32) | reactor, or ~0
};

// Reactor p of the concatenation of classes [c0, c1): class index and reactor, or -1.
__device__ __forceinline__ int locate(const MultiArgs &a, const int *cnt, int c0, int c1, int p, int64_t &r) {
    for (int c = c0; c < c1; ++c) {
        if (p < cnt[c]) {
            r = int64_t(a.lists[int64_t(a.cls[c].ci) * a.B + p]);
            return c;
        }
        p -= cnt[c];
    }
    return -1;
}

// The end of reactor r's first pass (one thread): mixed form, unconverged -> re-solve list.
__device__ __forceinline__ void first_pass_done(const MultiArgs &a, const Batch &bt, int c, int64_t r) {
    if (a.fb_passes > 0 && bt.status[r] != PSR_CONVERGED) {
        const int idx = atomicAdd(a.ctl + kNF, 1);
        atomicExch(a.relist + idx, (static_cast<unsigned long long>(c) << 32) | static_cast<unsigned long long>(r));
        __threadfence();
    }
    atomicAdd(a.ctl + kDone, 1);
}

// Phase 3 claim (thread 0): the next re-solve entry, or ~0 once the first pass is over and
// no entry is left for this claim (or the wait gave up).
__device__ unsigned long long claim_resolve(const MultiArgs &a, int total) {
    const int p = atomicAdd(a.ctl + kQF, 1);
    if (p >= total) return ~0ull;
    volatile unsigned long long *slot = a.relist + p;
    volatile int *done = a.ctl + kDone;
    for (long long it = 0; it < a.spin_limit; ++it) {
        unsigned long long v = *slot;
        if (v != ~0ull) return v;
        if (*done >= total) {
            __threadfence();
            return *slot;   // every producer published its entry before counting itself done
        }
        __nanosleep(1000);
    }
    atomicExch(a.ctl + kErr, 1);
    return ~0ull;
}

// Claim without waiting (thread 0): a re-solve entry some producer has already reserved
// (it publishes it right after), or ~0 when none is reserved beyond the claims so far.
__device__ unsigned long long try_claim_resolve(const MultiArgs &a) {
    volatile int *qf = a.ctl + kQF, *nf = a.ctl + kNF;
    while (true) {
        const int cur = *qf;
        if (cur >= *nf) return ~0ull;
        if (atomicCAS(a.ctl + kQF, cur, cur + 1) != cur) continue;   // another block took it
        volatile unsigned long long *slot = a.relist + cur;
        for (long long it = 0; it < a.spin_limit; ++it) {
            const unsigned long long v = *slot;
            if (v != ~0ull) return v;
            __nanosleep(100);
        }
        atomicExch(a.ctl + kErr, 1);
        return ~0ull;
    }
}

// FP64 re-solve (mixed form) of re-solve entry v, one block: warp-solver reactors that the
// FP32 pass stopped at its iteration cap are first continued from its final iterate, then
// restarted from the initial guess where that fails; the others (block-solver classes, and
// reactors whose FP32 pass ended in exhausted pseudo-time stepping, an iterate the FP64
// continuation almost never finishes) are restarted at once, as the per-mechanism launches do.
__device__ void resolve_fp64(const MultiArgs &a, const Batch &bt, blk::BCtx &cx, char *smem,
                             unsigned long long v) {
    const int c = int(v >> 32);
    const int64_t r = int64_t(v & 0xffffffffull);
    const DevMech &M = a.cls[c].M;
    cx.M = M;
    cx.K = M.K;
    cx.n = M.K + 1;
    double *Jg = a.cls[c].j_smem64 ? nullptr : reinterpret_cast<double *>(a.jglob + blockIdx.x * a.jslot);
    const blk::BWS<double> w = blk::bcarve<double>(smem, M.K, M.I, M.n_troe, M.K + 1, Jg, 0);
    Batch b2 = bt;
    b2.fallback = 1;   // counters add up; success reports PSR_REFINE_FALLBACK
    if (a.fb_passes == 2 && c >= a.n_block && bt.status[r] == PSR_MAX_ITER) {
        // continued from the FP32 pass's final iterate (read before it is overwritten)
        Batch bc = b2;
        bc.Y0 = bt.Y_out;
        if (cx.o.energy != PSR_FIXED_T) bc.T0 = bt.T_out;   // else T0 is the specified temperature
        blk::b_solve_one<double>(cx, w, bc, r);
        const int32_t s = bt.status[r];   // written by thread 0 before the solver's last barrier
        if (s == PSR_CONVERGED || s == PSR_REFINE_FALLBACK) return;
    }
    blk::b_solve_one<double>(cx, w, b2, r);   // restarted from the initial guess
}

template <class TJ>
__global__ void __launch_bounds__(kMT, kMinB) multi_solve_kernel(MultiArgs a, Batch bt, Opts o1, Opts o) {
    extern __shared__ __align__(128) char smem[];
    __shared__ int s_cnt[kMaxClasses];
    __shared__ unsigned long long s_claim;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t < a.n_cls) s_cnt[t] = a.counts[a.cls[t].ci];
    __syncthreads();
    int total = 0, nB = 0;
    for (int c = 0; c < a.n_cls; ++c) {
        total += s_cnt[c];
        if (c < a.n_block) nB += s_cnt[c];
    }
    blk::BCtx cx64;   // the FP64 re-solves (mixed form)
    cx64.o = o;
    cx64.mult = bt.rate_mult;
    cx64.fn = INFINITY;
    constexpr unsigned long long kFirst = 1ull << 63;   // tags a first-pass claim
    // ---- phase 1: block-solver classes, one block per reactor; in the mixed form an FP64
    // re-solve already listed goes first (the longest work starts earliest)
    if (nB > 0) {
        blk::BCtx cx;
        cx.o = o1;
        cx.mult = bt.rate_mult;
        cx.fn = INFINITY;
        while (true) {
            if (t == 0) {
                unsigned long long v = ~0ull;
                if (sizeof(TJ) == 4 && a.fb_passes > 0) v = try_claim_resolve(a);
                if (v == ~0ull) v = kFirst | static_cast<unsigned long long>(atomicAdd(a.ctl + kQB, 1));
                s_claim = v;
            }
            __syncthreads();
            const unsigned long long v = s_claim;
            __syncthreads();
            if constexpr (sizeof(TJ) == 4) {
                if (!(v & kFirst)) {
                    resolve_fp64(a, bt, cx64, smem, v);
                    continue;
                }
            }
            int64_t r = 0;
            const int c = locate(a, s_cnt, 0, a.n_block, int(v & 0x7fffffffull), r);
            if (c < 0) break;
            const DevMech &M = a.cls[c].M;
            cx.M = M;
            cx.K = M.K;
            cx.n = M.K + 1;
            TJ *Jg = a.cls[c].j_smem ? nullptr : reinterpret_cast<TJ *>(a.jglob + blockIdx.x * a.jslot);
            const blk::BWS<TJ> w = blk::bcarve<TJ>(smem, M.K, M.I, M.n_troe, M.K + 1, Jg, 0);
            blk::b_solve_one<TJ>(cx, w, bt, r);
            if (t == 0) first_pass_done(a, bt, c, r);
        }
    }
    // ---- phase 2: warp-solver classes, one warp per reactor
    if (warp < a.warps_active && a.n_block < a.n_cls) {
        char *base = smem + size_t(warp) * a.ws_per_warp;
        Ctx cx;
        cx.o = o1;
        cx.mult = bt.rate_mult;
        cx.idle = a.ctl + kErr;   // never consulted: handoff_at = 0
        cx.handoff_at = 0;
        while (true) {
            int p = 0;
            if (lane == 0) p = atomicAdd(a.ctl + kQW, 1);
            p = __shfl_sync(kFull, p, 0);
            int64_t r = 0;
            const int c = locate(a, s_cnt, a.n_block, a.n_cls, p, r);
            if (c < 0) break;
            const DevMech &M = a.cls[c].M;
            cx.M = M;
            cx.K = M.K;
            cx.n = M.K + 1;
            const WS<TJ> w = carve<TJ>(base, M.K, M.I, M.K + 1, M.n_troe, 0);
            solve_one<TJ, false, false>(cx, w, bt, r);
            if (lane == 0) first_pass_done(a, bt, c, r);
            __syncwarp();
        }
    }
    __syncthreads();
    // ---- phase 3 (mixed form): FP64 re-solve of the reactors the first pass left
    if constexpr (sizeof(TJ) == 4) {
        if (a.fb_passes <= 0) return;
        while (true) {
            if (t == 0) s_claim = claim_resolve(a, total);
            __syncthreads();
            const unsigned long long v = s_claim;
            __syncthreads();
            if (v == ~0ull) break;
            resolve_fp64(a, bt, cx64, smem, v);
        }
    }
}

// Host side of the persistent launch. Returns PSR_E_UNSUPPORTED (without launching)
// when the batch needs what this kernel leaves out: soot moments, the finite-difference
// Jacobian, the tensor-core LU, or a class with K + 1 > kMT on the block solver.
template <class TJ>
int multi_launch(const Mech *const *ms, const int32_t *class_of, int n_cls, int n_block, const int32_t *counts,
                 const int32_t *lists, const Batch &bt, const Opts &o, const Opts &o1, int fb_passes,
                 long long spin_limit, cudaStream_t st) {
    if (n_cls < 1 || n_cls > kMaxClasses) return set_error(PSR_E_ARG, "persistent launch: 1..8 classes");
    if (o.jac_fd || o.lu_tc) return set_error(PSR_E_UNSUPPORTED, "persistent launch: analytic Jacobian, CUDA-core LU");
    constexpr bool mixed = sizeof(TJ) == 4;
    const void *kern = reinterpret_cast<const void *>(&multi_solve_kernel<TJ>);
    int dev = 0, max_smem = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return cuda_error("cudaFuncGetAttributes", e);
    max_smem -= int(fa.sharedSizeBytes);   // the kernel's static shared memory
    MultiArgs a{};
    a.n_cls = n_cls;
    a.n_block = n_block;
    a.counts = counts;
    a.lists = lists;
    a.B = bt.B;
    a.fb_passes = mixed ? fb_passes : 0;
    a.spin_limit = spin_limit;
    size_t smem = 0, wsw = 0, jslot = 0;
    const size_t tj = mixed ? sizeof(float) : sizeof(double);
    for (int k = 0; k < n_cls; ++k) {
        const Mech &m = *ms[k];
        if (m.dev.nsoot) return set_error(PSR_E_UNSUPPORTED, "persistent launch: gas mechanisms only");
        const int K = m.K, n = K + 1;
        MultiClass &c = a.cls[k];
        c.M = m.dev;
        c.ci = class_of[k];
        const size_t slot_tj = tj * size_t(n) * blk::pitch_of(n), slot64 = 8 * size_t(n) * blk::pitch_of(n);
        if (k < n_block) {
            if (n > kMT) return set_error(PSR_E_UNSUPPORTED, "persistent launch: block classes need K + 1 <= 256");
            const size_t with_j = mixed ? blk::bws_bytes<float>(K, m.I, m.n_troe, n, true)
                                        : blk::bws_bytes<double>(K, m.I, m.n_troe, n, true);
            const size_t no_j = mixed ? blk::bws_bytes<float>(K, m.I, m.n_troe, n, false)
                                      : blk::bws_bytes<double>(K, m.I, m.n_troe, n, false);
            c.j_smem = with_j <= size_t(max_smem);
            smem = std::max(smem, c.j_smem ? with_j : no_j);
            if (!c.j_smem) jslot = std::max(jslot, slot_tj);
        } else {
            c.j_smem = 0;
            wsw = std::max(wsw, mixed ? ws_bytes<float>(K, m.I, n, m.n_troe) : ws_bytes<double>(K, m.I, n, m.n_troe));
        }
        c.j_smem64 = 0;
        if (a.fb_passes > 0) {
            if (n > kMT) return set_error(PSR_E_UNSUPPORTED, "persistent launch: FP64 re-solve needs K + 1 <= 256");
            const size_t with_j = blk::bws_bytes<double>(K, m.I, m.n_troe, n, true);
            c.j_smem64 = with_j <= size_t(max_smem);
            smem = std::max(smem, c.j_smem64 ? with_j : blk::bws_bytes<double>(K, m.I, m.n_troe, n, false));
            if (!c.j_smem64) jslot = std::max(jslot, slot64);
        }
    }
    if (smem > size_t(max_smem)) return set_error(PSR_E_UNSUPPORTED, "persistent launch: tables exceed shared memory");
    if (wsw) {
        wsw = (wsw + 127) & ~size_t(127);
        if (wsw > size_t(max_smem)) return set_error(PSR_E_UNSUPPORTED, "persistent launch: warp workspace too large");
        // warp slices: kMW of them, or as many as fit with kMinB blocks per SM, at least one;
        // a block whose other phases need more shared memory gives its warps slices of that
        int sm_total = 0;
        cudaDeviceGetAttribute(&sm_total, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        const size_t share = std::min<size_t>(size_t(max_smem), size_t(sm_total) / kMinB - 1024 - fa.sharedSizeBytes);
        smem = std::max(smem, std::max(wsw, std::min(size_t(kMW) * wsw, share / wsw * wsw)));
        a.warps_active = int(std::min<size_t>(kMW, smem / wsw));
    }
    a.ws_per_warp = wsw;
    jslot = (jslot + 255) & ~size_t(255);   // every block's slot aligned for FP64 and FP32 alike
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return cuda_error("cudaFuncSetAttribute", e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMT, smem);
    if (e != cudaSuccess) return cuda_error("occupancy", e);
    if (per_sm < 1) return set_error(PSR_E_UNSUPPORTED, "persistent kernel does not fit on an SM");
    const int grid = per_sm * nsm;
    // control words, the re-solve list and the global Jacobian slots in one allocation
    const size_t list_bytes = a.fb_passes > 0 ? sizeof(unsigned long long) * size_t(bt.B) : 0;
    const size_t ctl_bytes = 256, jg_off = ctl_bytes + ((list_bytes + 255) & ~size_t(255));
    const size_t bytes = jg_off + jslot * size_t(grid);
    char *scr = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void **>(&scr), bytes, st);
    if (e != cudaSuccess) return set_error(PSR_E_OOM, "persistent launch: scratch");
    a.ctl = reinterpret_cast<int *>(scr);
    a.relist = reinterpret_cast<unsigned long long *>(scr + ctl_bytes);
    a.jglob = jslot ? scr + jg_off : nullptr;
    a.jslot = jslot;
    e = cudaMemsetAsync(scr, 0, ctl_bytes, st);
    if (e == cudaSuccess && list_bytes) e = cudaMemsetAsync(scr + ctl_bytes, 0xff, list_bytes, st);
    if (e == cudaSuccess) {
        multi_solve_kernel<TJ><<<grid, kMT, smem, st>>>(a, bt, o1, o);
        e = cudaGetLastError();
    }
    cudaFreeAsync(scr, st);
    if (e != cudaSuccess) return cuda_error("multi_solve_kernel launch", e);
    return PSR_OK;
}

}  // namespace

int PSR_MULTI_ENTRY(const Mech *const *ms, const int32_t *class_of, int n_cls, int n_block, const int32_t *counts,
                    const int32_t *lists, const Batch &bt, const Opts &o, const Opts &o1, int fb_passes,
                    long long spin_limit, cudaStream_t st) {
    return multi_launch<PSR_MULTI_TJ>(ms, class_of, n_cls, n_block, counts, lists, bt, o, o1, fb_passes, spin_limit,
                                      st);
}

}  // namespace psr
