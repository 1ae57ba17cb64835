// Fifth-generation tensor cores (tcgen05) for the block solver's LU trailing update
// A22 -= L21 U12 (sm_100a / sm_103a): TF32 operands staged in shared memory in the
// canonical no-swizzle K-major layout, the FP32 accumulator in tensor memory, one thread
// issuing the MMAs, completion tracked by an mbarrier with a bounded wait.
//
// Layout of a staged operand tile (R rows x 16 K-elements of 4 bytes): core matrices of
// 8 rows x 16 bytes (4 elements), 128 contiguous bytes each; the 4 core matrices of an
// 8-row group follow one another along K (leading byte offset 128), consecutive 8-row
// groups are 512 bytes apart (stride byte offset). Element (r, k) sits at byte
//   (r / 8) * 512 + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4.
// One MMA of kind::tf32 consumes K = 8 (two core matrices along K); the second K-step of
// a 16-wide tile starts 256 bytes further.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace psr {
namespace tc {

constexpr int kTileM = 128;        // MMA rows (accumulator lanes)
constexpr int kTileK = 16;         // K elements staged per round
constexpr int kGroupBytes = 512;   // one 8-row group of a staged tile: 8 x 16 elements x 4 B
constexpr int kTmemCols = 128;     // accumulator columns allocated per block (N <= 128 per MMA)
constexpr long long kWaitLimit = 1 << 22;   // mbarrier polls before a wait is declared failed

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (r, k) in a staged tile
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
    return uint32_t((r >> 3) * kGroupBytes + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// FP32 -> TF32, round to nearest (ties away), as a float bit pattern
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (8-row group)
// byte offsets, descriptor version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFF) >> 4);
    d |= uint64_t(128 >> 4) << 16;
    d |= uint64_t(kGroupBytes >> 4) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// whole warp: allocate ncols tensor-memory columns, address written to *slot (shared)
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// whole warp (the one that allocated)
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the completion of phase `parity`; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// generic-proxy writes to shared memory made visible to the tensor cores' (async) reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A x B, one thread
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the mbarrier arrives once the MMAs this thread issued before have completed
__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// whole warp: 16 consecutive accumulator columns of the warp's 32 lanes (lane i of the
// warp gets row 32 (warp % 4) + i)
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace psr
