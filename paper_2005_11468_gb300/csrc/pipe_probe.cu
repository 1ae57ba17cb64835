// Pipe-throughput probes (measurement service, see psr_probe.h): dependency chains of one
// operation per thread, enough chains per thread and threads per SM to keep the pipe
// full, so that operations / launch time is the pipe's sustained rate.
#include <cuda_runtime.h>

#include <cmath>

#include "psr.h"
#include "psr_internal.h"
#include "psr_probe.h"

namespace psr {
namespace {

__global__ void fma64_probe(int64_t iters, double *sink) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = 1.0 + 1e-3 * (t % 97) + 1e-4 * c;
    const double b = 0.99999999, d = 1e-8;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = fma(a[c], b, d);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    sink[t] = s;
}

__global__ void fma32_probe(int64_t iters, double *sink) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float a[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) a[c] = 1.0f + 1e-3f * float(t % 97) + 1e-4f * float(c);
    const float b = 0.9999999f, d = 1e-7f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 16; ++c) a[c] = fmaf(a[c], b, d);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 16; ++c) s += a[c];
    sink[t] = double(s);
}

// kind 2: exp, 3: log, 4: division; arguments stay in a moderate range
template <int KIND>
__global__ void math64_probe(int64_t iters, double *sink) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double x[8], acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        x[c] = (KIND == 2 ? -1.0 : 1.5) + 1e-3 * (t % 89) + 1e-2 * c;
        acc[c] = 0.0;
    }
    const double step = 1e-9;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (KIND == 2) acc[c] += exp(x[c]);
            else if (KIND == 3) acc[c] += log(x[c]);
            else acc[c] += 1.0 / x[c];
            x[c] += step;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += acc[c];
    sink[t] = s;
}

// kinds 5-8: shared-memory atomicAdd of float / double, 8 per iteration, to 32 distinct
// words per warp (lane-indexed) or all lanes to one word (the worst collision)
template <class T, bool SAME>
__global__ void smem_atomic_probe(int64_t iters, double *sink) {
    __shared__ T buf[8 * 32 * 8];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = (threadIdx.x >> 5) & 7;
    for (int i = threadIdx.x; i < 8 * 32 * 8; i += blockDim.x) buf[i] = T(0);
    __syncthreads();
    T *base = buf + wid * 32 * 8;
    const T v = T(1) + T(lane) * T(1e-3);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) atomicAdd(base + c * 32 + (SAME ? 0 : lane), v);
    }
    __syncthreads();
    sink[t] = double(buf[threadIdx.x % (8 * 32 * 8)]);
}

}  // namespace
}  // namespace psr

extern "C" int psr_pipe_probe(int32_t kind, int64_t iters, int32_t blocks, int32_t threads, double *sink,
                              void *stream) {
    using namespace psr;
    if (iters < 1 || blocks < 1 || threads < 32 || threads > 256 || (threads & 31) || !sink)
        return set_error(PSR_E_ARG, "psr_pipe_probe: bad sizes or NULL sink");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (kind) {
        case PSR_PROBE_FMA64: fma64_probe<<<blocks, threads, 0, st>>>(iters, sink); break;
        case PSR_PROBE_FMA32: fma32_probe<<<blocks, threads, 0, st>>>(iters, sink); break;
        case PSR_PROBE_EXP64: math64_probe<2><<<blocks, threads, 0, st>>>(iters, sink); break;
        case PSR_PROBE_LOG64: math64_probe<3><<<blocks, threads, 0, st>>>(iters, sink); break;
        case PSR_PROBE_DIV64: math64_probe<4><<<blocks, threads, 0, st>>>(iters, sink); break;
        case PSR_PROBE_SATOM32: smem_atomic_probe<float, false><<<blocks, threads, 0, st>>>(iters, sink); break;
        case PSR_PROBE_SATOM32_SAME: smem_atomic_probe<float, true><<<blocks, threads, 0, st>>>(iters, sink); break;
        case PSR_PROBE_SATOM64: smem_atomic_probe<double, false><<<blocks, threads, 0, st>>>(iters, sink); break;
        case PSR_PROBE_SATOM64_SAME: smem_atomic_probe<double, true><<<blocks, threads, 0, st>>>(iters, sink); break;
        default: return set_error(PSR_E_ARG, "psr_pipe_probe: unknown kind");
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error("psr_pipe_probe launch", e);
    return PSR_OK;
}
