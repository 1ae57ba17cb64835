/* psr_probe.h -- pipe-throughput probes of libpsr (measurement service).
 *
 * The paper has no counterpart: these kernels measure the peak rates the solver's
 * roofline is reported against on the GPU at hand, because the FP64 pipe, the FP32 FMA
 * pipe and the double-precision exp and log of the CUDA math library bound the PSR
 * solve, and none of them is among the measured peaks (HBM copy, bf16 GEMM).
 *
 * psr_pipe_probe launches one probe kernel of `blocks` x `threads` threads on `stream`;
 * every thread runs `iters` iterations of independent dependency chains:
 *   PSR_PROBE_FMA64  8 chains a = fma(a, b, c) in FP64:   16 flops per iteration
 *   PSR_PROBE_FMA32  16 chains a = fma(a, b, c) in FP32:  32 flops per iteration
 *   PSR_PROBE_EXP64  8 calls exp(x) in FP64 per iteration (plus one add and one
 *                    accumulate per call)
 *   PSR_PROBE_LOG64  8 calls log(x) in FP64 per iteration (same overhead)
 *   PSR_PROBE_DIV64  8 FP64 divisions per iteration (same overhead)
 *   PSR_PROBE_SATOM32 / _SAME  8 shared-memory float atomicAdd per iteration, each warp's
 *                    lanes to 32 distinct words / all to one word (full collision)
 *   PSR_PROBE_SATOM64 / _SAME  the same with double
 * threads: a multiple of 32, at most 256.
 * The operation count of a launch is blocks x threads x iters x the per-iteration count;
 * the caller times the launch (CUDA events on `stream`). `sink` (device, >= blocks x
 * threads doubles) receives one value per thread so that no chain is optimised away.
 * Errors: PSR_E_ARG (unknown kind, non-positive sizes, NULL sink), PSR_E_CUDA. */
#ifndef PSR_PROBE_H
#define PSR_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSR_PROBE_FMA64 0
#define PSR_PROBE_FMA32 1
#define PSR_PROBE_EXP64 2
#define PSR_PROBE_LOG64 3
#define PSR_PROBE_DIV64 4
#define PSR_PROBE_SATOM32 5
#define PSR_PROBE_SATOM32_SAME 6
#define PSR_PROBE_SATOM64 7
#define PSR_PROBE_SATOM64_SAME 8

int psr_pipe_probe(int32_t kind, int64_t iters, int32_t blocks, int32_t threads, double *sink, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PSR_PROBE_H */
