// One instantiation of the warp-per-reactor solve_kernel per build of this file.
//
// The build compiles it once for each (Jacobian precision, soot, finite-difference
// Jacobian) combination the launchers use, passing PSR_INST_TJ (float | double),
// PSR_INST_SOOT and PSR_INST_FDJ (0 | 1), so that the six large kernels compile in
// parallel. Each build defines solve_kernel_entry for its combination: the kernel's host
// address, which the launchers in psr_solve.cu hand to cudaLaunchKernel.
#include "psr_warp.cuh"

#if !defined(PSR_INST_TJ) || !defined(PSR_INST_SOOT) || !defined(PSR_INST_FDJ)
#error "psr_solve_inst.cu needs PSR_INST_TJ, PSR_INST_SOOT and PSR_INST_FDJ"
#endif

namespace psr {
template <>
const void *solve_kernel_entry<PSR_INST_TJ, bool(PSR_INST_SOOT), bool(PSR_INST_FDJ)>() {
    return reinterpret_cast<const void *>(&solve_kernel<PSR_INST_TJ, bool(PSR_INST_SOOT), bool(PSR_INST_FDJ)>);
}
}  // namespace psr
