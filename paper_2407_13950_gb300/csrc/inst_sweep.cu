// Explicit instantiation of the sweep kernels for one (levels, subsystems) shape, selected with
// -DMSQOC_L=<levels> -DMSQOC_Q=<subsystems>; this file is compiled once per supported shape.
#include "msqoc_sweep.cuh"

#ifndef MSQOC_L
#error "MSQOC_L must be defined"
#endif
#ifndef MSQOC_Q
#error "MSQOC_Q must be defined"
#endif

#define MSQOC_CAT2(a, b, c) a##_L##b##_Q##c
#define MSQOC_CAT(a, b, c) MSQOC_CAT2(a, b, c)

namespace msqoc {

template <int SOLVER, bool BWD, bool ROLLOUT = false>
static cudaError_t launch_one(const SweepArgs& a, int ntiles, cudaStream_t s) {
    auto kern = k_sweep<MSQOC_L, MSQOC_Q, SOLVER, BWD, ROLLOUT>;
    const size_t smem = sweep_smem_bytes(a);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    if (ntiles <= 0) return cudaSuccess;
    kern<<<ntiles, a.nthreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int SOLVER, bool BWD>
static int occupancy_one(const SweepArgs& a) {
    auto kern = k_sweep<MSQOC_L, MSQOC_Q, SOLVER, BWD>;
    const size_t smem = sweep_smem_bytes(a);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, a.nthreads, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t MSQOC_CAT(launch_sweep, MSQOC_L, MSQOC_Q)(const SweepArgs& a, int ntiles, cudaStream_t s) {
    if (a.mode == SWEEP_ROLLOUT)
        return a.solver == SOLVER_FP64 ? launch_one<SOLVER_FP64, false, true>(a, ntiles, s)
                                       : launch_one<SOLVER_MIXED, false, true>(a, ntiles, s);
    const bool bwd = a.mode == SWEEP_ADJOINT;
    if (a.solver == SOLVER_FP64)
        return bwd ? launch_one<SOLVER_FP64, true>(a, ntiles, s) : launch_one<SOLVER_FP64, false>(a, ntiles, s);
    return bwd ? launch_one<SOLVER_MIXED, true>(a, ntiles, s) : launch_one<SOLVER_MIXED, false>(a, ntiles, s);
}

int MSQOC_CAT(sweep_occupancy, MSQOC_L, MSQOC_Q)(const SweepArgs& a) {
    const bool bwd = a.mode == SWEEP_ADJOINT;
    if (a.solver == SOLVER_FP64) return bwd ? occupancy_one<SOLVER_FP64, true>(a) : occupancy_one<SOLVER_FP64, false>(a);
    return bwd ? occupancy_one<SOLVER_MIXED, true>(a) : occupancy_one<SOLVER_MIXED, false>(a);
}

}  // namespace msqoc
