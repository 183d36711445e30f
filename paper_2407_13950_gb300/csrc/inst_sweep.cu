// Explicit instantiation of the sweep kernels (both families: one thread per fiber and a lane
// pair per fiber) for one (levels, subsystems) shape, selected with -DMSQOC_L=<levels>
// -DMSQOC_Q=<subsystems>; this file is compiled once per supported shape.
#include "msqoc_sweep.cuh"
#include "msqoc_sweep_pair.cuh"

#ifndef MSQOC_L
#error "MSQOC_L must be defined"
#endif
#ifndef MSQOC_Q
#error "MSQOC_Q must be defined"
#endif

#define MSQOC_CAT2(a, b, c) a##_L##b##_Q##c
#define MSQOC_CAT(a, b, c) MSQOC_CAT2(a, b, c)

namespace msqoc {

template <int SOLVER, bool BWD, bool ROLLOUT, bool PAIR>
static auto kernel_of() {
    if constexpr (PAIR)
        return k_sweep_pair<MSQOC_L, MSQOC_Q, SOLVER, BWD, ROLLOUT>;
    else
        return k_sweep<MSQOC_L, MSQOC_Q, SOLVER, BWD, ROLLOUT>;
}

template <int SOLVER, bool BWD, bool ROLLOUT, bool PAIR>
static cudaError_t launch_one(const SweepArgs& a, int ntiles, cudaStream_t s) {
    auto kern = kernel_of<SOLVER, BWD, ROLLOUT, PAIR>();
    const size_t smem = sweep_smem_bytes(a);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    if (ntiles <= 0) return cudaSuccess;
    kern<<<ntiles, a.nthreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int SOLVER, bool BWD, bool PAIR>
static int occupancy_one(const SweepArgs& a) {
    auto kern = kernel_of<SOLVER, BWD, false, PAIR>();
    const size_t smem = sweep_smem_bytes(a);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, a.nthreads, smem) != cudaSuccess) return 0;
    return n;
}

template <bool PAIR>
static cudaError_t launch_family(const SweepArgs& a, int ntiles, cudaStream_t s) {
    if (a.mode == SWEEP_ROLLOUT)
        return a.solver == SOLVER_FP64 ? launch_one<SOLVER_FP64, false, true, PAIR>(a, ntiles, s)
                                       : launch_one<SOLVER_MIXED, false, true, PAIR>(a, ntiles, s);
    const bool bwd = a.mode == SWEEP_ADJOINT;
    if (a.solver == SOLVER_FP64)
        return bwd ? launch_one<SOLVER_FP64, true, false, PAIR>(a, ntiles, s)
                   : launch_one<SOLVER_FP64, false, false, PAIR>(a, ntiles, s);
    return bwd ? launch_one<SOLVER_MIXED, true, false, PAIR>(a, ntiles, s)
               : launch_one<SOLVER_MIXED, false, false, PAIR>(a, ntiles, s);
}

template <bool PAIR>
static int occupancy_family(const SweepArgs& a) {
    const bool bwd = a.mode == SWEEP_ADJOINT;
    if (a.solver == SOLVER_FP64)
        return bwd ? occupancy_one<SOLVER_FP64, true, PAIR>(a) : occupancy_one<SOLVER_FP64, false, PAIR>(a);
    return bwd ? occupancy_one<SOLVER_MIXED, true, PAIR>(a) : occupancy_one<SOLVER_MIXED, false, PAIR>(a);
}

cudaError_t MSQOC_CAT(launch_sweep, MSQOC_L, MSQOC_Q)(const SweepArgs& a, int ntiles, cudaStream_t s) {
    return a.pair ? launch_family<true>(a, ntiles, s) : launch_family<false>(a, ntiles, s);
}

int MSQOC_CAT(sweep_occupancy, MSQOC_L, MSQOC_Q)(const SweepArgs& a) {
    return a.pair ? occupancy_family<true>(a) : occupancy_family<false>(a);
}

}  // namespace msqoc
