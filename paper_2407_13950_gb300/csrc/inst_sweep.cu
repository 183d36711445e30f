// Explicit instantiation of the sweep kernels (the families: one thread per fiber, a lane pair
// per fiber and, for 2-level shapes, a lane quad per fiber) for one (levels, subsystems) shape,
// selected with -DMSQOC_L=<levels> -DMSQOC_Q=<subsystems>; this file is compiled once per
// supported shape.
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

// FAM: log2 of the threads per fiber (0: k_sweep; 1, 2: k_sweep_pair with one or two entry groups),
// or 3: k_sweep with the 168-register budget (one thread per fiber, up to 12 warps an SM)
template <int SOLVER, bool BWD, bool ROLLOUT, int FAM>
static auto kernel_of() {
    if constexpr (FAM == 3)
        return k_sweep<MSQOC_L, MSQOC_Q, SOLVER, BWD, ROLLOUT, MAX_LEAN_TILE_THREADS>;
    else if constexpr (FAM == 2)
        return k_sweep_pair<MSQOC_L, MSQOC_Q, SOLVER, BWD, ROLLOUT, 2>;
    else if constexpr (FAM == 1)
        return k_sweep_pair<MSQOC_L, MSQOC_Q, SOLVER, BWD, ROLLOUT, 1>;
    else
        return k_sweep<MSQOC_L, MSQOC_Q, SOLVER, BWD, ROLLOUT>;
}

// Dynamic shared memory above 48 KB needs the kernel's opt-in attribute, and the 48 KB limit
// counts the kernel's static shared memory too.  The static size of each instantiation is read
// once from the runtime (cudaFuncGetAttributes); the opt-in is set when static + dynamic bytes
// exceed 48 KB.
constexpr size_t SMEM_DEFAULT_LIMIT = 48 * 1024;

// one static per kernel instantiation (the template parameters name the kernel)
template <int SOLVER, bool BWD, bool ROLLOUT, int FAM>
static bool needs_opt_in(size_t smem) {
    static const size_t static_bytes = [] {
        cudaFuncAttributes fa{};
        // an unreadable attribute counts as the largest static size, so the opt-in is taken
        return cudaFuncGetAttributes(&fa, kernel_of<SOLVER, BWD, ROLLOUT, FAM>()) == cudaSuccess ? fa.sharedSizeBytes
                                                                                                 : SMEM_DEFAULT_LIMIT;
    }();
    return smem + static_bytes > SMEM_DEFAULT_LIMIT;
}

template <int SOLVER, bool BWD, bool ROLLOUT, int FAM>
static cudaError_t launch_one(const SweepArgs& a, int ntiles, cudaStream_t s) {
    auto kern = kernel_of<SOLVER, BWD, ROLLOUT, FAM>();
    const size_t smem = sweep_smem_bytes(a);
    if (needs_opt_in<SOLVER, BWD, ROLLOUT, FAM>(smem)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    if (ntiles <= 0) return cudaSuccess;
    kern<<<ntiles, a.nthreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int SOLVER, bool BWD, int FAM>
static int occupancy_one(const SweepArgs& a) {
    auto kern = kernel_of<SOLVER, BWD, false, FAM>();
    const size_t smem = sweep_smem_bytes(a);
    if (needs_opt_in<SOLVER, BWD, false, FAM>(smem) &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, a.nthreads, smem) != cudaSuccess) return 0;
    return n;
}

template <int FAM>
static cudaError_t launch_family(const SweepArgs& a, int ntiles, cudaStream_t s) {
    if (a.mode == SWEEP_ROLLOUT)
        return a.solver == SOLVER_FP64 ? launch_one<SOLVER_FP64, false, true, FAM>(a, ntiles, s)
                                       : launch_one<SOLVER_MIXED, false, true, FAM>(a, ntiles, s);
    const bool bwd = a.mode == SWEEP_ADJOINT;
    if (a.solver == SOLVER_FP64)
        return bwd ? launch_one<SOLVER_FP64, true, false, FAM>(a, ntiles, s)
                   : launch_one<SOLVER_FP64, false, false, FAM>(a, ntiles, s);
    return bwd ? launch_one<SOLVER_MIXED, true, false, FAM>(a, ntiles, s)
               : launch_one<SOLVER_MIXED, false, false, FAM>(a, ntiles, s);
}

template <int FAM>
static int occupancy_family(const SweepArgs& a) {
    const bool bwd = a.mode == SWEEP_ADJOINT;
    if (a.solver == SOLVER_FP64)
        return bwd ? occupancy_one<SOLVER_FP64, true, FAM>(a) : occupancy_one<SOLVER_FP64, false, FAM>(a);
    return bwd ? occupancy_one<SOLVER_MIXED, true, FAM>(a) : occupancy_one<SOLVER_MIXED, false, FAM>(a);
}

cudaError_t MSQOC_CAT(launch_sweep, MSQOC_L, MSQOC_Q)(const SweepArgs& a, int ntiles, cudaStream_t s) {
    if (a.pair == 0) return a.lean ? launch_family<3>(a, ntiles, s) : launch_family<0>(a, ntiles, s);
    if (a.pair == 1) return launch_family<1>(a, ntiles, s);
#if MSQOC_L == 2
    if (a.pair == 2) return launch_family<2>(a, ntiles, s);
#endif
    return cudaErrorInvalidValue;
}

int MSQOC_CAT(sweep_occupancy, MSQOC_L, MSQOC_Q)(const SweepArgs& a) {
    if (a.pair == 0) return a.lean ? occupancy_family<3>(a) : occupancy_family<0>(a);
    if (a.pair == 1) return occupancy_family<1>(a);
#if MSQOC_L == 2
    if (a.pair == 2) return occupancy_family<2>(a);
#endif
    return 0;
}

}  // namespace msqoc
