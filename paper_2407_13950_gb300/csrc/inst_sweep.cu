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

template <int SOLVER, bool BWD>
static cudaError_t launch_one(const ProbDev& pd, bool want_hist, cudaStream_t s) {
    auto kern = k_sweep<MSQOC_L, MSQOC_Q, SOLVER, BWD>;
    static bool configured = false;
    if (!configured) {
        int dev = 0, maxsmem = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsmem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const size_t smem = sweep_smem_bytes(pd, BWD);
    kern<<<pd.ntiles, pd.nthreads, smem, s>>>(pd, want_hist ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t MSQOC_CAT(launch_sweep, MSQOC_L, MSQOC_Q)(const ProbDev& pd, bool bwd, bool want_hist, cudaStream_t s) {
    if (pd.solver == SOLVER_FP64)
        return bwd ? launch_one<SOLVER_FP64, true>(pd, want_hist, s) : launch_one<SOLVER_FP64, false>(pd, want_hist, s);
    return bwd ? launch_one<SOLVER_MIXED, true>(pd, want_hist, s) : launch_one<SOLVER_MIXED, false>(pd, want_hist, s);
}

}  // namespace msqoc
