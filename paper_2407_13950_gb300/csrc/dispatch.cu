// Dispatch of the sweep launch to the kernel instantiated for the problem's shape.
#include "msqoc_internal.h"
#include "msqoc_sweep_common.cuh"

namespace msqoc {

#define MSQOC_DECL(L, Q)                                                                       \
    cudaError_t launch_sweep_L##L##_Q##Q(const SweepArgs&, int, cudaStream_t);                 \
    int sweep_occupancy_L##L##_Q##Q(const SweepArgs&);
MSQOC_DECL(2, 1) MSQOC_DECL(2, 2) MSQOC_DECL(2, 3) MSQOC_DECL(2, 4) MSQOC_DECL(2, 5) MSQOC_DECL(2, 6)
MSQOC_DECL(3, 1) MSQOC_DECL(3, 2) MSQOC_DECL(3, 3) MSQOC_DECL(3, 4) MSQOC_DECL(3, 5)
#undef MSQOC_DECL

#define MSQOC_SHAPES(X) \
    X(2, 1) X(2, 2) X(2, 3) X(2, 4) X(2, 5) X(2, 6) X(3, 1) X(3, 2) X(3, 3) X(3, 4) X(3, 5)

size_t sweep_smem_bytes(const SweepArgs& a) {
    const int N = ipow_c(a.L, a.q);
    return sweep_layout(a.q, a.L, N, a.cpt, a.nthreads, a.gmax, a.solver, a.mode == SWEEP_ADJOINT, a.pair,
                        a.hdepth).total;
}

cudaError_t launch_sweep(const SweepArgs& a, int ntiles, cudaStream_t s) {
#define MSQOC_CASE(LV, QV) \
    if (a.L == LV && a.q == QV) return launch_sweep_L##LV##_Q##QV(a, ntiles, s);
    MSQOC_SHAPES(MSQOC_CASE)
#undef MSQOC_CASE
    return cudaErrorInvalidValue;
}

int sweep_ctas_per_sm(const SweepArgs& a) {
#define MSQOC_CASE(LV, QV) \
    if (a.L == LV && a.q == QV) return sweep_occupancy_L##LV##_Q##QV(a);
    MSQOC_SHAPES(MSQOC_CASE)
#undef MSQOC_CASE
    return 0;
}

}  // namespace msqoc
