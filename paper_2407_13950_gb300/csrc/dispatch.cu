// Dispatch of the sweep launch to the kernel instantiated for the problem's shape.
#include "msqoc_internal.h"

namespace msqoc {

#define MSQOC_DECL(L, Q) cudaError_t launch_sweep_L##L##_Q##Q(const ProbDev&, bool, bool, cudaStream_t);
MSQOC_DECL(2, 1) MSQOC_DECL(2, 2) MSQOC_DECL(2, 3) MSQOC_DECL(2, 4) MSQOC_DECL(2, 5) MSQOC_DECL(2, 6)
MSQOC_DECL(3, 1) MSQOC_DECL(3, 2) MSQOC_DECL(3, 3) MSQOC_DECL(3, 4) MSQOC_DECL(3, 5)
#undef MSQOC_DECL

cudaError_t launch_sweep(const ProbDev& pd, bool bwd, bool want_hist, cudaStream_t s) {
#define MSQOC_CASE(LV, QV) \
    if (pd.L == LV && pd.q == QV) return launch_sweep_L##LV##_Q##QV(pd, bwd, want_hist, s);
    MSQOC_CASE(2, 1) MSQOC_CASE(2, 2) MSQOC_CASE(2, 3) MSQOC_CASE(2, 4) MSQOC_CASE(2, 5) MSQOC_CASE(2, 6)
    MSQOC_CASE(3, 1) MSQOC_CASE(3, 2) MSQOC_CASE(3, 3) MSQOC_CASE(3, 4) MSQOC_CASE(3, 5)
#undef MSQOC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace msqoc
