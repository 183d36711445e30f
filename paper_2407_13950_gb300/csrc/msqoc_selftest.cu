// Self-test of the sweeps' failure path: the bounded mbarrier wait (the one the adjoint sweep
// uses for its midpoint-history fetches) on a barrier that nothing completes gives up after its
// spin limit, and the launch reports it through the status word as MSQOC_ERR_TIMEOUT instead of
// hanging the GPU.  The context stays usable afterwards.
#include <cuda_runtime.h>

#include "../../include/msqoc.h"
#include "msqoc_host.h"
#include "msqoc_sweep_common.cuh"

namespace msqoc {
namespace {

// thread 0: a one-arrival mbarrier, completed first (arrive != 0) or never, then waited on
__global__ void k_wait_probe(int64_t spins, int arrive, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (arrive) mbar_arrive(&bar);
        if (!mbar_wait(&bar, 0, spins)) atomicOr(status, ST_TIMEOUT);
    }
}

}  // namespace
}  // namespace msqoc

using namespace msqoc;

extern "C" msqoc_status msqoc_selftest_bounded_wait(int64_t spins, int32_t arrive, double* seconds_out) {
    if (spins < 1 || spins > MBAR_WAIT_SPINS) return fail(MSQOC_ERR_INVALID_ARG, "spins %lld not in [1, %lld]",
                                                          (long long)spins, (long long)MBAR_WAIT_SPINS);
    int* st = nullptr;
    CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&st), sizeof(int)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaMemset(st, 0, sizeof(int));
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) ce = cudaEventRecord(e0, nullptr);
    if (ce == cudaSuccess) {
        k_wait_probe<<<1, 32>>>(spins, arrive ? 1 : 0, st);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, nullptr);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    int h = 0;
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaMemcpy(&h, st, sizeof(int), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(st);
    if (ce != cudaSuccess) return fail(MSQOC_ERR_CUDA, "bounded-wait self-test: %s", cudaGetErrorString(ce));
    if (seconds_out) *seconds_out = double(ms) * 1e-3;
    if (h & ST_TIMEOUT) return fail(MSQOC_ERR_TIMEOUT, "a bounded device wait gave up after %lld spins", (long long)spins);
    return MSQOC_OK;
}
