// Self-tests of pieces of the sweeps:
//  * the failure path: the bounded mbarrier wait (the one the adjoint sweep uses for its
//    midpoint-history fetches) on a barrier that nothing completes gives up after its spin
//    limit, and the launch reports it through the status word as MSQOC_ERR_TIMEOUT instead of
//    hanging the GPU.  The context stays usable afterwards.
//  * the compensated FP32 arithmetic of the mixed solver (msqoc_split.cuh), on the host or in a
//    one-thread kernel: the split of doubles into two floats, a real dot product formed the way
//    the adjoint forms its gradient products, and steps of the compensated state update.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/msqoc.h"
#include "msqoc_host.h"
#include "msqoc_split.cuh"
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

__global__ void k_split_probe(const double* x, int64_t n, int sh, float* hi, float* lo) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float2 v = split_scaled(x[i], sh);
        hi[i] = v.x;
        lo[i] = v.y;
    }
}

// sum_i x_i y_i with the split operands (x 2^-shx, y 2^-shy) and the compensated accumulation,
// scaled back by 2^(shx + shy)
__host__ __device__ double dot_split(const double* x, const double* y, int64_t n, int shx, int shy) {
    DF acc{0.f, 0.f};
    for (int64_t i = 0; i < n; ++i) {
        const float2 a = split_scaled(x[i], shx), b = split_scaled(y[i], shy);
        df_mac(acc, a.x, a.y, b.x, b.y);
    }
    return df_to_f64_scaled(acc, shx + shy);
}

__global__ void k_dot_probe(const double* x, const double* y, int64_t n, int shx, int shy, double* out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *out = dot_split(x, y, n, shx, shy);
}

// n steps of the compensated state update on one complex entry from u0 with the preconditioner
// entry P and the corrections d_j (absolute), in units 2^-sh; out = the final u + carry
__host__ __device__ void carry_steps(const double* u0, const double* P, const double* d, int64_t n, int sh,
                                     double* out) {
    double2 u = make_double2(u0[0], u0[1]);
    const double2 p = make_double2(P[0], P[1]);
    const float4 Ps = split_scaled(p, 0);
    const float2 P3 = make_float2(split_third(p.x, make_float2(Ps.x, Ps.z)), split_third(p.y, make_float2(Ps.y, Ps.w)));
    const double k2d = -2.0 * p.y / p.x;
    const float2 k2 = split_scaled(k2d, 0);
    const float k3 = split_third(k2d, k2);
    float2 car = make_float2(0.f, 0.f);
    for (int64_t j = 0; j < n; ++j) {
        DF bre, bim;
        carry_rhs(split_scaled(u, sh), Ps, P3, car, bre, bim);
        const float2 dr = split_scaled(d[2 * j], sh), di = split_scaled(d[2 * j + 1], sh);
        u = carry_update(u, bre, bim, k2, k3, DF{dr.x, dr.y}, DF{di.x, di.y}, sh, car);
    }
    const double2 r = carry_finish(u, car, sh);
    out[0] = r.x;
    out[1] = r.y;
}

__global__ void k_carry_probe(const double* u0, const double* P, const double* d, int64_t n, int sh, double* out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) carry_steps(u0, P, d, n, sh, out);
}

// device copies of n doubles; frees what it allocated on failure
struct DevBufs {
    std::vector<void*> p;
    ~DevBufs() {
        for (void* b : p) cudaFree(b);
    }
    template <typename T>
    cudaError_t alloc(T** out, size_t n) {
        void* b = nullptr;
        const cudaError_t e = cudaMalloc(&b, n ? n * sizeof(T) : sizeof(T));
        if (e == cudaSuccess) p.push_back(b);
        *out = static_cast<T*>(b);
        return e;
    }
};

}  // namespace
}  // namespace msqoc

using namespace msqoc;

extern "C" msqoc_status msqoc_selftest_split(const double* x, int64_t n, int32_t sh, int32_t on_device, float* hi,
                                             float* lo) {
    if (n < 0 || (n > 0 && (!x || !hi || !lo))) return fail(MSQOC_ERR_INVALID_ARG, "split self-test: bad arrays");
    if (sh < -2000 || sh > 2000) return fail(MSQOC_ERR_INVALID_ARG, "split self-test: scale %d out of range", sh);
    if (!on_device) {
        for (int64_t i = 0; i < n; ++i) {
            const float2 v = split_scaled(x[i], sh);
            hi[i] = v.x;
            lo[i] = v.y;
        }
        return MSQOC_OK;
    }
    if (n == 0) return MSQOC_OK;
    DevBufs d;
    double* xd = nullptr;
    float *hd = nullptr, *ld = nullptr;
    cudaError_t e = d.alloc(&xd, n);
    if (e == cudaSuccess) e = d.alloc(&hd, n);
    if (e == cudaSuccess) e = d.alloc(&ld, n);
    if (e == cudaSuccess) e = cudaMemcpy(xd, x, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_split_probe<<<static_cast<int>(std::min<int64_t>((n + 255) / 256, 1024)), 256>>>(xd, n, sh, hd, ld);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(hi, hd, n * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(lo, ld, n * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(MSQOC_ERR_CUDA, "split self-test: %s", cudaGetErrorString(e));
    return MSQOC_OK;
}

extern "C" msqoc_status msqoc_selftest_dot(const double* x, const double* y, int64_t n, int32_t shx, int32_t shy,
                                           int32_t on_device, double* out) {
    if (n < 0 || !out || (n > 0 && (!x || !y))) return fail(MSQOC_ERR_INVALID_ARG, "dot self-test: bad arrays");
    if (shx < -2000 || shx > 2000 || shy < -2000 || shy > 2000)
        return fail(MSQOC_ERR_INVALID_ARG, "dot self-test: scales %d, %d out of range", shx, shy);
    if (!on_device) {
        *out = dot_split(x, y, n, shx, shy);
        return MSQOC_OK;
    }
    DevBufs d;
    double *xd = nullptr, *yd = nullptr, *od = nullptr;
    cudaError_t e = d.alloc(&xd, n);
    if (e == cudaSuccess) e = d.alloc(&yd, n);
    if (e == cudaSuccess) e = d.alloc(&od, 1);
    if (e == cudaSuccess && n) e = cudaMemcpy(xd, x, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n) e = cudaMemcpy(yd, y, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_dot_probe<<<1, 32>>>(xd, yd, n, shx, shy, od);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, od, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(MSQOC_ERR_CUDA, "dot self-test: %s", cudaGetErrorString(e));
    return MSQOC_OK;
}

extern "C" msqoc_status msqoc_selftest_carry(const double* u0, const double* P, const double* d, int64_t n,
                                             int32_t sh, int32_t on_device, double* out) {
    if (n < 0 || !u0 || !P || !out || (n > 0 && !d)) return fail(MSQOC_ERR_INVALID_ARG, "carry self-test: bad arrays");
    if (sh < -SCALE_SHIFT_MAX || sh > SCALE_SHIFT_MAX)
        return fail(MSQOC_ERR_INVALID_ARG, "carry self-test: scale %d out of range", sh);
    if (!(P[0] > 0.5 && P[0] <= 1.0)) return fail(MSQOC_ERR_INVALID_ARG, "carry self-test: Re P not in (1/2, 1]");
    const double k2 = -2.0 * P[1] / P[0];
    if (!(k2 * k2 <= CARRY_UPDATE_K2))
        return fail(MSQOC_ERR_INVALID_ARG, "carry self-test: |2 kappa| above the compensated update's bound");
    if (!on_device) {
        carry_steps(u0, P, d, n, sh, out);
        return MSQOC_OK;
    }
    DevBufs b;
    double *ud = nullptr, *pdv = nullptr, *dd = nullptr, *od = nullptr;
    cudaError_t e = b.alloc(&ud, 2);
    if (e == cudaSuccess) e = b.alloc(&pdv, 2);
    if (e == cudaSuccess) e = b.alloc(&dd, std::max<int64_t>(2 * n, 1));
    if (e == cudaSuccess) e = b.alloc(&od, 2);
    if (e == cudaSuccess) e = cudaMemcpy(ud, u0, 2 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pdv, P, 2 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n) e = cudaMemcpy(dd, d, 2 * n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_carry_probe<<<1, 32>>>(ud, pdv, dd, n, sh, od);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, od, 2 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(MSQOC_ERR_CUDA, "carry self-test: %s", cudaGetErrorString(e));
    return MSQOC_OK;
}

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
