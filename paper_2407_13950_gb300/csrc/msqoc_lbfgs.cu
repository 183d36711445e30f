// Limited-memory BFGS steps of the client optimiser on the device: the search direction by the
// two-loop recursion, the projected trial point of the line search and the memory update.
// Each is one CTA that sweeps the n-vectors in a fixed order, so results are deterministic and
// one optimiser iteration costs a few launches instead of dozens of small vector operations.
#include <cstdint>

#include "../../include/msqoc.h"
#include "msqoc_host.h"

namespace msqoc {
namespace {

constexpr int LB_THREADS = 1024;

// sum of v over the block in a fixed order (every thread gets the result): an xor butterfly in
// each warp (lanes i and i ^ o add the same two values, so every lane ends with the same sum),
// then the same over the warps' sums.  sh: at least 33 doubles.
__device__ double lb_block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        double r = sh[lane];   // LB_THREADS / 32 = 32 warps
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if (lane == 0) sh[32] = r;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();   // sh is reused by the next sum
    return r;
}
static_assert(LB_THREADS == 1024, "lb_block_sum reduces 32 warps");

// x_i at a bound with the gradient pushing it outward (held fixed for the iteration)
__device__ __forceinline__ bool lb_active(int64_t i, int64_t nb, const double* x, const double* g,
                                          const double* lim) {
    if (i >= nb) return false;
    const double xi = x[i], gi = g[i], li = lim[i];
    return (xi >= li && gi < 0.0) || (xi <= -li && gi > 0.0);
}

// d = -H pg (two-loop recursion over the m newest of the ring slots, newest = head - 1), zero on
// the active set; slope = <pg, d>.  alpha_s holds the first loop's coefficients (m <= MAXMEM).
__global__ void __launch_bounds__(LB_THREADS) k_lbfgs_direction(int64_t n, int64_t nb, const double* x,
                                                                const double* g, const double* lim,
                                                                const double* S, const double* Y,
                                                                const double* rho, const double* yy, int cap,
                                                                int m, int head, double* d, double* slope) {
    __shared__ double sh[LB_THREADS];
    __shared__ double alpha_s[MSQOC_LBFGS_MAXMEM];
    const int t = threadIdx.x;
    for (int64_t i = t; i < n; i += LB_THREADS) d[i] = lb_active(i, nb, x, g, lim) ? 0.0 : g[i];
    __syncthreads();
    auto slot_of = [&](int j) { return ((head - m + j) % cap + cap) % cap; };   // j = 0: oldest
    for (int j = m - 1; j >= 0; --j) {
        const int s = slot_of(j);
        const double* Sj = S + size_t(s) * n;
        const double* Yj = Y + size_t(s) * n;
        double acc = 0.0;
#pragma unroll 4
        for (int64_t i = t; i < n; i += LB_THREADS) acc += Sj[i] * d[i];
        const double a = rho[s] * lb_block_sum(acc, sh);
        if (t == 0) alpha_s[j] = a;
#pragma unroll 4
        for (int64_t i = t; i < n; i += LB_THREADS) d[i] -= a * Yj[i];
        __syncthreads();
    }
    double gamma;
    if (m > 0) {
        const int s = slot_of(m - 1);
        gamma = (1.0 / rho[s]) / yy[s];   // <s, y> / <y, y> of the newest pair
    } else {
        double acc = 0.0;
#pragma unroll 4
        for (int64_t i = t; i < n; i += LB_THREADS) acc += d[i] * d[i];
        gamma = 1.0 / fmax(sqrt(lb_block_sum(acc, sh)), 1e-300);   // first step: unit length
    }
    for (int64_t i = t; i < n; i += LB_THREADS) d[i] *= gamma;
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        const int s = slot_of(j);
        const double* Sj = S + size_t(s) * n;
        const double* Yj = Y + size_t(s) * n;
        double acc = 0.0;
#pragma unroll 4
        for (int64_t i = t; i < n; i += LB_THREADS) acc += Yj[i] * d[i];
        const double c = alpha_s[j] - rho[s] * lb_block_sum(acc, sh);
#pragma unroll 4
        for (int64_t i = t; i < n; i += LB_THREADS) d[i] += c * Sj[i];
        __syncthreads();
    }
    double acc = 0.0;
    for (int64_t i = t; i < n; i += LB_THREADS) {
        const bool a = lb_active(i, nb, x, g, lim);
        const double di = a ? 0.0 : -d[i];
        d[i] = di;
        acc += (a ? 0.0 : g[i]) * di;
    }
    const double sl = lb_block_sum(acc, sh);
    if (t == 0) *slope = sl;
}

// x_new = projection of x + step d onto the box (the first nb entries), dec = <g, x_new - x>
__global__ void __launch_bounds__(LB_THREADS) k_lbfgs_trial(int64_t n, int64_t nb, const double* x,
                                                            const double* d, double step, const double* lim,
                                                            const double* g, double* x_new, double* dec) {
    __shared__ double sh[LB_THREADS];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += LB_THREADS) {
        double v = x[i] + step * d[i];
        if (i < nb) v = fmin(fmax(v, -lim[i]), lim[i]);
        x_new[i] = v;
        acc += g[i] * (v - x[i]);
    }
    const double s = lb_block_sum(acc, sh);
    if (threadIdx.x == 0) *dec = s;
}

// s = x_new - x, y = g_new - g into one ring slot; sy_yy = (<s, y>, <y, y>)
__global__ void __launch_bounds__(LB_THREADS) k_lbfgs_update(int64_t n, const double* x, const double* x_new,
                                                             const double* g, const double* g_new, double* Sk,
                                                             double* Yk, double* sy_yy) {
    __shared__ double sh[LB_THREADS];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += LB_THREADS) {
        const double s = x_new[i] - x[i], y = g_new[i] - g[i];
        Sk[i] = s;
        Yk[i] = y;
        a += s * y;
        b += y * y;
    }
    const double sy = lb_block_sum(a, sh);
    const double yy = lb_block_sum(b, sh);
    if (threadIdx.x == 0) {
        sy_yy[0] = sy;
        sy_yy[1] = yy;
    }
}

bool all_device(std::initializer_list<const void*> ps) {
    for (const void* p : ps)
        if (p && !is_device_ptr(p)) return false;
    return true;
}

}  // namespace
}  // namespace msqoc

using namespace msqoc;

extern "C" {

msqoc_status msqoc_lbfgs_direction(int64_t n, int64_t nb, const double* x, const double* g, const double* lim,
                                   const double* S, const double* Y, const double* rho, const double* yy,
                                   int32_t cap, int32_t m, int32_t head, double* d_out, double* slope_out,
                                   void* stream) {
    if (n < 1 || nb < 0 || nb > n) return fail(MSQOC_ERR_INVALID_ARG, "n %lld, nb %lld", (long long)n, (long long)nb);
    if (cap < 0 || cap > MSQOC_LBFGS_MAXMEM || m < 0 || m > cap || (cap > 0 && (head < 0 || head >= cap)))
        return fail(MSQOC_ERR_INVALID_ARG, "memory cap %d (<= %d), m %d, head %d", cap, MSQOC_LBFGS_MAXMEM, m, head);
    if (!x || !g || !d_out || !slope_out || (nb > 0 && !lim) || (m > 0 && (!S || !Y || !rho || !yy)))
        return fail(MSQOC_ERR_INVALID_ARG, "a required array is NULL");
    if (!all_device({x, g, lim, S, Y, rho, yy, d_out, slope_out}))
        return fail(MSQOC_ERR_INVALID_ARG, "the L-BFGS arrays must be device memory");
    k_lbfgs_direction<<<1, LB_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(n, nb, x, g, lim, S, Y, rho, yy,
                                                                                 cap, m, head, d_out, slope_out);
    CUDA_TRY(cudaGetLastError());
    return MSQOC_OK;
}

msqoc_status msqoc_lbfgs_trial(int64_t n, int64_t nb, const double* x, const double* d, double step,
                               const double* lim, const double* g, double* x_new, double* dec_out, void* stream) {
    if (n < 1 || nb < 0 || nb > n) return fail(MSQOC_ERR_INVALID_ARG, "n %lld, nb %lld", (long long)n, (long long)nb);
    if (!x || !d || !g || !x_new || !dec_out || (nb > 0 && !lim))
        return fail(MSQOC_ERR_INVALID_ARG, "a required array is NULL");
    if (!all_device({x, d, lim, g, x_new, dec_out}))
        return fail(MSQOC_ERR_INVALID_ARG, "the L-BFGS arrays must be device memory");
    k_lbfgs_trial<<<1, LB_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(n, nb, x, d, step, lim, g, x_new,
                                                                             dec_out);
    CUDA_TRY(cudaGetLastError());
    return MSQOC_OK;
}

msqoc_status msqoc_lbfgs_update(int64_t n, const double* x, const double* x_new, const double* g,
                                const double* g_new, double* s_out, double* y_out, double* sy_yy_out, void* stream) {
    if (n < 1) return fail(MSQOC_ERR_INVALID_ARG, "n %lld < 1", (long long)n);
    if (!x || !x_new || !g || !g_new || !s_out || !y_out || !sy_yy_out)
        return fail(MSQOC_ERR_INVALID_ARG, "a required array is NULL");
    if (!all_device({x, x_new, g, g_new, s_out, y_out, sy_yy_out}))
        return fail(MSQOC_ERR_INVALID_ARG, "the L-BFGS arrays must be device memory");
    k_lbfgs_update<<<1, LB_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(n, x, x_new, g, g_new, s_out, y_out,
                                                                              sy_yy_out);
    CUDA_TRY(cudaGetLastError());
    return MSQOC_OK;
}

}  // extern "C"
