// Forward and adjoint sweeps of one multiple-shooting evaluation (sm_103a).
//
// One CTA owns a tile = (window m, block of cb state columns) and keeps those columns
// resident in shared memory / registers for every time step of the window.  Each thread owns
// one "fiber": the L entries of one column that differ only in the level of the last
// subsystem (stride 1), so that subsystem's ladder terms stay in registers; the other
// subsystems' ladder terms are tensor-product strided shifts read from shared memory
// through a per-thread neighbour list.  Fibers are sorted on the host so that the lanes of
// a warp share the same neighbour-list shape: every branch below is warp-uniform.
//
// Step equation (implicit midpoint rule, Sec. 5), with X = (h/2) H(t_{n+1/2}),
// H = D + C(t), D the diagonal drift and C the control ladder terms (Eq. ctrl-ham):
//   forward : (I + iX) Ubar = U_n,           U_{n+1} = 2 Ubar - U_n
//   adjoint : (I - iX) Lbar = Lambda_{n+1},  Lambda_n = 2 Lbar - Lambda_{n+1}
// (the exact discrete adjoint: Lambda_n = C_n^+ Lambda_{n+1} with C_n the Cayley map).
// Both are solved with the diagonal preconditioner P = (I + i h/2 D)^-1 (conj(P) for the
// adjoint): x - s P (iX_C) x = P rhs with s = -1 (forward) / +1 (adjoint).  The contraction
// factor rho_n = ||P iX_C|| <= (h/2) lam sum_k |d_k(t)| is evaluated every step and sets the
// iteration counts (warp-uniform).
//   SOLVER_FP64 : K fixed-point sweeps in FP64, K = ceil(log(2^-56)/log rho) - 1.
//   SOLVER_MIXED: mixed-precision iterative refinement.  FP32 sweeps give d = Ubar - P rhs,
//     the FP64 residual r = P rhs - z + s P (iX_C) z of z = P rhs + d is formed once with an
//     FP64 apply, and the FP32 correction e (I + ...)e = r is added in FP64.  Conversions
//     between f64 and f32 are done with integer bit operations because the hardware
//     conversions issue on the (slow) FP64 pipe.
// The adjoint sweep fuses the gradient quadrature of Eq. grad-int at the midpoints:
//   z_k = <Lbar, a_k Ubar>_F, y_k = <Lbar, a_k^+ Ubar>_F (summed over the tile's columns),
//   dP/dalpha1_kfs += -2h B_s Im(e^{i W t} z_k + e^{-i W t} y_k),
//   dP/dalpha2_kfs += -2h B_s Re(e^{i W t} z_k - e^{-i W t} y_k).
#pragma once

#include <cstdint>

#include "msqoc_internal.h"

namespace msqoc {

__host__ __device__ constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }
__host__ __device__ constexpr int next_pow2_c(int v) { return v <= 1 ? 1 : 2 * next_pow2_c((v + 1) / 2); }
__host__ __device__ constexpr int log2_c(int v) { return v <= 1 ? 0 : 1 + log2_c(v / 2); }

// ------------------------------------------------------------------ precision conversions
// f64 -> f32 rounded to nearest (ties away from zero) for |x| in [2^-126, 2^127); smaller
// magnitudes become signed zero.  Pure integer operations.
__device__ __forceinline__ float f32_of(double x) {
    unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned int ahi = static_cast<unsigned int>(bits >> 32) & 0x7fffffffu;
    bits += (1ull << 28);
    const unsigned int hi = static_cast<unsigned int>(bits >> 32);
    const unsigned int lo = static_cast<unsigned int>(bits);
    const unsigned int t = __funnelshift_l(lo, hi, 3);
    unsigned int fb = ((t ^ 0x40000000u) & 0x7fffffffu) | (hi & 0x80000000u);
    fb = (ahi < 0x38100000u) ? (hi & 0x80000000u) : fb;
    return __uint_as_float(fb);
}
// f32 -> f64 exactly for normal floats (denormals become signed zero).  Integer operations.
__device__ __forceinline__ double f64_of(float f) {
    const unsigned int fb = __float_as_uint(f);
    const unsigned int s = fb & 0x80000000u;
    const unsigned int a = fb & 0x7fffffffu;
    unsigned int hi = s | ((a >> 3) + 0x38000000u);
    unsigned int lo = a << 29;
    hi = (a < 0x00800000u) ? s : hi;
    lo = (a < 0x00800000u) ? 0u : lo;
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}
__device__ __forceinline__ float2 f32_of(double2 v) { return make_float2(f32_of(v.x), f32_of(v.y)); }
__device__ __forceinline__ double2 f64_of(float2 v) { return make_double2(f64_of(v.x), f64_of(v.y)); }

// ------------------------------------------------------------------ complex helpers
template <typename T2> struct cx;
template <> struct cx<double2> { using T = double; };
template <> struct cx<float2> { using T = float; };

// w += c * x
__device__ __forceinline__ void cmac(double2& w, double2 c, double2 x) {
    w.x = fma(c.x, x.x, w.x);
    w.x = fma(-c.y, x.y, w.x);
    w.y = fma(c.x, x.y, w.y);
    w.y = fma(c.y, x.x, w.y);
}
__device__ __forceinline__ void cmac(float2& w, float2 c, float2 x) {
    w.x = fmaf(c.x, x.x, w.x);
    w.x = fmaf(-c.y, x.y, w.x);
    w.y = fmaf(c.x, x.y, w.y);
    w.y = fmaf(c.y, x.x, w.y);
}
// w += conj(a) * b
__device__ __forceinline__ void cjmac(double2& w, double2 a, double2 b) {
    w.x = fma(a.x, b.x, w.x);
    w.x = fma(a.y, b.y, w.x);
    w.y = fma(a.x, b.y, w.y);
    w.y = fma(-a.y, b.x, w.y);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + s * (c * w) for s = +-1, complex c: 4 FMA (the signs are FMA operand negations)
template <int S>
__device__ __forceinline__ double2 cadd_scaled(double2 acc, double2 c, double2 w) {
    double2 r;
    if constexpr (S > 0) {
        r.x = fma(c.x, w.x, fma(-c.y, w.y, acc.x));
        r.y = fma(c.x, w.y, fma(c.y, w.x, acc.y));
    } else {
        r.x = fma(-c.x, w.x, fma(c.y, w.y, acc.x));
        r.y = fma(-c.x, w.y, fma(-c.y, w.x, acc.y));
    }
    return r;
}
template <int S>
__device__ __forceinline__ float2 cadd_scaled(float2 acc, float2 c, float2 w) {
    float2 r;
    if constexpr (S > 0) {
        r.x = fmaf(c.x, w.x, fmaf(-c.y, w.y, acc.x));
        r.y = fmaf(c.x, w.y, fmaf(c.y, w.x, acc.y));
    } else {
        r.x = fmaf(-c.x, w.x, fmaf(c.y, w.y, acc.x));
        r.y = fmaf(-c.x, w.y, fmaf(-c.y, w.x, acc.y));
    }
    return r;
}

// -d + s * (c * w): the FP64 residual of the refinement when the current iterate is b + d
// (the negations are FMA operand modifiers; nothing is materialized)
template <int S>
__device__ __forceinline__ double2 resid_from(double2 d, double2 c, double2 w) {
    double2 r;
    if constexpr (S > 0) {
        r.x = fma(c.x, w.x, fma(-c.y, w.y, -d.x));
        r.y = fma(c.x, w.y, fma(c.y, w.x, -d.y));
    } else {
        r.x = fma(-c.x, w.x, fma(c.y, w.y, -d.x));
        r.y = fma(-c.x, w.y, fma(-c.y, w.x, -d.y));
    }
    return r;
}
// 2 z - u as one FMA per component
__device__ __forceinline__ double2 reflect(double2 z, double2 u) {
    return make_double2(fma(2.0, z.x, -u.x), fma(2.0, z.y, -u.y));
}
// sqrt(l) for small l, as compile-time constants
__host__ __device__ constexpr double sqrt_small(int l) {
    return l == 0 ? 0.0 : l == 1 ? 1.0 : l == 2 ? 1.4142135623730951 : l == 3 ? 1.7320508075688772 : 2.0;
}

// ------------------------------------------------------------------ async bulk copies (TMA, 1D)
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy completing on an mbarrier (bytes multiple of 16, 16B-aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// shared -> global bulk copy (bulk-group completion)
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// bounded wait on an mbarrier phase; returns false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ------------------------------------------------------------------ per-thread neighbour lists
template <int L, int Q>
struct Fiber {
    static constexpr int NFIX = Q - 1;
    static constexpr int NA = NFIX > 0 ? NFIX : 1;
    int xo;            // offset of the fiber's first entry in a [cb][N] buffer
    int nb1[NA];       // offset of neighbour fiber (first entry) for subsystem k, entry 1
    int nb2[NA];       // entry 2 (exists when the level is interior)
    int sl1[NA];       // coefficient slot of entry 1
    int sl2[NA];
    bool two[NA];      // entry 2 exists (warp-uniform by construction)
    bool plus1[NA];    // entry 1 is the a_k (lowering, "+") term
    double w1[NA];     // product weight sqrt(level factor) of entry 1
    double w2[NA];

    __device__ void init(int c, int f, const ProbDev& pd) {
        constexpr int N = ipow_c(L, Q);
        xo = c * N + f * L;
#pragma unroll
        for (int k = 0; k < NFIX; ++k) {
            const int sf = ipow_c(L, Q - 2 - k);   // stride of subsystem k in fiber units
            const int lk = (f / sf) % L;
            if (lk < L - 1) {
                nb1[k] = c * N + (f + sf) * L;
                sl1[k] = (k * L + lk) * 2 + 0;
                plus1[k] = true;
                w1[k] = pd.wsq[2 * lk + 0];
                two[k] = lk > 0;
                nb2[k] = c * N + (f - (lk > 0 ? sf : 0)) * L;
                sl2[k] = (k * L + lk) * 2 + 1;
                w2[k] = pd.wsq[2 * lk + 1];
            } else {
                nb1[k] = c * N + (f - sf) * L;
                sl1[k] = (k * L + lk) * 2 + 1;
                plus1[k] = false;
                w1[k] = pd.wsq[2 * lk + 1];
                two[k] = false;
                nb2[k] = nb1[k];
                sl2[k] = sl1[k];
                w2[k] = 0.0;
            }
        }
    }
};

// w = (iX_C x) on the fiber: ladder terms of the last subsystem from registers (xr), the
// others from the shared buffer.  cf: per-slot coefficients i(h/2)sqrt(.)d_k for this step.
template <int L, int Q, typename T2>
__device__ __forceinline__ void apply_off(const T2* __restrict__ buf, const T2* __restrict__ cf,
                                          const Fiber<L, Q>& fb, const T2 (&xr)[L], T2 (&w)[L]) {
#pragma unroll
    for (int l = 0; l < L; ++l) {
        w[l].x = 0;
        w[l].y = 0;
    }
    constexpr int kl = Q - 1;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        if (l < L - 1) cmac(w[l], cf[(kl * L + l) * 2 + 0], xr[l + 1]);
        if (l > 0) cmac(w[l], cf[(kl * L + l) * 2 + 1], xr[l - 1]);
    }
#pragma unroll
    for (int k = 0; k < Fiber<L, Q>::NFIX; ++k) {
        const T2 c1 = cf[fb.sl1[k]];
        const T2* p1 = buf + fb.nb1[k];
#pragma unroll
        for (int l = 0; l < L; ++l) cmac(w[l], c1, p1[l]);
        if (fb.two[k]) {
            const T2 c2 = cf[fb.sl2[k]];
            const T2* p2 = buf + fb.nb2[k];
#pragma unroll
            for (int l = 0; l < L; ++l) cmac(w[l], c2, p2[l]);
        }
    }
}

// ------------------------------------------------------------------ shared memory layout
struct SweepSmem {
    size_t coef_d, coef_f, params, mbar, red, zy, galpha, D0, D1, FA, FB, H, UB0, UB1, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline SweepSmem sweep_layout(int q, int L, int N, int cb, int nthreads, int d, int solver,
                                                  bool bwd) {
    SweepSmem s{};
    const int nslot = q * L * 2;
    const int nwarps = nthreads / 32;
    const int V = next_pow2_c(4 * q);
    const size_t buf_d = size_t(cb) * N * 16, buf_f = size_t(cb) * N * 8;
    size_t o = 0;
    s.coef_d = o; o = align16(o + 2 * nslot * 16);
    s.coef_f = o; o = align16(o + 2 * nslot * 8);
    s.params = o; o = align16(o + 2 * 4 * 4);
    s.mbar = o;   o = align16(o + 2 * 8);
    s.red = o;    o = align16(o + (bwd ? size_t(2) * nwarps * V * 8 : 0));
    s.zy = o;     o = align16(o + (bwd ? size_t(2) * 4 * q * 8 : 0));
    s.galpha = o; o = align16(o + (bwd ? size_t(d) * 8 : 0));
    s.D0 = o;     o = align16(o + buf_d);
    s.D1 = o;     o = align16(o + (solver == SOLVER_FP64 ? buf_d : 0));
    s.FA = o;     o = align16(o + (solver == SOLVER_MIXED ? buf_f : 0));
    s.FB = o;     o = align16(o + (solver == SOLVER_MIXED ? buf_f : 0));
    s.H = o;      o = align16(o + (bwd ? 0 : buf_d));
    s.UB0 = o;    o = align16(o + (bwd ? buf_d : 0));
    s.UB1 = o;    o = align16(o + (bwd ? buf_d : 0));
    s.total = o;
    return s;
}

// ------------------------------------------------------------------ per-step coefficients
// Warp 0: slot (k, l, dir) -> i (h/2) sqrt(l+1) d_k (dir 0, a_k) or i (h/2) sqrt(l) conj(d_k)
// (dir 1, a_k^+); lane k' < NSLOT holds d_k of its slot's subsystem.  The iteration counts of
// the step (packed by step_counts in the controls kernel) are unpacked into prm.
template <int L, int Q>
__device__ __forceinline__ void step_coefficients(const ProbDev& pd, int lane, double2 dk, int cnt, double2* cfd,
                                                  float2* cff, int* prm) {
    constexpr int NSLOT = Q * L * 2;
    if (lane < NSLOT) {
        const int dir = lane & 1;
        const int l = (lane >> 1) % L;
        const bool valid = dir == 0 ? (l < L - 1) : (l > 0);
        const double s = pd.sc[2 * l + dir];
        double2 v = make_double2(0.0, 0.0);
        if (valid) v = dir == 0 ? make_double2(-s * dk.y, s * dk.x) : make_double2(s * dk.y, s * dk.x);
        cfd[lane] = v;
        cff[lane] = f32_of(v);
    }
    if (lane == 0) {
        prm[0] = cnt & 0xff;
        prm[1] = (cnt >> 8) & 0xff;
        prm[2] = (cnt >> 16) & 0xff;
        prm[3] = (cnt >> 24) & 0xff;
    }
}

// Barrier of the tile's threads; a warp barrier when the tile is a single warp (blockDim is
// uniform, so the branch is too).
__device__ __forceinline__ void tile_sync() {
    if (blockDim.x == 32)
        __syncwarp();
    else
        __syncthreads();
}
__device__ __forceinline__ int tile_sync_or(int p) {
    if (blockDim.x == 32) return __any_sync(0xffffffffu, p);
    return __syncthreads_or(p);
}

// ------------------------------------------------------------------ the sweep kernel
template <int L, int Q, int SOLVER, bool BWD>
__global__ void __launch_bounds__(MAX_TILE_THREADS, 1) k_sweep(const ProbDev pd, const int want_hist) {
    constexpr int N = ipow_c(L, Q);
    constexpr int F = N / L;
    constexpr int NSLOT = Q * L * 2;
    constexpr int S = BWD ? +1 : -1;       // sign of the preconditioned off-diagonal term
    constexpr int V = next_pow2_c(4 * Q);  // padded count of reduced gradient values
    constexpr int NH = log2_c(V);          // halving levels of the warp reduce-scatter

    extern __shared__ __align__(128) unsigned char smem[];
    const SweepSmem lay = sweep_layout(Q, L, N, pd.cb, pd.nthreads, pd.d, SOLVER, BWD);
    double2* coef_d = reinterpret_cast<double2*>(smem + lay.coef_d);
    float2* coef_f = reinterpret_cast<float2*>(smem + lay.coef_f);
    int* params = reinterpret_cast<int*>(smem + lay.params);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + lay.mbar);
    double* red = reinterpret_cast<double*>(smem + lay.red);
    double* zy = reinterpret_cast<double*>(smem + lay.zy);
    double* galpha = reinterpret_cast<double*>(smem + lay.galpha);
    double2* D0 = reinterpret_cast<double2*>(smem + lay.D0);
    double2* D1 = reinterpret_cast<double2*>(smem + lay.D1);
    float2* FA = reinterpret_cast<float2*>(smem + lay.FA);
    float2* FB = reinterpret_cast<float2*>(smem + lay.FB);
    double2* H = reinterpret_cast<double2*>(smem + lay.H);
    double2* UB0 = reinterpret_cast<double2*>(smem + lay.UB0);
    double2* UB1 = reinterpret_cast<double2*>(smem + lay.UB1);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int cb = pd.cb;
    const int tile = blockIdx.x;
    const int m = tile / pd.nblk + 1;               // window, 1-based
    const int blk = tile % pd.nblk;
    const int64_t n0 = ((int64_t)(m - 1) * pd.nsteps) / pd.M;
    const int64_t n1 = ((int64_t)m * pd.nsteps) / pd.M;
    const int ns = static_cast<int>(n1 - n0);
    const int nact = cb * F;
    const bool act = tid < nact;
    const int tt = act ? tid : nact - 1;            // inactive lanes mirror a valid fiber, store nothing
    const int c = tt % cb;
    const int f = pd.fiber_order[tt / cb];
    const int col = blk * cb + c;
    const size_t blk_elems = size_t(cb) * N;
    const uint32_t blk_bytes = static_cast<uint32_t>(blk_elems * sizeof(double2));

    Fiber<L, Q> fb;
    fb.init(c, f, pd);

    // preconditioner on the fiber: P (forward) or conj(P) (adjoint)
    double2 Pd[L];
    float2 Pf[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        double2 p = pd.P[f * L + l];
        if (BWD) p.y = -p.y;
        Pd[l] = p;
        Pf[l] = f32_of(p);
    }

    // initial state: forward U^m(t_{m-1}) = W^{m-1} (identity embedding for m = 1);
    // adjoint Lambda^m(t_m) from the terminal kernel
    double2 u[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const int i = f * L + l;
        if (BWD) {
            u[l] = pd.Lterm[(size_t(m - 1) * pd.E + col) * N + i];
        } else if (m == 1) {
            u[l] = make_double2(pd.emb[col] == i ? 1.0 : 0.0, 0.0);
        } else {
            u[l] = pd.W[(size_t(m - 2) * pd.E + col) * N + i];
        }
    }

    if (BWD) {
        for (int j = tid; j < pd.d; j += blockDim.x) galpha[j] = 0.0;
        if (tid == 0) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
            fence_mbar_init();
        }
        tile_sync();
        if (tid == 0 && ns > 0) {
            const int64_t n = n0 + ns - 1;
            mbar_expect_tx(&mbar[0], blk_bytes);
            bulk_g2s(UB0, pd.hist + (size_t(n) * pd.nblk + blk) * blk_elems, blk_bytes, &mbar[0]);
        }
    }

    // warp 0 keeps d_k of the next step in registers (lane -> subsystem of its slot)
    const int my_k = (lane < NSLOT) ? (lane / (2 * L)) : 0;
    double2 dk_next = make_double2(0.0, 0.0);
    int cnt_next = 0;
    auto load_ctrl = [&](int64_t n) {
        if (warp == 0) {
            dk_next = lane < NSLOT ? pd.ctrl[size_t(n) * pd.q + my_k] : make_double2(0.0, 0.0);
            cnt_next = pd.spl[n].cnt;
        }
    };
    // warp 0 lanes that scatter gradient entries: (k, f, j) with 3 active splines per carrier
    const int nscat = pd.nfsum * 3;

    bool timed_out = false;
    int fsel = 0;
    double2* Dc = D0;   // FP64-solver ping-pong buffers
    double2* Dn = D1;
    load_ctrl(BWD ? n0 + ns - 1 : n0);

    for (int jj = 0; jj < ns; ++jj) {
        const int j = BWD ? ns - 1 - jj : jj;      // local step index
        const int64_t n = n0 + j;                  // global step index
        const int par = jj & 1;
        double2* cfd = coef_d + par * NSLOT;
        float2* cff = coef_f + par * NSLOT;
        int* prm = params + par * 4;

        if (warp == 0) {
            const double2 dk = dk_next;
            const int cnt = cnt_next;
            if (jj + 1 < ns) load_ctrl(BWD ? n - 1 : n + 1);
            step_coefficients<L, Q>(pd, lane, dk, cnt, cfd, cff, prm);
        }
        // adjoint: warp 0 fetches what the gradient fold of the previous step (n + 1) needs
        // now, so the loads are in flight during the solve
        Spline4 sp_prev{};
        double2 ph_prev = make_double2(0.0, 0.0);
        if (BWD && jj > 0 && warp == 0) {
            sp_prev = pd.spl[n + 1];
            if (lane < nscat) ph_prev = pd.phase[size_t(n + 1) * pd.nfsum + lane / 3];
        }

        // right-hand side of the preconditioned step equation: b = P u (conj(P) for the adjoint)
        double2 b[L];
#pragma unroll
        for (int l = 0; l < L; ++l) b[l] = cmul(Pd[l], u[l]);

        double2 z[L];   // the midpoint state being solved for (Ubar or Lbar)

        if constexpr (SOLVER == SOLVER_FP64) {
            // Dc/Dn alternate on every write (persisting across steps): a buffer is never
            // rewritten before the sync that follows its last read.
#pragma unroll
            for (int l = 0; l < L; ++l) z[l] = b[l];
            if (act) {
#pragma unroll
                for (int l = 0; l < L; ++l) Dc[fb.xo + l] = z[l];
            }
            tile_sync();
            // first sync of the step: publish the previous step's history block / issue prefetch
            if (!BWD && want_hist && tid == 0 && jj > 0) {
                fence_proxy_async_smem();
                bulk_s2g(pd.hist + (size_t(n - 1) * pd.nblk + blk) * blk_elems, H, blk_bytes);
            }
            if (BWD && tid == 0 && jj + 1 < ns) {
                const int nx = (jj + 1) & 1;
                mbar_expect_tx(&mbar[nx], blk_bytes);
                bulk_g2s(nx ? UB1 : UB0, pd.hist + (size_t(n - 1) * pd.nblk + blk) * blk_elems, blk_bytes,
                         &mbar[nx]);
            }
            const int K = prm[0];
            for (int it = 0; it < K; ++it) {
                if (it > 0) {
                    if (act) {
#pragma unroll
                        for (int l = 0; l < L; ++l) Dc[fb.xo + l] = z[l];
                    }
                    tile_sync();
                }
                double2 w[L];
                apply_off<L, Q, double2>(Dc, cfd, fb, z, w);
#pragma unroll
                for (int l = 0; l < L; ++l) z[l] = cadd_scaled<S>(b[l], Pd[l], w[l]);
                double2* tmp = Dc;
                Dc = Dn;
                Dn = tmp;
            }
            (void)Dn;
        } else {
            // ---- FP32 stage: d = Ubar - b from the preconditioned fixed point d = s P w(b + d)
            float2 bf[L], df[L], y[L];
#pragma unroll
            for (int l = 0; l < L; ++l) {
                bf[l] = f32_of(b[l]);
                y[l] = bf[l];
            }
            {
                float2* Fb = fsel ? FB : FA;
                fsel ^= 1;
                if (act) {
#pragma unroll
                    for (int l = 0; l < L; ++l) Fb[fb.xo + l] = y[l];
                }
                tile_sync();
                if (!BWD && want_hist && tid == 0 && jj > 0) {
                    fence_proxy_async_smem();
                    bulk_s2g(pd.hist + (size_t(n - 1) * pd.nblk + blk) * blk_elems, H, blk_bytes);
                }
                if (BWD && tid == 0 && jj + 1 < ns) {
                    const int nx = (jj + 1) & 1;
                    mbar_expect_tx(&mbar[nx], blk_bytes);
                    bulk_g2s(nx ? UB1 : UB0, pd.hist + (size_t(n - 1) * pd.nblk + blk) * blk_elems, blk_bytes,
                             &mbar[nx]);
                }
                float2 w[L];
                apply_off<L, Q, float2>(Fb, cff, fb, y, w);
#pragma unroll
                for (int l = 0; l < L; ++l) df[l] = cadd_scaled<S>(make_float2(0.f, 0.f), Pf[l], w[l]);
            }
            const int j1 = prm[0], j2 = prm[1], R = prm[2];
            for (int it = 1; it < j1; ++it) {
#pragma unroll
                for (int l = 0; l < L; ++l) y[l] = make_float2(bf[l].x + df[l].x, bf[l].y + df[l].y);
                float2* Fb = fsel ? FB : FA;
                fsel ^= 1;
                if (act) {
#pragma unroll
                    for (int l = 0; l < L; ++l) Fb[fb.xo + l] = y[l];
                }
                tile_sync();
                float2 w[L];
                apply_off<L, Q, float2>(Fb, cff, fb, y, w);
#pragma unroll
                for (int l = 0; l < L; ++l) df[l] = cadd_scaled<S>(make_float2(0.f, 0.f), Pf[l], w[l]);
            }
            // ---- FP64 refinement: z = b + d, residual r = (b - z) + s P w(z), correction in FP32.
            // dacc accumulates z - b (= d, then d + e, ...); b - z = -dacc up to the rounding of z.
            double2 dacc[L];
#pragma unroll
            for (int l = 0; l < L; ++l) {
                dacc[l] = f64_of(df[l]);
                z[l] = make_double2(b[l].x + dacc[l].x, b[l].y + dacc[l].y);
            }
            for (int pass = 0;; ++pass) {
                if (act) {
#pragma unroll
                    for (int l = 0; l < L; ++l) D0[fb.xo + l] = z[l];
                }
                tile_sync();
                double2 w[L];
                apply_off<L, Q, double2>(D0, cfd, fb, z, w);
                float2 rf[L], e[L];
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    const double2 r = resid_from<S>(dacc[l], Pd[l], w[l]);
                    rf[l] = f32_of(r);
                    e[l] = rf[l];
                }
                for (int it = 0; it < j2; ++it) {
                    float2* Fb = fsel ? FB : FA;
                    fsel ^= 1;
                    if (act) {
#pragma unroll
                        for (int l = 0; l < L; ++l) Fb[fb.xo + l] = e[l];
                    }
                    tile_sync();
                    float2 wf[L];
                    apply_off<L, Q, float2>(Fb, cff, fb, e, wf);
#pragma unroll
                    for (int l = 0; l < L; ++l) e[l] = cadd_scaled<S>(rf[l], Pf[l], wf[l]);
                }
                double2 ed[L];
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    ed[l] = f64_of(e[l]);
                    z[l] = make_double2(z[l].x + ed[l].x, z[l].y + ed[l].y);
                }
                if (pass + 1 >= R) break;
                // another pass: dacc accumulates the correction; it rewrites D0, so every thread
                // must be done reading it
#pragma unroll
                for (int l = 0; l < L; ++l) dacc[l] = make_double2(dacc[l].x + ed[l].x, dacc[l].y + ed[l].y);
                tile_sync();
            }
        }

        if (tid == 0 && prm[3]) atomicOr(pd.status, ST_SOLVER_RANGE);

        if constexpr (!BWD) {
            // ---- history of midpoint states for the adjoint sweep (async bulk store)
            if (want_hist) {
                if (tid == 0) bulk_wait_read_all();
                tile_sync();
                if (act) {
#pragma unroll
                    for (int l = 0; l < L; ++l) H[fb.xo + l] = z[l];
                }
                fence_proxy_async_smem();
            }
#pragma unroll
            for (int l = 0; l < L; ++l) u[l] = reflect(z[l], u[l]);
        } else {
            // ---- gradient quadrature on the midpoints (fused): needs Ubar_n of the tile
            const int slot = jj & 1;
            double2* UB = slot ? UB1 : UB0;
            const bool ok = mbar_wait(&mbar[slot], (jj >> 1) & 1);
            if (tile_sync_or(!ok)) {
                timed_out = true;
                break;
            }
            double acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = 0.0;
            {
                // last subsystem (stride 1) from the fiber itself
                constexpr int kl = Q - 1;
                double2 zq = make_double2(0.0, 0.0), yq = make_double2(0.0, 0.0);
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    // z: conj(Lbar_l) sqrt(l+1) Ubar_{l+1};  y: conj(Lbar_l) sqrt(l) Ubar_{l-1}
                    if (l < L - 1) {
                        const double wz = sqrt_small(l + 1);   // folded after unrolling
                        if (wz == 1.0) {
                            cjmac(zq, z[l], UB[fb.xo + l + 1]);
                        } else {
                            double2 p = make_double2(0.0, 0.0);
                            cjmac(p, z[l], UB[fb.xo + l + 1]);
                            zq.x = fma(wz, p.x, zq.x);
                            zq.y = fma(wz, p.y, zq.y);
                        }
                    }
                    if (l > 0) {
                        const double wy = sqrt_small(l);
                        if (wy == 1.0) {
                            cjmac(yq, z[l], UB[fb.xo + l - 1]);
                        } else {
                            double2 p = make_double2(0.0, 0.0);
                            cjmac(p, z[l], UB[fb.xo + l - 1]);
                            yq.x = fma(wy, p.x, yq.x);
                            yq.y = fma(wy, p.y, yq.y);
                        }
                    }
                }
                acc[4 * kl + 0] = zq.x;
                acc[4 * kl + 1] = zq.y;
                acc[4 * kl + 2] = yq.x;
                acc[4 * kl + 3] = yq.y;
            }
#pragma unroll
            for (int k = 0; k < Fiber<L, Q>::NFIX; ++k) {
                double2 p = make_double2(0.0, 0.0);
                const double2* q1 = UB + fb.nb1[k];
#pragma unroll
                for (int l = 0; l < L; ++l) cjmac(p, z[l], q1[l]);
                const double px = fb.w1[k] * p.x, py = fb.w1[k] * p.y;
                acc[4 * k + 0] = fb.plus1[k] ? px : 0.0;
                acc[4 * k + 1] = fb.plus1[k] ? py : 0.0;
                acc[4 * k + 2] = fb.plus1[k] ? 0.0 : px;
                acc[4 * k + 3] = fb.plus1[k] ? 0.0 : py;
                if (fb.two[k]) {
                    double2 p2 = make_double2(0.0, 0.0);
                    const double2* q2 = UB + fb.nb2[k];
#pragma unroll
                    for (int l = 0; l < L; ++l) cjmac(p2, z[l], q2[l]);
                    acc[4 * k + 2] = fb.w2[k] * p2.x;
                    acc[4 * k + 3] = fb.w2[k] * p2.y;
                }
            }
            if (!act) {
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = 0.0;
            }
            // warp reduce-scatter: lane ends with value (lane >> (5 - NH)) summed over the warp
            {
                int cnt = V;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    if (cnt > 1) {
                        const int half = cnt >> 1;
                        const bool upper = (lane & o) != 0;
#pragma unroll
                        for (int q2 = 0; q2 < V / 2; ++q2) {
                            if (q2 < half) {
                                const double send = upper ? acc[q2] : acc[q2 + half];
                                const double keep = upper ? acc[q2 + half] : acc[q2];
                                acc[q2] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                            }
                        }
                        cnt = half;
                    } else {
                        acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
                    }
                }
                const int vi = lane >> (5 - NH);
                if ((lane & ((1 << (5 - NH)) - 1)) == 0) red[(par * nwarps + warp) * V + vi] = acc[0];
            }
            // Lambda_n = 2 Lbar - Lambda_{n+1}
#pragma unroll
            for (int l = 0; l < L; ++l) u[l] = reflect(z[l], u[l]);
        }

        // warp 0 folds the previous step's reduced products into the alpha-gradient
        if (BWD && jj > 0 && warp == 0) {
            // (the sync that published red[par ^ 1] was this step's first sync)
            const int pp = par ^ 1;
            const int64_t np = n + 1;   // global step of the previous iteration
            if (lane < 4 * Q) {
                double s = 0.0;
                for (int w2 = 0; w2 < nwarps; ++w2) s += red[(pp * nwarps + w2) * V + lane];
                zy[pp * 4 * Q + lane] = s;
            }
            __syncwarp();
            const Spline4 sp = sp_prev;
            const int s0 = sp.s;
            for (int i = lane; i < nscat; i += 32) {
                const int kf = i / 3, jw = i % 3;
                int k = 0;
                while (k + 1 < Q && pd.cof[k + 1] <= kf) ++k;
                const double2 zk = make_double2(zy[pp * 4 * Q + 4 * k + 0], zy[pp * 4 * Q + 4 * k + 1]);
                const double2 yk = make_double2(zy[pp * 4 * Q + 4 * k + 2], zy[pp * 4 * Q + 4 * k + 3]);
                const double2 ph = i == lane ? ph_prev : pd.phase[size_t(np) * pd.nfsum + kf];
                const double wgt = -2.0 * pd.h * (jw == 0 ? sp.w0 : (jw == 1 ? sp.w1 : sp.w2));
                const double A = zk.y + yk.y, B = zk.x - yk.x;
                const int idx = (kf * pd.d1 + s0 + jw) * 2;
                galpha[idx + 0] += wgt * fma(ph.x, A, ph.y * B);
                galpha[idx + 1] += wgt * fma(ph.x, B, -ph.y * A);
            }
        }
    }

    if (!timed_out) {
        tile_sync();
        if (!BWD) {
            if (want_hist && tid == 0 && ns > 0) {
                fence_proxy_async_smem();
                bulk_s2g(pd.hist + (size_t(n0 + ns - 1) * pd.nblk + blk) * blk_elems, H, blk_bytes);
                bulk_wait_all();
            }
            if (act) {
#pragma unroll
                for (int l = 0; l < L; ++l) pd.Uend[(size_t(m - 1) * pd.E + col) * N + f * L + l] = u[l];
            }
        } else {
            if (warp == 0 && ns > 0) {
                const int pp = (ns - 1) & 1;
                const int64_t np = n0;
                if (lane < 4 * Q) {
                    double s = 0.0;
                    for (int w2 = 0; w2 < nwarps; ++w2) s += red[(pp * nwarps + w2) * V + lane];
                    zy[pp * 4 * Q + lane] = s;
                }
                __syncwarp();
                const Spline4 sp = pd.spl[np];
                const int s0 = sp.s;
                for (int i = lane; i < nscat; i += 32) {
                    const int kf = i / 3, jw = i % 3;
                    int k = 0;
                    while (k + 1 < Q && pd.cof[k + 1] <= kf) ++k;
                    const double2 zk = make_double2(zy[pp * 4 * Q + 4 * k + 0], zy[pp * 4 * Q + 4 * k + 1]);
                    const double2 yk = make_double2(zy[pp * 4 * Q + 4 * k + 2], zy[pp * 4 * Q + 4 * k + 3]);
                    const double2 ph = pd.phase[size_t(np) * pd.nfsum + kf];
                    const double wgt = -2.0 * pd.h * (jw == 0 ? sp.w0 : (jw == 1 ? sp.w1 : sp.w2));
                    const double A = zk.y + yk.y, B = zk.x - yk.x;
                    const int idx = (kf * pd.d1 + s0 + jw) * 2;
                    galpha[idx + 0] += wgt * fma(ph.x, A, ph.y * B);
                    galpha[idx + 1] += wgt * fma(ph.x, B, -ph.y * A);
                }
            }
            tile_sync();
            for (int jx = tid; jx < pd.d; jx += blockDim.x) pd.gpart[size_t(tile) * pd.d + jx] = galpha[jx];
            if (act) {
#pragma unroll
                for (int l = 0; l < L; ++l) pd.Lam0[(size_t(m - 1) * pd.E + col) * N + f * L + l] = u[l];
            }
        }
    } else if (tid == 0) {
        atomicOr(pd.status, ST_TIMEOUT);
    }
}

}  // namespace msqoc
