// Pieces shared by the sweep kernel families (msqoc_sweep.cuh: one thread per fiber;
// msqoc_sweep_pair.cuh: a lane pair, or for 2-level subsystems a lane quad, per fiber):
// precision conversions, 1D bulk async copies and bounded mbarrier waits, the per-thread
// neighbour lists, the shared-memory layout, the tile barrier, the spline origin of a window
// and the write-out of a tile's gradient partial.
#pragma once

#include <cstdint>

#include "msqoc_internal.h"
#include "msqoc_split.cuh"

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

// The same conversions of a state entry with a per-column binary scale 2^-sh (|sh| <=
// SCALE_SHIFT_MAX): f32_of_scaled gives x 2^-sh rounded to f32 as above, f64_of_scaled gives
// f 2^sh exactly.  The scale is an offset of the exponent field, applied to the high word (no
// FP64 instruction); the per-column constants are formed once per launch (ColScale).  Scaled
// magnitudes below 2^-126 become signed zero.  The column scale bounds every scaled entry, the
// corrections and residuals included, below 1, so no overflow handling is needed.
constexpr int SCALE_SHIFT_MAX = 896;
struct ColScale {
    unsigned int sub;    // sh 2^20 (mod 2^32): subtracted from the high word
    int flush;           // |high word| below this flushes: 0x38100000 + sh 2^20
    unsigned int bias;   // f32 -> f64 exponent bias with the scale: 0x38000000 + sh 2^20
};
__device__ __forceinline__ ColScale col_scale(int sh) {
    const unsigned int s20 = static_cast<unsigned int>(sh) * (1u << 20);
    return ColScale{s20, 0x38100000 + sh * (1 << 20), 0x38000000u + s20};
}
__device__ __forceinline__ float f32_of_scaled(double x, const ColScale& cs) {
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned int hi0 = static_cast<unsigned int>(bits >> 32);
    const unsigned int sgn = hi0 & 0x80000000u;
    const int ahi = static_cast<int>(hi0 & 0x7fffffffu);
    const unsigned long long adj = (static_cast<unsigned long long>(hi0 - cs.sub) << 32 |
                                    static_cast<unsigned int>(bits)) + (1ull << 28);
    const unsigned int hi = static_cast<unsigned int>(adj >> 32);
    const unsigned int lo = static_cast<unsigned int>(adj);
    const unsigned int t = __funnelshift_l(lo, hi, 3);
    const unsigned int fb = ((t ^ 0x40000000u) & 0x7fffffffu) | sgn;
    return __uint_as_float(ahi < cs.flush ? sgn : fb);
}
__device__ __forceinline__ double f64_of_scaled(float f, const ColScale& cs) {
    const unsigned int fb = __float_as_uint(f);
    const unsigned int s = fb & 0x80000000u;
    const unsigned int a = fb & 0x7fffffffu;
    unsigned int hi = s | ((a >> 3) + cs.bias);
    unsigned int lo = a << 29;
    hi = (a < 0x00800000u) ? s : hi;
    lo = (a < 0x00800000u) ? 0u : lo;
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}
__device__ __forceinline__ float2 f32_of_scaled(double2 v, const ColScale& cs) {
    return make_float2(f32_of_scaled(v.x, cs), f32_of_scaled(v.y, cs));
}
__device__ __forceinline__ double2 f64_of_scaled(float2 v, const ColScale& cs) {
    return make_double2(f64_of_scaled(v.x, cs), f64_of_scaled(v.y, cs));
}
// biased exponent field of a double (0 for zero and subnormals)
__device__ __forceinline__ int exp_field(double x) {
    return static_cast<int>(static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7ff;
}
// Scale of a column of the mixed-precision solver: the step preserves every column's 2-norm (the
// Cayley map of a Hermitian H is unitary, forward and adjoint), so the largest entry exponent
// ce of the column's state at the start of a launch bounds every entry of every later step by
// 2^(ce - 1022) sqrt(N) < 2^(ce - 1018) (N <= 256).  Entries scaled by 2^-sh with
// sh = ce - 1018 stay below 1, and the FP32 stage's range limits apply relative to the column
// norm instead of to absolute magnitudes (the flush below 2^-126 of the column's scale).
__device__ __forceinline__ int column_shift(int ce) {
    if (ce == 0) return 0;   // an all-zero column
    const int sh = ce - 1018;
    return sh > SCALE_SHIFT_MAX ? SCALE_SHIFT_MAX : (sh < -SCALE_SHIFT_MAX ? -SCALE_SHIFT_MAX : sh);
}
// tile columns at most (E = 2^q for 2-level shapes, q <= MAXQ)
constexpr int MAX_TILE_COLS = 1 << MAXQ;

template <typename T2> struct cx;
template <> struct cx<double2> { using T = double; };
template <> struct cx<float2> { using T = float; };

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
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
// polls of a bounded mbarrier wait before it gives up: a poll of a phase that does not complete
// suspends ~3.8 us on this GPU (measured by msqoc_selftest_bounded_wait), so a stuck wait ends
// after about a second
constexpr int64_t MBAR_WAIT_SPINS = int64_t(1) << 18;
// bounded wait on an mbarrier phase; returns false if it gave up after max_spins polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int64_t max_spins = MBAR_WAIT_SPINS) {
    const uint32_t a = smem_u32(bar);
    for (int64_t it = 0; it < max_spins; ++it) {
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
// exchange-coupled pairs whose sources a fiber keeps precomputed (more use the general form)
constexpr int MAXEXF = 6;
template <int L, int Q>
struct Fiber {
    static constexpr int NFIX = Q - 1;
    static constexpr int NA = NFIX > 0 ? NFIX : 1;
    int f;             // fiber index
    int xo;            // offset of the fiber's first entry in a [cb][N] buffer
    int nb1[NA];       // offset of neighbour fiber (first entry) for subsystem k, entry 1
    int nb2[NA];       // entry 2 (exists when the level is interior)
    int sl1[NA];       // coefficient slot of entry 1
    int sl2[NA];
    bool two[NA];      // entry 2 exists (warp-uniform by construction)
    bool plus1[NA];    // entry 1 is the a_k (lowering, "+") term
    double w1[NA];     // product weight sqrt(level factor) of entry 1
    double w2[NA];
    // dipole exchange of a 2-level (qubit) problem with at most MAXEXF coupled pairs: the source
    // of pair e's term for entry l (an entry index in a [cb][N] buffer, or the buffer's zero
    // entry when the pair gives that entry no term), so the apply is the same for every lane
    int exs[MAXEXF][L];

    // c: tile column, f: fiber, zero: index of the shared buffers' zero entry
    __device__ void init(int c, int f, const ProbDev& pd, int zero) {
        constexpr int N = ipow_c(L, Q);
        this->f = f;
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
        if constexpr (L == 2 && Q >= 2) init_exchange(pd, zero);
    }

    // For 2 levels every weight of the exchange terms is 1 and a coupled pair (j, k) gives the
    // fiber at most one term.  k the last subsystem: level 1 of the fiber takes level 0 of the
    // fiber with l_j + 1 (a_k^+ a_j, when l_j = 0), or level 0 takes level 1 of the fiber with
    // l_j - 1 (a_k a_j^+, when l_j = 1).  k not the last: every entry takes the same level of
    // the fiber with (l_j + 1, l_k - 1) when (l_j, l_k) = (0, 1), or (l_j - 1, l_k + 1) when
    // (1, 0).  Computed once per launch instead of in every apply.
    __device__ void init_exchange(const ProbDev& pd, int zero) {
#pragma unroll
        for (int e = 0; e < MAXEXF; ++e) {
#pragma unroll
            for (int l = 0; l < L; ++l) exs[e][l] = zero;
            if (e < pd.nex) {
                const int j = pd.ex_j[e], k = pd.ex_k[e];
                int sfj = 1, sfk = 1;                          // fiber strides (j is never the last)
                for (int t = j; t < Q - 2; ++t) sfj *= 2;
                for (int t = k; t < Q - 2; ++t) sfk *= 2;
                const int lj = (f / sfj) % 2;
                if (k == Q - 1) {
                    if (lj == 0)
                        exs[e][1] = xo + sfj * 2;
                    else
                        exs[e][0] = xo - sfj * 2 + 1;
                } else {
                    const int lk = (f / sfk) % 2;
#pragma unroll
                    for (int l = 0; l < L; ++l) {
                        if (lk == 1 && lj == 0) exs[e][l] = xo + (sfj - sfk) * 2 + l;
                        if (lk == 0 && lj == 1) exs[e][l] = xo + (sfk - sfj) * 2 + l;
                    }
                }
            }
        }
    }
};

// ------------------------------------------------------------------ shared memory layout
// Per-slot arrays are sized for the two windows a tile can cover.  Lane-pair tiles (pair = 1)
// keep each coefficient in the form of either part, so their coefficient arrays are twice as
// large.
struct SweepSmem {
    size_t coef_d, coef_f, coef_s, params, mbar, red, zy, galpha, gdf, cq, D0, D1, FA, FB, H, UB0, UB1, total;
};
// steps between flushes of the mixed solver's two-float gradient accumulator into the FP64 one
constexpr int FOLD_FLUSH = 8;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline SweepSmem sweep_layout(int q, int L, int N, int cpt, int nthreads, int gmax, int solver,
                                                  bool bwd, int pair, int hdepth = 1) {
    SweepSmem s{};
    const int nslot = q * L * 2;
    const int nwarps = nthreads / 32;
    const int ncoef = pair ? 2 : 1;
    int V = 1;
    while (V < 4 * q) V <<= 1;
    // apply buffers hold cpt N entries plus a zero entry (index cpt N, never written by the
    // sweeps: the source of the exchange terms an entry does not have)
    const size_t buf_d = (size_t(cpt) * N + 1) * 16, buf_f = (size_t(cpt) * N + 1) * 8;
    size_t o = 0;
    s.coef_d = o; o = align16(o + size_t(2) * 2 * ncoef * nslot * 16);  // [parity][slot][part][NSLOT]
    s.coef_f = o; o = align16(o + size_t(2) * 2 * ncoef * nslot * 8);
    // the coefficients split into two floats (hi, lo) for the compensated apply of the mixed
    // solver's one-thread families
    s.coef_s = o; o = align16(o + (!pair && solver == SOLVER_MIXED ? size_t(2) * 2 * nslot * 16 : 0));
    s.params = o; o = align16(o + 2 * 2 * 4 * 4);                      // [parity][slot][4]
    s.mbar = o;   o = align16(o + 2 * 8);
    s.red = o;    o = align16(o + (bwd ? size_t(2) * 2 * nwarps * V * 8 : 0));   // [parity][slot][warp][V]
    s.zy = o;     o = align16(o + (bwd ? size_t(2) * 2 * 4 * q * 8 : 0));        // [parity][slot][4q]
    s.galpha = o; o = align16(o + (bwd ? size_t(2) * gmax * 8 : 0));             // [slot][nfsum][gspan][2]
    // the mixed solver's one-thread families: the same, two-float, holding the last steps' terms
    s.gdf = o;    o = align16(o + (bwd && !pair && solver == SOLVER_MIXED ? size_t(2) * gmax * 8 : 0));
    // the mixed solver's one-thread families: per fiber entry the third parts of the splits of
    // 2 kappa and P (the compensated state update)
    s.cq = o;     o = align16(o + (!pair && solver == SOLVER_MIXED ? size_t(N) * 16 : 0));
    s.D0 = o;     o = align16(o + buf_d);
    s.D1 = o;     o = align16(o + (solver == SOLVER_FP64 ? buf_d : 0));
    s.FA = o;     o = align16(o + (solver == SOLVER_MIXED ? buf_f : 0));
    s.FB = o;     o = align16(o + (solver == SOLVER_MIXED ? buf_f : 0));
    // history staging: hdepth blocks of cpt N states (forward H; adjoint UB0 / UB1, one group each)
    const size_t hist_b = size_t(hdepth) * cpt * N * 16;
    s.H = o;      o = align16(o + (bwd ? 0 : hist_b));
    s.UB0 = o;    o = align16(o + (bwd ? hist_b : 0));
    s.UB1 = o;    o = align16(o + (bwd ? hist_b : 0));
    s.total = o;
    return s;
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


// first spline active at the midpoint of global step n (the controls kernel's spline table
// holds the same index for every step)
__device__ __forceinline__ int spline_first(const ProbDev& pd, int64_t n) {
    return spline_index((double(n) + 0.5) * pd.h, pd.dtau, pd.d1);
}

// The tile's alpha-gradient partial gp[d] ([carrier][spline][re, im]) from the window-local
// sums of its slots (slot s holds splines [slo_s, slo_s + gspan) of every carrier at
// galpha + s gmax; slo_1 < 0: one slot), stored (first launch of the adjoint) or added.  Kept
// out of line: it runs once per launch, and inlined into the lane-pair adjoint of some shapes
// it crashed the assembler.
static __device__ __noinline__ void store_grad_partial(double* gp, const double* galpha, const ProbDev& pd, int gmax,
                                                int slo_0, int slo_1, bool first) {
    for (int jx = threadIdx.x; jx < pd.d; jx += blockDim.x) {
        const int kf = jx / (2 * pd.d1), sx = (jx >> 1) - kf * pd.d1;
        const int l0 = sx - slo_0, l1 = sx - slo_1;
        double v = 0.0;
        if (l0 >= 0 && l0 < pd.gspan) v += galpha[(kf * pd.gspan + l0) * 2 + (jx & 1)];
        if (slo_1 >= 0 && l1 >= 0 && l1 < pd.gspan) v += galpha[gmax + (kf * pd.gspan + l1) * 2 + (jx & 1)];
        gp[jx] = first ? v : gp[jx] + v;
    }
}

// first global step of local window m (1-based); window m owns [win_start(m), win_start(m + 1))
// of the whole problem's grid
__device__ __forceinline__ int64_t win_start(const ProbDev& pd, int m) {
    return (static_cast<int64_t>(pd.m_off + m - 1) * pd.nsteps) / pd.M_glob;
}

}  // namespace msqoc
