// Forward and adjoint sweeps with a lane pair per fiber (sm_103a): the variant of the sweeps of
// msqoc_sweep.cuh (same tiles, step equation, solvers, history and fused gradient quadrature)
// for problems whose tiles are too few to fill the GPU.
//
// A warp issues one FP64 instruction per 64 cycles on its SM sub-partition, so when an SM holds
// few warps a step's latency is set by the FP64 instruction count of its threads.  Here the two
// threads of a pair (lanes 2i, 2i + 1) share a fiber: one computes the real, the other the
// imaginary component of every complex result, which halves each thread's FP64 instructions
// (the other component comes from the partner lane by a shuffle, or from shared memory).  The
// cost is twice the threads and a lower register budget (384-thread tiles), so the one-thread
// family stays the choice for problems that fill the GPU.
//
// The same kernel with SPLIT = 2 is the lane-quad family for 2-level subsystems: four threads
// per fiber, a lane pair per entry of the fiber (lanes 4i + 2e and 4i + 2e + 1 own entry e).
// Each thread then computes one component of one entry, half of a lane pair's work; the
// entry the pair does not hold (the in-fiber ladder term) is read from the shared buffer like
// any neighbour.  Tiles of up to 384 threads, like lane pairs (at 512 threads the 128-register
// budget cost the adjoint 2-4%).
#pragma once

#include "msqoc_sweep_common.cuh"

namespace msqoc {

// ------------------------------------------------------------------ complex arithmetic over a lane pair
// The two threads of a pair (lanes 2i and 2i + 1) own the same fiber.  Part p = lane & 1
// computes component p (0: real, 1: imaginary) of every complex result and holds component p of
// the fiber's state, so each part does half of the fiber's FP64 work.  A product c x costs a
// part two real FMAs:
//   (c x)_p = ca x_p + cb x_{1-p},   (ca, cb) = (Re c, -Im c) for p = 0, (Re c, Im c) for p = 1,
// so coefficients are kept as per-part pairs (ca, cb).  The other component of a value the
// part holds comes from the partner lane (one shuffle) or from shared memory.
__device__ __forceinline__ double2 part_pair(double2 c, int p) { return make_double2(c.x, p ? c.y : -c.y); }
__device__ __forceinline__ float2 part_pair(float2 c, int p) { return make_float2(c.x, p ? c.y : -c.y); }
// the partner lane's value (every lane of the warp takes part)
__device__ __forceinline__ double partner(double v) { return __shfl_xor_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float partner(float v) { return __shfl_xor_sync(0xffffffffu, v, 1); }
// component p of the complex value v
__device__ __forceinline__ double comp(double2 v, int p) { return p ? v.y : v.x; }
// acc + (c x)_p for a per-part pair c and the components (xa, xb) = (x_p, x_{1-p})
__device__ __forceinline__ double pmac(double acc, double2 c, double xa, double xb) {
    return fma(c.x, xa, fma(c.y, xb, acc));
}
__device__ __forceinline__ float pmac(float acc, float2 c, float xa, float xb) {
    return fmaf(c.x, xa, fmaf(c.y, xb, acc));
}

// Dipole exchange on the fiber (fiber index f, entries at fb.xo of a [cols][N] buffer), part p:
// w += (i (h/2) J_jk (a_k^+ a_j + a_k a_j^+) x)_p for every coupled pair j < k.  a_k^+ a_j moves
// one quantum from j to k: the source has l_j + 1 and l_k - 1, weight sqrt(l_k) sqrt(l_j + 1);
// a_k a_j^+ the opposite, weight sqrt(l_k + 1) sqrt(l_j).  When k is the last subsystem the
// source is an entry of the neighbour fiber in subsystem j at the shifted level; otherwise a
// fiber that differs in both digits, at the same level.  (i c x)_p = (p ? c : -c) x_{1-p}, so
// only the other component of each source is read (xb: the buffer's component 1 - p).  The
// pairs are warp-uniform; the level tests are per lane.
template <int L, int Q, typename R>
__device__ __forceinline__ void apply_exchange_pair(const R* __restrict__ xb, const ProbDev& pd, int f, int xo, int p,
                                               R (&w)[L]) {
    for (int e = 0; e < pd.nex; ++e) {
        const int j = pd.ex_j[e], k = pd.ex_k[e];
        int sfj = 1, sfk = 1;                                  // fiber strides (j is never the last)
        for (int t = j; t < Q - 2; ++t) sfj *= L;
        for (int t = k; t < Q - 2; ++t) sfk *= L;
        const int lj = (f / sfj) % L;
        const R c = static_cast<R>(p ? pd.ex_c[e] : -pd.ex_c[e]);
        if (k == Q - 1) {
#pragma unroll
            for (int l = 0; l < L; ++l) {
                // a_k^+ a_j: from (l_j + 1, l - 1)
                if (l >= 1 && lj <= L - 2) {
                    const R wt = c * static_cast<R>(sqrt_small(l) * sqrt_small(lj + 1));
                    w[l] += wt * xb[2 * (xo + sfj * L + (l - 1))];
                }
                // a_k a_j^+: from (l_j - 1, l + 1)
                if (l <= L - 2 && lj >= 1) {
                    const R wt = c * static_cast<R>(sqrt_small(l + 1) * sqrt_small(lj));
                    w[l] += wt * xb[2 * (xo - sfj * L + (l + 1))];
                }
            }
        } else {
            const int lk = (f / sfk) % L;
            if (lk >= 1 && lj <= L - 2) {
                const R wt = c * static_cast<R>(sqrt_small(lk) * sqrt_small(lj + 1));
                const int o = 2 * (xo + (sfj - sfk) * L);
#pragma unroll
                for (int l = 0; l < L; ++l) w[l] += wt * xb[o + 2 * l];
            }
            if (lk <= L - 2 && lj >= 1) {
                const R wt = c * static_cast<R>(sqrt_small(lk + 1) * sqrt_small(lj));
                const int o = 2 * (xo + (sfk - sfj) * L);
#pragma unroll
                for (int l = 0; l < L; ++l) w[l] += wt * xb[o + 2 * l];
            }
        }
    }
}

// w = (iX_C x)_p on the fiber, part p: ladder terms of the last subsystem from the fiber itself,
// the others from the shared buffer (entries interleaved re, im; both parts of the pair have
// written theirs before the barrier).  xa: this part's components of the fiber (registers);
// cf: this part's coefficient pairs of the step's slots, i(h/2)sqrt(.)d_k.
//
// SPLIT = 2 (lane quads, L = 2): the thread holds entry le of the fiber only (xa[0], w[0]); the
// other entry of the in-fiber ladder term comes from the buffer, and exo[e] is the source of
// exchange pair e for entry le (the problem has at most MAXEXF pairs: the host admits the
// family only then).
template <int L, int Q, typename T2, int SPLIT>
__device__ __forceinline__ void apply_off_pair(const T2* __restrict__ buf, const T2* __restrict__ cf,
                                               const Fiber<L, Q>& fb, const typename cx<T2>::T (&xa)[L / SPLIT],
                                               typename cx<T2>::T (&w)[L / SPLIT], int p, int le,
                                               const int (&exo)[MAXEXF], const ProbDev& pd) {
    using R = typename cx<T2>::T;
    constexpr int LS = L / SPLIT;
    const R* ba = reinterpret_cast<const R*>(buf) + p;        // component p of entry i: ba[2 i]
    const R* bb = reinterpret_cast<const R*>(buf) + (p ^ 1);  // component 1 - p
#pragma unroll
    for (int l = 0; l < LS; ++l) w[l] = 0;
    constexpr int kl = Q - 1;
    if constexpr (SPLIT == 1) {
#pragma unroll
        for (int l = 0; l < L; ++l) {
            if (l < L - 1) w[l] = pmac(w[l], cf[(kl * L + l) * 2 + 0], xa[l + 1], bb[2 * (fb.xo + l + 1)]);
            if (l > 0) w[l] = pmac(w[l], cf[(kl * L + l) * 2 + 1], xa[l - 1], bb[2 * (fb.xo + l - 1)]);
        }
    } else {
        static_assert(SPLIT == 2 && L == 2, "lane quads are for 2-level subsystems");
        // entry 0 takes entry 1 (slot (kl, 0, a_k)), entry 1 takes entry 0 (slot (kl, 1, a_k^+))
        const int src = 2 * (fb.xo + 1 - le);
        w[0] = pmac(w[0], cf[(kl * L + le) * 2 + le], ba[src], bb[src]);
    }
#pragma unroll
    for (int k = 0; k < Fiber<L, Q>::NFIX; ++k) {
        const T2 c1 = cf[fb.sl1[k]];
        const int o1 = 2 * (fb.nb1[k] + le);
#pragma unroll
        for (int l = 0; l < LS; ++l) w[l] = pmac(w[l], c1, ba[o1 + 2 * l], bb[o1 + 2 * l]);
        if (fb.two[k]) {
            const T2 c2 = cf[fb.sl2[k]];
            const int o2 = 2 * (fb.nb2[k] + le);
#pragma unroll
            for (int l = 0; l < LS; ++l) w[l] = pmac(w[l], c2, ba[o2 + 2 * l], bb[o2 + 2 * l]);
        }
    }
    // exchange-coupled problems are 2-level qubit models (the only shapes compiled with it):
    // w += (i (h/2) J x_src)_p from the fiber's precomputed sources (a zero entry where a pair
    // gives an entry no term), or, lane pairs only, the general form beyond MAXEXF pairs
    if constexpr (L == 2 && Q >= 2) {
        bool general = false;
        if constexpr (SPLIT == 1) general = pd.nex > MAXEXF;
        if (general) {
            if constexpr (SPLIT == 1) apply_exchange_pair<L, Q, R>(bb, pd, fb.f, fb.xo, p, w);
        } else if (pd.nex) {
#pragma unroll
            for (int e = 0; e < MAXEXF; ++e) {
                if (e >= pd.nex) break;                        // warp-uniform
                const R c = static_cast<R>(p ? pd.ex_c[e] : -pd.ex_c[e]);
#pragma unroll
                for (int l = 0; l < LS; ++l) w[l] += c * bb[2 * (SPLIT == 1 ? fb.exs[e][l] : exo[e])];
            }
        }
    }
}

// this part's components of LS consecutive entries (from entry xo) into an interleaved (re, im)
// buffer
template <int LS, typename T2>
__device__ __forceinline__ void store_part(T2* buf, int xo, int p, const typename cx<T2>::T (&v)[LS]) {
    using R = typename cx<T2>::T;
    R* b = reinterpret_cast<R*>(buf) + 2 * xo + p;
#pragma unroll
    for (int l = 0; l < LS; ++l) b[2 * l] = v[l];
}

// ------------------------------------------------------------------ per-step coefficients
// Warp 0: slot (k, l, dir) -> i (h/2) sqrt(l+1) d_k (dir 0, a_k) or i (h/2) sqrt(l) conj(d_k)
// (dir 1, a_k^+), stored as the pair of part 0 (cfd[slot]) and of part 1 (cfd[NSLOT + slot]);
// lane k' < NSLOT holds d_k of its slot's subsystem.  The iteration counts of the step (packed
// by step_counts in the controls kernel) are unpacked into prm.
template <int L, int Q>
__device__ __forceinline__ void step_coefficients_pair(const ProbDev& pd, int lane, double2 dk, int cnt, double2* cfd,
                                                  float2* cff, int* prm) {
    constexpr int NSLOT = Q * L * 2;
    if (lane < NSLOT) {
        const int dir = lane & 1;
        const int l = (lane >> 1) % L;
        const bool valid = dir == 0 ? (l < L - 1) : (l > 0);
        const double s = pd.sc[2 * l + dir];
        double2 v = make_double2(0.0, 0.0);
        if (valid) v = dir == 0 ? make_double2(-s * dk.y, s * dk.x) : make_double2(s * dk.y, s * dk.x);
        const float2 vf = f32_of(v);
        cfd[lane] = part_pair(v, 0);
        cfd[NSLOT + lane] = part_pair(v, 1);
        cff[lane] = part_pair(vf, 0);
        cff[NSLOT + lane] = part_pair(vf, 1);
    }
    if (lane == 0) {
        prm[0] = cnt & 0xff;
        prm[1] = (cnt >> 8) & 0xff;
        prm[2] = (cnt >> 16) & 0xff;
        prm[3] = (cnt >> 24) & 1;
    }
}

// Reduce-scatter of VH values over the 16 lanes of one part (lanes of equal parity): the
// halving levels use lane bits 4..1, so lane ends with value (lane >> (5 - NH)) of its part
// summed over the part's lanes (NH = log2 VH <= 4); bit 0, the part, is never mixed.
template <int VH, int NH>
__device__ __forceinline__ double part_reduce_scatter(double (&acc)[VH], int lane) {
    int cnt = VH;
#pragma unroll
    for (int o = 16; o > 1; o >>= 1) {
        if (cnt > 1) {
            const int half = cnt >> 1;
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int q2 = 0; q2 < VH / 2; ++q2) {
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
    return acc[0];
}

// ------------------------------------------------------------------ the sweep kernel
// One CTA per tile.  A tile covers one or two windows ("slots"); each slot has its own step
// range, per-step coefficients, iteration counts and gradient fold, computed by warp `slot`
// (the host only builds two-slot tiles with at least two warps).  Loops run to the longer of
// the slots' ranges; a thread whose slot has no step at an iteration keeps its state.  A lane
// pair (parts 0 and 1) works on each (column, fiber) for SPLIT = 1, on each of its entries for
// SPLIT = 2 (lane quads).
template <int L, int Q, int SOLVER, bool BWD, bool ROLLOUT = false, int SPLIT = 1>
__global__ void __launch_bounds__(SPLIT > 1 ? MAX_QUAD_TILE_THREADS : MAX_PAIR_TILE_THREADS, 1)
    k_sweep_pair(const SweepArgs a) {
    static_assert(!(BWD && ROLLOUT), "the roll-out is a forward sweep");
    static_assert(SPLIT == 1 || (SPLIT == 2 && L == 2), "lane quads are for 2-level subsystems");
    constexpr int LS = L / SPLIT;          // entries of the fiber this thread holds
    constexpr int N = ipow_c(L, Q);
    constexpr int NSLOT = Q * L * 2;
    constexpr int S = BWD ? +1 : -1;       // sign of the preconditioned off-diagonal term
    constexpr int V = next_pow2_c(4 * Q);  // padded count of reduced gradient values (both parts)
    constexpr int VH = V / 2;              // values of one part: z_k and y_k components, k < Q
    constexpr int NH = log2_c(VH);         // halving levels of the part reduce-scatter

    const Tile tile = a.tiles[blockIdx.x];
    const ProbDev& pd = a.pds[tile.prob];

    extern __shared__ __align__(128) unsigned char smem[];
    const SweepSmem lay = sweep_layout(Q, L, N, a.cpt, blockDim.x, a.gmax, SOLVER, BWD, SPLIT, a.hdepth);
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
    const int part = tid & 1;              // component this thread computes (0: re, 1: im)
    const int le = SPLIT > 1 ? ((tid >> 1) & (SPLIT - 1)) * LS : 0;   // first entry it holds
    const int E = pd.E;
    const int ncol = tile.ncol, ncol0 = tile.ncol0;
    const int nslot = ncol0 < ncol ? 2 : 1;
    const bool segmented = a.mode == SWEEP_RECOMPUTE || a.mode == SWEEP_ADJOINT;
    const bool idle_launch = a.mode == SWEEP_RECOMPUTE && pd.nseg == 1;   // nothing to recompute
    constexpr bool rollout = ROLLOUT;   // one window over the whole grid (compiled separately)

    // ---- the slots' windows and step ranges (local step indices [lo, lo + cnt) of the window)
    const int64_t wn0_0 = rollout ? 0 : win_start(pd, tile.m0);
    const int wns_0 = rollout ? static_cast<int>(pd.nsteps) : static_cast<int>(win_start(pd, tile.m0 + 1) - wn0_0);
    const int64_t wn0_1 = nslot > 1 ? win_start(pd, tile.m0 + 1) : 0;
    const int wns_1 = nslot > 1 ? static_cast<int>(win_start(pd, tile.m0 + 2) - wn0_1) : 0;
    const int lo_0 = segmented ? a.seg * pd.kseg : 0;
    const int lo_1 = lo_0;
    const int cnt_0 = idle_launch ? 0 : max(0, (segmented ? min(wns_0, lo_0 + pd.kseg) : wns_0) - lo_0);
    const int cnt_1 = nslot > 1 && !idle_launch ? max(0, (segmented ? min(wns_1, lo_1 + pd.kseg) : wns_1) - lo_1) : 0;
    const int nit = max(cnt_0, cnt_1);
    // first spline active in each slot's window: the origin of the slot's window-local
    // alpha-gradient (adjoint)
    const int slo_0 = BWD ? spline_first(pd, wn0_0) : 0;
    const int slo_1 = BWD && nslot > 1 ? spline_first(pd, wn0_1) : 0;
    // every step's splines fit the slot's window-local range (the index grows with the step, so
    // a window's last step bounds them all; the host sizes the range with a margin): checked
    // once per launch, a failure reported in the status word and the gradient left unfolded
    const bool grad_fits =
        !BWD || (spline_first(pd, wn0_0 + wns_0 - 1) - slo_0 + 2 < pd.gspan &&
                 (nslot < 2 || spline_first(pd, wn0_1 + wns_1 - 1) - slo_1 + 2 < pd.gspan));
    if (!grad_fits && threadIdx.x == 0) atomicOr(pd.status, ST_GRAD_RANGE);
    // global step of slot s at iteration jj, clamped into the slot's range (a slot without steps
    // in this launch maps to its window's first step, which exists)
    auto step_of = [&](int s, int jj) -> int64_t {
        const int cnt = s ? cnt_1 : cnt_0;
        const int lo = s ? lo_1 : lo_0;
        const int64_t n0 = s ? wn0_1 : wn0_0;
        if (cnt <= 0) return n0;
        const int jc = min(jj, cnt - 1);
        return BWD ? n0 + lo + cnt - 1 - jc : n0 + lo + jc;
    };

    // ---- this thread's fiber (the threads of a pair, or quad, read the same entry)
    const int lm = a.lanemap[tile.map * static_cast<int>(blockDim.x) + tid];
    const bool act = lm >= 0;                       // idle lanes mirror an active unit, store nothing
    const int lmv = act ? lm : ~lm;
    const int c = lmv >> 16;                        // tile column
    const int f = lmv & 0xffff;                     // fiber
    const int slot = c < ncol0 ? 0 : 1;
    const int m = tile.m0 + slot;                   // window, 1-based
    const int col = slot == 0 ? tile.c0 + c : c - ncol0;
    const int my_cnt = slot ? cnt_1 : cnt_0;
    const int my_lo = slot ? lo_1 : lo_0;
    const int my_ns = slot ? wns_1 : wns_0;
    const size_t wcol = (size_t(m - 1) * E + col) * N;   // (window, column) in [M][E][N] arrays

    Fiber<L, Q> fb;
    fb.init(c, f, pd, a.cpt * N);
    // lane quads: the exchange sources of this thread's entry
    int exo[MAXEXF] = {};
    if constexpr (SPLIT > 1) {
#pragma unroll
        for (int e = 0; e < MAXEXF; ++e) exo[e] = le ? fb.exs[e][1] : fb.exs[e][0];
    }
    // the apply buffers' zero entry (read by the exchange terms a fiber entry does not have; the
    // first barrier of the time loop orders these stores before any read)
    if (tid == 0) {
        const size_t z = size_t(a.cpt) * N;
        D0[z] = make_double2(0.0, 0.0);
        if (SOLVER == SOLVER_FP64) D1[z] = make_double2(0.0, 0.0);
        if (SOLVER == SOLVER_MIXED) {
            FA[z] = make_float2(0.f, 0.f);
            FB[z] = make_float2(0.f, 0.f);
        }
    }

    // preconditioner on the fiber (P forward, conj(P) adjoint) as this part's pairs, times the
    // sign S of the off-diagonal term: (S P w)_p = SP.x w_p + SP.y w_{1-p}
    double2 Pp[LS], SPp[LS];
    float2 SPf[LS];
#pragma unroll
    for (int l = 0; l < LS; ++l) {
        double2 pv = pd.P[f * L + le + l];
        if (BWD) pv.y = -pv.y;
        Pp[l] = part_pair(pv, part);
        SPp[l] = make_double2(S * Pp[l].x, S * Pp[l].y);
        SPf[l] = make_float2(f32_of(SPp[l].x), f32_of(SPp[l].y));
    }

    // ---- initial state (this part's component)
    //   forward, whole window : U^m(t_{m-1}) = W^{m-1} (identity embedding for the first window
    //                           of the whole problem)
    //   forward, recompute    : the segment's checkpoint
    //   adjoint               : Lambda^m(t_m) for the window's last segment, else the state the
    //                           previous (later) segment left
    double u[LS];
#pragma unroll
    for (int l = 0; l < LS; ++l) {
        const int i = f * L + le + l;
        if (my_cnt == 0) {
            u[l] = 0.0;
        } else if (BWD) {
            u[l] = comp((my_lo + my_cnt == my_ns) ? pd.Lterm[wcol + i] : pd.Lstate[wcol + i], part);
        } else if (a.mode == SWEEP_RECOMPUTE) {
            u[l] = comp(pd.ckpt[((size_t(m - 1) * pd.nseg + a.seg) * E + col) * N + i], part);
        } else if (m + pd.m_off == 1) {
            u[l] = (part == 0 && pd.emb[col] == i) ? 1.0 : 0.0;
        } else {
            u[l] = comp(pd.W[(size_t(m - 2) * E + col) * N + i], part);
        }
    }
    // ---- the mixed solver's per-column scale, from the launch's initial state (column_shift)
    int sh = 0;   // the column's scale exponent (ColScale cs below)
    if constexpr (SOLVER == SOLVER_MIXED) {
        __shared__ int colexp_s[MAX_TILE_COLS];
        for (int j = tid; j < MAX_TILE_COLS; j += blockDim.x) colexp_s[j] = 0;
        tile_sync();
        int ce = 0;
#pragma unroll
        for (int l = 0; l < LS; ++l) ce = max(ce, exp_field(u[l]));
        if (act && ce > 0 && c < MAX_TILE_COLS) atomicMax(&colexp_s[c], ce);
        tile_sync();
        sh = column_shift(colexp_s[c < MAX_TILE_COLS ? c : 0]);
    }
    const ColScale cs = col_scale(sh);
    // this part's components of a [..][N] complex array at the fiber
    auto store_fiber = [&](double2* dst) {
        double* d = reinterpret_cast<double*>(dst) + 2 * (size_t(f) * L + le) + part;
#pragma unroll
        for (int l = 0; l < LS; ++l) d[2 * l] = u[l];
    };

    // ---- history blocks: slot s of a tile covers a contiguous column range of its window
    const bool want_hist = !BWD && ((a.mode == SWEEP_HISTORY && pd.nseg == 1) || a.mode == SWEEP_RECOMPUTE);
    const bool want_ckpt = !BWD && a.mode == SWEEP_HISTORY && pd.nseg > 1;
    const uint32_t bytes_0 = static_cast<uint32_t>(size_t(ncol0) * N * sizeof(double2));
    const uint32_t bytes_1 = static_cast<uint32_t>(size_t(ncol - ncol0) * N * sizeof(double2));
    auto hist_ptr = [&](int s, int jj) -> double2* {
        const int64_t n0 = s ? wn0_1 : wn0_0;
        const int lo = s ? lo_1 : lo_0;
        const int jr = static_cast<int>(step_of(s, jj) - n0) - lo;   // step within the segment
        return pd.hist + ((size_t(tile.m0 + s - 1) * pd.kseg + jr) * E + (s ? 0 : tile.c0)) * N;
    };
    // Steps per history synchronisation: the midpoint states move in groups of hd iterations
    // (iterations g hd .. g hd + hd - 1), one block of the tile's cpt N states per iteration.  The
    // forward stages a group in H and stores it with one wait per group; the adjoint fetches
    // group g into UB0 / UB1 (g even / odd) on mbar[g & 1], one group ahead.
    const int hd = a.hdepth;
    const size_t hstride = size_t(a.cpt) * N;
    // forward (thread 0): store the staged group starting at iteration g0 (every slot with a step)
    auto publish_group = [&](int g0) {
        const int g1 = min(g0 + hd, nit);
        for (int j = g0; j < g1; ++j) {
            const double2* src = H + size_t(j - g0) * hstride;
            if (j < cnt_0) bulk_s2g(hist_ptr(0, j), src, bytes_0);
            if (j < cnt_1) bulk_s2g(hist_ptr(1, j), src + size_t(ncol0) * N, bytes_1);
        }
    };
    // adjoint (thread 0): fetch the group starting at iteration g0 into dst, completing on bar
    auto fetch_group = [&](double2* dst, int g0, uint64_t* bar) {
        const int g1 = min(g0 + hd, nit);
        uint32_t total = 0;
        for (int j = g0; j < g1; ++j) total += (j < cnt_0 ? bytes_0 : 0u) + (j < cnt_1 ? bytes_1 : 0u);
        mbar_expect_tx(bar, total);
        for (int j = g0; j < g1; ++j) {
            double2* d = dst + size_t(j - g0) * hstride;
            if (j < cnt_0) bulk_g2s(d, hist_ptr(0, j), bytes_0, bar);
            if (j < cnt_1) bulk_g2s(d + size_t(ncol0) * N, hist_ptr(1, j), bytes_1, bar);
        }
    };

    if (BWD) {
        for (int j = tid; j < 2 * a.gmax; j += blockDim.x) galpha[j] = 0.0;
        if (tid == 0) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
            fence_mbar_init();
        }
        tile_sync();
        if (tid == 0 && nit > 0) fetch_group(UB0, 0, &mbar[0]);
    }

    // warp s < nslot computes slot s's coefficients and folds its gradient; it keeps d_k and
    // the iteration counts of the slot's next step in registers (lane -> subsystem of its slot)
    const bool coef_warp = warp < nslot;
    const int cslot = coef_warp ? warp : 0;
    const int my_k = (lane < NSLOT) ? (lane / (2 * L)) : 0;
    double2 dk_next = make_double2(0.0, 0.0);
    int cnt_next = 0;
    auto load_ctrl = [&](int jj) {
        if (coef_warp) {
            const int64_t n = step_of(cslot, jj);
            dk_next = lane < NSLOT ? pd.ctrl[size_t(n) * pd.q + my_k] : make_double2(0.0, 0.0);
            cnt_next = pd.spl[n].cnt;
        }
    };
    // gradient entries of a step: (carrier, spline of the 3 active) pairs, one per lane; the
    // carrier, spline offset and subsystem of this lane's first entry are fixed for the launch
    const int nscat = pd.nfsum * 3;
    const int f_kf = lane / 3, f_jw = lane % 3;
    int f_k = 0;
    while (f_k + 1 < Q && pd.cof[f_k + 1] <= f_kf) ++f_k;
    // warps whose lanes belong to both slots reduce each slot separately
    const unsigned mask1 = __ballot_sync(0xffffffffu, act && slot == 1);
    const unsigned mask0 = __ballot_sync(0xffffffffu, act && slot == 0);

    // fold slot s's reduced products of step np (parity pp of the reduction buffers) into the
    // slot's alpha-gradient: dP/dalpha1_kfs += -2h B_s Im(e^{iWt} z_k + e^{-iWt} y_k),
    // dP/dalpha2_kfs += -2h B_s Re(e^{iWt} z_k - e^{-iWt} y_k)  (Eq. grad-int at the midpoint).
    // Value v = 4k + j (j: Re z, Im z, Re y, Im y) was reduced by part j & 1 at index 2k + (j >> 1).
    auto fold = [&](int s, int pp, int64_t np, const Spline4& sp, double2 ph_lane, bool prefetched) {
        if (lane < 4 * Q) {
            const int j = lane & 3, kk = lane >> 2;
            const int pos = (j & 1) * VH + 2 * kk + (j >> 1);
            double sum = 0.0;
            for (int w2 = 0; w2 < nwarps; ++w2) sum += red[((pp * 2 + s) * nwarps + w2) * V + pos];
            zy[(pp * 2 + s) * 4 * Q + lane] = sum;
        }
        __syncwarp();
        if (!grad_fits) return;
        const int s0 = sp.s - (s ? slo_1 : slo_0);   // first active spline, window-local
        double* ga = galpha + size_t(s) * a.gmax;
        for (int i = lane; i < nscat; i += 32) {
            int kf = f_kf, jw = f_jw, k = f_k;   // this lane's first entry, precomputed
            if (i != lane) {
                kf = i / 3;
                jw = i % 3;
                k = 0;
                while (k + 1 < Q && pd.cof[k + 1] <= kf) ++k;
            }
            const double* zyk = zy + (pp * 2 + s) * 4 * Q + 4 * k;
            const double2 zk = make_double2(zyk[0], zyk[1]);
            const double2 yk = make_double2(zyk[2], zyk[3]);
            const double2 ph = (prefetched && i == lane) ? ph_lane : pd.phase[size_t(np) * pd.nfsum + kf];
            const double wgt = -2.0 * pd.h * (jw == 0 ? sp.w0 : (jw == 1 ? sp.w1 : sp.w2));
            const double A = zk.y + yk.y, B = zk.x - yk.x;
            const int idx = (kf * pd.gspan + s0 + jw) * 2;
            ga[idx + 0] += wgt * fma(ph.x, A, ph.y * B);
            ga[idx + 1] += wgt * fma(ph.x, B, -ph.y * A);
        }
    };

    __shared__ int tflag_s;   // a bounded history wait gave up (adjoint)
    int* tflag = &tflag_s;
    if (tid == 0) tflag_s = 0;
    // (the first barrier of the loop orders this store before every read of the flag)
    bool timed_out = false;
    int fsel = 0;
    double2* Dc = D0;   // FP64-solver ping-pong buffers
    double2* Dn = D1;
    if (nit > 0) load_ctrl(0);

    int hpos = 0, hgrp = 0;   // iteration jj = hgrp hd + hpos (history group and position)
    for (int jj = 0; jj < nit; ++jj) {
        const int par = jj & 1;
        const bool live = jj < my_cnt;
        if (coef_warp) {
            const double2 dk = dk_next;
            const int cnt = cnt_next;
            if (jj + 1 < nit) load_ctrl(jj + 1);
            step_coefficients_pair<L, Q>(pd, lane, dk, cnt, coef_d + (par * 2 + cslot) * 2 * NSLOT,
                                    coef_f + (par * 2 + cslot) * 2 * NSLOT, params + (par * 2 + cslot) * 4);
        }
        // adjoint: the folding warps fetch what the fold of iteration jj - 1 needs now, so the
        // loads are in flight during the solve
        Spline4 sp_prev{};
        double2 ph_prev = make_double2(0.0, 0.0);
        if (BWD && jj > 0 && coef_warp && jj - 1 < (cslot ? cnt_1 : cnt_0)) {
            const int64_t np = step_of(cslot, jj - 1);
            sp_prev = pd.spl[np];
            if (lane < nscat) ph_prev = pd.phase[size_t(np) * pd.nfsum + lane / 3];
        }
        // checkpoint: the state at the start of every segment (forward over whole windows)
        if (want_ckpt && live && act && jj % pd.kseg == 0)
            store_fiber(pd.ckpt + ((size_t(m - 1) * pd.nseg + jj / pd.kseg) * E + col) * N);
        const double2* cfd = coef_d + ((par * 2 + slot) * 2 + part) * NSLOT;
        const float2* cff = coef_f + ((par * 2 + slot) * 2 + part) * NSLOT;
        const int* prm = params + (par * 2 + slot) * 4;          // this thread's slot
        const int* prm0 = params + (par * 2) * 4;
        const int* prm1 = params + (par * 2 + 1) * 4;

        // right-hand side of the preconditioned step equation: b = P u (conj(P) for the adjoint)
        double b[LS];
#pragma unroll
        for (int l = 0; l < LS; ++l) {
            const double uo = partner(u[l]);
            b[l] = fma(Pp[l].x, u[l], Pp[l].y * uo);
        }

        double z[LS];   // this part of the midpoint state being solved for (Ubar or Lbar)

        // first barrier of the step: the coefficients are published; thread 0 stores the
        // previous iteration's midpoints (forward) or fetches the next iteration's (adjoint)
        auto first_sync_work = [&]() {
            if (BWD && *tflag) timed_out = true;   // uniform: read after a barrier
            if (!BWD && want_hist && tid == 0 && jj > 0 && hpos == 0) {
                fence_proxy_async_smem();
                publish_group(jj - hd);
            }
            if (BWD && tid == 0 && hpos == 0 && jj + hd < nit) {
                const int gn = hgrp + 1;
                fetch_group((gn & 1) ? UB1 : UB0, jj + hd, &mbar[gn & 1]);
            }
        };

        if constexpr (SOLVER == SOLVER_FP64) {
            // Dc/Dn alternate on every write (persisting across steps): a buffer is never
            // rewritten before the sync that follows its last read.
#pragma unroll
            for (int l = 0; l < LS; ++l) z[l] = b[l];
            if (act) store_part<LS, double2>(Dc, fb.xo + le, part, z);
            tile_sync();
            first_sync_work();
            if (timed_out) break;
            const int Kown = prm[0];
            const int Kmax = nslot > 1 ? max(prm0[0], prm1[0]) : prm0[0];
            for (int it = 0; it < Kmax; ++it) {
                if (it > 0) {
                    if (act) store_part<LS, double2>(Dc, fb.xo + le, part, z);
                    tile_sync();
                }
                double w[LS];
                apply_off_pair<L, Q, double2, SPLIT>(Dc, cfd, fb, z, w, part, le, exo, pd);
                double wo[LS];
#pragma unroll
                for (int l = 0; l < LS; ++l) wo[l] = partner(w[l]);
                if (it < Kown) {
#pragma unroll
                    for (int l = 0; l < LS; ++l) z[l] = fma(SPp[l].x, w[l], fma(SPp[l].y, wo[l], b[l]));
                }
                double2* tmp = Dc;
                Dc = Dn;
                Dn = tmp;
            }
        } else {
            // ---- FP32 stage: d = Ubar - b from the preconditioned fixed point d = s P w(b + d)
            float bf[LS], df[LS], y[LS];
#pragma unroll
            for (int l = 0; l < LS; ++l) {
                bf[l] = f32_of_scaled(b[l], cs);
                y[l] = bf[l];
            }
            {
                float2* Fb = fsel ? FB : FA;
                fsel ^= 1;
                if (act) store_part<LS, float2>(Fb, fb.xo + le, part, y);
                tile_sync();
                first_sync_work();
                if (timed_out) break;
                float w[LS];
                apply_off_pair<L, Q, float2, SPLIT>(Fb, cff, fb, y, w, part, le, exo, pd);
#pragma unroll
                for (int l = 0; l < LS; ++l) {
                    const float wo = partner(w[l]);
                    df[l] = fmaf(SPf[l].x, w[l], SPf[l].y * wo);
                }
            }
            const int j1 = prm[0], j2 = prm[1], R = prm[2];
            const int j1max = nslot > 1 ? max(prm0[0], prm1[0]) : prm0[0];
            const int j2max = nslot > 1 ? max(prm0[1], prm1[1]) : prm0[1];
            const int Rmax = nslot > 1 ? max(prm0[2], prm1[2]) : prm0[2];
            for (int it = 1; it < j1max; ++it) {
#pragma unroll
                for (int l = 0; l < LS; ++l) y[l] = bf[l] + df[l];
                float2* Fb = fsel ? FB : FA;
                fsel ^= 1;
                if (act) store_part<LS, float2>(Fb, fb.xo + le, part, y);
                tile_sync();
                float w[LS], wo[LS];
                apply_off_pair<L, Q, float2, SPLIT>(Fb, cff, fb, y, w, part, le, exo, pd);
#pragma unroll
                for (int l = 0; l < LS; ++l) wo[l] = partner(w[l]);
                if (it < j1) {
#pragma unroll
                    for (int l = 0; l < LS; ++l) df[l] = fmaf(SPf[l].x, w[l], SPf[l].y * wo[l]);
                }
            }
            // ---- FP64 refinement: z = b + d, residual r = (b - z) + s P w(z), correction in FP32.
            // dacc accumulates z - b (= d, then d + e, ...); b - z = -dacc up to the rounding of z.
            double dacc[LS];
#pragma unroll
            for (int l = 0; l < LS; ++l) {
                dacc[l] = f64_of_scaled(df[l], cs);
                z[l] = b[l] + dacc[l];
            }
            for (int pass = 0;; ++pass) {
                if (act) store_part<LS, double2>(D0, fb.xo + le, part, z);
                // forward: the staged midpoints of the previous step must have been read by their
                // bulk store (issued at this step's first barrier) before this step's are staged;
                // waiting here, ahead of a barrier every step has, makes the staging barrier-free
                if (!BWD && want_hist && pass == 0 && tid == 0 && hpos == 0) bulk_wait_read_all();
                tile_sync();
                double w[LS];
                apply_off_pair<L, Q, double2, SPLIT>(D0, cfd, fb, z, w, part, le, exo, pd);
                float rf[LS], e[LS];
#pragma unroll
                for (int l = 0; l < LS; ++l) {
                    const double wo = partner(w[l]);
                    const double r = fma(SPp[l].x, w[l], fma(SPp[l].y, wo, -dacc[l]));
                    rf[l] = f32_of_scaled(r, cs);
                    e[l] = rf[l];
                }
                for (int it = 0; it < j2max; ++it) {
                    float2* Fb = fsel ? FB : FA;
                    fsel ^= 1;
                    if (act) store_part<LS, float2>(Fb, fb.xo + le, part, e);
                    tile_sync();
                    float wf[LS], wfo[LS];
                    apply_off_pair<L, Q, float2, SPLIT>(Fb, cff, fb, e, wf, part, le, exo, pd);
#pragma unroll
                    for (int l = 0; l < LS; ++l) wfo[l] = partner(wf[l]);
                    if (it < j2) {
#pragma unroll
                        for (int l = 0; l < LS; ++l) e[l] = fmaf(SPf[l].x, wf[l], fmaf(SPf[l].y, wfo[l], rf[l]));
                    }
                }
                double ed[LS];
#pragma unroll
                for (int l = 0; l < LS; ++l) ed[l] = f64_of_scaled(e[l], cs);
                if (pass < R) {
#pragma unroll
                    for (int l = 0; l < LS; ++l) z[l] = z[l] + ed[l];
                }
                if (pass + 1 >= Rmax) break;
                // another pass: dacc accumulates the correction; it rewrites D0, so every thread
                // must be done reading it
                if (pass + 1 < R) {
#pragma unroll
                    for (int l = 0; l < LS; ++l) dacc[l] = dacc[l] + ed[l];
                }
                tile_sync();
            }
        }

        if (tid == 0 && (prm0[3] || (nslot > 1 && prm1[3]))) atomicOr(pd.status, ST_SOLVER_RANGE);

        if constexpr (!BWD) {
            // ---- midpoint states for the adjoint sweep (async bulk store at the next step)
            if (want_hist) {
                if constexpr (SOLVER == SOLVER_FP64) {
                    // (the FP64 solver's step may have no barrier after the first one)
                    if (hpos == 0) {
                        if (tid == 0) bulk_wait_read_all();
                        tile_sync();
                    }
                }
                if (act && live) store_part<LS, double2>(H + size_t(hpos) * hstride, fb.xo + le, part, z);
                fence_proxy_async_smem();
            }
            if (live) {
#pragma unroll
                for (int l = 0; l < LS; ++l) u[l] = fma(2.0, z[l], -u[l]);
            }
            // roll-out: U(t_m) when the step ends on a window boundary t_m, i.e. when n + 1 =
            // floor(m N_T / M) for some 1 <= m < M; the only candidate is m = ceil((n+1) M / N_T)
            if (rollout && live && act) {
                const int64_t n1 = wn0_0 + jj + 1;
                const int64_t mb = (n1 * pd.M + pd.nsteps - 1) / pd.nsteps;
                if (mb >= 1 && mb < pd.M && (mb * pd.nsteps) / pd.M == n1)
                    store_fiber(a.out + (size_t(mb - 1) * E + col) * N);
            }
        } else {
            // ---- gradient quadrature on the midpoints (fused): needs Ubar_n of the tile
            double2* UB = ((hgrp & 1) ? UB1 : UB0) + size_t(hpos) * hstride;
            // this part's products conj(Lbar) x Ubar: Re (part 0) = Lr Ur + Li Ui = za Ur + zb Ui,
            // Im (part 1) = Lr Ui - Li Ur = za Ur + zb Ui with (za, zb) = (-Li, Lr)
            double za[LS], zb[LS];
#pragma unroll
            for (int l = 0; l < LS; ++l) {
                const double zo = partner(z[l]);
                za[l] = part ? -z[l] : z[l];
                zb[l] = zo;
            }
            // a wait that gives up raises the tile's flag, read after the next barrier (the
            // products below then use whatever landed; the evaluation reports the timeout)
            if (hpos == 0 && !mbar_wait(&mbar[hgrp & 1], (hgrp >> 1) & 1)) *tflag = 1;
            double acc[VH];   // index 2k: z_k, 2k + 1: y_k (this part's component)
#pragma unroll
            for (int v = 0; v < VH; ++v) acc[v] = 0.0;
            auto prod = [&](double s0, int l, double2 x) { return fma(za[l], x.x, fma(zb[l], x.y, s0)); };
            if constexpr (SPLIT > 1) {
                // last subsystem, lane quads (L = 2): entry 0 gives z (conj(Lbar_0) Ubar_1),
                // entry 1 gives y (conj(Lbar_1) Ubar_0); every weight is 1
                constexpr int kl = Q - 1;
                const double pq = prod(0.0, 0, UB[fb.xo + 1 - le]);
                acc[2 * kl + 0] = le ? 0.0 : pq;
                acc[2 * kl + 1] = le ? pq : 0.0;
            } else {
                // last subsystem (stride 1) from the fiber itself
                constexpr int kl = Q - 1;
                double zq = 0.0, yq = 0.0;
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    // z: conj(Lbar_l) sqrt(l+1) Ubar_{l+1};  y: conj(Lbar_l) sqrt(l) Ubar_{l-1}
                    if (l < L - 1) {
                        const double wz = sqrt_small(l + 1);   // folded after unrolling
                        if (wz == 1.0)
                            zq = prod(zq, l, UB[fb.xo + l + 1]);
                        else
                            zq = fma(wz, prod(0.0, l, UB[fb.xo + l + 1]), zq);
                    }
                    if (l > 0) {
                        const double wy = sqrt_small(l);
                        if (wy == 1.0)
                            yq = prod(yq, l, UB[fb.xo + l - 1]);
                        else
                            yq = fma(wy, prod(0.0, l, UB[fb.xo + l - 1]), yq);
                    }
                }
                acc[2 * kl + 0] = zq;
                acc[2 * kl + 1] = yq;
            }
#pragma unroll
            for (int k = 0; k < Fiber<L, Q>::NFIX; ++k) {
                double p1 = 0.0;
                const double2* q1 = UB + fb.nb1[k] + le;
#pragma unroll
                for (int l = 0; l < LS; ++l) p1 = prod(p1, l, q1[l]);
                const double pv = fb.w1[k] * p1;
                acc[2 * k + 0] = fb.plus1[k] ? pv : 0.0;
                acc[2 * k + 1] = fb.plus1[k] ? 0.0 : pv;
                if (fb.two[k]) {
                    double p2 = 0.0;
                    const double2* q2 = UB + fb.nb2[k] + le;
#pragma unroll
                    for (int l = 0; l < LS; ++l) p2 = prod(p2, l, q2[l]);
                    acc[2 * k + 1] = fb.w2[k] * p2;
                }
            }
            if (!act || !live) {
#pragma unroll
                for (int v = 0; v < VH; ++v) acc[v] = 0.0;
            }
            // per-slot sums over each part's lanes: lane (lane >> (5 - NH)) == vi of part p holds
            // value vi of part p, stored at p VH + vi
            {
                const int vi = lane >> (5 - NH);
                const bool writer = (lane & ((1 << (5 - NH)) - 2)) == 0;
                const int pos = part * VH + vi;
                double* r0 = red + ((par * 2 + 0) * nwarps + warp) * V;
                double* r1 = red + ((par * 2 + 1) * nwarps + warp) * V;
                if (mask0 && mask1) {
                    // lanes of both windows: reduce the window-1 lanes on a copy first
                    double t[VH];
#pragma unroll
                    for (int v = 0; v < VH; ++v) t[v] = slot == 1 ? acc[v] : 0.0;
                    const double s1 = part_reduce_scatter<VH, NH>(t, lane);
#pragma unroll
                    for (int v = 0; v < VH; ++v) acc[v] = slot == 0 ? acc[v] : 0.0;
                    const double s0 = part_reduce_scatter<VH, NH>(acc, lane);
                    if (writer) {
                        r0[pos] = s0;
                        r1[pos] = s1;
                    }
                } else {
                    const double sv = part_reduce_scatter<VH, NH>(acc, lane);
                    if (writer) {
                        r0[pos] = mask1 ? 0.0 : sv;
                        if (nslot > 1) r1[pos] = mask1 ? sv : 0.0;
                    }
                }
            }
            // Lambda_n = 2 Lbar - Lambda_{n+1}
            if (live) {
#pragma unroll
                for (int l = 0; l < LS; ++l) u[l] = fma(2.0, z[l], -u[l]);
            }
        }

        // the folding warps add iteration jj - 1's reduced products into the alpha-gradient
        // (the barrier that published red[par ^ 1] was this iteration's first one)
        if (BWD && jj > 0 && coef_warp && jj - 1 < (cslot ? cnt_1 : cnt_0))
            fold(cslot, par ^ 1, step_of(cslot, jj - 1), sp_prev, ph_prev, true);
        if (++hpos == hd) {
            hpos = 0;
            ++hgrp;
        }
    }

    if (!timed_out) {
        tile_sync();
        if (BWD && *tflag) timed_out = true;   // the last step's wait (uniform: after the barrier)
    }
    if (!timed_out) {
        if constexpr (!BWD) {
            if (want_hist && tid == 0 && nit > 0) {
                fence_proxy_async_smem();
                publish_group(((nit - 1) / hd) * hd);
                bulk_wait_all();
            }
            if (a.mode != SWEEP_RECOMPUTE && !rollout && act && my_cnt > 0) store_fiber(pd.Uend + wcol);
        } else {
            // the last fold of every slot whose range ends at the last iteration
            if (coef_warp && nit > 0 && (cslot ? cnt_1 : cnt_0) == nit) {
                const int64_t np = step_of(cslot, nit - 1);
                fold(cslot, (nit - 1) & 1, np, pd.spl[np], make_double2(0.0, 0.0), false);
            }
            tile_sync();
            // the tile's alpha-gradient partial, accumulated over the segment launches (the first
            // adjoint launch is the last segment's)
            double* gp = pd.gpart + size_t(tile.tloc) * pd.d;
            const bool first_launch = a.seg == pd.nseg - 1;
            store_grad_partial(gp, galpha, pd, a.gmax, slo_0, nslot > 1 ? slo_1 : -1, first_launch);
            // Lambda at the segment start: Lambda^m(t_{m-1}) for the window's first segment
            if (act && my_cnt > 0) store_fiber((my_lo == 0 ? pd.Lam0 : pd.Lstate) + wcol);
        }
    } else if (tid == 0) {
        atomicOr(pd.status, ST_TIMEOUT);
        // let the bulk copies this tile issued land before its shared memory is released
        for (int p2 = 0; p2 < 2; ++p2) (void)mbar_wait(&mbar[p2], 0), (void)mbar_wait(&mbar[p2], 1);
    }
}

}  // namespace msqoc
