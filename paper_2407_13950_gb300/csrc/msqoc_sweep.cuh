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
//     conversions issue on the (slow) FP64 pipe; they carry a per-column binary scale taken
//     from the launch's initial state (the step preserves column norms), so the FP32 stage
//     works relative to the column norm whatever the state's magnitude.
// The adjoint sweep fuses the gradient quadrature of Eq. grad-int at the midpoints:
//   z_k = <Lbar, a_k Ubar>_F, y_k = <Lbar, a_k^+ Ubar>_F (summed over the tile's columns),
//   dP/dalpha1_kfs += -2h B_s Im(e^{i W t} z_k + e^{-i W t} y_k),
//   dP/dalpha2_kfs += -2h B_s Re(e^{i W t} z_k - e^{-i W t} y_k).
#pragma once

#include <type_traits>

#include "msqoc_sweep_common.cuh"

namespace msqoc {

// ------------------------------------------------------------------ complex helpers
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
// the mixed solver's 2 z - u for z = P u + d: R u + 2 d with R = 2P - 1 (FP64; d a two-float
// sum in units 2^-sh, doubled exactly through the scale): three FP64 instructions a component
__device__ __forceinline__ double2 cayley_update(double2 R, double2 u, DF dre, DF dim, int sh) {
    const double tx = df_to_f64_scaled(dre, sh + 1), ty = df_to_f64_scaled(dim, sh + 1);
    return make_double2(fma(R.x, u.x, fma(-R.y, u.y, tx)), fma(R.x, u.y, fma(R.y, u.x, ty)));
}

// Dipole exchange on the fiber (fiber index f, entries at fb.xo of a [cols][N] buffer):
// w += i (h/2) J_jk (a_k^+ a_j + a_k a_j^+) x for every coupled pair j < k.  a_k^+ a_j moves one
// quantum from j to k: the source has l_j + 1 and l_k - 1, weight sqrt(l_k) sqrt(l_j + 1); a_k a_j^+
// the opposite, weight sqrt(l_k + 1) sqrt(l_j).  When k is the last subsystem the source is an
// entry of the neighbour fiber in subsystem j at the shifted level; otherwise a fiber that
// differs in both digits, at the same level.  The pairs are warp-uniform; the level tests are
// per lane.
template <int L, int Q, typename T2>
__device__ __forceinline__ void apply_exchange(const T2* __restrict__ buf, const ProbDev& pd, int f, int xo,
                                               T2 (&w)[L]) {
    using R = typename cx<T2>::T;
    for (int e = 0; e < pd.nex; ++e) {
        const int j = pd.ex_j[e], k = pd.ex_k[e];
        int sfj = 1, sfk = 1;                                  // fiber strides (j is never the last)
        for (int t = j; t < Q - 2; ++t) sfj *= L;
        for (int t = k; t < Q - 2; ++t) sfk *= L;
        const int lj = (f / sfj) % L;
        const R c = static_cast<R>(pd.ex_c[e]);
        if (k == Q - 1) {
#pragma unroll
            for (int l = 0; l < L; ++l) {
                // a_k^+ a_j: from (l_j + 1, l - 1)
                if (l >= 1 && lj <= L - 2) {
                    const R wt = c * static_cast<R>(sqrt_small(l) * sqrt_small(lj + 1));
                    const T2 x = buf[xo + sfj * L + (l - 1)];
                    w[l].x -= wt * x.y;
                    w[l].y += wt * x.x;
                }
                // a_k a_j^+: from (l_j - 1, l + 1)
                if (l <= L - 2 && lj >= 1) {
                    const R wt = c * static_cast<R>(sqrt_small(l + 1) * sqrt_small(lj));
                    const T2 x = buf[xo - sfj * L + (l + 1)];
                    w[l].x -= wt * x.y;
                    w[l].y += wt * x.x;
                }
            }
        } else {
            const int lk = (f / sfk) % L;
            if (lk >= 1 && lj <= L - 2) {
                const R wt = c * static_cast<R>(sqrt_small(lk) * sqrt_small(lj + 1));
                const T2* src = buf + xo + (sfj - sfk) * L;
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    w[l].x -= wt * src[l].y;
                    w[l].y += wt * src[l].x;
                }
            }
            if (lk <= L - 2 && lj >= 1) {
                const R wt = c * static_cast<R>(sqrt_small(lk + 1) * sqrt_small(lj));
                const T2* src = buf + xo + (sfk - sfj) * L;
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    w[l].x -= wt * src[l].y;
                    w[l].y += wt * src[l].x;
                }
            }
        }
    }
}

// w = (iX_C x) on the fiber: ladder terms of the last subsystem from registers (xr), the
// others from the shared buffer.  cf: per-slot coefficients i(h/2)sqrt(.)d_k for this step.
template <int L, int Q, typename T2>
__device__ __forceinline__ void apply_off(const T2* __restrict__ buf, const T2* __restrict__ cf,
                                          const Fiber<L, Q>& fb, const T2 (&xr)[L], T2 (&w)[L],
                                          const ProbDev& pd) {
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
    // exchange-coupled problems are 2-level qubit models (the only shapes compiled with it):
    // w += i (h/2) J x_src from the fiber's precomputed sources, or the general form
    if constexpr (L == 2 && Q >= 2) {
        if (pd.nex > MAXEXF) {
            apply_exchange<L, Q, T2>(buf, pd, fb.f, fb.xo, w);
        } else if (pd.nex) {
            using R = typename cx<T2>::T;
#pragma unroll
            for (int e = 0; e < MAXEXF; ++e) {
                if (e >= pd.nex) break;                        // warp-uniform
                const R c = static_cast<R>(pd.ex_c[e]);
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    const T2 x = buf[fb.exs[e][l]];            // the zero entry where no term
                    w[l].x -= c * x.y;
                    w[l].y += c * x.x;
                }
            }
        }
    }
}


// ------------------------------------------------------------------ per-step coefficients
// Warp 0: slot (k, l, dir) -> i (h/2) sqrt(l+1) d_k (dir 0, a_k) or i (h/2) sqrt(l) conj(d_k)
// (dir 1, a_k^+); lane k' < NSLOT holds d_k of its slot's subsystem.  The coefficients go out
// in FP64, FP32 and (mixed solver, cfs != nullptr) split into two floats.  The iteration counts
// of the step (packed by step_counts in the controls kernel) are unpacked into prm; prm[3] holds
// the solver-range flag (bit 0) and the FP64-apply flag (bit 1).
template <int L, int Q>
__device__ __forceinline__ void step_coefficients(const ProbDev& pd, int lane, double2 dk, int cnt, double2* cfd,
                                                  float2* cff, float4* cfs, int* prm) {
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
        if (cfs) cfs[lane] = split_scaled(v, 0);
    }
    if (lane == 0) {
        prm[0] = cnt & 0xff;
        prm[1] = (cnt >> 8) & 0xff;
        prm[2] = (cnt >> 16) & 0xff;
        prm[3] = (cnt >> 24) & 3;
    }
}

// sums of the gradient products: FP64 (FP64 solver) or two-float (mixed solver; exact two-sums
// of the leading parts, no FP64 instruction)
__device__ __forceinline__ double gsum_add(double a, double b) { return a + b; }
__device__ __forceinline__ DF gsum_add(DF a, DF b) { return df_add(a, b); }
__device__ __forceinline__ double gsum_shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ DF gsum_shfl_xor(DF v, int o) {
    return DF{__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.c, o)};
}
__device__ __forceinline__ void gsum_zero(double& v) { v = 0.0; }
__device__ __forceinline__ void gsum_zero(DF& v) { v = DF{0.f, 0.f}; }

// warp reduce-scatter of V values: lane ends with value (lane >> (5 - NH)) summed over the warp
template <int V, int NH, typename T>
__device__ __forceinline__ T warp_reduce_scatter(T (&acc)[V], int lane) {
    int cnt = V;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (cnt > 1) {
            const int half = cnt >> 1;
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int q2 = 0; q2 < V / 2; ++q2) {
                if (q2 < half) {
                    const T send = upper ? acc[q2] : acc[q2 + half];
                    const T keep = upper ? acc[q2 + half] : acc[q2];
                    acc[q2] = gsum_add(keep, gsum_shfl_xor(send, o));
                }
            }
            cnt = half;
        } else {
            acc[0] = gsum_add(acc[0], gsum_shfl_xor(acc[0], o));
        }
    }
    return acc[0];
}

// ------------------------------------------------------------------ compensated apply
// w += c x for split complex operands (hi.x, hi.y, lo.x, lo.y); w[0] real, w[1] imaginary part
__device__ __forceinline__ void cmac_df(DF (&w)[2], const float4& c, const float4& x) {
    df_mac(w[0], c.x, c.z, x.x, x.z);
    df_mac(w[0], -c.y, -c.w, x.y, x.w);
    df_mac(w[1], c.x, c.z, x.y, x.w);
    df_mac(w[1], c.y, c.w, x.x, x.z);
}
// w = iX_C x on the fiber (apply_off without exchange terms) from split entries: the fiber's own
// in xr, the neighbours' in buf, the coefficients in cf; compensated FP32 sums (about 2^-47 of
// the terms' magnitudes).  The mixed solver's residual needs P w to within 2^-53 |x| only, and
// |P w| <= rho |x| with rho <= 2^-7 wherever this form is used.
// exc / nex: the exchange pairs' coefficients (h/2) J split into two floats and their count
// (2-level problems with at most MAXEXF pairs; terms i (h/2) J x_src from the fiber's sources)
template <int L, int Q>
__device__ __forceinline__ void apply_off_df(const float4* __restrict__ buf, const float4* __restrict__ cf,
                                             const Fiber<L, Q>& fb, const float4 (&xr)[L], DF (&w)[L][2],
                                             const float2 (&exc)[MAXEXF], int nex) {
    // the first term of each entry's sum initialises it (no two-sum with zero)
    constexpr int kl = Q - 1;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        if (l < L - 1) cmul_df(xr[l + 1], cf[(kl * L + l) * 2 + 0], w[l][0], w[l][1]);
        if (l > 0) {
            if (l < L - 1)
                cmac_df(w[l], cf[(kl * L + l) * 2 + 1], xr[l - 1]);
            else
                cmul_df(xr[l - 1], cf[(kl * L + l) * 2 + 1], w[l][0], w[l][1]);
        }
    }
#pragma unroll
    for (int k = 0; k < Fiber<L, Q>::NFIX; ++k) {
        const float4 c1 = cf[fb.sl1[k]];
        const float4* p1 = buf + fb.nb1[k];
#pragma unroll
        for (int l = 0; l < L; ++l) cmac_df(w[l], c1, p1[l]);
        if (fb.two[k]) {
            const float4 c2 = cf[fb.sl2[k]];
            const float4* p2 = buf + fb.nb2[k];
#pragma unroll
            for (int l = 0; l < L; ++l) cmac_df(w[l], c2, p2[l]);
        }
    }
    if constexpr (L == 2 && Q >= 2) {
#pragma unroll
        for (int e = 0; e < MAXEXF; ++e) {
            if (e >= nex) break;   // uniform
#pragma unroll
            for (int l = 0; l < L; ++l) {
                const float4 x = buf[fb.exs[e][l]];   // the zero entry where the pair gives no term
                df_mac(w[l][0], -exc[e].x, -exc[e].y, x.y, x.w);
                df_mac(w[l][1], exc[e].x, exc[e].y, x.x, x.z);
            }
        }
    }
}
// the residual -d + s P w of the refinement in scaled units, rounded to FP32: d = dh + dl and
// P = (hi, lo) split, w from apply_off_df
template <int S>
__device__ __forceinline__ float2 resid_df(float2 dh, float2 dl, const float4& P, const DF (&w)[2]) {
    DF re{-dh.x, -dl.x}, im{-dh.y, -dl.y};
    constexpr float s = S > 0 ? 1.f : -1.f;
    df_mac(re, s * P.x, s * P.z, w[0].s, w[0].c);
    df_mac(re, -s * P.y, -s * P.w, w[1].s, w[1].c);
    df_mac(im, s * P.x, s * P.z, w[1].s, w[1].c);
    df_mac(im, s * P.y, s * P.w, w[0].s, w[0].c);
    return make_float2(fadd_n(re.s, re.c), fadd_n(im.s, im.c));
}

// ------------------------------------------------------------------ FP64 residual, out of line
// The mixed solver's refinement residual in FP64, for the steps whose contraction factor is
// above the compensated form's bound (step_counts) and for exchange-coupled problems.  Out of
// line: it is rare on the workloads that fill the GPU, and inlined into the step loop (with the
// FP64 midpoint state and the FP64 apply it needs) it slowed the common path by 4-9%.  Values
// travel by value; the fiber's neighbour list is rebuilt from (column, fiber).
template <int L> struct SplitVals { float4 v[L]; };
template <int L> struct ResidIn { float4 zs[L]; DF dre[L], dim[L]; };
template <int L> struct ResidOut { float2 r[L]; };

// the midpoint state z = zs 2^sh in FP64 into the shared apply buffer (the fiber's entries)
template <int L>
static __device__ __noinline__ void store_z64(double2* dst, SplitVals<L> zs, int sh) {
#pragma unroll
    for (int l = 0; l < L; ++l)
        dst[l] = make_double2(df_to_f64_scaled(DF{zs.v[l].x, zs.v[l].z}, sh),
                              df_to_f64_scaled(DF{zs.v[l].y, zs.v[l].w}, sh));
}
// r = s P (iX_C) z - d_total in FP64, rounded to FP32 in the column's scaled units
template <int L, int Q, int S, bool BWD>
static __device__ __noinline__ ResidOut<L> resid_fp64(const double2* D0, const double2* cfd, const ProbDev& pd, int c,
                                                      int f, int zero, ResidIn<L> in, int sh) {
    Fiber<L, Q> fb;
    fb.init(c, f, pd, zero);
    double2 z[L];
#pragma unroll
    for (int l = 0; l < L; ++l)
        z[l] = make_double2(df_to_f64_scaled(DF{in.zs[l].x, in.zs[l].z}, sh),
                            df_to_f64_scaled(DF{in.zs[l].y, in.zs[l].w}, sh));
    double2 w[L];
    apply_off<L, Q, double2>(D0, cfd, fb, z, w, pd);
    const ColScale cs = col_scale(sh);
    ResidOut<L> o;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        double2 p = pd.P[f * L + l];
        if (BWD) p.y = -p.y;
        const double2 dacc = make_double2(df_to_f64_scaled(in.dre[l], sh), df_to_f64_scaled(in.dim[l], sh));
        o.r[l] = f32_of_scaled(resid_from<S>(dacc, p, w[l]), cs);
    }
    return o;
}

// ------------------------------------------------------------------ gradient products, split form
// (R, I) += (Re, Im) of conj(x) u for split entries x, u = (hi.x, hi.y, lo.x, lo.y); sr = -1
// subtracts the real part instead
template <int SR>
__device__ __forceinline__ void cjmac_split(DF& R, DF& I, const float4& x, const float4& u) {
    if constexpr (SR > 0) {
        df_mac(R, x.x, x.z, u.x, u.z);
        df_mac(R, x.y, x.w, u.y, u.w);
    } else {
        df_mac(R, -x.x, -x.z, u.x, u.z);
        df_mac(R, -x.y, -x.w, u.y, u.w);
    }
    df_mac(I, x.x, x.z, u.y, u.w);
    df_mac(I, -x.y, -x.w, u.x, u.z);
}
// the same as the first term of the sums (R = SR Re(conj(x) u), I = Im(conj(x) u)): no
// two-sum with zero
template <int SR>
__device__ __forceinline__ void cjmul_split(DF& R, DF& I, const float4& x, const float4& u) {
    if constexpr (SR > 0)
        R = dot2_df(x.x, x.z, u.x, u.z, x.y, x.w, u.y, u.w);
    else
        R = dot2_df(-x.x, -x.z, u.x, u.z, -x.y, -x.w, u.y, u.w);
    I = dot2_df(x.x, x.z, u.y, u.w, -x.y, -x.w, u.x, u.z);
}

// The mixed solver's gradient products of one fiber (the FP64 form is in the adjoint below):
// acc[2k] = A_k and acc[2k + 1] = B_k, the fiber's rows of A_k = Im z_k + Im y_k and
// B_k = Re z_k - Re y_k with z_k = <Lbar, a_k Ubar>, y_k = <Lbar, a_k^+ Ubar>.  Lbar comes split
// into two floats (zs, in units of its column's scale 2^shL), the midpoint states Ubar split by
// the forward sweep (ub, scale 2^shU).  Each value is a compensated FP32 sum (about 2^-47 times
// its terms' magnitudes) in units 2^(shL + shU), multiplied by pscale (a power of two) into the
// tile's common units.
//   last subsystem, weight class j = 1 .. L-1 (weight sqrt j): the pairs (Lbar_{j-1}, Ubar_j)
//     (a_k, real part +) and (Lbar_j, Ubar_{j-1}) (a_k^+, real part -);
//   other subsystems: entry 1 of the neighbour list (weight sqrt(l_k + 1) for a_k, real part +;
//     sqrt(l_k) for a_k^+ at the top level, real part -) and, at interior levels, entry 2
//     (a_k^+, weight sqrt(l_k), real part -).
template <int L, int Q>
__device__ __forceinline__ void products_split(const float4 (&zs)[L], const float4* __restrict__ ub,
                                               const Fiber<L, Q>& fb, float pscale, DF* acc) {
    {
        constexpr int kl = Q - 1;
        DF A{0.f, 0.f}, B{0.f, 0.f};
#pragma unroll
        for (int j = 1; j < L; ++j) {
            DF R, I;
            cjmul_split<+1>(R, I, zs[j - 1], ub[fb.xo + j]);
            cjmac_split<-1>(R, I, zs[j], ub[fb.xo + j - 1]);
            if (j == 1) {
                A = I;
                B = R;
            } else {
                A = df_add(A, df_scale_sqrt(I, j));
                B = df_add(B, df_scale_sqrt(R, j));
            }
        }
        acc[2 * kl + 0] = DF{fmul_n(A.s, pscale), fmul_n(A.c, pscale)};
        acc[2 * kl + 1] = DF{fmul_n(B.s, pscale), fmul_n(B.c, pscale)};
    }
#pragma unroll
    for (int k = 0; k < Fiber<L, Q>::NFIX; ++k) {
        const int lk = (fb.f / ipow_c(L, Q - 2 - k)) % L;   // the fiber's level in subsystem k
        DF R, I;
        const float4* u1 = ub + fb.nb1[k];
        cjmul_split<+1>(R, I, zs[0], u1[0]);
#pragma unroll
        for (int l = 1; l < L; ++l) cjmac_split<+1>(R, I, zs[l], u1[l]);
        // entry 1: a_k (weight sqrt(l_k + 1)) or, at the top level, a_k^+ (sqrt(l_k), real part -)
        DF A = df_scale_sqrt(I, fb.plus1[k] ? lk + 1 : lk);
        DF B = df_scale_sqrt(R, fb.plus1[k] ? lk + 1 : lk);
        if (!fb.plus1[k]) B = df_neg(B);
        if (fb.two[k]) {   // an interior level (warp-uniform: lanes are sorted by class)
            DF R2, I2;
            const float4* u2 = ub + fb.nb2[k];
            cjmul_split<-1>(R2, I2, zs[0], u2[0]);
#pragma unroll
            for (int l = 1; l < L; ++l) cjmac_split<-1>(R2, I2, zs[l], u2[l]);
            A = df_add(A, df_scale_sqrt(I2, lk));
            B = df_add(B, df_scale_sqrt(R2, lk));
        }
        acc[2 * k + 0] = DF{fmul_n(A.s, pscale), fmul_n(A.c, pscale)};
        acc[2 * k + 1] = DF{fmul_n(B.s, pscale), fmul_n(B.c, pscale)};
    }
}

// ------------------------------------------------------------------ gradient fold (adjoint)
// One step's fold of a window slot, run by that slot's folding warp: the warps' partial sums
// red[w][v] (fixed order) of A_k = Im z_k + Im y_k and B_k = Re z_k - Re y_k into zy, then, per
// (carrier kf, active spline jw) entry, dP/dalpha1_kfs += -2h B_s (p.x A + p.y B) and
// dP/dalpha2_kfs += -2h B_s (p.x B - p.y A) with p = e^{i W t} at the midpoint (Eq. grad-int).
// Kept out of line: it runs once per step on one warp, and inlined it enlarged the adjoint's
// step loop, whose instruction fetches already stall its warps.
template <int Q, int V>
static __device__ __noinline__ void fold_step(const ProbDev& pd, const double* red, double* zy, double* ga,
                                              int nwarps, int64_t np, Spline4 sp, double2 ph_lane, bool prefetched,
                                              int s0, int lane) {
    if (lane < 2 * Q) {
        const double* r = red + lane;
        double s_even = 0.0, s_odd = 0.0;
        for (int w2 = 0; w2 < nwarps; w2 += 2) {
            s_even += r[w2 * V];
            if (w2 + 1 < nwarps) s_odd += r[(w2 + 1) * V];
        }
        zy[lane] = s_even + s_odd;
    }
    __syncwarp();
    const int nscat = pd.nfsum * 3;
    const double m2h = -2.0 * pd.h;
    for (int i = lane; i < nscat; i += 32) {
        const int kf = i / 3, jw = i % 3;
        int k = 0;
        while (k + 1 < Q && pd.cof[k + 1] <= kf) ++k;
        const double2 ph = (prefetched && i == lane) ? ph_lane : pd.phase[size_t(np) * pd.nfsum + kf];
        const double wgt = m2h * (jw == 0 ? sp.w0 : (jw == 1 ? sp.w1 : sp.w2));
        const double A = zy[2 * k], B = zy[2 * k + 1];
        const int idx = (kf * pd.gspan + s0 + jw) * 2;
        ga[idx + 0] = fma(wgt, fma(ph.x, A, ph.y * B), ga[idx + 0]);
        ga[idx + 1] = fma(wgt, fma(ph.x, B, -ph.y * A), ga[idx + 1]);
    }
}

// The mixed solver's fold (the same sums as fold_step): the partial sums and zy are two-float
// sums in units of 2^S (the tile's product scale, see the adjoint), the phase and spline weight
// are split on the fly, and each step's contribution goes into a two-float copy gdf of the
// slot's gradient, which is added into the FP64 gradient ga every FOLD_FLUSH steps (flush: one
// FP64 add and FMA per element), so a window's hundreds of steps still accumulate in FP64.
__device__ __forceinline__ void df_mac_full(DF& a, float xh, float xl, float yh, float yl) {
    df_mac(a, xh, xl, yh, yl);
    a.c = ffma_n(xl, yl, a.c);   // the low parts' product too: y may be a sum that cancelled
}
template <int Q, int V>
static __device__ __noinline__ void fold_step_df(const ProbDev& pd, const DF* red, DF* zy, double* ga, DF* gdf,
                                                 int gmax, int nwarps, int64_t np, Spline4 sp, double2 ph_lane,
                                                 bool prefetched, int s0, int S, bool flush, int lane) {
    if (lane < 2 * Q) {
        const DF* r = red + lane;
        DF s_even{0.f, 0.f}, s_odd{0.f, 0.f};
        for (int w2 = 0; w2 < nwarps; w2 += 2) {
            s_even = df_add(s_even, r[w2 * V]);
            if (w2 + 1 < nwarps) s_odd = df_add(s_odd, r[(w2 + 1) * V]);
        }
        zy[lane] = df_add(s_even, s_odd);
    }
    __syncwarp();
    const int nscat = pd.nfsum * 3;
    for (int i = lane; i < nscat; i += 32) {
        const int kf = i / 3, jw = i % 3;
        int k = 0;
        while (k + 1 < Q && pd.cof[k + 1] <= kf) ++k;
        const double2 ph = (prefetched && i == lane) ? ph_lane : pd.phase[size_t(np) * pd.nfsum + kf];
        const float2 px = split_scaled(ph.x, 0), py = split_scaled(ph.y, 0);
        const float2 wg = split_scaled(jw == 0 ? sp.w0 : (jw == 1 ? sp.w1 : sp.w2), 0);
        const DF A = zy[2 * k], B = zy[2 * k + 1];
        DF t1{0.f, 0.f}, t2{0.f, 0.f};
        df_mac_full(t1, px.x, px.y, A.s, A.c);
        df_mac_full(t1, py.x, py.y, B.s, B.c);
        df_mac_full(t2, px.x, px.y, B.s, B.c);
        df_mac_full(t2, -py.x, -py.y, A.s, A.c);
        DF* g = gdf + (kf * pd.gspan + s0 + jw) * 2;
        g[0] = df_add(g[0], df_scale(t1, wg.x, wg.y));
        g[1] = df_add(g[1], df_scale(t2, wg.x, wg.y));
    }
    if (flush) {
        __syncwarp();
        const double m2h = -2.0 * pd.h;
        for (int e = lane; e < gmax; e += 32) {
            const DF v = gdf[e];
            if (v.s != 0.f || v.c != 0.f) {
                ga[e] = fma(m2h, df_to_f64_scaled(v, S), ga[e]);
                gdf[e] = DF{0.f, 0.f};
            }
        }
    }
}

// ------------------------------------------------------------------ the sweep kernel
// One CTA per tile.  A tile covers one or two windows ("slots"); each slot has its own step
// range, per-step coefficients and iteration counts, computed by warp `slot`, and gradient fold,
// run by warp nwarps - 1 - slot (the host only builds two-slot tiles with at least two warps).  Loops run to the longer of
// the slots' ranges; a thread whose slot has no step at an iteration keeps its state.
// MAXT: the largest tile the instantiation serves; it sets the register budget (255 registers a
// thread for MAX_TILE_THREADS, 168 for MAX_LEAN_TILE_THREADS: 12 warps on an SM).
template <int L, int Q, int SOLVER, bool BWD, bool ROLLOUT = false, int MAXT = MAX_TILE_THREADS>
__global__ void __launch_bounds__(MAXT, 1) k_sweep(const SweepArgs a) {
    static_assert(!(BWD && ROLLOUT), "the roll-out is a forward sweep");
    constexpr int N = ipow_c(L, Q);
    constexpr int NSLOT = Q * L * 2;
    constexpr int S = BWD ? +1 : -1;       // sign of the preconditioned off-diagonal term
    // reduced gradient values per subsystem: A_k = Im z_k + Im y_k and B_k = Re z_k - Re y_k, the
    // only combinations of the products the quadrature needs (padded to a power of two)
    constexpr int V = next_pow2_c(2 * Q);
    constexpr int NH = log2_c(V);          // halving levels of the warp reduce-scatter

    const Tile tile = a.tiles[blockIdx.x];
    const ProbDev& pd = a.pds[tile.prob];

    extern __shared__ __align__(128) unsigned char smem[];
    const SweepSmem lay = sweep_layout(Q, L, N, a.cpt, blockDim.x, a.gmax, SOLVER, BWD, 0, a.hdepth);
    double2* coef_d = reinterpret_cast<double2*>(smem + lay.coef_d);
    float2* coef_f = reinterpret_cast<float2*>(smem + lay.coef_f);
    float4* coef_s = SOLVER == SOLVER_MIXED ? reinterpret_cast<float4*>(smem + lay.coef_s) : nullptr;
    int* params = reinterpret_cast<int*>(smem + lay.params);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + lay.mbar);
    // sums of the gradient products: two-float (mixed solver, in units 2^S_tile) or FP64; the
    // tile's window gradients are FP64
    using GT = std::conditional_t<SOLVER == SOLVER_MIXED, DF, double>;
    GT* red = reinterpret_cast<GT*>(smem + lay.red);
    GT* zy = reinterpret_cast<GT*>(smem + lay.zy);
    double* galpha = reinterpret_cast<double*>(smem + lay.galpha);
    DF* gdf = reinterpret_cast<DF*>(smem + lay.gdf);   // two-float gradient terms (mixed solver)
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

    // ---- this thread's fiber
    const int lm = a.lanemap[tile.map * static_cast<int>(blockDim.x) + tid];
    const bool act = lm >= 0;                       // idle lanes mirror an active one, store nothing
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
    // the exchange coefficients split for the compensated apply (2-level problems)
    float2 exc[MAXEXF];
#pragma unroll
    for (int e = 0; e < MAXEXF; ++e)
        exc[e] = (L == 2 && Q >= 2 && e < pd.nex) ? split_scaled(pd.ex_c[e], 0) : make_float2(0.f, 0.f);
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

    // preconditioner on the fiber: P (forward) or conj(P) (adjoint)
    double2 Pd[L];
    float2 Pf[L];
    float4 Ps[L];   // split (mixed solver's right-hand side and compensated residual)
    // 2 kappa = -2 Im P / Re P split (P = 1 / (1 + i kappa)), for the mixed solver's state update
    float2 k2s[L];
    float4* cq = SOLVER == SOLVER_MIXED ? reinterpret_cast<float4*>(smem + lay.cq) : nullptr;
    bool carry_ok = true;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        double2 p = pd.P[f * L + l];
        if (BWD) p.y = -p.y;
        Pd[l] = p;
        Ps[l] = split_scaled(p, 0);
        Pf[l] = make_float2(Ps[l].x, Ps[l].y);   // p rounded to FP32
        const double k2 = -2.0 * p.y / p.x;
        k2s[l] = split_scaled(k2, 0);
        carry_ok = carry_ok && k2 * k2 <= CARRY_UPDATE_K2;
        // the splits' third parts, per entry of the fiber (the same for every column)
        if (SOLVER == SOLVER_MIXED && act && c == 0)
            cq[f * L + l] = make_float4(split_third(k2, k2s[l]), split_third(p.x, make_float2(Ps[l].x, Ps[l].z)),
                                        split_third(p.y, make_float2(Ps[l].y, Ps[l].w)), 0.f);
    }
    // the compensated state update for the whole tile (the same P table for every tile of the
    // problem, so the same choice), else R u + 2 d in FP64
    const bool carry_upd = SOLVER == SOLVER_MIXED && tile_sync_or(act && !carry_ok) == 0;
    float2 car[L];   // the state's FP32 carry (compensated update), zero otherwise
#pragma unroll
    for (int l = 0; l < L; ++l) car[l] = make_float2(0.f, 0.f);

    // ---- initial state
    //   forward, whole window : U^m(t_{m-1}) = W^{m-1} (identity embedding for the first window
    //                           of the whole problem)
    //   forward, recompute    : the segment's checkpoint
    //   adjoint               : Lambda^m(t_m) for the window's last segment, else the state the
    //                           previous (later) segment left
    double2 u[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const int i = f * L + l;
        if (my_cnt == 0) {
            u[l] = make_double2(0.0, 0.0);
        } else if (BWD) {
            u[l] = (my_lo + my_cnt == my_ns) ? pd.Lterm[wcol + i] : pd.Lstate[wcol + i];
        } else if (a.mode == SWEEP_RECOMPUTE) {
            u[l] = pd.ckpt[((size_t(m - 1) * pd.nseg + a.seg) * E + col) * N + i];
        } else if (m + pd.m_off == 1) {
            u[l] = make_double2(pd.emb[col] == i ? 1.0 : 0.0, 0.0);
        } else {
            u[l] = pd.W[(size_t(m - 2) * E + col) * N + i];
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
        for (int l = 0; l < L; ++l) ce = max(ce, max(exp_field(u[l].x), exp_field(u[l].y)));
        if (act && ce > 0 && c < MAX_TILE_COLS) atomicMax(&colexp_s[c], ce);
        tile_sync();
        sh = column_shift(colexp_s[c < MAX_TILE_COLS ? c : 0]);
    }
    const ColScale cs = col_scale(sh);
    // the history's column scale exponent: written by the forward launch that stores the
    // segment's midpoint states, read by the adjoint launch of the segment
    const int hseg = a.mode == SWEEP_HISTORY ? 0 : a.seg;
    int* const hsh_col = pd.hsh + (size_t(m - 1) * pd.nseg + hseg) * E + col;
    int shU = 0;
    // adjoint, mixed solver: the gradient products of column c are in units 2^(sh + shU); the
    // tile sums them in units 2^S_tile, the largest over its columns (pscale = 2^(sh + shU -
    // S_tile) <= 1, set after the barrier below)
    __shared__ int stile_s;
    int S_tile = 0;
    float pscale = 1.f;
    if constexpr (SOLVER == SOLVER_MIXED) {
        if (!BWD && ((a.mode == SWEEP_HISTORY && pd.nseg == 1) || a.mode == SWEEP_RECOMPUTE) && act && f == 0 &&
            my_cnt > 0)
            *hsh_col = sh;
        if (BWD) {
            if (tid == 0) stile_s = -(1 << 20);
            tile_sync();
            if (my_cnt > 0) shU = *hsh_col;
            if (act && my_cnt > 0) atomicMax(&stile_s, sh + shU);
        }
    }

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
        if constexpr (SOLVER == SOLVER_MIXED)
            for (int j = tid; j < 2 * a.gmax; j += blockDim.x) gdf[j] = DF{0.f, 0.f};
        if (tid == 0) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
            fence_mbar_init();
        }
        tile_sync();
        if (tid == 0 && nit > 0) fetch_group(UB0, 0, &mbar[0]);
        if constexpr (SOLVER == SOLVER_MIXED) {
            S_tile = stile_s > -(1 << 20) ? stile_s : 0;
            const int k = sh + shU - S_tile;   // <= 0
            pscale = k >= -126 ? float_of(static_cast<uint32_t>(127 + k) << 23)
                               : (k >= -149 ? float_of(1u << (k + 149)) : 0.f);
        }
    }

    // warp s < nslot computes slot s's coefficients and keeps d_k and the iteration counts of
    // the slot's next step in registers (lane -> subsystem of its slot); warp nwarps - 1 - s folds
    // the slot's gradient (the two extra jobs of a step on different warps where there are two)
    const bool coef_warp = warp < nslot;
    const bool fold_warp = nwarps - 1 - warp < nslot;
    const int fslot = fold_warp ? nwarps - 1 - warp : 0;
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
    // gradient entries of a step: (carrier, spline of the 3 active) pairs, one per lane of the
    // folding warp (whose phases are prefetched for the lane's first entry)
    const int nscat = pd.nfsum * 3;
    // warps whose lanes belong to both slots reduce each slot separately
    const unsigned mask1 = __ballot_sync(0xffffffffu, act && slot == 1);
    const unsigned mask0 = __ballot_sync(0xffffffffu, act && slot == 0);

    // fold slot s's reduced products of step np (parity pp of the reduction buffers) into the
    // slot's alpha-gradient: dP/dalpha1_kfs += -2h B_s Im(e^{iWt} z_k + e^{-iWt} y_k),
    // dP/dalpha2_kfs += -2h B_s Re(e^{iWt} z_k - e^{-iWt} y_k)  (Eq. grad-int at the midpoint),
    // i.e. with (A, B) = (Im z + Im y, Re z - Re y) and the phase p: -2h B_s (p.x A + p.y B) and
    // -2h B_s (p.x B - p.y A)
    auto fold = [&](int s, int pp, int64_t np, const Spline4& sp, double2 ph_lane, bool prefetched, bool flush) {
        if (!grad_fits) {
            // the sums are not needed; keep the warp's lanes together as fold_step would
            __syncwarp();
            return;
        }
        if constexpr (SOLVER == SOLVER_MIXED)
            fold_step_df<Q, V>(pd, red + ((pp * 2 + s) * nwarps) * V, zy + (pp * 2 + s) * 4 * Q,
                               galpha + size_t(s) * a.gmax, gdf + size_t(s) * a.gmax, a.gmax, nwarps, np, sp,
                               ph_lane, prefetched, sp.s - (s ? slo_1 : slo_0), S_tile, flush, lane);
        else
            fold_step<Q, V>(pd, red + ((pp * 2 + s) * nwarps) * V, zy + (pp * 2 + s) * 4 * Q,
                            galpha + size_t(s) * a.gmax, nwarps, np, sp, ph_lane, prefetched,
                            sp.s - (s ? slo_1 : slo_0), lane);
    };

    // the step's state update: 2 z - u (FP64 solver); R u + 2 d in FP64 or the compensated form
    // with the carry (mixed solver; the FP64 form reads R's P from the table: rare)
    auto state_update = [&](double2 (&uu)[L], const double2 (&zz)[L], const DF (&br)[L], const DF (&bi)[L],
                            const DF (&dr)[L], const DF (&di)[L]) {
        if constexpr (SOLVER == SOLVER_MIXED) {
            if (carry_upd) {
#pragma unroll
                for (int l = 0; l < L; ++l)
                    uu[l] = carry_update(uu[l], br[l], bi[l], k2s[l], cq[f * L + l].x, dr[l], di[l], sh, car[l]);
            } else {
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    double2 p = pd.P[f * L + l];
                    if (BWD) p.y = -p.y;
                    uu[l] = cayley_update(make_double2(fma(2.0, p.x, -1.0), 2.0 * p.y), uu[l], dr[l], di[l], sh);
                }
            }
        } else {
#pragma unroll
            for (int l = 0; l < L; ++l) uu[l] = reflect(zz[l], uu[l]);
        }
    };
    // the state as stored (u + carry)
    auto state_out = [&](int l) { return carry_upd ? carry_finish(u[l], car[l], sh) : u[l]; };

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
            step_coefficients<L, Q>(pd, lane, dk, cnt, coef_d + (par * 2 + cslot) * NSLOT,
                                    coef_f + (par * 2 + cslot) * NSLOT,
                                    coef_s ? coef_s + (par * 2 + cslot) * NSLOT : nullptr,
                                    params + (par * 2 + cslot) * 4);
        }
        // adjoint: the folding warps fetch what the fold of iteration jj - 1 needs now, so the
        // loads are in flight during the solve
        Spline4 sp_prev{};
        double2 ph_prev = make_double2(0.0, 0.0);
        if (BWD && jj > 0 && fold_warp && jj - 1 < (fslot ? cnt_1 : cnt_0)) {
            const int64_t np = step_of(fslot, jj - 1);
            sp_prev = pd.spl[np];
            if (lane < nscat) ph_prev = pd.phase[size_t(np) * pd.nfsum + lane / 3];
        }
        // checkpoint: the state at the start of every segment (forward over whole windows)
        // (the carry is folded into u there, so that a segment recomputed from its checkpoint
        // repeats these steps bit for bit)
        if (want_ckpt && live && jj % pd.kseg == 0) {
            if (carry_upd) {
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    u[l] = carry_finish(u[l], car[l], sh);
                    car[l] = make_float2(0.f, 0.f);
                }
            }
            if (act) {
                double2* ck = pd.ckpt + ((size_t(m - 1) * pd.nseg + jj / pd.kseg) * E + col) * N + f * L;
#pragma unroll
                for (int l = 0; l < L; ++l) ck[l] = u[l];
            }
        }
        const double2* cfd = coef_d + (par * 2 + slot) * NSLOT;
        const float2* cff = coef_f + (par * 2 + slot) * NSLOT;
        const float4* cfs = coef_s + (par * 2 + slot) * NSLOT;
        const int* prm = params + (par * 2 + slot) * 4;          // this thread's slot
        const int* prm0 = params + (par * 2) * 4;
        const int* prm1 = params + (par * 2 + 1) * 4;

        // the midpoint state being solved for (Ubar or Lbar): FP64 (FP64 solver) or, for the
        // mixed solver, the two-float sum zf = b + d_total in the column's scaled units (about
        // 2^-47 |z|), which the forward's history and the adjoint's gradient products use; the
        // mixed solver's state update needs only the correction d_total (dre, dim: two-float)
        double2 z[L];
        float4 zf[L];
        DF dre[L], dim[L];
        DF bre[L], bim[L];   // mixed solver: b = P u (conj(P) for the adjoint), two-float

        // first barrier of the step: the coefficients are published; thread 0 stores the
        // previous iteration's midpoints (forward) or fetches the next iteration's (adjoint)
        // the folding warps add iteration jj - 1's reduced products into the alpha-gradient right
        // after this iteration's first barrier (which published red[par ^ 1]): the other warps
        // then run FP32 sweeps, so the fold's FP64 chain does not queue behind the FP64 work
        // every warp issues at the ends of a step
        auto fold_previous = [&]() {
            if (BWD && jj > 0 && fold_warp && jj - 1 < (fslot ? cnt_1 : cnt_0))
                fold(fslot, par ^ 1, step_of(fslot, jj - 1), sp_prev, ph_prev, true,
                     ((jj - 1) & (FOLD_FLUSH - 1)) == FOLD_FLUSH - 1 || jj == (fslot ? cnt_1 : cnt_0));
        };
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
            // right-hand side of the preconditioned step equation: b = P u (conj(P) for the adjoint)
            double2 b[L];
#pragma unroll
            for (int l = 0; l < L; ++l) b[l] = cmul(Pd[l], u[l]);
            // Dc/Dn alternate on every write (persisting across steps): a buffer is never
            // rewritten before the sync that follows its last read.
#pragma unroll
            for (int l = 0; l < L; ++l) z[l] = b[l];
            if (act) {
#pragma unroll
                for (int l = 0; l < L; ++l) Dc[fb.xo + l] = z[l];
            }
            tile_sync();
            first_sync_work();
            if (timed_out) break;
            fold_previous();
            const int Kown = prm[0];
            const int Kmax = nslot > 1 ? max(prm0[0], prm1[0]) : prm0[0];
            for (int it = 0; it < Kmax; ++it) {
                if (it > 0) {
                    if (act) {
#pragma unroll
                        for (int l = 0; l < L; ++l) Dc[fb.xo + l] = z[l];
                    }
                    tile_sync();
                }
                double2 w[L];
                apply_off<L, Q, double2>(Dc, cfd, fb, z, w, pd);
                if (it < Kown) {
#pragma unroll
                    for (int l = 0; l < L; ++l) z[l] = cadd_scaled<S>(b[l], Pd[l], w[l]);
                }
                double2* tmp = Dc;
                Dc = Dn;
                Dn = tmp;
            }
        } else {
            // ---- b = P u (conj(P) for the adjoint) as a two-float sum in the column's scaled
            // units: the FP32 stage's right-hand side and the point at which the refinement
            // evaluates the off-diagonal apply.  The residual below is that of the exact P u
            // (it is formed as s P w(z) - d_total), so b's 2^-47 error enters the solve only
            // through the evaluation point of a term of size rho.  The state update takes R u
            // either in FP64 (R = 2P - 1) or, compensated, as u + 2 kappa (Im b, -Re b), where
            // b's error enters times |2 kappa| <= 2^-4.5; there the state is u + carry, and
            // P carry (|carry| <= half an FP32 unit of the last increment) joins the low parts.
#pragma unroll
            for (int l = 0; l < L; ++l) {
                const float4 t = cq[f * L + l];
                carry_rhs(split_scaled(u[l], sh), Ps[l], make_float2(t.y, t.z), car[l], bre[l], bim[l]);
            }
            // ---- FP32 stage: d = Ubar - b from the preconditioned fixed point d = s P w(b + d)
            float2 bf[L], df[L], y[L];
#pragma unroll
            for (int l = 0; l < L; ++l) {
                bf[l] = make_float2(fadd_n(bre[l].s, bre[l].c), fadd_n(bim[l].s, bim[l].c));
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
                first_sync_work();
                if (timed_out) break;
                fold_previous();
                float2 w[L];
                apply_off<L, Q, float2>(Fb, cff, fb, y, w, pd);
#pragma unroll
                for (int l = 0; l < L; ++l) df[l] = cadd_scaled<S>(make_float2(0.f, 0.f), Pf[l], w[l]);
            }
            const int j1 = prm[0], j2 = prm[1], R = prm[2];
            const int j1max = nslot > 1 ? max(prm0[0], prm1[0]) : prm0[0];
            const int j2max = nslot > 1 ? max(prm0[1], prm1[1]) : prm0[1];
            const int Rmax = nslot > 1 ? max(prm0[2], prm1[2]) : prm0[2];
            for (int it = 1; it < j1max; ++it) {
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
                apply_off<L, Q, float2>(Fb, cff, fb, y, w, pd);
                if (it < j1) {
#pragma unroll
                    for (int l = 0; l < L; ++l) df[l] = cadd_scaled<S>(make_float2(0.f, 0.f), Pf[l], w[l]);
                }
            }
            // ---- refinement: z = b + d_total, residual r = s P w(z) - d_total (that of the exact
            // P u), an FP32 correction e added to d_total (two-float, scaled units)
#pragma unroll
            for (int l = 0; l < L; ++l) {
                dre[l] = DF{df[l].x, 0.f};
                dim[l] = DF{df[l].y, 0.f};
            }
            // the residual's apply in compensated FP32 (split entries in D0) where the step's
            // contraction factor (exchange included) allows it (step_counts) and the exchange
            // terms, if any, have precomputed sources, else in FP64; uniform over a slot, so a
            // column's entries in D0 have one form
            const bool dfa = (pd.nex == 0 || (L == 2 && pd.nex <= MAXEXF)) && !(prm[3] & 2);
            float4* D0s = reinterpret_cast<float4*>(D0);
            for (int pass = 0;; ++pass) {
                float4 zs[L];
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    const DF zr = df_add(bre[l], dre[l]), zi = df_add(bim[l], dim[l]);
                    zs[l] = make_float4(zr.s, zi.s, zr.c, zi.c);
                }
                if (dfa) {
                    if (act) {
#pragma unroll
                        for (int l = 0; l < L; ++l) D0s[fb.xo + l] = zs[l];
                    }
                } else if (act) {
                    SplitVals<L> zv;
#pragma unroll
                    for (int l = 0; l < L; ++l) zv.v[l] = zs[l];
                    store_z64<L>(D0 + fb.xo, zv, sh);
                }
                // forward: the staged midpoints of the previous step must have been read by their
                // bulk store (issued at this step's first barrier) before this step's are staged;
                // waiting here, ahead of a barrier every step has, makes the staging barrier-free
                if (!BWD && want_hist && pass == 0 && tid == 0 && hpos == 0) bulk_wait_read_all();
                tile_sync();
                float2 rf[L], e[L];
                if (dfa) {
                    DF w[L][2];
                    apply_off_df<L, Q>(D0s, cfs, fb, zs, w, exc, pd.nex);
#pragma unroll
                    for (int l = 0; l < L; ++l) {
                        rf[l] = resid_df<S>(make_float2(dre[l].s, dim[l].s), make_float2(dre[l].c, dim[l].c), Ps[l],
                                            w[l]);
                        e[l] = rf[l];
                    }
                } else {
                    ResidIn<L> in;
#pragma unroll
                    for (int l = 0; l < L; ++l) {
                        in.zs[l] = zs[l];
                        in.dre[l] = dre[l];
                        in.dim[l] = dim[l];
                    }
                    const ResidOut<L> o = resid_fp64<L, Q, S, BWD>(D0, cfd, pd, c, f, a.cpt * N, in, sh);
#pragma unroll
                    for (int l = 0; l < L; ++l) {
                        rf[l] = o.r[l];
                        e[l] = rf[l];
                    }
                }
                for (int it = 0; it < j2max; ++it) {
                    float2* Fb = fsel ? FB : FA;
                    fsel ^= 1;
                    if (act) {
#pragma unroll
                        for (int l = 0; l < L; ++l) Fb[fb.xo + l] = e[l];
                    }
                    tile_sync();
                    float2 wf[L];
                    apply_off<L, Q, float2>(Fb, cff, fb, e, wf, pd);
                    if (it < j2) {
#pragma unroll
                        for (int l = 0; l < L; ++l) e[l] = cadd_scaled<S>(rf[l], Pf[l], wf[l]);
                    }
                }
                if (pass < R) {
#pragma unroll
                    for (int l = 0; l < L; ++l) {
                        dre[l] = df_add(dre[l], DF{e[l].x, 0.f});
                        dim[l] = df_add(dim[l], DF{e[l].y, 0.f});
                    }
                }
                if (pass + 1 >= Rmax) break;
                // another pass rewrites D0: every thread must be done reading it
                tile_sync();
            }
#pragma unroll
            for (int l = 0; l < L; ++l) {
                const DF zr = df_add(bre[l], dre[l]), zi = df_add(bim[l], dim[l]);
                zf[l] = make_float4(zr.s, zi.s, zr.c, zi.c);
            }
        }
        if (tid == 0 && ((prm0[3] & 1) || (nslot > 1 && (prm1[3] & 1)))) atomicOr(pd.status, ST_SOLVER_RANGE);
        // the state update (U_{n+1} = 2 Ubar - U_n; Lambda_n = 2 Lbar - Lambda_{n+1}) as soon as
        // the step is solved: what follows (history, gradient products) needs only the midpoint
        if (live) state_update(u, z, bre, bim, dre, dim);

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
                if (act && live) {
                    if constexpr (SOLVER == SOLVER_MIXED) {
                        // the adjoint's gradient products read the split form (products_split)
                        float4* Hs = reinterpret_cast<float4*>(H) + size_t(hpos) * hstride + fb.xo;
#pragma unroll
                        for (int l = 0; l < L; ++l) Hs[l] = zf[l];
                    } else {
#pragma unroll
                        for (int l = 0; l < L; ++l) H[size_t(hpos) * hstride + fb.xo + l] = z[l];
                    }
                }
                fence_proxy_async_smem();
            }
            // roll-out: U(t_m) when the step ends on a window boundary t_m, i.e. when n + 1 =
            // floor(m N_T / M) for some 1 <= m < M; the only candidate is m = ceil((n+1) M / N_T)
            if (rollout && live && act) {
                const int64_t n1 = wn0_0 + jj + 1;
                const int64_t mb = (n1 * pd.M + pd.nsteps - 1) / pd.nsteps;
                if (mb >= 1 && mb < pd.M && (mb * pd.nsteps) / pd.M == n1) {
                    double2* dst = a.out + (size_t(mb - 1) * E + col) * N + f * L;
#pragma unroll
                    for (int l = 0; l < L; ++l) dst[l] = state_out(l);
                }
            }
        } else {
            // ---- gradient quadrature on the midpoints (fused): needs Ubar_n of the tile
            double2* UB = ((hgrp & 1) ? UB1 : UB0) + size_t(hpos) * hstride;
            // a wait that gives up raises the tile's flag, read after the next barrier (the
            // products below then use whatever landed; the evaluation reports the timeout)
            if (hpos == 0 && !mbar_wait(&mbar[hgrp & 1], (hgrp >> 1) & 1)) *tflag = 1;
            GT acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) gsum_zero(acc[v]);
            if constexpr (SOLVER == SOLVER_MIXED) {
                products_split<L, Q>(zf, reinterpret_cast<const float4*>(UB), fb, pscale, acc);
            } else {
            {
                // last subsystem (stride 1) from the fiber itself, grouped by entry l of Lbar:
                // A += Im(conj(Lbar_l) v+), B += Re(conj(Lbar_l) v-) with
                // v+- = sqrt(l+1) Ubar_{l+1} +- sqrt(l) Ubar_{l-1} (the z and y terms of entry l)
                constexpr int kl = Q - 1;
                double A = 0.0, B = 0.0;
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    constexpr double kOne = 1.0;
                    const double wp = l < L - 1 ? sqrt_small(l + 1) : 0.0;   // folded after unrolling
                    const double wm = l > 0 ? sqrt_small(l) : 0.0;
                    const double2 zl = z[l];
                    if (wp != 0.0 && wm != 0.0) {
                        const double2 up = UB[fb.xo + l + 1], um = UB[fb.xo + l - 1];
                        double2 vp, vm;
                        if (wp == kOne) {
                            vp = make_double2(up.x + wm * um.x, up.y + wm * um.y);
                            vm = make_double2(up.x - wm * um.x, up.y - wm * um.y);
                        } else if (wm == kOne) {
                            vp = make_double2(fma(wp, up.x, um.x), fma(wp, up.y, um.y));
                            vm = make_double2(fma(wp, up.x, -um.x), fma(wp, up.y, -um.y));
                        } else {
                            vp = make_double2(fma(wp, up.x, wm * um.x), fma(wp, up.y, wm * um.y));
                            vm = make_double2(fma(wp, up.x, -wm * um.x), fma(wp, up.y, -wm * um.y));
                        }
                        A = fma(zl.x, vp.y, fma(-zl.y, vp.x, A));
                        B = fma(zl.x, vm.x, fma(zl.y, vm.y, B));
                    } else {
                        // one term: plus (first entry) or minus (last), weight w
                        const bool plus = wp != 0.0;
                        const double w = plus ? wp : wm;
                        const double2 u = UB[fb.xo + (plus ? l + 1 : l - 1)];
                        if (w == kOne) {
                            A = fma(zl.x, u.y, fma(-zl.y, u.x, A));
                            B = plus ? fma(zl.x, u.x, fma(zl.y, u.y, B)) : fma(-zl.x, u.x, fma(-zl.y, u.y, B));
                        } else {
                            const double ti = fma(zl.x, u.y, -zl.y * u.x), tr = fma(zl.x, u.x, zl.y * u.y);
                            A = fma(w, ti, A);
                            B = fma(plus ? w : -w, tr, B);
                        }
                    }
                }
                acc[2 * kl + 0] = A;
                acc[2 * kl + 1] = B;
            }
#pragma unroll
            for (int k = 0; k < Fiber<L, Q>::NFIX; ++k) {
                double2 p = make_double2(0.0, 0.0);
                const double2* q1 = UB + fb.nb1[k];
#pragma unroll
                for (int l = 0; l < L; ++l) cjmac(p, z[l], q1[l]);
                // entry 1 is a z_k term (a_k) or, for a fiber at the top level, a y_k term
                // (a_k^+); entry 2, where there is one, a y_k term: A = Im z + Im y, B = Re z - Re y
                double A, B;
                if (fb.two[k]) {   // an interior level (warp-uniform: lanes are sorted by class)
                    double2 p2 = make_double2(0.0, 0.0);
                    const double2* q2 = UB + fb.nb2[k];
#pragma unroll
                    for (int l = 0; l < L; ++l) cjmac(p2, z[l], q2[l]);
                    if constexpr (L == 3) {   // level 1 of 3: weights sqrt(2) (a_k) and 1 (a_k^+)
                        A = fma(fb.w1[k], p.y, p2.y);
                        B = fma(fb.w1[k], p.x, -p2.x);
                    } else {
                        A = fma(fb.w1[k], p.y, fb.w2[k] * p2.y);
                        B = fma(fb.w1[k], p.x, -fb.w2[k] * p2.x);
                    }
                } else {
                    const double sw1 = fb.plus1[k] ? fb.w1[k] : -fb.w1[k];
                    A = fb.w1[k] * p.y;
                    B = sw1 * p.x;
                }
                acc[2 * k + 0] = A;
                acc[2 * k + 1] = B;
            }
            }   // FP64 products
            if (!act || !live) {
#pragma unroll
                for (int v = 0; v < V; ++v) gsum_zero(acc[v]);
            }
            // per-slot warp sums: lane (lane >> (5 - NH)) == v holds value v
            {
                const int vi = lane >> (5 - NH);
                const bool writer = (lane & ((1 << (5 - NH)) - 1)) == 0;
                GT* r0 = red + ((par * 2 + 0) * nwarps + warp) * V;
                GT* r1 = red + ((par * 2 + 1) * nwarps + warp) * V;
                GT zero;
                gsum_zero(zero);
                // a warp with lanes of both windows reduces each window's lanes in a pass of its
                // own (one copy of the reduction in the code: the step loop's instruction fetches
                // already stall the adjoint's warps)
                const bool both = mask0 && mask1;
                for (int pass = 0; pass < (both ? 2 : 1); ++pass) {
                    GT t[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) t[v] = (!both || slot == pass) ? acc[v] : zero;
                    const GT sv = warp_reduce_scatter<V, NH>(t, lane);
                    if (writer) {
                        if (!both) {
                            r0[vi] = mask1 ? zero : sv;
                            if (nslot > 1) r1[vi] = mask1 ? sv : zero;
                        } else {
                            (pass == 0 ? r0 : r1)[vi] = sv;
                        }
                    }
                }
            }
        }

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
            if (a.mode != SWEEP_RECOMPUTE && !rollout && act && my_cnt > 0) {
#pragma unroll
                for (int l = 0; l < L; ++l) pd.Uend[wcol + f * L + l] = state_out(l);
            }
        } else {
            // the last fold of every slot whose range ends at the last iteration
            if (fold_warp && nit > 0 && (fslot ? cnt_1 : cnt_0) == nit) {
                const int64_t np = step_of(fslot, nit - 1);
                fold(fslot, (nit - 1) & 1, np, pd.spl[np], make_double2(0.0, 0.0), false, true);
            }
            tile_sync();
            // the tile's alpha-gradient partial, accumulated over the segment launches (the first
            // adjoint launch is the last segment's)
            double* gp = pd.gpart + size_t(tile.tloc) * pd.d;
            const bool first_launch = a.seg == pd.nseg - 1;
            store_grad_partial(gp, galpha, pd, a.gmax, slo_0, nslot > 1 ? slo_1 : -1, first_launch);
            // Lambda at the segment start: Lambda^m(t_{m-1}) for the window's first segment
            if (act && my_cnt > 0) {
                double2* dst = my_lo == 0 ? pd.Lam0 : pd.Lstate;
#pragma unroll
                for (int l = 0; l < L; ++l) dst[wcol + f * L + l] = state_out(l);
            }
        }
    } else if (tid == 0) {
        atomicOr(pd.status, ST_TIMEOUT);
        // let the bulk copies this tile issued land before its shared memory is released
        for (int p2 = 0; p2 < 2; ++p2) (void)mbar_wait(&mbar[p2], 0), (void)mbar_wait(&mbar[p2], 1);
    }
}

}  // namespace msqoc
