// Small kernels around the sweeps: control evaluation, window terminal conditions and the
// deterministic final reductions.
#pragma once

#include "msqoc_internal.h"

namespace msqoc {

// Iteration counts of the implicit-midpoint solve of one step from the contraction bound
// rho = ||P iX_C|| <= (h/2) lam sum_k |d_k(t_{n+1/2})| of the diagonally preconditioned
// fixed point (P = (I + i h/2 D)^-1).  Packed as j1 | j2 << 8 | passes << 16 | bad << 24.
//   FP64 solver : j1 = K sweeps with rho^(K+1) <= 2^-56.
//   mixed solver: the FP32 stage leaves the error e1 = c u32 rho + rho^(j1+1) relative to
//     |P rhs| (FP32 rounding of the right-hand side and of the sweeps, times the contraction,
//     plus truncation); each FP64 residual + FP32 correction multiplies it by
//     phi = c u32 + rho^(j2+1).  c = 4 rounding units per FP32 sweep output; target: the FP64
//     unit roundoff 2^-53.  An FP64 pass costs far more than FP32 sweeps, so the fewest passes R
//     are taken first, then the fewest FP32 sweeps j1 + j2 (each sweep is a barrier of the
//     tile), then the smaller j2.
//   bad: rho >= 1/2, outside the range the counts are derived for.
__device__ inline int step_counts(int solver, float rho) {
    int a = 1, b = 1, r = 1, bad = 0;
    if (rho > 1e-30f) {
        const float lr = logf(rho);
        if (solver == SOLVER_FP64) {
            a = int(ceilf(-38.8162f / lr)) - 1;   // log(2^-56) = -38.816
            a = a < 1 ? 1 : (a > 60 ? 60 : a);
        } else {
            const float u32 = 5.9604645e-8f, c = 4.f, target = 1.1102230e-16f;
            const int j0 = max(1, min(30, int(ceilf(logf(u32) / lr))));   // rho^j0 <= u32
            r = 0;
            for (int pass = 1; pass <= 6 && r == 0; ++pass) {
                int best = 0;
                for (int ja = 1; ja <= j0 + 2; ++ja) {
                    const float e1 = c * u32 * rho + __powf(rho, float(ja + 1));
                    for (int jb = 1; jb <= j0 + 1; ++jb) {
                        const float phi = c * u32 + __powf(rho, float(jb + 1));
                        float e = e1;
                        for (int t = 0; t < pass; ++t) e *= phi;
                        if (e <= target && (best == 0 || ja + jb < best || (ja + jb == best && jb < b))) {
                            best = ja + jb;
                            a = ja;
                            b = jb;
                        }
                    }
                }
                if (best) r = pass;
            }
            if (r == 0) {
                a = min(30, j0 + 2);
                b = min(30, j0 + 1);
                r = 6;
            }
        }
        if (rho >= 0.5f) bad = 1;
    }
    // the compensated FP32 apply of the residual (error about 2^-47 |P iX_C z| <= 2^-47 rho |z|)
    // stays below the FP64 rounding of z (2^-53 |z|) for rho <= 2^-7; above, the FP64 apply
    const int f64_apply = rho > 0.0078125f ? 1 : 0;
    return a | (b << 8) | (r << 16) | (bad << 24) | (f64_apply << 25);
}

// The quadratic cardinal B-splines active at time t: on [j dtau, (j+1) dtau) the three
// non-zero splines are s = j, j+1, j+2 with weights (1-x)^2/2, 3/4 - (x-1/2)^2, x^2/2
// (x = t/dtau - j); j is clamped to [0, d1 - 3].
struct SplineAt {
    int s0;
    double w0, w1, w2;
};

__device__ __forceinline__ SplineAt spline_at(const ProbDev& pd, double t) {
    const double tau = t / pd.dtau;
    const int s0 = spline_index(t, pd.dtau, pd.d1);
    const double x = tau - s0;
    return SplineAt{s0, 0.5 * (1.0 - x) * (1.0 - x), 0.75 - (x - 0.5) * (x - 0.5), 0.5 * x * x};
}

// Controls at every step midpoint t_{n+1/2} = (n + 1/2) h (Eq. dj-ctrl with the quadratic
// B-spline envelope of Sec. 2): d_k(t) = sum_f e^{i Omega_kf t} sum_s (a1 + i a2)_kfs B_s(t),
// and the step solver's iteration counts (step_counts).  Also stores the spline weights for the
// gradient quadrature of the adjoint sweep.  The carrier phases come from the problem's phase
// table (k_phases).
__global__ void k_controls(const ProbDev pd) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < pd.nsteps; n += stride) {
        const double t = (double(n) + 0.5) * pd.h;
        const SplineAt sp = spline_at(pd, t);
        double mag = 0.0;   // sum_k |d_k| for the contraction bound
        for (int k = 0; k < pd.q; ++k) {
            double2 dk = make_double2(0.0, 0.0);
            for (int fi = pd.cof[k]; fi < pd.cof[k + 1]; ++fi) {
                const double2 ph = pd.phase[size_t(n) * pd.nfsum + fi];
                const double cs = ph.x, sn = ph.y;
                const double* a = pd.alpha + (size_t(fi) * pd.d1 + sp.s0) * 2;
                const double er = a[0] * sp.w0 + a[2] * sp.w1 + a[4] * sp.w2;
                const double ei = a[1] * sp.w0 + a[3] * sp.w1 + a[5] * sp.w2;
                dk.x += cs * er - sn * ei;
                dk.y += cs * ei + sn * er;
            }
            pd.ctrl[size_t(n) * pd.q + k] = dk;
            mag += sqrt(dk.x * dk.x + dk.y * dk.y);
        }
        const float rho = float(0.5 * pd.h * pd.lam * mag + pd.rho_ex) * 1.0001f;
        pd.spl[n] = Spline4{sp.s0, step_counts(pd.solver, rho), sp.w0, sp.w1, sp.w2};
    }
}

// The carrier phases e^{i Omega_f t} at every step midpoint t_{n+1/2} = (n + 1/2) h: they
// depend on the time grid and the carriers only, so the table is filled once per problem
// (per call for the allocation-free objective) and read by the controls, the adjoint's gradient
// quadrature and the regularization.
__global__ void k_phases(const ProbDev pd) {
    const int64_t total = pd.nsteps * pd.nfsum;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int64_t n = i / pd.nfsum;
        const int fi = static_cast<int>(i - n * pd.nfsum);
        const double t = (double(n) + 0.5) * pd.h;
        double sn, cs;
        sincos(pd.omega[fi] * t, &sn, &cs);
        pd.phase[i] = make_double2(cs, sn);
    }
}

// block-wide sum with a fixed reduction order (deterministic)
template <int NT>
__device__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
#pragma unroll
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

constexpr int TERM_THREADS = 256;

// Terminal conditions per window (Eq. terminal) and the window's objective term:
//   m < M: pen_m = mu/2 ||U^m - W^m||^2,  Lambda^m(t_m) = mu/2 (W^m - U^m)
//   m = M: gamma = <V, U^M>, J = ||U^M||^2/E - |gamma|^2/E^2, Lambda^M(t_M) = (gamma V - E U^M)/E^2
// (m and M global: a shard's last window is the problem's last only when it ends the grid)
__global__ void __launch_bounds__(TERM_THREADS) k_terminal(const ProbDev pd, const int want_lambda) {
    __shared__ double sh[TERM_THREADS];
    const int m = blockIdx.x + 1;
    const size_t ne = size_t(pd.N) * pd.E;
    const double2* U = pd.Uend + size_t(m - 1) * ne;
    double2* Lt = pd.Lterm + size_t(m - 1) * ne;
    if (m + pd.m_off < pd.M_glob) {
        const double2* Wm = pd.W + size_t(m - 1) * ne;
        double s = 0.0;
        for (size_t e = threadIdx.x; e < ne; e += TERM_THREADS) {
            const double2 u = U[e], w = Wm[e];
            const double cx = u.x - w.x, cy = u.y - w.y;
            s = fma(cx, cx, fma(cy, cy, s));
            if (want_lambda) Lt[e] = make_double2(-0.5 * pd.mu * cx, -0.5 * pd.mu * cy);
        }
        s = block_sum<TERM_THREADS>(s, sh);
        if (threadIdx.x == 0) pd.term[m - 1] = 0.5 * pd.mu * s;
    } else {
        double gr = 0.0, gi = 0.0, nr = 0.0;
        for (size_t e = threadIdx.x; e < ne; e += TERM_THREADS) {
            const double2 u = U[e], v = pd.V[e];
            gr = fma(v.x, u.x, fma(v.y, u.y, gr));
            gi = fma(v.x, u.y, fma(-v.y, u.x, gi));
            nr = fma(u.x, u.x, fma(u.y, u.y, nr));
        }
        gr = block_sum<TERM_THREADS>(gr, sh);
        gi = block_sum<TERM_THREADS>(gi, sh);
        nr = block_sum<TERM_THREADS>(nr, sh);
        const double E = pd.E;
        if (threadIdx.x == 0) pd.term[m - 1] = nr / E - (gr * gr + gi * gi) / (E * E);
        if (want_lambda) {
            const double inv = 1.0 / (E * E);
            for (size_t e = threadIdx.x; e < ne; e += TERM_THREADS) {
                const double2 u = U[e], v = pd.V[e];
                const double lx = (gr * v.x - gi * v.y) - E * u.x;
                const double ly = (gr * v.y + gi * v.x) - E * u.y;
                Lt[e] = make_double2(lx * inv, ly * inv);
            }
        }
    }
}

// P = J + sum_m pen_m (window order), J and pen outputs, and the alpha-gradient as the sum of
// the per-tile partials in tile order.  A shard sums its own windows' terms; J is 0 unless its
// last window is the problem's last.
__global__ void k_finalize_scalars(const ProbDev pd, double* P_out, double* J_out, double* pen_out,
                                   double* galpha_out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const bool has_last = pd.m_off + pd.M == pd.M_glob;
        double P = 0.0;
        for (int m = 1; m <= pd.M; ++m) P += pd.term[m - 1];
        if (P_out) *P_out = P;
        if (J_out) *J_out = has_last ? pd.term[pd.M - 1] : 0.0;
        if (pen_out)
            for (int m = 1; m <= pd.M - (has_last ? 1 : 0); ++m) pen_out[m - 1] = pd.term[m - 1];
    }
    if (galpha_out) {
        for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < pd.d; l += gridDim.x * blockDim.x) {
            double s = 0.0;
            for (int t = 0; t < pd.ntiles; ++t) s += pd.gpart[size_t(t) * pd.d + l];
            galpha_out[l] = s;
        }
    }
}

// Roll-out infidelity estimate (Eq. rollout-infid-est) from the last evaluation's window terms:
//   J + (2 / sqrt(n)) sqrt(J) S + S^2 / n,  S = sum_{m<M} ||C^m||_F,  ||C^m||_F = sqrt(2 pen_m / mu),
// with n := E (as in the generalized infidelity).  Window order sum (deterministic).
__global__ void k_rollout_estimate(const ProbDev pd, double* est) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double S = 0.0;
        for (int m = 1; m < pd.M; ++m) S += sqrt(2.0 * pd.term[m - 1] / pd.mu);
        const double J = pd.term[pd.M - 1];
        const double n = pd.E;
        *est = J + 2.0 / sqrt(n) * sqrt(fmax(J, 0.0)) * S + S * S / n;
    }
}

// dP/dW^k = mu (W^k - U^k(t_k)) - 2 Lambda^{k+1}(t_k) = 2 (Lambda^k(t_k) - Lambda^{k+1}(t_k))
// (Eq. dP-dW with the factor of Appendix B, Eq. dT-dW-j), k = 1..M-1.  A shard (global windows
// m_off + 1 .. m_off + M) writes, for the window states it reads (k = max(m_off, 1) ..
// min(m_off + M, M_glob - 1)), the terms it owns: 2 Lambda^k(t_k) if window k is its own,
// -2 Lambda^{k+1}(t_k) if window k + 1 is.
__global__ void k_grad_W(const ProbDev pd, double2* gW, int nblocks) {
    const size_t ne = size_t(pd.N) * pd.E;
    const size_t total = ne * size_t(nblocks);
    const int kfirst = pd.m_off > 1 ? pd.m_off : 1;
    for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += size_t(gridDim.x) * blockDim.x) {
        const int k = kfirst + static_cast<int>(e / ne);
        const size_t i = e % ne;
        const int jk = k - pd.m_off;                  // local index of window k (own if >= 1)
        const bool own_k = jk >= 1, own_next = jk + 1 <= pd.M;
        const double2 lt = own_k ? pd.Lterm[size_t(jk - 1) * ne + i] : make_double2(0.0, 0.0);
        const double2 l0 = own_next ? pd.Lam0[size_t(jk) * ne + i] : make_double2(0.0, 0.0);
        gW[e] = own_k && own_next ? make_double2(2.0 * (lt.x - l0.x), 2.0 * (lt.y - l0.y))
                                  : (own_k ? make_double2(2.0 * lt.x, 2.0 * lt.y)
                                           : make_double2(-2.0 * l0.x, -2.0 * l0.y));
    }
}

constexpr int REG_THREADS = 256;

// Regularization of the optimisation problem (Sec. 5): R = (gamma_tik/2) ||alpha||^2 +
// gamma_energy E with the time-averaged control-pulse energy E = (h/T) sum_n sum_k
// |d_k(t_{n+1/2})|^2 (the midpoint rule of (1/T) int_0^T sum_k |d_k|^2 dt on the time grid).
// One block per (subsystem k, spline s), over the steps where spline s is active (its weight
// B = w_{s - s0}):
//   dR/d alpha1_kfs = gamma_tik alpha1_kfs + 2 gamma_energy (h/T) sum_n B Re(conj(d_k) e^{i Omega_kf t}),
//   dR/d alpha2_kfs = gamma_tik alpha2_kfs - 2 gamma_energy (h/T) sum_n B Im(conj(d_k) e^{i Omega_kf t}),
// and the block's share of the energy, (h/T) sum |d_k|^2 over the steps whose first active
// spline is s (each step is counted by exactly one block per k).  Every sum has a fixed order.
// A pass over the steps evaluates d_k once per step and accumulates the energy and up to
// REG_CHUNK carriers' sums (the paper's subsystems have 2-3 carriers: one pass).
constexpr int REG_CHUNK = 4;
__global__ void __launch_bounds__(REG_THREADS) k_regularization(const ProbDev pd, const double* alpha,
                                                                 double gamma_tik, double gamma_energy,
                                                                 double* grad, double* epart) {
    __shared__ double sh[REG_THREADS];
    const int k = blockIdx.x / pd.d1, s = blockIdx.x % pd.d1;
    // steps whose midpoint lies in [(s - 2) dtau, (s + 1) dtau), widened by two steps on each side
    // (membership is decided exactly by spline_at below)
    const double r = pd.dtau / pd.h;
    const int64_t lo = max(int64_t(0), int64_t(floor((s - 2) * r - 0.5)) - 2);
    const int64_t hi = min(pd.nsteps, int64_t(ceil((s + 1) * r)) + 2);
    const int f0 = pd.cof[k], nfk = pd.cof[k + 1] - f0;
    const double wt = pd.h / pd.T;   // midpoint weight of the time average
    for (int c0 = 0; c0 < nfk; c0 += REG_CHUNK) {   // carriers f0 + c0 .. f0 + c0 + REG_CHUNK - 1
        double are[REG_CHUNK], aim[REG_CHUNK], en = 0.0;
#pragma unroll
        for (int c = 0; c < REG_CHUNK; ++c) are[c] = aim[c] = 0.0;
        for (int64_t n = lo + threadIdx.x; n < hi; n += REG_THREADS) {
            const double t = (double(n) + 0.5) * pd.h;
            const SplineAt sp = spline_at(pd, t);
            const int j = s - sp.s0;
            if (j < 0 || j > 2) continue;
            double2 dk = make_double2(0.0, 0.0);
            double2 ph[REG_CHUNK];
#pragma unroll
            for (int c = 0; c < REG_CHUNK; ++c) ph[c] = make_double2(0.0, 0.0);
            for (int g = f0; g < f0 + nfk; ++g) {
                const double2 pg = pd.phase[size_t(n) * pd.nfsum + g];   // the problem's phase table
                const double cs = pg.x, sn = pg.y;
                const double* a = alpha + (size_t(g) * pd.d1 + sp.s0) * 2;
                const double er = a[0] * sp.w0 + a[2] * sp.w1 + a[4] * sp.w2;
                const double ei = a[1] * sp.w0 + a[3] * sp.w1 + a[5] * sp.w2;
                dk.x += cs * er - sn * ei;
                dk.y += cs * ei + sn * er;
#pragma unroll
                for (int c = 0; c < REG_CHUNK; ++c)
                    if (g == f0 + c0 + c) ph[c] = pg;
            }
            if (c0 == 0 && j == 0) en += dk.x * dk.x + dk.y * dk.y;
            const double B = j == 0 ? sp.w0 : (j == 1 ? sp.w1 : sp.w2);
#pragma unroll
            for (int c = 0; c < REG_CHUNK; ++c) {   // conj(d_k) e^{i Omega t}
                are[c] += B * (dk.x * ph[c].x + dk.y * ph[c].y);
                aim[c] += B * (dk.x * ph[c].y - dk.y * ph[c].x);
            }
        }
        if (c0 == 0) {
            const double se = block_sum<REG_THREADS>(en, sh);
            if (threadIdx.x == 0) epart[blockIdx.x] = wt * se;
        }
#pragma unroll
        for (int c = 0; c < REG_CHUNK; ++c) {
            if (c0 + c >= nfk) break;                  // block-uniform
            const double sre = block_sum<REG_THREADS>(are[c], sh);
            const double sim = block_sum<REG_THREADS>(aim[c], sh);
            if (threadIdx.x == 0) {
                const size_t i = (size_t(f0 + c0 + c) * pd.d1 + s) * 2;
                grad[i] = gamma_tik * alpha[i] + 2.0 * gamma_energy * wt * sre;
                grad[i + 1] = gamma_tik * alpha[i + 1] - 2.0 * gamma_energy * wt * sim;
            }
        }
    }
}

// R from the energy shares of k_regularization and ||alpha||^2 (one block, fixed order)
__global__ void __launch_bounds__(REG_THREADS) k_regularization_total(const ProbDev pd, const double* alpha,
                                                                       double gamma_tik, double gamma_energy,
                                                                       const double* epart, double* R) {
    __shared__ double sh[REG_THREADS];
    double a2 = 0.0, en = 0.0;
    for (int i = threadIdx.x; i < pd.d; i += REG_THREADS) a2 += alpha[i] * alpha[i];
    for (int i = threadIdx.x; i < pd.q * pd.d1; i += REG_THREADS) en += epart[i];
    a2 = block_sum<REG_THREADS>(a2, sh);
    en = block_sum<REG_THREADS>(en, sh);
    if (threadIdx.x == 0) *R = 0.5 * gamma_tik * a2 + gamma_energy * en;
}

}  // namespace msqoc
