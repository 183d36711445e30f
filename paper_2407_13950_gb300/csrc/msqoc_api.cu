// Host side of libmsqoc: problem packing, tile layout, device memory, launches and the C ABI.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/msqoc.h"
#include "msqoc_aux.cuh"
#include "msqoc_internal.h"
#include "msqoc_host.h"
#include "msqoc_sweep_common.cuh"

using namespace msqoc;

namespace msqoc {

thread_local std::string g_last_error;

msqoc_status fail(msqoc_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}


int ipow_i(int b, int e) {
    int r = 1;
    while (e-- > 0) r *= b;
    return r;
}

// is p readable by kernels on the current device?
bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

constexpr int kMaxRows = 243;    // largest N of a supported shape (L = 3, q = 5)

bool shape_supported(int L, int q) { return (L == 3 && q >= 1 && q <= 5) || (L == 2 && q >= 1 && q <= 6); }

double ladder_norm(int L) {
    // largest eigenvalue of a + a^+ on L levels (zeros of the Hermite polynomial H_L / sqrt 2)
    switch (L) {
        case 2: return 1.0;
        case 3: return std::sqrt(3.0);
        case 4: return std::sqrt(3.0 + std::sqrt(6.0));
        default: return std::sqrt(2.0 * L);  // safe upper bound (Gershgorin)
    }
}

// Drift diagonal D_i of row i: self-Kerr -xi_k/2 l_k(l_k-1), optional detuning, cross-Kerr
// -xi_kl l_k l_l (the rotating-frame transmon form of Eq. sys-ham).
double drift_entry(const msqoc_hamiltonian* H, int q, int L, int i) {
    int lv[MAXQ];
    for (int k = 0; k < q; ++k) lv[k] = (i / ipow_i(L, q - 1 - k)) % L;
    double e = 0.0;
    for (int k = 0; k < q; ++k) {
        e += -0.5 * H->xi[k] * lv[k] * (lv[k] - 1);
        if (H->detune) e += H->detune[k] * lv[k];
        for (int l = k + 1; l < q; ++l)
            if (H->xi_cross) e -= H->xi_cross[k * q + l] * lv[k] * lv[l];
    }
    return e;
}

// diagonal preconditioner entry 1/(1 + i a), a = h D_i / 2
double2 precond_entry(double h, double D) {
    const double a = 0.5 * h * D;
    const double den = 1.0 + a * a;
    return make_double2(1.0 / den, -a / den);
}

// full row index of essential column e (base-ness digits -> base-L digits)
int essential_row(int q, int L, int ness, int e) {
    int i = 0, r = e;
    for (int k = q - 1, w = 1; k >= 0; --k, w *= L) {
        i += (r % ness) * w;
        r /= ness;
    }
    return i;
}

// QFT_E entry (e, j) = exp(2 pi i e j / E) / sqrt(E) (Sec. 5)
double2 qft_entry(int E, int e, int j) {
    const double s = 1.0 / std::sqrt(double(E));
    const long long pw = (long long)e * j % E;
    const double ang = 2.0 * M_PI * double(pw) / double(E);
    return make_double2(s * std::cos(ang), s * std::sin(ang));
}

// ------------------------------------------------------------------ tile layout
// Class of a fiber: bitmask of the fixed subsystems (all but the last) at an interior level,
// i.e. with a neighbour on both sides.  Lanes of one class take the same branches in the apply.
int fiber_class(int L, int q, int f) {
    int mask = 0;
    for (int k = 0; k < q - 1; ++k) {
        const int lk = (f / ipow_i(L, q - 2 - k)) % L;
        if (lk > 0 && lk < L - 1) mask |= 1 << k;
    }
    return mask;
}
// position of a mask in the reflected Gray-code sequence (neighbours differ in one bit)
int gray_rank(int g) {
    int r = 0;
    for (; g; g >>= 1) r ^= g;
    return r;
}

// Threads of a tile with ncol columns, the first ncol0 of window m0: each window's
// (column, fiber) pairs are ordered by the Gray rank of the fiber class, so that a warp spans
// few classes (its branch cost is the union of its lanes' branches); window m0's pairs come
// first so at most one warp has lanes of both windows.  Each (column, fiber) goes to one thread,
// to a lane pair for lane-pair tiles (pair = 1: threads 2i and 2i + 1, the real and the
// imaginary part) or to a lane quad (pair = 2: threads 4i..4i + 3, a pair per entry).  Idle
// lanes mirror the last active entry.  Writes out[nthreads]; no allocation.
void build_lanemap(int L, int q, int ncol, int ncol0, int nthreads, int pair, int* out) {
    const int F = ipow_i(L, q) / L;
    int key[MAX_ANY_TILE_THREADS], val[MAX_ANY_TILE_THREADS];
    if (ncol * F > MAX_ANY_TILE_THREADS || nthreads > MAX_ANY_TILE_THREADS) return;   // rejected by tile_width_ok
    int n = 0;
    for (int part = 0; part < 2; ++part) {
        const int first = n;
        const int ca = part == 0 ? 0 : ncol0, cb = part == 0 ? ncol0 : ncol;
        for (int f = 0; f < F; ++f)
            for (int c = ca; c < cb; ++c) {
                // stable insertion by key within this window's pairs
                const int k = gray_rank(fiber_class(L, q, f));
                int pos = n++;
                while (pos > first && key[pos - 1] > k) {
                    key[pos] = key[pos - 1];
                    val[pos] = val[pos - 1];
                    --pos;
                }
                key[pos] = k;
                val[pos] = (c << 16) | f;
            }
    }
    const int sh = pair;
    for (int t = 0; t < nthreads; ++t) out[t] = (t >> sh) < n ? val[t >> sh] : ~val[n - 1];
}

// Tile t of one problem for `cpt` columns per tile: a consecutive run of the window-major column
// list (windows m = 1..M, columns 0..E-1 each).  cpt <= E, so a tile covers at most two windows.
// Lane map index: ncol0 - 1 for full tiles, cpt for the (single, last) partial tile.
Tile tile_at(long t, int M, int E, int cpt, int prob) {
    const long total = long(M) * E, g0 = t * cpt;
    Tile x{};
    x.prob = prob;
    x.ncol = static_cast<int>(std::min<long>(cpt, total - g0));
    x.m0 = static_cast<int>(g0 / E) + 1;
    x.c0 = static_cast<int>(g0 % E);
    x.ncol0 = std::min(x.ncol, E - x.c0);
    x.map = x.ncol == cpt ? x.ncol0 - 1 : cpt;
    x.tloc = static_cast<int>(t);
    return x;
}
long tile_count(int M, int E, int cpt) { return (long(M) * E + cpt - 1) / cpt; }

// The cpt + 1 lane maps of a problem's tiles (out[(cpt + 1) * nthreads]); map cpt serves the
// last tile when it is partial.
void build_lanemaps(int L, int q, int M, int E, int cpt, int nthreads, int pair, int* out) {
    for (int k = 0; k < cpt; ++k) build_lanemap(L, q, cpt, k + 1, nthreads, pair, out + size_t(k) * nthreads);
    const Tile last = tile_at(tile_count(M, E, cpt) - 1, M, E, cpt, 0);
    build_lanemap(L, q, last.ncol, last.ncol0, nthreads, pair, out + size_t(cpt) * nthreads);
}

// one thread, a lane pair or a lane quad (2^pair threads) per (column, fiber)
int tile_threads(int cpt, int F, int pair) { return (((1 << pair) * cpt * F + 31) / 32) * 32; }
int max_tile_threads(int pair, int lean = 0) {
    return pair == 2 ? MAX_QUAD_TILE_THREADS : pair ? MAX_PAIR_TILE_THREADS : lean ? MAX_LEAN_TILE_THREADS : MAX_TILE_THREADS;
}

// Is `cpt` columns per tile usable in the given kernel family?  Tiles must fit the family's
// thread limit and the shared memory; a tile that covers two windows needs two warps (one per
// window's coefficients), so a one-warp tile must divide the window's columns.  g: doubles of
// the adjoint's shared alpha-gradient per window slot.
bool tile_width_ok(int cpt, int E, int F, int q, int L, int N, int g, int solver, int pair, int lean = 0) {
    if (cpt < 1 || cpt > E || (1 << pair) * cpt * F > max_tile_threads(pair, lean)) return false;
    const int nthreads = tile_threads(cpt, F, pair);
    if (nthreads == 32 && E % cpt) return false;
    const size_t s1 = sweep_layout(q, L, N, cpt, nthreads, g, solver, true, pair).total;
    const size_t s0 = sweep_layout(q, L, N, cpt, nthreads, g, solver, false, pair).total;
    return std::max(s0, s1) <= 200 * 1024;
}

// Lane quads serve 2-level subsystems whose exchange-coupled pairs all have precomputed sources.
bool quad_admitted(const ProbDev& pd) { return pd.L == 2 && pd.nex <= MAXEXF; }

// Kernel family and columns per tile.  Makespan model, from FP64 throughput probes and sweep
// timings on this GPU: a warp issues one FP64 instruction per 64 cycles on its SM sub-partition,
// an SM with four or more warps of FP64 work runs at its full rate, and every thread of a tile
// does the same FP64 work per step (idle lanes cost as much as busy ones).  In units of the
// step time of one one-thread-per-fiber warp alone on a sub-partition, a step of an SM holding
// w warps costs max(w c / 4, c0): c = c0 = 1 for that family; for lane pairs (half the FP64
// instructions a thread, plus shuffles) c = 0.6 at full SM load and c0 = 0.7 alone (measured:
// equal to the one-thread family on the 4-transmon tiles, 1.4x faster steps on small
// problems); for lane quads (2-level subsystems, a quarter of a fiber's work a thread)
// c = 0.38 and c0 = 0.52 (measured on the paper's QFT cases: steps 1.33-1.38x faster than lane
// pairs where the tiles are too few to fill the GPU; under load, from QFT-16 at 64 windows,
// seven one-warp quad tiles per SM take 0.73 of the time of one-thread tiles at the floor).
// Tiles that do not fit at once run in waves of the CTAs an SM holds (the kernels'
// occupancy at that width).  A tile over two windows pays a second coefficient set, gradient
// reduction and fold each step and wider class mixing in its warps: about one more warp's work
// per step, so its cost is taken (w + 1) / w times that of w warps (measured on the 4-transmon
// tiles: 6-warp two-window tiles as slow as 7-warp one-window ones, at 64 windows; 8-warp
// two-window tiles in three waves 7% faster than 7-warp one-window tiles in four, at 256
// windows, where (w + 1) / w predicts 4%).  Candidates are ranked by
//   1. the makespan: an SM's ceil(tiles / SMs) tiles in waves of `resident`, summed over the
//      waves;
//   2. tiles that stay inside one window;
//   3. where every wave sits at the single-warp floor (problems too small to fill the GPU, whose
//      candidates all tie there): tiles of 2 or 3 warps, then of 1, then of more (measured
//      there, 2-3 warp tiles step fastest:
//      fewer threads meet at each barrier than in wider tiles, and the coefficient and gradient
//      work of a tile is not serialised with the step as in one-warp tiles);
//   4. the idle-lane fraction of a tile.
// fixed_cpt > 0 restricts the width, layout (MSQOC_LAYOUT_*) the family; quad_ok: the problem
// admits lane quads.  cpt = -1: none fits.
constexpr double QUAD_C = 0.38, QUAD_C0 = 0.52;
// the one-thread family with 168 registers a thread: an SM holds 12 warps.  While the sweeps
// were bound by the FP64 pipe, two or more of its tiles on an SM did better than their warp
// count (each has its own barriers, so one tile's FP32 sweeps overlapped another's FP64 work)
// and a warp of such tiles counted 0.9.  With the mixed solver's compensated FP32 arithmetic
// the sweeps are bound by issue and dependency latency instead, and on the 4-transmon tiles one
// 14-column tile of 12 warps per SM steps 5% faster than two 7-column tiles (autotuner probes at
// 256 windows: 2.78 against 2.93 ms), so the lean build's warps count like any others
constexpr double LEAN_C = 1.0;
TileChoice choose_tile_layout(int M, int E, int F, int q, int L, int N, int g, int solver, int sms, int fixed_cpt,
                              int layout, bool quad_ok) {
    TileChoice best{-1, 0, 0};
    double best_a = 0.0, best_c = 0.0;
    int best_b = 0, best_w = 0;
    for (int fam = MSQOC_LAYOUT_FIBER; fam <= MSQOC_LAYOUT_FIBER_LEAN; ++fam) {
        if (layout != MSQOC_LAYOUT_AUTO && layout != fam) continue;
        const int pair = fam == MSQOC_LAYOUT_FIBER_LEAN ? 0 : fam - MSQOC_LAYOUT_FIBER;
        const int lean = fam == MSQOC_LAYOUT_FIBER_LEAN ? 1 : 0;
        if (pair == 2 && !quad_ok) continue;
        const double c_load = pair == 2 ? QUAD_C : pair ? 0.6 : 1.0;
        const double c_alone = pair == 2 ? QUAD_C0 : pair ? 0.7 : 1.0;
        const int hi = fixed_cpt > 0 ? fixed_cpt : std::min(E, max_tile_threads(pair, lean) / ((1 << pair) * F));
        const int lo = fixed_cpt > 0 ? fixed_cpt : 1;
        for (int cpt = hi; cpt >= lo; --cpt) {
            if (!tile_width_ok(cpt, E, F, q, L, N, g, solver, pair, lean)) continue;
            const long tiles = (long(M) * E + cpt - 1) / cpt;
            const int threads = tile_threads(cpt, F, pair);
            const int warps = threads / 32;
            SweepArgs a{};
            a.cpt = cpt;
            a.gmax = g;
            a.L = L;
            a.q = q;
            a.solver = solver;
            a.nthreads = threads;
            a.pair = pair;
            a.lean = lean;
            a.hdepth = 1;
            a.mode = SWEEP_HISTORY;
            const int r0 = sweep_ctas_per_sm(a);
            a.mode = SWEEP_ADJOINT;
            const int r1 = sweep_ctas_per_sm(a);
            const long resident = std::max(1, std::min(r0, r1));
            const long per_sm = (tiles + sms - 1) / sms;
            const long waves = (per_sm + resident - 1) / resident;
            const long last = per_sm - (waves - 1) * resident;
            const int cb = (E % cpt) ? 1 : 0;
            const double two = cb ? double(warps + 1) / double(warps) : 1.0;
            // a wave of n tiles on an SM; the lean build's warps count LEAN_C when two or more
            // of its tiles share the SM (independent tiles fall out of step)
            auto wave = [&](long n) {
                const double c = (lean && n >= 2 && warps >= 4) ? LEAN_C : c_load;
                return std::max(double(n * warps) * c / 4.0, c_alone);
            };
            const double ca = two * (double(waves - 1) * wave(resident) + wave(last));
            const double cc = 1.0 - double((1 << pair) * cpt * F) / (32.0 * warps);
            const bool at_floor = ca <= two * double(waves) * c_alone + 1e-9;
            const int cw = !at_floor ? 0 : ((warps == 2 || warps == 3) ? 0 : (warps == 1 ? 1 : 2));
            const bool tie_a = ca < best_a + 1e-9, tie_b = cb == best_b, tie_w = cw == best_w;
            const bool better = best.cpt < 0 || ca < best_a - 1e-9 ||
                                (tie_a && (cb < best_b || (tie_b && (cw < best_w || (tie_w && cc < best_c - 1e-9)))));
            if (better) {
                best = TileChoice{cpt, pair, lean};
                best_a = ca;
                best_b = cb;
                best_w = cw;
                best_c = cc;
            }
        }
    }
    return best;
}

// Validation of a problem description shared by every entry point that takes one.
msqoc_status check_description(const msqoc_hamiltonian* H, const msqoc_controls* C, double T, int64_t nsteps,
                               int32_t nwindows) {
    if (!H || !C) return fail(MSQOC_ERR_INVALID_ARG, "hamiltonian or controls is NULL");
    const int q = H->nqubits, L = H->nlevels, ness = H->ness;
    if (q < 1 || q > MAXQ || L < 2 || ness < 1 || ness > L || !H->xi)
        return fail(MSQOC_ERR_INVALID_ARG, "invalid subsystem description (q=%d L=%d ness=%d)", q, L, ness);
    if (!shape_supported(L, q))
        return fail(MSQOC_ERR_UNSUPPORTED, "no kernel for L=%d levels and q=%d subsystems", L, q);
    if (H->jx)
        for (int e = 0; e < q * q; ++e) {
            if (!std::isfinite(H->jx[e])) return fail(MSQOC_ERR_INVALID_ARG, "dipole exchange jx[%d] is not finite", e);
            if (H->jx[e] != 0.0 && L != 2)
                return fail(MSQOC_ERR_UNSUPPORTED, "dipole exchange is implemented for 2-level subsystems only");
        }
    if (!C->ncarriers || !C->carriers || C->nsplines < 3)
        return fail(MSQOC_ERR_INVALID_ARG, "invalid control description");
    if (!(T > 0) || !std::isfinite(T) || nsteps < 1 || nwindows < 1 || nwindows > nsteps)
        return fail(MSQOC_ERR_INVALID_ARG, "invalid time grid (T=%g nsteps=%lld M=%d)", T, (long long)nsteps, nwindows);
    if (nsteps > (int64_t(1) << 40)) return fail(MSQOC_ERR_INVALID_ARG, "nsteps too large");
    int nfsum = 0;
    for (int k = 0; k < q; ++k) {
        if (C->ncarriers[k] < 1) return fail(MSQOC_ERR_INVALID_ARG, "subsystem %d has no carrier", k);
        nfsum += C->ncarriers[k];
    }
    if (nfsum > MAXNF) return fail(MSQOC_ERR_INVALID_ARG, "too many carriers (%d > %d)", nfsum, MAXNF);
    return MSQOC_OK;
}

// Shape, time grid, model scalars and tile geometry of a validated description (every field
// of pd except the device pointers and the history segmentation).  col_block 0 = automatic.
msqoc_status shape_problem(const msqoc_hamiltonian* H, const msqoc_controls* C, double T, int64_t nsteps,
                           int32_t nwindows, double mu, int solver, int col_block, int layout, int sms, ProbDev& pd,
                           int wfirst = 0, int wlast = 0) {
    const int q = H->nqubits, L = H->nlevels, ness = H->ness;
    int nfsum = 0;
    for (int k = 0; k < q; ++k) nfsum += C->ncarriers[k];
    pd.q = q;
    pd.L = L;
    pd.ness = ness;
    pd.N = ipow_i(L, q);
    pd.E = ipow_i(ness, q);
    pd.F = pd.N / L;
    pd.d1 = C->nsplines;
    // windows: every one, or the shard wfirst..wlast (validated by the caller)
    pd.M_glob = nwindows;
    pd.m_off = wfirst > 0 ? wfirst - 1 : 0;
    pd.M = wfirst > 0 ? wlast - wfirst + 1 : nwindows;
    pd.nfsum = nfsum;
    pd.d = 2 * pd.d1 * nfsum;
    pd.nsteps = nsteps;
    pd.T = T;
    pd.h = T / double(nsteps);
    pd.mu = mu > 0 ? mu : 2.0 / pd.E;
    pd.dtau = T / double(pd.d1 - 2);
    pd.lam = ladder_norm(L);
    pd.solver = solver;
    pd.cof[0] = 0;
    for (int k = 0; k < q; ++k) {
        pd.nf[k] = C->ncarriers[k];
        pd.cof[k + 1] = pd.cof[k] + C->ncarriers[k];
    }
    for (int i = 0; i < nfsum; ++i) pd.omega[i] = C->carriers[i];
    // dipole exchange pairs (j < k): constant off-diagonal terms of the step operator; their norm
    // joins the contraction bound (||a_k^+ a_j|| <= L - 1, two terms per pair)
    pd.nex = 0;
    pd.rho_ex = 0.0;
    if (H->jx)
        for (int j = 0; j < q; ++j)
            for (int k = j + 1; k < q; ++k)
                if (H->jx[j * q + k] != 0.0) {
                    pd.ex_j[pd.nex] = j;
                    pd.ex_k[pd.nex] = k;
                    pd.ex_c[pd.nex] = 0.5 * pd.h * H->jx[j * q + k];
                    pd.rho_ex += pd.h * (L - 1) * std::fabs(H->jx[j * q + k]);
                    ++pd.nex;
                }
    for (int l = 0; l < MAXL; ++l) {
        pd.sc[2 * l + 0] = 0.5 * pd.h * std::sqrt(double(l + 1));
        pd.sc[2 * l + 1] = 0.5 * pd.h * std::sqrt(double(l));
        pd.wsq[2 * l + 0] = std::sqrt(double(l + 1));
        pd.wsq[2 * l + 1] = std::sqrt(double(l));
    }
    // the tiles' shared alpha-gradient: the splines active in one window (the most over the
    // windows, from each window's first active spline), plus a margin of two
    int span = 3;
    for (int m = pd.m_off + 1; m <= pd.m_off + pd.M; ++m) {
        const int64_t n0 = (int64_t(m - 1) * nsteps) / pd.M_glob, n1 = (int64_t(m) * nsteps) / pd.M_glob;
        if (n1 <= n0) continue;
        const int s_first = spline_index((double(n0) + 0.5) * pd.h, pd.dtau, pd.d1);
        const int s_last = spline_index((double(n1 - 1) + 0.5) * pd.h, pd.dtau, pd.d1);
        span = std::max(span, s_last - s_first + 3);
    }
    pd.gspan = std::min(pd.d1, span + 2);
    pd.glocal = 2 * nfsum * pd.gspan;
    if (layout < MSQOC_LAYOUT_AUTO || layout > MSQOC_LAYOUT_FIBER_LEAN)
        return fail(MSQOC_ERR_INVALID_ARG, "layout %d is not an MSQOC_LAYOUT_* value", layout);
    if (layout == MSQOC_LAYOUT_QUAD && !quad_admitted(pd))
        return fail(MSQOC_ERR_INVALID_ARG, "lane quads need 2-level subsystems and at most %d exchange-coupled pairs",
                    MAXEXF);
    if (col_block < 0) return fail(MSQOC_ERR_INVALID_ARG, "column block %d < 0", col_block);
    const TileChoice tc =
        choose_tile_layout(pd.M, pd.E, pd.F, q, L, pd.N, pd.glocal, solver, sms, col_block, layout, quad_admitted(pd));
    if (tc.cpt < 0)
        return fail(MSQOC_ERR_INVALID_ARG,
                    "column block %d invalid for E=%d (needs 1 <= cb <= E, cb N/L <= %d threads with one thread "
                    "per fiber (%d with the lean build), 2 cb N/L <= %d with lane pairs or 4 cb N/L <= %d with lane "
                    "quads, cb | E for one-warp tiles, and the shared memory)",
                    col_block, pd.E, MAX_TILE_THREADS, MAX_LEAN_TILE_THREADS, MAX_PAIR_TILE_THREADS,
                    MAX_QUAD_TILE_THREADS);
    const int cpt = tc.cpt;
    pd.cb = cpt;
    pd.pair = tc.pair;
    pd.lean = tc.lean;
    pd.nthreads = tile_threads(cpt, pd.F, tc.pair);
    pd.ntiles = static_cast<int>((long(pd.M) * pd.E + cpt - 1) / cpt);
    // whole windows in one history segment unless a checkpoint interval is set later
    const int64_t max_ns = (nsteps + nwindows - 1) / nwindows;
    pd.kseg = static_cast<int>(max_ns);
    pd.nseg = 1;
    pd.hdepth = 1;
    return MSQOC_OK;
}

// the sweeps' shared memory fits with history groups of `depth` steps
bool history_depth_ok(const ProbDev& pd, int depth) {
    if (depth < 1 || depth > MAX_HDEPTH) return false;
    for (int bwd = 0; bwd < 2; ++bwd)
        if (sweep_layout(pd.q, pd.L, pd.N, pd.cb, pd.nthreads, pd.glocal, pd.solver, bwd != 0, pd.pair, depth).total >
            200 * 1024)
            return false;
    return true;
}

// history segmentation for a checkpoint interval K (1 = keep every midpoint state)
void set_segments(ProbDev& pd, int K) {
    const int64_t max_ns = (pd.nsteps + pd.M_glob - 1) / pd.M_glob;
    pd.kseg = (K <= 1 || K >= max_ns) ? static_cast<int>(max_ns) : K;
    pd.nseg = static_cast<int>((max_ns + pd.kseg - 1) / pd.kseg);
}

// sweep launch arguments of a single problem
SweepArgs sweep_args(const ProbDev& pd, const ProbDev* pds_dev, const Tile* tiles, const int* lanemap, int mode,
                     int seg) {
    SweepArgs a{};
    a.pds = pds_dev;
    a.tiles = tiles;
    a.lanemap = lanemap;
    a.cpt = pd.cb;
    a.gmax = pd.glocal;
    a.mode = mode;
    a.seg = seg;
    a.L = pd.L;
    a.q = pd.q;
    a.solver = pd.solver;
    a.nthreads = pd.nthreads;
    a.pair = pd.pair;
    a.lean = pd.lean;
    a.hdepth = pd.hdepth;
    return a;
}

OutLayout out_layout(int npen, int d, size_t nW) {
    OutLayout o;
    o.pen = 2;
    o.ga = (o.pen + size_t(npen) + 1) & ~size_t(1);
    o.gw = (o.ga + size_t(d) + 1) & ~size_t(1);
    o.total = o.gw + nW + 2;
    return o;
}

int w_blocks(const ProbDev& pd) {
    const int kfirst = std::max(pd.m_off, 1), klast = std::min(pd.m_off + pd.M, pd.M_glob - 1);
    return std::max(0, klast - kfirst + 1);
}

int pen_count(const ProbDev& pd) { return pd.M - (pd.m_off + pd.M == pd.M_glob ? 1 : 0); }

bool is_shard(const ProbDev& pd) { return pd.M != pd.M_glob; }

}  // namespace msqoc

namespace {

void free_problem(msqoc_problem* p) {
    void* bufs[] = {p->tiles_ro, p->lanemap_ro,
                    p->pds,   p->tiles, p->lanemap, p->P,     p->emb,   p->V,     p->alpha_dev, p->W_dev,
                    p->ctrl,  p->spl,   p->phase,   p->hist,  p->ckpt,  p->Lstate, p->Uend,     p->Lterm,
                    p->Lam0,  p->term,  p->gpart,   p->status, p->out_dev, p->reg_dev};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (p->status_host) cudaFreeHost(p->status_host);
    for (auto& e : p->ev)
        for (auto& x : e)
            if (x) cudaEventDestroy(x);
}

// brackets a stretch of launches with profiling events when enabled
struct Mark {
    msqoc_problem* p;
    int k;
    cudaStream_t s;
    Mark(msqoc_problem* p_, int k_, cudaStream_t s_) : p(p_), k(k_), s(s_) {
        if (p->profile) {
            cudaEventRecord(p->ev[k][0], s);
            p->ran[k] = true;
        }
    }
    ~Mark() {
        if (p->profile) cudaEventRecord(p->ev[k][1], s);
    }
};

// doubles of the regularization scratch: alpha[d], gradient[d], energy shares[q d1], R
size_t reg_doubles(const ProbDev& pd) { return 2 * size_t(pd.d) + size_t(pd.q) * pd.d1 + 2; }

// device bytes of the history, checkpoints and segment state of one problem
// 16-byte blocks after the history that hold its column scale exponents ([M][nseg][E] ints)
size_t hist_scale_blocks(const ProbDev& pd) { return (size_t(pd.M) * pd.nseg * pd.E * sizeof(int) + 15) / 16; }

size_t gradient_bytes(const ProbDev& pd) {
    const size_t ne = size_t(pd.N) * pd.E;
    size_t b = (size_t(pd.M) * pd.kseg * ne + hist_scale_blocks(pd)) * sizeof(double2);
    if (pd.nseg > 1) b += (size_t(pd.M) * pd.nseg * ne + size_t(pd.M) * ne) * sizeof(double2);
    return b;
}

}  // namespace

extern "C" {

int32_t msqoc_version(void) { return 200; }

int32_t msqoc_last_error(char* buf, size_t len) {
    if (buf && len) {
        size_t n = std::min(len - 1, g_last_error.size());
        memcpy(buf, g_last_error.data(), n);
        buf[n] = 0;
    }
    return static_cast<int32_t>(g_last_error.size());
}

}  // extern "C"

namespace {

// frees a problem under construction unless released
struct ProblemOwner {
    msqoc_problem* p = nullptr;
    ~ProblemOwner() {
        if (p) {
            free_problem(p);
            delete p;
        }
    }
    msqoc_problem* release() {
        msqoc_problem* q = p;
        p = nullptr;
        return q;
    }
};

msqoc_status create_problem(const msqoc_hamiltonian* H, const msqoc_controls* C, const double* target, double T,
                            int64_t nsteps, int32_t nwindows, double mu, const msqoc_options* opt,
                            msqoc_problem** out) {
    if (!out) return fail(MSQOC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    msqoc_status st0 = check_description(H, C, T, nsteps, nwindows);
    if (st0 != MSQOC_OK) return st0;

    msqoc_options o{};
    if (opt) o = *opt;
    const int solver = o.solver == MSQOC_SOLVER_FP64 ? SOLVER_FP64 : SOLVER_MIXED;
    if (o.ckpt_interval < 0) return fail(MSQOC_ERR_INVALID_ARG, "checkpoint interval %d < 0", o.ckpt_interval);
    if (o.profile != 0 && o.profile != 1) return fail(MSQOC_ERR_INVALID_ARG, "profile must be 0 or 1");
    if (o.steps_per_sync < 0 || o.steps_per_sync > MAX_HDEPTH)
        return fail(MSQOC_ERR_INVALID_ARG, "steps_per_sync %d is not within 0..%d", o.steps_per_sync, MAX_HDEPTH);
    if ((o.window_first == 0) != (o.window_last == 0) ||
        (o.window_first != 0 && (o.window_first < 1 || o.window_first > o.window_last || o.window_last > nwindows)))
        return fail(MSQOC_ERR_INVALID_ARG, "window range %d..%d is not within 1..%d (0 and 0 = every window)",
                    o.window_first, o.window_last, nwindows);

    ProblemOwner owner{new (std::nothrow) msqoc_problem()};
    msqoc_problem* p = owner.p;
    if (!p) return fail(MSQOC_ERR_OUT_OF_MEMORY, "host allocation failed");
    ProbDev& pd = p->pd;
    cudaGetDevice(&p->device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (sms <= 0) sms = 1;
    st0 = shape_problem(H, C, T, nsteps, nwindows, mu, solver, o.col_block, o.layout, sms, pd, o.window_first,
                        o.window_last);
    if (st0 != MSQOC_OK) return st0;
    const int q = pd.q, L = pd.L, nfsum = pd.nfsum;
    // checkpoint interval: 0 = automatic (every midpoint state unless that history would take
    // more than a quarter of the device memory, else every 64 steps)
    int K = o.ckpt_interval;
    if (K == 0) {
        size_t freeb = 0, totalb = 0;
        cudaMemGetInfo(&freeb, &totalb);
        set_segments(pd, 1);
        K = (totalb && gradient_bytes(pd) > totalb / 4) ? 64 : 1;
    }
    p->ckpt_interval = K;
    set_segments(pd, K);
    // steps per history synchronisation: 0 = one (every step)
    pd.hdepth = o.steps_per_sync > 0 ? o.steps_per_sync : 1;
    if (!history_depth_ok(pd, pd.hdepth))
        return fail(MSQOC_ERR_INVALID_ARG, "history groups of %d steps do not fit the tile's shared memory",
                    pd.hdepth);

    // ---- host-side model tables and tile layout
    const int N = pd.N, E = pd.E;
    p->ne = size_t(N) * E;
    p->nWs = w_blocks(pd);
    p->npen = pen_count(pd);
    p->nW = 2 * p->ne * size_t(p->nWs);
    std::vector<double2> P(N);
    for (int i = 0; i < N; ++i) P[i] = precond_entry(pd.h, drift_entry(H, q, L, i));
    std::vector<int> emb(E);
    for (int e = 0; e < E; ++e) emb[e] = essential_row(q, L, pd.ness, e);
    std::vector<double2> Vh(p->ne, make_double2(0.0, 0.0));
    if (target) {
        for (size_t e = 0; e < p->ne; ++e) Vh[e] = make_double2(target[2 * e], target[2 * e + 1]);
    } else {
        for (int j = 0; j < E; ++j)
            for (int e = 0; e < E; ++e) Vh[size_t(j) * N + emb[e]] = qft_entry(E, e, j);
    }
    std::vector<Tile> tiles(pd.ntiles);
    for (int t = 0; t < pd.ntiles; ++t) tiles[t] = tile_at(t, pd.M, E, pd.cb, 0);
    std::vector<int> maps(size_t(pd.cb + 1) * pd.nthreads);
    build_lanemaps(L, q, pd.M, E, pd.cb, pd.nthreads, pd.pair, maps.data());
    // the roll-out sweep's tiles: the same widths over a single window
    p->ntiles_ro = static_cast<int>(tile_count(1, E, pd.cb));
    std::vector<Tile> tiles_ro(p->ntiles_ro);
    for (int t = 0; t < p->ntiles_ro; ++t) tiles_ro[t] = tile_at(t, 1, E, pd.cb, 0);
    std::vector<int> maps_ro(size_t(pd.cb + 1) * pd.nthreads);
    build_lanemaps(L, q, 1, E, pd.cb, pd.nthreads, pd.pair, maps_ro.data());

    // ---- device buffers
    const size_t M = pd.M;
    msqoc_status st = MSQOC_OK;
    auto A = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && st == MSQOC_OK)
            st = fail(e == cudaErrorMemoryAllocation ? MSQOC_ERR_OUT_OF_MEMORY : MSQOC_ERR_CUDA,
                      "allocating %s: %s", what, cudaGetErrorString(e));
    };
    A(dalloc(&p->pds, 1), "problem record");
    A(dalloc(&p->tiles, tiles.size()), "tiles");
    A(dalloc(&p->lanemap, maps.size()), "lane maps");
    A(dalloc(&p->tiles_ro, tiles_ro.size()), "roll-out tiles");
    A(dalloc(&p->lanemap_ro, maps_ro.size()), "roll-out lane maps");
    A(dalloc(&p->P, N), "P");
    A(dalloc(&p->emb, E), "embedding");
    A(dalloc(&p->V, p->ne), "target");
    A(dalloc(&p->alpha_dev, pd.d), "alpha");
    A(dalloc(&p->W_dev, std::max<size_t>(p->nW, 2)), "W");
    A(dalloc(&p->ctrl, size_t(nsteps) * q), "controls");
    A(dalloc(&p->spl, size_t(nsteps)), "splines");
    A(dalloc(&p->phase, size_t(nsteps) * nfsum), "phases");
    A(dalloc(&p->Uend, M * p->ne), "Uend");
    A(dalloc(&p->Lterm, M * p->ne), "Lterm");
    A(dalloc(&p->Lam0, M * p->ne), "Lam0");
    A(dalloc(&p->term, M), "terms");
    A(dalloc(&p->gpart, size_t(pd.ntiles) * pd.d), "gradient partials");
    A(dalloc(&p->status, 1), "status");
    A(dalloc(&p->out_dev, out_layout(p->npen, pd.d, p->nW).total), "outputs");
    A(dalloc(&p->reg_dev, reg_doubles(pd)), "regularization scratch");
    A(cudaMallocHost(reinterpret_cast<void**>(&p->status_host), sizeof(int)), "pinned status");
    p->profile = o.profile == 1;
    if (p->profile)
        for (auto& e : p->ev)
            for (auto& x : e) A(cudaEventCreate(&x), "profiling event");
    if (st == MSQOC_OK) {
        pd.P = p->P;
        pd.emb = p->emb;
        pd.V = p->V;
        pd.alpha = p->alpha_dev;
        // a shard past the first window reads its first window's initial state at index -1
        pd.W = reinterpret_cast<const double2*>(p->W_dev) + (pd.m_off >= 1 ? p->ne : 0);
        pd.ctrl = p->ctrl;
        pd.spl = p->spl;
        pd.phase = p->phase;
        pd.Uend = p->Uend;
        pd.Lterm = p->Lterm;
        pd.Lam0 = p->Lam0;
        pd.term = p->term;
        pd.gpart = p->gpart;
        pd.status = p->status;
        A(cudaMemcpy(p->tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice), "tiles copy");
        A(cudaMemcpy(p->lanemap, maps.data(), maps.size() * sizeof(int), cudaMemcpyHostToDevice), "lane map copy");
        A(cudaMemcpy(p->tiles_ro, tiles_ro.data(), tiles_ro.size() * sizeof(Tile), cudaMemcpyHostToDevice),
          "roll-out tiles copy");
        A(cudaMemcpy(p->lanemap_ro, maps_ro.data(), maps_ro.size() * sizeof(int), cudaMemcpyHostToDevice),
          "roll-out lane map copy");
        A(cudaMemcpy(p->P, P.data(), N * sizeof(double2), cudaMemcpyHostToDevice), "P copy");
        A(cudaMemcpy(p->emb, emb.data(), E * sizeof(int), cudaMemcpyHostToDevice), "emb copy");
        A(cudaMemcpy(p->V, Vh.data(), p->ne * sizeof(double2), cudaMemcpyHostToDevice), "target copy");
        A(cudaMemset(p->W_dev, 0, std::max<size_t>(p->nW, 2) * sizeof(double)), "W init");
        A(cudaMemset(p->status, 0, sizeof(int)), "status init");
        A(cudaMemcpy(p->pds, &pd, sizeof(ProbDev), cudaMemcpyHostToDevice), "problem record copy");
        // the carrier phase table: a constant of the time grid, filled once
        if (st == MSQOC_OK) {
            k_phases<<<phase_blocks(pd), 256>>>(pd);
            A(cudaGetLastError(), "phase table");
            A(cudaDeviceSynchronize(), "phase table");
        }
    }
    if (st != MSQOC_OK) return st;
    p->bytes = sizeof(double2) * (N + p->ne * (1 + 3 * M) + size_t(nsteps) * (q + nfsum)) +
               sizeof(Spline4) * size_t(nsteps) + sizeof(double) * (pd.d + p->nW + M + size_t(pd.ntiles) * pd.d + out_layout(p->npen, pd.d, p->nW).total +
                                reg_doubles(pd)) +
               sizeof(int) * (E + 1 + maps.size() + maps_ro.size()) + sizeof(Tile) * (tiles.size() + tiles_ro.size()) +
               sizeof(ProbDev);
    p->grad_bytes = gradient_bytes(pd);
    *out = owner.release();
    return MSQOC_OK;
}

}  // namespace

extern "C" {

msqoc_status msqoc_create_problem(const msqoc_hamiltonian* H, const msqoc_controls* C, const double* target,
                                  double T, int64_t nsteps, int32_t nwindows, double mu,
                                  const msqoc_options* opt, msqoc_problem** out) {
    if (out) *out = nullptr;
    return guarded([&] { return create_problem(H, C, target, T, nsteps, nwindows, mu, opt, out); });
}

msqoc_status msqoc_query(const msqoc_problem* p, int64_t* d, int64_t* nW, size_t* device_bytes) {
    if (!p) return fail(MSQOC_ERR_INVALID_ARG, "problem is NULL");
    if (d) *d = p->pd.d;
    if (nW) *nW = static_cast<int64_t>(p->nW);
    if (device_bytes) *device_bytes = p->bytes + (p->hist ? 0 : p->grad_bytes);
    return MSQOC_OK;
}

msqoc_status msqoc_query_layout(const msqoc_problem* p, int32_t* col_block, int32_t* tiles, int32_t* threads,
                                int32_t* ckpt_interval, int32_t* layout, int32_t* steps_per_sync) {
    if (!p) return fail(MSQOC_ERR_INVALID_ARG, "problem is NULL");
    if (steps_per_sync) *steps_per_sync = p->pd.hdepth;
    if (col_block) *col_block = p->pd.cb;
    if (tiles) *tiles = p->pd.ntiles;
    if (threads) *threads = p->pd.nthreads;
    if (ckpt_interval) *ckpt_interval = p->ckpt_interval;
    if (layout) *layout = p->pd.lean ? MSQOC_LAYOUT_FIBER_LEAN : MSQOC_LAYOUT_FIBER + p->pd.pair;
    return MSQOC_OK;
}

msqoc_status msqoc_destroy_problem(msqoc_problem* p) {
    if (!p) return MSQOC_OK;
    cudaDeviceSynchronize();
    free_problem(p);
    delete p;
    return MSQOC_OK;
}

}  // extern "C"

namespace msqoc {

// copy the evaluation's inputs into the problem's input buffers (stream-ordered)
msqoc_status stage_inputs(msqoc_problem* p, const double* alpha, const double* W, cudaStream_t s) {
    if (!alpha) return fail(MSQOC_ERR_INVALID_ARG, "alpha is NULL");
    if (p->nW > 0 && !W) return fail(MSQOC_ERR_INVALID_ARG, "W is NULL but the problem reads window states");
    CUDA_TRY(cudaMemcpyAsync(p->alpha_dev, alpha, p->pd.d * sizeof(double), cudaMemcpyDefault, s));
    if (p->nW > 0) CUDA_TRY(cudaMemcpyAsync(p->W_dev, W, p->nW * sizeof(double), cudaMemcpyDefault, s));
    return MSQOC_OK;
}

// the history, checkpoints and segment state, on the first gradient evaluation
msqoc_status ensure_gradient_buffers(msqoc_problem* p, cudaStream_t s) {
    if (p->hist) return MSQOC_OK;
    ProbDev& pd = p->pd;
    const size_t M = pd.M;
    cudaError_t e = dalloc(&p->hist, M * pd.kseg * p->ne + hist_scale_blocks(pd));
    if (e == cudaSuccess && pd.nseg > 1) e = dalloc(&p->ckpt, M * pd.nseg * p->ne);
    if (e == cudaSuccess && pd.nseg > 1) e = dalloc(&p->Lstate, M * p->ne);
    if (e != cudaSuccess) {
        for (void* b : {static_cast<void*>(p->hist), static_cast<void*>(p->ckpt), static_cast<void*>(p->Lstate)})
            if (b) cudaFree(b);
        p->hist = p->ckpt = p->Lstate = nullptr;
        cudaGetLastError();
        return fail(MSQOC_ERR_OUT_OF_MEMORY, "history buffers (%zu bytes, checkpoint interval %d): %s", p->grad_bytes,
                    p->ckpt_interval, cudaGetErrorString(e));
    }
    pd.hist = p->hist;
    pd.hsh = reinterpret_cast<int*>(p->hist + M * pd.kseg * p->ne);
    pd.ckpt = p->ckpt;
    pd.Lstate = p->Lstate;
    p->bytes += p->grad_bytes;
    // a pageable host-to-device copy has consumed its source when the call returns
    CUDA_TRY(cudaMemcpyAsync(p->pds, &pd, sizeof(ProbDev), cudaMemcpyHostToDevice, s));
    return MSQOC_OK;
}

msqoc_status sweep(msqoc_problem* p, int mode, int seg, cudaStream_t s) {
    const SweepArgs a = sweep_args(p->pd, p->pds, p->tiles, p->lanemap, mode, seg);
    CUDA_TRY(launch_sweep(a, p->pd.ntiles, s));
    return MSQOC_OK;
}

// blocks of 256 threads for the phase table (grid-stride loop)
int phase_blocks(const ProbDev& pd) {
    return static_cast<int>(std::min<int64_t>((pd.nsteps * pd.nfsum + 255) / 256, 4096));
}

msqoc_status launch_controls(msqoc_problem* p, cudaStream_t s) {
    const ProbDev& pd = p->pd;
    Mark mk(p, MSQOC_KERNEL_CONTROLS, s);
    const int threads = 256;
    const int blocks = static_cast<int>(std::min<int64_t>((pd.nsteps + threads - 1) / threads, 4096));
    k_controls<<<blocks, threads, 0, s>>>(pd);
    CUDA_TRY(cudaGetLastError());
    return MSQOC_OK;
}

msqoc_status launch_terminal(msqoc_problem* p, bool want_lambda, cudaStream_t s) {
    Mark mk(p, MSQOC_KERNEL_TERMINAL, s);
    k_terminal<<<p->pd.M, TERM_THREADS, 0, s>>>(p->pd, want_lambda ? 1 : 0);
    CUDA_TRY(cudaGetLastError());
    return MSQOC_OK;
}

msqoc_status launch_objective_outputs(msqoc_problem* p, double* P, double* J, double* pen, cudaStream_t s) {
    Mark mk(p, MSQOC_KERNEL_FINALIZE, s);
    k_finalize_scalars<<<1, 32, 0, s>>>(p->pd, P, J, p->npen > 0 ? pen : nullptr, nullptr);
    CUDA_TRY(cudaGetLastError());
    return MSQOC_OK;
}

msqoc_status launch_gradient_outputs(msqoc_problem* p, double* P, double* ga, double* gw, cudaStream_t s) {
    const ProbDev& pd = p->pd;
    Mark mk(p, MSQOC_KERNEL_FINALIZE, s);
    k_finalize_scalars<<<std::max(1, (pd.d + 255) / 256), 256, 0, s>>>(pd, P, nullptr, nullptr, ga);
    CUDA_TRY(cudaGetLastError());
    if (p->nWs > 0) {
        const size_t total = p->ne * size_t(p->nWs);
        const int blocks = static_cast<int>(std::min<size_t>((total + 255) / 256, 8192));
        k_grad_W<<<blocks, 256, 0, s>>>(pd, reinterpret_cast<double2*>(gw), p->nWs);
        CUDA_TRY(cudaGetLastError());
    }
    return MSQOC_OK;
}

// controls, forward sweep over whole windows, terminal conditions
msqoc_status launch_forward_part(msqoc_problem* p, int mode, cudaStream_t s) {
    for (bool& r : p->ran) r = false;
    msqoc_status st = launch_controls(p, s);
    if (st) return st;
    {
        Mark mk(p, MSQOC_KERNEL_FORWARD, s);
        st = sweep(p, mode, 0, s);
        if (st) return st;
    }
    return launch_terminal(p, mode != SWEEP_OBJECTIVE, s);
}

msqoc_status status_error(int st) {
    if (st & ST_TIMEOUT) return fail(MSQOC_ERR_TIMEOUT, "a bounded device wait gave up (status %d)", st);
    if (st & ST_SOLVER_RANGE)
        return fail(MSQOC_ERR_UNSUPPORTED, "time step too large for the step solver (h*|H_c|/2 >= 0.5)");
    if (st & ST_GRAD_RANGE)
        return fail(MSQOC_ERR_INTERNAL, "a gradient spline index fell outside its tile's window range (status %d)", st);
    return fail(MSQOC_ERR_INTERNAL, "device status %d", st);
}

msqoc_status check_status_sync(msqoc_problem* p, cudaStream_t s) {
    CUDA_TRY(cudaMemcpyAsync(p->status_host, p->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const int st = *p->status_host;
    if (st) {
        cudaMemsetAsync(p->status, 0, sizeof(int), s);
        return status_error(st);
    }
    return MSQOC_OK;
}

}  // namespace msqoc

extern "C" {

msqoc_status msqoc_eval_objective(msqoc_problem* p, const double* alpha, const double* W, double* P_out,
                                  double* J_out, double* pen_out, void* stream) {
    if (!p) return fail(MSQOC_ERR_INVALID_ARG, "problem is NULL");
    if (!P_out) return fail(MSQOC_ERR_INVALID_ARG, "P_out is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    msqoc_status st = stage_inputs(p, alpha, W, s);
    if (st) return st;
    st = launch_forward_part(p, SWEEP_OBJECTIVE, s);
    if (st) return st;
    const ProbDev& pd = p->pd;
    const bool dP = is_device_ptr(P_out), dJ = !J_out || is_device_ptr(J_out), dpen = !pen_out || is_device_ptr(pen_out);
    double* o = p->out_dev;
    st = launch_objective_outputs(p, dP ? P_out : o, J_out ? (dJ ? J_out : o + 1) : nullptr,
                                  pen_out ? (dpen ? pen_out : o + 2) : nullptr, s);
    if (st) return st;
    const bool all_dev = dP && dJ && dpen;
    if (all_dev) return MSQOC_OK;
    if (!dP) CUDA_TRY(cudaMemcpyAsync(P_out, o, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (J_out && !dJ) CUDA_TRY(cudaMemcpyAsync(J_out, o + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (pen_out && !dpen && p->npen > 0)
        CUDA_TRY(cudaMemcpyAsync(pen_out, o + 2, p->npen * sizeof(double), cudaMemcpyDeviceToHost, s));
    return check_status_sync(p, s);
}

msqoc_status msqoc_eval_gradient(msqoc_problem* p, const double* alpha, const double* W, double* P_out,
                                 double* grad_alpha, double* grad_W, void* stream) {
    if (!p) return fail(MSQOC_ERR_INVALID_ARG, "problem is NULL");
    if (!grad_alpha) return fail(MSQOC_ERR_INVALID_ARG, "grad_alpha is NULL");
    if (p->nW > 0 && !grad_W) return fail(MSQOC_ERR_INVALID_ARG, "grad_W is NULL but the problem reads window states");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    msqoc_status st = ensure_gradient_buffers(p, s);
    if (st) return st;
    st = stage_inputs(p, alpha, W, s);
    if (st) return st;
    const ProbDev& pd = p->pd;
    // one history segment: every midpoint state in the forward sweep; otherwise checkpoints
    // at the segment starts, and each segment is recomputed before its adjoint sweep
    st = launch_forward_part(p, SWEEP_HISTORY, s);
    if (st) return st;
    {
        Mark mk(p, MSQOC_KERNEL_ADJOINT, s);
        for (int seg = pd.nseg - 1; seg >= 0; --seg) {
            if (pd.nseg > 1) {
                st = sweep(p, SWEEP_RECOMPUTE, seg, s);
                if (st) return st;
            }
            st = sweep(p, SWEEP_ADJOINT, seg, s);
            if (st) return st;
        }
    }
    const bool dP = !P_out || is_device_ptr(P_out), dga = is_device_ptr(grad_alpha),
               dgw = p->nW == 0 || is_device_ptr(grad_W);
    double* o = p->out_dev;
    const OutLayout ol = out_layout(p->npen, pd.d, p->nW);
    if (p->nW > 0 && dgw && reinterpret_cast<uintptr_t>(grad_W) % 16)
        return fail(MSQOC_ERR_INVALID_ARG, "device grad_W must be 16-byte aligned");
    double* ga_dst = dga ? grad_alpha : o + ol.ga;
    double* gw_dst = p->nW == 0 ? nullptr : (dgw ? grad_W : o + ol.gw);
    st = launch_gradient_outputs(p, P_out ? (dP ? P_out : o) : nullptr, ga_dst, gw_dst, s);
    if (st) return st;
    if (dP && dga && dgw) return MSQOC_OK;
    if (P_out && !dP) CUDA_TRY(cudaMemcpyAsync(P_out, o, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (!dga) CUDA_TRY(cudaMemcpyAsync(grad_alpha, ga_dst, pd.d * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (!dgw) CUDA_TRY(cudaMemcpyAsync(grad_W, gw_dst, p->nW * sizeof(double), cudaMemcpyDeviceToHost, s));
    return check_status_sync(p, s);
}

msqoc_status msqoc_rollout(msqoc_problem* p, const double* alpha, double* W_out, void* stream) {
    if (!p) return fail(MSQOC_ERR_INVALID_ARG, "problem is NULL");
    if (is_shard(p->pd)) return fail(MSQOC_ERR_UNSUPPORTED, "the roll-out takes a whole problem, not a window range");
    if (p->pd.M > 1 && !W_out) return fail(MSQOC_ERR_INVALID_ARG, "W_out is NULL but M > 1");
    if (!alpha) return fail(MSQOC_ERR_INVALID_ARG, "alpha is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->pd.M == 1) return MSQOC_OK;
    CUDA_TRY(cudaMemcpyAsync(p->alpha_dev, alpha, p->pd.d * sizeof(double), cudaMemcpyDefault, s));
    msqoc_status st;
    const bool dev = is_device_ptr(W_out) && reinterpret_cast<uintptr_t>(W_out) % 16 == 0;
    double* dst = dev ? W_out : p->out_dev + out_layout(p->npen, p->pd.d, p->nW).gw;
    for (bool& r : p->ran) r = false;
    if ((st = launch_controls(p, s))) return st;
    SweepArgs a = sweep_args(p->pd, p->pds, p->tiles_ro, p->lanemap_ro, SWEEP_ROLLOUT, 0);
    a.out = reinterpret_cast<double2*>(dst);
    {
        Mark mk(p, MSQOC_KERNEL_FORWARD, s);
        CUDA_TRY(launch_sweep(a, p->ntiles_ro, s));
    }
    if (dev) return MSQOC_OK;
    CUDA_TRY(cudaMemcpyAsync(W_out, dst, p->nW * sizeof(double), cudaMemcpyDefault, s));
    return check_status_sync(p, s);
}

msqoc_status msqoc_rollout_estimate(msqoc_problem* p, double* est_out, void* stream) {
    if (!p || !est_out) return fail(MSQOC_ERR_INVALID_ARG, "problem or est_out is NULL");
    if (is_shard(p->pd))
        return fail(MSQOC_ERR_UNSUPPORTED, "the roll-out estimate takes a whole problem, not a window range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool dev = is_device_ptr(est_out);
    // a spare slot at the end of the output staging (the other slots hold the last results)
    double* dst = dev ? est_out : p->out_dev + out_layout(p->npen, p->pd.d, p->nW).total - 1;
    k_rollout_estimate<<<1, 32, 0, s>>>(p->pd, dst);
    CUDA_TRY(cudaGetLastError());
    if (dev) return MSQOC_OK;
    CUDA_TRY(cudaMemcpyAsync(est_out, dst, sizeof(double), cudaMemcpyDeviceToHost, s));
    return check_status_sync(p, s);
}

msqoc_status msqoc_eval_regularization(msqoc_problem* p, const double* alpha, double gamma_tik,
                                       double gamma_energy, double* R_out, double* grad_alpha, void* stream) {
    if (!p) return fail(MSQOC_ERR_INVALID_ARG, "problem is NULL");
    if (!alpha || !R_out) return fail(MSQOC_ERR_INVALID_ARG, "alpha or R_out is NULL");
    if (!(gamma_tik >= 0.0) || !(gamma_energy >= 0.0) || std::isinf(gamma_tik) || std::isinf(gamma_energy))
        return fail(MSQOC_ERR_INVALID_ARG, "gamma_tik %g and gamma_energy %g must be finite and >= 0", gamma_tik,
                    gamma_energy);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ProbDev& pd = p->pd;
    double* a = p->reg_dev;
    double* g = a + pd.d;
    double* ep = g + pd.d;
    double* R = ep + size_t(pd.q) * pd.d1;
    const bool dR = is_device_ptr(R_out);
    const bool dg = grad_alpha && is_device_ptr(grad_alpha);
    CUDA_TRY(cudaMemcpyAsync(a, alpha, pd.d * sizeof(double), cudaMemcpyDefault, s));
    k_regularization<<<pd.q * pd.d1, REG_THREADS, 0, s>>>(pd, a, gamma_tik, gamma_energy, dg ? grad_alpha : g, ep);
    CUDA_TRY(cudaGetLastError());
    k_regularization_total<<<1, REG_THREADS, 0, s>>>(pd, a, gamma_tik, gamma_energy, ep, dR ? R_out : R);
    CUDA_TRY(cudaGetLastError());
    if (dR && (dg || !grad_alpha)) return MSQOC_OK;
    if (!dR) CUDA_TRY(cudaMemcpyAsync(R_out, R, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (grad_alpha && !dg) CUDA_TRY(cudaMemcpyAsync(grad_alpha, g, pd.d * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return MSQOC_OK;
}

msqoc_status msqoc_kernel_times(msqoc_problem* p, float* ms) {
    if (!p || !ms) return fail(MSQOC_ERR_INVALID_ARG, "problem or ms is NULL");
    if (!p->profile) return fail(MSQOC_ERR_INVALID_ARG, "problem was created without options.profile = 1");
    for (int k = 0; k < MSQOC_NKERNELS; ++k) {
        ms[k] = 0.f;
        if (!p->ran[k]) continue;
        CUDA_TRY(cudaEventSynchronize(p->ev[k][1]));
        CUDA_TRY(cudaEventElapsedTime(&ms[k], p->ev[k][0], p->ev[k][1]));
    }
    return MSQOC_OK;
}

}  // extern "C"
// ------------------------------------------------------------------ autotuning the tile width
namespace {

msqoc_status autotune(const msqoc_hamiltonian* H, const msqoc_controls* C, double T, int64_t nsteps, int32_t nwindows,
                      double mu, const msqoc_options* opt, const double* alpha, int32_t probe_steps,
                      int32_t* col_block, int32_t* layout, int32_t* steps_per_sync, int32_t* widths, int32_t* layouts,
                      int32_t* depths, float* ms, int32_t max_out, int32_t* n_out) {
    if (!col_block) return fail(MSQOC_ERR_INVALID_ARG, "col_block is NULL");
    *col_block = 0;
    if (layout) *layout = 0;
    if (steps_per_sync) *steps_per_sync = 0;
    if (n_out) *n_out = 0;
    msqoc_status st = check_description(H, C, T, nsteps, nwindows);
    if (st != MSQOC_OK) return st;
    if (probe_steps < 1) return fail(MSQOC_ERR_INVALID_ARG, "probe_steps %d < 1", probe_steps);
    msqoc_options o{};
    if (opt) o = *opt;
    o.profile = 0;
    o.window_first = o.window_last = 0;   // the probes are whole problems
    const int solver = o.solver == MSQOC_SOLVER_FP64 ? SOLVER_FP64 : SOLVER_MIXED;
    // the probe: same shape, step size and window count, probe_steps steps per window
    const int64_t psteps = std::min<int64_t>(nsteps, int64_t(nwindows) * probe_steps);
    const double pT = T * double(psteps) / double(nsteps);
    ProbDev pd{};
    st = shape_problem(H, C, pT, psteps, nwindows, mu, solver, 1, o.layout, 1, pd);
    if (st != MSQOC_OK && st != MSQOC_ERR_INVALID_ARG) return st;
    std::vector<double> a(static_cast<size_t>(pd.d));
    for (int j = 0; j < pd.d; ++j)   // default iterate: alternating amplitudes of the workloads' scale
        a[j] = alpha ? alpha[j] : ((j & 1) ? -1.0 : 1.0) * 2.0 * M_PI * 0.002;
    const size_t nW = 2 * size_t(pd.N) * pd.E * size_t(nwindows - 1);
    std::vector<double> W(std::max<size_t>(nW, 2), 0.0), ga(pd.d), gW(std::max<size_t>(nW, 2));
    double* dbuf = nullptr;
    CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&dbuf), (pd.d + nW + 2) * sizeof(double)));
    double* d_alpha = dbuf;
    double* d_W = dbuf + pd.d;
    double* d_out = nullptr;
    cudaError_t ce = cudaMalloc(reinterpret_cast<void**>(&d_out), (1 + pd.d + nW + 2) * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMemcpy(d_alpha, a.data(), pd.d * sizeof(double), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(d_W, 0, (nW + 2) * sizeof(double));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaFree(dbuf);
        if (d_out) cudaFree(d_out);
        if (e0) cudaEventDestroy(e0);
        return fail(MSQOC_ERR_CUDA, "autotune buffers: %s", cudaGetErrorString(ce));
    }
    double* o_P = d_out;
    double* o_ga = d_out + 2;   // keep grad_W 16-byte aligned: it starts at an even offset
    double* o_gW = o_ga + ((pd.d + 1) & ~1);
    float best_ms = 0.f;
    int best = 0, nrec = 0;
    int best_layout = 0, best_depth = 1;
    const int fam_lo = o.layout == MSQOC_LAYOUT_AUTO ? MSQOC_LAYOUT_FIBER : o.layout;
    const int fam_hi = o.layout == MSQOC_LAYOUT_AUTO ? MSQOC_LAYOUT_FIBER_LEAN : o.layout;
    // candidates: every (family, width) with one step per history synchronisation, then the
    // best pair with 2, 4 and 8 steps per synchronisation
    std::vector<std::array<int, 3>> cands;
    for (int fam = fam_lo; fam <= fam_hi; ++fam)
        for (int cb = std::min(pd.E, MAX_LEAN_TILE_THREADS / pd.F); cb >= 1; --cb)
            if (choose_tile_layout(pd.M, pd.E, pd.F, pd.q, pd.L, pd.N, pd.glocal, solver, 1, cb, fam,
                                   quad_admitted(pd)).cpt >= 0)
                cands.push_back({fam, cb, o.steps_per_sync > 0 ? o.steps_per_sync : 1});
    const size_t n_first = cands.size();
    for (size_t ci = 0; ci < cands.size() && st == MSQOC_OK; ++ci) {
        const int fam = cands[ci][0], cb = cands[ci][1], dp = cands[ci][2];
        msqoc_options oc = o;
        oc.col_block = cb;
        oc.layout = fam;
        oc.steps_per_sync = dp;
        msqoc_problem* p = nullptr;
        msqoc_status cs = msqoc_create_problem(H, C, nullptr, pT, psteps, nwindows, mu, &oc, &p);
        if (cs == MSQOC_ERR_INVALID_ARG && ci >= n_first) continue;   // that depth does not fit
        if (cs != MSQOC_OK) {
            st = cs;
            break;
        }
        float t = 0.f;
        for (int it = 0; it < 3 && cs == MSQOC_OK; ++it) {   // one warm-up, two timed
            if (it == 1) cudaEventRecord(e0, nullptr);
            cs = msqoc_eval_gradient(p, d_alpha, nwindows > 1 ? d_W : nullptr, o_P, o_ga, nwindows > 1 ? o_gW : nullptr,
                                     nullptr);
        }
        if (cs == MSQOC_OK) {
            cudaEventRecord(e1, nullptr);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&t, e0, e1);
            t *= 0.5f;
            cs = check_status_sync(p, nullptr);
        }
        msqoc_destroy_problem(p);
        if (cs != MSQOC_OK) {
            st = cs;
            break;
        }
        if (widths && ms && nrec < max_out) {
            widths[nrec] = cb;
            ms[nrec] = t;
            if (layouts) layouts[nrec] = fam;
            if (depths) depths[nrec] = dp;
        }
        ++nrec;
        if (best == 0 || t < best_ms) {
            best = cb;
            best_layout = fam;
            best_depth = dp;
            best_ms = t;
        }
        // the depth candidates are appended once the (family, width) sweep is done
        if (ci + 1 == n_first && best > 0 && o.steps_per_sync == 0)
            for (int dp2 : {2, 4, 8}) cands.push_back({best_layout, best, dp2});
    }
    cudaFree(dbuf);
    cudaFree(d_out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MSQOC_OK) return st;
    if (best == 0) return fail(MSQOC_ERR_UNSUPPORTED, "no admissible tile width");
    *col_block = best;
    if (layout) *layout = best_layout;
    if (steps_per_sync) *steps_per_sync = best_depth;
    if (n_out) *n_out = std::min(nrec, max_out);
    return MSQOC_OK;
}

}  // namespace

extern "C" msqoc_status msqoc_autotune(const msqoc_hamiltonian* H, const msqoc_controls* C, double T, int64_t nsteps,
                                       int32_t nwindows, double mu, const msqoc_options* opt, const double* alpha,
                                       int32_t probe_steps, int32_t* col_block, int32_t* layout,
                                       int32_t* steps_per_sync, int32_t* widths, int32_t* layouts, int32_t* depths,
                                       float* ms, int32_t max_out, int32_t* n_out) {
    return guarded([&] {
        return autotune(H, C, T, nsteps, nwindows, mu, opt, alpha, probe_steps, col_block, layout, steps_per_sync,
                        widths, layouts, depths, ms, max_out, n_out);
    });
}

// ------------------------------------------------------------------ objective without allocation
// Scratch of msqoc_eval_objective_noalloc: every table and intermediate of one objective
// evaluation, carved into 256-byte-aligned regions.  Static device storage: the module holds
// it on every GPU where it is loaded, and no call allocates.  In host code the name below is
// only a stand-in registered with the runtime; the device address comes from
// cudaGetSymbolAddress (noalloc_scratch below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[MSQOC_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of the scratch array on the current device.  It is looked up on every call,
// with the calling device current: a cached address would go stale when the context is torn
// down and recreated (cudaDeviceReset), since the module and its static storage are then
// loaded again, possibly elsewhere.  The lookup is a host-side table query.
msqoc_status noalloc_scratch(unsigned char** base) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
        return fail(MSQOC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch on device %d failed: %s", dev,
                    cudaGetErrorString(e));
    *base = static_cast<unsigned char*>(ptr);
    return MSQOC_OK;
}

// byte offsets of consecutive 256-byte-aligned regions
struct Carve {
    size_t off = 0;
    template <typename T>
    size_t take(size_t n) {
        const size_t at = off;
        off = (off + n * sizeof(T) + 255) & ~size_t(255);
        return at;
    }
};

}  // namespace

namespace {

msqoc_status eval_objective_noalloc(const msqoc_hamiltonian* H, const msqoc_controls* C, const double* target,
                                   double T, int64_t nsteps, int32_t nwindows, double mu, int32_t solver,
                                   const double* alpha, const double* W, double* P_out, double* J_out,
                                   double* pen_out, void* stream) {
    if (!alpha || !P_out) return fail(MSQOC_ERR_INVALID_ARG, "alpha or P_out is NULL");
    msqoc_status st = check_description(H, C, T, nsteps, nwindows);
    if (st != MSQOC_OK) return st;
    if (nwindows > 1 && !W) return fail(MSQOC_ERR_INVALID_ARG, "W is NULL but M > 1");
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ProbDev pd{};
    st = shape_problem(H, C, T, nsteps, nwindows, mu, solver == MSQOC_SOLVER_FP64 ? SOLVER_FP64 : SOLVER_MIXED, 0,
                       MSQOC_LAYOUT_AUTO, std::max(sms, 1), pd);
    if (st != MSQOC_OK) return st;

    // ---- scratch layout; the limit depends on the problem's size only
    const size_t N = pd.N, E = pd.E, ne = N * E, M = pd.M, nt = size_t(nsteps);
    const size_t nW = 2 * ne * (M - 1);
    const size_t nmap = size_t(pd.cb + 1) * pd.nthreads;
    Carve cv;
    const size_t o_status = cv.take<int>(1), o_term = cv.take<double>(M), o_out = cv.take<double>(M + 1),
                 o_pd = cv.take<ProbDev>(1), o_tiles = cv.take<Tile>(pd.ntiles), o_map = cv.take<int>(nmap),
                 o_P = cv.take<double2>(N), o_emb = cv.take<int>(E), o_V = cv.take<double2>(ne),
                 o_alpha = cv.take<double>(pd.d), o_W = cv.take<double>(nW), o_ctrl = cv.take<double2>(nt * pd.q),
                 o_spl = cv.take<Spline4>(nt), o_phase = cv.take<double2>(nt * pd.nfsum),
                 o_Uend = cv.take<double2>(M * ne);
    if (cv.off > MSQOC_NOALLOC_SCRATCH_BYTES)
        return fail(MSQOC_ERR_INVALID_ARG,
                    "problem needs %zu bytes of scratch; the allocation-free objective holds at most %zu "
                    "(MSQOC_NOALLOC_SCRATCH_BYTES)",
                    cv.off, size_t(MSQOC_NOALLOC_SCRATCH_BYTES));
    unsigned char* base = nullptr;
    st = noalloc_scratch(&base);
    if (st != MSQOC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    pd.status = reinterpret_cast<int*>(base + o_status);
    pd.term = reinterpret_cast<double*>(base + o_term);
    double2* Pd = reinterpret_cast<double2*>(base + o_P);
    int* emb_d = reinterpret_cast<int*>(base + o_emb);
    double2* V_d = reinterpret_cast<double2*>(base + o_V);
    ProbDev* pd_d = reinterpret_cast<ProbDev*>(base + o_pd);
    Tile* tiles_d = reinterpret_cast<Tile*>(base + o_tiles);
    int* map_d = reinterpret_cast<int*>(base + o_map);
    pd.P = Pd;
    pd.emb = emb_d;
    pd.V = V_d;
    pd.ctrl = reinterpret_cast<double2*>(base + o_ctrl);
    pd.spl = reinterpret_cast<Spline4*>(base + o_spl);
    pd.phase = reinterpret_cast<double2*>(base + o_phase);
    pd.Uend = reinterpret_cast<double2*>(base + o_Uend);
    double* outs = reinterpret_cast<double*>(base + o_out);   // P, J, pen[M-1]

    // ---- inputs: device arrays in place, host arrays copied into the scratch
    if (is_device_ptr(alpha)) {
        pd.alpha = alpha;
    } else {
        CUDA_TRY(cudaMemcpyAsync(base + o_alpha, alpha, pd.d * sizeof(double), cudaMemcpyHostToDevice, s));
        pd.alpha = reinterpret_cast<const double*>(base + o_alpha);
    }
    pd.W = reinterpret_cast<const double2*>(base + o_W);
    if (M > 1) {
        if (is_device_ptr(W)) {
            if (reinterpret_cast<uintptr_t>(W) % 16) return fail(MSQOC_ERR_INVALID_ARG, "device W must be 16-byte aligned");
            pd.W = reinterpret_cast<const double2*>(W);
        } else {
            CUDA_TRY(cudaMemcpyAsync(base + o_W, W, nW * sizeof(double), cudaMemcpyHostToDevice, s));
        }
    }

    // ---- model tables, tiles and lane maps, built in small host buffers and copied in (a
    // pageable host-to-device copy has consumed its source when cudaMemcpyAsync returns, so the
    // buffers are reused)
    CUDA_TRY(cudaMemsetAsync(pd.status, 0, sizeof(int), s));
    CUDA_TRY(cudaMemcpyAsync(pd_d, &pd, sizeof(ProbDev), cudaMemcpyHostToDevice, s));
    {
        double2 rows[kMaxRows];
        for (size_t i = 0; i < N; ++i) rows[i] = precond_entry(pd.h, drift_entry(H, pd.q, pd.L, int(i)));
        CUDA_TRY(cudaMemcpyAsync(Pd, rows, N * sizeof(double2), cudaMemcpyHostToDevice, s));
        int emb[kMaxRows];
        for (size_t e = 0; e < E; ++e) emb[e] = essential_row(pd.q, pd.L, pd.ness, int(e));
        CUDA_TRY(cudaMemcpyAsync(emb_d, emb, E * sizeof(int), cudaMemcpyHostToDevice, s));
        if (target) {
            CUDA_TRY(cudaMemcpyAsync(V_d, target, ne * sizeof(double2), cudaMemcpyDefault, s));
        } else {
            for (size_t j = 0; j < E; ++j) {   // QFT_E on the essential rows, one column at a time
                for (size_t i = 0; i < N; ++i) rows[i] = make_double2(0.0, 0.0);
                for (size_t e = 0; e < E; ++e) rows[emb[e]] = qft_entry(int(E), int(e), int(j));
                CUDA_TRY(cudaMemcpyAsync(V_d + j * N, rows, N * sizeof(double2), cudaMemcpyHostToDevice, s));
            }
        }
        Tile chunk[128];
        for (long t0 = 0; t0 < pd.ntiles; t0 += 128) {
            const long n = std::min<long>(128, pd.ntiles - t0);
            for (long t = 0; t < n; ++t) chunk[t] = tile_at(t0 + t, pd.M, pd.E, pd.cb, 0);
            CUDA_TRY(cudaMemcpyAsync(tiles_d + t0, chunk, n * sizeof(Tile), cudaMemcpyHostToDevice, s));
        }
        constexpr int kMapMax = MAX_ANY_TILE_THREADS;
        int map[kMapMax];
        if (pd.nthreads > kMapMax)
            return fail(MSQOC_ERR_INVALID_ARG, "tile of %d threads exceeds the %d-entry lane map", pd.nthreads, kMapMax);
        const Tile last = tile_at(pd.ntiles - 1, pd.M, pd.E, pd.cb, 0);
        for (int k = 0; k <= pd.cb; ++k) {
            build_lanemap(pd.L, pd.q, k < pd.cb ? pd.cb : last.ncol, k < pd.cb ? k + 1 : last.ncol0, pd.nthreads,
                          pd.pair, map);
            CUDA_TRY(cudaMemcpyAsync(map_d + size_t(k) * pd.nthreads, map, pd.nthreads * sizeof(int),
                                     cudaMemcpyHostToDevice, s));
        }
    }

    // ---- the objective's kernels (controls, forward sweep, terminal terms, reduction)
    {
        const int threads = 256;
        const int blocks = static_cast<int>(std::min<int64_t>((pd.nsteps + threads - 1) / threads, 4096));
        k_phases<<<phase_blocks(pd), threads, 0, s>>>(pd);
        CUDA_TRY(cudaGetLastError());
        k_controls<<<blocks, threads, 0, s>>>(pd);
        CUDA_TRY(cudaGetLastError());
    }
    CUDA_TRY(launch_sweep(sweep_args(pd, pd_d, tiles_d, map_d, SWEEP_OBJECTIVE, 0), pd.ntiles, s));
    k_terminal<<<pd.M, TERM_THREADS, 0, s>>>(pd, 0);
    CUDA_TRY(cudaGetLastError());
    k_finalize_scalars<<<1, 32, 0, s>>>(pd, outs, outs + 1, M > 1 ? outs + 2 : nullptr, nullptr);
    CUDA_TRY(cudaGetLastError());

    // ---- results to the caller (host or device) and the device status word
    CUDA_TRY(cudaMemcpyAsync(P_out, outs, sizeof(double), cudaMemcpyDefault, s));
    if (J_out) CUDA_TRY(cudaMemcpyAsync(J_out, outs + 1, sizeof(double), cudaMemcpyDefault, s));
    if (pen_out && M > 1) CUDA_TRY(cudaMemcpyAsync(pen_out, outs + 2, (M - 1) * sizeof(double), cudaMemcpyDefault, s));
    int status_word = 0;
    CUDA_TRY(cudaMemcpyAsync(&status_word, pd.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (status_word) return status_error(status_word);
    return MSQOC_OK;
}

}  // namespace

extern "C" msqoc_status msqoc_eval_objective_noalloc(const msqoc_hamiltonian* H, const msqoc_controls* C,
                                                     const double* target, double T, int64_t nsteps,
                                                     int32_t nwindows, double mu, int32_t solver,
                                                     const double* alpha, const double* W, double* P_out,
                                                     double* J_out, double* pen_out, void* stream) {
    return guarded([&] {
        return eval_objective_noalloc(H, C, target, T, nsteps, nwindows, mu, solver, alpha, W, P_out, J_out, pen_out,
                                      stream);
    });
}
