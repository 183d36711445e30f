// Internal definitions shared by the host API and the kernels of libmsqoc.
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>

namespace msqoc {

constexpr int MAXQ = 6;       // subsystems
constexpr int MAXEX = 15;     // exchange-coupled pairs (q (q - 1) / 2)
constexpr int MAXNF = 64;     // carriers over all subsystems
constexpr int MAXL = 4;       // levels per subsystem handled by the sweep kernels
constexpr int MAX_TILE_THREADS = 256;       // threads of a one-thread-per-fiber tile (255 registers a thread)
constexpr int MAX_LEAN_TILE_THREADS = 384;  // the same family compiled for 168 registers a thread: tiles of
                                            // up to 12 warps, or two 6-warp tiles on an SM
constexpr int MAX_PAIR_TILE_THREADS = 384;  // threads of a lane-pair tile (168 registers a thread)
constexpr int MAX_QUAD_TILE_THREADS = 384;  // threads of a lane-quad tile (168 registers a thread)
constexpr int MAX_HDEPTH = 8;               // steps per history group at most
// threads of any tile (host arrays of a tile's lane map are sized by it)
constexpr int MAX_ANY_TILE_THREADS = 384;
static_assert(MAX_TILE_THREADS <= MAX_ANY_TILE_THREADS && MAX_LEAN_TILE_THREADS <= MAX_ANY_TILE_THREADS &&
                  MAX_PAIR_TILE_THREADS <= MAX_ANY_TILE_THREADS && MAX_QUAD_TILE_THREADS <= MAX_ANY_TILE_THREADS,
              "a tile limit exceeds MAX_ANY_TILE_THREADS");

enum Solver { SOLVER_FP64 = 1, SOLVER_MIXED = 2 };

// device status word bits
enum Status { ST_OK = 0, ST_TIMEOUT = 1, ST_BAD_LAUNCH = 2, ST_SOLVER_RANGE = 4, ST_GRAD_RANGE = 8 };

// Index of the first of the three quadratic B-splines (spacing dtau, d1 of them) active at time
// t, clamped to the grid.  The controls kernel, the sweeps and the host's sizing of the shared
// gradient all take it from here.
__host__ __device__ inline int spline_index(double t, double dtau, int d1) {
    const int s0 = static_cast<int>(floor(t / dtau));
    return s0 < 0 ? 0 : (s0 > d1 - 3 ? d1 - 3 : s0);
}

// Per-step table: first active spline index, the step solver's iteration counts packed as
// j1 | j2 << 8 | passes << 16 | out-of-range << 24, and the three spline weights.
struct __align__(16) Spline4 {
    int s;
    int cnt;
    double w0, w1, w2;
};

// Everything a kernel needs about one problem.  The small kernels take it by value; the sweep
// kernels read it from a device copy (several problems share a batched sweep launch).
struct ProbDev {
    // shape
    int q, L, N, E, F, ness, d1, M, nfsum, d;
    int m_off;     // global index of the first window minus one (0 unless the problem is a shard)
    int M_glob;    // windows of the whole problem (M for a whole problem; windows are local
                   // 1..M, global m_off + 1 .. m_off + M, on the whole problem's time grid)
    int cb;        // columns of a full tile
    int nthreads;  // threads per tile (multiple of 32)
    int pair;      // kernel family: log2 of the threads per fiber (0: one thread, 1: a lane pair,
                   // the real and the imaginary part; 2: a lane quad, a pair per entry of a
                   // 2-level fiber)
    int lean;      // one thread per fiber compiled for 168 registers (more warps per SM), pair = 0
    int ntiles;    // tiles of the problem's sweeps
    int gspan;     // splines per carrier in a tile's shared alpha-gradient: every spline active in
                   // one window (from the window's first active spline), with a margin
    int glocal;    // doubles of that gradient per window slot: nfsum gspan 2
    int solver;
    int kseg;      // steps per history segment (checkpoint interval; >= the longest window when
                   // every midpoint state is kept)
    int nseg;      // segments per window: ceil(longest window / kseg)
    int hdepth;    // steps per history synchronisation: midpoint states staged and stored (forward)
                   // or fetched (adjoint) in groups of hdepth steps, one wait per group
    int64_t nsteps;
    double T, h, mu, dtau;
    double lam;    // ||a + a^+|| on L levels (bound of the ladder-term norm per unit |d|)
    int nf[MAXQ];
    int cof[MAXQ + 1];           // carrier offsets
    double omega[MAXNF];
    double sc[2 * MAXL];         // (h/2) sqrt(l+1) [dir +] and (h/2) sqrt(l) [dir -], index 2l+dir
    // dipole exchange J_jk (a_k^+ a_j + a_k a_j^+), j < k, a constant part of the off-diagonal
    // operator of the step: pairs, (h/2) J_jk, and its contribution to the contraction bound
    int nex;
    int ex_j[MAXEX], ex_k[MAXEX];
    double ex_c[MAXEX];
    double rho_ex;
    double wsq[2 * MAXL];        // sqrt(l+1) [dir +] and sqrt(l) [dir -]: product weights
    // constant tables
    const double2* P;            // [N] (1 + i h/2 D_i)^-1
    const int* emb;              // [E] full row index of essential column e
    const double2* V;            // [E][N] target
    // inputs of this evaluation (device memory)
    const double* alpha;         // [d]
    const double2* W;            // [M-1][E][N]; W + (m - 2) E N is the initial state of local
                                 // window m (a shard that starts past the first window reads its
                                 // first window's initial state at index -1)
    // scratch
    double2* ctrl;               // [nsteps][q] d_k(t_{n+1/2})
    Spline4* spl;                // [nsteps] (first spline index, solver counts, w0, w1, w2)
    double2* phase;              // [nsteps][nfsum] exp(i Omega t_{n+1/2})
    double2* hist;               // [M][kseg][E][N] midpoint states Ubar of one segment of every window
                                 // (the mixed solver's one-thread families store each entry as the
                                 // two-float split of Ubar 2^-hsh, hsh the column's scale exponent)
    int* hsh;                    // [M][nseg][E] column scale exponent of each window segment's
                                 // history (mixed solver, one thread per fiber), after hist
    double2* ckpt;               // [M][nseg][E][N] states at the segment starts (kseg < longest window)
    double2* Uend;               // [M][E][N] U^m(t_m)
    double2* Lterm;              // [M][E][N] Lambda^m(t_m)
    double2* Lam0;               // [M][E][N] Lambda^m(t_{m-1})
    double2* Lstate;             // [M][E][N] adjoint state between segments
    double* term;                // [M] pen_m (m < M), J (m = M)
    double* gpart;               // [ntiles][d] per-tile alpha-gradient partials
    int* status;                 // status word (ST_* bits)
};

// One sweep tile (one CTA): `ncol` consecutive columns of problem `prob` in window-major column
// order, starting at column c0 of window m0 (1-based).  The first `ncol0` columns belong to
// window m0, the rest to window m0 + 1 (a tile covers at most two windows).  `map` selects the
// thread -> (column, fiber) assignment in the launch's lane maps; `tloc` is the tile's index
// among its problem's tiles (row of the problem's gradient partials).
struct Tile {
    int prob, m0, c0, ncol, ncol0, map, tloc, pad;
};

// What a sweep launch does.
enum SweepMode {
    SWEEP_OBJECTIVE = 0,  // forward over whole windows; end states U^m(t_m)
    SWEEP_HISTORY = 1,    // forward over whole windows for a gradient; also every midpoint state
                          // (a problem with one history segment) or the states at the segment
                          // starts (checkpoints, more segments)
    SWEEP_RECOMPUTE = 3,  // forward over segment `seg` from its checkpoint; midpoint states
                          // (no work for a problem with one segment)
    SWEEP_ADJOINT = 4,    // adjoint over segment `seg` with the fused gradient quadrature
    SWEEP_ROLLOUT = 5     // forward over the whole time grid as one window from the identity
                          // embedding; the state at every window boundary t_m into `out`
};

// Arguments of one sweep launch (uniform over its tiles; problems share shape and solver).
struct SweepArgs {
    const ProbDev* pds;   // [problems] device copies
    const Tile* tiles;    // [tiles] one per CTA
    const int* lanemap;   // [maps][threads]: (column << 16 | fiber), ~value for idle lanes
    int cpt;              // columns of the widest tile (shared-memory sizing)
    int gmax;             // largest shared alpha-gradient per window slot (doubles) over the problems
    int mode;             // SweepMode
    int seg;              // segment (SWEEP_RECOMPUTE, SWEEP_ADJOINT)
    int L, q, solver, nthreads;
    int pair;             // kernel family: log2 of the threads per fiber (0, 1 or 2)
    int lean;             // pair = 0 with the 168-register build (ProbDev::lean)
    int hdepth;           // steps per history group (ProbDev::hdepth), >= 1
    double2* out;         // SWEEP_ROLLOUT: [M-1][E][N] states at the window boundaries
};

// shared-memory bytes of a sweep launch
size_t sweep_smem_bytes(const SweepArgs& a);

// launcher (dispatches on L, q, solver, direction); returns cudaError_t
cudaError_t launch_sweep(const SweepArgs& a, int ntiles, cudaStream_t s);

// resident CTAs per SM of a sweep kernel at this launch shape (0 on error)
int sweep_ctas_per_sm(const SweepArgs& a);

}  // namespace msqoc
