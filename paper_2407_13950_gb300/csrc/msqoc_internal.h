// Internal definitions shared by the host API and the kernels of libmsqoc.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace msqoc {

constexpr int MAXQ = 6;       // subsystems
constexpr int MAXNF = 64;     // carriers over all subsystems
constexpr int MAXL = 4;       // levels per subsystem handled by the sweep kernels
constexpr int MAX_TILE_THREADS = 256;  // threads of one sweep tile (leaves 255 registers a thread)

enum Solver { SOLVER_FP64 = 1, SOLVER_MIXED = 2 };

// device status word bits
enum Status { ST_OK = 0, ST_TIMEOUT = 1, ST_BAD_LAUNCH = 2, ST_SOLVER_RANGE = 4 };

// Per-step table: first active spline index, the step solver's iteration counts packed as
// j1 | j2 << 8 | passes << 16 | out-of-range << 24, and the three spline weights.
struct __align__(16) Spline4 {
    int s;
    int cnt;
    double w0, w1, w2;
};

// Everything a kernel needs about one problem and one evaluation.  Passed by value.
struct ProbDev {
    // shape
    int q, L, N, E, F, ness, d1, M, nfsum, d;
    int cb;        // columns per tile
    int nblk;      // E / cb
    int nthreads;  // threads per tile (multiple of 32)
    int ntiles;    // M * nblk
    int solver;
    int64_t nsteps;
    double T, h, mu, dtau;
    double lam;    // ||a + a^+|| on L levels (bound of the ladder-term norm per unit |d|)
    int nf[MAXQ];
    int cof[MAXQ + 1];           // carrier offsets
    double omega[MAXNF];
    double sc[2 * MAXL];         // (h/2) sqrt(l+1) [dir +] and (h/2) sqrt(l) [dir -], index 2l+dir
    double wsq[2 * MAXL];        // sqrt(l+1) [dir +] and sqrt(l) [dir -]: product weights
    // constant tables
    const double2* P;            // [N] (1 + i h/2 D_i)^-1
    const int* fiber_order;      // [F] fibers sorted by neighbour class
    const int* emb;              // [E] full row index of essential column e
    const double2* V;            // [E][N] target
    // inputs of this evaluation (device memory)
    const double* alpha;         // [d]
    const double2* W;            // [M-1][E][N]
    // scratch
    double2* ctrl;               // [nsteps][q] d_k(t_{n+1/2})
    Spline4* spl;                // [nsteps] (first spline index, solver counts, w0, w1, w2)
    double2* phase;              // [nsteps][nfsum] exp(i Omega t_{n+1/2})
    double2* hist;               // [nsteps][nblk][cb][N] midpoint states Ubar_n
    double2* Uend;               // [M][E][N] U^m(t_m)
    double2* Lterm;              // [M][E][N] Lambda^m(t_m)
    double2* Lam0;               // [M][E][N] Lambda^m(t_{m-1})
    double* term;                // [M] pen_m (m < M), J (m = M)
    double* gpart;               // [ntiles][d] per-tile alpha-gradient partials
    int* status;                 // status word (ST_* bits)
};

// shared-memory bytes of a sweep launch
size_t sweep_smem_bytes(const ProbDev& pd, bool bwd);

// launchers (defined per subsystem count in inst_q*.cu); return cudaError_t
cudaError_t launch_sweep(const ProbDev& pd, bool bwd, bool want_hist, cudaStream_t s);

}  // namespace msqoc
