// Host-side definitions shared by the C-ABI translation units of libmsqoc (problems, batches).
#pragma once

#include <cstddef>
#include <cstdint>
#include <new>

#include "../../include/msqoc.h"
#include "msqoc_internal.h"

// One problem on one device: the model tables, its tile layout and every buffer an evaluation
// needs.  Created by msqoc_create_problem, which owns all of it.
struct msqoc_problem {
    msqoc::ProbDev pd{};
    int device = 0;
    int ckpt_interval = 1;   // K (1 = every midpoint state kept)
    size_t nW = 0;           // doubles in W
    int nWs = 0;             // window states in W (M - 1, or those a shard reads)
    int npen = 0;            // penalty terms (M - 1, or those a shard owns)
    size_t ne = 0;           // N*E
    // owned device buffers
    msqoc::ProbDev* pds = nullptr;   // device copy of pd (read by the sweeps)
    msqoc::Tile* tiles = nullptr;
    int* lanemap = nullptr;
    msqoc::Tile* tiles_ro = nullptr;   // the roll-out sweep: one window over the whole grid
    int* lanemap_ro = nullptr;
    int ntiles_ro = 0;
    double2* P = nullptr;
    int* emb = nullptr;
    double2* V = nullptr;
    double* alpha_dev = nullptr;   // the evaluation's inputs (copied from the caller's arrays)
    double* W_dev = nullptr;
    double2* ctrl = nullptr;
    msqoc::Spline4* spl = nullptr;
    double2* phase = nullptr;
    double2* hist = nullptr;       // allocated by the first gradient evaluation
    double2* ckpt = nullptr;       // (with hist, when K > 1)
    double2* Lstate = nullptr;     // (with hist, when K > 1)
    double2* Uend = nullptr;
    double2* Lterm = nullptr;
    double2* Lam0 = nullptr;
    double* term = nullptr;
    double* gpart = nullptr;
    int* status = nullptr;
    double* out_dev = nullptr;     // outputs of the last evaluation: P, J, pen[M-1], galpha[d], gW[nW]
    double* reg_dev = nullptr;     // regularization: alpha[d], gradient[d], energy shares[q d1], R
    int* status_host = nullptr;    // pinned
    size_t bytes = 0;              // device bytes held now
    size_t grad_bytes = 0;         // bytes the first gradient evaluation adds
    // profiling: CUDA events around each kernel of an evaluation
    bool profile = false;
    cudaEvent_t ev[MSQOC_NKERNELS][2] = {};
    bool ran[MSQOC_NKERNELS] = {};
};

namespace msqoc {

// records the calling thread's last error message; returns code
msqoc_status fail(msqoc_status code, const char* fmt, ...);

#define CUDA_TRY(expr)                                                                              \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess)                                                                      \
            return ::msqoc::fail(_e == cudaErrorMemoryAllocation ? MSQOC_ERR_OUT_OF_MEMORY           \
                                                                 : MSQOC_ERR_CUDA,                  \
                                 "%s failed: %s", #expr, cudaGetErrorString(_e));                   \
    } while (0)

bool is_device_ptr(const void* p);

// Runs f and turns a C++ exception (a failed host allocation in a std container) into a status:
// nothing may unwind across the C ABI.
template <class F>
msqoc_status guarded(F&& f) noexcept {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return fail(MSQOC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail(MSQOC_ERR_INTERNAL, "unexpected C++ exception");
    }
}

// tile layout (see msqoc_api.cu)
void build_lanemap(int L, int q, int ncol, int ncol0, int nthreads, int pair, int* out);
// kernel family (pair: log2 of the threads per fiber, 0, 1 or 2) and columns per tile of a problem
struct TileChoice {
    int cpt, pair, lean;
};
Tile tile_at(long t, int M, int E, int cpt, int prob);
long tile_count(int M, int E, int cpt);
SweepArgs sweep_args(const ProbDev& pd, const ProbDev* pds_dev, const Tile* tiles, const int* lanemap, int mode,
                     int seg);

// Output staging layout in out_dev (doubles): P, J, pen[npen], grad_alpha[d], grad_W[nW].
// grad_alpha and grad_W start at even offsets: grad_W is written as double2 (16-byte aligned).
struct OutLayout {
    size_t pen, ga, gw, total;
};
OutLayout out_layout(int npen, int d, size_t nW);
// window states a problem reads (W blocks) and penalty terms it owns: M - 1 each for a whole
// problem; for a shard, W^k for k = max(m_off, 1) .. min(m_off + M, M_glob - 1) and pen_m for
// its windows m < M_glob
int w_blocks(const ProbDev& pd);
int pen_count(const ProbDev& pd);
bool is_shard(const ProbDev& pd);

// steps of an evaluation of one problem (stream-ordered)
msqoc_status stage_inputs(msqoc_problem* p, const double* alpha, const double* W, cudaStream_t s);
msqoc_status ensure_gradient_buffers(msqoc_problem* p, cudaStream_t s);
int phase_blocks(const ProbDev& pd);   // blocks of 256 threads for k_phases
msqoc_status launch_controls(msqoc_problem* p, cudaStream_t s);
msqoc_status launch_terminal(msqoc_problem* p, bool want_lambda, cudaStream_t s);
// P, J (may be NULL), pen (may be NULL) of the last forward sweep into device arrays
msqoc_status launch_objective_outputs(msqoc_problem* p, double* P, double* J, double* pen, cudaStream_t s);
// P (may be NULL), dP/dalpha, dP/dW (NULL when there is no window state) of the last adjoint
// sweep into device arrays
msqoc_status launch_gradient_outputs(msqoc_problem* p, double* P, double* ga, double* gw, cudaStream_t s);
msqoc_status status_error(int st);
msqoc_status check_status_sync(msqoc_problem* p, cudaStream_t s);

}  // namespace msqoc
