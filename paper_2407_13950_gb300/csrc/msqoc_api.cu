// Host side of libmsqoc: problem packing, device memory, launches and the C ABI.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/msqoc.h"
#include "msqoc_aux.cuh"
#include "msqoc_internal.h"
#include "msqoc_sweep.cuh"

using namespace msqoc;

namespace {

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

#define CUDA_TRY(expr)                                                                              \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess)                                                                      \
            return fail(_e == cudaErrorMemoryAllocation ? MSQOC_ERR_OUT_OF_MEMORY : MSQOC_ERR_CUDA, \
                        "%s failed: %s", #expr, cudaGetErrorString(_e));                           \
    } while (0)

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

}  // namespace

struct msqoc_problem {
    ProbDev pd{};
    int device = 0;
    size_t nW = 0;         // doubles in W
    size_t ne = 0;         // N*E
    // owned device buffers
    double2* P = nullptr;
    int* fiber_order = nullptr;
    int* emb = nullptr;
    double2* V = nullptr;
    double* alpha_dev = nullptr;   // staging of host inputs
    double* W_dev = nullptr;
    double2* ctrl = nullptr;
    Spline4* spl = nullptr;
    double2* phase = nullptr;
    double2* hist = nullptr;
    double2* Uend = nullptr;
    double2* Lterm = nullptr;
    double2* Lam0 = nullptr;
    double* term = nullptr;
    double* gpart = nullptr;
    int* status = nullptr;
    double* out_dev = nullptr;     // staging of outputs: P, J, pen[M-1], galpha[d], gW[nW]
    int* status_host = nullptr;    // pinned
    size_t bytes = 0;
    // profiling: CUDA events around each kernel of an evaluation
    bool profile = false;
    cudaEvent_t ev[MSQOC_NKERNELS][2] = {};
    bool ran[MSQOC_NKERNELS] = {};
};

namespace {

void free_problem(msqoc_problem* p) {
    void* bufs[] = {p->P, p->fiber_order, p->emb, p->V, p->alpha_dev, p->W_dev, p->ctrl, p->spl, p->phase,
                    p->hist, p->Uend, p->Lterm, p->Lam0, p->term, p->gpart, p->status, p->out_dev};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (p->status_host) cudaFreeHost(p->status_host);
    for (auto& e : p->ev)
        for (auto& x : e)
            if (x) cudaEventDestroy(x);
}

// brackets a kernel launch with profiling events when enabled
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

double ladder_norm(int L) {
    // largest eigenvalue of a + a^+ on L levels (zeros of the Hermite polynomial H_L / sqrt 2)
    switch (L) {
        case 2: return 1.0;
        case 3: return std::sqrt(3.0);
        case 4: return std::sqrt(3.0 + std::sqrt(6.0));
        default: return std::sqrt(2.0 * L);  // safe upper bound (Gershgorin)
    }
}

// Output staging layout in out_dev (doubles): P, J, pen[M-1], grad_alpha[d], grad_W[nW].
// grad_alpha and grad_W start at even offsets: grad_W is written as double2 (16-byte aligned).
struct OutLayout {
    size_t pen, ga, gw, total;
};
OutLayout out_layout(int M, int d, size_t nW) {
    OutLayout o;
    o.pen = 2;
    o.ga = (o.pen + size_t(M - 1) + 1) & ~size_t(1);
    o.gw = (o.ga + size_t(d) + 1) & ~size_t(1);
    o.total = o.gw + nW + 2;
    return o;
}

bool shape_supported(int L, int q) { return (L == 3 && q >= 1 && q <= 5) || (L == 2 && q >= 1 && q <= 6); }

constexpr int kMaxRows = 243;    // largest N of a supported shape (L = 3, q = 5)
constexpr int kMaxFibers = 81;   // largest N / L

// Fibers sorted so that lanes of a warp share their neighbour-list shape: key = bitmask of the
// fixed subsystems whose level is interior (two neighbours), ordered by popcount then mask.
// Stable insertion sort into order[N/L] (equal keys keep ascending fiber order).
void fiber_order_into(int L, int q, int* order) {
    const int F = ipow_i(L, q) / L;
    int key[kMaxFibers];
    for (int f = 0; f < F; ++f) {
        int mask = 0;
        for (int k = 0; k < q - 1; ++k) {
            const int lk = (f / ipow_i(L, q - 2 - k)) % L;
            if (lk > 0 && lk < L - 1) mask |= 1 << k;
        }
        const int kf = (__builtin_popcount(mask) << 16) | mask;
        int pos = f;
        while (pos > 0 && key[pos - 1] > kf) {
            key[pos] = key[pos - 1];
            order[pos] = order[pos - 1];
            --pos;
        }
        key[pos] = kf;
        order[pos] = f;
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

int choose_col_block(int E, int F, int M, int q, int L, int N, int d, int solver, int sms) {
    // Makespan model: a tile occupies one SM for the whole window; an SM's time grows with the
    // warps (lanes, idle ones included) of the tiles it runs.  Tiles are spread evenly, so the
    // busiest SM runs ceil(tiles / sms) of them.  Ties go to the larger block (fewer tiles).
    int best = -1;
    double best_cost = 0.0;
    for (int cb = E; cb >= 1; --cb) {
        if (E % cb) continue;
        if (cb * F > MAX_TILE_THREADS) continue;
        const int nthreads = ((cb * F + 31) / 32) * 32;
        const size_t s1 = sweep_layout(q, L, N, cb, nthreads, d, solver, true).total;
        const size_t s0 = sweep_layout(q, L, N, cb, nthreads, d, solver, false).total;
        if (std::max(s0, s1) > 200 * 1024) continue;
        const long tiles = long(M) * (E / cb);
        const double cost = double((tiles + sms - 1) / sms) * nthreads;
        if (best < 0 || cost < best_cost * 0.999) {
            best = cb;
            best_cost = cost;
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
        for (int e = 0; e < q * q; ++e)
            if (H->jx[e] != 0.0) return fail(MSQOC_ERR_UNSUPPORTED, "dipole exchange (jx) is not supported");
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
// of pd except the device pointers).  col_block 0 = automatic.
msqoc_status shape_problem(const msqoc_hamiltonian* H, const msqoc_controls* C, double T, int64_t nsteps,
                           int32_t nwindows, double mu, int solver, int col_block, int sms, ProbDev& pd) {
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
    pd.M = nwindows;
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
    for (int l = 0; l < MAXL; ++l) {
        pd.sc[2 * l + 0] = 0.5 * pd.h * std::sqrt(double(l + 1));
        pd.sc[2 * l + 1] = 0.5 * pd.h * std::sqrt(double(l));
        pd.wsq[2 * l + 0] = std::sqrt(double(l + 1));
        pd.wsq[2 * l + 1] = std::sqrt(double(l));
    }
    int cb = col_block;
    if (cb == 0) cb = choose_col_block(pd.E, pd.F, pd.M, q, L, pd.N, pd.d, solver, sms);
    if (cb <= 0 || pd.E % cb || cb * pd.F > MAX_TILE_THREADS)
        return fail(MSQOC_ERR_INVALID_ARG, "column block %d invalid for E=%d (needs cb | E, cb*N/L <= %d)", cb, pd.E,
                    MAX_TILE_THREADS);
    pd.cb = cb;
    pd.nblk = pd.E / cb;
    pd.nthreads = ((cb * pd.F + 31) / 32) * 32;
    pd.ntiles = pd.M * pd.nblk;
    if (std::max(sweep_layout(q, L, pd.N, cb, pd.nthreads, pd.d, solver, true).total,
                 sweep_layout(q, L, pd.N, cb, pd.nthreads, pd.d, solver, false).total) > 227 * 1024)
        return fail(MSQOC_ERR_INVALID_ARG, "column block %d needs too much shared memory", cb);
    return MSQOC_OK;
}

}  // namespace

namespace msqoc {
size_t sweep_smem_bytes(const ProbDev& pd, bool bwd) {
    return sweep_layout(pd.q, pd.L, pd.N, pd.cb, pd.nthreads, pd.d, pd.solver, bwd).total;
}
}  // namespace msqoc

extern "C" {

int32_t msqoc_version(void) { return 100; }

int32_t msqoc_last_error(char* buf, size_t len) {
    if (buf && len) {
        size_t n = std::min(len - 1, g_last_error.size());
        memcpy(buf, g_last_error.data(), n);
        buf[n] = 0;
    }
    return static_cast<int32_t>(g_last_error.size());
}

msqoc_status msqoc_create_problem(const msqoc_hamiltonian* H, const msqoc_controls* C, const double* target,
                                  double T, int64_t nsteps, int32_t nwindows, double mu,
                                  const msqoc_options* opt, msqoc_problem** out) {
    if (!out) return fail(MSQOC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    msqoc_status st0 = check_description(H, C, T, nsteps, nwindows);
    if (st0 != MSQOC_OK) return st0;

    msqoc_options o{};
    if (opt) o = *opt;
    const int solver = o.solver == MSQOC_SOLVER_FP64 ? SOLVER_FP64 : SOLVER_MIXED;
    if (o.ckpt_interval != 0 && o.ckpt_interval != 1)
        return fail(MSQOC_ERR_UNSUPPORTED, "checkpoint interval %d not implemented (use 1)", o.ckpt_interval);
    if (o.profile != 0 && o.profile != 1) return fail(MSQOC_ERR_INVALID_ARG, "profile must be 0 or 1");

    auto* p = new (std::nothrow) msqoc_problem();
    if (!p) return fail(MSQOC_ERR_OUT_OF_MEMORY, "host allocation failed");
    ProbDev& pd = p->pd;
    cudaGetDevice(&p->device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (sms <= 0) sms = 1;
    st0 = shape_problem(H, C, T, nsteps, nwindows, mu, solver, o.col_block, sms, pd);
    if (st0 != MSQOC_OK) {
        delete p;
        return st0;
    }
    const int q = pd.q, L = pd.L, nfsum = pd.nfsum;

    // ---- host-side model tables
    const int N = pd.N, E = pd.E;
    p->ne = size_t(N) * E;
    p->nW = 2 * p->ne * size_t(pd.M - 1);
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
    std::vector<int> order(pd.F);
    fiber_order_into(L, q, order.data());

    // ---- device buffers
    const size_t M = pd.M;
    msqoc_status st = MSQOC_OK;
    auto A = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && st == MSQOC_OK)
            st = fail(e == cudaErrorMemoryAllocation ? MSQOC_ERR_OUT_OF_MEMORY : MSQOC_ERR_CUDA,
                      "allocating %s: %s", what, cudaGetErrorString(e));
    };
    A(dalloc(&p->P, N), "P");
    A(dalloc(&p->fiber_order, pd.F), "fiber order");
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
    A(dalloc(&p->out_dev, out_layout(pd.M, pd.d, p->nW).total), "outputs");
    A(cudaMallocHost(reinterpret_cast<void**>(&p->status_host), sizeof(int)), "pinned status");
    p->profile = o.profile == 1;
    if (p->profile)
        for (auto& e : p->ev)
            for (auto& x : e) A(cudaEventCreate(&x), "profiling event");
    if (st == MSQOC_OK) {
        A(cudaMemcpy(p->P, P.data(), N * sizeof(double2), cudaMemcpyHostToDevice), "P copy");
        A(cudaMemcpy(p->fiber_order, order.data(), pd.F * sizeof(int), cudaMemcpyHostToDevice), "order copy");
        A(cudaMemcpy(p->emb, emb.data(), E * sizeof(int), cudaMemcpyHostToDevice), "emb copy");
        A(cudaMemcpy(p->V, Vh.data(), p->ne * sizeof(double2), cudaMemcpyHostToDevice), "target copy");
        A(cudaMemset(p->status, 0, sizeof(int)), "status init");
    }
    if (st != MSQOC_OK) {
        free_problem(p);
        delete p;
        return st;
    }
    pd.P = p->P;
    pd.fiber_order = p->fiber_order;
    pd.emb = p->emb;
    pd.V = p->V;
    pd.ctrl = p->ctrl;
    pd.spl = p->spl;
    pd.phase = p->phase;
    pd.Uend = p->Uend;
    pd.Lterm = p->Lterm;
    pd.Lam0 = p->Lam0;
    pd.term = p->term;
    pd.gpart = p->gpart;
    pd.status = p->status;
    p->bytes = sizeof(double2) * (N + p->ne * (1 + 3 * M) + size_t(nsteps) * (q + nfsum)) +
               sizeof(Spline4) * size_t(nsteps) + sizeof(double) * (pd.d + p->nW + M + size_t(pd.ntiles) * pd.d) +
               sizeof(int) * (pd.F + E + 1);
    *out = p;
    return MSQOC_OK;
}

msqoc_status msqoc_query(const msqoc_problem* p, int64_t* d, int64_t* nW, size_t* device_bytes) {
    if (!p) return fail(MSQOC_ERR_INVALID_ARG, "problem is NULL");
    if (d) *d = p->pd.d;
    if (nW) *nW = static_cast<int64_t>(p->nW);
    if (device_bytes)
        *device_bytes = p->bytes + size_t(p->pd.nsteps) * p->ne * sizeof(double2);  // + history
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

namespace {

// stage the inputs on the device (copies host arrays; device arrays are used in place)
msqoc_status stage_inputs(msqoc_problem* p, const double* alpha, const double* W, cudaStream_t s) {
    if (!alpha) return fail(MSQOC_ERR_INVALID_ARG, "alpha is NULL");
    if (p->pd.M > 1 && !W) return fail(MSQOC_ERR_INVALID_ARG, "W is NULL but M > 1");
    if (is_device_ptr(alpha)) {
        p->pd.alpha = alpha;
    } else {
        CUDA_TRY(cudaMemcpyAsync(p->alpha_dev, alpha, p->pd.d * sizeof(double), cudaMemcpyHostToDevice, s));
        p->pd.alpha = p->alpha_dev;
    }
    if (p->pd.M > 1) {
        if (is_device_ptr(W)) {
            if (reinterpret_cast<uintptr_t>(W) % 16) return fail(MSQOC_ERR_INVALID_ARG, "device W must be 16-byte aligned");
            p->pd.W = reinterpret_cast<const double2*>(W);
        } else {
            CUDA_TRY(cudaMemcpyAsync(p->W_dev, W, p->nW * sizeof(double), cudaMemcpyHostToDevice, s));
            p->pd.W = reinterpret_cast<const double2*>(p->W_dev);
        }
    } else {
        p->pd.W = reinterpret_cast<const double2*>(p->W_dev);
    }
    return MSQOC_OK;
}

msqoc_status launch_forward_part(msqoc_problem* p, bool want_hist, cudaStream_t s) {
    ProbDev& pd = p->pd;
    for (bool& r : p->ran) r = false;
    {
        Mark mk(p, MSQOC_KERNEL_CONTROLS, s);
        const int threads = 256;
        int blocks = static_cast<int>(std::min<int64_t>((pd.nsteps + threads - 1) / threads, 4096));
        k_controls<<<blocks, threads, 0, s>>>(pd);
        CUDA_TRY(cudaGetLastError());
    }
    {
        Mark mk(p, MSQOC_KERNEL_FORWARD, s);
        CUDA_TRY(launch_sweep(pd, false, want_hist, s));
    }
    {
        Mark mk(p, MSQOC_KERNEL_TERMINAL, s);
        k_terminal<<<pd.M, TERM_THREADS, 0, s>>>(pd, want_hist ? 1 : 0);
        CUDA_TRY(cudaGetLastError());
    }
    return MSQOC_OK;
}

msqoc_status check_status_sync(msqoc_problem* p, cudaStream_t s) {
    CUDA_TRY(cudaMemcpyAsync(p->status_host, p->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const int st = *p->status_host;
    if (st) {
        cudaMemsetAsync(p->status, 0, sizeof(int), s);
        if (st & ST_TIMEOUT) return fail(MSQOC_ERR_TIMEOUT, "a bounded device wait gave up (status %d)", st);
        if (st & ST_SOLVER_RANGE)
            return fail(MSQOC_ERR_UNSUPPORTED, "time step too large for the step solver (h*|H_c|/2 >= 0.5)");
        return fail(MSQOC_ERR_INTERNAL, "device status %d", st);
    }
    return MSQOC_OK;
}

}  // namespace

extern "C" {

msqoc_status msqoc_eval_objective(msqoc_problem* p, const double* alpha, const double* W, double* P_out,
                                  double* J_out, double* pen_out, void* stream) {
    if (!p) return fail(MSQOC_ERR_INVALID_ARG, "problem is NULL");
    if (!P_out) return fail(MSQOC_ERR_INVALID_ARG, "P_out is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    msqoc_status st = stage_inputs(p, alpha, W, s);
    if (st) return st;
    st = launch_forward_part(p, false, s);
    if (st) return st;
    const ProbDev& pd = p->pd;
    const bool dP = is_device_ptr(P_out), dJ = !J_out || is_device_ptr(J_out), dpen = !pen_out || is_device_ptr(pen_out);
    double* o = p->out_dev;
    {
        Mark mk(p, MSQOC_KERNEL_FINALIZE, s);
            k_finalize_scalars<<<1, 32, 0, s>>>(pd, dP ? P_out : o, J_out ? (dJ ? J_out : o + 1) : nullptr,
                                           pen_out && pd.M > 1 ? (dpen ? pen_out : o + 2) : nullptr, nullptr);
        CUDA_TRY(cudaGetLastError());
    }
    const bool all_dev = dP && dJ && dpen;
    if (all_dev) return MSQOC_OK;
    if (!dP) CUDA_TRY(cudaMemcpyAsync(P_out, o, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (J_out && !dJ) CUDA_TRY(cudaMemcpyAsync(J_out, o + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (pen_out && !dpen && pd.M > 1)
        CUDA_TRY(cudaMemcpyAsync(pen_out, o + 2, (pd.M - 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    return check_status_sync(p, s);
}

msqoc_status msqoc_eval_gradient(msqoc_problem* p, const double* alpha, const double* W, double* P_out,
                                 double* grad_alpha, double* grad_W, void* stream) {
    if (!p) return fail(MSQOC_ERR_INVALID_ARG, "problem is NULL");
    if (!grad_alpha) return fail(MSQOC_ERR_INVALID_ARG, "grad_alpha is NULL");
    if (p->pd.M > 1 && !grad_W) return fail(MSQOC_ERR_INVALID_ARG, "grad_W is NULL but M > 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!p->hist) {
        const size_t n = size_t(p->pd.nsteps) * p->ne;
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p->hist), n * sizeof(double2));
        if (e != cudaSuccess) {
            p->hist = nullptr;
            return fail(MSQOC_ERR_OUT_OF_MEMORY, "history buffer (%zu bytes): %s", n * sizeof(double2),
                        cudaGetErrorString(e));
        }
        p->pd.hist = p->hist;
    }
    msqoc_status st = stage_inputs(p, alpha, W, s);
    if (st) return st;
    st = launch_forward_part(p, true, s);
    if (st) return st;
    const ProbDev& pd = p->pd;
    {
        Mark mk(p, MSQOC_KERNEL_ADJOINT, s);
        CUDA_TRY(launch_sweep(pd, true, false, s));
    }
    const bool dP = !P_out || is_device_ptr(P_out), dga = is_device_ptr(grad_alpha),
               dgw = pd.M == 1 || is_device_ptr(grad_W);
    double* o = p->out_dev;
    const OutLayout ol = out_layout(pd.M, pd.d, p->nW);
    if (pd.M > 1 && dgw && reinterpret_cast<uintptr_t>(grad_W) % 16)
        return fail(MSQOC_ERR_INVALID_ARG, "device grad_W must be 16-byte aligned");
    double* ga_dst = dga ? grad_alpha : o + ol.ga;
    double* gw_dst = pd.M == 1 ? nullptr : (dgw ? grad_W : o + ol.gw);
    {
        Mark mk(p, MSQOC_KERNEL_FINALIZE, s);
        k_finalize_scalars<<<std::max(1, (pd.d + 255) / 256), 256, 0, s>>>(pd, P_out ? (dP ? P_out : o) : nullptr,
                                                                          nullptr, nullptr, ga_dst);
        CUDA_TRY(cudaGetLastError());
        if (pd.M > 1) {
            const size_t total = p->ne * (pd.M - 1);
            const int blocks = static_cast<int>(std::min<size_t>((total + 255) / 256, 8192));
            k_grad_W<<<blocks, 256, 0, s>>>(pd, reinterpret_cast<double2*>(gw_dst));
            CUDA_TRY(cudaGetLastError());
        }
    }
    if (dP && dga && dgw) return MSQOC_OK;
    if (P_out && !dP) CUDA_TRY(cudaMemcpyAsync(P_out, o, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (!dga) CUDA_TRY(cudaMemcpyAsync(grad_alpha, ga_dst, pd.d * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (!dgw) CUDA_TRY(cudaMemcpyAsync(grad_W, gw_dst, p->nW * sizeof(double), cudaMemcpyDeviceToHost, s));
    return check_status_sync(p, s);
}

}  // extern "C"

extern "C" msqoc_status msqoc_kernel_times(msqoc_problem* p, float* ms) {
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

// ------------------------------------------------------------------ objective without allocation
// Scratch of msqoc_eval_objective_noalloc: every table and intermediate of one objective
// evaluation, carved into 256-byte-aligned regions.  Static device storage: the module holds
// it on every GPU where it is loaded, and no call allocates.  In host code the name below is
// only a stand-in registered with the runtime; the device address comes from
// cudaGetSymbolAddress (noalloc_scratch below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[MSQOC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_base[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up on the first call
// for that device (with that device current) and cached.
msqoc_status noalloc_scratch(unsigned char** base) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(MSQOC_ERR_UNSUPPORTED, "device %d is beyond the %d devices this entry point serves", dev,
                    kMaxDevices);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_base[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(MSQOC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch on device %d failed: %s", dev,
                        cudaGetErrorString(e));
        g_noalloc_base[dev] = static_cast<unsigned char*>(ptr);
    }
    *base = g_noalloc_base[dev];
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

extern "C" msqoc_status msqoc_eval_objective_noalloc(const msqoc_hamiltonian* H, const msqoc_controls* C,
                                                     const double* target, double T, int64_t nsteps,
                                                     int32_t nwindows, double mu, int32_t solver,
                                                     const double* alpha, const double* W, double* P_out,
                                                     double* J_out, double* pen_out, void* stream) {
    if (!alpha || !P_out) return fail(MSQOC_ERR_INVALID_ARG, "alpha or P_out is NULL");
    msqoc_status st = check_description(H, C, T, nsteps, nwindows);
    if (st != MSQOC_OK) return st;
    if (nwindows > 1 && !W) return fail(MSQOC_ERR_INVALID_ARG, "W is NULL but M > 1");
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ProbDev pd{};
    st = shape_problem(H, C, T, nsteps, nwindows, mu, solver == MSQOC_SOLVER_FP64 ? SOLVER_FP64 : SOLVER_MIXED, 0,
                       std::max(sms, 1), pd);
    if (st != MSQOC_OK) return st;

    // ---- scratch layout; the limit depends on the problem's size only
    const size_t N = pd.N, E = pd.E, ne = N * E, M = pd.M, nt = size_t(nsteps);
    const size_t nW = 2 * ne * (M - 1);
    Carve cv;
    const size_t o_status = cv.take<int>(1), o_term = cv.take<double>(M), o_out = cv.take<double>(M + 1),
                 o_P = cv.take<double2>(N), o_order = cv.take<int>(pd.F), o_emb = cv.take<int>(E),
                 o_V = cv.take<double2>(ne), o_alpha = cv.take<double>(pd.d), o_W = cv.take<double>(nW),
                 o_ctrl = cv.take<double2>(nt * pd.q), o_spl = cv.take<Spline4>(nt),
                 o_phase = cv.take<double2>(nt * pd.nfsum), o_Uend = cv.take<double2>(M * ne);
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
    int* order_d = reinterpret_cast<int*>(base + o_order);
    int* emb_d = reinterpret_cast<int*>(base + o_emb);
    double2* V_d = reinterpret_cast<double2*>(base + o_V);
    pd.P = Pd;
    pd.fiber_order = order_d;
    pd.emb = emb_d;
    pd.V = V_d;
    pd.ctrl = reinterpret_cast<double2*>(base + o_ctrl);
    pd.spl = reinterpret_cast<Spline4*>(base + o_spl);
    pd.phase = reinterpret_cast<double2*>(base + o_phase);
    pd.Uend = reinterpret_cast<double2*>(base + o_Uend);
    double* outs = reinterpret_cast<double*>(base + o_out);   // P, J, pen[M-1]

    // ---- model tables, built in small host buffers and copied in (a pageable host-to-device
    // copy has consumed its source when cudaMemcpyAsync returns, so the buffers are reused)
    CUDA_TRY(cudaMemsetAsync(pd.status, 0, sizeof(int), s));
    {
        double2 rows[kMaxRows];
        for (size_t i = 0; i < N; ++i) rows[i] = precond_entry(pd.h, drift_entry(H, pd.q, pd.L, int(i)));
        CUDA_TRY(cudaMemcpyAsync(Pd, rows, N * sizeof(double2), cudaMemcpyHostToDevice, s));
        int order[kMaxFibers];
        fiber_order_into(pd.L, pd.q, order);
        CUDA_TRY(cudaMemcpyAsync(order_d, order, pd.F * sizeof(int), cudaMemcpyHostToDevice, s));
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
    }
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

    // ---- the objective's kernels (controls, forward sweep, terminal terms, reduction)
    {
        const int threads = 256;
        const int blocks = static_cast<int>(std::min<int64_t>((pd.nsteps + threads - 1) / threads, 4096));
        k_controls<<<blocks, threads, 0, s>>>(pd);
        CUDA_TRY(cudaGetLastError());
    }
    CUDA_TRY(launch_sweep(pd, false, false, s));
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
    if (status_word & ST_TIMEOUT) return fail(MSQOC_ERR_TIMEOUT, "a bounded device wait gave up (status %d)", status_word);
    if (status_word & ST_SOLVER_RANGE)
        return fail(MSQOC_ERR_UNSUPPORTED, "time step too large for the step solver (h*|H_c|/2 >= 0.5)");
    if (status_word) return fail(MSQOC_ERR_INTERNAL, "device status %d", status_word);
    return MSQOC_OK;
}
