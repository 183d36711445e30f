/*
 * Plain FP64 CPU oracle for one multiple-shooting objective + gradient evaluation.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
 * CPU-baseline leg are the only users.  It shares no code, header, table or helper with
 * the CUDA library; it is deliberately slow and dense so that every step can be checked
 * against the paper by eye:
 *
 *  - model (Sec. 2, Eqs. sys-ham, ctrl-ham, dj-ctrl and the B-spline envelope): dense
 *    lowering matrices A_k = I x .. x a x .. x I, drift and control Hamiltonians built from
 *    dense matrix products of them, controls summed literally over every spline and carrier;
 *  - time stepping (Sec. 5: implicit midpoint rule): per step the dense matrices
 *    A = I + i(h/2)H(t_{n+1/2}) and B = I - i(h/2)H(t_{n+1/2}) are formed and
 *    A U_{n+1} = B U_n is solved by complex LU with partial pivoting;
 *  - windows (Sec. 3, Eqs. sch-op, sch-ic): window m starts from W^{m-1}, W^0 = identity
 *    embedding of the essential subspace;
 *  - objective (Eqs. mod-infid, penalty-fcn): generalized infidelity on the last window plus
 *    (mu/2) sum ||U^m(t_m) - W^m||_F^2;
 *  - adjoint (Eqs. lambda-de, terminal; Sec. 5 "discretize-then-optimize"): the exact
 *    discrete adjoint of the midpoint rule, B Lambda_n = A Lambda_{n+1}, with the
 *    gradient (Eq. grad-int) as the midpoint sum 2h Re<Lbar_n, i dH/dalpha Ubar_n>_F;
 *  - window-state gradient (Eq. dP-dW with the factor 2 derived in Appendix B, Eq. dT-dW-j):
 *    mu (W^m - U^m(t_m)) - 2 Lambda^{m+1}(t_m).
 *
 * Readings where the paper is silent (all listed with reasons in the design notes):
 * controls are evaluated at the step midpoint t_{n+1/2}; the global grid h = T/nsteps is
 * split into windows at n_m = floor(m nsteps / M); splines are centred at (s - 1/2) dtau with
 * dtau = T/(d1 - 2); the infidelity uses n := E (number of essential columns) and the
 * default penalty weight is mu = 2/E (Sec. 5).
 *
 * Layouts (all complex numbers interleaved re, im): matrices are column-major; W is
 * [M-1][E][N]; alpha is [k][f][s][alpha^(1), alpha^(2)].
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    int q;                 /* number of subsystems */
    int L;                 /* levels per subsystem */
    int ness;              /* essential levels per subsystem */
    const double* xi;      /* [q] self-Kerr (rad/ns) */
    const double* xi_cross;/* [q*q] row-major, entry (k,l) with k<l used (rad/ns) */
    const double* detune;  /* [q] or NULL: omega_k - omega_rot (paper's Eq. sys-ham) */
    const double* jx;      /* [q*q] or NULL: dipole exchange J_kl, k<l used */
    const int* nf;         /* [q] carriers per subsystem */
    const double* omega;   /* [sum nf] carrier frequencies, subsystem-major (rad/ns) */
    int d1;                /* B-spline coefficients per carrier */
    double T;              /* gate duration (ns) */
    int64_t nsteps;        /* global number of time steps */
    int M;                 /* number of windows */
    double mu;             /* penalty weight; <= 0 selects 2/E */
    const double* target;  /* N*E complex column-major, or NULL for QFT_E on essentials */
} oracle_problem;

/* ------------------------------------------------------------------ small helpers */

static int ipow_i(int b, int e) { int r = 1; while (e-- > 0) r *= b; return r; }

static void dims(const oracle_problem* p, int* N, int* E, int* d) {
    int nfs = 0;
    for (int k = 0; k < p->q; ++k) nfs += p->nf[k];
    *N = ipow_i(p->L, p->q);
    *E = ipow_i(p->ness, p->q);
    *d = 2 * p->d1 * nfs;
}

int oracle_dims(const oracle_problem* p, int* N, int* E, int* d) {
    if (!p || p->q < 1 || p->L < 2 || p->ness < 1 || p->ness > p->L || p->d1 < 3 ||
        p->nsteps < 1 || p->M < 1 || p->M > p->nsteps || !(p->T > 0))
        return -1;
    dims(p, N, E, d);
    return 0;
}

static double penalty_weight(const oracle_problem* p) {
    int N, E, d;
    dims(p, &N, &E, &d);
    return p->mu > 0 ? p->mu : 2.0 / E;
}

/* digit of subsystem k (0 = most significant) in the full index i */
static int level_of(const oracle_problem* p, int i, int k) {
    return (i / ipow_i(p->L, p->q - 1 - k)) % p->L;
}

/* first step of window m (1-based); window m covers [wstart(m), wstart(m+1)) */
static int64_t wstart(const oracle_problem* p, int m) {
    return (int64_t)(((__int128)(m - 1) * p->nsteps) / p->M);
}

void oracle_window_range(const oracle_problem* p, int m, int64_t* n0, int64_t* n1) {
    *n0 = wstart(p, m);
    *n1 = wstart(p, m + 1);
}

/* C = A * B for n x n column-major complex matrices */
static void matmul(int n, const cplx* A, const cplx* B, cplx* C) {
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            cplx s = 0;
            for (int l = 0; l < n; ++l) s += A[i + (size_t)l * n] * B[l + (size_t)j * n];
            C[i + (size_t)j * n] = s;
        }
}

static void adjoint(int n, const cplx* A, cplx* Ah) {
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) Ah[j + (size_t)i * n] = conj(A[i + (size_t)j * n]);
}

/* ------------------------------------------------------------------ model (Sec. 2) */

/* dense lowering matrix of subsystem k: <l-1| a |l> = sqrt(l), identity elsewhere */
static void build_lowering(const oracle_problem* p, int k, cplx* A) {
    int N = ipow_i(p->L, p->q);
    int s = ipow_i(p->L, p->q - 1 - k);
    memset(A, 0, sizeof(cplx) * (size_t)N * N);
    for (int j = 0; j < N; ++j) {
        int l = level_of(p, j, k);
        if (l > 0) A[(j - s) + (size_t)j * N] = sqrt((double)l);
    }
}

/* system Hamiltonian: sum_k -xi_k/2 a_k^+ a_k^+ a_k a_k - sum_{k<l} xi_kl a_k^+a_k a_l^+a_l
 * (+ the paper's sum_k detune_k a_k^+ a_k + sum_{k<l} J_kl (a_l^+ a_k + a_l a_k^+)) */
static void build_system_hamiltonian(const oracle_problem* p, cplx* const* A, cplx* Hs) {
    int N = ipow_i(p->L, p->q);
    size_t nn = (size_t)N * N;
    cplx* Ad = malloc(sizeof(cplx) * nn);
    cplx* t1 = malloc(sizeof(cplx) * nn);
    cplx* t2 = malloc(sizeof(cplx) * nn);
    cplx* num = malloc(sizeof(cplx) * nn * p->q);
    memset(Hs, 0, sizeof(cplx) * nn);
    for (int k = 0; k < p->q; ++k) {
        adjoint(N, A[k], Ad);
        matmul(N, Ad, A[k], num + nn * k);            /* number operator a^+ a */
        matmul(N, Ad, Ad, t1);                         /* a^+ a^+ */
        matmul(N, A[k], A[k], t2);                     /* a a */
        cplx* t3 = malloc(sizeof(cplx) * nn);
        matmul(N, t1, t2, t3);                         /* a^+ a^+ a a */
        for (size_t e = 0; e < nn; ++e) Hs[e] += -0.5 * p->xi[k] * t3[e];
        if (p->detune)
            for (size_t e = 0; e < nn; ++e) Hs[e] += p->detune[k] * num[nn * k + e];
        free(t3);
    }
    for (int k = 0; k < p->q; ++k)
        for (int l = k + 1; l < p->q; ++l) {
            double c = p->xi_cross ? p->xi_cross[k * p->q + l] : 0.0;
            if (c != 0.0) {
                matmul(N, num + nn * k, num + nn * l, t1);
                for (size_t e = 0; e < nn; ++e) Hs[e] += -c * t1[e];
            }
            double J = p->jx ? p->jx[k * p->q + l] : 0.0;
            if (J != 0.0) {
                adjoint(N, A[l], Ad);
                matmul(N, Ad, A[k], t1);               /* a_l^+ a_k */
                adjoint(N, A[k], Ad);
                matmul(N, A[l], Ad, t2);               /* a_l a_k^+ */
                for (size_t e = 0; e < nn; ++e) Hs[e] += J * (t1[e] + t2[e]);
            }
        }
    free(Ad); free(t1); free(t2); free(num);
}

/* centred quadratic cardinal B-spline (unit knot spacing, support [-3/2, 3/2]) */
double oracle_bspline(double tau) {
    if (tau < -1.5 || tau > 1.5) return 0.0;
    if (tau < -0.5) return 0.5 * (tau + 1.5) * (tau + 1.5);
    if (tau < 0.5) return 0.75 - tau * tau;
    return 0.5 * (tau - 1.5) * (tau - 1.5);
}

/* value of basis function s (0-based) at time t: centre (s - 1/2) dtau, dtau = T/(d1-2) */
static double basis(const oracle_problem* p, int s, double t) {
    double dtau = p->T / (p->d1 - 2);
    return oracle_bspline((t - (s - 0.5) * dtau) / dtau);
}

/* d_k(t) = sum_f exp(i Omega_kf t) sum_s (alpha1 + i alpha2)_kfs B_s(t)  (Eq. dj-ctrl) */
void oracle_controls(const oracle_problem* p, const double* alpha, double t, double* d_out) {
    int off = 0;
    for (int k = 0; k < p->q; ++k) {
        cplx dk = 0;
        for (int f = 0; f < p->nf[k]; ++f) {
            cplx env = 0;
            const double* a = alpha + (size_t)2 * p->d1 * (off + f);
            for (int s = 0; s < p->d1; ++s) env += (a[2 * s] + I * a[2 * s + 1]) * basis(p, s, t);
            dk += cexp(I * p->omega[off + f] * t) * env;
        }
        d_out[2 * k] = creal(dk);
        d_out[2 * k + 1] = cimag(dk);
        off += p->nf[k];
    }
}

/* H(t) = Hs + sum_k d_k A_k + conj(d_k) A_k^+   (Eq. ctrl-ham) */
static void build_hamiltonian(const oracle_problem* p, const cplx* Hs, cplx* const* A,
                              const double* alpha, double t, cplx* H) {
    int N = ipow_i(p->L, p->q);
    size_t nn = (size_t)N * N;
    double* dk = malloc(sizeof(double) * 2 * p->q);
    oracle_controls(p, alpha, t, dk);
    memcpy(H, Hs, sizeof(cplx) * nn);
    for (int k = 0; k < p->q; ++k) {
        cplx d = dk[2 * k] + I * dk[2 * k + 1];
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                H[i + (size_t)j * N] += d * A[k][i + (size_t)j * N] + conj(d) * conj(A[k][j + (size_t)i * N]);
            }
    }
    free(dk);
}

/* target: QFT_E on the essential subspace, {V}_{jk} = kappa^{jk}/sqrt(E), kappa = e^{2 pi i/E}
 * (Sec. 5), rows of guard states zero; or the user's N x E matrix */
static void build_target(const oracle_problem* p, cplx* V) {
    int N, E, d;
    dims(p, &N, &E, &d);
    if (p->target) {
        for (int e = 0; e < N * E; ++e) V[e] = p->target[2 * e] + I * p->target[2 * e + 1];
        return;
    }
    memset(V, 0, sizeof(cplx) * (size_t)N * E);
    for (int j = 0; j < E; ++j)
        for (int e = 0; e < E; ++e) {
            /* full index of essential state e: its base-ness digits placed in base L */
            int i = 0, r = e;
            for (int k = p->q - 1, w = 1; k >= 0; --k, w *= p->L) { i += (r % p->ness) * w; r /= p->ness; }
            double ang = 2.0 * M_PI * (double)(((int64_t)e * j) % E) / E;
            V[i + (size_t)j * N] = cexp(I * ang) / sqrt((double)E);
        }
}

/* W^0: identity embedding of the essential subspace (Eq. sch-ic) */
static void build_identity_state(const oracle_problem* p, cplx* W0) {
    int N, E, d;
    dims(p, &N, &E, &d);
    memset(W0, 0, sizeof(cplx) * (size_t)N * E);
    for (int e = 0; e < E; ++e) {
        int i = 0, r = e;
        for (int k = p->q - 1, w = 1; k >= 0; --k, w *= p->L) { i += (r % p->ness) * w; r /= p->ness; }
        W0[i + (size_t)e * N] = 1.0;
    }
}

/* ------------------------------------------------------------------ dense LU */

/* in-place LU with partial pivoting, column-major; returns 0 or -1 on a zero pivot */
static int lu_factor(int n, cplx* A, int* piv) {
    for (int c = 0; c < n; ++c) {
        int pr = c;
        double best = cabs(A[c + (size_t)c * n]);
        for (int r = c + 1; r < n; ++r) {
            double v = cabs(A[r + (size_t)c * n]);
            if (v > best) { best = v; pr = r; }
        }
        piv[c] = pr;
        if (best == 0.0) return -1;
        if (pr != c)
            for (int j = 0; j < n; ++j) {
                cplx t = A[c + (size_t)j * n];
                A[c + (size_t)j * n] = A[pr + (size_t)j * n];
                A[pr + (size_t)j * n] = t;
            }
        cplx inv = 1.0 / A[c + (size_t)c * n];
        for (int r = c + 1; r < n; ++r) A[r + (size_t)c * n] *= inv;
        for (int j = c + 1; j < n; ++j) {
            cplx f = A[c + (size_t)j * n];
            if (f != 0)
                for (int r = c + 1; r < n; ++r) A[r + (size_t)j * n] -= A[r + (size_t)c * n] * f;
        }
    }
    return 0;
}

/* solve (LU) X = B for ncols right-hand sides stored column-major with leading dim n */
static void lu_solve(int n, const cplx* LU, const int* piv, cplx* B, int ncols) {
    for (int j = 0; j < ncols; ++j) {
        cplx* b = B + (size_t)j * n;
        for (int c = 0; c < n; ++c)
            if (piv[c] != c) { cplx t = b[c]; b[c] = b[piv[c]]; b[piv[c]] = t; }
        for (int c = 0; c < n; ++c)
            for (int r = c + 1; r < n; ++r) b[r] -= LU[r + (size_t)c * n] * b[c];
        for (int c = n - 1; c >= 0; --c) {
            b[c] /= LU[c + (size_t)c * n];
            for (int r = 0; r < c; ++r) b[r] -= LU[r + (size_t)c * n] * b[c];
        }
    }
}

/* Y = X (n x n) * Z (n x ncols) */
static void matmat(int n, const cplx* X, const cplx* Z, int ncols, cplx* Y) {
    for (int j = 0; j < ncols; ++j)
        for (int i = 0; i < n; ++i) {
            cplx s = 0;
            for (int l = 0; l < n; ++l) s += X[i + (size_t)l * n] * Z[l + (size_t)j * n];
            Y[i + (size_t)j * n] = s;
        }
}

/* ------------------------------------------------------------------ shared model state */

typedef struct {
    const oracle_problem* p;
    int N, E, d;
    double h, mu;
    cplx** A;   /* q dense lowering matrices */
    cplx* Hs;   /* dense drift */
    cplx* V;    /* target N x E */
} model;

static int model_init(model* m, const oracle_problem* p) {
    if (oracle_dims(p, &m->N, &m->E, &m->d)) return -1;
    m->p = p;
    m->h = p->T / (double)p->nsteps;
    m->mu = penalty_weight(p);
    size_t nn = (size_t)m->N * m->N;
    m->A = malloc(sizeof(cplx*) * p->q);
    for (int k = 0; k < p->q; ++k) { m->A[k] = malloc(sizeof(cplx) * nn); build_lowering(p, k, m->A[k]); }
    m->Hs = malloc(sizeof(cplx) * nn);
    build_system_hamiltonian(p, m->A, m->Hs);
    m->V = malloc(sizeof(cplx) * (size_t)m->N * m->E);
    build_target(p, m->V);
    return 0;
}

static void model_free(model* m) {
    for (int k = 0; k < m->p->q; ++k) free(m->A[k]);
    free(m->A); free(m->Hs); free(m->V);
}

/* A = I + i(h/2)H and B = I - i(h/2)H at t_{n+1/2} = (n + 1/2) h */
static void step_matrices(const model* m, const double* alpha, int64_t n, cplx* H, cplx* Am, cplx* Bm) {
    int N = m->N;
    double t = ((double)n + 0.5) * m->h;
    build_hamiltonian(m->p, m->Hs, m->A, alpha, t, H);
    for (size_t e = 0; e < (size_t)N * N; ++e) {
        Am[e] = I * (0.5 * m->h) * H[e];
        Bm[e] = -Am[e];
    }
    for (int i = 0; i < N; ++i) { Am[i + (size_t)i * N] += 1.0; Bm[i + (size_t)i * N] += 1.0; }
}

/* one implicit-midpoint step: A U_{n+1} = B U_n (U is N x ncols), in place */
static int imr_forward_step(const model* m, const double* alpha, int64_t n, cplx* U, int ncols,
                            cplx* H, cplx* Am, cplx* Bm, cplx* tmp, int* piv) {
    step_matrices(m, alpha, n, H, Am, Bm);
    matmat(m->N, Bm, U, ncols, tmp);
    if (lu_factor(m->N, Am, piv)) return -1;
    lu_solve(m->N, Am, piv, tmp, ncols);
    memcpy(U, tmp, sizeof(cplx) * (size_t)m->N * ncols);
    return 0;
}

/* one discrete-adjoint step: B Lambda_n = A Lambda_{n+1}, in place */
static int imr_adjoint_step(const model* m, const double* alpha, int64_t n, cplx* Lam, int ncols,
                            cplx* H, cplx* Am, cplx* Bm, cplx* tmp, int* piv) {
    step_matrices(m, alpha, n, H, Am, Bm);
    matmat(m->N, Am, Lam, ncols, tmp);
    if (lu_factor(m->N, Bm, piv)) return -1;
    lu_solve(m->N, Bm, piv, tmp, ncols);
    memcpy(Lam, tmp, sizeof(cplx) * (size_t)m->N * ncols);
    return 0;
}

/* <X, Y>_F = sum conj(X) Y over n entries */
static cplx frob(const cplx* X, const cplx* Y, size_t n) {
    cplx s = 0;
    for (size_t e = 0; e < n; ++e) s += conj(X[e]) * Y[e];
    return s;
}

/* generalized infidelity J(U) = ||U||^2/E - |<V,U>|^2/E^2  (Eq. mod-infid with n := E) */
static double infidelity(const model* m, const cplx* U, cplx* gamma_out) {
    size_t ne = (size_t)m->N * m->E;
    double nrm2 = creal(frob(U, U, ne));
    cplx g = frob(m->V, U, ne);
    if (gamma_out) *gamma_out = g;
    double E = m->E;
    return nrm2 / E - (creal(g) * creal(g) + cimag(g) * cimag(g)) / (E * E);
}

/* ------------------------------------------------------------------ public pieces */

static void load_cplx(cplx* dst, const double* src, size_t n) {
    for (size_t e = 0; e < n; ++e) dst[e] = src[2 * e] + I * src[2 * e + 1];
}
static void store_cplx(double* dst, const cplx* src, size_t n) {
    for (size_t e = 0; e < n; ++e) { dst[2 * e] = creal(src[e]); dst[2 * e + 1] = cimag(src[e]); }
}

int oracle_system_hamiltonian(const oracle_problem* p, double* Hs_out) {
    model m;
    if (model_init(&m, p)) return -1;
    store_cplx(Hs_out, m.Hs, (size_t)m.N * m.N);
    model_free(&m);
    return 0;
}

int oracle_hamiltonian(const oracle_problem* p, const double* alpha, double t, double* H_out) {
    model m;
    if (model_init(&m, p)) return -1;
    cplx* H = malloc(sizeof(cplx) * (size_t)m.N * m.N);
    build_hamiltonian(p, m.Hs, m.A, alpha, t, H);
    store_cplx(H_out, H, (size_t)m.N * m.N);
    free(H);
    model_free(&m);
    return 0;
}

int oracle_lowering(const oracle_problem* p, int k, double* A_out) {
    model m;
    if (model_init(&m, p) || k < 0 || k >= p->q) return -1;
    store_cplx(A_out, m.A[k], (size_t)m.N * m.N);
    model_free(&m);
    return 0;
}

int oracle_target(const oracle_problem* p, double* V_out) {
    model m;
    if (model_init(&m, p)) return -1;
    store_cplx(V_out, m.V, (size_t)m.N * m.E);
    model_free(&m);
    return 0;
}

int oracle_identity_state(const oracle_problem* p, double* W0_out) {
    int N, E, d;
    if (oracle_dims(p, &N, &E, &d)) return -1;
    cplx* W0 = malloc(sizeof(cplx) * (size_t)N * E);
    build_identity_state(p, W0);
    store_cplx(W0_out, W0, (size_t)N * E);
    free(W0);
    return 0;
}

double oracle_infidelity(const oracle_problem* p, const double* U_in) {
    model m;
    if (model_init(&m, p)) return NAN;
    cplx* U = malloc(sizeof(cplx) * (size_t)m.N * m.E);
    load_cplx(U, U_in, (size_t)m.N * m.E);
    double J = infidelity(&m, U, NULL);
    free(U);
    model_free(&m);
    return J;
}

/* propagate an N x ncols state from global step n0 to n1 (n0 <= n1) with the midpoint rule */
int oracle_propagate(const oracle_problem* p, const double* alpha, int64_t n0, int64_t n1,
                     const double* U_in, double* U_out, int ncols) {
    model m;
    if (model_init(&m, p) || n0 < 0 || n1 < n0 || n1 > p->nsteps || ncols < 1) return -1;
    size_t nn = (size_t)m.N * m.N, nc = (size_t)m.N * ncols;
    cplx *H = malloc(sizeof(cplx) * nn), *Am = malloc(sizeof(cplx) * nn), *Bm = malloc(sizeof(cplx) * nn);
    cplx *U = malloc(sizeof(cplx) * nc), *tmp = malloc(sizeof(cplx) * nc);
    int* piv = malloc(sizeof(int) * m.N);
    int rc = 0;
    load_cplx(U, U_in, nc);
    for (int64_t n = n0; n < n1 && !rc; ++n) rc = imr_forward_step(&m, alpha, n, U, ncols, H, Am, Bm, tmp, piv);
    store_cplx(U_out, U, nc);
    free(H); free(Am); free(Bm); free(U); free(tmp); free(piv);
    model_free(&m);
    return rc;
}

/* discrete adjoint propagation from step n1 back to n0 */
int oracle_propagate_adjoint(const oracle_problem* p, const double* alpha, int64_t n0, int64_t n1,
                             const double* L_in, double* L_out, int ncols) {
    model m;
    if (model_init(&m, p) || n0 < 0 || n1 < n0 || n1 > p->nsteps || ncols < 1) return -1;
    size_t nn = (size_t)m.N * m.N, nc = (size_t)m.N * ncols;
    cplx *H = malloc(sizeof(cplx) * nn), *Am = malloc(sizeof(cplx) * nn), *Bm = malloc(sizeof(cplx) * nn);
    cplx *Lm = malloc(sizeof(cplx) * nc), *tmp = malloc(sizeof(cplx) * nc);
    int* piv = malloc(sizeof(int) * m.N);
    int rc = 0;
    load_cplx(Lm, L_in, nc);
    for (int64_t n = n1 - 1; n >= n0 && !rc; --n) rc = imr_adjoint_step(&m, alpha, n, Lm, ncols, H, Am, Bm, tmp, piv);
    store_cplx(L_out, Lm, nc);
    free(H); free(Am); free(Bm); free(Lm); free(tmp); free(piv);
    model_free(&m);
    return rc;
}

/* roll-out (Sec. 5): W^m = U(t_m) of the single-shooting solution from W^0, m = 1..M-1 */
int oracle_rollout(const oracle_problem* p, const double* alpha, double* W_out) {
    model m;
    if (model_init(&m, p)) return -1;
    size_t nn = (size_t)m.N * m.N, ne = (size_t)m.N * m.E;
    cplx *H = malloc(sizeof(cplx) * nn), *Am = malloc(sizeof(cplx) * nn), *Bm = malloc(sizeof(cplx) * nn);
    cplx *U = malloc(sizeof(cplx) * ne), *tmp = malloc(sizeof(cplx) * ne);
    int* piv = malloc(sizeof(int) * m.N);
    int rc = 0;
    build_identity_state(p, U);
    for (int w = 1; w < p->M && !rc; ++w) {
        for (int64_t n = wstart(p, w); n < wstart(p, w + 1) && !rc; ++n)
            rc = imr_forward_step(&m, alpha, n, U, m.E, H, Am, Bm, tmp, piv);
        store_cplx(W_out + 2 * ne * (w - 1), U, ne);
    }
    free(H); free(Am); free(Bm); free(U); free(tmp); free(piv);
    model_free(&m);
    return rc;
}

/* Regularization of the optimisation problem (Sec. 5): a Tikhonov term (gamma_tik/2)||alpha||^2
 * on the control vector plus gamma_energy times the time-averaged control-pulse energy
 * (1/T) int_0^T sum_k |d_k(t)|^2 dt.  The integral is the midpoint rule on the time grid (the
 * quadrature of the gradient integral, Eq. grad-int), so h/T = 1/nsteps weights each step.  The
 * gradient differentiates each term literally: with
 * d_k = sum_f exp(i Omega_kf t) sum_s (alpha1 + i alpha2)_kfs B_s(t),
 *   d|d_k|^2 / d alpha1_kfs = 2 Re(conj(d_k) exp(i Omega_kf t) B_s(t)),
 *   d|d_k|^2 / d alpha2_kfs = 2 Re(conj(d_k) i exp(i Omega_kf t) B_s(t)).
 * Step sums are accumulated in blocks of BLOCK_REG steps.  grad may be NULL. */
#define BLOCK_REG 256
double oracle_regularization(const oracle_problem* p, const double* alpha, double gamma_tik, double gamma_energy,
                             double* grad) {
    int N, E, d;
    dims(p, &N, &E, &d);
    double h = p->T / (double)p->nsteps;
    double* dk = malloc(sizeof(double) * 2 * p->q);
    double* gblk = calloc((size_t)d, sizeof(double));
    double* gsum = calloc((size_t)d, sizeof(double));
    double energy = 0.0, eblk = 0.0;
    for (int64_t n = 0; n < p->nsteps; ++n) {
        double t = ((double)n + 0.5) * h;
        oracle_controls(p, alpha, t, dk);
        int off = 0;
        for (int k = 0; k < p->q; ++k) {
            cplx dkc = dk[2 * k] + I * dk[2 * k + 1];
            eblk += creal(dkc) * creal(dkc) + cimag(dkc) * cimag(dkc);
            for (int f = 0; f < p->nf[k]; ++f) {
                cplx e = cexp(I * p->omega[off + f] * t);
                for (int s = 0; s < p->d1; ++s) {
                    double B = basis(p, s, t);
                    size_t j = (size_t)2 * ((size_t)(off + f) * p->d1 + s);
                    gblk[j] += 2.0 * creal(conj(dkc) * e * B);
                    gblk[j + 1] += 2.0 * creal(conj(dkc) * I * e * B);
                }
            }
            off += p->nf[k];
        }
        if ((n + 1) % BLOCK_REG == 0 || n + 1 == p->nsteps) {
            energy += eblk;
            eblk = 0.0;
            for (int j = 0; j < d; ++j) { gsum[j] += gblk[j]; gblk[j] = 0.0; }
        }
    }
    double tik = 0.0;
    for (int j = 0; j < d; ++j) tik += alpha[j] * alpha[j];
    double wt = h / p->T;   /* midpoint weight of the time average */
    double R = 0.5 * gamma_tik * tik + gamma_energy * wt * energy;
    if (grad)
        for (int j = 0; j < d; ++j) grad[j] = gamma_tik * alpha[j] + gamma_energy * wt * gsum[j];
    free(dk); free(gblk); free(gsum);
    return R;
}

/* ------------------------------------------------------------------ one window's work */

typedef struct {
    const model* m;
    const double* alpha;
    const double* W;      /* [M-1][E][N] complex interleaved */
    int want_grad;
    int w;                /* window index, 1-based */
    /* outputs */
    double term;          /* pen_m (m < M) or J (m = M) */
    cplx* Uend;           /* U^m(t_m), N x E */
    cplx* Lam0;           /* Lambda^m(t_{m-1}), N x E */
    double* galpha;       /* this window's contribution to dP/dalpha, [d] */
    int rc;
} window_job;

#define BLOCK_STEPS 256

static void run_window(window_job* job) {
    const model* m = job->m;
    const oracle_problem* p = m->p;
    int N = m->N, E = m->E, w = job->w;
    size_t nn = (size_t)N * N, ne = (size_t)N * E;
    int64_t n0 = wstart(p, w), n1 = wstart(p, w + 1), ns = n1 - n0;
    cplx *H = malloc(sizeof(cplx) * nn), *Am = malloc(sizeof(cplx) * nn), *Bm = malloc(sizeof(cplx) * nn);
    cplx* tmp = malloc(sizeof(cplx) * ne);
    int* piv = malloc(sizeof(int) * N);
    /* all states of the window, U_{n0} .. U_{n1} (kept for the adjoint sweep) */
    cplx* Us = malloc(sizeof(cplx) * ne * (size_t)(job->want_grad ? ns + 1 : 1));
    cplx* U = Us;
    job->rc = 0;

    /* initial condition W^{w-1}, W^0 = identity embedding (Eq. sch-ic) */
    if (w == 1) build_identity_state(p, U);
    else load_cplx(U, job->W + 2 * ne * (w - 2), ne);

    /* forward sweep */
    for (int64_t j = 0; j < ns && !job->rc; ++j) {
        cplx* next = job->want_grad ? Us + ne * (j + 1) : Us;
        if (job->want_grad) memcpy(next, Us + ne * j, sizeof(cplx) * ne);
        job->rc = imr_forward_step(m, job->alpha, n0 + j, next, E, H, Am, Bm, tmp, piv);
    }
    cplx* Ufin = job->want_grad ? Us + ne * ns : Us;
    memcpy(job->Uend, Ufin, sizeof(cplx) * ne);

    /* terminal term and adjoint terminal condition (Eqs. penalty-fcn, terminal) */
    cplx* Lam = malloc(sizeof(cplx) * ne);
    if (w < p->M) {
        cplx* Wm = malloc(sizeof(cplx) * ne);
        load_cplx(Wm, job->W + 2 * ne * (w - 1), ne);
        double s = 0;
        for (size_t e = 0; e < ne; ++e) {
            cplx c = Ufin[e] - Wm[e];
            s += creal(c) * creal(c) + cimag(c) * cimag(c);
            Lam[e] = 0.5 * m->mu * (Wm[e] - Ufin[e]);
        }
        job->term = 0.5 * m->mu * s;
        free(Wm);
    } else {
        cplx g;
        job->term = infidelity(m, Ufin, &g);
        for (size_t e = 0; e < ne; ++e) Lam[e] = (g * m->V[e] - (double)E * Ufin[e]) / ((double)E * E);
    }

    if (job->want_grad && !job->rc) {
        /* backward sweep with the gradient quadrature (Eq. grad-int at the midpoints) */
        cplx* Lprev = malloc(sizeof(cplx) * ne);
        cplx* Lbar = malloc(sizeof(cplx) * ne);
        cplx* Ubar = malloc(sizeof(cplx) * ne);
        cplx* AU = malloc(sizeof(cplx) * ne);
        cplx* AdU = malloc(sizeof(cplx) * ne);
        cplx* Ad = malloc(sizeof(cplx) * nn);
        double* blk = calloc((size_t)m->d, sizeof(double));
        memset(job->galpha, 0, sizeof(double) * m->d);
        for (int64_t j = ns - 1; j >= 0 && !job->rc; --j) {
            int64_t n = n0 + j;
            double t = ((double)n + 0.5) * m->h;
            memcpy(Lprev, Lam, sizeof(cplx) * ne);              /* Lambda_{n+1} */
            job->rc = imr_adjoint_step(m, job->alpha, n, Lam, E, H, Am, Bm, tmp, piv);  /* Lambda_n */
            for (size_t e = 0; e < ne; ++e) {
                Lbar[e] = 0.5 * (Lam[e] + Lprev[e]);
                Ubar[e] = 0.5 * (Us[ne * j + e] + Us[ne * (j + 1) + e]);
            }
            /* dH/dalpha1_kfs = B_s(t)(e^{i W t} A_k + e^{-i W t} A_k^+),
             * dH/dalpha2_kfs = B_s(t)(i e^{i W t} A_k - i e^{-i W t} A_k^+) */
            int off = 0;
            for (int k = 0; k < p->q; ++k) {
                adjoint(N, m->A[k], Ad);
                matmat(N, m->A[k], Ubar, E, AU);
                matmat(N, Ad, Ubar, E, AdU);
                cplx z = frob(Lbar, AU, ne), y = frob(Lbar, AdU, ne);
                for (int f = 0; f < p->nf[k]; ++f) {
                    cplx ph = cexp(I * p->omega[off + f] * t);
                    cplx g1 = I * (ph * z + conj(ph) * y);              /* <Lbar, i dH/da1 Ubar> / B_s */
                    cplx g2 = I * (I * ph * z - I * conj(ph) * y);      /* <Lbar, i dH/da2 Ubar> / B_s */
                    double* b = blk + (size_t)2 * p->d1 * (off + f);
                    for (int s = 0; s < p->d1; ++s) {
                        double Bs = basis(p, s, t);
                        b[2 * s] += 2.0 * m->h * Bs * creal(g1);
                        b[2 * s + 1] += 2.0 * m->h * Bs * creal(g2);
                    }
                }
                off += p->nf[k];
            }
            if ((ns - 1 - j) % BLOCK_STEPS == BLOCK_STEPS - 1 || j == 0) {
                for (int l = 0; l < m->d; ++l) { job->galpha[l] += blk[l]; blk[l] = 0; }
            }
        }
        memcpy(job->Lam0, Lam, sizeof(cplx) * ne);
        free(Lprev); free(Lbar); free(Ubar); free(AU); free(AdU); free(Ad); free(blk);
    }
    free(Lam); free(H); free(Am); free(Bm); free(tmp); free(piv); free(Us);
}

typedef struct {
    window_job* jobs;
    int njobs;
    int next;
    pthread_mutex_t lock;
} job_pool;

static void* worker(void* arg) {
    job_pool* pool = arg;
    for (;;) {
        pthread_mutex_lock(&pool->lock);
        int j = pool->next++;
        pthread_mutex_unlock(&pool->lock);
        if (j >= pool->njobs) return NULL;
        run_window(&pool->jobs[j]);
    }
}

/*
 * Evaluate P (and optionally its gradient) for windows [wlo, whi] (1-based, inclusive).
 * Full evaluation: wlo = 1, whi = M.  Outputs (any may be NULL):
 *   P_out: J + sum pen over the evaluated windows; J_out: J if window M was evaluated;
 *   pen_out[M-1]: pen_m of evaluated windows m < M; grad_alpha[d]: sum of the evaluated
 *   windows' contributions; grad_W[(M-1)*E*N*2]: for m with both m and m+1 evaluated;
 *   Uend_out[M][E][N] and Lam0_out[M][E][N]: per-window final state and initial adjoint.
 */
int oracle_eval_windows(const oracle_problem* p, const double* alpha, const double* W,
                        int wlo, int whi, int nthreads,
                        double* P_out, double* J_out, double* pen_out,
                        double* grad_alpha, double* grad_W, double* Uend_out, double* Lam0_out) {
    model m;
    if (model_init(&m, p)) return -1;
    if (wlo < 1 || whi > p->M || wlo > whi) { model_free(&m); return -1; }
    int want_grad = grad_alpha || grad_W || Lam0_out;
    int nj = whi - wlo + 1;
    size_t ne = (size_t)m.N * m.E;
    window_job* jobs = calloc(nj, sizeof(window_job));
    for (int j = 0; j < nj; ++j) {
        jobs[j].m = &m; jobs[j].alpha = alpha; jobs[j].W = W; jobs[j].want_grad = want_grad;
        jobs[j].w = wlo + j;
        jobs[j].Uend = malloc(sizeof(cplx) * ne);
        jobs[j].Lam0 = calloc(ne, sizeof(cplx));
        jobs[j].galpha = calloc((size_t)m.d, sizeof(double));
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nj) nthreads = nj;
    job_pool pool = {jobs, nj, 0, PTHREAD_MUTEX_INITIALIZER};
    pthread_t* th = malloc(sizeof(pthread_t) * nthreads);
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, worker, &pool);
    worker(&pool);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);

    int rc = 0;
    double P = 0;
    for (int j = 0; j < nj; ++j) {
        if (jobs[j].rc) rc = -2;
        P += jobs[j].term;
        if (jobs[j].w < p->M) { if (pen_out) pen_out[jobs[j].w - 1] = jobs[j].term; }
        else if (J_out) *J_out = jobs[j].term;
        if (Uend_out) store_cplx(Uend_out + 2 * ne * (jobs[j].w - 1), jobs[j].Uend, ne);
        if (Lam0_out) store_cplx(Lam0_out + 2 * ne * (jobs[j].w - 1), jobs[j].Lam0, ne);
    }
    if (P_out) *P_out = P;
    if (grad_alpha) {
        memset(grad_alpha, 0, sizeof(double) * m.d);
        for (int j = 0; j < nj; ++j)
            for (int l = 0; l < m.d; ++l) grad_alpha[l] += jobs[j].galpha[l];
    }
    if (grad_W) {
        /* dP/dW^w = mu (W^w - U^w(t_w)) - 2 Lambda^{w+1}(t_w), real and imaginary parts */
        for (int j = 0; j + 1 < nj; ++j) {
            int w = jobs[j].w;
            const double* Ww = W + 2 * ne * (w - 1);
            double* g = grad_W + 2 * ne * (w - 1);
            for (size_t e = 0; e < ne; ++e) {
                cplx Wv = Ww[2 * e] + I * Ww[2 * e + 1];
                cplx gv = m.mu * (Wv - jobs[j].Uend[e]) - 2.0 * jobs[j + 1].Lam0[e];
                g[2 * e] = creal(gv);
                g[2 * e + 1] = cimag(gv);
            }
        }
    }
    for (int j = 0; j < nj; ++j) { free(jobs[j].Uend); free(jobs[j].Lam0); free(jobs[j].galpha); }
    free(jobs);
    model_free(&m);
    return rc;
}

int oracle_eval(const oracle_problem* p, const double* alpha, const double* W, int nthreads,
                double* P_out, double* J_out, double* pen_out, double* grad_alpha, double* grad_W) {
    return oracle_eval_windows(p, alpha, W, 1, p->M, nthreads, P_out, J_out, pen_out,
                               grad_alpha, grad_W, NULL, NULL);
}
