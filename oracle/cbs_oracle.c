/*
 * cbs_oracle.c -- plain FP64 CPU oracle for the split-preconditioned Born
 * iteration on the first-order (particle velocity, pressure) Helmholtz system
 * with heterogeneous sound speed, density and absorption.
 *
 * Source of every formula: A. Stanziola, S. R. Arridge, B. E. Treeby,
 * B. T. Cox, "Iterative Born solver for the acoustic Helmholtz equation with
 * heterogeneous sound speed and density" (arXiv 2507.16087).  Citations below
 * name the paper's section, equation, algorithm or appendix.
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously-correct reference the
 * GPU library is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header, table or
 * helper with the CUDA library, and the CUDA library never loads it.
 *
 * Everything is double precision and complex<double> (C99 _Complex).  No
 * blocking, fusion or reordering beyond what the formulas state: each step is
 * the paper's formula written out per voxel / per wavenumber.  Its own FFT is a
 * textbook recursive decimation-in-time transform (smallest prime factor
 * first, naive DFT for a prime length); OpenMP only splits independent lines.
 *
 * Array layout: a grid of D dims has n[0] (x, fastest) .. n[D-1]; a field has C
 * = D+1 components ordered (u_x, u_y, [u_z], p), each a contiguous block of
 * N = prod(n) complex values.  Velocity component eta lives at the staggered
 * points x + (dx/2) e_eta (App. B.1).
 *
 * Readings where the paper is silent or garbled (all shared with the GPU path
 * by statement, never by code):
 *  - absorbing layer gamma: quadratic profile inside the grid, depth
 *    min(1, max(0, (n_lo - xi)/n_lo, (xi - (N-1-n_hi))/n_hi)), summed over axes;
 *    staggered values evaluated at xi + 1/2 (Sec. 2.1 names gamma but gives no
 *    profile; App. B.1 says gamma is evaluated analytically at staggered points).
 *  - shifts a1, a2: midrange (bounding-box centre) of the diagonal values by
 *    default; componentwise median is the Algorithm 1 example (rule 1); the
 *    centre of the minimum enclosing circle, recommended in Sec. 4 (rule 2).
 *  - lambda_j = max|diag_j - a_j| / beta (eq. C); if that max is 0, lambda_j =
 *    |a_j| (and setup fails if a_j is 0 too).
 *  - pressure row divided by rho c^2 with the complex c^2 of eq. 118 (eq.
 *    HH1stOrderSH); velocity row multiplied by the staggered density.
 *  - adjoint: per-wavenumber conjugate transpose of the staggered (L+I)^-1
 *    symbol, conj(B) in place of B (App. B's elementwise-conjugate shortcut
 *    assumes a symmetric symbol, which the staggered one is not).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

#define ORC_MAXD 3
#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------- */
/* FFT (own implementation)                                                   */
/* ------------------------------------------------------------------------- */

static long smallest_factor(long n)
{
    for (long p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* Recursive decimation in time.  x: input with stride `stride`, X: n outputs.
 * tw: table of N roots exp(sign*2*pi*i*j/N) of the top-level length N; a
 * sub-transform of length n uses root index (e * N/n) mod N.  scratch: >= n. */
static void fft_rec(const cplx* x, long stride, cplx* X, long n, long N, const cplx* tw, cplx* scratch)
{
    if (n == 1) { X[0] = x[0]; return; }
    const long step = N / n; /* root of unity w_n = tw[step] */
    long p = smallest_factor(n);
    if (p == n) { /* prime length: the DFT sum itself */
        for (long k = 0; k < n; ++k) {
            cplx acc = 0;
            for (long j = 0; j < n; ++j) acc += x[j * stride] * tw[((j * k) % n) * step];
            X[k] = acc;
        }
        return;
    }
    long m = n / p;
    /* X_k = sum_q w_n^{q k} Y_q[k mod m],  Y_q = DFT_m of x[q + p j] */
    for (long q = 0; q < p; ++q) fft_rec(x + q * stride, stride * p, X + q * m, m, N, tw, scratch);
    memcpy(scratch, X, (size_t)n * sizeof(cplx));
    for (long k = 0; k < n; ++k) {
        cplx acc = 0;
        for (long q = 0; q < p; ++q) acc += tw[((q * k) % n) * step] * scratch[q * m + (k % m)];
        X[k] = acc;
    }
}

static void make_roots(long N, int sign, cplx* tw)
{
    for (long j = 0; j < N; ++j) {
        double ang = sign * 2.0 * ORC_PI * (double)j / (double)N;
        tw[j] = cos(ang) + I * sin(ang);
    }
}

/* 1-D DFT of length n of a strided array, in place.  sign=-1: forward
 * (sum x_j e^{-2 pi i jk/n}); sign=+1: inverse without the 1/n factor. */
void orc_fft1d(cplx* data, long n, long stride, int sign)
{
    cplx* tw = malloc(sizeof(cplx) * n);
    cplx* in = malloc(sizeof(cplx) * n);
    cplx* out = malloc(sizeof(cplx) * n);
    cplx* scr = malloc(sizeof(cplx) * n);
    make_roots(n, sign, tw);
    for (long j = 0; j < n; ++j) in[j] = data[j * stride];
    fft_rec(in, 1, out, n, n, tw, scr);
    for (long j = 0; j < n; ++j) data[j * stride] = out[j];
    free(tw); free(in); free(out); free(scr);
}

/* D-dim DFT of one component block (N = prod n values), axis by axis.
 * sign=-1 forward; sign=+1 inverse including the 1/N factor. */
void orc_fftn(cplx* data, int ndim, const int64_t* n, int sign)
{
    long total = 1;
    for (int a = 0; a < ndim; ++a) total *= (long)n[a];
    long stride = 1;
    for (int a = 0; a < ndim; ++a) {
        long len = (long)n[a];
        long nlines = total / len;
        cplx* tw = malloc(sizeof(cplx) * len);
        make_roots(len, sign, tw);
        #pragma omp parallel
        {
            cplx* in = malloc(sizeof(cplx) * len);
            cplx* out = malloc(sizeof(cplx) * len);
            cplx* scr = malloc(sizeof(cplx) * len);
            #pragma omp for schedule(static)
            for (long l = 0; l < nlines; ++l) {
                /* line l: the index with axis a removed, split into below/above */
                long lo = l % stride, hi = l / stride;
                long base = lo + hi * stride * len;
                for (long j = 0; j < len; ++j) in[j] = data[base + j * stride];
                fft_rec(in, 1, out, len, len, tw, scr);
                for (long j = 0; j < len; ++j) data[base + j * stride] = out[j];
            }
            free(in); free(out); free(scr);
        }
        free(tw);
        stride *= len;
    }
    if (sign > 0) {
        double s = 1.0 / (double)total;
        for (long i = 0; i < total; ++i) data[i] *= s;
    }
}

/* ------------------------------------------------------------------------- */
/* Problem set-up (Sec. 2.1, 2.3.1, Algorithm 1 preprocessing, App. B.1)       */
/* ------------------------------------------------------------------------- */

typedef struct orc_problem {
    int ndim, ncomp;
    int64_t n[ORC_MAXD];
    long N;
    double dx, omega;
    int adjoint_ready;
    cplx a1, a2;        /* shifts, eq. LV */
    double lam1, lam2;  /* scaling, eq. C */
    double maxdev1, maxdev2;
    cplx* v;            /* [C][N] scaled potential V = C^-1/2 (diag - a) C^-1/2 */
    cplx* rho_stag;     /* [D][N] staggered density (App. B.1 linear interpolation) */
    cplx* inv_rho_c2;   /* [N] 1/(rho c^2), complex c^2 of eq. 118 */
    double* k;          /* [D][nmax] continuous wavenumbers 2 pi fftfreq(n, dx) */
    int64_t kstride;
    int collocated;     /* 1: velocity at the cell centres (App. B), 0: staggered (App. B.1) */
} orc_problem;

/* depth of the absorbing layer at continuous cell coordinate xi (reading of
 * the unspecified profile; see header) */
static double layer_depth(double xi, long N, int n_lo, int n_hi)
{
    double d = 0.0;
    if (n_lo > 0) {
        double t = ((double)n_lo - xi) / (double)n_lo;
        if (t > d) d = t;
    }
    if (n_hi > 0) {
        double t = (xi - (double)(N - 1 - n_hi)) / (double)n_hi;
        if (t > d) d = t;
    }
    return d > 1.0 ? 1.0 : d;
}

static double layer_axis(double xi, long N, const int* nabs2, double gamma_max, double power)
{
    double d = layer_depth(xi, N, nabs2[0], nabs2[1]);
    return d > 0.0 ? gamma_max * pow(d, power) : 0.0;
}

static void unravel(long i, int ndim, const int64_t* n, long* idx)
{
    for (int a = 0; a < ndim; ++a) { idx[a] = i % (long)n[a]; i /= (long)n[a]; }
}

static long neighbour_plus(long i, int axis, int ndim, const int64_t* n)
{
    long idx[ORC_MAXD];
    unravel(i, ndim, n, idx);
    idx[axis] = (idx[axis] + 1) % (long)n[axis];
    long j = 0;
    for (int a = ndim - 1; a >= 0; --a) j = j * (long)n[a] + idx[a];
    return j;
}

/* gamma at a point given by continuous cell coordinates (sum over axes) */
static double gamma_at(const double* xi, int ndim, const int64_t* n, const int* nabs, double gmax, double power)
{
    double g = 0.0;
    for (int a = 0; a < ndim; ++a) g += layer_axis(xi[a], (long)n[a], nabs + 2 * a, gmax, power);
    return g;
}

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

static double median_of(double* v, long m)
{
    qsort(v, (size_t)m, sizeof(double), cmp_double);
    return (m % 2) ? v[m / 2] : 0.5 * (v[m / 2 - 1] + v[m / 2]);
}

/* circle through three points (NULL-safe for collinear input: returns 0) */
static int circumcircle(cplx a, cplx b, cplx c, cplx* centre, double* radius)
{
    double ax = creal(a), ay = cimag(a), bx = creal(b), by = cimag(b), cx = creal(c), cy = cimag(c);
    double d = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by));
    if (d == 0.0) return 0;
    double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
    double ux = (a2 * (by - cy) + b2 * (cy - ay) + c2 * (ay - by)) / d;
    double uy = (a2 * (cx - bx) + b2 * (ax - cx) + c2 * (bx - ax)) / d;
    *centre = ux + I * uy;
    *radius = cabs(a - *centre);
    return 1;
}

/* Minimum enclosing circle of a point set (the shift that minimises max|v - a|,
 * i.e. the norm of V0, Sec. 2.3.1 / Sec. 4): Welzl's randomised incremental
 * algorithm in its iterative form, over a fixed pseudo-random order. */
static cplx min_enclosing_centre(const cplx* vals, long m)
{
    long* idx = malloc(sizeof(long) * m);
    for (long i = 0; i < m; ++i) idx[i] = i;
    unsigned long long st = 0x9E3779B97F4A7C15ull;
    for (long i = m - 1; i > 0; --i) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        long j = (long)((st >> 33) % (unsigned long long)(i + 1));
        long t = idx[i]; idx[i] = idx[j]; idx[j] = t;
    }
    const double tol = 1e-12;
    cplx c = vals[idx[0]];
    double r = 0.0;
    for (long i = 1; i < m; ++i) {
        cplx pi = vals[idx[i]];
        if (cabs(pi - c) <= r * (1 + tol)) continue;
        c = pi;
        r = 0.0;
        for (long j = 0; j < i; ++j) {
            cplx pj = vals[idx[j]];
            if (cabs(pj - c) <= r * (1 + tol)) continue;
            c = 0.5 * (pi + pj);
            r = 0.5 * cabs(pi - pj);
            for (long k = 0; k < j; ++k) {
                cplx pk = vals[idx[k]];
                if (cabs(pk - c) <= r * (1 + tol)) continue;
                cplx cc;
                double rr;
                if (circumcircle(pi, pj, pk, &cc, &rr)) { c = cc; r = rr; }
            }
        }
    }
    free(idx);
    return c;
}

/* complex shift over a set of values: 0 = midrange (bounding-box centre),
 * 1 = componentwise median (Algorithm 1's example), 2 = centre of the minimum
 * enclosing circle (Sec. 4's recommendation) */
static cplx choose_shift(const cplx* vals, long m, int rule)
{
    if (rule == 2) return min_enclosing_centre(vals, m);
    if (rule == 1) {
        double* re = malloc(sizeof(double) * m);
        double* im = malloc(sizeof(double) * m);
        for (long i = 0; i < m; ++i) { re[i] = creal(vals[i]); im[i] = cimag(vals[i]); }
        cplx a = median_of(re, m) + I * median_of(im, m);
        free(re); free(im);
        return a;
    }
    double rmin = INFINITY, rmax = -INFINITY, imin = INFINITY, imax = -INFINITY;
    for (long i = 0; i < m; ++i) {
        double r = creal(vals[i]), q = cimag(vals[i]);
        if (r < rmin) rmin = r;
        if (r > rmax) rmax = r;
        if (q < imin) imin = q;
        if (q > imax) imax = q;
    }
    return 0.5 * (rmin + rmax) + I * 0.5 * (imin + imax);
}

/* Returns NULL on invalid input (non-finite, c<=0, rho<=0, alpha<0, degenerate
 * scaling).  nabs: [D][2] cells (low side, high side) per axis. */
orc_problem* orc_create(int ndim, const int64_t* n, double dx, double omega,
                        const double* c0, const double* rho, const double* alpha,
                        const int* nabs, double gamma_max, double power,
                        double beta, int shift_rule, int collocated)
{
    if (ndim < 1 || ndim > ORC_MAXD || !(dx > 0) || !(omega > 0) || !(beta > 0 && beta < 1)) return NULL;
    orc_problem* P = calloc(1, sizeof(orc_problem));
    P->ndim = ndim;
    P->ncomp = ndim + 1;
    P->N = 1;
    for (int a = 0; a < ndim; ++a) { P->n[a] = n[a]; P->N *= (long)n[a]; }
    P->dx = dx;
    P->omega = omega;
    P->collocated = collocated;
    const long N = P->N;
    for (long i = 0; i < N; ++i)
        if (!isfinite(c0[i]) || !isfinite(rho[i]) || !isfinite(alpha[i]) || !(c0[i] > 0) || !(rho[i] > 0) || !(alpha[i] >= 0)) {
            free(P);
            return NULL;
        }

    /* complex sound speed, eq. 118: c^2 = c0^2 / (1 - 2 i alpha c0 / omega) */
    P->inv_rho_c2 = malloc(sizeof(cplx) * N);
    cplx* gam_c = malloc(sizeof(cplx) * N);
    cplx* q = malloc(sizeof(cplx) * N);
    for (long i = 0; i < N; ++i) {
        cplx c2 = c0[i] * c0[i] / (1.0 - 2.0 * I * alpha[i] * c0[i] / omega);
        P->inv_rho_c2[i] = 1.0 / (rho[i] * c2);
    }
    /* gamma at the cell centres and at the staggered points (App. B.1) */
    P->rho_stag = malloc(sizeof(cplx) * ndim * N);
    cplx* d = malloc(sizeof(cplx) * ndim * N);
    for (long i = 0; i < N; ++i) {
        long idx[ORC_MAXD];
        double xi[ORC_MAXD];
        unravel(i, ndim, n, idx);
        for (int a = 0; a < ndim; ++a) xi[a] = (double)idx[a];
        double g = gamma_at(xi, ndim, n, nabs, gamma_max, power);
        gam_c[i] = g;
        /* pressure diagonal: (i omega + gamma) / (rho c^2), eq. HH1stOrderSH */
        q[i] = (I * omega + g) * P->inv_rho_c2[i];
        for (int eta = 0; eta < ndim; ++eta) {
            double xs[ORC_MAXD];
            memcpy(xs, xi, sizeof xs);
            if (!collocated) xs[eta] += 0.5;
            double gs = gamma_at(xs, ndim, n, nabs, gamma_max, power);
            /* staggered density: mean of the two neighbours along eta (collocated: rho itself) */
            double rs = collocated ? rho[i] : 0.5 * (rho[i] + rho[neighbour_plus(i, eta, ndim, n)]);
            P->rho_stag[eta * N + i] = rs;
            /* velocity diagonal: (S+ rho)(S+ gamma + i omega), App. B.1 */
            d[eta * N + i] = rs * (gs + I * omega);
        }
    }
    /* shifts (Algorithm 1 preprocessing) and scaling (eq. C) */
    P->a1 = choose_shift(d, ndim * N, shift_rule);
    P->a2 = choose_shift(q, N, shift_rule);
    double m1 = 0.0, m2 = 0.0;
    for (long i = 0; i < ndim * N; ++i) { double t = cabs(d[i] - P->a1); if (t > m1) m1 = t; }
    for (long i = 0; i < N; ++i) { double t = cabs(q[i] - P->a2); if (t > m2) m2 = t; }
    P->maxdev1 = m1;
    P->maxdev2 = m2;
    P->lam1 = m1 > 0 ? m1 / beta : cabs(P->a1);
    P->lam2 = m2 > 0 ? m2 / beta : cabs(P->a2);
    if (!(P->lam1 > 0) || !(P->lam2 > 0)) {
        free(gam_c); free(q); free(d); free(P->inv_rho_c2); free(P->rho_stag); free(P);
        return NULL;
    }
    /* V = C^-1/2 (diag - a) C^-1/2 (eq. LV); C is constant per block */
    P->v = malloc(sizeof(cplx) * P->ncomp * N);
    for (int eta = 0; eta < ndim; ++eta)
        for (long i = 0; i < N; ++i) P->v[eta * N + i] = (d[eta * N + i] - P->a1) / P->lam1;
    for (long i = 0; i < N; ++i) P->v[ndim * N + i] = (q[i] - P->a2) / P->lam2;
    free(gam_c); free(q); free(d);

    /* k_eta = 2 pi fftfreq(n_eta, dx) */
    long nmax = 0;
    for (int a = 0; a < ndim; ++a) if (n[a] > nmax) nmax = (long)n[a];
    P->kstride = nmax;
    P->k = calloc((size_t)ndim * nmax, sizeof(double));
    for (int a = 0; a < ndim; ++a) {
        long L = (long)n[a];
        for (long j = 0; j < L; ++j) {
            long f = (j < (L + 1) / 2) ? j : j - L;
            P->k[a * nmax + j] = 2.0 * ORC_PI * (double)f / ((double)L * dx);
        }
    }
    return P;
}

void orc_destroy(orc_problem* P)
{
    if (!P) return;
    free(P->v); free(P->rho_stag); free(P->inv_rho_c2); free(P->k);
    free(P);
}

/* scalars: out[0..5] = Re a1, Im a1, Re a2, Im a2, lambda1, lambda2 */
void orc_scalars(const orc_problem* P, double* out)
{
    out[0] = creal(P->a1); out[1] = cimag(P->a1);
    out[2] = creal(P->a2); out[3] = cimag(P->a2);
    out[4] = P->lam1; out[5] = P->lam2;
}

void orc_get_v(const orc_problem* P, cplx* v) { memcpy(v, P->v, sizeof(cplx) * P->ncomp * P->N); }

/* y = C^-1/2 s_hat with s_hat_u = (S+ rho) s_u, s_hat_p = s_p / (rho c^2)
 * (eq. HH1stOrderSH, scaled source of Sec. 2.3.1).  adjoint != 0: the adjoint
 * right-hand side is taken as given (no row scaling), y = C^-1/2 g. */
void orc_scale_source(const orc_problem* P, const cplx* s, cplx* y, int adjoint)
{
    const long N = P->N;
    const int D = P->ndim;
    const double r1 = 1.0 / sqrt(P->lam1), r2 = 1.0 / sqrt(P->lam2);
    for (int eta = 0; eta < D; ++eta)
        for (long i = 0; i < N; ++i)
            y[eta * N + i] = (adjoint ? s[eta * N + i] : P->rho_stag[eta * N + i] * s[eta * N + i]) * r1;
    for (long i = 0; i < N; ++i)
        y[D * N + i] = (adjoint ? s[D * N + i] : s[D * N + i] * P->inv_rho_c2[i]) * r2;
}

/* (u, p) = C^-1/2 x  (Algorithm 1 output) */
void orc_unscale(const orc_problem* P, const cplx* x, cplx* field)
{
    const long N = P->N;
    const int D = P->ndim;
    const double r1 = 1.0 / sqrt(P->lam1), r2 = 1.0 / sqrt(P->lam2);
    for (int eta = 0; eta < D; ++eta)
        for (long i = 0; i < N; ++i) field[eta * N + i] = x[eta * N + i] * r1;
    for (long i = 0; i < N; ++i) field[D * N + i] = x[D * N + i] * r2;
}

/* ------------------------------------------------------------------------- */
/* Fourier-domain operators (App. B, App. B.1)                                 */
/* ------------------------------------------------------------------------- */

static void k_vector(const orc_problem* P, long i, double* kv)
{
    long idx[ORC_MAXD];
    unravel(i, P->ndim, P->n, idx);
    for (int a = 0; a < P->ndim; ++a) kv[a] = P->k[a * P->kstride + idx[a]];
}

/* Staggered (L+I)^-1 at one wavenumber, written entry by entry as in App. B.1
 * with the appendix notation a = a1, lambda_0 = lambda1, b = a2,
 * lambda_1(appendix) = lambda2:
 *   G_{eta eta}  = lambda_0 (mu - k_eta^2) / ((a + lambda_0) mu)
 *   G_{eta nu}   = -lambda_0 k_eta k_nu S_eta^nu / ((a + lambda_0) mu)
 *   G_{eta p}    = -i k_eta sqrt(lambda_0 lambda_1) S_eta / mu
 *   G_{p eta}    = -i k_eta sqrt(lambda_0 lambda_1) S^eta / mu
 *   G_{p p}      = lambda_1 (a + lambda_0) / mu
 * with mu = k^2 + (a + lambda_0)(b + lambda_1), S_eta = e^{i k_eta dx/2},
 * S^eta = conj(S_eta), S_eta^nu = S_eta S^nu. */
static void green_matrix(const orc_problem* P, const double* kv, cplx G[ORC_MAXD + 1][ORC_MAXD + 1])
{
    const int D = P->ndim;
    const cplx a = P->a1, b = P->a2;
    const double l0 = P->lam1, l1 = P->lam2;
    double k2 = 0.0;
    cplx S[ORC_MAXD];
    for (int e = 0; e < D; ++e) {
        k2 += kv[e] * kv[e];
        /* collocated grid (App. B): no half-cell shift filters */
        S[e] = P->collocated ? 1.0 : cexp(I * kv[e] * P->dx / 2.0);
    }
    const cplx mu = k2 + (a + l0) * (b + l1);
    const double sq = sqrt(l0 * l1);
    for (int e = 0; e < D; ++e) {
        for (int f = 0; f < D; ++f) {
            if (e == f) G[e][f] = l0 * (mu - kv[e] * kv[e]) / ((a + l0) * mu);
            else G[e][f] = -l0 * kv[e] * kv[f] * (S[e] * conj(S[f])) / ((a + l0) * mu);
        }
        G[e][D] = -I * kv[e] * sq * S[e] / mu;
        G[D][e] = -I * kv[e] * sq * conj(S[e]) / mu;
    }
    G[D][D] = l1 * (a + l0) / mu;
}

/* Scaled L symbol at one wavenumber (eq. LV with the staggered derivative
 * symbols of App. B.1: S+ d_eta -> i k_eta S_eta, d_eta S- -> i k_eta S^eta):
 *   L = [[ a1/lambda1 I , i k S / sqrt(l1 l2) ], [ i k^T S^ / sqrt(l1 l2), a2/lambda2 ]] */
static void l_matrix(const orc_problem* P, const double* kv, cplx Lm[ORC_MAXD + 1][ORC_MAXD + 1])
{
    const int D = P->ndim;
    const double sq = sqrt(P->lam1 * P->lam2);
    for (int e = 0; e <= D; ++e)
        for (int f = 0; f <= D; ++f) Lm[e][f] = 0;
    for (int e = 0; e < D; ++e) {
        cplx Se = P->collocated ? 1.0 : cexp(I * kv[e] * P->dx / 2.0);
        Lm[e][e] = P->a1 / P->lam1;
        Lm[e][D] = I * kv[e] * Se / sq;
        Lm[D][e] = I * kv[e] * conj(Se) / sq;
    }
    Lm[D][D] = P->a2 / P->lam2;
}

/* Apply a per-wavenumber (C x C) matrix to a field: out = F^-1 M(k) F in.
 * mode 0: M = (L+I)^-1, 1: M = L, 2: M = [(L+I)^-1]^H, 3: M = L^H. */
static void fourier_apply(const orc_problem* P, const cplx* in, cplx* out, int mode)
{
    const long N = P->N;
    const int C = P->ncomp;
    cplx* F = malloc(sizeof(cplx) * C * N);
    memcpy(F, in, sizeof(cplx) * C * N);
    for (int c = 0; c < C; ++c) orc_fftn(F + c * N, P->ndim, P->n, -1);
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        double kv[ORC_MAXD];
        cplx M[ORC_MAXD + 1][ORC_MAXD + 1], vin[ORC_MAXD + 1];
        k_vector(P, i, kv);
        if (mode == 0 || mode == 2) green_matrix(P, kv, M);
        else l_matrix(P, kv, M);
        for (int c = 0; c < C; ++c) vin[c] = F[c * N + i];
        for (int r = 0; r < C; ++r) {
            cplx acc = 0;
            for (int c = 0; c < C; ++c) acc += (mode >= 2 ? conj(M[c][r]) : M[r][c]) * vin[c];
            F[r * N + i] = acc;
        }
    }
    for (int c = 0; c < C; ++c) orc_fftn(F + c * N, P->ndim, P->n, +1);
    memcpy(out, F, sizeof(cplx) * C * N);
    free(F);
}

/* out = (L+I)^-1 in  (adjoint: [(L+I)^-1]^H in) */
void orc_green(const orc_problem* P, const cplx* in, cplx* out, int adjoint)
{
    fourier_apply(P, in, out, adjoint ? 2 : 0);
}

/* out = A_s x = L x + V x  (adjoint: A_s^H x = L^H x + conj(V) x), eq. LV */
void orc_apply(const orc_problem* P, const cplx* x, cplx* out, int adjoint)
{
    const long CN = (long)P->ncomp * P->N;
    fourier_apply(P, x, out, adjoint ? 3 : 1);
    for (long i = 0; i < CN; ++i) out[i] += (adjoint ? conj(P->v[i]) : P->v[i]) * x[i];
}

static double norm2(const cplx* a, long m)
{
    double s = 0.0;
    for (long i = 0; i < m; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

/* ||y - A_s x|| / ||y||  (true scaled residual) */
double orc_residual(const orc_problem* P, const cplx* x, const cplx* y, int adjoint)
{
    const long CN = (long)P->ncomp * P->N;
    cplx* r = malloc(sizeof(cplx) * CN);
    orc_apply(P, x, r, adjoint);
    for (long i = 0; i < CN; ++i) r[i] = y[i] - r[i];
    double rr = sqrt(norm2(r, CN) / norm2(y, CN));
    free(r);
    return rr;
}

/* Born iterations, eq. BornAlt / Algorithm 1:
 *   z = (L+I)^-1 (B x + y);  x <- x + nu B (z - x),  B = I - V.
 * Runs n_iter iterations in place on x.  incr (optional, n_iter values):
 * ||x_{k+1} - x_k|| / ||x_{k+1}||, the quantity Algorithm 1 tests. */
void orc_iterate(const orc_problem* P, const cplx* y, cplx* x, long n_iter, double nu, int adjoint, double* incr)
{
    const long CN = (long)P->ncomp * P->N;
    cplx* w = malloc(sizeof(cplx) * CN);
    cplx* z = malloc(sizeof(cplx) * CN);
    for (long it = 0; it < n_iter; ++it) {
        for (long i = 0; i < CN; ++i) {
            cplx B = 1.0 - (adjoint ? conj(P->v[i]) : P->v[i]);
            w[i] = B * x[i] + y[i];
        }
        orc_green(P, w, z, adjoint);
        double dd = 0.0, xx = 0.0;
        for (long i = 0; i < CN; ++i) {
            cplx B = 1.0 - (adjoint ? conj(P->v[i]) : P->v[i]);
            cplx delta = nu * B * (z[i] - x[i]);
            x[i] += delta;
            dd += creal(delta) * creal(delta) + cimag(delta) * cimag(delta);
            xx += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
        }
        if (incr) incr[it] = xx > 0 ? sqrt(dd / xx) : 0.0;
    }
    free(w); free(z);
}

/* Iterate until the true scaled residual <= tol, checked every check_every
 * iterations (and at max_iter).  Returns the iteration count; *res gets the
 * last residual.  x holds the start value on entry. */
long orc_solve(const orc_problem* P, const cplx* y, cplx* x, double nu, double tol, long max_iter,
               long check_every, int adjoint, double* res)
{
    long it = 0;
    double r = orc_residual(P, x, y, adjoint);
    while (r > tol && it < max_iter) {
        long blk = check_every;
        if (it + blk > max_iter) blk = max_iter - it;
        orc_iterate(P, y, x, blk, nu, adjoint, NULL);
        it += blk;
        r = orc_residual(P, x, y, adjoint);
    }
    if (res) *res = r;
    return it;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
