/*
 * cbs.h -- C ABI of the GB300 Born solver for the acoustic Helmholtz equation
 * with heterogeneous sound speed, density and absorption.
 *
 * Method: A. Stanziola, S. R. Arridge, B. E. Treeby, B. T. Cox, "Iterative
 * Born solver for the acoustic Helmholtz equation with heterogeneous sound
 * speed and density" (arXiv 2507.16087).  The solver iterates eq. BornAlt
 * (Algorithm 1) on the row-scaled first-order system (eq. HH1stOrderSH) on a
 * staggered grid (App. B.1):
 *
 *   [ (S+ rho)(S+ gamma + i omega)   S+ grad            ] [ u ]   [ (S+ rho) s_u     ]
 *   [ div S-                         (i omega + gamma)/(rho c^2) ] [ p ] = [ s_p / (rho c^2) ]
 *
 * with the complex sound speed c^2 = c0^2 / (1 - 2 i alpha c0 / omega)
 * (eq. 118), split A = L + V with shifts a1, a2 and scaling C = diag(lambda1,
 * lambda2) (eq. LV, eq. C), and (L+I)^-1 applied in the Fourier domain
 * (App. B.1).
 *
 * Conventions shared by every entry point:
 *  - Grid: ndim = 2 or 3, extents n[0] (x, fastest), n[1] (y), n[2] (z);
 *    every extent is one of 8,12,16,24,32,48,64,96,128,192,256,512,1024,2048
 *    (3D grids with an extent above 512 are accepted but need ~350 B/voxel).
 *  - Field / source arrays: caller-owned DEVICE buffers of (ndim+1)*N
 *    complex128 values (interleaved re, im; 16-byte aligned), component-major
 *    [u_x][u_y][(u_z)][p], each component laid out [n2][n1][n0].  Velocity
 *    component eta sits at the staggered points x + (dx/2) e_eta.
 *  - Medium arrays c0 (m/s), rho (kg/m^3), alpha (Np/m): caller-owned DEVICE
 *    buffers of N float64 values [n2][n1][n0].  They are read during
 *    solver_create only; the solver keeps its own derived copies.
 *  - Every call enqueues its work on the solver's internal stream after the
 *    work already queued on opt->stream, and returns only when its work is
 *    complete.  Results (info, scalars) are valid on return.
 *  - Errors are return codes; cbs_last_error gives a message.  Nothing aborts,
 *    exits or throws across the ABI.  A call with invalid arguments changes no
 *    output.
 */
#ifndef CBS_H
#define CBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CBS_OK = 0,
    CBS_EINVAL = 1,     /* invalid argument, unsupported size, rejected medium */
    CBS_ENOMEM = 2,     /* device allocation failed */
    CBS_ECUDA = 3,      /* a CUDA call failed */
    CBS_ENOCONV = 4,    /* max_iter reached before tol; field holds the last iterate */
    CBS_EDIVERGED = 5,  /* non-finite or growing iterate; field holds the last finite iterate */
    CBS_ETIMEOUT = 6    /* a staged bulk copy did not complete within its bounded wait */
} cbs_status;

enum { CBS_FP64 = 0, CBS_FP32_REFINE = 1, CBS_FP32 = 2 };
enum { CBS_SHIFT_MIDRANGE = 0, CBS_SHIFT_MEDIAN = 1, CBS_SHIFT_MEC = 2 };
enum { CBS_GRID_STAGGERED = 0, CBS_GRID_COLLOCATED = 1 };

typedef struct {
    int ndim;      /* 2 or 3 */
    int64_t n[3];  /* n[0] = x (fastest) .. n[ndim-1]; unused entries ignored */
} cbs_grid;

/* Absorbing layer gamma(x) (the paper names it, Sec. 2.1, but gives no
 * profile): n_abs[a][0/1] cells on the low/high side of axis a, inside the
 * grid; depth(xi) = min(1, max(0, (lo - xi)/lo, (xi - (n-1-hi))/hi)) at cell
 * coordinate xi; gamma = gamma_max * sum_a depth_a^power; the staggered
 * values are taken at xi + 1/2 (App. B.1). */
typedef struct {
    int n_abs[3][2];
    double gamma_max; /* 1/s */
    double power;
} cbs_boundary;

/* Optional device allocator for the solver's own arrays, so that a framework's caching allocator (torch's,
 * for instance) can serve them instead of cudaMalloc / cudaFree.  dev_alloc(bytes, stream, ctx) gets
 * options.stream as `stream` and returns device memory aligned to at least 256 bytes (the staged bulk
 * and tensor copies need 16), or NULL on failure; dev_free(ptr, ctx) takes back what dev_alloc gave.
 * The solver calls them from solver_create (its arrays and set-up temporaries) and solver_destroy, on the
 * calling thread, after its own work on the memory is complete.  The paper has no counterpart. */
typedef void* (*cbs_dev_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*cbs_dev_free_fn)(void* ptr, void* ctx);

typedef struct {
    int precision;     /* CBS_FP64 (default), CBS_FP32_REFINE, CBS_FP32 */
    double nu;         /* 0 < nu < 1 (eq. BornAlt); 0 -> 0.8 */
    double beta;       /* 0 < beta < 1 (eq. C); 0 -> 0.95 */
    int shift_rule;    /* CBS_SHIFT_MIDRANGE (default), CBS_SHIFT_MEDIAN, or CBS_SHIFT_MEC: centre of
                          the minimum enclosing circle of the support points of the value set in
                          64 directions (Sec. 4's recommendation, to within the polygon's sag) */
    double tol;        /* relative scaled residual ||y - A_s x|| / ||y||; <= 0: run exactly max_iter */
    double tol_inner;  /* FP32_REFINE: inner relative reduction per outer step; 0 -> 1e-4 */
    int max_iter;      /* Born iterations (all inner iterations for FP32_REFINE); 0 -> 100000 */
    int check_every;   /* iterations between residual checks; 0 -> 50 */
    void* stream;      /* cudaStream_t the caller's work is queued on (may be 0) */
    int grid_kind;     /* CBS_GRID_STAGGERED (default, App. B.1: velocity at x + dx/2 e_eta, staggered
                          density, symbol i k e^{i k dx/2}) or CBS_GRID_COLLOCATED (App. B: velocity at
                          the cell centres, unshifted density and gamma, symbol i k) */
    cbs_dev_alloc_fn dev_alloc;  /* NULL (default): cudaMalloc; else set dev_free too (CBS_EINVAL otherwise) */
    cbs_dev_free_fn dev_free;
    void* alloc_ctx;             /* passed to dev_alloc / dev_free */
} cbs_options;

typedef struct {
    int iters;              /* Born iterations run (FP32 inner iterations for FP32_REFINE) */
    int outer_iters;        /* refinement steps (FP32_REFINE), else 0 */
    int residual_checks;    /* true-residual evaluations */
    double rel_residual;    /* last true scaled residual (FP64 for FP64 and FP32_REFINE) */
    double rel_increment;   /* last ||x_{k+1} - x_k|| / ||x_{k+1}|| (Algorithm 1's criterion) */
    double a1[2], a2[2];    /* shifts (re, im) */
    double lambda1, lambda2;/* scaling (eq. C) */
    double t_setup_ms;      /* solver_create device time */
    double t_solve_ms;      /* this call's device time */
    long long kernel_launches; /* kernels this call launched (graph nodes included) */
} cbs_info;

typedef struct cbs_solver cbs_solver;

/* Build a solver for one medium, frequency and grid (Algorithm 1
 * preprocessing): complex sound speed (eq. 118), staggered density
 * (App. B.1), diagonal values, shifts a1, a2 (midrange of the diagonal values
 * by default; componentwise median or minimum enclosing circle on request), lambda_j = max|diag - a_j| /
 * beta (eq. C; lambda_j = |a_j| when that max is 0), per-axis wavenumber and
 * twiddle tables.  c0, rho, alpha: device float64 [N].  Rejects (CBS_EINVAL)
 * non-finite values, c0 <= 0, rho <= 0, alpha < 0, unsupported extents,
 * nu/beta outside (0,1).  On success *out owns all device memory it uses until
 * solver_destroy. */
cbs_status solver_create(const cbs_grid* grid, double dx, double omega, const double* c0, const double* rho,
                         const double* alpha, const cbs_boundary* boundary, const cbs_options* opt,
                         cbs_solver** out);

/* Solve A (u, p) = (S+ rho s_u, s_p / (rho c^2)) for the physical field
 * (Algorithm 1: x = 0 or x0, iterate, output C^-1/2 x).  src, field: device
 * complex128 [C][N] (physical s_u, s_p in; physical u, p out).  x0_or_null:
 * optional physical start field.  Stops when the true scaled residual
 * ||y - A_s x|| / ||y|| <= tol (checked every check_every iterations); FP64:
 * all arithmetic in float64; FP32_REFINE: inner Born iterations in float32 on
 * r / ||r|| with the residual r = y - A_s x, its norm and the correction
 * accumulation in float64; FP32: everything in float32 (residual in float32).
 * info may be NULL. */
cbs_status solve_forward(cbs_solver* s, const void* src, void* field, const void* x0_or_null, cbs_info* info);

/* Solve the adjoint system A^H lambda = g (Sec. 2.3: A^H is accretive for
 * alpha >= 0, so the same iteration applies with conj(B) and the per-wavenumber
 * conjugate transpose of the staggered (L+I)^-1 symbol).  g is taken as the
 * adjoint right-hand side as given (no row scaling).  Same layouts and stopping
 * rule as solve_forward. */
cbs_status solve_adjoint(cbs_solver* s, const void* src, void* field, const void* x0_or_null, cbs_info* info);

/* Relative scaled residual of a physical field for a physical source,
 * ||y - A_s C^1/2 (u,p)|| / ||y|| with y the scaled source (adjoint != 0: the
 * adjoint system), computed in float64 on the device. */
cbs_status residual_norm(cbs_solver* s, const void* field, const void* src, int adjoint, double* rel);

/* Run exactly n_iter Born iterations (eq. BornAlt) in the solver's precision
 * (FP64, or FP32 for FP32 / FP32_REFINE) on the scaled variables, starting from
 * the scaled iterate x (device complex128 [C][N], updated in place) with the
 * scaled right-hand side y (device complex128).  incr (host, n_iter doubles,
 * may be NULL) receives ||x_{k+1}-x_k|| / ||x_{k+1}|| per iteration. */
cbs_status born_iterate(cbs_solver* s, const void* y, void* x, int n_iter, int adjoint, double* incr);

/* out = (L+I)^-1 in (adjoint: [(L+I)^-1]^H in) on scaled fields (device
 * complex128 [C][N]), in the solver's iteration precision (App. B.1). */
cbs_status green_apply(cbs_solver* s, const void* in, void* out, int adjoint);

/* out = A_s x = L x + V x (adjoint: A_s^H x) on scaled fields, float64 (eq. LV). */
cbs_status operator_apply(cbs_solver* s, const void* x, void* out, int adjoint);

/* y = C^-1/2 (S+ rho s_u, s_p / (rho c^2))  (adjoint: y = C^-1/2 g), and the
 * inverse map field = C^-1/2 x of Algorithm 1's output.  Device complex128. */
cbs_status scale_source(cbs_solver* s, const void* src, void* y, int adjoint);
cbs_status unscale_field(cbs_solver* s, const void* x, void* field);

/* Adjoint-state medium gradient (Sec. 2.3: the adjoint A^H lambda = g is
 * solved by solve_adjoint).  Per voxel, in float64:
 *   grad_c0  = Re conj(lambda_p) (db_p/dc0 - dq/dc0 p)
 *   grad_rho = Re conj(lambda_p) (db_p/drho - dq/drho p)
 *            + sum_eta 1/2 Re conj(lambda_eta) (s_u,eta - (S+ gamma_eta + i omega) u_eta)
 *              at x and at x - e_eta (the staggered density, App. B.1)
 * with q = (i omega + gamma)/(rho c^2), b_p = s_p/(rho c^2) (eq. HH1stOrderSH,
 * eq. 118): i.e. dJ/dm for a misfit J with dJ = Re<g, dX>.  c0, rho, alpha:
 * the device medium the solver was created from; src, field, adj_field: device
 * complex128 [C][N] physical source, forward field and adjoint field;
 * grad_c0, grad_rho: device float64 [N], overwritten (accumulate = 0) or added
 * to (accumulate != 0). */
cbs_status medium_gradient(cbs_solver* s, const double* c0, const double* rho, const double* alpha, const void* src,
                           const void* field, const void* adj_field, double* grad_c0, double* grad_rho, int accumulate);

/* Shifts and scaling: out[0..5] = Re a1, Im a1, Re a2, Im a2, lambda1, lambda2. */
cbs_status solver_scalars(const cbs_solver* s, double* out);

/* Average device time (ms) per launch of each kernel of one Born iteration
 * (the per-block norm reduction, one launch per check_every iterations, is not
 * included),
 * measured with CUDA events on the solver's stream over n_iter iterations
 * after one untimed iteration (scaled iterate and source taken as given,
 * updated in place by all n_iter + 1 iterations).  names
 * receives up to max_k NUL-separated kernel names; ms receives one time per
 * kernel; *nk the kernel count. */
cbs_status solver_time_kernels(cbs_solver* s, const void* y, void* x, int n_iter, char* names, int names_len,
                               double* ms, int max_k, int* nk);

/* Allocation-free (L+I)^-1 apply, for callers that cannot call cudaMalloc
 * (code that must stay inside another framework's memory pool or a fixed
 * device-memory budget).  The paper has no counterpart: it is the float64
 * transform green_apply runs for a solver on the staggered grid (App. B.1, the
 * default grid kind; a collocated-grid solver's green_apply differs), without a
 * solver object.  grid as for
 * solver_create (extents <= 512, at most 2,097,152 voxels, else CBS_EINVAL with
 * a message from cbs_last_error(NULL)); scalars[0..5] = Re a1, Im a1, Re a2,
 * Im a2, lambda1, lambda2 (as solver_scalars returns them); in, out: distinct
 * caller-owned device complex128 [C][N] buffers; out is also the work array.
 * Work is enqueued on `stream` (cudaStream_t, may be 0) and the call
 * synchronises that stream before it returns.  It allocates no device memory:
 * its tables and norm partials live in a static device array of 124 KiB that
 * every GPU loading the library holds until exit.  The first call on each
 * device looks up that array's device address (cudaGetSymbolAddress) and keeps
 * it for the life of the process, so make the first call on a device before
 * any stream capture, and do not call it on a device after cudaDeviceReset.
 * All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller. */
cbs_status green_apply_noalloc(const cbs_grid* grid, double dx, const double* scalars, const void* in, void* out,
                               int adjoint, void* stream);

/* Comparison build of the iteration (timed only; the solver never calls it): n_iter float32 Born
 * iterations of eq. BornAlt with the App. B.1 symbol, the transforms done by cuFFT (batched
 * complex-to-complex plans over the C components, made on first use and kept by the solver) and the
 * rest by plain pointwise kernels: w = B x + y, FFT, symbol, IFFT, x += nu B (w - x).  y: scaled source,
 * x: scaled iterate, updated in place (device complex128 [C][N], as born_iterate).  *ms_per_iter: CUDA-event
 * time per iteration on the solver's stream, casts excluded.  CBS_EINVAL for a float64 solver. */
cbs_status cufft_baseline_iterate(cbs_solver* s, const void* y, void* x, int n_iter, int adjoint, double* ms_per_iter);

/* Failure-detection self-test (no counterpart in the paper).  which =
 * CBS_SELFTEST_BULK_TIMEOUT launches one block whose bulk copy delivers half
 * the bytes its shared-memory barrier expects, so the barrier never completes:
 * the kernel's bounded wait gives up, records the timeout in an error word and
 * returns, as the Born row kernels do.  *result = CBS_ETIMEOUT when the wait
 * expired and was reported, CBS_OK otherwise.  Returns CBS_ECUDA if a CUDA
 * call failed (the context stays usable after a timeout).  Allocates and
 * frees 24 bytes of device memory. */
enum { CBS_SELFTEST_BULK_TIMEOUT = 1 };
cbs_status cbs_selftest(int which, int* result);

/* Float64 arithmetic rate of the current device, for stating the float64 path against the roof that
 * binds it (the paper has no counterpart; not on the solver's path).  Runs eight independent chains of
 * double-precision fused multiply-adds in every thread of 16 blocks of 256 threads per SM and times the
 * second of two launches with CUDA events on the default stream; *tflops = 2 * FMAs / time / 1e12.
 * Allocates and frees 8 bytes of device memory.  CBS_EINVAL for a NULL pointer, CBS_ECUDA / CBS_ENOMEM
 * when a CUDA call fails. */
cbs_status cbs_fp64_rate(double* tflops);

void solver_destroy(cbs_solver* s);

/* Message of the last failure on this solver (or of the last failed
 * solver_create when s is NULL).  Never NULL. */
const char* cbs_last_error(const cbs_solver* s);

#ifdef __cplusplus
}
#endif
#endif /* CBS_H */
