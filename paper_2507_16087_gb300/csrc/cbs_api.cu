// cbs_api.cu -- C ABI of the Born solver: set-up (Algorithm 1 preprocessing),
// the FP64 / FP32 / FP32+FP64-refinement drivers, the adjoint, and the
// operator entry points used for step-by-step checks.  All compute runs in
// the kernels of born.cuh and the set-up/utility kernels below; the host
// only computes O(n) per-axis tables and scalars.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "cbs.h"
#include "launch.cuh"
#include "baseline_cufft.cuh"

namespace cbs {
CBS_EXTERN_LAUNCHERS(float)
CBS_EXTERN_LAUNCHERS(double)
}  // namespace cbs

using namespace cbs;

namespace {

constexpr int kHostBuf = 8192;  // pinned host doubles

// Pinned host buffers for the norm read-backs, kept in a process-wide pool and never freed while the library is
// loaded: cudaFreeHost may synchronise the whole device, which would stall the streams of every other solver
// running when one solver is destroyed (the serving loop creates and destroys solvers while others run).
std::mutex g_pinned_mu;
std::vector<double*> g_pinned_free;

double* pinned_get()
{
    {
        std::lock_guard<std::mutex> lk(g_pinned_mu);
        if (!g_pinned_free.empty()) {
            double* p = g_pinned_free.back();
            g_pinned_free.pop_back();
            return p;
        }
    }
    double* p = nullptr;
    if (cudaMallocHost(&p, kHostBuf * sizeof(double)) != cudaSuccess) return nullptr;
    return p;
}

void pinned_put(double* p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    g_pinned_free.push_back(p);
}
constexpr int kSetupThreads = 256;
constexpr double kPi = 3.14159265358979323846264338327950288;

thread_local std::string g_create_error = "no error";

bool trace_on()
{
    static int on = -1;
    if (on < 0) on = std::getenv("CBS_TRACE") != nullptr;
    return on == 1;
}
#define TRACE(...)                                                                                                   \
    do {                                                                                                             \
        if (trace_on()) { std::fprintf(stderr, "[cbs] " __VA_ARGS__); std::fprintf(stderr, "\n"); std::fflush(stderr); } \
    } while (0)

// ---------------------------------------------------------------- set-up kernels
struct SetupIn {
    int colloc;  // 1: collocated grid (no half-cell shifts)
    int D, n0, n1, n2;
    long long N;
    double omega;
    const double* c0;
    const double* rho;
    const double* alpha;
    const double* gc[3];
    const double* gs[3];
};

__device__ __forceinline__ void unravel(const SetupIn& s, long long i, int& i0, int& i1, int& i2)
{
    i0 = (int)(i % s.n0);
    long long r = i / s.n0;
    i1 = (int)(r % s.n1);
    i2 = (int)(r / s.n1);
}

__device__ __forceinline__ long long plus_one(const SetupIn& s, int eta, int i0, int i1, int i2)
{
    if (s.colloc) return ((long long)i2 * s.n1 + i1) * s.n0 + i0;  // unshifted: the voxel itself
    if (eta == 0) i0 = (i0 + 1) % s.n0;
    else if (eta == 1) i1 = (i1 + 1) % s.n1;
    else i2 = (i2 + 1) % s.n2;
    return ((long long)i2 * s.n1 + i1) * s.n0 + i0;
}

__device__ __forceinline__ double gamma_c(const SetupIn& s, int i0, int i1, int i2)
{
    double g = s.gc[0][i0] + s.gc[1][i1];
    if (s.D == 3) g += s.gc[2][i2];
    return g;
}

__device__ __forceinline__ double gamma_s(const SetupIn& s, int eta, int i0, int i1, int i2)
{
    double g = (eta == 0 ? s.gs[0][i0] : s.gc[0][i0]) + (eta == 1 ? s.gs[1][i1] : s.gc[1][i1]);
    if (s.D == 3) g += (eta == 2 ? s.gs[2][i2] : s.gc[2][i2]);
    return g;
}

// diagonal values of the row-scaled system (eq. HH1stOrderSH, App. B.1):
//   d_eta = (S+ rho)_eta (S+ gamma_eta + i omega),  q = (i omega + gamma) / (rho c^2)
// with 1 / (rho c^2) = (1 - i 2 alpha c0 / omega) / (rho c0^2)   (eq. 118)
__device__ __forceinline__ void diag_values(const SetupIn& s, long long i, double2* d, double2& q)
{
    int i0, i1, i2;
    unravel(s, i, i0, i1, i2);
    const double rho = s.rho[i], c0 = s.c0[i], al = s.alpha[i];
    const double kap = 1.0 / (rho * c0 * c0), et = 2.0 * al * c0 / s.omega;
    const double g = gamma_c(s, i0, i1, i2);
    q = make_double2(kap * (g + et * s.omega), kap * (s.omega - g * et));
    for (int eta = 0; eta < s.D; ++eta) {
        const double rs = 0.5 * (rho + s.rho[plus_one(s, eta, i0, i1, i2)]);
        d[eta] = make_double2(rs * gamma_s(s, eta, i0, i1, i2), rs * s.omega);
    }
}

// per block: min/max of Re, Im over d (all eta) and q; invalid-input flag
__global__ void k_setup_minmax(SetupIn s, double* part, int* bad)
{
    double v[8] = {INFINITY, -INFINITY, INFINITY, -INFINITY, INFINITY, -INFINITY, INFINITY, -INFINITY};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.N; i += (long long)gridDim.x * blockDim.x) {
        const double c0 = s.c0[i], rho = s.rho[i], al = s.alpha[i];
        if (!(isfinite(c0) && isfinite(rho) && isfinite(al)) || !(c0 > 0.0) || !(rho > 0.0) || !(al >= 0.0)) {
            atomicOr(bad, 1);
            continue;
        }
        double2 d[3], q;
        diag_values(s, i, d, q);
        for (int e = 0; e < s.D; ++e) {
            v[0] = fmin(v[0], d[e].x); v[1] = fmax(v[1], d[e].x);
            v[2] = fmin(v[2], d[e].y); v[3] = fmax(v[3], d[e].y);
        }
        v[4] = fmin(v[4], q.x); v[5] = fmax(v[5], q.x);
        v[6] = fmin(v[6], q.y); v[7] = fmax(v[7], q.y);
    }
    __shared__ double sh[8][kSetupThreads];
    for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 8; ++k)
                sh[k][threadIdx.x] = (k & 1) ? fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + o])
                                             : fmin(sh[k][threadIdx.x], sh[k][threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) part[blockIdx.x * 8 + k] = sh[k][0];
}

// per block: max |d - a1|, max |q - a2|
__global__ void k_setup_maxdev(SetupIn s, double2 a1, double2 a2, double* part)
{
    double m1 = 0.0, m2 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.N; i += (long long)gridDim.x * blockDim.x) {
        double2 d[3], q;
        diag_values(s, i, d, q);
        for (int e = 0; e < s.D; ++e) m1 = fmax(m1, hypot(d[e].x - a1.x, d[e].y - a1.y));
        m2 = fmax(m2, hypot(q.x - a2.x, q.y - a2.y));
    }
    __shared__ double sh[2][kSetupThreads];
    sh[0][threadIdx.x] = m1;
    sh[1][threadIdx.x] = m2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][threadIdx.x + o]);
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[blockIdx.x * 2] = sh[0][0]; part[blockIdx.x * 2 + 1] = sh[1][0]; }
}

// all diagonal values (for the median shift rule): dv[eta*N + i], qv[i]
__global__ void k_setup_values(SetupIn s, double2* dv, double2* qv)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.N; i += (long long)gridDim.x * blockDim.x) {
        double2 d[3], q;
        diag_values(s, i, d, q);
        for (int e = 0; e < s.D; ++e) dv[e * s.N + i] = d[e];
        qv[i] = q;
    }
}

// Support points of a value set: for each of kSupportDirs directions theta_k,
// the value maximising Re(z e^{-i theta_k}).  Per block: the best value of
// each direction (projections compared in float32; the values are exact).
constexpr int kSupportDirs = 64;
__global__ void k_setup_support(const double2* __restrict__ vals, long long n, double2* __restrict__ best)
{
    float bp[kSupportDirs];
    int bi[kSupportDirs];
#pragma unroll
    for (int k = 0; k < kSupportDirs; ++k) { bp[k] = -INFINITY; bi[k] = -1; }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = (float)vals[i].x, y = (float)vals[i].y;
#pragma unroll
        for (int k = 0; k < kSupportDirs; ++k) {
            float sk, ck;
            sincospif(2.0f * (float)k / (float)kSupportDirs, &sk, &ck);
            const float p = x * ck + y * sk;
            if (p > bp[k]) { bp[k] = p; bi[k] = (int)i; }
        }
    }
    __shared__ float sp[kSupportDirs][32];
    __shared__ int si[kSupportDirs][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kSupportDirs; ++k) {
        float p = bp[k];
        int ix = bi[k];
        for (int o = 16; o > 0; o >>= 1) {
            const float po = __shfl_down_sync(0xffffffffu, p, o);
            const int io = __shfl_down_sync(0xffffffffu, ix, o);
            if (po > p) { p = po; ix = io; }
        }
        if (lane == 0) { sp[k][w] = p; si[k][w] = ix; }
    }
    __syncthreads();
    if (threadIdx.x < kSupportDirs) {
        const int k = threadIdx.x;
        float p = -INFINITY;
        int ix = -1;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j)
            if (si[k][j] >= 0 && sp[k][j] > p) { p = sp[k][j]; ix = si[k][j]; }
        best[(long long)blockIdx.x * kSupportDirs + k] = ix >= 0 ? vals[ix] : make_double2(NAN, NAN);
    }
}

// per-voxel arrays the iteration kernels read: rs_eta = (S+ rho)_eta / lambda1,
// kp = 1 / (rho c0^2 lambda2), et = 2 alpha c0 / omega  (float64 and float32)
__global__ void k_setup_store(SetupIn s, double il1, double il2, double* rs64_0, double* rs64_1, double* rs64_2,
                              double* kp64, double* et64, float* rs32_0, float* rs32_1, float* rs32_2, float* kp32,
                              float* et32)
{
    double* rs64[3] = {rs64_0, rs64_1, rs64_2};
    float* rs32[3] = {rs32_0, rs32_1, rs32_2};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.N; i += (long long)gridDim.x * blockDim.x) {
        int i0, i1, i2;
        unravel(s, i, i0, i1, i2);
        const double rho = s.rho[i], c0 = s.c0[i];
        for (int e = 0; e < s.D; ++e) {
            const double r = 0.5 * (rho + s.rho[plus_one(s, e, i0, i1, i2)]) * il1;
            rs64[e][i] = r;
            rs32[e][i] = (float)r;
        }
        const double kp = 1.0 / (rho * c0 * c0) * il2;
        const double et = 2.0 * s.alpha[i] * c0 / s.omega;
        kp64[i] = kp;
        et64[i] = et;
        kp32[i] = (float)kp;
        et32[i] = (float)et;
    }
}

// ---------------------------------------------------------------- gradient
// Re <lambda, db/dm - (dA/dm) X> per voxel for m = c0 and m = rho (adjoint-state
// gradient of a misfit; A^H lambda = g, Sec. 2.3).  A depends on the medium only
// through its diagonal: q = (i omega + gamma) / (rho c^2) (eq. HH1stOrderSH,
// eq. 118) and d_eta = (S+ rho)_eta (S+ gamma_eta + i omega) (App. B.1), whose
// staggered density couples rho(x) to the velocity rows at x and x - e_eta.
struct GradIn {
    SetupIn m;
    const double2* src;
    const double2* X;
    const double2* L;
};

__device__ __forceinline__ double re_conj_mul(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }  // Re(conj(a) b)

__global__ void k_medium_gradient(GradIn g, double* __restrict__ grad_c, double* __restrict__ grad_r, int accumulate)
{
    const SetupIn& s = g.m;
    const long long N = s.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int i0, i1, i2;
        unravel(s, i, i0, i1, i2);
        const double rho = s.rho[i], c0 = s.c0[i], al = s.alpha[i], w = s.omega;
        const double gam = gamma_c(s, i0, i1, i2);
        // fac = d/dc0 [(1 - 2 i alpha c0 / omega) / c0^2] = -2/c0^3 + 2 i alpha / (omega c0^2)
        const double2 fac = make_double2(-2.0 / (c0 * c0 * c0), 2.0 * al / (w * c0 * c0));
        // 1/(rho c^2) = (1 - 2 i alpha c0 / omega) / (rho c0^2)
        const double k = 1.0 / (rho * c0 * c0);
        const double2 ic2 = make_double2(k, -k * 2.0 * al * c0 / w);
        const double2 iwg = make_double2(gam, w);  // i omega + gamma
        const long long ip = (long long)s.D * N + i;
        const double2 p = g.X[ip], lp = g.L[ip], sp = g.src[ip];
        // c0: conj(lp) (sp fac - (i w + gam) fac p) / rho
        const double2 dq = cmul(iwg, fac);
        const double2 tc = csub(cmul(sp, fac), cmul(dq, p));
        const double gc = re_conj_mul(lp, tc) / rho;
        // rho: conj(lp) (-bp + q p) / rho with bp = sp / (rho c^2), q = (i w + gam) / (rho c^2)
        const double2 bp = cmul(sp, ic2);
        const double2 q = cmul(iwg, ic2);
        double gr = re_conj_mul(lp, csub(cmul(q, p), bp)) / rho;
        for (int e = 0; e < s.D; ++e) {
            // staggered rows at x and at x - e_eta share rho(x) with weight 1/2
            for (int side = 0; side < 2; ++side) {
                int j0 = i0, j1 = i1, j2 = i2;
                if (side == 1 && !s.colloc) {
                    if (e == 0) j0 = (i0 + s.n0 - 1) % s.n0;
                    else if (e == 1) j1 = (i1 + s.n1 - 1) % s.n1;
                    else j2 = (i2 + s.n2 - 1) % s.n2;
                }
                const long long j = ((long long)j2 * s.n1 + j1) * s.n0 + j0;
                const long long f = (long long)e * N + j;
                const double gs = gamma_s(s, e, j0, j1, j2);
                const double2 t = csub(g.src[f], cmul(make_double2(gs, w), g.X[f]));
                gr += 0.5 * re_conj_mul(g.L[f], t);
            }
        }
        grad_c[i] = (accumulate ? grad_c[i] : 0.0) + gc;
        grad_r[i] = (accumulate ? grad_r[i] : 0.0) + gr;
    }
}

// ---------------------------------------------------------------- field kernels
struct ScaleIn {
    int D;
    long long N;
    const double* rs[3];
    const double* kp;
    const double* et;
    double sl1, sl2;  // sqrt(lambda1), sqrt(lambda2)
};

// y = C^-1/2 s_hat,  s_hat_u = (S+ rho) s_u,  s_hat_p = s_p / (rho c^2)
// (rs sqrt(l1) = (S+ rho)/sqrt(l1);  kp sqrt(l2) (1 - i et) = 1/(rho c^2 sqrt(l2)))
__global__ void k_scale_source(ScaleIn p, const double2* __restrict__ src, double2* __restrict__ y, int adjoint)
{
    const long long total = (long long)(p.D + 1) * p.N;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total; j += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(j / p.N);
        const long long i = j - (long long)c * p.N;
        const double2 v = src[j];
        if (adjoint) {
            const double f = 1.0 / (c < p.D ? p.sl1 : p.sl2);
            y[j] = make_double2(v.x * f, v.y * f);
        } else if (c < p.D) {
            const double f = p.rs[c][i] * p.sl1;
            y[j] = make_double2(v.x * f, v.y * f);
        } else {
            const double k = p.kp[i] * p.sl2, e = p.et[i];
            // v * k (1 - i e)
            y[j] = make_double2(k * (v.x + e * v.y), k * (v.y - e * v.x));
        }
    }
}

// out = C^{mode} in with mode -1/2 (unscale) or +1/2 (physical -> scaled)
__global__ void k_scale_blocks(int D, long long N, double f1, double f2, const double2* __restrict__ in,
                               double2* __restrict__ out)
{
    const long long total = (long long)(D + 1) * N;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total; j += (long long)gridDim.x * blockDim.x) {
        const double f = (j < (long long)D * N) ? f1 : f2;
        const double2 v = in[j];
        out[j] = make_double2(v.x * f, v.y * f);
    }
}

__global__ void k_cast_64_32(const double2* __restrict__ a, float2* __restrict__ b, double s, long long n)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const double2 v = a[j];
        b[j] = make_float2((float)(v.x * s), (float)(v.y * s));
    }
}

__global__ void k_cast_32_64(const float2* __restrict__ a, double2* __restrict__ b, long long n)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const float2 v = a[j];
        b[j] = make_double2((double)v.x, (double)v.y);
    }
}

// x64 += s * x32   (refinement correction accumulated in float64)
__global__ void k_axpy_32_64(double2* __restrict__ x, const float2* __restrict__ d, double s, long long n)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const float2 v = d[j];
        double2 a = x[j];
        a.x = fma(s, (double)v.x, a.x);
        a.y = fma(s, (double)v.y, a.y);
        x[j] = a;
    }
}

// per-block partial sums of |a|^2 (grid-stride, fixed assignment -> deterministic)
__global__ void k_norm2(const double2* __restrict__ a, long long n, double* part)
{
    double s = 0.0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const double2 v = a[j];
        s += v.x * v.x + v.y * v.y;
    }
    block_sum2(s, 0.0, part + 2 * blockIdx.x);
}

// Block b: fixed-order sum of the nblk partial pairs of slot b -> out[2b], out[2b+1].
__global__ void k_reduce(const double* __restrict__ part, int nblk, double* out)
{
    const double* p = part + (long long)blockIdx.x * nblk * 2;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        a += p[2 * i];
        b += p[2 * i + 1];
    }
    block_sum2(a, b, out + 2 * blockIdx.x);
}

inline int grid_for(long long n, int threads = 256)
{
    long long g = (n + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

// ====================================================================== solver
struct cbs_solver {
    int D = 0, C = 0;
    int n[3] = {1, 1, 1};
    long long N = 0;
    double dx = 0, omega = 0;
    cbs_options opt{};
    cbs_boundary bnd{};
    double a1r = 0, a1i = 0, a2r = 0, a2i = 0, lam1 = 0, lam2 = 0;
    double t_setup_ms = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev_user = nullptr, ev0 = nullptr, ev1 = nullptr;
    std::string err = "no error";
    std::vector<void*> allocs;
    cufftHandle fft_plan = 0;  // comparison baseline only (cufft_baseline_iterate), made on first use
    bool fft_plan_ok = false;

    double *rs64[3] = {}, *kp64 = nullptr, *et64 = nullptr;
    float *rs32[3] = {}, *kp32 = nullptr, *et32 = nullptr;
    double *gc64[3] = {}, *gs64[3] = {};
    float *gc32[3] = {}, *gs32[3] = {};
    double2* kt64[3] = {};
    double* k264[3] = {};
    float2* kt32[3] = {};
    float* k232[3] = {};
    double2* tw64[3] = {};
    float2* tw32[3] = {};

    double2 *x64 = nullptr, *y64 = nullptr, *w64 = nullptr;
    float2 *x32 = nullptr, *y32 = nullptr, *w32 = nullptr;
    double* partials = nullptr;
    int npart = 0;
    int kslots = 1;             // iterations whose norm partials are kept between reductions
    double* red = nullptr;      // [2] result of the last single reduction
    double* hist = nullptr;     // [kslots][2] per-iteration (|dx|^2, |x|^2) of the last block
    double* host_red = nullptr; // pinned [kHostBuf]

    Plan<double> P64{};
    Plan<float> P32{};
    cudaGraphExec_t graph64[2] = {nullptr, nullptr};
    cudaGraphExec_t graph32[2] = {nullptr, nullptr};
    bool warmed64 = false, warmed32 = false;
    int hist_n = 0;          // entries of hist written by the last block
    int* errword = nullptr;  // device error word of the bulk-staged kernels
    cudaAccessPolicyWindow l2_window{};
    bool l2_window_set = false;
    long long launches = 0;  // kernels launched by the current call
};

namespace {

struct Fail {
    cbs_status code;
};

#define CUDA_TRY(expr)                                                                                                \
    do {                                                                                                              \
        cudaError_t e_ = (expr);                                                                                      \
        if (e_ != cudaSuccess) {                                                                                      \
            throw CudaError{e_, #expr, __LINE__};                                                                     \
        }                                                                                                             \
    } while (0)

struct CudaError {
    cudaError_t e;
    const char* what;
    int line;
};

// device memory from the caller's allocator (options.dev_alloc) or cudaMalloc
void* dev_get(cbs_solver* s, size_t bytes)
{
    void* p = nullptr;
    if (s->opt.dev_alloc) {
        p = s->opt.dev_alloc(bytes, s->opt.stream, s->opt.alloc_ctx);
        if (!p) throw Fail{CBS_ENOMEM};
        if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {
            s->opt.dev_free(p, s->opt.alloc_ctx);
            throw Fail{CBS_EINVAL};
        }
        return p;
    }
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        throw Fail{CBS_ENOMEM};
    }
    return p;
}

void dev_put(cbs_solver* s, void* p)
{
    if (s->opt.dev_free) s->opt.dev_free(p, s->opt.alloc_ctx);
    else cudaFree(p);
}

template <typename T> T* dalloc(cbs_solver* s, size_t count)
{
    if (count == 0) count = 1;
    void* p = dev_get(s, count * sizeof(T));
    s->allocs.push_back(p);
    return static_cast<T*>(p);
}

// release a set-up temporary before solver_destroy
void dfree(cbs_solver* s, void* p)
{
    auto it = std::find(s->allocs.begin(), s->allocs.end(), p);
    if (it != s->allocs.end()) {
        cudaStreamSynchronize(s->st);
        dev_put(s, p);
        s->allocs.erase(it);
    }
}

cbs_status set_err(cbs_solver* s, cbs_status code, const std::string& msg)
{
    if (s) s->err = msg;
    else g_create_error = msg;
    return code;
}

// ---------------------------------------------------------------- host tables
double layer_depth(double xi, long n, int lo, int hi)
{
    double d = 0.0;
    if (lo > 0) d = std::max(d, (lo - xi) / lo);
    if (hi > 0) d = std::max(d, (xi - (double)(n - 1 - hi)) / hi);
    return std::min(1.0, d);
}

double layer_gamma(double xi, long n, int lo, int hi, double gmax, double power)
{
    const double d = layer_depth(xi, n, lo, hi);
    return d > 0.0 ? gmax * std::pow(d, power) : 0.0;
}

template <typename T> void upload(cbs_solver* s, T* dst, const std::vector<T>& v)
{
    CUDA_TRY(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s->st));
}

// ---------------------------------------------------------------- iteration pieces
template <typename R> struct Bufs;
template <> struct Bufs<double> {
    static Plan<double>& plan(cbs_solver* s) { return s->P64; }
    static double2* x(cbs_solver* s) { return s->x64; }
    static double2* y(cbs_solver* s) { return s->y64; }
    static double2* w(cbs_solver* s) { return s->w64; }
    static cudaGraphExec_t* graph(cbs_solver* s) { return s->graph64; }
    static bool& warmed(cbs_solver* s) { return s->warmed64; }
};
template <> struct Bufs<float> {
    static Plan<float>& plan(cbs_solver* s) { return s->P32; }
    static float2* x(cbs_solver* s) { return s->x32; }
    static float2* y(cbs_solver* s) { return s->y32; }
    static float2* w(cbs_solver* s) { return s->w32; }
    static cudaGraphExec_t* graph(cbs_solver* s) { return s->graph32; }
    static bool& warmed(cbs_solver* s) { return s->warmed32; }
};

// sum the partials of `nslots` slots into out[2 * slot]
void reduce_slots(cbs_solver* s, int nblk, int nslots, double* out)
{
    k_reduce<<<nslots, 256, 0, s->st>>>(s->partials, nblk, out);
    CUDA_TRY(cudaGetLastError());
    s->launches += 1;
}

// one Born iteration on the precision-R buffers (eq. BornAlt); its norm
// partials go to slot `slot`
template <typename R> int iter_blocks(const Plan<R>& P) { return P.plane ? plane_blocks<R>(P) : rows_blocks<R>(P); }
template <typename R> int iter_kernels(const Plan<R>& P) { return P.plane ? 3 : (P.d.D == 3 ? 5 : 3); }

template <typename R> void iterate_once(cbs_solver* s, bool adj, int slot)
{
    Plan<R>& P = Bufs<R>::plan(s);
    auto x = Bufs<R>::x(s);
    auto y = Bufs<R>::y(s);
    auto w = Bufs<R>::w(s);
    const int nblk = iter_blocks<R>(P);
    if (P.plane) {  // x-y plane kernels around the last-axis symbol kernel
        CUDA_TRY(launch_plane_fwd<R>(P, x, y, w, adj, s->st));
        CUDA_TRY(launch_last<R>(P, w, adj ? SYM_GREEN_ADJ : SYM_GREEN, s->st));
        CUDA_TRY(launch_plane_inv<R>(P, x, w, adj, (R)s->opt.nu, s->partials + (size_t)slot * nblk * 2, s->st));
        s->launches += 3;
        return;
    }
    CUDA_TRY(launch_rows_fwd<R>(P, x, y, w, FWD_BORN, adj, s->st));
    if (s->D == 3) CUDA_TRY(launch_axis<R>(P, w, -1, s->st));
    CUDA_TRY(launch_last<R>(P, w, adj ? SYM_GREEN_ADJ : SYM_GREEN, s->st));
    if (s->D == 3) CUDA_TRY(launch_axis<R>(P, w, +1, s->st));
    CUDA_TRY(launch_rows_inv<R>(P, x, y, w, INV_BORN, adj, (R)s->opt.nu, s->partials + (size_t)slot * nblk * 2, s->st));
    s->launches += (s->D == 3) ? 5 : 3;
}

// n <= kslots iterations and one reduction of their norms into hist[0..n).  With fused rows the update of
// iteration k and the forward row transform of iteration k+1 are one kernel: the block launches the forward
// row kernel once, then per iteration the strided-axis / last-axis kernels and the fused row kernel, the last
// iteration ending with the plain update kernel.
template <typename R> void iterate_block(cbs_solver* s, int n, bool adj)
{
    Plan<R>& P = Bufs<R>::plan(s);
    if (P.plane || !P.fused_rows) {
        for (int k = 0; k < n; ++k) iterate_once<R>(s, adj, k);
    } else {
        auto x = Bufs<R>::x(s);
        auto y = Bufs<R>::y(s);
        auto w = Bufs<R>::w(s);
        const int nblk = rows_blocks<R>(P);
        const R nu = (R)s->opt.nu;
        CUDA_TRY(launch_rows_fwd<R>(P, x, y, w, FWD_BORN, adj, s->st));
        s->launches += 1;
        for (int k = 0; k < n; ++k) {
            if (s->D == 3) CUDA_TRY(launch_axis<R>(P, w, -1, s->st));
            CUDA_TRY(launch_last<R>(P, w, adj ? SYM_GREEN_ADJ : SYM_GREEN, s->st));
            if (s->D == 3) CUDA_TRY(launch_axis<R>(P, w, +1, s->st));
            double* part = s->partials + (size_t)k * nblk * 2;
            if (k + 1 < n) CUDA_TRY(launch_rows_inv_fwd<R>(P, x, y, w, adj, nu, part, s->st));
            else CUDA_TRY(launch_rows_inv<R>(P, x, y, w, INV_BORN, adj, nu, part, s->st));
            s->launches += (s->D == 3) ? 4 : 2;
        }
    }
    reduce_slots(s, iter_blocks<R>(P), n, s->hist);
}

// run n iterations in blocks of K = kslots; full blocks replay a captured CUDA graph
template <typename R> void run_iterations(cbs_solver* s, int n, bool adj)
{
    const int K = s->kslots;
    bool& warmed = Bufs<R>::warmed(s);
    while (n > 0) {
        const int blk = std::min(n, K);
        if (!warmed || blk < K) {
            iterate_block<R>(s, blk, adj);
            warmed = true;
        } else {
            cudaGraphExec_t& ge = Bufs<R>::graph(s)[adj ? 1 : 0];
            if (ge == nullptr) {
                cudaGraph_t g = nullptr;
                const long long l0 = s->launches;
                CUDA_TRY(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
                try {
                    iterate_block<R>(s, K, adj);
                } catch (...) {
                    cudaStreamEndCapture(s->st, &g);
                    if (g) cudaGraphDestroy(g);
                    throw;
                }
                s->launches = l0;
                CUDA_TRY(cudaStreamEndCapture(s->st, &g));
                if (s->l2_window_set) {
                    size_t nn = 0;
                    cudaGraphGetNodes(g, nullptr, &nn);
                    std::vector<cudaGraphNode_t> nodes(nn);
                    cudaGraphGetNodes(g, nodes.data(), &nn);
                    cudaKernelNodeAttrValue kv{};
                    kv.accessPolicyWindow = s->l2_window;
                    for (auto nd : nodes) {
                        cudaGraphNodeType t;
                        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                            cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributeAccessPolicyWindow, &kv);
                    }
                    cudaGetLastError();
                }
                cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                CUDA_TRY(e);
            }
            CUDA_TRY(cudaGraphLaunch(ge, s->st));
            s->launches += (long long)K * iter_kernels<R>(Bufs<R>::plan(s)) + 1;
        }
        s->hist_n = blk;
        n -= blk;
    }
}

// w <- y - A_s x (mode INV_RESID) or w <- A_s x (INV_APPLY); red = (|w|^2, |y|^2)
template <typename R> void apply_operator(cbs_solver* s, bool adj, int mode)
{
    Plan<R>& P = Bufs<R>::plan(s);
    auto x = Bufs<R>::x(s);
    auto y = Bufs<R>::y(s);
    auto w = Bufs<R>::w(s);
    CUDA_TRY(launch_rows_fwd<R>(P, x, y, w, FWD_COPY, adj, s->st));
    if (s->D == 3) CUDA_TRY(launch_axis<R>(P, w, -1, s->st));
    CUDA_TRY(launch_last<R>(P, w, adj ? SYM_L_ADJ : SYM_L, s->st));
    if (s->D == 3) CUDA_TRY(launch_axis<R>(P, w, +1, s->st));
    CUDA_TRY(launch_rows_inv<R>(P, x, y, w, mode, adj, (R)0, s->partials, s->st));
    s->launches += (s->D == 3) ? 5 : 3;
    reduce_slots(s, rows_blocks<R>(P), 1, s->red);
}

// w <- (L+I)^-1 x (or its adjoint)
template <typename R> void apply_green(cbs_solver* s, bool adj)
{
    Plan<R>& P = Bufs<R>::plan(s);
    auto x = Bufs<R>::x(s);
    auto y = Bufs<R>::y(s);
    auto w = Bufs<R>::w(s);
    CUDA_TRY(launch_rows_fwd<R>(P, x, y, w, FWD_COPY, adj, s->st));
    if (s->D == 3) CUDA_TRY(launch_axis<R>(P, w, -1, s->st));
    CUDA_TRY(launch_last<R>(P, w, adj ? SYM_GREEN_ADJ : SYM_GREEN, s->st));
    if (s->D == 3) CUDA_TRY(launch_axis<R>(P, w, +1, s->st));
    CUDA_TRY(launch_rows_inv<R>(P, x, y, w, INV_PLAIN, adj, (R)0, s->partials, s->st));
    s->launches += (s->D == 3) ? 5 : 3;
}

void read_red(cbs_solver* s, double* out2)
{
    CUDA_TRY(cudaMemcpyAsync(s->host_red, s->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CUDA_TRY(cudaStreamSynchronize(s->st));
    out2[0] = s->host_red[0];
    out2[1] = s->host_red[1];
}

// last history entry (|dx|^2, |x|^2) of the last block -> relative increment
double read_last_increment(cbs_solver* s)
{
    const int k = s->hist_n - 1;
    CUDA_TRY(cudaMemcpyAsync(s->host_red, s->hist + 2 * k, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CUDA_TRY(cudaStreamSynchronize(s->st));
    return s->host_red[1] > 0 ? std::sqrt(s->host_red[0] / s->host_red[1]) : 0.0;
}

void norm2_64(cbs_solver* s, const double2* a, long long n, double* out)
{
    const int g = std::min(grid_for(n), s->npart);
    k_norm2<<<g, 256, 0, s->st>>>(a, n, s->partials);
    CUDA_TRY(cudaGetLastError());
    s->launches += 1;
    reduce_slots(s, g, 1, s->red);
    double r[2];
    read_red(s, r);
    *out = r[0];
}

void begin_call(cbs_solver* s)
{
    cudaStream_t us = (cudaStream_t)s->opt.stream;
    CUDA_TRY(cudaEventRecord(s->ev_user, us));
    CUDA_TRY(cudaStreamWaitEvent(s->st, s->ev_user, 0));
}

ScaleIn scale_in(cbs_solver* s)
{
    ScaleIn p;
    p.D = s->D;
    p.N = s->N;
    for (int e = 0; e < 3; ++e) p.rs[e] = s->rs64[e];
    p.kp = s->kp64;
    p.et = s->et64;
    p.sl1 = std::sqrt(s->lam1);
    p.sl2 = std::sqrt(s->lam2);
    return p;
}

long long field_len(cbs_solver* s) { return (long long)s->C * s->N; }

// physical source -> y64 ; optional start field -> x64 (C^1/2 (u,p)) else 0
void prepare(cbs_solver* s, const void* src, const void* x0, bool adj)
{
    const long long n = field_len(s);
    k_scale_source<<<grid_for(n), 256, 0, s->st>>>(scale_in(s), (const double2*)src, s->y64, adj ? 1 : 0);
    CUDA_TRY(cudaGetLastError());
    s->launches += x0 ? 2 : 1;
    if (x0) {
        k_scale_blocks<<<grid_for(n), 256, 0, s->st>>>(s->D, s->N, std::sqrt(s->lam1), std::sqrt(s->lam2),
                                                       (const double2*)x0, s->x64);
        CUDA_TRY(cudaGetLastError());
    } else {
        CUDA_TRY(cudaMemsetAsync(s->x64, 0, n * sizeof(double2), s->st));
    }
}

void finish_field(cbs_solver* s, void* field)
{
    const long long n = field_len(s);
    k_scale_blocks<<<grid_for(n), 256, 0, s->st>>>(s->D, s->N, 1.0 / std::sqrt(s->lam1), 1.0 / std::sqrt(s->lam2),
                                                   s->x64, (double2*)field);
    CUDA_TRY(cudaGetLastError());
    s->launches += 1;
}

bool finite(double v) { return std::isfinite(v); }

// plain FP64 (or plain FP32) solve on the scaled variables; x64/y64 prepared
// Skips residual checks that cannot stop the iteration yet.  For the stationary Born iteration the
// residual and the increment ||x_{k+1} - x_k|| / ||x_{k+1}|| decay together once the slowest mode
// dominates, so after a check has measured the ratio residual / increment, a block whose increment
// predicts a residual above twice the target skips the check (an operator apply and a host round trip).
// A wrong prediction costs iterations, never accuracy: the loop stops only on a measured residual.
struct ResidualGate {
    double ratio = -1.0;
    bool skip(double inc, double target) const { return ratio > 0 && inc > 0 && inc * ratio > 2.0 * target; }
    void learn(double res, double inc) { ratio = (inc > 0 && res > 0) ? res / inc : -1.0; }
};

template <typename R> cbs_status solve_plain(cbs_solver* s, bool adj, cbs_info* info)
{
    const long long n = field_len(s);
    double ny2;
    norm2_64(s, s->y64, n, &ny2);
    if (!(ny2 > 0)) {  // zero source: zero field
        CUDA_TRY(cudaMemsetAsync(s->x64, 0, n * sizeof(double2), s->st));
        info->rel_residual = 0;
        return CBS_OK;
    }
    // the float32 path iterates on y / ||y|| (and x / ||y||) so that squared
    // magnitudes stay far from float32 underflow whatever the source scale
    const double ys = std::sqrt(ny2);
    if (std::is_same<R, float>::value) {
        k_cast_64_32<<<grid_for(n), 256, 0, s->st>>>(s->y64, s->y32, 1.0 / ys, n);
        k_cast_64_32<<<grid_for(n), 256, 0, s->st>>>(s->x64, s->x32, 1.0 / ys, n);
        CUDA_TRY(cudaGetLastError());
        s->launches += 2;
    }
    const double tol = s->opt.tol;
    const int maxit = s->opt.max_iter;
    int it = 0;
    double rel = 1.0, inc = 0.0;
    cbs_status st = CBS_OK;
    ResidualGate gate;
    while (it < maxit) {
        const int blk = std::min(s->opt.check_every, maxit - it);
        run_iterations<R>(s, blk, adj);
        it += blk;
        inc = read_last_increment(s);
        if (tol > 0 && finite(inc) && gate.skip(inc, tol) && it < maxit) continue;
        if (tol > 0) {
            apply_operator<R>(s, adj, INV_RESID);
            double r[2];
            read_red(s, r);
            info->residual_checks++;
            rel = std::sqrt(r[0] / r[1]);
            if (!finite(rel) || !finite(inc)) { st = CBS_EDIVERGED; break; }
            gate.learn(rel, inc);
            if (rel <= tol) break;
        } else if (!finite(inc)) {
            st = CBS_EDIVERGED;
            break;
        }
    }
    if (st == CBS_OK && tol > 0 && rel > tol) st = CBS_ENOCONV;
    if (std::is_same<R, float>::value) {
        CUDA_TRY(cudaMemsetAsync(s->x64, 0, n * sizeof(double2), s->st));
        k_axpy_32_64<<<grid_for(n), 256, 0, s->st>>>(s->x64, s->x32, ys, n);
        CUDA_TRY(cudaGetLastError());
        s->launches += 1;
    }
    info->iters = it;
    info->rel_residual = tol > 0 ? rel : -1.0;
    info->rel_increment = inc;
    return st;
}

// FP32 inner Born iterations with FP64 residual, norm and correction
// zero_start: x64 = 0 on entry, so the first residual is y itself (no float64 operator apply)
cbs_status solve_refine(cbs_solver* s, bool adj, cbs_info* info, bool zero_start)
{
    const long long n = field_len(s);
    double ny2;
    norm2_64(s, s->y64, n, &ny2);
    if (!(ny2 > 0)) {
        CUDA_TRY(cudaMemsetAsync(s->x64, 0, n * sizeof(double2), s->st));
        info->rel_residual = 0;
        return CBS_OK;
    }
    const double tol = s->opt.tol > 0 ? s->opt.tol : 1e-6;
    const int maxit = s->opt.max_iter;
    // r = y - A_s x in float64 (into w64)
    double r[2];
    double rn2 = ny2;
    if (zero_start) {
        CUDA_TRY(cudaMemcpyAsync(s->w64, s->y64, n * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
    } else {
        apply_operator<double>(s, adj, INV_RESID);
        read_red(s, r);
        info->residual_checks++;
        rn2 = r[0];
    }
    double rel = std::sqrt(rn2 / ny2), inc = 0.0;
    int it = 0, outer = 0;
    cbs_status st = CBS_OK;
    while (rel > tol && it < maxit) {
        const double rn = std::sqrt(rn2);
        // inner right-hand side r / ||r|| in float32; inner iterate from zero
        k_cast_64_32<<<grid_for(n), 256, 0, s->st>>>(s->w64, s->y32, 1.0 / rn, n);
        CUDA_TRY(cudaGetLastError());
        s->launches += 1;
        CUDA_TRY(cudaMemsetAsync(s->x32, 0, n * sizeof(float2), s->st));
        const double target = std::max(s->opt.tol_inner, 0.5 * tol / rel);
        ResidualGate gate;
        while (it < maxit) {
            const int blk = std::min(s->opt.check_every, maxit - it);
            run_iterations<float>(s, blk, adj);
            it += blk;
            inc = read_last_increment(s);
            if (!finite(inc)) { st = CBS_EDIVERGED; break; }
            if (gate.skip(inc, target) && it < maxit) continue;
            apply_operator<float>(s, adj, INV_RESID);  // inner residual (float32)
            double ri[2];
            read_red(s, ri);
            const double rr = std::sqrt(ri[0] / ri[1]);
            if (!finite(rr)) { st = CBS_EDIVERGED; break; }
            gate.learn(rr, inc);
            if (rr <= target) break;
        }
        if (st != CBS_OK) break;
        // x64 += ||r|| x32 ;  r = y - A_s x64  (float64)
        k_axpy_32_64<<<grid_for(n), 256, 0, s->st>>>(s->x64, s->x32, rn, n);
        CUDA_TRY(cudaGetLastError());
        s->launches += 1;
        apply_operator<double>(s, adj, INV_RESID);
        read_red(s, r);
        info->residual_checks++;
        rn2 = r[0];
        rel = std::sqrt(rn2 / ny2);
        ++outer;
        if (!finite(rel)) { st = CBS_EDIVERGED; break; }
    }
    if (st == CBS_OK && rel > tol) st = CBS_ENOCONV;
    info->iters = it;
    info->outer_iters = outer;
    info->rel_residual = rel;
    info->rel_increment = inc;
    return st;
}

cbs_status solve_common(cbs_solver* s, const void* src, void* field, const void* x0, cbs_info* info_out, bool adj)
{
    if (!s) return CBS_EINVAL;
    if (!src || !field) return set_err(s, CBS_EINVAL, "src and field must be device pointers");
    cbs_info info{};
    try {
        begin_call(s);
        s->launches = 0;
        CUDA_TRY(cudaEventRecord(s->ev0, s->st));
        prepare(s, src, x0, adj);
        cbs_status st;
        if (s->opt.precision == CBS_FP32_REFINE) st = solve_refine(s, adj, &info, x0 == nullptr);
        else if (s->opt.precision == CBS_FP32) st = solve_plain<float>(s, adj, &info);
        else st = solve_plain<double>(s, adj, &info);
        finish_field(s, field);
        CUDA_TRY(cudaEventRecord(s->ev1, s->st));
        int herr = 0;
        CUDA_TRY(cudaMemcpyAsync(&herr, s->errword, sizeof(int), cudaMemcpyDeviceToHost, s->st));
        CUDA_TRY(cudaStreamSynchronize(s->st));
        if (herr != 0) {
            CUDA_TRY(cudaMemsetAsync(s->errword, 0, sizeof(int), s->st));
            CUDA_TRY(cudaStreamSynchronize(s->st));
            st = herr == kErrTileAlign ? CBS_ECUDA : CBS_ETIMEOUT;
        }
        float ms = 0;
        CUDA_TRY(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
        info.t_solve_ms = ms;
        info.t_setup_ms = s->t_setup_ms;
        info.a1[0] = s->a1r; info.a1[1] = s->a1i;
        info.a2[0] = s->a2r; info.a2[1] = s->a2i;
        info.lambda1 = s->lam1;
        info.lambda2 = s->lam2;
        info.kernel_launches = s->launches;
        if (info_out) *info_out = info;
        if (st == CBS_ENOCONV) s->err = "max_iter reached before tol";
        if (st == CBS_EDIVERGED) s->err = "iteration produced a non-finite value";
        if (st == CBS_ETIMEOUT) s->err = "a bulk copy did not complete within its wait limit";
        if (herr == kErrTileAlign) s->err = "shared-memory tile not 128-byte aligned for tensor copies";
        return st;
    } catch (const CudaError& e) {
        return set_err(s, CBS_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e.e) + " in " + e.what);
    } catch (const Fail& f) {
        return set_err(s, f.code, "allocation failed");
    }
}


// Minimum enclosing circle of a small host point set (the <= 64 support points),
// by exhaustion: the smallest enclosing circle passes through two points that
// are a diameter of it, or through three, so it is the smallest circle among
// all pair-diameter circles and all three-point circumcircles that contain
// every point.  O(n^4) for n <= 64 is a few million distance tests.
double2 mec_centre(const std::vector<double2>& pts)
{
    const size_t n = pts.size();
    if (n == 0) return make_double2(0.0, 0.0);
    double best_r = INFINITY;
    double2 best = pts[0];
    auto contains_all = [&](double2 ctr, double r) {
        const double lim = r * (1.0 + 1e-9);
        for (const double2& p : pts)
            if (std::hypot(p.x - ctr.x, p.y - ctr.y) > lim) return false;
        return true;
    };
    auto consider = [&](double2 ctr, double r) {
        if (r < best_r && contains_all(ctr, r)) { best_r = r; best = ctr; }
    };
    if (n == 1) return pts[0];
    for (size_t i = 0; i < n; ++i)
        for (size_t j = i + 1; j < n; ++j)
            consider(make_double2(0.5 * (pts[i].x + pts[j].x), 0.5 * (pts[i].y + pts[j].y)),
                     0.5 * std::hypot(pts[j].x - pts[i].x, pts[j].y - pts[i].y));
    for (size_t i = 0; i < n; ++i)
        for (size_t j = i + 1; j < n; ++j)
            for (size_t k = j + 1; k < n; ++k) {
                // centre o = p_i + u with 2 (p_j - p_i).u = |p_j - p_i|^2 and 2 (p_k - p_i).u = |p_k - p_i|^2
                const double bx = pts[j].x - pts[i].x, by = pts[j].y - pts[i].y;
                const double cx = pts[k].x - pts[i].x, cy = pts[k].y - pts[i].y;
                const double det = 2.0 * (bx * cy - by * cx);
                const double scale = (bx * bx + by * by) + (cx * cx + cy * cy);
                if (!(std::fabs(det) > 1e-14 * scale)) continue;  // (nearly) collinear: a pair circle covers it
                const double bb = bx * bx + by * by, cc = cx * cx + cy * cy;
                const double ux = (bb * cy - cc * by) / det, uy = (bx * cc - cx * bb) / det;
                consider(make_double2(pts[i].x + ux, pts[i].y + uy), std::hypot(ux, uy));
            }
    return best;
}

// centre of the minimum enclosing circle of the support points of a device value set
double2 support_mec(cbs_solver* s, const double2* vals, long long n)
{
    const int g = grid_for(n, kSetupThreads);
    double2* best = dalloc<double2>(s, (size_t)g * kSupportDirs);
    k_setup_support<<<g, kSetupThreads, 0, s->st>>>(vals, n, best);
    CUDA_TRY(cudaGetLastError());
    std::vector<double2> hb((size_t)g * kSupportDirs);
    CUDA_TRY(cudaMemcpyAsync(hb.data(), best, hb.size() * sizeof(double2), cudaMemcpyDeviceToHost, s->st));
    CUDA_TRY(cudaStreamSynchronize(s->st));
    dfree(s, best);
    std::vector<double2> pts;
    for (int k = 0; k < kSupportDirs; ++k) {
        const double ck = std::cos(2.0 * kPi * k / kSupportDirs), sk = std::sin(2.0 * kPi * k / kSupportDirs);
        double bp = -INFINITY;
        double2 bv = make_double2(NAN, NAN);
        for (int b = 0; b < g; ++b) {
            const double2 v = hb[(size_t)b * kSupportDirs + k];
            if (std::isnan(v.x)) continue;
            const double p = v.x * ck + v.y * sk;
            if (p > bp) { bp = p; bv = v; }
        }
        if (!std::isnan(bv.x)) pts.push_back(bv);
    }
    return mec_centre(pts);
}

// Solvers holding a persisting-L2 window, and the context's persisting-L2 limit before the first of them
// raised it: when the last one is destroyed the persisting lines are reset and the limit restored, so the
// set-aside part of L2 does not stay reserved for kernels that no longer run.
std::mutex g_l2_mu;
int g_l2_users = 0;
size_t g_l2_limit0 = 0;

// Keep the float32 work array resident in L2 across the five kernels of an
// iteration: an access-policy window marks it persisting (the others stream).
// The persisting-L2 limit is a property of this process's CUDA context (it
// ends with the context); it is raised only up to the device maximum.
void set_l2_window(cbs_solver* s, void* base, size_t bytes)
{
    int dev = 0, max_persist = 0, max_window = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev);
    cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev);
    if (max_persist <= 0 || max_window <= 0) return;
    // Only a field that fits in the persisting carve-out gets a window.  A window over a larger field
    // marks most of its accesses streaming (evict first) and measured 1.7-1.9x slower per iteration
    // on GB300 at 256^3 and 512^3; at 128^3 (67 MB) the window makes an iteration 7 % faster.
    if (bytes > (size_t)max_persist || bytes > (size_t)max_window) return;
    const size_t win = bytes;
    size_t cur = 0;
    {
        std::lock_guard<std::mutex> lk(g_l2_mu);
        cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
        if (g_l2_users == 0) g_l2_limit0 = cur;
        ++g_l2_users;
        if (cur < std::min(win, (size_t)max_persist))
            cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, std::min(win, (size_t)max_persist));
        cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    }
    cudaStreamAttrValue v{};
    v.accessPolicyWindow.base_ptr = base;
    v.accessPolicyWindow.num_bytes = win;
    v.accessPolicyWindow.hitRatio = (float)std::min(1.0, (double)cur / (double)win);
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cudaStreamSetAttribute(s->st, cudaStreamAttributeAccessPolicyWindow, &v);
    s->l2_window = v.accessPolicyWindow;
    s->l2_window_set = true;
    TRACE("L2 window %zu bytes, persisting limit %zu, hit ratio %f", win, cur, v.accessPolicyWindow.hitRatio);
    cudaGetLastError();
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against the driver library)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// Tensor-copy descriptor of the float32 work field for the tile-staged last-axis kernel: the field
// [C][n2][n1][n0] seen as {n0, n1, C*n2} 8-byte elements, box {COLS, 1, n2}.  The tile kernel is
// opt-in (environment variable CBS_TILE_LAST): on GB300 it measured no faster than the register
// kernel (41.0 us at 128^3) and slower at 64^3 and 256^3.  Leaves tile_field null (register kernel)
// when not asked for, when the sizes do not qualify, or when the descriptor cannot be made.
template <typename R> void fill_tile_map(cbs_solver* s, Plan<R>& P, const void* field)
{
    P.tile_field = nullptr;
    const int n2 = s->n[2];
    if (s->D != 3 || field == nullptr || !tile_ok<R>(n2) || s->n[0] % cols_tile<R>(n2) != 0) return;
    if (std::getenv("CBS_TILE_LAST") == nullptr) return;
    auto enc = tensor_map_encoder();
    if (!enc) return;
    const cuuint64_t gdim[3] = {(cuuint64_t)s->n[0], (cuuint64_t)s->n[1], (cuuint64_t)s->C * n2};
    const cuuint64_t gstride[2] = {(cuuint64_t)s->n[0] * sizeof(cplx<R>),
                                   (cuuint64_t)s->n[0] * s->n[1] * sizeof(cplx<R>)};
    const cuuint32_t box[3] = {(cuuint32_t)cols_tile<R>(n2), 1u, (cuuint32_t)n2};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    static_assert(sizeof(cplx<R>) == 8, "the descriptor treats one complex value as one 8-byte element");
    const CUresult r = enc(&P.tmap_last, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(field), gdim, gstride,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS) P.tile_field = field;
    TRACE("tile map for the last axis: %s", r == CUDA_SUCCESS ? "yes" : "no");
}

// The float32 last-axis step runs on a cluster of C CTAs (one component each) for 2D grids whose last axis
// has 2048 points: measured on GB300, 2048^2 takes 142.5 instead of 170.7 us (8-column tiles, 64-byte rows,
// instead of 2-column tiles holding all three components).  Elsewhere the one-CTA kernel is faster (128^3:
// 37.9 against 53.5 us; 512^3: 3.25 against 4.26 ms; 1024^2: 32.9 against 34.9 us).  CBS_LAST_CLUSTER=1 /
// =0 forces it on (extents 64 .. 2048) / off.
bool last_cluster_preferred(const cbs_solver* s)
{
    const int nl = s->n[s->D - 1];
    if (!last_cluster_ok<float>(nl)) return false;
    const char* e = std::getenv("CBS_LAST_CLUSTER");
    if (e != nullptr) return e[0] == '1';
    return s->D == 2 && nl >= 2048;
}

// Tensor-copy descriptor and persistent grid of the pipelined strided-axis kernel (3D float32, n1 <= 256,
// n0 % COLS == 0): the field as {n0, n1, C*n2} 8-byte elements, box {COLS, n1, 1}.  Opt-in with
// CBS_AXIS_PIPE=1.
template <typename R> void fill_axis_map(cbs_solver* s, Plan<R>& P, const void* field)
{
    P.axis_field = nullptr;
    P.axis_grid = 0;
    const int n1 = s->n[1];
    if (s->D != 3 || field == nullptr || !axis_pipe_ok<R>(n1) || s->n[0] % cols_axis<R>(n1) != 0) return;
    if (std::getenv("CBS_AXIS_PIPE") == nullptr) return;
    auto enc = tensor_map_encoder();
    if (!enc) return;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const int per_sm = axis_pipe_blocks_per_sm<R>(n1);
    if (per_sm <= 0) return;
    const cuuint64_t gdim[3] = {(cuuint64_t)s->n[0], (cuuint64_t)n1, (cuuint64_t)s->C * s->n[2]};
    const cuuint64_t gstride[2] = {(cuuint64_t)s->n[0] * sizeof(cplx<R>), (cuuint64_t)s->n[0] * n1 * sizeof(cplx<R>)};
    const cuuint32_t box[3] = {(cuuint32_t)cols_axis<R>(n1), (cuuint32_t)n1, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = enc(&P.tmap_axis, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(field), gdim, gstride,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return;
    P.axis_field = field;
    P.axis_grid = sms * per_sm;
    TRACE("pipelined axis kernel: %d CTAs", P.axis_grid);
}

template <typename R> void fill_plan(cbs_solver* s, Plan<R>& P)
{
    P.d.D = s->D;
    P.d.n0 = s->n[0];
    P.d.n1 = s->n[1];
    P.d.n2 = s->n[2];
    P.d.N = s->N;
    const bool f = std::is_same<R, float>::value;
    for (int e = 0; e < 3; ++e) {
        P.M.rs[e] = f ? (const R*)s->rs32[e] : (const R*)s->rs64[e];
        P.M.gc[e] = f ? (const R*)s->gc32[e] : (const R*)s->gc64[e];
        P.M.gs[e] = f ? (const R*)s->gs32[e] : (const R*)s->gs64[e];
        P.Sy.kt[e] = f ? (const cplx<R>*)s->kt32[e] : (const cplx<R>*)s->kt64[e];
        P.Sy.k2[e] = f ? (const R*)s->k232[e] : (const R*)s->k264[e];
        P.tw[e] = f ? (const cplx<R>*)s->tw32[e] : (const cplx<R>*)s->tw64[e];
    }
    P.M.kp = f ? (const R*)s->kp32 : (const R*)s->kp64;
    P.M.et = f ? (const R*)s->et32 : (const R*)s->et64;
    P.M.omega = (R)s->omega;
    P.M.a1r = (R)(s->a1r / s->lam1);
    P.M.a1i = (R)(s->a1i / s->lam1);
    P.M.a2r = (R)(s->a2r / s->lam2);
    P.M.a2i = (R)(s->a2i / s->lam2);
    // symbol constants (App. B.1 with a = a1, lambda_0 = lambda1, b = a2, lambda_1 = lambda2)
    const double l1 = s->lam1, l2 = s->lam2;
    const double apr = s->a1r + l1, api = s->a1i;   // a1 + lambda1
    const double bpr = s->a2r + l2, bpi = s->a2i;   // a2 + lambda2
    const double den = apr * apr + api * api;
    const double Pr = l1 * apr / den, Pi = -l1 * api / den;  // lambda1 / (a1 + lambda1)
    const double scale = 1.0 / (double)s->N;
    const double sq = std::sqrt(l1 * l2);
    P.Sy.Pu = mk<cplx<R>, R>((R)Pr, (R)Pi);
    P.Sy.P = mk<cplx<R>, R>((R)(Pr * scale), (R)(Pi * scale));
    P.Sy.c1 = mk<cplx<R>, R>((R)0, (R)sq);
    P.Sy.c2 = mk<cplx<R>, R>((R)(l2 * apr), (R)(l2 * api));
    P.Sy.c3 = mk<cplx<R>, R>((R)(apr * bpr - api * bpi), (R)(apr * bpi + api * bpr));
    P.Sy.la1 = mk<cplx<R>, R>((R)(s->a1r / l1), (R)(s->a1i / l1));
    P.Sy.la2 = mk<cplx<R>, R>((R)(s->a2r / l2), (R)(s->a2i / l2));
    P.Sy.isq = (R)(1.0 / sq);
    P.Sy.scale = (R)scale;
}

// Failure-detection self-test: thread 0 arms the barrier for two elements but
// the bulk copy sends one, so the phase never completes.  The bounded wait
// gives up after `limit` rounds, the kernel records the timeout in the error
// word and returns; nothing faults and the context stays usable.  The one copy
// that was issued has landed by then (16 bytes from device memory).
__global__ void k_selftest_bulk_timeout(const double2* src, int* err, int* out, int limit)
{
    __shared__ __align__(128) double2 buf[2];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar, 2 * sizeof(double2));
        bulk_g2s(buf, src, sizeof(double2), &bar);
    }
    const bool ok = mbar_wait_bounded(&bar, 0, limit);
    if (threadIdx.x == 0) {
        if (!ok) atomicExch(err, kErrBulkTimeout);
        out[0] = ok ? 0 : 1;
    }
}

}  // namespace

namespace cbs {
// lets other translation units of the library report through cbs_last_error(NULL)
void set_create_error(const std::string& msg) { g_create_error = msg; }
}  // namespace cbs

// ====================================================================== C ABI
extern "C" {

const char* cbs_last_error(const cbs_solver* s) { return s ? s->err.c_str() : g_create_error.c_str(); }

void solver_destroy(cbs_solver* s)
{
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    // the last solver holding a window resets the persisting lines and restores the persisting-L2 limit, so the
    // set-aside part of L2 is not kept from the process's later kernels
    if (s->l2_window_set) {
        std::lock_guard<std::mutex> lk(g_l2_mu);
        if (--g_l2_users == 0) {
            cudaCtxResetPersistingL2Cache();
            cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_l2_limit0);
        }
        cudaGetLastError();
    }
    for (int a = 0; a < 2; ++a) {
        if (s->graph64[a]) cudaGraphExecDestroy(s->graph64[a]);
        if (s->graph32[a]) cudaGraphExecDestroy(s->graph32[a]);
    }
    if (s->fft_plan_ok) cufftDestroy(s->fft_plan);
    for (void* p : s->allocs) dev_put(s, p);
    pinned_put(s->host_red);
    if (s->ev_user) cudaEventDestroy(s->ev_user);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
}

cbs_status solver_create(const cbs_grid* grid, double dx, double omega, const double* c0, const double* rho,
                         const double* alpha, const cbs_boundary* boundary, const cbs_options* opt, cbs_solver** out)
{
    if (!out) return set_err(nullptr, CBS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !c0 || !rho || !alpha) return set_err(nullptr, CBS_EINVAL, "NULL grid or medium pointer");
    if (grid->ndim != 2 && grid->ndim != 3) return set_err(nullptr, CBS_EINVAL, "ndim must be 2 or 3");
    for (int a = 0; a < grid->ndim; ++a)
        if (!size_supported(grid->n[a]))
            return set_err(nullptr, CBS_EINVAL, "unsupported extent " + std::to_string((long long)grid->n[a]));
    if (!(dx > 0) || !(omega > 0) || !std::isfinite(dx) || !std::isfinite(omega))
        return set_err(nullptr, CBS_EINVAL, "dx and omega must be positive");
    cbs_options o{};
    if (opt) o = *opt;
    if (o.nu == 0) o.nu = 0.8;
    if (o.beta == 0) o.beta = 0.95;
    if (o.tol_inner == 0) o.tol_inner = 1e-4;
    if (o.max_iter == 0) o.max_iter = 100000;
    if (o.check_every <= 0) o.check_every = 50;
    if (!(o.nu > 0 && o.nu < 1) || !(o.beta > 0 && o.beta < 1))
        return set_err(nullptr, CBS_EINVAL, "nu and beta must lie in (0, 1)");
    if (o.precision < CBS_FP64 || o.precision > CBS_FP32) return set_err(nullptr, CBS_EINVAL, "bad precision");
    if (o.grid_kind != CBS_GRID_STAGGERED && o.grid_kind != CBS_GRID_COLLOCATED)
        return set_err(nullptr, CBS_EINVAL, "bad grid kind");
    if (o.shift_rule != CBS_SHIFT_MIDRANGE && o.shift_rule != CBS_SHIFT_MEDIAN && o.shift_rule != CBS_SHIFT_MEC)
        return set_err(nullptr, CBS_EINVAL, "bad shift rule");
    if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr))
        return set_err(nullptr, CBS_EINVAL, "dev_alloc and dev_free must be set together");
    cbs_boundary b{};
    if (boundary) b = *boundary;
    if (b.power == 0) b.power = 2.0;
    if (!(b.gamma_max >= 0) || !std::isfinite(b.gamma_max)) return set_err(nullptr, CBS_EINVAL, "bad gamma_max");
    for (int a = 0; a < grid->ndim; ++a)
        for (int k = 0; k < 2; ++k)
            if (b.n_abs[a][k] < 0 || b.n_abs[a][k] >= grid->n[a])
                return set_err(nullptr, CBS_EINVAL, "bad absorbing layer width");

    cbs_solver* s = new cbs_solver();
    s->D = grid->ndim;
    s->C = s->D + 1;
    for (int a = 0; a < s->D; ++a) s->n[a] = (int)grid->n[a];
    s->N = (long long)s->n[0] * s->n[1] * s->n[2];
    s->dx = dx;
    s->omega = omega;
    s->opt = o;
    s->bnd = b;
    try {
        TRACE("create: stream");
        CUDA_TRY(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
        TRACE("create: events");
        CUDA_TRY(cudaEventCreateWithFlags(&s->ev_user, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreate(&s->ev0));
        CUDA_TRY(cudaEventCreate(&s->ev1));
        s->host_red = pinned_get();
        if (!s->host_red) throw CudaError{cudaErrorMemoryAllocation, "cudaMallocHost", __LINE__};
        TRACE("create: begin_call");
        begin_call(s);
        TRACE("create: tables");
        CUDA_TRY(cudaEventRecord(s->ev0, s->st));
        const long long N = s->N;
        const int D = s->D;
        // per-axis tables (host, float64): gamma, wavenumbers, twiddles
        for (int a = 0; a < 3; ++a) {
            const int n = s->n[a];
            std::vector<double> gc(n, 0.0), gs(n, 0.0), k2(n, 0.0);
            std::vector<double2> kt(n), tw(n);
            std::vector<float> gc32(n), gs32(n), k232(n);
            std::vector<float2> kt32(n), tw32(n);
            for (int i = 0; i < n; ++i) {
                const bool colloc = o.grid_kind == CBS_GRID_COLLOCATED;
                if (a < D) {
                    gc[i] = layer_gamma((double)i, n, b.n_abs[a][0], b.n_abs[a][1], b.gamma_max, b.power);
                    gs[i] = colloc ? gc[i] : layer_gamma(i + 0.5, n, b.n_abs[a][0], b.n_abs[a][1], b.gamma_max, b.power);
                }
                const int f = (i < (n + 1) / 2) ? i : i - n;
                const double k = 2.0 * kPi * f / (n * dx);
                // t = k e^{i k dx/2} (staggered derivative symbol / i), or k on the collocated grid
                kt[i] = colloc ? make_double2(k, 0.0) : make_double2(k * std::cos(k * dx / 2), k * std::sin(k * dx / 2));
                k2[i] = k * k;
                const double ang = -2.0 * kPi * (double)i / (double)n;
                tw[i] = make_double2(std::cos(ang), std::sin(ang));
                gc32[i] = (float)gc[i];
                gs32[i] = (float)gs[i];
                k232[i] = (float)k2[i];
                kt32[i] = make_float2((float)kt[i].x, (float)kt[i].y);
                tw32[i] = make_float2((float)tw[i].x, (float)tw[i].y);
            }
            s->gc64[a] = dalloc<double>(s, n); upload(s, s->gc64[a], gc);
            s->gs64[a] = dalloc<double>(s, n); upload(s, s->gs64[a], gs);
            s->k264[a] = dalloc<double>(s, n); upload(s, s->k264[a], k2);
            s->kt64[a] = dalloc<double2>(s, n); upload(s, s->kt64[a], kt);
            s->tw64[a] = dalloc<double2>(s, n); upload(s, s->tw64[a], tw);
            s->gc32[a] = dalloc<float>(s, n); upload(s, s->gc32[a], gc32);
            s->gs32[a] = dalloc<float>(s, n); upload(s, s->gs32[a], gs32);
            s->k232[a] = dalloc<float>(s, n); upload(s, s->k232[a], k232);
            s->kt32[a] = dalloc<float2>(s, n); upload(s, s->kt32[a], kt32);
            s->tw32[a] = dalloc<float2>(s, n); upload(s, s->tw32[a], tw32);
            CUDA_TRY(cudaStreamSynchronize(s->st));  // host vectors go out of scope
        }
        SetupIn si;
        si.colloc = o.grid_kind == CBS_GRID_COLLOCATED ? 1 : 0;
        si.D = D; si.n0 = s->n[0]; si.n1 = s->n[1]; si.n2 = s->n[2]; si.N = N; si.omega = omega;
        si.c0 = c0; si.rho = rho; si.alpha = alpha;
        for (int a = 0; a < 3; ++a) { si.gc[a] = s->gc64[a]; si.gs[a] = s->gs64[a]; }
        TRACE("create: minmax");
        const int sg = grid_for(N, kSetupThreads);
        double* part = dalloc<double>(s, (size_t)sg * 8);
        int* bad = dalloc<int>(s, 1);
        CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s->st));
        k_setup_minmax<<<sg, kSetupThreads, 0, s->st>>>(si, part, bad);
        CUDA_TRY(cudaGetLastError());
        std::vector<double> hp((size_t)sg * 8);
        int hbad = 0;
        CUDA_TRY(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
        CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s->st));
        CUDA_TRY(cudaStreamSynchronize(s->st));
        TRACE("create: minmax done bad=%d", hbad);
        if (hbad) {
            solver_destroy(s);
            return set_err(nullptr, CBS_EINVAL, "medium rejected: non-finite value, c0 <= 0, rho <= 0 or alpha < 0");
        }
        if (o.shift_rule == CBS_SHIFT_MIDRANGE) {
            double mm[8] = {INFINITY, -INFINITY, INFINITY, -INFINITY, INFINITY, -INFINITY, INFINITY, -INFINITY};
            for (int bi = 0; bi < sg; ++bi)
                for (int k = 0; k < 8; ++k)
                    mm[k] = (k & 1) ? std::max(mm[k], hp[bi * 8 + k]) : std::min(mm[k], hp[bi * 8 + k]);
            s->a1r = 0.5 * (mm[0] + mm[1]);
            s->a1i = 0.5 * (mm[2] + mm[3]);
            s->a2r = 0.5 * (mm[4] + mm[5]);
            s->a2i = 0.5 * (mm[6] + mm[7]);
        } else if (o.shift_rule == CBS_SHIFT_MEC) {
            double2* dv = dalloc<double2>(s, (size_t)D * N);
            double2* qv = dalloc<double2>(s, (size_t)N);
            k_setup_values<<<sg, kSetupThreads, 0, s->st>>>(si, dv, qv);
            CUDA_TRY(cudaGetLastError());
            const double2 c1 = support_mec(s, dv, (long long)D * N);
            const double2 c2 = support_mec(s, qv, (long long)N);
            s->a1r = c1.x; s->a1i = c1.y; s->a2r = c2.x; s->a2i = c2.y;
            dfree(s, dv);
            dfree(s, qv);
        } else {
            double2* dv = dalloc<double2>(s, (size_t)D * N);
            double2* qv = dalloc<double2>(s, (size_t)N);
            k_setup_values<<<sg, kSetupThreads, 0, s->st>>>(si, dv, qv);
            CUDA_TRY(cudaGetLastError());
            std::vector<double2> hd((size_t)D * N), hq((size_t)N);
            CUDA_TRY(cudaMemcpyAsync(hd.data(), dv, hd.size() * sizeof(double2), cudaMemcpyDeviceToHost, s->st));
            CUDA_TRY(cudaMemcpyAsync(hq.data(), qv, hq.size() * sizeof(double2), cudaMemcpyDeviceToHost, s->st));
            CUDA_TRY(cudaStreamSynchronize(s->st));
            auto median = [](std::vector<double>& v) {
                const size_t m = v.size();
                std::sort(v.begin(), v.end());
                return (m % 2) ? v[m / 2] : 0.5 * (v[m / 2 - 1] + v[m / 2]);
            };
            std::vector<double> re, im;
            re.reserve(hd.size()); im.reserve(hd.size());
            for (auto& z : hd) { re.push_back(z.x); im.push_back(z.y); }
            s->a1r = median(re); s->a1i = median(im);
            re.clear(); im.clear();
            for (auto& z : hq) { re.push_back(z.x); im.push_back(z.y); }
            s->a2r = median(re); s->a2i = median(im);
            dfree(s, dv);
            dfree(s, qv);
        }
        TRACE("create: maxdev");
        k_setup_maxdev<<<sg, kSetupThreads, 0, s->st>>>(si, make_double2(s->a1r, s->a1i), make_double2(s->a2r, s->a2i), part);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(hp.data(), part, (size_t)sg * 2 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
        CUDA_TRY(cudaStreamSynchronize(s->st));
        double m1 = 0, m2 = 0;
        for (int bi = 0; bi < sg; ++bi) { m1 = std::max(m1, hp[bi * 2]); m2 = std::max(m2, hp[bi * 2 + 1]); }
        s->lam1 = m1 > 0 ? m1 / o.beta : std::hypot(s->a1r, s->a1i);
        s->lam2 = m2 > 0 ? m2 / o.beta : std::hypot(s->a2r, s->a2i);
        if (!(s->lam1 > 0) || !(s->lam2 > 0) || !std::isfinite(s->lam1) || !std::isfinite(s->lam2)) {
            solver_destroy(s);
            return set_err(nullptr, CBS_EINVAL, "degenerate scaling: a diagonal block is identically zero");
        }
        TRACE("create: store lam1=%g lam2=%g", s->lam1, s->lam2);
        for (int e = 0; e < 3; ++e) {
            s->rs64[e] = dalloc<double>(s, e < D ? N : 1);
            s->rs32[e] = dalloc<float>(s, e < D ? N : 1);
        }
        s->kp64 = dalloc<double>(s, N); s->et64 = dalloc<double>(s, N);
        s->kp32 = dalloc<float>(s, N); s->et32 = dalloc<float>(s, N);
        k_setup_store<<<sg, kSetupThreads, 0, s->st>>>(si, 1.0 / s->lam1, 1.0 / s->lam2, s->rs64[0], s->rs64[1],
                                                       s->rs64[2], s->kp64, s->et64, s->rs32[0], s->rs32[1],
                                                       s->rs32[2], s->kp32, s->et32);
        CUDA_TRY(cudaGetLastError());
        // working fields
        const long long n = (long long)s->C * N;
        s->x64 = dalloc<double2>(s, n);
        s->y64 = dalloc<double2>(s, n);
        s->w64 = dalloc<double2>(s, n);
        if (o.precision != CBS_FP64) {
            s->x32 = dalloc<float2>(s, n);
            s->y32 = dalloc<float2>(s, n);
            s->w32 = dalloc<float2>(s, n);
            if (std::getenv("CBS_NO_L2_WINDOW") == nullptr) set_l2_window(s, s->w32, (size_t)n * sizeof(float2));
        }
        TRACE("create: plans");
        fill_plan<double>(s, s->P64);
        fill_plan<float>(s, s->P32);
        fill_tile_map<float>(s, s->P32, s->w32);
        fill_axis_map<float>(s, s->P32, s->w32);
        // CBS_PLANE=1 / CBS_NO_PLANE=1 force the plane kernels on (where they exist) / off
        s->P32.plane = o.precision != CBS_FP64 && std::getenv("CBS_NO_PLANE") == nullptr &&
                       (std::getenv("CBS_PLANE") != nullptr ? plane_ok<float>(s->P32) : plane_preferred<float>(s->P32));
        s->P32.last_cluster = o.precision != CBS_FP64 && last_cluster_preferred(s);
        // CBS_PLANE_CL=4: four CTAs per x-y plane (quarter planes) in place of a pair
        {
            const char* e = std::getenv("CBS_PLANE_CL");
            s->P32.plane_cl = (e != nullptr && e[0] == '4') ? 4 : 2;
        }
        const int nb = std::max(std::max(rows_blocks<double>(s->P64), rows_blocks<float>(s->P32)),
                                std::max(grid_for(n), plane_blocks<float>(s->P32)));
        s->npart = nb;
        s->kslots = std::min(o.check_every, kHostBuf / 2);
        TRACE("create: partials %d x %d", nb, s->kslots);
        s->partials = dalloc<double>(s, (size_t)nb * 2 * s->kslots);
        s->red = dalloc<double>(s, 2);
        s->hist = dalloc<double>(s, (size_t)s->kslots * 2);
        s->errword = dalloc<int>(s, 1);
        CUDA_TRY(cudaMemsetAsync(s->errword, 0, sizeof(int), s->st));
        s->P64.err = s->errword;
        s->P32.err = s->errword;
        // one kernel for the update of an iteration and the forward row transform of the next, where the rows
        // are bulk-staged; CBS_NO_FUSED_ROWS=1 keeps them apart
        {
            const bool off = std::getenv("CBS_NO_FUSED_ROWS") != nullptr;
            s->P64.fused_rows = !off && fused_rows_ok<double>(s->P64);
            s->P32.fused_rows = !off && o.precision != CBS_FP64 && fused_rows_ok<float>(s->P32);
            const char* v = std::getenv("CBS_FUSED_VAR");  // measured variants of the fused row kernel
            s->P32.fused_var = (v != nullptr && ((v[0] >= '0' && v[0] <= '3') || v[0] == '6')) ? v[0] - '0' : -1;
        }
        CUDA_TRY(cudaEventRecord(s->ev1, s->st));
        CUDA_TRY(cudaStreamSynchronize(s->st));
        float ms = 0;
        CUDA_TRY(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
        s->t_setup_ms = ms;
    } catch (const CudaError& e) {
        std::string msg = std::string("CUDA error ") + cudaGetErrorString(e.e) + " in " + e.what;
        solver_destroy(s);
        return set_err(nullptr, CBS_ECUDA, msg);
    } catch (const Fail& f) {
        solver_destroy(s);
        return set_err(nullptr, f.code, f.code == CBS_EINVAL ? "dev_alloc returned memory not aligned to 256 bytes"
                                                             : "device allocation failed");
    }
    *out = s;
    return CBS_OK;
}

cbs_status solve_forward(cbs_solver* s, const void* src, void* field, const void* x0, cbs_info* info)
{
    return solve_common(s, src, field, x0, info, false);
}

cbs_status solve_adjoint(cbs_solver* s, const void* src, void* field, const void* x0, cbs_info* info)
{
    return solve_common(s, src, field, x0, info, true);
}

cbs_status residual_norm(cbs_solver* s, const void* field, const void* src, int adjoint, double* rel)
{
    if (!s) return CBS_EINVAL;
    if (!field || !src || !rel) return set_err(s, CBS_EINVAL, "NULL argument");
    try {
        begin_call(s);
        prepare(s, src, field, adjoint != 0);
        apply_operator<double>(s, adjoint != 0, INV_RESID);
        double r[2];
        read_red(s, r);
        *rel = r[1] > 0 ? std::sqrt(r[0] / r[1]) : 0.0;
        return CBS_OK;
    } catch (const CudaError& e) {
        return set_err(s, CBS_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e.e) + " in " + e.what);
    }
}

cbs_status born_iterate(cbs_solver* s, const void* y, void* x, int n_iter, int adjoint, double* incr)
{
    if (!s) return CBS_EINVAL;
    if (!y || !x || n_iter < 0) return set_err(s, CBS_EINVAL, "bad argument");
    try {
        begin_call(s);
        const long long n = field_len(s);
        const bool f32 = s->opt.precision != CBS_FP64;
        if (f32) {
            k_cast_64_32<<<grid_for(n), 256, 0, s->st>>>((const double2*)y, s->y32, 1.0, n);
            k_cast_64_32<<<grid_for(n), 256, 0, s->st>>>((const double2*)x, s->x32, 1.0, n);
            CUDA_TRY(cudaGetLastError());
        } else {
            CUDA_TRY(cudaMemcpyAsync(s->y64, y, n * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
            CUDA_TRY(cudaMemcpyAsync(s->x64, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
        }
        int done = 0;
        while (done < n_iter) {
            const int blk = std::min(s->kslots, n_iter - done);
            if (f32) iterate_block<float>(s, blk, adjoint != 0);
            else iterate_block<double>(s, blk, adjoint != 0);
            if (incr) {
                CUDA_TRY(cudaMemcpyAsync(s->host_red, s->hist, 2 * blk * sizeof(double), cudaMemcpyDeviceToHost, s->st));
                CUDA_TRY(cudaStreamSynchronize(s->st));
                for (int k = 0; k < blk; ++k) {
                    const double a = s->host_red[2 * k], b = s->host_red[2 * k + 1];
                    incr[done + k] = b > 0 ? std::sqrt(a / b) : 0.0;
                }
            }
            done += blk;
        }
        if (f32) k_cast_32_64<<<grid_for(n), 256, 0, s->st>>>(s->x32, (double2*)x, n);
        else CUDA_TRY(cudaMemcpyAsync(x, s->x64, n * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaStreamSynchronize(s->st));
        return CBS_OK;
    } catch (const CudaError& e) {
        return set_err(s, CBS_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e.e) + " in " + e.what);
    }
}

cbs_status green_apply(cbs_solver* s, const void* in, void* out, int adjoint)
{
    if (!s) return CBS_EINVAL;
    if (!in || !out) return set_err(s, CBS_EINVAL, "NULL argument");
    try {
        begin_call(s);
        const long long n = field_len(s);
        if (s->opt.precision != CBS_FP64) {
            k_cast_64_32<<<grid_for(n), 256, 0, s->st>>>((const double2*)in, s->x32, 1.0, n);
            CUDA_TRY(cudaGetLastError());
            apply_green<float>(s, adjoint != 0);
            k_cast_32_64<<<grid_for(n), 256, 0, s->st>>>(s->w32, (double2*)out, n);
            CUDA_TRY(cudaGetLastError());
        } else {
            CUDA_TRY(cudaMemcpyAsync(s->x64, in, n * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
            apply_green<double>(s, adjoint != 0);
            CUDA_TRY(cudaMemcpyAsync(out, s->w64, n * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
        }
        CUDA_TRY(cudaStreamSynchronize(s->st));
        return CBS_OK;
    } catch (const CudaError& e) {
        return set_err(s, CBS_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e.e) + " in " + e.what);
    }
}

cbs_status operator_apply(cbs_solver* s, const void* x, void* out, int adjoint)
{
    if (!s) return CBS_EINVAL;
    if (!x || !out) return set_err(s, CBS_EINVAL, "NULL argument");
    try {
        begin_call(s);
        const long long n = field_len(s);
        CUDA_TRY(cudaMemcpyAsync(s->x64, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
        apply_operator<double>(s, adjoint != 0, INV_APPLY);
        CUDA_TRY(cudaMemcpyAsync(out, s->w64, n * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
        CUDA_TRY(cudaStreamSynchronize(s->st));
        return CBS_OK;
    } catch (const CudaError& e) {
        return set_err(s, CBS_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e.e) + " in " + e.what);
    }
}

cbs_status scale_source(cbs_solver* s, const void* src, void* y, int adjoint)
{
    if (!s) return CBS_EINVAL;
    if (!src || !y) return set_err(s, CBS_EINVAL, "NULL argument");
    try {
        begin_call(s);
        const long long n = field_len(s);
        k_scale_source<<<grid_for(n), 256, 0, s->st>>>(scale_in(s), (const double2*)src, (double2*)y, adjoint ? 1 : 0);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaStreamSynchronize(s->st));
        return CBS_OK;
    } catch (const CudaError& e) {
        return set_err(s, CBS_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e.e) + " in " + e.what);
    }
}

cbs_status unscale_field(cbs_solver* s, const void* x, void* field)
{
    if (!s) return CBS_EINVAL;
    if (!x || !field) return set_err(s, CBS_EINVAL, "NULL argument");
    try {
        begin_call(s);
        const long long n = field_len(s);
        k_scale_blocks<<<grid_for(n), 256, 0, s->st>>>(s->D, s->N, 1.0 / std::sqrt(s->lam1), 1.0 / std::sqrt(s->lam2),
                                                       (const double2*)x, (double2*)field);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaStreamSynchronize(s->st));
        return CBS_OK;
    } catch (const CudaError& e) {
        return set_err(s, CBS_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e.e) + " in " + e.what);
    }
}

cbs_status medium_gradient(cbs_solver* s, const double* c0, const double* rho, const double* alpha, const void* src,
                           const void* field, const void* adj_field, double* grad_c0, double* grad_rho, int accumulate)
{
    if (!s) return CBS_EINVAL;
    if (!c0 || !rho || !alpha || !src || !field || !adj_field || !grad_c0 || !grad_rho)
        return set_err(s, CBS_EINVAL, "NULL argument");
    try {
        begin_call(s);
        GradIn g;
        g.m.colloc = s->opt.grid_kind == CBS_GRID_COLLOCATED ? 1 : 0;
        g.m.D = s->D; g.m.n0 = s->n[0]; g.m.n1 = s->n[1]; g.m.n2 = s->n[2]; g.m.N = s->N; g.m.omega = s->omega;
        g.m.c0 = c0; g.m.rho = rho; g.m.alpha = alpha;
        for (int a = 0; a < 3; ++a) { g.m.gc[a] = s->gc64[a]; g.m.gs[a] = s->gs64[a]; }
        g.src = (const double2*)src;
        g.X = (const double2*)field;
        g.L = (const double2*)adj_field;
        k_medium_gradient<<<grid_for(s->N), 256, 0, s->st>>>(g, grad_c0, grad_rho, accumulate ? 1 : 0);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaStreamSynchronize(s->st));
        return CBS_OK;
    } catch (const CudaError& e) {
        return set_err(s, CBS_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e.e) + " in " + e.what);
    }
}

cbs_status solver_scalars(const cbs_solver* s, double* out)
{
    if (!s || !out) return CBS_EINVAL;
    out[0] = s->a1r; out[1] = s->a1i; out[2] = s->a2r; out[3] = s->a2i; out[4] = s->lam1; out[5] = s->lam2;
    return CBS_OK;
}

cbs_status solver_time_kernels(cbs_solver* s, const void* y, void* x, int n_iter, char* names, int names_len,
                               double* ms, int max_k, int* nk)
{
    if (!s) return CBS_EINVAL;
    if (!y || !x || n_iter <= 0 || !ms || !nk) return set_err(s, CBS_EINVAL, "bad argument");
    const bool f32 = s->opt.precision != CBS_FP64;
    const char* kn3[5] = {"rows_fwd", "axis_fwd", "last_symbol", "axis_inv", "rows_inv"};
    const char* kn2[3] = {"rows_fwd", "last_symbol", "rows_inv"};
    const char* knp[3] = {"plane_fwd", "last_symbol", "plane_inv"};
    const char* knf3[4] = {"axis_fwd", "last_symbol", "axis_inv", "rows_inv_fwd"};
    const char* knf2[2] = {"last_symbol", "rows_inv_fwd"};
    const bool plane = f32 && s->P32.plane;
    const bool fused = !plane && (f32 ? s->P32.fused_rows : s->P64.fused_rows);
    const int K = fused ? (s->D == 3 ? 4 : 2) : ((s->D == 3 && !plane) ? 5 : 3);
    const char** kn = fused ? (s->D == 3 ? knf3 : knf2) : (plane ? knp : (s->D == 3 ? kn3 : kn2));
    try {
        begin_call(s);
        const long long n = field_len(s);
        if (f32) {
            k_cast_64_32<<<grid_for(n), 256, 0, s->st>>>((const double2*)y, s->y32, 1.0, n);
            k_cast_64_32<<<grid_for(n), 256, 0, s->st>>>((const double2*)x, s->x32, 1.0, n);
        } else {
            CUDA_TRY(cudaMemcpyAsync(s->y64, y, n * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
            CUDA_TRY(cudaMemcpyAsync(s->x64, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
        }
        std::vector<cudaEvent_t> ev(K + 1);
        for (auto& e : ev) CUDA_TRY(cudaEventCreate(&e));
        std::vector<double> acc(K, 0.0);
        // fused rows: the forward row kernel runs once before the timed iterations, each of which is then the
        // strided-axis and last-axis kernels and the fused update + next forward row kernel
        if (fused) {
            if (f32) CUDA_TRY(launch_rows_fwd<float>(s->P32, s->x32, s->y32, s->w32, FWD_BORN, 0, s->st));
            else CUDA_TRY(launch_rows_fwd<double>(s->P64, s->x64, s->y64, s->w64, FWD_BORN, 0, s->st));
        }
        // one untimed iteration first: the first launch of each kernel in a process also loads it
        for (int it = -1; it < n_iter; ++it) {
            int k = 0;
            auto mark = [&]() { CUDA_TRY(cudaEventRecord(ev[k++], s->st)); };
            mark();
            if (fused) {
                auto one = [&](auto& P, auto* x, auto* y, auto* w, auto nu) {
                    if (s->D == 3) { CUDA_TRY(launch_axis(P, w, -1, s->st)); mark(); }
                    CUDA_TRY(launch_last(P, w, SYM_GREEN, s->st)); mark();
                    if (s->D == 3) { CUDA_TRY(launch_axis(P, w, +1, s->st)); mark(); }
                    CUDA_TRY(launch_rows_inv_fwd(P, x, y, w, 0, nu, s->partials, s->st)); mark();
                };
                if (f32) one(s->P32, s->x32, s->y32, s->w32, (float)s->opt.nu);
                else one(s->P64, s->x64, s->y64, s->w64, s->opt.nu);
                CUDA_TRY(cudaStreamSynchronize(s->st));
                for (int j = 0; j < K && it >= 0; ++j) {
                    float tj = 0;
                    CUDA_TRY(cudaEventElapsedTime(&tj, ev[j], ev[j + 1]));
                    acc[j] += tj;
                }
                continue;
            }
            if (f32) {
                Plan<float>& P = s->P32;
                if (plane) {
                    CUDA_TRY(launch_plane_fwd<float>(P, s->x32, s->y32, s->w32, 0, s->st)); mark();
                    CUDA_TRY(launch_last<float>(P, s->w32, SYM_GREEN, s->st)); mark();
                    CUDA_TRY(launch_plane_inv<float>(P, s->x32, s->w32, 0, (float)s->opt.nu, s->partials, s->st)); mark();
                    CUDA_TRY(cudaStreamSynchronize(s->st));
                    for (int j = 0; j < K && it >= 0; ++j) {
                        float tj = 0;
                        CUDA_TRY(cudaEventElapsedTime(&tj, ev[j], ev[j + 1]));
                        acc[j] += tj;
                    }
                    continue;
                }
                CUDA_TRY(launch_rows_fwd<float>(P, s->x32, s->y32, s->w32, FWD_BORN, 0, s->st)); mark();
                if (s->D == 3) { CUDA_TRY(launch_axis<float>(P, s->w32, -1, s->st)); mark(); }
                CUDA_TRY(launch_last<float>(P, s->w32, SYM_GREEN, s->st)); mark();
                if (s->D == 3) { CUDA_TRY(launch_axis<float>(P, s->w32, +1, s->st)); mark(); }
                CUDA_TRY(launch_rows_inv<float>(P, s->x32, s->y32, s->w32, INV_BORN, 0, (float)s->opt.nu, s->partials, s->st)); mark();
            } else {
                Plan<double>& P = s->P64;
                CUDA_TRY(launch_rows_fwd<double>(P, s->x64, s->y64, s->w64, FWD_BORN, 0, s->st)); mark();
                if (s->D == 3) { CUDA_TRY(launch_axis<double>(P, s->w64, -1, s->st)); mark(); }
                CUDA_TRY(launch_last<double>(P, s->w64, SYM_GREEN, s->st)); mark();
                if (s->D == 3) { CUDA_TRY(launch_axis<double>(P, s->w64, +1, s->st)); mark(); }
                CUDA_TRY(launch_rows_inv<double>(P, s->x64, s->y64, s->w64, INV_BORN, 0, s->opt.nu, s->partials, s->st)); mark();
            }
            CUDA_TRY(cudaStreamSynchronize(s->st));
            for (int j = 0; j < K && it >= 0; ++j) {
                float t = 0;
                CUDA_TRY(cudaEventElapsedTime(&t, ev[j], ev[j + 1]));
                acc[j] += t;
            }
        }
        for (auto& e : ev) cudaEventDestroy(e);
        const int m = std::min(K, max_k);
        for (int j = 0; j < m; ++j) ms[j] = acc[j] / n_iter;
        *nk = m;
        if (names && names_len > 0) {
            std::string all;
            for (int j = 0; j < m; ++j) { all += kn[j]; all.push_back('\0'); }
            std::memcpy(names, all.data(), std::min((size_t)names_len, all.size()));
        }
        if (f32) k_cast_32_64<<<grid_for(n), 256, 0, s->st>>>(s->x32, (double2*)x, n);
        else CUDA_TRY(cudaMemcpyAsync(x, s->x64, n * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
        CUDA_TRY(cudaStreamSynchronize(s->st));
        return CBS_OK;
    } catch (const CudaError& e) {
        return set_err(s, CBS_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e.e) + " in " + e.what);
    }
}

cbs_status cbs_selftest(int which, int* result)
{
    if (!result || which != CBS_SELFTEST_BULK_TIMEOUT) return CBS_EINVAL;
    double2* src = nullptr;
    int* words = nullptr;
    cudaError_t e = cudaMalloc(&src, sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&words, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(src, 0, sizeof(double2));
    if (e == cudaSuccess) e = cudaMemset(words, 0, 2 * sizeof(int));
    if (e == cudaSuccess) {
        k_selftest_bulk_timeout<<<1, 32>>>(src, words, words + 1, 256);
        e = cudaGetLastError();
    }
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, words, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(src);
    cudaFree(words);
    if (e != cudaSuccess) return CBS_ECUDA;
    *result = (h[0] == kErrBulkTimeout && h[1] == 1) ? CBS_ETIMEOUT : CBS_OK;
    return CBS_OK;
}

cbs_status cufft_baseline_iterate(cbs_solver* s, const void* y, void* x, int n_iter, int adjoint, double* ms_per_iter)
{
    if (!s) return CBS_EINVAL;
    if (!y || !x || n_iter <= 0 || !ms_per_iter) return set_err(s, CBS_EINVAL, "bad argument");
    if (s->opt.precision == CBS_FP64)
        return set_err(s, CBS_EINVAL, "the cuFFT baseline runs the float32 iteration: create the solver in float32");
    try {
        begin_call(s);
        const long long n = field_len(s);
        if (!s->fft_plan_ok) {
            int dims[3] = {s->n[2], s->n[1], s->n[0]};  // slowest axis first
            int* d0 = s->D == 3 ? dims : dims + 1;
            if (cufftPlanMany(&s->fft_plan, s->D, d0, nullptr, 1, (int)s->N, nullptr, 1, (int)s->N, CUFFT_C2C, s->C) !=
                CUFFT_SUCCESS)
                return set_err(s, CBS_ECUDA, "cufftPlanMany failed");
            s->fft_plan_ok = true;
        }
        if (cufftSetStream(s->fft_plan, s->st) != CUFFT_SUCCESS) return set_err(s, CBS_ECUDA, "cufftSetStream failed");
        k_cast_64_32<<<grid_for(n), 256, 0, s->st>>>((const double2*)y, s->y32, 1.0, n);
        k_cast_64_32<<<grid_for(n), 256, 0, s->st>>>((const double2*)x, s->x32, 1.0, n);
        CUDA_TRY(cudaGetLastError());
        Plan<float>& P = s->P32;
        const int g = grid_for(n), gs = grid_for(s->N);
        const int mode = adjoint ? SYM_GREEN_ADJ : SYM_GREEN;
        cufftComplex* w = reinterpret_cast<cufftComplex*>(s->w32);
        CUDA_TRY(cudaEventRecord(s->ev0, s->st));
        for (int it = 0; it < n_iter; ++it) {
            k_base_pre<float><<<g, 256, 0, s->st>>>(P.d, P.M, s->x32, s->y32, s->w32, adjoint);
            CUDA_TRY(cudaGetLastError());
            if (cufftExecC2C(s->fft_plan, w, w, CUFFT_FORWARD) != CUFFT_SUCCESS)
                return set_err(s, CBS_ECUDA, "cufftExecC2C failed");
            if (s->D == 3) k_base_symbol<float, 4><<<gs, 256, 0, s->st>>>(P.d, P.Sy, s->w32, mode);
            else k_base_symbol<float, 3><<<gs, 256, 0, s->st>>>(P.d, P.Sy, s->w32, mode);
            CUDA_TRY(cudaGetLastError());
            if (cufftExecC2C(s->fft_plan, w, w, CUFFT_INVERSE) != CUFFT_SUCCESS)
                return set_err(s, CBS_ECUDA, "cufftExecC2C failed");
            k_base_update<float><<<g, 256, 0, s->st>>>(P.d, P.M, s->x32, s->w32, adjoint, (float)s->opt.nu, s->partials);
            CUDA_TRY(cudaGetLastError());
        }
        CUDA_TRY(cudaEventRecord(s->ev1, s->st));
        k_cast_32_64<<<grid_for(n), 256, 0, s->st>>>(s->x32, (double2*)x, n);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaStreamSynchronize(s->st));
        float ms = 0;
        CUDA_TRY(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
        *ms_per_iter = ms / n_iter;
        return CBS_OK;
    } catch (const CudaError& e) {
        return set_err(s, CBS_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e.e) + " in " + e.what);
    }
}

}  // extern "C"
