// noalloc.cu -- (L+I)^-1 apply that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or under a fixed memory budget, plug-ins that must
// not grow the process's device footprint, or processes where the CUDA
// allocator is locked down.  green_apply_noalloc serves them: the caller
// passes the input and output buffers, and every other piece of device memory
// the transform needs (twiddle and wavenumber tables, the inverse-x kernel's
// per-block norm partials) lives in the file-scope array below.  That array
// is part of the library image: every GPU that loads the library holds it
// (kNoAllocScratchDoubles * 8 bytes = 124 KiB) until the process exits.
//
// The kernels are the same ones green_apply runs for a solver on the
// staggered grid (App. B.1, the default grid kind); the output buffer doubles
// as the transform's work array.  The collocated grid kind is not offered
// here: its symbol uses i k in place of i k e^{i k dx / 2}.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "cbs.h"
#include "launch.cuh"

namespace cbs {
CBS_EXTERN_LAUNCHERS(double)
void set_create_error(const std::string& msg);  // message returned by cbs_last_error(NULL)
}  // namespace cbs

using namespace cbs;

namespace {

constexpr int kMaxAxis = 512;                    // largest supported extent
constexpr long long kMaxVoxels = 1LL << 21;      // N <= 2,097,152 (e.g. 128^3, 512 x 64 x 64, 512 x 512)
constexpr int kMaxPartialBlocks = 4096;          // inverse-x kernel blocks for N <= kMaxVoxels
constexpr int kTwOff = 0;                                   // double2 tw[3][kMaxAxis]
constexpr int kKtOff = kTwOff + 3 * kMaxAxis * 2;           // double2 kt[3][kMaxAxis]
constexpr int kK2Off = kKtOff + 3 * kMaxAxis * 2;           // double  k2[3][kMaxAxis]
constexpr int kPartOff = kK2Off + 3 * kMaxAxis;             // double  partials[2 * kMaxPartialBlocks]
constexpr int kNoAllocScratchDoubles = kPartOff + 2 * kMaxPartialBlocks;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The name
// g_noalloc_scratch in host code is only a host-side stand-in, so the address
// is looked up once per device with that device current (the first call on
// that device) and kept for the life of the process; a process that resets a
// device with cudaDeviceReset must not call this entry point on that device
// afterwards, since the kept address belonged to the destroyed context.
cudaError_t scratch_address(double** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// per-axis twiddles exp(-2 pi i j / n), t = k e^{i k dx/2} and k^2 with
// k = 2 pi fftfreq(n, dx), written into the scratch tables
__global__ void k_noalloc_tables(int D, int n0, int n1, int n2, double dx, double* scratch)
{
    const int a = blockIdx.y;
    const int n = a == 0 ? n0 : (a == 1 ? n1 : n2);
    double2* tw = reinterpret_cast<double2*>(scratch + kTwOff) + a * kMaxAxis;
    double2* kt = reinterpret_cast<double2*>(scratch + kKtOff) + a * kMaxAxis;
    double* k2 = scratch + kK2Off + a * kMaxAxis;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)j / (double)n, &s, &c);
        tw[j] = make_double2(c, s);
        const int f = (j < (n + 1) / 2) ? j : j - n;
        const double k = 2.0 * 3.14159265358979323846 * (double)f / ((double)n * dx);
        double sh, ch;
        sincos(0.5 * k * dx, &sh, &ch);
        kt[j] = make_double2(k * ch, k * sh);
        k2[j] = k * k;
    }
    (void)D;
}

cbs_status fail(cbs_status st, const std::string& msg)
{
    set_create_error("green_apply_noalloc: " + msg);
    return st;
}

}  // namespace

extern "C" {

cbs_status green_apply_noalloc(const cbs_grid* grid, double dx, const double* scalars, const void* in, void* out,
                               int adjoint, void* stream)
{
    if (!grid || !scalars || !in || !out) return fail(CBS_EINVAL, "NULL argument");
    if (in == out) return fail(CBS_EINVAL, "in and out must be different buffers");
    if (grid->ndim != 2 && grid->ndim != 3) return fail(CBS_EINVAL, "ndim must be 2 or 3");
    long long N = 1;
    int n[3] = {1, 1, 1};
    for (int a = 0; a < grid->ndim; ++a) {
        if (!size_supported(grid->n[a]) || grid->n[a] > kMaxAxis)
            return fail(CBS_EINVAL, "unsupported extent " + std::to_string((long long)grid->n[a]));
        n[a] = (int)grid->n[a];
        N *= grid->n[a];
    }
    if (N > kMaxVoxels)
        return fail(CBS_EINVAL, "grid of " + std::to_string(N) + " voxels exceeds the allocation-free maximum of " +
                                    std::to_string(kMaxVoxels));
    const double l1 = scalars[4], l2 = scalars[5];
    if (!(dx > 0) || !(l1 > 0) || !(l2 > 0) || !std::isfinite(l1) || !std::isfinite(l2))
        return fail(CBS_EINVAL, "dx, lambda1 and lambda2 must be positive");
    double* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return fail(CBS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;

    Plan<double> P{};
    P.d.D = grid->ndim;
    P.d.n0 = n[0];
    P.d.n1 = n[1];
    P.d.n2 = n[2];
    P.d.N = N;
    const int nblk = rows_blocks<double>(P);
    if (nblk > kMaxPartialBlocks) return fail(CBS_EINVAL, "grid needs more norm partials than the scratch holds");
    for (int a = 0; a < 3; ++a) {
        P.tw[a] = reinterpret_cast<const double2*>(scratch + kTwOff) + a * kMaxAxis;
        P.Sy.kt[a] = reinterpret_cast<const double2*>(scratch + kKtOff) + a * kMaxAxis;
        P.Sy.k2[a] = scratch + kK2Off + a * kMaxAxis;
        // the copy / plain modes read the layer tables only as unused row
        // constants: any readable table of n_a values serves
        P.M.gc[a] = P.Sy.k2[a];
        P.M.gs[a] = P.Sy.k2[a];
    }
    // (L+I)^-1 symbol constants (App. B.1, a = a1, lambda_0 = lambda1, b = a2, lambda_1 = lambda2)
    const double apr = scalars[0] + l1, api = scalars[1];
    const double bpr = scalars[2] + l2, bpi = scalars[3];
    const double den = apr * apr + api * api;
    const double Pr = l1 * apr / den, Pi = -l1 * api / den;
    const double scale = 1.0 / (double)N;
    const double sq = std::sqrt(l1 * l2);
    P.Sy.Pu = make_double2(Pr, Pi);
    P.Sy.P = make_double2(Pr * scale, Pi * scale);
    P.Sy.c1 = make_double2(0.0, sq);
    P.Sy.c2 = make_double2(l2 * apr, l2 * api);
    P.Sy.c3 = make_double2(apr * bpr - api * bpi, apr * bpi + api * bpr);
    P.Sy.la1 = make_double2(scalars[0] / l1, scalars[1] / l1);
    P.Sy.la2 = make_double2(scalars[2] / l2, scalars[3] / l2);
    P.Sy.isq = 1.0 / sq;
    P.Sy.scale = scale;

    k_noalloc_tables<<<dim3(4, 3), 128, 0, st>>>(grid->ndim, n[0], n[1], n[2], dx, scratch);
    e = cudaGetLastError();
    const double2* x = static_cast<const double2*>(in);
    double2* w = static_cast<double2*>(out);
    double* partials = scratch + kPartOff;
    if (e == cudaSuccess) e = launch_rows_fwd<double>(P, x, nullptr, w, FWD_COPY, 0, st);
    if (e == cudaSuccess && P.d.D == 3) e = launch_axis<double>(P, w, -1, st);
    if (e == cudaSuccess) e = launch_last<double>(P, w, adjoint ? SYM_GREEN_ADJ : SYM_GREEN, st);
    if (e == cudaSuccess && P.d.D == 3) e = launch_axis<double>(P, w, +1, st);
    if (e == cudaSuccess) e = launch_rows_inv<double>(P, nullptr, nullptr, w, INV_PLAIN, 0, 0.0, partials, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(CBS_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e));
    return CBS_OK;
}

}  // extern "C"
