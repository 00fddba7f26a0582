// launch.cuh -- host-side launchers of the Born kernels for one precision.
// Each launcher dispatches on the axis extent to the kernel instantiated for
// that size (the FFT plans are compile-time).  Included by exactly one
// translation unit per precision (kernels_f32.cu, kernels_f64.cu).
#pragma once
#include <cuda_runtime.h>

#include "born.cuh"
#include "last_cluster.cuh"
#include "plane.cuh"

namespace cbs {

// Elements per thread of one transform (RX for row/axis kernels, RL for the
// all-components pencil kernel, which keeps C transforms in registers).
// float32 rows of 128 and more points: 16 values a thread (radix-16 passes: 128 = 16*8, 2048 = 16*16*8), measured
// on the fused row kernel 438.9 instead of 479.7 us at 256^3, 144.4 instead of 169.8 us at 2048^2, 3.94 instead of
// 4.06 ms at 512^3 (59.7 either way at 128^3); float32 3*2^k rows of 192 and more points: 24 (passes 3, 8, 8),
// 295 instead of 308 us at 192^3
template <typename R> __host__ __device__ constexpr int r_rows(int n)
{
    return (n % 3 == 0) ? ((sizeof(R) == 4 && n >= 192) ? 24 : 12) : ((sizeof(R) == 4 && n >= 128) ? 16 : 8);
}
// strided-axis transforms: 16 values per thread for float32 128 / 256 (two passes, radix 16 then 8 or 16) and 512
// (16, 16, 2: 1.52 instead of 1.94 ms at 512^3, 8 columns; 16 columns measured 2.27 ms)
template <typename R> __host__ __device__ constexpr int r_axis(int n)
{
    return (n % 3 == 0) ? 12 : ((sizeof(R) == 4 && (n == 128 || n == 256 || n == 512)) ? 16 : 8);
}
template <typename R> __host__ __device__ constexpr int r_last(int n, int c = 4)
{
    // float32 3D 3*2^k pencils of 96 and 192 points: 12 values a thread (passes 3,4,4,...) instead of 6
    // (3,2,2,...): measured 174 instead of 224 us at 192^3, 22.6 instead of 26.7 us at 96^3
    return sizeof(R) == 4 ? ((n % 3 == 0) ? ((c == 4 && n >= 96) ? 12 : 6) : 8) : ((n % 3 == 0) ? 6 : 4);
}
template <typename R> __host__ __device__ constexpr int cols_axis(int n)
{
    return sizeof(R) == 4 ? (n == 128 ? 32 : (n <= 256 ? 16 : (n <= 512 ? 8 : 4))) : (n <= 128 ? 8 : (n <= 512 ? 4 : 2));
}
template <typename R> __host__ __device__ constexpr int cols_last(int n, int c)
{
    if (sizeof(R) == 4 && c == 3 && n == 512) return 4;  // 2D: the grid is n0 / COLS blocks, keep it wide
    // float32 512: 8 columns (64-byte rows) measured 3.27 ms instead of 4.73 ms with 4 at 512^3; 16 columns at
    // 256 measured slower than 8; 3D 96 / 192 with 12 values a thread: 32 / 16 columns (256 threads)
    if (sizeof(R) == 4 && c == 4 && n % 3 == 0 && n >= 96) return n <= 96 ? 32 : 16;
    return sizeof(R) == 4 ? (n <= 128 ? 16 : (n <= 256 ? 8 : (n <= 512 ? 8 : (n <= 1024 ? 4 : 2))))
                          : (n <= 128 ? 8 : (n <= 256 ? 4 : (n <= 512 ? 2 : (n <= 1024 ? 2 : 1))));
}

// tile-staged last-axis kernel (3D float32, 16 <= n2 <= 256: one tensor-copy box per component)
template <typename R> __host__ __device__ constexpr int r_tile(int n) { return (n % 3 == 0) ? 6 : 8; }
template <typename R> __host__ __device__ constexpr int cols_tile(int n) { return n <= 64 ? 32 : (n <= 128 ? 16 : 8); }
template <typename R> __host__ __device__ constexpr bool tile_ok(int n)
{
    return sizeof(R) == 4 && n >= 16 && n <= 256;
}

#define CBS_FOR_EACH_SIZE(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(512) X(1024) X(2048)

inline bool size_supported(long long n)
{
    switch (n) {
#define CBS_CASE(n) case n:
        CBS_FOR_EACH_SIZE(CBS_CASE)
#undef CBS_CASE
        return true;
    default:
        return false;
    }
}

template <typename R> struct Plan {
    Dims d;
    Medium<R> M;
    Symbol<R> Sy;
    const cplx<R>* tw[3];  // twiddle table of each axis length
    int* err = nullptr;    // device error word of the bulk-staged kernels (nullptr: plain kernels only)
    // tensor-copy descriptor of one work field for the tile-staged last-axis kernel; used when the kernel
    // is given that field (tile_field) and the error word is set
    CUtensorMap tmap_last;
    const void* tile_field = nullptr;
    // tensor-copy descriptor of the same field for the pipelined strided-axis kernel (box {COLS, n1, 1})
    CUtensorMap tmap_axis;
    const void* axis_field = nullptr;
    int axis_grid = 0;  // persistent CTAs: SMs x resident blocks
    bool plane = false;    // the Born iteration uses the x-y plane kernels (see plane_ok)
    bool last_cluster = false;  // float32 last-axis step on a cluster of C CTAs (see last_cluster_ok)
    int plane_cl = 2;           // CTAs per x-y plane of the plane kernels (2 or 4)
    bool fused_rows = false;    // update + next forward row transform in one kernel (see fused_rows_ok)
    int fused_var = -1;         // variant of the fused row kernel (float32, 128- to 512-point rows); -1: default
};

// x-y plane kernels: 3D float32 with n0, n1 in {32, 64, 128}; one CTA pair per (component, z) plane.
// The Born iteration uses them for planes of at most 4096 values: measured on GB300, 64^3 takes 33.0
// instead of 41.0 us per iteration, while 128 x 128 planes (64 KiB half-planes, two CTAs per SM) take
// 173 instead of 157 us, so larger planes keep the row + strided-axis kernels.
constexpr int kPlaneCL = 2;
constexpr long long kPlaneMaxValues = 4096;
inline bool plane_size(int n) { return n == 32 || n == 64 || n == 128; }
template <typename R> inline bool plane_ok(const Plan<R>& P)
{
    return sizeof(R) == 4 && P.d.D == 3 && plane_size(P.d.n0) && plane_size(P.d.n1);
}
template <typename R> inline bool plane_preferred(const Plan<R>& P)
{
    return plane_ok<R>(P) && (long long)P.d.n0 * P.d.n1 <= kPlaneMaxValues;
}
template <typename R> inline int plane_blocks(const Plan<R>& P) { return (P.d.D + 1) * P.d.n2 * P.plane_cl; }

// the Born row kernels stage their rows with bulk copies when every block's
// rows lie in one component and the rows' exchange fits in place
template <typename R, int N> inline bool bulk_rows_ok(const Plan<R>& P)
{
    using Cfg = BulkCfg<R, N, r_rows<R>(N)>;
    return Cfg::OK && P.err != nullptr && (P.d.N / N) % Cfg::ROWS == 0;
}

template <typename R> inline int rows_blocks(const Plan<R>& P)
{
    int n0 = P.d.n0;
    long long rows = (long long)(P.d.D + 1) * (P.d.N / n0);
    int per = 1;
    switch (n0) {
#define CBS_CASE(n) case n: per = RowCfg<R, n, r_rows<R>(n)>::ROWS; break;
        CBS_FOR_EACH_SIZE(CBS_CASE)
#undef CBS_CASE
    default: return 0;
    }
    return (int)((rows + per - 1) / per);
}

template <typename R, int N> cudaError_t rows_fwd_n(const Plan<R>& P, const cplx<R>* x, const cplx<R>* y, cplx<R>* w,
                                                    int mode, int adj, cudaStream_t st)
{
    constexpr int RX = r_rows<R>(N);
    using Cfg = RowCfg<R, N, RX>;
    long long rows = (long long)(P.d.D + 1) * (P.d.N / N);
    int grid = (int)((rows + Cfg::ROWS - 1) / Cfg::ROWS);
    if constexpr (BulkCfg<R, N, RX>::OK) {
        if (mode == FWD_BORN && bulk_rows_ok<R, N>(P)) {
            using B = BulkCfg<R, N, RX>;
            auto kern = k_rows_fwd_bulk<R, N, RX>;
            // once per process, thread-safe (function-local static)
            static const cudaError_t attr =
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B::SMEM);
            if (attr != cudaSuccess) return attr;
            kern<<<grid, B::THREADS, B::SMEM, st>>>(P.d, P.M, x, y, w, P.tw[0], adj, P.err);
            return cudaGetLastError();
        }
    }
    k_rows_fwd<R, N, RX><<<grid, Cfg::THREADS, 0, st>>>(P.d, P.M, x, y, w, P.tw[0], mode, adj);
    return cudaGetLastError();
}

template <typename R, int N> cudaError_t rows_inv_n(const Plan<R>& P, cplx<R>* x, const cplx<R>* y, cplx<R>* w, int mode,
                                                    int adj, R nu, double* partials, cudaStream_t st)
{
    constexpr int RX = r_rows<R>(N);
    using Cfg = RowCfg<R, N, RX>;
    long long rows = (long long)(P.d.D + 1) * (P.d.N / N);
    int grid = (int)((rows + Cfg::ROWS - 1) / Cfg::ROWS);
    if constexpr (BulkCfg<R, N, RX>::OK) {
        if (mode == INV_BORN && bulk_rows_ok<R, N>(P)) {
            using B = BulkCfg<R, N, RX>;
            auto kern = k_rows_inv_bulk<R, N, RX>;
            // once per process, thread-safe (function-local static)
            static const cudaError_t attr =
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B::SMEM);
            if (attr != cudaSuccess) return attr;
            kern<<<grid, B::THREADS, B::SMEM, st>>>(P.d, P.M, x, w, P.tw[0], adj, nu, partials, P.err);
            return cudaGetLastError();
        }
    }
    if (mode == INV_BORN)
        k_rows_inv<R, N, RX, true><<<grid, Cfg::THREADS, 0, st>>>(P.d, P.M, x, y, w, P.tw[0], mode, adj, nu, partials);
    else
        k_rows_inv<R, N, RX, false><<<grid, Cfg::THREADS, 0, st>>>(P.d, P.M, x, y, w, P.tw[0], mode, adj, nu, partials);
    return cudaGetLastError();
}

// update of iteration k fused with the forward row transform of iteration k+1 (bulk-staged rows)
template <typename R, int N> inline bool fused_rows_ok_n(const Plan<R>& P)
{
    using Cfg = FusedCfg<R, N, r_rows<R>(N)>;
    return Cfg::OK && P.err != nullptr && (P.d.N / N) % Cfg::ROWS == 0;
}

template <typename R> inline bool fused_rows_ok(const Plan<R>& P)
{
    switch (P.d.n0) {
#define CBS_CASE(n) case n: return fused_rows_ok_n<R, n>(P);
        CBS_FOR_EACH_SIZE(CBS_CASE)
#undef CBS_CASE
    default: return false;
    }
}

template <typename R, int N, int VAR> cudaError_t rows_inv_fwd_var(const Plan<R>& P, cplx<R>* x, const cplx<R>* y,
                                                                   cplx<R>* w, int adj, R nu, double* partials,
                                                                   cudaStream_t st)
{
    constexpr int RX = r_rows<R>(N);
    using Cfg = FusedCfg<R, N, RX, VAR>;
    auto kern = k_rows_inv_fwd_bulk<R, N, RX, VAR>;
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (attr != cudaSuccess) return attr;
    const long long rows = (long long)(P.d.D + 1) * (P.d.N / N);
    kern<<<(unsigned)(rows / Cfg::ROWS), Cfg::THREADS, Cfg::SMEM, st>>>(P.d, P.M, x, y, w, P.tw[0], adj, nu, partials,
                                                                        P.err);
    return cudaGetLastError();
}

template <typename R, int N> cudaError_t rows_inv_fwd_n(const Plan<R>& P, cplx<R>* x, const cplx<R>* y, cplx<R>* w,
                                                        int adj, R nu, double* partials, cudaStream_t st)
{
    constexpr int RX = r_rows<R>(N);
    using Cfg = FusedCfg<R, N, RX>;
    if constexpr (Cfg::OK) {
        if (!fused_rows_ok_n<R, N>(P)) return cudaErrorNotSupported;
        if constexpr (sizeof(R) == 4 && (N == 128 || N == 256 || N == 512)) {
            // default: y staged into the transform's buffer (measured: 128^3 59.6 instead of 64.0 us, 512^3 4.06
            // instead of 4.30 ms; 256^3 480 instead of 502 us with the four-block variant); L2 hints on the copies
            // gained nothing with the persisting window on w
            const int var = P.fused_var >= 0 ? P.fused_var : 2;
            switch (var) {
            case 1: return rows_inv_fwd_var<R, N, 1>(P, x, y, w, adj, nu, partials, st);
            case 2: return rows_inv_fwd_var<R, N, 2>(P, x, y, w, adj, nu, partials, st);
            case 3: return rows_inv_fwd_var<R, N, 3>(P, x, y, w, adj, nu, partials, st);
            case 6: return rows_inv_fwd_var<R, N, 6>(P, x, y, w, adj, nu, partials, st);
            default: break;
            }
        } else if constexpr (sizeof(R) == 4 && FusedCfg<R, N, RX, 2>::OK) {
            // the other float32 row lengths (192, 1024, 2048): y staged into the transform's buffer too (measured
            // 192^3 289 instead of 298 us, 1024^2 35.2 instead of 37.2 us, 2048^2 133.3 instead of 142.4 us);
            // CBS_FUSED_VAR=0 keeps three field buffers
            if (P.fused_var != 0) return rows_inv_fwd_var<R, N, 2>(P, x, y, w, adj, nu, partials, st);
        }
        return rows_inv_fwd_var<R, N, 0>(P, x, y, w, adj, nu, partials, st);
    } else {
        return cudaErrorNotSupported;
    }
}

template <typename R> cudaError_t launch_rows_inv_fwd(const Plan<R>& P, cplx<R>* x, const cplx<R>* y, cplx<R>* w, int adj,
                                                      R nu, double* partials, cudaStream_t st)
{
    switch (P.d.n0) {
#define CBS_CASE(n) case n: return rows_inv_fwd_n<R, n>(P, x, y, w, adj, nu, partials, st);
        CBS_FOR_EACH_SIZE(CBS_CASE)
#undef CBS_CASE
    default: return cudaErrorInvalidValue;
    }
}

// pipelined strided-axis kernel: 3D float32, n1 <= 256 (one box per tile)
template <typename R> __host__ __device__ constexpr bool axis_pipe_ok(int n) { return sizeof(R) == 4 && n >= 16 && n <= 256; }

template <typename R, int N, int S> cudaError_t axis_n(const Plan<R>& P, cplx<R>* w, cudaStream_t st)
{
    constexpr int RA = r_axis<R>(N);
    constexpr int COLS = cols_axis<R>(N);
    constexpr int T = N / RA;
    if constexpr (axis_pipe_ok<R>(N)) {
        if (P.axis_field != nullptr && P.axis_field == (const void*)w && P.err != nullptr && P.axis_grid > 0 &&
            P.d.n0 % COLS == 0) {
            using PC = AxisPipeCfg<R, N, COLS>;
            auto kp = k_axis_fft_pipe<R, N, RA, COLS, S>;
            static const cudaError_t attr =
                cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PC::SMEM);
            if (attr != cudaSuccess) return attr;
            const long long tiles = (long long)(P.d.D + 1) * P.d.n2 * (P.d.n0 / COLS);
            const int grid = (int)(tiles < P.axis_grid ? tiles : P.axis_grid);
            kp<<<grid, T * COLS, PC::SMEM, st>>>(P.tmap_axis, P.d, w, P.tw[1], P.err);
            return cudaGetLastError();
        }
    }
    const size_t smem = (size_t)N * COLS * sizeof(cplx<R>);
    auto kern = k_axis_fft<R, N, RA, COLS, S>;
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    int xblocks = (P.d.n0 + COLS - 1) / COLS;
    long long grid = (long long)(P.d.D + 1) * P.d.n2 * xblocks;
    kern<<<(unsigned)grid, T * COLS, smem, st>>>(P.d, w, P.tw[1]);
    return cudaGetLastError();
}

template <typename R, int N, int C> cudaError_t last_tile_n(const Plan<R>& P, cplx<R>* w, int mode, cudaStream_t st)
{
    constexpr int RL = r_tile<R>(N);
    constexpr int COLS = cols_tile<R>(N);
    using Cfg = LastTileCfg<R, N, RL, COLS, C>;
    auto kern = k_last_symbol_tile<R, N, RL, COLS, C>;
    static const cudaError_t attr =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (attr != cudaSuccess) return attr;
    const long long grid = (long long)P.d.n1 * (P.d.n0 / COLS);
    kern<<<(unsigned)grid, Cfg::THREADS, Cfg::SMEM, st>>>(P.tmap_last, P.d, P.Sy, P.tw[2], mode, P.err);
    return cudaGetLastError();
}

// last-axis step on a cluster of C CTAs (one component each): float32, extents 64 .. 2048
template <typename R> __host__ __device__ constexpr int r_lastcl(int n) { return (n % 3 == 0) ? 12 : 16; }
template <typename R> __host__ __device__ constexpr int cols_lastcl(int n, int c)
{
    return c == 4 ? (n <= 128 ? 32 : (n <= 512 ? 16 : (n <= 1024 ? 8 : 4))) : (n <= 256 ? 16 : 8);
}
template <typename R> __host__ __device__ constexpr bool last_cluster_ok(int n)
{
    return sizeof(R) == 4 && n >= 64 && n <= 2048;
}
template <typename R, int N, int C> cudaError_t last_cluster_n(const Plan<R>& P, cplx<R>* w, int mode, cudaStream_t st);

template <typename R, int N, int C> cudaError_t last_n(const Plan<R>& P, cplx<R>* w, int mode, cudaStream_t st)
{
    if constexpr (last_cluster_ok<R>(N)) {
        if (P.last_cluster) return last_cluster_n<R, N, C>(P, w, mode, st);
    }
    if constexpr (C == 4 && tile_ok<R>(N)) {
        if (P.tile_field != nullptr && P.tile_field == (const void*)w && P.err != nullptr &&
            P.d.n0 % cols_tile<R>(N) == 0)
            return last_tile_n<R, N, C>(P, w, mode, st);
    }
    constexpr int RL = r_last<R>(N, C);
    constexpr int COLS = cols_last<R>(N, C);
    constexpr int T = N / RL;
    const size_t smem = (size_t)C * N * COLS * sizeof(cplx<R>);
    auto kern = k_last_symbol<R, N, RL, COLS, C>;
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    int xblocks = (P.d.n0 + COLS - 1) / COLS;
    long long grid = (long long)(C == 4 ? P.d.n1 : 1) * xblocks;
    kern<<<(unsigned)grid, T * COLS, smem, st>>>(P.d, P.Sy, w, P.tw[P.d.D - 1], mode);
    return cudaGetLastError();
}

template <typename R> cudaError_t launch_rows_fwd(const Plan<R>& P, const cplx<R>* x, const cplx<R>* y, cplx<R>* w,
                                                  int mode, int adj, cudaStream_t st)
{
    switch (P.d.n0) {
#define CBS_CASE(n) case n: return rows_fwd_n<R, n>(P, x, y, w, mode, adj, st);
        CBS_FOR_EACH_SIZE(CBS_CASE)
#undef CBS_CASE
    default: return cudaErrorInvalidValue;
    }
}

template <typename R> cudaError_t launch_rows_inv(const Plan<R>& P, cplx<R>* x, const cplx<R>* y, cplx<R>* w, int mode,
                                                  int adj, R nu, double* partials, cudaStream_t st)
{
    switch (P.d.n0) {
#define CBS_CASE(n) case n: return rows_inv_n<R, n>(P, x, y, w, mode, adj, nu, partials, st);
        CBS_FOR_EACH_SIZE(CBS_CASE)
#undef CBS_CASE
    default: return cudaErrorInvalidValue;
    }
}

template <typename R> cudaError_t launch_axis(const Plan<R>& P, cplx<R>* w, int sign, cudaStream_t st)
{
    switch (P.d.n1) {
#define CBS_CASE(n) case n: return sign < 0 ? axis_n<R, n, -1>(P, w, st) : axis_n<R, n, +1>(P, w, st);
        CBS_FOR_EACH_SIZE(CBS_CASE)
#undef CBS_CASE
    default: return cudaErrorInvalidValue;
    }
}

template <typename R> cudaError_t launch_last(const Plan<R>& P, cplx<R>* w, int mode, cudaStream_t st)
{
    const int nl = P.d.D == 3 ? P.d.n2 : P.d.n1;
    if (P.d.D == 3) {
        switch (nl) {
#define CBS_CASE(n) case n: return last_n<R, n, 4>(P, w, mode, st);
            CBS_FOR_EACH_SIZE(CBS_CASE)
#undef CBS_CASE
        default: return cudaErrorInvalidValue;
        }
    }
    switch (nl) {
#define CBS_CASE(n) case n: return last_n<R, n, 3>(P, w, mode, st);
        CBS_FOR_EACH_SIZE(CBS_CASE)
#undef CBS_CASE
    default: return cudaErrorInvalidValue;
    }
}

template <int CL = kPlaneCL, typename Kern, typename... Args>
cudaError_t launch_clustered(Kern kern, int grid, int threads, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = CL > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename R, int N, int C> cudaError_t last_cluster_n(const Plan<R>& P, cplx<R>* w, int mode, cudaStream_t st)
{
    constexpr int RL = r_lastcl<R>(N);
    constexpr int COLS = cols_lastcl<R>(N, C);
    using Cfg = LastClusterCfg<R, N, RL, COLS, C>;
    auto kern = k_last_cluster<R, N, RL, COLS, C>;
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (attr != cudaSuccess) return attr;
    const long long tiles = (long long)(C == 4 ? P.d.n1 : 1) * ((P.d.n0 + COLS - 1) / COLS);
    return launch_clustered<C>(kern, (int)(C * tiles), Cfg::THREADS, Cfg::SMEM, st, P.d, P.Sy, w, P.tw[P.d.D - 1], mode);
}

template <typename R, int NX, int NY, int CL>
cudaError_t plane_fwd_cl(const Plan<R>& P, const cplx<R>* x, const cplx<R>* y, cplx<R>* w, int adj, cudaStream_t st)
{
    using Cfg = PlaneCfg<R, NX, NY, CL>;
    auto kern = k_plane_fwd<R, NX, NY, CL>;
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (attr != cudaSuccess) return attr;
    return launch_clustered<CL>(kern, plane_blocks<R>(P), Cfg::THREADS, Cfg::SMEM, st, P.d, P.M, x, y, w, P.tw[0],
                                P.tw[1], adj);
}

template <typename R, int NX, int NY, int CL>
cudaError_t plane_inv_cl(const Plan<R>& P, cplx<R>* x, const cplx<R>* w, int adj, R nu, double* partials, cudaStream_t st)
{
    using Cfg = PlaneCfg<R, NX, NY, CL>;
    auto kern = k_plane_inv<R, NX, NY, CL>;
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (attr != cudaSuccess) return attr;
    return launch_clustered<CL>(kern, plane_blocks<R>(P), Cfg::THREADS, Cfg::SMEM, st, P.d, P.M, x, w, P.tw[0], P.tw[1],
                                adj, nu, partials);
}

template <typename R, int NX, int NY>
cudaError_t plane_fwd_n(const Plan<R>& P, const cplx<R>* x, const cplx<R>* y, cplx<R>* w, int adj, cudaStream_t st)
{
    if (P.plane_cl == 4) return plane_fwd_cl<R, NX, NY, 4>(P, x, y, w, adj, st);
    return plane_fwd_cl<R, NX, NY, 2>(P, x, y, w, adj, st);
}

template <typename R, int NX, int NY>
cudaError_t plane_inv_n(const Plan<R>& P, cplx<R>* x, const cplx<R>* w, int adj, R nu, double* partials, cudaStream_t st)
{
    if (P.plane_cl == 4) return plane_inv_cl<R, NX, NY, 4>(P, x, w, adj, nu, partials, st);
    return plane_inv_cl<R, NX, NY, 2>(P, x, w, adj, nu, partials, st);
}

#define CBS_FOR_EACH_PLANE(X) X(32, 32) X(32, 64) X(32, 128) X(64, 32) X(64, 64) X(64, 128) X(128, 32) X(128, 64) X(128, 128)

// w = FFT_y FFT_x (B x + y) over every (component, z) plane
template <typename R>
cudaError_t launch_plane_fwd(const Plan<R>& P, const cplx<R>* x, const cplx<R>* y, cplx<R>* w, int adj, cudaStream_t st)
{
    if constexpr (sizeof(R) == 4) {
#define CBS_CASE(a, b) if (P.d.n0 == a && P.d.n1 == b) return plane_fwd_n<R, a, b>(P, x, y, w, adj, st);
        CBS_FOR_EACH_PLANE(CBS_CASE)
#undef CBS_CASE
    }
    return cudaErrorInvalidValue;
}

// x += nu B (IFFT_x IFFT_y w - x) over every plane; norm partials per block
template <typename R>
cudaError_t launch_plane_inv(const Plan<R>& P, cplx<R>* x, const cplx<R>* w, int adj, R nu, double* partials,
                             cudaStream_t st)
{
    if constexpr (sizeof(R) == 4) {
#define CBS_CASE(a, b) if (P.d.n0 == a && P.d.n1 == b) return plane_inv_n<R, a, b>(P, x, w, adj, nu, partials, st);
        CBS_FOR_EACH_PLANE(CBS_CASE)
#undef CBS_CASE
    }
    return cudaErrorInvalidValue;
}

// resident CTAs of the pipelined axis kernel for extent n1 (0 when it does not apply)
template <typename R> int axis_pipe_blocks_per_sm(int n1)
{
    int nb = 0;
    switch (n1) {
#define CBS_CASE(n)                                                                                              \
    case n:                                                                                                      \
        if constexpr (axis_pipe_ok<R>(n)) {                                                                      \
            constexpr int RA = r_axis<R>(n), COLS = cols_axis<R>(n);                                             \
            auto kp = k_axis_fft_pipe<R, n, RA, COLS, -1>;                                                       \
            if (cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize,                            \
                                     (int)AxisPipeCfg<R, n, COLS>::SMEM) != cudaSuccess ||                       \
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kp, (n / RA) * COLS,                          \
                                                              AxisPipeCfg<R, n, COLS>::SMEM) != cudaSuccess)     \
                nb = 0;                                                                                          \
        }                                                                                                        \
        break;
        CBS_FOR_EACH_SIZE(CBS_CASE)
#undef CBS_CASE
    default: break;
    }
    cudaGetLastError();
    return nb;
}

// explicit instantiation helper
#define CBS_INSTANTIATE_LAUNCHERS(R)                                                                                 \
    template int rows_blocks<R>(const Plan<R>&);                                                                     \
    template int axis_pipe_blocks_per_sm<R>(int);                                                                    \
    template cudaError_t launch_rows_fwd<R>(const Plan<R>&, const cplx<R>*, const cplx<R>*, cplx<R>*, int, int,      \
                                            cudaStream_t);                                                           \
    template cudaError_t launch_rows_inv<R>(const Plan<R>&, cplx<R>*, const cplx<R>*, cplx<R>*, int, int, R, double*, \
                                            cudaStream_t);                                                           \
    template cudaError_t launch_rows_inv_fwd<R>(const Plan<R>&, cplx<R>*, const cplx<R>*, cplx<R>*, int, R, double*,  \
                                                cudaStream_t);                                                       \
    template bool fused_rows_ok<R>(const Plan<R>&);                                                                  \
    template cudaError_t launch_axis<R>(const Plan<R>&, cplx<R>*, int, cudaStream_t);                                \
    template cudaError_t launch_last<R>(const Plan<R>&, cplx<R>*, int, cudaStream_t);                                \
    template cudaError_t launch_plane_fwd<R>(const Plan<R>&, const cplx<R>*, const cplx<R>*, cplx<R>*, int,          \
                                             cudaStream_t);                                                          \
    template cudaError_t launch_plane_inv<R>(const Plan<R>&, cplx<R>*, const cplx<R>*, int, R, double*, cudaStream_t);

}  // namespace cbs

namespace cbs {
// declarations for translation units that only call the launchers
#define CBS_EXTERN_LAUNCHERS(R)                                                                                      \
    extern template int rows_blocks<R>(const Plan<R>&);                                                              \
    extern template int axis_pipe_blocks_per_sm<R>(int);                                                             \
    extern template cudaError_t launch_rows_fwd<R>(const Plan<R>&, const cplx<R>*, const cplx<R>*, cplx<R>*, int, int, \
                                                   cudaStream_t);                                                    \
    extern template cudaError_t launch_rows_inv<R>(const Plan<R>&, cplx<R>*, const cplx<R>*, cplx<R>*, int, int, R,   \
                                                   double*, cudaStream_t);                                           \
    extern template cudaError_t launch_rows_inv_fwd<R>(const Plan<R>&, cplx<R>*, const cplx<R>*, cplx<R>*, int, R,    \
                                                       double*, cudaStream_t);                                       \
    extern template bool fused_rows_ok<R>(const Plan<R>&);                                                           \
    extern template cudaError_t launch_axis<R>(const Plan<R>&, cplx<R>*, int, cudaStream_t);                         \
    extern template cudaError_t launch_last<R>(const Plan<R>&, cplx<R>*, int, cudaStream_t);                         \
    extern template cudaError_t launch_plane_fwd<R>(const Plan<R>&, const cplx<R>*, const cplx<R>*, cplx<R>*, int,   \
                                                    cudaStream_t);                                                   \
    extern template cudaError_t launch_plane_inv<R>(const Plan<R>&, cplx<R>*, const cplx<R>*, int, R, double*,       \
                                                    cudaStream_t);
}  // namespace cbs
