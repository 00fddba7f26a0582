// plane.cuh -- x-y plane kernels of the Born iteration for 3D float32 fields.
//
// The forward half of one iteration (eq. BornAlt) needs w = FFT_xy(B x + y)
// before the last-axis symbol kernel, and the inverse half needs
// x <- x + nu B (IFFT_xy(w) - x) after it.  The row kernels do the x transform
// and the axis kernels the y transform in separate passes over HBM; here one
// pair of CTAs (a cluster of CL = 2) owns a whole (component, z) plane of
// NY x NX values, so both transforms happen on chip and each plane crosses HBM
// once per half-iteration: 116 B per voxel each way instead of 116 + 64.
//
// Each CTA of the pair holds half the plane's rows (ROWS_OWN rows of NX, row
// layout swizzled as in the row kernels) in shared memory.  The y transform of
// a column needs rows held by both CTAs: a CTA transforms its half of the
// columns, reading (forward) or writing (inverse) the other half-plane through
// distributed shared memory.  Cluster barriers separate the phases; nothing
// in these kernels waits on anything but those barriers and __syncthreads.
#pragma once
#include <cooperative_groups.h>

#include "born.cuh"

namespace cbs {

template <typename R, int NX, int NY, int CL> struct PlaneCfg {
    static constexpr int RX = 8, TX = NX / RX;  // x transform: TX threads per row
    static constexpr int RY = 8, TY = NY / RY;  // y transform: TY threads per column
    static constexpr int ROWS_OWN = NY / CL;    // plane rows held by one CTA
    static constexpr int COLS_OWN = NX / CL;    // columns one CTA transforms along y
    static constexpr int T0 = TX * ROWS_OWN < TY * COLS_OWN ? TX * ROWS_OWN : TY * COLS_OWN;
    static constexpr int TMAX = CL >= 4 ? 256 : 512;  // quarter planes: smaller CTAs, more of them an SM
    static constexpr int THREADS = T0 < TMAX ? T0 : TMAX;
    static constexpr int RB = THREADS / TX;     // rows per x batch
    static constexpr int CB = THREADS / TY;     // columns per y batch
    static constexpr int SL = sm_len<NX, true>();
    static constexpr size_t H_BYTES = (size_t)ROWS_OWN * SL * sizeof(cplx<R>);
    static constexpr size_t X_BYTES = (size_t)CB * NY * sizeof(cplx<R>);  // y-transform exchange
    static constexpr size_t SMEM = H_BYTES + X_BYTES;
    static constexpr int MINB = 1024 / THREADS;  // 64 registers a thread
    static_assert(THREADS % 32 == 0 && THREADS % TX == 0 && THREADS % TY == 0, "plane block shape");
    static_assert(ROWS_OWN % RB == 0 && COLS_OWN % CB == 0, "plane batches");
    static_assert(TX <= 32, "a row's threads must lie in one warp");
    static_assert(CL == 1 || CL == 2 || CL == 4, "one CTA, a pair or four per plane");
};

template <int CL> __device__ __forceinline__ unsigned plane_rank()
{
    if constexpr (CL == 1) return 0u;
    else return cooperative_groups::this_cluster().block_rank();
}

template <int CL> __device__ __forceinline__ void plane_sync()
{
    if constexpr (CL == 1) __syncthreads();
    else cooperative_groups::this_cluster().sync();
}

// shared-memory base of the part of the plane held by CTA `q` of the cluster
template <int CL, typename CT> __device__ __forceinline__ CT* plane_half(CT* H, unsigned q)
{
    if constexpr (CL == 1) return H;
    else return cooperative_groups::this_cluster().map_shared_rank(H, q);
}

// the plane row i1 (of NY) as held in the cluster: CTA i1 / ROWS_OWN, local row i1 % ROWS_OWN
template <int CL, int ROWS_OWN, int SL, typename CT> __device__ __forceinline__ CT* plane_row(CT* H, int i1)
{
    if constexpr (CL == 1) return H + i1 * SL;
    else return plane_half<CL>(H, (unsigned)(i1 / ROWS_OWN)) + (i1 % ROWS_OWN) * SL;
}

// w[c, z] = FFT_y FFT_x (B x + y) of plane (c, z) = blockIdx.x / CL.
// grid: C * n2 * CL (clusters of CL along x); block: THREADS.
template <typename R, int NX, int NY, int CL>
__global__ void __launch_bounds__(PlaneCfg<R, NX, NY, CL>::THREADS, PlaneCfg<R, NX, NY, CL>::MINB)
k_plane_fwd(Dims d, Medium<R> M, const cplx<R>* __restrict__ x, const cplx<R>* __restrict__ y,
            cplx<R>* __restrict__ w, const cplx<R>* __restrict__ twx, const cplx<R>* __restrict__ twy, int adj)
{
    using CT = cplx<R>;
    using Cfg = PlaneCfg<R, NX, NY, CL>;
    constexpr int RX = Cfg::RX, TX = Cfg::TX, RY = Cfg::RY, TY = Cfg::TY, SL = Cfg::SL;
    extern __shared__ __align__(16) unsigned char smraw[];
    CT* H = reinterpret_cast<CT*>(smraw);
    CT* X = reinterpret_cast<CT*>(smraw + Cfg::H_BYTES);
    const unsigned rank = plane_rank<CL>();
    const long long plane = blockIdx.x / CL;
    const int c = (int)(plane / d.n2), z = (int)(plane % d.n2);
    const long long pbase = (long long)z * NY * NX;  // voxel index of the plane's first value
    const long long fplane = (long long)c * d.N + pbase;
    // x transforms of the rows this CTA holds: w_row = FFT_x(B x + y)
    {
        const int lr = threadIdx.x / TX, t = threadIdx.x % TX;
        TwCache<NX, RX, CT> tc;
        tw_load<NX, RX, TX>(tc, t, twx);
        constexpr int np = plan_npass(NX, RX);
#pragma unroll 1
        for (int b = 0; b < Cfg::ROWS_OWN / Cfg::RB; ++b) {
            const int yl = b * Cfg::RB + lr;
            const int i1 = (int)rank * Cfg::ROWS_OWN + yl;
            const long long vbase = pbase + (long long)i1 * NX;
            const long long fbase = fplane + (long long)i1 * NX;
            const RowB<R> rb = row_B(M, d.D, c, i1, z, vbase);
            CT v[RX];
#pragma unroll
            for (int s = 0; s < RX; ++s) {
                const int i0 = t + TX * slot_q<NX, RX, 0>(s);
                const CT b_ = born_B(M, rb, i0, adj != 0);
                v[s] = cadd(cmul(b_, x[fbase + i0]), y[fbase + i0]);
            }
            CT* row = H + yl * SL;
            fft_run<NX, RX, -1, true>(v, row, 1, t, twx, tc, RowSync<TX>());
            RowSync<TX>()();
#pragma unroll
            for (int s = 0; s < RX; ++s) row[row_swizzle<NX>(t + TX * slot_q<NX, RX, np>(s))] = v[s];
        }
    }
    plane_sync<CL>();
    // y transforms of this CTA's columns, rows read from both halves
    {
        const int col = threadIdx.x % Cfg::CB, t = threadIdx.x / Cfg::CB;
        TwCache<NY, RY, CT> tc;
        tw_load<NY, RY, TY>(tc, t, twy);
        constexpr int np = plan_npass(NY, RY);
#pragma unroll 1
        for (int b = 0; b < Cfg::COLS_OWN / Cfg::CB; ++b) {
            const int i0 = (int)rank * Cfg::COLS_OWN + b * Cfg::CB + col;
            const int sw = row_swizzle<NX>(i0);
            CT v[RY];
#pragma unroll
            for (int s = 0; s < RY; ++s) {
                const int i1 = t + TY * slot_q<NY, RY, 0>(s);
                v[s] = plane_row<CL, Cfg::ROWS_OWN, SL>(H, i1)[sw];
            }
            fft_run<NY, RY, -1>(v, X + col, Cfg::CB, t, twy, tc, BlockSync());
#pragma unroll
            for (int s = 0; s < RY; ++s)
                w[fplane + (long long)(t + TY * slot_q<NY, RY, np>(s)) * NX + i0] = v[s];
        }
    }
    plane_sync<CL>();  // the other CTA has finished reading this half-plane
}

// x[c, z] += nu B (IFFT_x IFFT_y w - x) on plane (c, z), with the per-block
// norm partials (|dx|^2, |x|^2) of the update in partials[2 * blockIdx.x].
template <typename R, int NX, int NY, int CL>
__global__ void __launch_bounds__(PlaneCfg<R, NX, NY, CL>::THREADS, PlaneCfg<R, NX, NY, CL>::MINB)
k_plane_inv(Dims d, Medium<R> M, cplx<R>* __restrict__ x, const cplx<R>* __restrict__ w,
            const cplx<R>* __restrict__ twx, const cplx<R>* __restrict__ twy, int adj, R nu,
            double* __restrict__ partials)
{
    using CT = cplx<R>;
    using Cfg = PlaneCfg<R, NX, NY, CL>;
    constexpr int RX = Cfg::RX, TX = Cfg::TX, RY = Cfg::RY, TY = Cfg::TY, SL = Cfg::SL;
    extern __shared__ __align__(16) unsigned char smraw[];
    CT* H = reinterpret_cast<CT*>(smraw);
    CT* X = reinterpret_cast<CT*>(smraw + Cfg::H_BYTES);
    const unsigned rank = plane_rank<CL>();
    const long long plane = blockIdx.x / CL;
    const int c = (int)(plane / d.n2), z = (int)(plane % d.n2);
    const long long pbase = (long long)z * NY * NX;
    const long long fplane = (long long)c * d.N + pbase;
    // inverse y transforms of this CTA's columns, results written to the half that holds each row
    {
        const int col = threadIdx.x % Cfg::CB, t = threadIdx.x / Cfg::CB;
        TwCache<NY, RY, CT> tc;
        tw_load<NY, RY, TY>(tc, t, twy);
        constexpr int np = plan_npass(NY, RY);
#pragma unroll 1
        for (int b = 0; b < Cfg::COLS_OWN / Cfg::CB; ++b) {
            const int i0 = (int)rank * Cfg::COLS_OWN + b * Cfg::CB + col;
            const int sw = row_swizzle<NX>(i0);
            CT v[RY];
#pragma unroll
            for (int s = 0; s < RY; ++s) v[s] = w[fplane + (long long)(t + TY * slot_q<NY, RY, 0>(s)) * NX + i0];
            fft_run<NY, RY, +1>(v, X + col, Cfg::CB, t, twy, tc, BlockSync());
#pragma unroll
            for (int s = 0; s < RY; ++s) {
                const int i1 = t + TY * slot_q<NY, RY, np>(s);
                plane_row<CL, Cfg::ROWS_OWN, SL>(H, i1)[sw] = v[s];
            }
        }
    }
    plane_sync<CL>();
    // inverse x transforms of the rows this CTA holds, then the Born update
    R s0 = (R)0, s1 = (R)0;
    {
        const int lr = threadIdx.x / TX, t = threadIdx.x % TX;
        const TwCache<NX, RX, CT> tc{};  // twiddles from the table: the prefetched update operands need the registers
        constexpr int np = plan_npass(NX, RX);
#pragma unroll 1
        for (int b = 0; b < Cfg::ROWS_OWN / Cfg::RB; ++b) {
            const int yl = b * Cfg::RB + lr;
            const int i1 = (int)rank * Cfg::ROWS_OWN + yl;
            const long long vbase = pbase + (long long)i1 * NX;
            const long long fbase = fplane + (long long)i1 * NX;
            const RowB<R> rb = row_B(M, d.D, c, i1, z, vbase);
            CT* row = H + yl * SL;
            CT v[RX];
#pragma unroll
            for (int s = 0; s < RX; ++s) v[s] = row[row_swizzle<NX>(t + TX * slot_q<NX, RX, 0>(s))];
            // the update's loads (x, B at the output positions) overlap the transform
            CT xv[RX], bv[RX];
#pragma unroll
            for (int s = 0; s < RX; ++s) {
                const int i0 = t + TX * slot_q<NX, RX, np>(s);
                xv[s] = x[fbase + i0];
                bv[s] = born_B(M, rb, i0, adj != 0);
            }
            fft_run<NX, RX, +1, true, 0, false>(v, row, 1, t, twx, tc, RowSync<TX>());
#pragma unroll
            for (int s = 0; s < RX; ++s) {
                const CT del = cscale(cmul(bv[s], csub(v[s], xv[s])), nu);
                const CT xn = cadd(xv[s], del);
                x[fbase + t + TX * slot_q<NX, RX, np>(s)] = xn;
                s0 += cabs2(del);
                s1 += cabs2(xn);
            }
        }
    }
    block_sum2(s0, s1, partials + 2 * (long long)blockIdx.x);
}

}  // namespace cbs
