// last_cluster.cuh -- the last-axis step of the Born iteration split over a
// thread-block cluster, one CTA per field component.
//
// The step (forward FFT along the last axis, the per-wavenumber (L+I)^-1
// symbol of App. B.1 on all C components, inverse FFT along the last axis)
// couples the C components only through the symbol.  Here a cluster of C CTAs
// owns a tile of COLS x-columns (at one y in 3D) by all NL points of the last
// axis: CTA c transforms component c's tile in its own shared memory, the
// cluster synchronises, each CTA applies the symbol to its share of the
// wavenumbers reading and writing all C components' values through
// distributed shared memory, the cluster synchronises again, and each CTA
// inverse-transforms its component and stores it.
//
// Compared with one CTA holding all C components of a pencil, a CTA needs a
// C-th of the shared memory and registers, so the tile can be wider (whole
// 128-byte rows of the field along x) and more CTAs fit an SM.  Nothing here
// waits on anything but __syncthreads and the two cluster barriers; no CTA
// touches another's shared memory after the second barrier.
#pragma once
#include <cooperative_groups.h>

#include "born.cuh"

namespace cbs {

template <typename R, int NL, int RL, int COLS, int C> struct LastClusterCfg {
    static constexpr int T = NL / RL;             // threads per column transform
    static constexpr int THREADS = T * COLS;
    static constexpr size_t SMEM = (size_t)NL * COLS * sizeof(cplx<R>);
    static constexpr int KPER = (NL + C - 1) / C;  // wavenumbers whose symbol one CTA applies
    // resident CTAs an SM is sized for (register cap 65536 / (THREADS * MINB))
    static constexpr int MINB = THREADS <= 128 ? 4 : (THREADS <= 256 ? 3 : 1);
    // twiddles kept in registers only for 8 values a thread; with 12 or 16 they come from the table (L1)
    static constexpr bool TC = RL <= 8;
    static_assert(THREADS % 32 == 0 && THREADS <= 1024, "last-axis cluster block shape");
};

// grid: C * (D == 3 ? n1 : 1) * ceil(n0 / COLS), clusters of C along x (the C CTAs of one tile are
// consecutive); block: THREADS; dynamic shared memory: SMEM.
template <typename R, int NL, int RL, int COLS, int C>
__global__ void __launch_bounds__(LastClusterCfg<R, NL, RL, COLS, C>::THREADS, LastClusterCfg<R, NL, RL, COLS, C>::MINB)
k_last_cluster(Dims d, Symbol<R> Sy, cplx<R>* __restrict__ w, const cplx<R>* __restrict__ tw, int mode)
{
    namespace cg = cooperative_groups;
    using CT = cplx<R>;
    using Cfg = LastClusterCfg<R, NL, RL, COLS, C>;
    constexpr int T = Cfg::T;
    constexpr int D = C - 1;
    constexpr int np = plan_npass(NL, RL);
    extern __shared__ __align__(16) unsigned char smraw[];
    CT* S = reinterpret_cast<CT*>(smraw);  // [NL][COLS]: this CTA's component of the tile
    cg::cluster_group cl = cg::this_cluster();
    const int comp = (int)cl.block_rank();
    const long long tile = blockIdx.x / C;
    const int col = threadIdx.x % COLS, t = threadIdx.x / COLS;
    const int xblocks = (d.n0 + COLS - 1) / COLS;
    const int xb = (int)(tile % xblocks);
    const int i1 = (D == 3) ? (int)(tile / xblocks) : 0;
    const int i0 = xb * COLS + col;
    const bool valid = i0 < d.n0;
    const int ic0 = valid ? i0 : 0;
    const long long astride = (D == 3) ? (long long)d.n0 * d.n1 : (long long)d.n0;
    const long long base = (long long)comp * d.N + (D == 3 ? (long long)i1 * d.n0 : 0) + ic0;
    TwCache<NL, RL, CT> tc;
    if constexpr (Cfg::TC) tw_load<NL, RL, T>(tc, t, tw);
    CT v[RL];
#pragma unroll
    for (int s = 0; s < RL; ++s) v[s] = w[base + (long long)(t + T * slot_q<NL, RL, 0>(s)) * astride];
    fft_run<NL, RL, -1, false, 0, Cfg::TC>(v, S + col, COLS, t, tw, tc, BlockSync());
    __syncthreads();  // the last exchange's reads are done
#pragma unroll
    for (int s = 0; s < RL; ++s) S[(t + T * slot_q<NL, RL, np>(s)) * COLS + col] = v[s];
    cl.sync();  // every component of the tile is transformed
    {
        CT* Sc[C];
#pragma unroll
        for (int c = 0; c < C; ++c) Sc[c] = cl.map_shared_rank(S, (unsigned)c);
        CT tx[D];
        R k2c = Sy.k2[0][ic0];
        tx[0] = Sy.kt[0][ic0];
        if (D == 3) {
            tx[1] = Sy.kt[1][i1];
            k2c += Sy.k2[1][i1];
        }
        const int k_lo = comp * Cfg::KPER;
        const int k_hi = (k_lo + Cfg::KPER < NL) ? k_lo + Cfg::KPER : NL;
#pragma unroll 1
        for (int k = k_lo + t; k < k_hi; k += T) {
            tx[D - 1] = Sy.kt[D - 1][k];
            const R k2 = k2c + Sy.k2[D - 1][k];
            CT vv[C];
#pragma unroll
            for (int c = 0; c < C; ++c) vv[c] = Sc[c][k * COLS + col];
            apply_symbol<R, C>(Sy, mode, tx, k2, vv);
#pragma unroll
            for (int c = 0; c < C; ++c) Sc[c][k * COLS + col] = vv[c];
        }
    }
    cl.sync();  // every wavenumber of the tile has its symbol applied; no remote access after this
#pragma unroll
    for (int s = 0; s < RL; ++s) v[s] = S[(t + T * slot_q<NL, RL, 0>(s)) * COLS + col];
    fft_run<NL, RL, +1, false, 0, Cfg::TC>(v, S + col, COLS, t, tw, tc, BlockSync());
    if (valid) {
#pragma unroll
        for (int s = 0; s < RL; ++s) w[base + (long long)(t + T * slot_q<NL, RL, np>(s)) * astride] = v[s];
    }
}

}  // namespace cbs
