// baseline_cufft.cuh -- the comparison build of the Born iteration: the same
// step (eq. BornAlt, the App. B.1 symbol) with the transforms done by cuFFT
// (batched complex-to-complex plans over the C components) and everything else
// by plain grid-stride pointwise kernels, one pass over the field each:
//     w = B x + y;  w = FFT(w);  w = G(k) w;  w = IFFT(w);  x += nu B (w - x)
// It exists to be timed beside the fused kernels; the solver never uses it.
#pragma once
#include "born.cuh"

namespace cbs {

__device__ __forceinline__ void voxel_coords(const Dims& d, long long v, int& i0, int& i1, int& i2)
{
    i0 = (int)(v % d.n0);
    const long long rest = v / d.n0;
    i1 = (int)(rest % d.n1);
    i2 = (int)(rest / d.n1);
}

// w = B x + y over all components
template <typename R>
__global__ void k_base_pre(Dims d, Medium<R> M, const cplx<R>* __restrict__ x, const cplx<R>* __restrict__ y,
                           cplx<R>* __restrict__ w, int adj)
{
    const long long n = (long long)(d.D + 1) * d.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / d.N);
        const long long v = i % d.N;
        int i0, i1, i2;
        voxel_coords(d, v, i0, i1, i2);
        const RowB<R> rb = row_B(M, d.D, c, i1, i2, v - i0);
        w[i] = cadd(cmul(born_B(M, rb, i0, adj != 0), x[i]), y[i]);
    }
}

// the per-wavenumber symbol on the C components of each k (the 1/N of the
// unnormalised inverse transform is in the symbol constants)
template <typename R, int C>
__global__ void k_base_symbol(Dims d, Symbol<R> Sy, cplx<R>* __restrict__ w, int mode)
{
    constexpr int D = C - 1;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < d.N; v += (long long)gridDim.x * blockDim.x) {
        int i0, i1, i2;
        voxel_coords(d, v, i0, i1, i2);
        cplx<R> t[D];
        t[0] = Sy.kt[0][i0];
        t[1] = Sy.kt[1][i1];
        R k2 = Sy.k2[0][i0] + Sy.k2[1][i1];
        if constexpr (D == 3) {
            t[2] = Sy.kt[2][i2];
            k2 += Sy.k2[2][i2];
        }
        cplx<R> vv[C];
#pragma unroll
        for (int c = 0; c < C; ++c) vv[c] = w[c * d.N + v];
        apply_symbol<R, C>(Sy, mode, t, k2, vv);
#pragma unroll
        for (int c = 0; c < C; ++c) w[c * d.N + v] = vv[c];
    }
}

// x += nu B (w - x); per-block (|dx|^2, |x|^2) into partials[2 * blockIdx.x]
template <typename R>
__global__ void k_base_update(Dims d, Medium<R> M, cplx<R>* __restrict__ x, const cplx<R>* __restrict__ w, int adj,
                              R nu, double* __restrict__ partials)
{
    const long long n = (long long)(d.D + 1) * d.N;
    R s0 = (R)0, s1 = (R)0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / d.N);
        const long long v = i % d.N;
        int i0, i1, i2;
        voxel_coords(d, v, i0, i1, i2);
        const RowB<R> rb = row_B(M, d.D, c, i1, i2, v - i0);
        const cplx<R> xv = x[i];
        const cplx<R> del = cscale(cmul(born_B(M, rb, i0, adj != 0), csub(w[i], xv)), nu);
        const cplx<R> xn = cadd(xv, del);
        x[i] = xn;
        s0 += cabs2(del);
        s1 += cabs2(xn);
    }
    block_sum2(s0, s1, partials + 2 * (long long)blockIdx.x);
}

}  // namespace cbs
