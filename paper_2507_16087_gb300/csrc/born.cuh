// born.cuh -- fused kernels of the split-preconditioned Born iteration.
//
// One iteration of eq. BornAlt / Algorithm 1 (Stanziola et al.),
//     z = (L+I)^-1 (B x + y),   x <- x + nu B (z - x),   B = I - V,
// on a D-dim grid (D = 2, 3) with C = D+1 components, runs as
//     rows_fwd     w = B x + y, forward FFT along x               (per row)
//     axis_fft     forward FFT along y (3D only)                  (per y-pencil tile)
//     last_symbol  forward FFT along the last axis, the per-wavenumber
//                  (L+I)^-1 symbol of App. B.1 on all C components,
//                  inverse FFT along the last axis                (per pencil tile)
//     axis_fft     inverse FFT along y (3D only)
//     rows_inv     inverse FFT along x, update of x, norm partials (per row)
// The same kernels with other modes give the scaled operator A_s x = L x + V x
// (residual y - A_s x) and the adjoint (A_s^H, conj(B), [(L+I)^-1]^H).
//
// Field layout: [C][n2][n1][n0] interleaved complex, x fastest.
// Medium layout: rs[eta][N] = (S+ rho)_eta / lambda1, kp[N] = 1/(rho c0^2 lambda2),
// et[N] = 2 alpha c0 / omega; gamma from per-axis tables at centres (gc) and
// at the staggered points (gs).  V is never stored: per voxel
//   v_eta = rs_eta * gamma_eta - a1/lambda1 + i (rs_eta omega)    ... minus i Im(a1)/lambda1
//   v_p   = kp [(gamma + et omega) + i (omega - gamma et)] - a2/lambda2
// (eq. LV with q = (i omega + gamma)/(rho c^2), c^2 of eq. 118).
#pragma once
#include <cuda.h>  // CUtensorMap (the tensor-copy descriptor type; no driver calls here)

#include "fft.cuh"

namespace cbs {

enum RowsFwdMode { FWD_BORN = 0, FWD_COPY = 1 };
enum RowsInvMode { INV_BORN = 0, INV_RESID = 1, INV_PLAIN = 2, INV_APPLY = 3 };
enum SymbolMode { SYM_GREEN = 0, SYM_GREEN_ADJ = 1, SYM_L = 2, SYM_L_ADJ = 3 };

struct Dims {
    int D;          // 2 or 3
    int n0, n1, n2; // extents (n2 = 1 in 2D)
    long long N;    // voxels
};

template <typename R> struct Medium {
    const R* rs[3];
    const R* kp;
    const R* et;
    const R* gc[3];
    const R* gs[3];
    R omega;
    R a1r, a1i, a2r, a2i;  // a_j / lambda_j
};

template <typename R> struct Symbol {
    cplx<R> P;     // lambda1 / (a1 + lambda1) * scale
    cplx<R> Pu;    // lambda1 / (a1 + lambda1)
    cplx<R> c1;    // i sqrt(lambda1 lambda2)
    cplx<R> c2;    // lambda2 (a1 + lambda1)
    cplx<R> c3;    // (a1 + lambda1)(a2 + lambda2)
    cplx<R> la1;   // a1 / lambda1
    cplx<R> la2;   // a2 / lambda2
    R isq;         // 1 / sqrt(lambda1 lambda2)
    R scale;       // 1 / N (inverse-transform normalisation)
    const cplx<R>* kt[3];  // t_eta = k_eta exp(i k_eta dx / 2)
    const R* k2[3];        // k_eta^2
};

// Per-row view of B = 1 - v for component c (conj for the adjoint).  Along a
// row only x varies, so the gamma terms of the other axes are row constants.
template <typename R> struct RowB {
    const R* g0;  // gamma along x: staggered table for u_x, centre table otherwise
    R grest;      // gamma contributions of y (and z)
    const R* m0;  // rs_c (velocity) or kp (pressure), at the row start
    const R* m1;  // et (pressure), at the row start
    bool pres;
};

template <typename R>
__device__ __forceinline__ RowB<R> row_B(const Medium<R>& M, int D, int c, int i1, int i2, long long vbase)
{
    RowB<R> rb;
    rb.pres = (c == D);
    rb.g0 = (c == 0) ? M.gs[0] : M.gc[0];
    R g = (c == 1) ? __ldg(M.gs[1] + i1) : __ldg(M.gc[1] + i1);
    if (D == 3) g += (c == 2) ? __ldg(M.gs[2] + i2) : __ldg(M.gc[2] + i2);
    rb.grest = g;
    const R* rsc = (c == 0) ? M.rs[0] : ((c == 1) ? M.rs[1] : M.rs[2]);
    rb.m0 = (rb.pres ? M.kp : rsc) + vbase;
    rb.m1 = M.et + vbase;
    return rb;
}

// B from the row's medium values already in registers (m0 = rs_c or kp, m1 = et)
template <typename R>
__device__ __forceinline__ cplx<R> born_B_vals(const Medium<R>& M, bool pres, R g, R m0, R m1, bool adj)
{
    R vr, vi;
    if (!pres) {
        vr = m0 * g - M.a1r;
        vi = m0 * M.omega - M.a1i;
    } else {
        vr = m0 * (g + m1 * M.omega) - M.a2r;
        vi = m0 * (M.omega - g * m1) - M.a2i;
    }
    return mk<cplx<R>, R>((R)1 - vr, adj ? vi : -vi);
}

template <typename R>
__device__ __forceinline__ cplx<R> born_B(const Medium<R>& M, const RowB<R>& rb, int i0, bool adj)
{
    const R g = __ldg(rb.g0 + i0) + rb.grest;
    R vr, vi;
    if (!rb.pres) {
        const R r = __ldg(rb.m0 + i0);
        vr = r * g - M.a1r;
        vi = r * M.omega - M.a1i;
    } else {
        const R k = __ldg(rb.m0 + i0), e = __ldg(rb.m1 + i0);
        vr = k * (g + e * M.omega) - M.a2r;
        vi = k * (M.omega - g * e) - M.a2i;
    }
    return mk<cplx<R>, R>((R)1 - vr, adj ? vi : -vi);
}

template <int T> struct RowSync {
    __device__ __forceinline__ void operator()() const
    {
        if constexpr (T <= 32) __syncwarp();
        else __syncthreads();
    }
};
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Block-wide sum of two values; thread 0 writes them to out[0..1].  Warps sum
// in the accumulator type A (float32 for the float32 path: float64 arithmetic
// is scarce on this GPU), the per-warp sums are combined in float64.
template <typename A> __device__ __forceinline__ void block_sum2(A a_in, A b_in, double* out)
{
    __shared__ double red[2][32];
    A aa = a_in, bb = b_in;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        aa += __shfl_down_sync(0xffffffffu, aa, o);
        bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    double a = (double)aa, b = (double)bb;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { red[0][w] = a; red[1][w] = b; }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = lane < nw ? red[0][lane] : 0.0;
        b = lane < nw ? red[1][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (lane == 0) { out[0] = a; out[1] = b; }
    }
}

// Rows of one block: 256 threads when the rows' shared memory fits in the
// static limit (48 KiB less the reduction scratch).
template <typename R, int NX, int RX> struct RowCfg {
    static constexpr int T = NX / RX;
    // 256 threads (8 or 12 values each), or 2048 values per block with 16 values per thread
    static constexpr int ROWS0 = (T >= 256) ? 1 : (RX >= 16 ? (2048 / NX < 1 ? 1 : 2048 / NX) : 256 / T);
    static constexpr int SL = sm_len<NX, true>();  // row length in shared memory (swizzled / skewed)
    static constexpr int CAP0 = 47104 / (SL * (int)sizeof(cplx<R>));
    static constexpr int CAP = CAP0 < 1 ? 1 : CAP0;
    static constexpr int G = T < 32 ? 32 / T : 1;  // rows per warp: blocks are whole warps
    static constexpr int ROWS1 = ((ROWS0 < CAP ? ROWS0 : CAP) / G) * G;
    static constexpr int ROWS = ROWS1 < G ? G : ROWS1;
    static constexpr int THREADS = T * ROWS;
};

// ---------------------------------------------------------------- rows_fwd
// grid: ceil(C * N / n0 / ROWS); block: THREADS.  w[row] = FFT_x(B x + y) (FWD_BORN)
// or FFT_x(x) (FWD_COPY).
template <typename R, int NX, int RX>
__global__ void __launch_bounds__(RowCfg<R, NX, RX>::THREADS, sizeof(R) == 4 ? 4 : 1)
k_rows_fwd(Dims d, Medium<R> M, const cplx<R>* __restrict__ x, const cplx<R>* __restrict__ y,
           cplx<R>* __restrict__ w, const cplx<R>* __restrict__ tw, int mode, int adj)
{
    using CT = cplx<R>;
    using Cfg = RowCfg<R, NX, RX>;
    constexpr int T = Cfg::T;
    __shared__ CT sm[Cfg::ROWS * Cfg::SL];
    const int lr = threadIdx.x / T, t = threadIdx.x % T;
    const long long rows_per_comp = d.N / NX;
    const long long C = d.D + 1;
    long long row = (long long)blockIdx.x * Cfg::ROWS + lr;
    const bool valid = row < C * rows_per_comp;
    if (!valid) row = 0;
    const int c = (int)(row / rows_per_comp);
    const long long rest = row % rows_per_comp;
    const int i1 = (int)(rest % d.n1), i2 = (int)(rest / d.n1);
    const long long vbase = rest * NX;
    const long long fbase = (long long)c * d.N + vbase;
    const RowB<R> rb = row_B(M, d.D, c, i1, i2, vbase);
    TwCache<NX, RX, CT> tc;
    tw_load<NX, RX, T>(tc, t, tw);
    CT v[RX];
#pragma unroll
    for (int s = 0; s < RX; ++s) {
        const int i0 = t + T * slot_q<NX, RX, 0>(s);
        CT xv = x[fbase + i0];
        if (mode == FWD_BORN) {
            const CT b = born_B(M, rb, i0, adj != 0);
            v[s] = cadd(cmul(b, xv), y[fbase + i0]);
        } else {
            v[s] = xv;
        }
    }
    fft_run<NX, RX, -1, true>(v, sm + lr * Cfg::SL, 1, t, tw, tc, RowSync<T>());
    if (valid) {
        constexpr int np = plan_npass(NX, RX);
#pragma unroll
        for (int s = 0; s < RX; ++s) w[fbase + t + T * slot_q<NX, RX, np>(s)] = v[s];
    }
}

// ---------------------------------------------------------------- rows_inv
// INV_BORN:  z = IFFT_x(w);  dx = nu B (z - x);  x += dx;  partial (|dx|^2, |x|^2)
// INV_RESID: z = IFFT_x(w) = L x;  r = y - z - v x;  w <- r;  partial (|r|^2, |y|^2)
// INV_APPLY: z = IFFT_x(w) = L x;  w <- z + v x;           partial (|w|^2, 0)
// INV_PLAIN: w <- IFFT_x(w);                               partial (|w|^2, 0)
// BORN = true: the hot Born-update instance (mode must be INV_BORN); false:
// the residual / apply / plain instance.
template <typename R, int NX, int RX, bool BORN>
__global__ void __launch_bounds__(RowCfg<R, NX, RX>::THREADS, (sizeof(R) == 4 && BORN) ? 3 : 1)
k_rows_inv(Dims d, Medium<R> M, cplx<R>* __restrict__ x, const cplx<R>* __restrict__ y, cplx<R>* __restrict__ w,
           const cplx<R>* __restrict__ tw, int mode_in, int adj, R nu, double* __restrict__ partials)
{
    const int mode = BORN ? (int)INV_BORN : mode_in;
    using CT = cplx<R>;
    using Cfg = RowCfg<R, NX, RX>;
    constexpr int T = Cfg::T;
    constexpr int np = plan_npass(NX, RX);
    __shared__ CT sm[Cfg::ROWS * Cfg::SL];
    const int lr = threadIdx.x / T, t = threadIdx.x % T;
    const long long rows_per_comp = d.N / NX;
    const long long C = d.D + 1;
    long long row = (long long)blockIdx.x * Cfg::ROWS + lr;
    const bool valid = row < C * rows_per_comp;
    if (!valid) row = 0;
    const int c = (int)(row / rows_per_comp);
    const long long rest = row % rows_per_comp;
    const int i1 = (int)(rest % d.n1), i2 = (int)(rest / d.n1);
    const long long vbase = rest * NX;
    const long long fbase = (long long)c * d.N + vbase;
    const RowB<R> rb = row_B(M, d.D, c, i1, i2, vbase);
    TwCache<NX, RX, CT> tc;
    tw_load<NX, RX, T>(tc, t, tw);
    CT v[RX];
#pragma unroll
    for (int s = 0; s < RX; ++s) v[s] = w[fbase + t + T * slot_q<NX, RX, 0>(s)];
    // issue the epilogue's loads (x, B, y at the output positions) before the
    // transform so their latency overlaps it
    CT xv[RX], bv[RX], yv[BORN ? 1 : RX];
    if (mode != INV_PLAIN) {
#pragma unroll
        for (int s = 0; s < RX; ++s) {
            const int i0 = t + T * slot_q<NX, RX, np>(s);
            xv[s] = x[fbase + i0];
            bv[s] = born_B(M, rb, i0, adj != 0);
            if constexpr (!BORN) {
                if (mode == INV_RESID) yv[s] = y[fbase + i0];
            }
        }
    }
    fft_run<NX, RX, +1, true>(v, sm + lr * Cfg::SL, 1, t, tw, tc, RowSync<T>());
    R s0 = (R)0, s1 = (R)0;
#pragma unroll
    for (int s = 0; s < RX; ++s) {
        const long long f = fbase + t + T * slot_q<NX, RX, np>(s);
        if (mode == INV_PLAIN) {
            if (valid) w[f] = v[s];
            s0 += cabs2(v[s]);
            continue;
        }
        const CT b = bv[s];
        if (mode == INV_BORN) {
            const CT del = cscale(cmul(b, csub(v[s], xv[s])), nu);
            const CT xn = cadd(xv[s], del);
            if (valid) x[f] = xn;
            s0 += cabs2(del);
            s1 += cabs2(xn);
        } else if constexpr (!BORN) {
            // v x = (1 - B) x
            const CT vx = csub(xv[s], cmul(b, xv[s]));
            if (mode == INV_RESID) {
                const CT r = csub(yv[s], cadd(v[s], vx));
                if (valid) w[f] = r;
                s0 += cabs2(r);
                s1 += cabs2(yv[s]);
            } else {
                const CT a = cadd(v[s], vx);
                if (valid) w[f] = a;
                s0 += cabs2(a);
            }
        }
    }
    if (!valid) { s0 = (R)0; s1 = (R)0; }
    block_sum2(s0, s1, partials + 2 * (long long)blockIdx.x);
}

// ---------------------------------------------------------------- axis_fft
// FFT along axis 1 (y) of a 3D field, in place, COLS x-columns per block.
// grid: C * n2 * ceil(n0 / COLS); block: (NA/RA) * COLS.
template <int NA, int RA, int COLS> struct AxisCfg {
    static constexpr int T = NA / RA;
    static constexpr int THREADS = T * COLS;
};

template <typename R, int NA, int RA, int COLS, int S>
__global__ void __launch_bounds__(AxisCfg<NA, RA, COLS>::THREADS)
k_axis_fft(Dims d, cplx<R>* __restrict__ w, const cplx<R>* __restrict__ tw)
{
    using CT = cplx<R>;
    constexpr int T = NA / RA;
    extern __shared__ __align__(16) unsigned char smraw[];
    CT* sm = reinterpret_cast<CT*>(smraw);
    const int col = threadIdx.x % COLS, t = threadIdx.x / COLS;
    const int xblocks = (d.n0 + COLS - 1) / COLS;
    const int xb = blockIdx.x % xblocks;
    const long long rest = blockIdx.x / xblocks;  // c * n2 + i2
    const int i0 = xb * COLS + col;
    const bool valid = i0 < d.n0;
    const long long base = rest * (long long)d.n0 * d.n1 + (valid ? i0 : 0);
    TwCache<NA, RA, CT> tc;
    tw_load<NA, RA, T>(tc, t, tw);
    CT v[RA];
#pragma unroll
    for (int s = 0; s < RA; ++s) v[s] = w[base + (long long)(t + T * slot_q<NA, RA, 0>(s)) * d.n0];
    fft_run<NA, RA, S>(v, sm + col, COLS, t, tw, tc, BlockSync());
    if (valid) {
        constexpr int np = plan_npass(NA, RA);
#pragma unroll
        for (int s = 0; s < RA; ++s) w[base + (long long)(t + T * slot_q<NA, RA, np>(s)) * d.n0] = v[s];
    }
}

// ------------------------------------------------------------- last_symbol
// Forward FFT along the last axis, per-wavenumber symbol on all C components,
// inverse FFT along the last axis.  grid: (D == 3 ? n1 : 1) * ceil(n0 / COLS).
// 1 / m for the symbol's scale / |mu|^2: float32 takes the approximate reciprocal (2 ulp), float64 the
// exact quotient
template <bool FAST, typename R> __device__ __forceinline__ R sym_quot(R a, R m)
{
    if constexpr (FAST && sizeof(R) == 4) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"((float)m));
        return a * r;
    } else {
        return a / m;
    }
}

template <typename R, int C, bool FAST = false>
__device__ __forceinline__ void apply_symbol(const Symbol<R>& Sy, int mode, const cplx<R>* t, R k2, cplx<R>* v)
{
    using CT = cplx<R>;
    constexpr int D = C - 1;
    if (mode == SYM_GREEN || mode == SYM_GREEN_ADJ) {
        const bool adj = mode == SYM_GREEN_ADJ;
        const CT P = adj ? cconj(Sy.P) : Sy.P;
        const CT Pu = adj ? cconj(Sy.Pu) : Sy.Pu;
        const CT c1 = adj ? cconj(Sy.c1) : Sy.c1;
        const CT c2 = adj ? cconj(Sy.c2) : Sy.c2;
        const CT c3 = adj ? cconj(Sy.c3) : Sy.c3;
        // mu = k^2 + (a1 + l1)(a2 + l2);  im = scale / mu
        const CT mu = mk<CT, R>(k2 + c3.x, c3.y);
        const R inv = sym_quot<FAST>(Sy.scale, cabs2(mu));
        const CT im = mk<CT, R>(mu.x * inv, -mu.y * inv);
        CT s = mk<CT, R>((R)0, (R)0);
#pragma unroll
        for (int e = 0; e < D; ++e) s = cadd(s, cmulc(v[e], t[e]));  // sum conj(t_e) v_e
        const CT vp = v[D];
        const CT tmp = cmul(cadd(cmul(Pu, s), cmul(c1, vp)), im);
#pragma unroll
        for (int e = 0; e < D; ++e) v[e] = csub(cmul(P, v[e]), cmul(t[e], tmp));
        v[D] = cmul(csub(cmul(c2, vp), cmul(c1, s)), im);
    } else {
        const bool adj = mode == SYM_L_ADJ;
        const CT la1 = adj ? cconj(Sy.la1) : Sy.la1;
        const CT la2 = adj ? cconj(Sy.la2) : Sy.la2;
        const R g = adj ? -Sy.isq * Sy.scale : Sy.isq * Sy.scale;  // off-diagonal i -> -i for L^H
        const CT vp = v[D];
        CT sp = cmul(la2, vp);
        sp = cscale(sp, Sy.scale);
#pragma unroll
        for (int e = 0; e < D; ++e) {
            const CT ve = v[e];
            // i t_e g v_p  and  i conj(t_e) g v_e
            v[e] = cadd(cscale(cmul(la1, ve), Sy.scale), cscale(mul_si<1>(cmul(t[e], vp)), g));
            sp = cadd(sp, cscale(mul_si<1>(cmulc(ve, t[e])), g));
        }
        v[D] = sp;
    }
}

// two blocks an SM when a block has fewer than 512 threads; with 512 (the 1024- and 2048-point and 512-point
// 8-column tiles) the C transforms keep their registers (a 64-register cap spilled them) at one block an SM
// VAR (measured variants): bit 0 approximate float32 reciprocal in the symbol, bit 1 each twiddle read once
// for all C transforms
template <typename R, int NL, int RL, int COLS, int C, int VAR = 0>
__global__ void __launch_bounds__((NL / RL) * COLS, ((NL / RL) * COLS >= 512) ? 1 : 2)
k_last_symbol(Dims d, Symbol<R> Sy, cplx<R>* __restrict__ w, const cplx<R>* __restrict__ tw, int mode)
{
    constexpr bool FAST = (VAR & 1) != 0;
    constexpr bool SHTW = (VAR & 2) != 0;
    using CT = cplx<R>;
    constexpr int T = NL / RL;
    constexpr int D = C - 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    CT* sm = reinterpret_cast<CT*>(smraw);
    const int col = threadIdx.x % COLS, t = threadIdx.x / COLS;
    const int xblocks = (d.n0 + COLS - 1) / COLS;
    const int xb = blockIdx.x % xblocks;
    const int i1 = (D == 3) ? (int)(blockIdx.x / xblocks) : 0;
    const int i0 = xb * COLS + col;
    const bool valid = i0 < d.n0;
    const long long astride = (D == 3) ? (long long)d.n0 * d.n1 : (long long)d.n0;
    const long long base = (D == 3 ? (long long)i1 * d.n0 : 0) + (valid ? i0 : 0);
    CT v[C][RL];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int s = 0; s < RL; ++s)
            v[c][s] = w[(long long)c * d.N + base + (long long)(t + T * slot_q<NL, RL, 0>(s)) * astride];
    const int cstride = NL * COLS;
    fft_run_multi<NL, RL, C, -1, 0, SHTW>(v, sm + col, COLS, cstride, t, tw, BlockSync());
    // per-wavenumber symbol
    constexpr int np = plan_npass(NL, RL);
    const int ic0 = valid ? i0 : 0;
    CT tx[D];
    R k2c = Sy.k2[0][ic0];
    tx[0] = Sy.kt[0][ic0];
    if (D == 3) {
        tx[1] = Sy.kt[1][i1];
        k2c += Sy.k2[1][i1];
    }
#pragma unroll
    for (int s = 0; s < RL; ++s) {
        const int il = t + T * slot_q<NL, RL, np>(s);
        tx[D - 1] = Sy.kt[D - 1][il];
        const R k2 = k2c + Sy.k2[D - 1][il];
        CT vv[C];
#pragma unroll
        for (int c = 0; c < C; ++c) vv[c] = v[c][s];
        apply_symbol<R, C, FAST>(Sy, mode, tx, k2, vv);
#pragma unroll
        for (int c = 0; c < C; ++c) v[c][s] = vv[c];
    }
    // the thread owns the same positions after the forward transform; reorder
    // its registers into the entry order of the inverse transform
#pragma unroll
    for (int c = 0; c < C; ++c) permute_slots<NL, RL, np, 0>(v[c]);
    fft_run_multi<NL, RL, C, +1, 0, SHTW>(v, sm + col, COLS, cstride, t, tw, BlockSync());
    if (valid) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int s = 0; s < RL; ++s)
                w[(long long)c * d.N + base + (long long)(t + T * slot_q<NL, RL, np>(s)) * astride] = v[c][s];
    }
}

// ------------------------------------------------- bulk (TMA) staged rows
// cp.async.bulk copies of a block's contiguous rows into shared memory,
// completed on an mbarrier.  Every wait is bounded: on timeout the kernel
// records an error code in *err and leaves without touching its outputs.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// the same copy with an L2 eviction-priority hint (an L2 cache policy made by createpolicy)
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
// L2 policies: data read once (evicted first) and data the next kernel reads again (evicted last)
__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

constexpr int kBulkWaitLimit = 1 << 22;  // try_wait rounds before a copy is declared lost
constexpr int kErrBulkTimeout = 1;
constexpr int kErrTileAlign = 2;  // a shared-memory tile not on the 128-byte boundary tensor copies want

// true when the phase completed; false after kBulkWaitLimit rounds
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, int limit = kBulkWaitLimit)
{
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// orders this thread's shared-memory accesses before later bulk / tensor copies that read or overwrite the buffer
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <typename R, int NX, int RX> struct BulkCfg {
    using Rc = RowCfg<R, NX, RX>;
    static constexpr int ROWS = Rc::ROWS;
    static constexpr int T = Rc::T;
    static constexpr int THREADS = Rc::THREADS;
    static constexpr int ELEMS = ROWS * NX;
    // field A (x or w), field B (y or x), medium m0, medium m1, two mbarriers
    static constexpr size_t SMEM = 2 * (size_t)ELEMS * sizeof(cplx<R>) + 2 * (size_t)ELEMS * sizeof(R) + 16;
    // the exchange reuses field A's rows in place; every copy is a multiple of 16 bytes
    static constexpr bool OK = (Rc::SL == NX) && ((size_t)ELEMS * sizeof(R)) % 16 == 0;
};

// Born forward rows with bulk-staged x, y and medium (requires every block's
// rows to lie in one component: rows_per_comp % ROWS == 0).
template <typename R, int NX, int RX>
__global__ void __launch_bounds__(BulkCfg<R, NX, RX>::THREADS, sizeof(R) == 4 ? 4 : 1)
k_rows_fwd_bulk(Dims d, Medium<R> M, const cplx<R>* __restrict__ x, const cplx<R>* __restrict__ y,
                cplx<R>* __restrict__ w, const cplx<R>* __restrict__ tw, int adj, int* err)
{
    using CT = cplx<R>;
    using Cfg = BulkCfg<R, NX, RX>;
    constexpr int T = Cfg::T;
    constexpr int E = Cfg::ELEMS;
    extern __shared__ __align__(128) unsigned char smraw[];
    CT* xs = reinterpret_cast<CT*>(smraw);
    CT* ys = xs + E;
    R* m0s = reinterpret_cast<R*>(ys + E);
    R* m1s = m0s + E;
    uint64_t* bar = reinterpret_cast<uint64_t*>(m1s + E);
    const int lr = threadIdx.x / T, t = threadIdx.x % T;
    const long long rows_per_comp = d.N / NX;
    const long long row0 = (long long)blockIdx.x * Cfg::ROWS;
    const int c = (int)(row0 / rows_per_comp);
    const long long rest0 = row0 % rows_per_comp;
    const long long vbase0 = rest0 * NX;
    const long long fbase0 = (long long)c * d.N + vbase0;
    const bool pres = (c == d.D);
    const R* m0g = (pres ? M.kp : (c == 0 ? M.rs[0] : (c == 1 ? M.rs[1] : M.rs[2]))) + vbase0;
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t fb = E * sizeof(CT), mb = E * sizeof(R);
        mbar_expect_tx(bar, 2 * fb + (pres ? 2 : 1) * mb);
        bulk_g2s(xs, x + fbase0, fb, bar);
        bulk_g2s(ys, y + fbase0, fb, bar);
        bulk_g2s(m0s, m0g, mb, bar);
        if (pres) bulk_g2s(m1s, M.et + vbase0, mb, bar);
    }
    // overlap: twiddles and row constants while the copies fly
    TwCache<NX, RX, CT> tc;
    tw_load<NX, RX, T>(tc, t, tw);
    const long long rest = rest0 + lr;
    const int i1 = (int)(rest % d.n1), i2 = (int)(rest / d.n1);
    const RowB<R> rb = row_B(M, d.D, c, i1, i2, rest * NX);
    // the decision to leave is block-uniform (no thread may leave while others reach a barrier)
    if (__syncthreads_or(!mbar_wait_bounded(bar, 0))) {
        if (threadIdx.x == 0) {
            atomicExch(err, kErrBulkTimeout);
            mbar_wait_bounded(bar, 0);
        }
        return;
    }
    CT v[RX];
#pragma unroll
    for (int s = 0; s < RX; ++s) {
        const int i0 = t + T * slot_q<NX, RX, 0>(s);
        const int e = lr * NX + i0;
        const R g = __ldg(rb.g0 + i0) + rb.grest;
        const CT b = born_B_vals(M, pres, g, m0s[e], pres ? m1s[e] : (R)0, adj != 0);
        v[s] = cadd(cmul(b, xs[e]), ys[e]);
    }
    fft_run<NX, RX, -1, true>(v, xs + lr * NX, 1, t, tw, tc, RowSync<T>());
    constexpr int np = plan_npass(NX, RX);
    const long long fbase = fbase0 + (long long)lr * NX;
#pragma unroll
    for (int s = 0; s < RX; ++s) w[fbase + t + T * slot_q<NX, RX, np>(s)] = v[s];
}

// Born inverse rows with bulk-staged w (first barrier) and x + medium (second
// barrier, needed only by the update after the transform).
template <typename R, int NX, int RX>
__global__ void __launch_bounds__(BulkCfg<R, NX, RX>::THREADS, sizeof(R) == 4 ? 4 : 1)
k_rows_inv_bulk(Dims d, Medium<R> M, cplx<R>* __restrict__ x, cplx<R>* __restrict__ w,
                const cplx<R>* __restrict__ tw, int adj, R nu, double* __restrict__ partials, int* err)
{
    using CT = cplx<R>;
    using Cfg = BulkCfg<R, NX, RX>;
    constexpr int T = Cfg::T;
    constexpr int E = Cfg::ELEMS;
    constexpr int np = plan_npass(NX, RX);
    extern __shared__ __align__(128) unsigned char smraw[];
    CT* ws = reinterpret_cast<CT*>(smraw);
    CT* xs = ws + E;
    R* m0s = reinterpret_cast<R*>(xs + E);
    R* m1s = m0s + E;
    uint64_t* bar = reinterpret_cast<uint64_t*>(m1s + E);
    const int lr = threadIdx.x / T, t = threadIdx.x % T;
    const long long rows_per_comp = d.N / NX;
    const long long row0 = (long long)blockIdx.x * Cfg::ROWS;
    const int c = (int)(row0 / rows_per_comp);
    const long long rest0 = row0 % rows_per_comp;
    const long long vbase0 = rest0 * NX;
    const long long fbase0 = (long long)c * d.N + vbase0;
    const bool pres = (c == d.D);
    const R* m0g = (pres ? M.kp : (c == 0 ? M.rs[0] : (c == 1 ? M.rs[1] : M.rs[2]))) + vbase0;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t fb = E * sizeof(CT), mb = E * sizeof(R);
        mbar_expect_tx(bar, fb);
        bulk_g2s(ws, w + fbase0, fb, bar);
        mbar_expect_tx(bar + 1, fb + (pres ? 2 : 1) * mb);
        bulk_g2s(xs, x + fbase0, fb, bar + 1);
        bulk_g2s(m0s, m0g, mb, bar + 1);
        if (pres) bulk_g2s(m1s, M.et + vbase0, mb, bar + 1);
    }
    TwCache<NX, RX, CT> tc;
    tw_load<NX, RX, T>(tc, t, tw);
    const long long rest = rest0 + lr;
    const int i1 = (int)(rest % d.n1), i2 = (int)(rest / d.n1);
    const RowB<R> rb = row_B(M, d.D, c, i1, i2, rest * NX);
    // each decision to leave is block-uniform (no thread may leave while others reach a barrier)
    if (__syncthreads_or(!mbar_wait_bounded(bar, 0))) {
        if (threadIdx.x == 0) {
            atomicExch(err, kErrBulkTimeout);
            mbar_wait_bounded(bar, 0);
            mbar_wait_bounded(bar + 1, 0);
        }
        return;
    }
    CT v[RX];
#pragma unroll
    for (int s = 0; s < RX; ++s) v[s] = ws[lr * NX + t + T * slot_q<NX, RX, 0>(s)];
    fft_run<NX, RX, +1, true>(v, ws + lr * NX, 1, t, tw, tc, RowSync<T>());
    if (__syncthreads_or(!mbar_wait_bounded(bar + 1, 0))) {
        if (threadIdx.x == 0) {
            atomicExch(err, kErrBulkTimeout);
            mbar_wait_bounded(bar + 1, 0);
        }
        return;
    }
    R s0 = (R)0, s1 = (R)0;
    const long long fbase = fbase0 + (long long)lr * NX;
#pragma unroll
    for (int s = 0; s < RX; ++s) {
        const int i0 = t + T * slot_q<NX, RX, np>(s);
        const int e = lr * NX + i0;
        const R g = __ldg(rb.g0 + i0) + rb.grest;
        const CT b = born_B_vals(M, pres, g, m0s[e], pres ? m1s[e] : (R)0, adj != 0);
        const CT xv = xs[e];
        const CT del = cscale(cmul(b, csub(v[s], xv)), nu);
        const CT xn = cadd(xv, del);
        x[fbase + i0] = xn;
        s0 += cabs2(del);
        s1 += cabs2(xn);
    }
    block_sum2(s0, s1, partials + 2 * (long long)blockIdx.x);
}

// ------------------------------------- rows: update of one iteration + start of the next
// Between two Born iterations the x rows are read and written twice: the
// inverse row kernel of iteration k updates x (x <- x + nu B (IFFT_x(w) - x))
// and the forward row kernel of iteration k+1 reads the same x rows again to
// form FFT_x(B x + y).  Both work row by row, so one kernel does both for a
// block of rows: w (from the inverse strided-axis pass), x, the medium and y
// are staged by bulk copies on three barriers (w first, then x and the medium
// for the update, then y for the next forward transform), B is formed once per
// value, the updated x is stored and kept in registers, and the next
// iteration's w = FFT_x(B x + y) is written in place of the consumed w.  Per
// voxel this moves w, x, y and the medium in and x, w out, instead of also
// reading x and the medium a second time.  Norm partials as in k_rows_inv_bulk.
// VAR (measured variants): bit 0 twiddles read from the table instead of registers, bit 1 y staged into w's
// buffer once the inverse transform is done (two field buffers instead of three), bit 2 L2 hints on the
// copies (x, y and the medium read once: evict first; w: evict last); bits 0 and 1: four blocks an SM
template <typename R, int NX, int RX, int VAR = 0> struct FusedCfg {
    using Rc = RowCfg<R, NX, RX>;
    static constexpr bool NOTC = (VAR & 1) != 0;
    static constexpr bool YWS = (VAR & 2) != 0;
    static constexpr bool HINT = (VAR & 4) != 0;
    static constexpr int ROWS = Rc::ROWS;
    static constexpr int T = Rc::T;
    static constexpr int THREADS = Rc::THREADS;
    static constexpr int ELEMS = ROWS * NX;
    static constexpr int NF = YWS ? 2 : 3;  // field buffers: w (also the exchange and, with YWS, y), x[, y]
    // field buffers, medium m0, m1, three mbarriers
    static constexpr size_t SMEM = NF * (size_t)ELEMS * sizeof(cplx<R>) + 2 * (size_t)ELEMS * sizeof(R) + 32;
    static constexpr int MINB = sizeof(R) == 4 ? ((VAR & 3) == 3 ? 4 : 3) : 1;
    static constexpr bool OK = (Rc::SL == NX) && ((size_t)ELEMS * sizeof(R)) % 16 == 0;
};

template <typename R, int NX, int RX, int VAR = 0>
__global__ void __launch_bounds__(FusedCfg<R, NX, RX, VAR>::THREADS, FusedCfg<R, NX, RX, VAR>::MINB)
k_rows_inv_fwd_bulk(Dims d, Medium<R> M, cplx<R>* __restrict__ x, const cplx<R>* __restrict__ y,
                    cplx<R>* __restrict__ w, const cplx<R>* __restrict__ tw, int adj, R nu,
                    double* __restrict__ partials, int* err)
{
    using CT = cplx<R>;
    using Cfg = FusedCfg<R, NX, RX, VAR>;
    constexpr int T = Cfg::T;
    constexpr int E = Cfg::ELEMS;
    constexpr int np = plan_npass(NX, RX);
    extern __shared__ __align__(128) unsigned char smraw[];
    CT* ws = reinterpret_cast<CT*>(smraw);
    CT* xs = ws + E;
    CT* ys = Cfg::YWS ? ws : xs + E;
    R* m0s = reinterpret_cast<R*>(xs + (Cfg::NF - 1) * E);
    R* m1s = m0s + E;
    uint64_t* bar = reinterpret_cast<uint64_t*>(m1s + E);
    const int lr = threadIdx.x / T, t = threadIdx.x % T;
    const long long rows_per_comp = d.N / NX;
    const long long row0 = (long long)blockIdx.x * Cfg::ROWS;
    const int c = (int)(row0 / rows_per_comp);
    const long long rest0 = row0 % rows_per_comp;
    const long long vbase0 = rest0 * NX;
    const long long fbase0 = (long long)c * d.N + vbase0;
    const bool pres = (c == d.D);
    const R* m0g = (pres ? M.kp : (c == 0 ? M.rs[0] : (c == 1 ? M.rs[1] : M.rs[2]))) + vbase0;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_init(bar + 2, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t fb = E * sizeof(CT), mb = E * sizeof(R);
        mbar_expect_tx(bar, fb);
        mbar_expect_tx(bar + 1, fb + (pres ? 2 : 1) * mb);
        if constexpr (Cfg::HINT) {
            const uint64_t once = l2_policy_evict_first(), again = l2_policy_evict_last();
            bulk_g2s_hint(ws, w + fbase0, fb, bar, again);
            bulk_g2s_hint(xs, x + fbase0, fb, bar + 1, once);
            bulk_g2s_hint(m0s, m0g, mb, bar + 1, once);
            if (pres) bulk_g2s_hint(m1s, M.et + vbase0, mb, bar + 1, once);
            if constexpr (!Cfg::YWS) {
                mbar_expect_tx(bar + 2, fb);
                bulk_g2s_hint(ys, y + fbase0, fb, bar + 2, once);
            }
        } else {
            bulk_g2s(ws, w + fbase0, fb, bar);
            bulk_g2s(xs, x + fbase0, fb, bar + 1);
            bulk_g2s(m0s, m0g, mb, bar + 1);
            if (pres) bulk_g2s(m1s, M.et + vbase0, mb, bar + 1);
            if constexpr (!Cfg::YWS) {
                mbar_expect_tx(bar + 2, fb);
                bulk_g2s(ys, y + fbase0, fb, bar + 2);
            }
        }
    }
    TwCache<NX, RX, CT> tc;
    if constexpr (!Cfg::NOTC) tw_load<NX, RX, T>(tc, t, tw);
    const long long rest = rest0 + lr;
    const int i1 = (int)(rest % d.n1), i2 = (int)(rest / d.n1);
    const RowB<R> rb = row_B(M, d.D, c, i1, i2, rest * NX);
    // a timed-out wait records the error, lets the block's remaining copies land and leaves
    auto fail = [&](int from) {
        if (threadIdx.x == 0) {
            atomicExch(err, kErrBulkTimeout);
            for (int k = from; k < 3; ++k) mbar_wait_bounded(bar + k, 0);
        }
    };
    // every decision to leave is block-uniform (no thread may leave while others reach a barrier)
    if (__syncthreads_or(!mbar_wait_bounded(bar, 0))) { fail(0); return; }
    CT v[RX];
#pragma unroll
    for (int s = 0; s < RX; ++s) v[s] = ws[lr * NX + t + T * slot_q<NX, RX, 0>(s)];
    fft_run<NX, RX, +1, true, 0, !Cfg::NOTC>(v, ws + lr * NX, 1, t, tw, tc, RowSync<T>());
    // (the barrier below also ends every read of w's buffer by the inverse transform)
    if (__syncthreads_or(!mbar_wait_bounded(bar + 1, 0))) { fail(1); return; }
    if constexpr (Cfg::YWS) {
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();  // the generic-proxy reads of the buffer come before the copy's writes
            mbar_expect_tx(bar + 2, E * sizeof(CT));
            if constexpr (Cfg::HINT) bulk_g2s_hint(ys, y + fbase0, E * sizeof(CT), bar + 2, l2_policy_evict_first());
            else bulk_g2s(ys, y + fbase0, E * sizeof(CT), bar + 2);
        }
    }
    R s0 = (R)0, s1 = (R)0;
    const long long fbase = fbase0 + (long long)lr * NX;
#pragma unroll
    for (int s = 0; s < RX; ++s) {
        const int i0 = t + T * slot_q<NX, RX, np>(s);
        const int e = lr * NX + i0;
        const R g = __ldg(rb.g0 + i0) + rb.grest;
        const CT b = born_B_vals(M, pres, g, m0s[e], pres ? m1s[e] : (R)0, adj != 0);
        const CT xv = xs[e];
        const CT del = cscale(cmul(b, csub(v[s], xv)), nu);
        const CT xn = cadd(xv, del);
        x[fbase + i0] = xn;
        s0 += cabs2(del);
        s1 += cabs2(xn);
        v[s] = cmul(b, xn);  // B x of the next iteration
    }
    block_sum2(s0, s1, partials + 2 * (long long)blockIdx.x);
    if (__syncthreads_or(!mbar_wait_bounded(bar + 2, 0))) { fail(2); return; }
#pragma unroll
    for (int s = 0; s < RX; ++s) v[s] = cadd(v[s], ys[lr * NX + t + T * slot_q<NX, RX, np>(s)]);
    // same positions, entry order of the forward transform
    permute_slots<NX, RX, np, 0>(v);
    if constexpr (Cfg::YWS) __syncthreads();  // every thread has read its y values from w's buffer
    fft_run<NX, RX, -1, true, 0, !Cfg::NOTC>(v, ws + lr * NX, 1, t, tw, tc, RowSync<T>());
#pragma unroll
    for (int s = 0; s < RX; ++s) w[fbase + t + T * slot_q<NX, RX, np>(s)] = v[s];
}

// ------------------------------------------ tensor-copy helpers (3D tiles)
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y, int z)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// returns once the committed stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }


// ------------------------------------------------ last_symbol, tile-staged
// The k_last_symbol step for 3D fields, with the block's data staged in shared
// memory: the tile [C][NL][COLS] (COLS x-columns at one y, all z, all C
// components) arrives by one tensor copy per component, each on its own
// mbarrier.  The C forward transforms along z run one after the other out of
// the tile (each result written back in natural order), the per-wavenumber
// symbol updates the tile in place, the inverse transforms run the same way,
// and the tile leaves by tensor stores.  Only one component's RL values are in
// registers at a time.  tmap describes the field as {n0, n1, C*n2} 8-byte
// elements with box {COLS, 1, NL}; n0 % COLS == 0.
// grid: n1 * (n0 / COLS); block: (NL / RL) * COLS.
template <typename R, int NL, int RL, int COLS, int C> struct LastTileCfg {
    static constexpr int T = NL / RL;
    static constexpr int THREADS = T * COLS;
    static constexpr int TILE = NL * COLS;
    static constexpr uint32_t TILE_BYTES = TILE * sizeof(cplx<R>);
    static constexpr size_t SMEM = (size_t)C * TILE_BYTES + C * sizeof(uint64_t);
};

template <typename R, int NL, int RL, int COLS, int C>
__global__ void __launch_bounds__(LastTileCfg<R, NL, RL, COLS, C>::THREADS)
k_last_symbol_tile(const __grid_constant__ CUtensorMap tmap, Dims d, Symbol<R> Sy, const cplx<R>* __restrict__ tw,
                   int mode, int* err)
{
    using CT = cplx<R>;
    using Cfg = LastTileCfg<R, NL, RL, COLS, C>;
    constexpr int T = Cfg::T;
    constexpr int D = C - 1;
    constexpr int TILE = Cfg::TILE;
    constexpr int np = plan_npass(NL, RL);
    extern __shared__ __align__(128) unsigned char smraw[];
    CT* tile = reinterpret_cast<CT*>(smraw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + (size_t)C * Cfg::TILE_BYTES);
    const int col = threadIdx.x % COLS, t = threadIdx.x / COLS;
    const int xblocks = d.n0 / COLS;
    const int x0 = (blockIdx.x % xblocks) * COLS;
    const int i1 = blockIdx.x / xblocks;
    if (smem_u32(smraw) & 127u) {  // block-uniform; no copy has been issued
        if (threadIdx.x == 0) atomicExch(err, kErrTileAlign);
        return;
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < C; ++c) mbar_init(&bar[c], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            mbar_expect_tx(&bar[c], Cfg::TILE_BYTES);
            tma_load_3d(tile + c * TILE, &tmap, x0, i1, c * NL, &bar[c]);
        }
    }
    TwCache<NL, RL, CT> tc;
    tw_load<NL, RL, T>(tc, t, tw);
    // forward transforms along z, one component at a time
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const bool ok = mbar_wait_bounded(&bar[c], 0);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(err, kErrBulkTimeout);
                for (int k = c; k < C; ++k) mbar_wait_bounded(&bar[k], 0);
            }
            return;
        }
        CT* tcp = tile + c * TILE;
        CT v[RL];
#pragma unroll
        for (int s = 0; s < RL; ++s) v[s] = tcp[(t + T * slot_q<NL, RL, 0>(s)) * COLS + col];
        fft_run<NL, RL, -1>(v, tcp + col, COLS, t, tw, tc, BlockSync());
        __syncthreads();
#pragma unroll
        for (int s = 0; s < RL; ++s) tcp[(t + T * slot_q<NL, RL, np>(s)) * COLS + col] = v[s];
    }
    __syncthreads();
    // per-wavenumber symbol on all C components (each position read and written by one thread)
    {
        const int ix = x0 + col;
        CT tx[D];
        R k2c = Sy.k2[0][ix];
        tx[0] = Sy.kt[0][ix];
        if (D == 3) {
            tx[1] = Sy.kt[1][i1];
            k2c += Sy.k2[1][i1];
        }
#pragma unroll 2
        for (int s = 0; s < RL; ++s) {
            const int iz = t + T * s;
            tx[D - 1] = Sy.kt[D - 1][iz];
            const R k2 = k2c + Sy.k2[D - 1][iz];
            CT vv[C];
#pragma unroll
            for (int c = 0; c < C; ++c) vv[c] = tile[c * TILE + iz * COLS + col];
            apply_symbol<R, C>(Sy, mode, tx, k2, vv);
#pragma unroll
            for (int c = 0; c < C; ++c) tile[c * TILE + iz * COLS + col] = vv[c];
        }
    }
    // inverse transforms, one component at a time
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if (c == 0) __syncthreads();
        CT* tcp = tile + c * TILE;
        CT v[RL];
#pragma unroll
        for (int s = 0; s < RL; ++s) v[s] = tcp[(t + T * slot_q<NL, RL, 0>(s)) * COLS + col];
        fft_run<NL, RL, +1>(v, tcp + col, COLS, t, tw, tc, BlockSync());
        __syncthreads();
#pragma unroll
        for (int s = 0; s < RL; ++s) tcp[(t + T * slot_q<NL, RL, np>(s)) * COLS + col] = v[s];
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < C; ++c) tma_store_3d(&tmap, tile + c * TILE, x0, i1, c * NL);
        bulk_commit();
        bulk_wait_read_all();
    }
}

// --------------------------------------------- axis_fft, persistent and pipelined
// The k_axis_fft transform with its column tiles staged by tensor copies: a
// persistent CTA walks the tiles (blockIdx.x, + gridDim.x, ...) with two
// shared-memory stages, so the copy of the next tile lands while the current
// one is transformed.  A tile [NA][COLS] (all y of COLS x-columns at one
// (component, z)) is one box {COLS, NA, 1} of tmap, which describes the field
// as {n0, n1, C*n2} 8-byte elements; n0 % COLS == 0.  The transform's exchanges
// run in the tile's own stage; results go to w with plain stores (each tile is
// read and written by one CTA, tiles are disjoint).
template <typename R, int NA, int COLS> struct AxisPipeCfg {
    static constexpr uint32_t TILE_BYTES = (uint32_t)NA * COLS * sizeof(cplx<R>);
    static constexpr size_t SMEM = 2 * (size_t)TILE_BYTES + 2 * sizeof(uint64_t);
};

template <typename R, int NA, int RA, int COLS, int S>
__global__ void __launch_bounds__(AxisCfg<NA, RA, COLS>::THREADS, 3)
k_axis_fft_pipe(const __grid_constant__ CUtensorMap tmap, Dims d, cplx<R>* __restrict__ w,
                const cplx<R>* __restrict__ tw, int* err)
{
    using CT = cplx<R>;
    using Cfg = AxisPipeCfg<R, NA, COLS>;
    constexpr int T = NA / RA;
    constexpr int np = plan_npass(NA, RA);
    extern __shared__ __align__(128) unsigned char smraw[];
    CT* stage0 = reinterpret_cast<CT*>(smraw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + 2 * (size_t)Cfg::TILE_BYTES);
    const int col = threadIdx.x % COLS, t = threadIdx.x / COLS;
    const int xblocks = d.n0 / COLS;
    const long long ntiles = (long long)(d.D + 1) * d.n2 * xblocks;
    if (smem_u32(smraw) & 127u) {  // block-uniform; no copy issued
        if (threadIdx.x == 0) atomicExch(err, kErrTileAlign);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    // thread 0 issues the copy of tile `tile` into stage `st`
    auto issue = [&](long long tile, int st) {
        const int xb = (int)(tile % xblocks);
        const int zc = (int)(tile / xblocks);  // c * n2 + i2
        mbar_expect_tx(&bar[st], Cfg::TILE_BYTES);
        tma_load_3d(stage0 + (size_t)st * NA * COLS, &tmap, xb * COLS, 0, zc, &bar[st]);
    };
    if (threadIdx.x == 0) {
        if ((long long)blockIdx.x < ntiles) issue(blockIdx.x, 0);
        if ((long long)blockIdx.x + gridDim.x < ntiles) issue((long long)blockIdx.x + gridDim.x, 1);
    }
    TwCache<NA, RA, CT> tc;
    tw_load<NA, RA, T>(tc, t, tw);
    uint32_t phases = 0u;  // bit st: parity of stage st's next completion
    int st = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, st ^= 1) {
        const uint32_t ph = (phases >> st) & 1u;
        const bool ok = mbar_wait_bounded(&bar[st], ph);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(err, kErrBulkTimeout);
                // let the copies still in flight land before the block leaves
                mbar_wait_bounded(&bar[st], ph);
                if (tile + gridDim.x < ntiles) mbar_wait_bounded(&bar[st ^ 1], (phases >> (st ^ 1)) & 1u);
            }
            return;
        }
        phases ^= 1u << st;
        CT* sm = stage0 + (size_t)st * NA * COLS;
        CT v[RA];
#pragma unroll
        for (int s = 0; s < RA; ++s) v[s] = sm[(t + T * slot_q<NA, RA, 0>(s)) * COLS + col];
        fft_run<NA, RA, S>(v, sm + col, COLS, t, tw, tc, BlockSync());
        const int xb = (int)(tile % xblocks);
        const long long zc = tile / xblocks;
        const long long base = zc * (long long)d.n0 * d.n1 + xb * COLS + col;
#pragma unroll
        for (int s = 0; s < RA; ++s) w[base + (long long)(t + T * slot_q<NA, RA, np>(s)) * d.n0] = v[s];
        fence_proxy_async_smem();  // this thread's exchange writes to the stage come before the next copy into it
        __syncthreads();           // every thread is done with this stage (inputs and exchanges)
        if (threadIdx.x == 0 && tile + 2LL * gridDim.x < ntiles) issue(tile + 2LL * gridDim.x, st);
    }
}

}  // namespace cbs
