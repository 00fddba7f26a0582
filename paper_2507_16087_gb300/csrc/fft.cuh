// fft.cuh -- register/shared-memory Stockham FFT engine for sm_103a.
//
// A length-N transform is done by T = N/R threads, each holding R complex
// values in registers.  The transform is a sequence of radix-r passes (r in
// {2,3,4,8,16}, r | R) in Stockham autosort order: pass p with sub-transform size
// Ns takes, for butterfly j, the inputs j + k N/r, multiplies input k by
// w^{(j mod Ns) k N/(Ns r)} (w = exp(-2 pi i / N)), runs an r-point DFT and
// writes output k to (j div Ns) Ns r + (j mod Ns) + k Ns.  Between passes the
// values are exchanged through shared memory.  Thread `tid` owns positions
// tid + T q, q = 0..R-1, both on entry and on exit, so loads and stores along
// a contiguous axis are coalesced across threads.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cbs {

// ----------------------------------------------------------------- complex
template <typename R> struct ctype;
template <> struct ctype<float> { using T = float2; };
template <> struct ctype<double> { using T = double2; };
template <typename R> using cplx = typename ctype<R>::T;

template <typename CT> struct real_of;
template <> struct real_of<float2> { using T = float; };
template <> struct real_of<double2> { using T = double; };

template <typename CT, typename R> __host__ __device__ __forceinline__ CT mk(R a, R b) { CT c; c.x = a; c.y = b; return c; }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// multiply by s*i  (s = +1 or -1)
template <int S> __host__ __device__ __forceinline__ float2 mul_si(float2 a) { return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }
template <int S> __host__ __device__ __forceinline__ double2 mul_si(double2 a) { return S > 0 ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x); }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// --------------------------------------------------------------- r-point DFTs
// X_q = sum_m x_m exp(S 2 pi i m q / r), S = -1 forward, +1 inverse.
template <int S, typename CT> __host__ __device__ __forceinline__ void dft2(CT* v)
{
    CT a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <int S, typename CT> __host__ __device__ __forceinline__ void dft4(CT* v)
{
    CT s0 = cadd(v[0], v[2]), d0 = csub(v[0], v[2]);
    CT s1 = cadd(v[1], v[3]), d1 = mul_si<S>(csub(v[1], v[3]));
    v[0] = cadd(s0, s1);
    v[2] = csub(s0, s1);
    v[1] = cadd(d0, d1);
    v[3] = csub(d0, d1);
}

template <int S, typename CT> __host__ __device__ __forceinline__ void dft3(CT* v)
{
    using R = typename real_of<CT>::T;
    const R h = (R)0.86602540378443864676372317075294;  // sin(2 pi / 3)
    CT t = cadd(v[1], v[2]);
    CT u = csub(v[1], v[2]);
    CT a = v[0];
    CT m = mk<CT, R>(a.x - (R)0.5 * t.x, a.y - (R)0.5 * t.y);
    CT iu = mul_si<S>(cscale(u, h));
    v[0] = cadd(a, t);
    v[1] = cadd(m, iu);
    v[2] = csub(m, iu);
}

// 8 = 2 x 4: even/odd 4-point DFTs combined with w8^q = exp(S 2 pi i q / 8)
template <int S, typename CT> __host__ __device__ __forceinline__ void dft8(CT* v)
{
    using R = typename real_of<CT>::T;
    const R c = (R)0.70710678118654752440084436210485;
    CT e[4] = {v[0], v[2], v[4], v[6]};
    CT o[4] = {v[1], v[3], v[5], v[7]};
    dft4<S>(e);
    dft4<S>(o);
    // w8^1 = c (1 + S i), w8^2 = S i, w8^3 = c (-1 + S i)
    CT o1 = mk<CT, R>(c * (o[1].x - (R)S * o[1].y), c * (o[1].y + (R)S * o[1].x));
    CT o2 = mul_si<S>(o[2]);
    CT o3 = mk<CT, R>(c * (-o[3].x - (R)S * o[3].y), c * (-o[3].y + (R)S * o[3].x));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2; inner 4-point DFTs over n1, twiddles
// w16^{n2 k1}, outer 4-point DFTs over n2 (w16 = exp(S 2 pi i / 16))
template <int S, typename CT> __host__ __device__ __forceinline__ void dft16(CT* v)
{
    using R = typename real_of<CT>::T;
    const R c1 = (R)0.92387953251128675612818318939679;  // cos(pi/8)
    const R s1 = (R)0.38268343236508977172845998403040;  // sin(pi/8)
    const R h = (R)0.70710678118654752440084436210485;
    CT a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        CT t[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
        dft4<S>(t);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = t[k1];
    }
    const CT w1 = mk<CT, R>(c1, (R)S * s1);
    const CT w2 = mk<CT, R>(h, (R)S * h);
    const CT w3 = mk<CT, R>(s1, (R)S * c1);
    const CT w6 = mk<CT, R>(-h, (R)S * h);
    const CT w9 = mk<CT, R>(-c1, -(R)S * s1);
    a[1][1] = cmul(a[1][1], w1);
    a[1][2] = cmul(a[1][2], w2);
    a[1][3] = cmul(a[1][3], w3);
    a[2][1] = cmul(a[2][1], w2);
    a[2][2] = mul_si<S>(a[2][2]);
    a[2][3] = cmul(a[2][3], w6);
    a[3][1] = cmul(a[3][1], w3);
    a[3][2] = cmul(a[3][2], w6);
    a[3][3] = cmul(a[3][3], w9);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        CT t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
        dft4<S>(t);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
}

template <int r, int S, typename CT> __host__ __device__ __forceinline__ void dft(CT* v)
{
    if constexpr (r == 2) dft2<S>(v);
    else if constexpr (r == 3) dft3<S>(v);
    else if constexpr (r == 4) dft4<S>(v);
    else if constexpr (r == 8) dft8<S>(v);
    else if constexpr (r == 16) dft16<S>(v);
}

// ------------------------------------------------------------------- plans
// Radix of the step that reduces `rem` (the part of N not yet transformed).
__host__ __device__ constexpr int plan_step(int rem, int R)
{
    return (rem % 3 == 0 && R % 3 == 0) ? 3
         : (rem % 16 == 0 && R % 16 == 0) ? 16
         : (rem % 8 == 0 && R % 8 == 0) ? 8
         : (rem % 4 == 0 && R % 4 == 0) ? 4
         : (rem % 2 == 0 && R % 2 == 0) ? 2 : 0;
}
__host__ __device__ constexpr int plan_radix(int N, int R, int p)
{
    int rem = N;
    for (int i = 0; i < p; ++i) rem /= plan_step(rem, R);
    return plan_step(rem, R);
}
__host__ __device__ constexpr int plan_npass(int N, int R)
{
    int rem = N, n = 0;
    while (rem > 1) {
        int r = plan_step(rem, R);
        if (r == 0) return -1;
        rem /= r;
        ++n;
    }
    return n;
}
__host__ __device__ constexpr int plan_ns(int N, int R, int p)
{
    int ns = 1;
    for (int i = 0; i < p; ++i) ns *= plan_radix(N, R, i);
    return ns;
}

// Position index q (tid + T q) held in register slot s on entry to pass p (or,
// with p = npass, on exit of the last pass): slot s = m r + k holds butterfly
// m's input/output k, i.e. position j + k N/r with j = tid + T m.
template <int N, int R, int P> __host__ __device__ __forceinline__ constexpr int slot_q(int s)
{
    constexpr int np = plan_npass(N, R);
    constexpr int r = (P < np) ? plan_radix(N, R, P) : plan_radix(N, R, np - 1);
    return (s % r) * (R / r) + s / r;
}
// inverse of slot_q: the slot that holds position index q
template <int N, int R, int P> __host__ __device__ __forceinline__ constexpr int q_slot(int q)
{
    constexpr int np = plan_npass(N, R);
    constexpr int r = (P < np) ? plan_radix(N, R, P) : plan_radix(N, R, np - 1);
    return (q % (R / r)) * r + q / (R / r);
}
// Reorder registers from the slot order of pass PA to that of pass PB (the
// thread owns the same positions in both; this is a compile-time permutation).
template <int N, int R, int PA, int PB, typename CT>
__device__ __forceinline__ void permute_slots(CT (&v)[R])
{
    CT tmp[R];
#pragma unroll
    for (int s = 0; s < R; ++s) tmp[s] = v[s];
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = tmp[q_slot<N, R, PA>(slot_q<N, R, PB>(s))];
}

// Twiddles a thread needs over all passes: pass P with NS > 1 uses, for its
// butterfly m and input k = 1..r-1, w^{(j mod NS) k N/(NS r)}.  When there are
// few of them they are loaded into registers once per kernel (TwCache), else
// read from the table at each pass.
__host__ __device__ constexpr int tw_count_before(int N, int R, int P)
{
    int c = 0;
    for (int p = 0; p < P; ++p) {
        const int r = plan_radix(N, R, p);
        if (plan_ns(N, R, p) > 1) c += (R / r) * (r - 1);
    }
    return c;
}
__host__ __device__ constexpr int tw_count(int N, int R) { return tw_count_before(N, R, plan_npass(N, R)); }
template <int N, int R> struct TwPolicy {
    static constexpr int count = tw_count(N, R);
    static constexpr bool cached = count > 0 && count <= 16;
    static constexpr int slots = cached ? count : 1;
};

template <int N, int R, typename CT> struct TwCache {
    CT w[TwPolicy<N, R>::slots];
};

template <int N, int R, int T, int P = 0, typename CT>
__device__ __forceinline__ void tw_load(TwCache<N, R, CT>& tc, int tid, const CT* __restrict__ tw)
{
    if constexpr (TwPolicy<N, R>::cached && P < plan_npass(N, R)) {
        constexpr int r = plan_radix(N, R, P);
        constexpr int NS = plan_ns(N, R, P);
        if constexpr (NS > 1) {
            constexpr int off = tw_count_before(N, R, P);
#pragma unroll
            for (int m = 0; m < R / r; ++m) {
                const int jj = (tid + T * m) % NS;
#pragma unroll
                for (int k = 1; k < r; ++k) tc.w[off + m * (r - 1) + k - 1] = __ldg(&tw[jj * k * (N / (NS * r))]);
            }
        }
        tw_load<N, R, T, P + 1>(tc, tid, tw);
    }
}

// twiddle table: tw[m] = exp(-2 pi i m / N), m < N
template <int N, int R, int T, int P, int S, bool USE_TC = true, typename CT>
__device__ __forceinline__ void pass_compute(CT (&v)[R], int tid, const CT* __restrict__ tw, const TwCache<N, R, CT>& tc)
{
    constexpr int r = plan_radix(N, R, P);
    constexpr int NS = plan_ns(N, R, P);
#pragma unroll
    for (int m = 0; m < R / r; ++m) {
        if constexpr (NS > 1) {
            const int j = tid + T * m;
            const int jj = j % NS;
#pragma unroll
            for (int k = 1; k < r; ++k) {
                CT w;
                if constexpr (USE_TC && TwPolicy<N, R>::cached) w = tc.w[tw_count_before(N, R, P) + m * (r - 1) + k - 1];
                else w = __ldg(&tw[jj * k * (N / (NS * r))]);
                v[m * r + k] = (S < 0) ? cmul(v[m * r + k], w) : cmulc(v[m * r + k], w);
            }
        }
        dft<r, S>(&v[m * r]);
    }
}

// Shared-memory address of element e.  Column tiles (PAD = false): e * ss.
// A row stored contiguously (PAD = true): a swizzle that keeps the Stockham
// writes (stride r) and reads (stride N/r) of a 16-lane phase on distinct
// banks: XOR of bits 3..6 into bits 0..3 when N >= 128, else a skew.
template <int N> __host__ __device__ constexpr int row_swizzle(int e)
{
    return (N >= 128 && N % 16 == 0) ? (e ^ ((e >> 3) & 15)) : (N == 64 ? e + (e >> 3) + (e >> 6) : e + (e >> 4));
}
template <int N, bool PAD> __device__ __forceinline__ int sm_addr(int e, int ss) { return PAD ? row_swizzle<N>(e) : e * ss; }
template <int N, bool PAD> __host__ __device__ constexpr int sm_len()
{
    return PAD ? ((N >= 128 && N % 16 == 0) ? N : row_swizzle<N>(N - 1) + 1) : N;
}

template <int N, int R, int T, int P, bool PAD, typename CT, typename Sync>
__device__ __forceinline__ void pass_exchange(CT (&v)[R], CT* sm, int ss, int tid, Sync sync)
{
    constexpr int r = plan_radix(N, R, P);
    constexpr int NS = plan_ns(N, R, P);
    constexpr int rn = plan_radix(N, R, P + 1);
    sync();
#pragma unroll
    for (int m = 0; m < R / r; ++m) {
        const int j = tid + T * m;
        const int idx = (j / NS) * NS * r + (j % NS);
#pragma unroll
        for (int k = 0; k < r; ++k) sm[sm_addr<N, PAD>(idx + k * NS, ss)] = v[m * r + k];
    }
    sync();
#pragma unroll
    for (int m = 0; m < R / rn; ++m) {
        const int j = tid + T * m;
#pragma unroll
        for (int k = 0; k < rn; ++k) v[m * rn + k] = sm[sm_addr<N, PAD>(j + k * (N / rn), ss)];
    }
}

// Full transform.  On entry v[s] holds position tid + T*slot_q<N,R,0>(s); on
// exit v[s] holds position tid + T*slot_q<N,R,npass>(s).
// USE_TC = false reads every twiddle from the table (for kernels with no registers to spare).
template <int N, int R, int S, bool PAD = false, int P = 0, bool USE_TC = true, typename CT, typename Sync>
__device__ __forceinline__ void fft_run(CT (&v)[R], CT* sm, int ss, int tid, const CT* __restrict__ tw,
                                        const TwCache<N, R, CT>& tc, Sync sync)
{
    constexpr int T = N / R;
    constexpr int np = plan_npass(N, R);
    static_assert(np > 0, "unsupported FFT size / register split");
    pass_compute<N, R, T, P, S, USE_TC>(v, tid, tw, tc);
    if constexpr (P + 1 < np) {
        pass_exchange<N, R, T, P, PAD>(v, sm, ss, tid, sync);
        fft_run<N, R, S, PAD, P + 1, USE_TC>(v, sm, ss, tid, tw, tc, sync);
    }
}

// One pass of C transforms that share the thread mapping: each twiddle is read
// from the table once and applied to all C components.
template <int N, int R, int T, int P, int S, int C, typename CT>
__device__ __forceinline__ void pass_compute_multi(CT (&v)[C][R], int tid, const CT* __restrict__ tw)
{
    constexpr int r = plan_radix(N, R, P);
    constexpr int NS = plan_ns(N, R, P);
#pragma unroll
    for (int m = 0; m < R / r; ++m) {
        if constexpr (NS > 1) {
            const int jj = (tid + T * m) % NS;
#pragma unroll
            for (int k = 1; k < r; ++k) {
                const CT w = __ldg(&tw[jj * k * (N / (NS * r))]);
#pragma unroll
                for (int c = 0; c < C; ++c)
                    v[c][m * r + k] = (S < 0) ? cmul(v[c][m * r + k], w) : cmulc(v[c][m * r + k], w);
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) dft<r, S>(&v[c][m * r]);
    }
}

// Same for C independent transforms that share the thread mapping (used to
// keep all components of a pencil in registers at once).
// (twiddles read from the table: with C transforms in registers there is no
// room to cache them; SHTW reads each one once for all C transforms)
template <int N, int R, int C, int S, int P = 0, bool SHTW = false, typename CT, typename Sync>
__device__ __forceinline__ void fft_run_multi(CT (&v)[C][R], CT* sm, int ss, int cstride, int tid,
                                              const CT* __restrict__ tw, Sync sync)
{
    constexpr int T = N / R;
    constexpr int np = plan_npass(N, R);
    static_assert(np > 0, "unsupported FFT size / register split");
    const TwCache<N, R, CT> none{};
    if constexpr (SHTW) {
        pass_compute_multi<N, R, T, P, S, C>(v, tid, tw);
    } else {
#pragma unroll
        for (int c = 0; c < C; ++c) pass_compute<N, R, T, P, S, false>(v[c], tid, tw, none);
    }
    if constexpr (P + 1 < np) {
        constexpr int r = plan_radix(N, R, P);
        constexpr int NS = plan_ns(N, R, P);
        constexpr int rn = plan_radix(N, R, P + 1);
        sync();
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int m = 0; m < R / r; ++m) {
                const int j = tid + T * m;
                const int idx = (j / NS) * NS * r + (j % NS);
#pragma unroll
                for (int k = 0; k < r; ++k) sm[c * cstride + (idx + k * NS) * ss] = v[c][m * r + k];
            }
        sync();
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int m = 0; m < R / rn; ++m) {
                const int j = tid + T * m;
#pragma unroll
                for (int k = 0; k < rn; ++k) v[c][m * rn + k] = sm[c * cstride + (j + k * (N / rn)) * ss];
            }
        fft_run_multi<N, R, C, S, P + 1, SHTW>(v, sm, ss, cstride, tid, tw, sync);
    }
}

}  // namespace cbs
