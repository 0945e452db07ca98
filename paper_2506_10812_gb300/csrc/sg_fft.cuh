// Register-resident Stockham FFT for one CTA (float or double).
//
// A length-L transform (L = 16 T, L a power of two >= 16) is held by T
// threads, 16 elements each, in the "strided" layout: thread t holds
// x[t + T e] in register v[e].  Each Stockham pass of radix R reads exactly
// those registers (butterfly j = t + T q combines x[j + r L/R]), so a pass
// is: twiddle, radix-R DFT in registers, and (except after the last pass)
// one scatter/gather through a padded shared-memory buffer.  Passes are
// radix 16 with a final radix 2, 4 or 8; output is in natural order in the
// same strided layout, so a forward transform, a pointwise product and an
// inverse transform need no reordering at all.
//
// Twiddles come from a table tw[m] = exp(-2 pi i m / M) (computed in FP64 on
// the host); a length-L transform uses tw[m * (M / L)].
#pragma once

#include <cuda_runtime.h>

namespace sg {

template <typename R> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename R> using cplx = typename cplx_of<R>::type;

template <typename T> __device__ __forceinline__ T mkc(decltype(T::x) a, decltype(T::x) b) { T c; c.x = a; c.y = b; return c; }
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return mkc<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return mkc<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ T cneg(T a) { return mkc<T>(-a.x, -a.y); }
template <typename T> __device__ __forceinline__ T cconj(T a) { return mkc<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ T cmul_i(T a) { return mkc<T>(-a.y, a.x); }   // i a
template <typename T> __device__ __forceinline__ T cmul_mi(T a) { return mkc<T>(a.y, -a.x); }  // -i a
template <typename T> __device__ __forceinline__ T cscale(T a, decltype(T::x) s) { return mkc<T>(a.x * s, a.y * s); }
// a * b
template <typename T> __device__ __forceinline__ T cmul(T a, T b)
{
    return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ T cmulc(T a, T b)
{
    return mkc<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// acc + a * b
template <typename T> __device__ __forceinline__ T cfma(T a, T b, T acc)
{
    acc.x += a.x * b.x - a.y * b.y;
    acc.y += a.x * b.y + a.y * b.x;
    return acc;
}
template <bool FWD, typename T> __device__ __forceinline__ T twmul(T a, T w)
{
    return FWD ? cmul(a, w) : cmulc(a, w);
}

// cos(pi/8), sin(pi/8), cos(pi/4)
#define SG_C16 0.92387953251128675613
#define SG_S16 0.38268343236508977173
#define SG_C8 0.70710678118654752440

// a * exp(-+ 2 pi i P / 16)  (minus sign for the forward transform)
template <bool FWD, int P, typename T> __device__ __forceinline__ T w16(T a)
{
    using R = decltype(T::x);
    constexpr int p = P & 15;
    if constexpr (p == 0) {
        return a;
    } else if constexpr (p == 4) {
        return FWD ? cmul_mi(a) : cmul_i(a);
    } else if constexpr (p == 8) {
        return cneg(a);
    } else if constexpr (p == 12) {
        return FWD ? cmul_i(a) : cmul_mi(a);
    } else {
        constexpr double cs[16] = {1.0, SG_C16, SG_C8, SG_S16, 0.0, -SG_S16, -SG_C8, -SG_C16,
                                   -1.0, -SG_C16, -SG_C8, -SG_S16, 0.0, SG_S16, SG_C8, SG_C16};
        constexpr double sn[16] = {0.0, SG_S16, SG_C8, SG_C16, 1.0, SG_C16, SG_C8, SG_S16,
                                   0.0, -SG_S16, -SG_C8, -SG_C16, -1.0, -SG_C16, -SG_C8, -SG_S16};
        const R c = (R)cs[p];
        const R s = FWD ? (R)sn[p] : (R)(-sn[p]);
        // (a.x + i a.y)(c - i s)
        return mkc<T>(a.x * c + a.y * s, a.y * c - a.x * s);
    }
}

template <bool FWD, typename T> __device__ __forceinline__ void dft2(T &a0, T &a1)
{
    T t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <bool FWD, typename T> __device__ __forceinline__ void dft4(T &a0, T &a1, T &a2, T &a3)
{
    T t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = csub(a1, a3);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    if (FWD) {
        a1 = cadd(t1, cmul_mi(t3));
        a3 = cadd(t1, cmul_i(t3));
    } else {
        a1 = cadd(t1, cmul_i(t3));
        a3 = cadd(t1, cmul_mi(t3));
    }
}

// In-place 8-point DFT on a[OFF + S*n], n = 0..7 (natural order in and out).
template <bool FWD, int OFF, int S, typename T> __device__ __forceinline__ void dft8(T (&a)[16])
{
    // n = 2 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle W8^{n2 k1}, DFT2 over n2
    T b[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) b[n] = a[OFF + S * n];
    dft4<FWD>(b[0], b[2], b[4], b[6]);
    dft4<FWD>(b[1], b[3], b[5], b[7]);
    // b[2 k1 + n2] now holds B[n2][k1]
    b[3] = w16<FWD, 2>(b[3]);
    b[5] = w16<FWD, 4>(b[5]);
    b[7] = w16<FWD, 6>(b[7]);
    dft2<FWD>(b[0], b[1]);
    dft2<FWD>(b[2], b[3]);
    dft2<FWD>(b[4], b[5]);
    dft2<FWD>(b[6], b[7]);
    // X[k1 + 4 k2] = b[2 k1 + k2]
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        a[OFF + S * k1] = b[2 * k1];
        a[OFF + S * (k1 + 4)] = b[2 * k1 + 1];
    }
}

// In-place 16-point DFT on a[0..15] (natural order in and out).
template <bool FWD, typename T> __device__ __forceinline__ void dft16(T (&a)[16])
{
    // n = 4 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle W16^{n2 k1}, DFT4 over n2
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<FWD>(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
    // a[4 k1 + n2] = B[n2][k1]
    a[5] = w16<FWD, 1>(a[5]);
    a[6] = w16<FWD, 2>(a[6]);
    a[7] = w16<FWD, 3>(a[7]);
    a[9] = w16<FWD, 2>(a[9]);
    a[10] = w16<FWD, 4>(a[10]);
    a[11] = w16<FWD, 6>(a[11]);
    a[13] = w16<FWD, 3>(a[13]);
    a[14] = w16<FWD, 6>(a[14]);
    a[15] = w16<FWD, 9>(a[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<FWD>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
    // X[k1 + 4 k2] = a[4 k1 + k2]: transpose the 4x4 index
    T b[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) b[i] = a[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = b[4 * k1 + k2];
}

// Padded shared-memory index: one extra slot every 16 elements makes the
// Stockham scatter (stride 16) and the strided gather conflict-free.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int L) { return L + (L >> 4) + 1; }

// Scatter after a radix-16 pass with stride Ns, gather back the strided layout.
template <typename T>
__device__ __forceinline__ void exchange16(T (&v)[16], int t, int T_, int Ns, T *xb)
{
    const int k = t & (Ns - 1);
    const int base = (t - k) * 16 + k;     // (t / Ns) Ns 16 + k
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) xb[pidx(base + r * Ns)] = v[r];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = xb[pidx(t + T_ * e)];
}

// Final Stockham pass of radix RL in {2, 4, 8} (Q = 16 / RL butterflies per
// thread; butterfly q combines registers q + r Q).  Lands in-register.
template <bool FWD, int RL, typename T>
__device__ __forceinline__ void final_pass(T (&v)[16], int t, int T_, int Ns,
                                           const T *__restrict__ tw, int twstride)
{
    constexpr int Q = 16 / RL;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k = (t + T_ * q) & (Ns - 1);
#pragma unroll
        for (int r = 1; r < RL; ++r)
            v[q + r * Q] = twmul<FWD>(v[q + r * Q], __ldg(&tw[(r * k) * twstride]));
    }
    if constexpr (RL == 2) {
#pragma unroll
        for (int q = 0; q < Q; ++q) dft2<FWD>(v[q], v[q + Q]);
    } else if constexpr (RL == 4) {
#pragma unroll
        for (int q = 0; q < Q; ++q) dft4<FWD>(v[q], v[q + Q], v[q + 2 * Q], v[q + 3 * Q]);
    } else {
        dft8<FWD, 0, 2>(v);
        dft8<FWD, 1, 2>(v);
    }
}

// Full length-L transform (L = 16 T_, power of two) of the strided register
// layout v[e] = x[t + T_ e]; result X[t + T_ e] in v[e].  Forward: X[k] =
// sum x[n] exp(-2 pi i n k / L); inverse: the same with +i (unnormalised).
// xb: this transform's shared buffer of padded_len(L) elements.  Every thread
// of the CTA must call this together (it contains __syncthreads).
// tw: twiddle table exp(-2 pi i m / M) with M = L * twstride.
template <bool FWD, typename T>
__device__ __forceinline__ void fft_reg(T (&v)[16], int L, int T_, int t, T *xb,
                                        const T *__restrict__ tw, int twstride)
{
    dft16<FWD>(v);                              // pass Ns = 1: no twiddles
    if (L == 16) return;
    int Ns = 16;
    exchange16(v, t, T_, 1, xb);
    while (Ns * 16 <= L) {
        const int k = t & (Ns - 1);
        const int step = (L / (Ns * 16)) * k * twstride;
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = twmul<FWD>(v[r], __ldg(&tw[r * step]));
        dft16<FWD>(v);
        if (Ns * 16 == L) return;
        exchange16(v, t, T_, Ns, xb);
        Ns *= 16;
    }
    const int RL = L / Ns;
    if (RL == 8) final_pass<FWD, 8>(v, t, T_, Ns, tw, twstride);
    else if (RL == 4) final_pass<FWD, 4>(v, t, T_, Ns, tw, twstride);
    else final_pass<FWD, 2>(v, t, T_, Ns, tw, twstride);
}

}  // namespace sg
