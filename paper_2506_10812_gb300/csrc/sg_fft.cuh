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
// Twiddles come from a per-pass table (computed in FP64 on the host): the
// pass with stride Ns and radix R reads W_{Ns R}^{r k} = exp(-2 pi i r k / (Ns R))
// at (r - 1) Ns + k, so the threads of a warp (consecutive k) read
// consecutive entries; the passes' segments follow one another (Ns = 16,
// 256, ... for the radix-16 passes, then the final pass).
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

// ---- packed FP32 pairs (Blackwell add/sub/fma.f32x2): one instruction per
// complex add or subtract.  Results are bit-identical to the scalar forms
// (each lane is one correctly rounded operation; x * (+-1) is exact).
__device__ __forceinline__ float2 padd(float2 a, float2 b)
{
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " add.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 psub(float2 a, float2 b)
{
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
// c + a * (sx, sy) with sx, sy = +-1
template <int SX, int SY>
__device__ __forceinline__ float2 pfma_sign(float2 a, float2 c)
{
    float2 d;
    asm("{\n .reg .b64 ra, rs, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rs, {%6, %7};\n"
        " mov.b64 rc, {%4, %5};\n fma.rn.f32x2 rd, ra, rs, rc;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(c.x), "f"(c.y), "f"((float)SX), "f"((float)SY));
    return d;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return padd(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return psub(a, b); }

template <bool FWD, typename T> __device__ __forceinline__ void dft2(T &a0, T &a1)
{
    T t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

// Packed radix 4: u = swap(a1 - a3) in scalar form, the +-i rotations as
// sign-vector FMAs (9 instructions instead of 16).
template <bool FWD> __device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 t0 = padd(a0, a2), t1 = psub(a0, a2), t2 = padd(a1, a3);
    const float2 u = make_float2(a1.y - a3.y, a1.x - a3.x);
    a0 = padd(t0, t2);
    a2 = psub(t0, t2);
    if (FWD) {   // t1 - i t3 = t1 + (u.x, -u.y),  t1 + i t3 = t1 + (-u.x, u.y)
        a1 = pfma_sign<1, -1>(u, t1);
        a3 = pfma_sign<-1, 1>(u, t1);
    } else {
        a1 = pfma_sign<-1, 1>(u, t1);
        a3 = pfma_sign<1, -1>(u, t1);
    }
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

// Second half of the 16-point DFT below (after its first radix-4 stage).
template <bool FWD, typename T> __device__ __forceinline__ void dft16_tail(T (&a)[16])
{
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

// In-place 16-point DFT on a[0..15] (natural order in and out).
template <bool FWD, typename T> __device__ __forceinline__ void dft16(T (&a)[16])
{
    // n = 4 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle W16^{n2 k1}, DFT4 over n2
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<FWD>(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
    dft16_tail<FWD>(a);
}

// The same DFT when a[8..15] are zero (the radially zero-padded half of a
// forward column transform): each first-stage radix 4 has two inputs,
// X = x0 + x1, x0 -+ i x1, x0 - x1, x0 +- i x1 (4 packed instructions
// instead of 9).  Zero operands cannot be folded by the compiler (x + 0 is not
// x for x = -0), so the pruning is explicit.
template <bool FWD> __device__ __forceinline__ void dft16_half(float2 (&a)[16])
{
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        const float2 x0 = a[n2], x1 = a[4 + n2];
        const float2 u = make_float2(x1.y, x1.x);
        a[n2] = padd(x0, x1);
        a[8 + n2] = psub(x0, x1);
        if (FWD) {   // x0 - i x1 = x0 + (u.x, -u.y),  x0 + i x1 = x0 + (-u.x, u.y)
            a[4 + n2] = pfma_sign<1, -1>(u, x0);
            a[12 + n2] = pfma_sign<-1, 1>(u, x0);
        } else {
            a[4 + n2] = pfma_sign<-1, 1>(u, x0);
            a[12 + n2] = pfma_sign<1, -1>(u, x0);
        }
    }
    dft16_tail<FWD>(a);
}
template <bool FWD, typename T> __device__ __forceinline__ void dft16_half(T (&a)[16])
{
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        const T x0 = a[n2], x1 = a[4 + n2];
        a[n2] = cadd(x0, x1);
        a[8 + n2] = csub(x0, x1);
        a[4 + n2] = cadd(x0, FWD ? cmul_mi(x1) : cmul_i(x1));
        a[12 + n2] = cadd(x0, FWD ? cmul_i(x1) : cmul_mi(x1));
    }
    dft16_tail<FWD>(a);
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
__device__ __forceinline__ void final_pass(T (&v)[16], int t, int T_, int Ns, const T *__restrict__ tp)
{
    constexpr int Q = 16 / RL;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k = (t + T_ * q) & (Ns - 1);
#pragma unroll
        for (int r = 1; r < RL; ++r) v[q + r * Q] = twmul<FWD>(v[q + r * Q], __ldg(&tp[(r - 1) * Ns + k]));
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
// twp: the per-pass twiddle table of length L (see pass_twiddle_count).
template <bool FWD, typename T>
__device__ __forceinline__ void fft_reg(T (&v)[16], int L, int T_, int t, T *xb, const T *__restrict__ twp)
{
    dft16<FWD>(v);                              // pass Ns = 1: no twiddles
    if (L == 16) return;
    int Ns = 16;
    const T *tp = twp;
    exchange16(v, t, T_, 1, xb);
    while (Ns * 16 <= L) {
        const int k = t & (Ns - 1);
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = twmul<FWD>(v[r], __ldg(&tp[(r - 1) * Ns + k]));
        dft16<FWD>(v);
        tp += 15 * Ns;
        if (Ns * 16 == L) return;
        exchange16(v, t, T_, Ns, xb);
        Ns *= 16;
    }
    const int RL = L / Ns;
    if (RL == 8) final_pass<FWD, 8>(v, t, T_, Ns, tp);
    else if (RL == 4) final_pass<FWD, 4>(v, t, T_, Ns, tp);
    else final_pass<FWD, 2>(v, t, T_, Ns, tp);
}

// ---------------------------------------------------------------------
// Compile-time-length variant (L >= 256): same passes and layout as
// fft_reg, but every stride is a constant, so the shared-memory and twiddle
// addresses are a per-thread base plus immediate offsets, and outputs the
// caller never reads are removed by the compiler.
//   pidx(16 t + r)           = 17 t + r                            (Ns = 1)
//   pidx(base + r Ns)        = base + (base >> 4) + r (Ns + Ns/16)   (Ns % 16 == 0)
//   pidx(t + T e)            = t + (t >> 4) + e (T + T/16)         (T % 16 == 0)
template <int Ns, int TT, typename T>
__device__ __forceinline__ void exchange_ct(T (&v)[16], int t, T *xb)
{
    T *w;
    constexpr int step = Ns == 1 ? 1 : Ns + Ns / 16;
    if constexpr (Ns == 1) {
        w = xb + 17 * t;
    } else {
        const int k = t & (Ns - 1);
        const int base = (t - k) * 16 + k;
        w = xb + base + (base >> 4);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) w[r * step] = v[r];
    __syncthreads();
    const T *rd = xb + t + (t >> 4);
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = rd[e * (TT + TT / 16)];
}

// Base twiddles of the compile-time pass with stride Ns, loaded before the
// exchange that precedes the pass so that their latency overlaps its
// barriers and shared-memory traffic:
//   radix-16 pass: W^{r k} (k = t mod Ns) for r = 1, 2, 3, 4, 8, 12; the
//   other nine are products of two loaded values (one extra rounding), which
//   spares the L1 data path 9 loads;
//   final radix-RL pass: for each of its Q = 16 / RL butterflies, r = 1..4
//   when RL = 8 (r = 5..7 as products of w4 and w1..w3), else r = 1..RL-1.
template <int L, int Ns, typename T>
__device__ __forceinline__ void load_pass_tw(const T *__restrict__ tp, int t, T (&b)[12])
{
    constexpr int TT = L / 16;
    if constexpr (Ns * 16 <= L) {
        const T *p = tp + (t & (Ns - 1));
        b[0] = __ldg(p);
        b[1] = __ldg(p + Ns);
        b[2] = __ldg(p + 2 * Ns);
        b[3] = __ldg(p + 3 * Ns);
        b[4] = __ldg(p + 7 * Ns);
        b[5] = __ldg(p + 11 * Ns);
    } else {
        constexpr int RL = L / Ns, Q = 16 / RL, NL = RL == 8 ? 4 : RL - 1;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const T *p = tp + ((t + TT * q) & (Ns - 1));
#pragma unroll
            for (int r = 0; r < NL; ++r) b[q * NL + r] = __ldg(p + r * Ns);
        }
    }
}

// The radix-16 butterflies of the compile-time passes, in registers; a
// policy with the same call operator (the tensor-core DFT engine) can stand
// in for it.
template <bool FWD> struct RegDft16 {
    template <typename T> __device__ __forceinline__ void operator()(T (&v)[16]) const { dft16<FWD>(v); }
    // first pass of a transform whose inputs v[8..15] are zero
    template <typename T> __device__ __forceinline__ void half(T (&v)[16]) const { dft16_half<FWD>(v); }
};

template <bool FWD, int L, int Ns, typename T, typename D16 = RegDft16<FWD>>
__device__ __forceinline__ void fft_ct_pass(T (&v)[16], int t, T *xb, const T *__restrict__ tp, const T (&b)[12],
                                            D16 &&d16 = D16{})
{
    constexpr int TT = L / 16;
    if constexpr (Ns * 16 <= L) {
        {
            T w[16];
            w[1] = b[0];
            w[2] = b[1];
            w[3] = b[2];
            w[4] = b[3];
            w[8] = b[4];
            w[12] = b[5];
            w[5] = cmul(w[4], w[1]);
            w[6] = cmul(w[4], w[2]);
            w[7] = cmul(w[4], w[3]);
            w[9] = cmul(w[8], w[1]);
            w[10] = cmul(w[8], w[2]);
            w[11] = cmul(w[8], w[3]);
            w[13] = cmul(w[12], w[1]);
            w[14] = cmul(w[12], w[2]);
            w[15] = cmul(w[12], w[3]);
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = twmul<FWD>(v[r], w[r]);
        }
        d16(v);
        if constexpr (Ns * 16 < L) {
            T nb[12];
            load_pass_tw<L, Ns * 16>(tp + 15 * Ns, t, nb);
            exchange_ct<Ns, TT>(v, t, xb);
            fft_ct_pass<FWD, L, Ns * 16>(v, t, xb, tp + 15 * Ns, nb, d16);
        }
    } else {
        constexpr int RL = L / Ns, Q = 16 / RL;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if constexpr (RL == 8) {
                T w[8];
#pragma unroll
                for (int r = 1; r <= 4; ++r) w[r] = b[q * 4 + r - 1];
                w[5] = cmul(w[4], w[1]);
                w[6] = cmul(w[4], w[2]);
                w[7] = cmul(w[4], w[3]);
#pragma unroll
                for (int r = 1; r < 8; ++r) v[q + r * Q] = twmul<FWD>(v[q + r * Q], w[r]);
            } else {
#pragma unroll
                for (int r = 1; r < RL; ++r) v[q + r * Q] = twmul<FWD>(v[q + r * Q], b[q * (RL - 1) + r - 1]);
            }
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
}

// HALF: the inputs v[8..15] (x[L/2 ..]) are zero and the first pass skips them.
template <bool FWD, int L, bool HALF = false, typename T, typename D16 = RegDft16<FWD>>
__device__ __forceinline__ void fft_ct(T (&v)[16], int t, T *xb, const T *__restrict__ twp, D16 &&d16 = D16{})
{
    static_assert(L >= 256 && (L & (L - 1)) == 0, "compile-time FFT needs a power of two >= 256");
    if constexpr (HALF) d16.half(v);
    else d16(v);
    T b[12];
    load_pass_tw<L, 16>(twp, t, b);
    exchange_ct<1, L / 16>(v, t, xb);
    fft_ct_pass<FWD, L, 16>(v, t, xb, twp, b, d16);
}

// Compile-time length when LC > 0, runtime length L otherwise (the
// butterfly policy d16 and the zero-half pruning HALF apply to the
// compile-time lengths).
template <bool FWD, int LC, bool HALF = false, typename T, typename D16 = RegDft16<FWD>>
__device__ __forceinline__ void fft_any(T (&v)[16], int L, int T_, int t, T *xb, const T *__restrict__ twp,
                                        D16 &&d16 = D16{})
{
    if constexpr (LC > 0) fft_ct<FWD, LC, HALF>(v, t, xb, twp, d16);
    else fft_reg<FWD>(v, L, T_, t, xb, twp);
}

// The butterfly policies of a column pass: the forward and the inverse
// transforms' radix-16 DFTs (registers by default).
struct RegEngine {
    template <bool FWD> __device__ __forceinline__ RegDft16<FWD> d16() const { return {}; }
};

// Number of complex entries of the per-pass twiddle table of length L.
__host__ __device__ constexpr int pass_twiddle_count(int L)
{
    int n = 0, Ns = 16;
    while (Ns * 16 <= L) {
        n += 15 * Ns;
        Ns *= 16;
    }
    if (Ns < L) n += (L / Ns - 1) * Ns;
    return n > 0 ? n : 1;
}

}  // namespace sg
