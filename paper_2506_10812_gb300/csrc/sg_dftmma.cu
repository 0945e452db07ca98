// Column pass with the DFT stages on tensor cores (split-precision
// DFT-as-GEMM), for the precision study of the FFT path (Sec. 5.2 FFT
// convolution; FP32 gas-only plans with 2 nr in {2048, 4096}).
//
// Each length-L column transform is the same Stockham sequence of stages as
// the CUDA-core FFT (radix 16, 16 and 16 or 8): stage s reads butterfly j's
// inputs x[j + (L/R) r], multiplies them by the per-pass twiddles
// W_{Ns R}^{r k} (k = j mod Ns, the same tables as the FFT) and writes the R
// outputs to (j - k) R + k + r Ns.  The R-point DFTs of eight butterflies are
// one real block-matrix product on mma.sync.m16n8k16 with FP32 accumulation:
//     [Yr; Yi] = [[Fr, -Fi], [Fi, Fr]] [Xr; Xi],   F = exp(-+2 pi i m r / R),
// with the Fr and Fi tiles as the A operand and the sign folded into the B
// operand.  Operands are split into a high and a low part (x = hi + lo in
// FP16 or BF16) and three products are summed (hi hi + hi lo + lo hi), or,
// in the single-term modes, one.
//
// Scaling: every stage multiplies its inputs by the power of two that
// brings their block-wide maximum into (1/2, 1], so FP16 operands neither
// overflow nor lose their low parts to underflow; the powers of two are
// undone exactly at the output.  Column 0 (the packed m = 0 and m = nphi/2 columns) stays on the
// FP32 column pass.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "sg_fft.cuh"
#include "sg_internal.h"
#include "sg_mem.cuh"

namespace sg {

namespace {

// Shared-memory padding of the length-L buffers: chosen so that the
// fragment gathers and scatters of every stage are at most 4-way (2.7 on
// average) bank conflicted.
template <int L>
__host__ __device__ constexpr int mpad(int i)
{
    return L == 4096 ? i + (i >> 3) + (i >> 7) : i + (i >> 3) + (i >> 6);
}
template <int L>
__host__ __device__ constexpr int mpad_len()
{
    return mpad<L>(L - 1) + 1;
}

template <int MODE> struct Op;
// MODE 1: FP16 hi + lo, 3 products; 3: FP16, 1 product
// MODE 2: BF16 hi + lo, 3 products; 4: BF16, 1 product
template <> struct Op<1> {
    static constexpr bool f16 = true, split = true;
};
template <> struct Op<2> {
    static constexpr bool f16 = false, split = true;
};
template <> struct Op<3> {
    static constexpr bool f16 = true, split = false;
};
template <> struct Op<4> {
    static constexpr bool f16 = false, split = false;
};

__device__ __forceinline__ uint32_t pack_h(float a, float b, float &ra, float &rb)
{
    const __half2 h = __floats2half2_rn(a, b);
    ra = __low2float(h);
    rb = __high2float(h);
    return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack_b(float a, float b, float &ra, float &rb)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    ra = __low2float(h);
    rb = __high2float(h);
    return *reinterpret_cast<const uint32_t *>(&h);
}
// (a, b) -> hi (and lo = (a, b) - hi) as packed pairs, lower index in the low half
template <bool F16>
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    float ra, rb, x, y;
    if constexpr (F16) {
        hi = pack_h(a, b, ra, rb);
        lo = pack_h(a - ra, b - rb, x, y);
    } else {
        hi = pack_b(a, b, ra, rb);
        lo = pack_b(a - ra, b - rb, x, y);
    }
}
__device__ __forceinline__ uint32_t neg2(uint32_t v) { return v ^ 0x80008000u; }

template <bool F16>
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    if constexpr (F16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// d += A B with the split terms of the mode
template <int MODE>
__device__ __forceinline__ void mma_split(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                          uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1)
{
    constexpr bool F16 = Op<MODE>::f16;
    mma<F16>(d, ah, bh0, bh1);
    if constexpr (Op<MODE>::split) {
        mma<F16>(d, ah, bl0, bl1);
        mma<F16>(d, al, bh0, bh1);
    }
}

// A-fragment table (built on the host, per precision): [set][lane][4] with
// sets 0/1 Fr16 hi/lo, 2/3 Fi16 hi/lo (forward sign, Fi = -sin), 4/5 the
// forward radix-8 block hi/lo, 6/7 the inverse radix-8 block hi/lo.
__device__ __forceinline__ void load_frag(const uint32_t *__restrict__ tab, int set, int lane, uint32_t (&a)[4])
{
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(tab) + set * 32 + lane);
    a[0] = v.x;
    a[1] = v.y;
    a[2] = v.z;
    a[3] = v.w;
}

// One radix-R Stockham stage in place on buf (the last stage writes dst):
// the warp's n-tiles are gathered (inputs times `scale`, a power of two),
// transformed and kept in registers, the block synchronises, then every
// warp scatters.  Returns the block's largest output magnitude (reduced
// through red[8] across the stage's own barrier).
template <int MODE, bool FWD, int L, int R>
__device__ __forceinline__ float mma_stage(float2 *buf, float2 *dst, int Ns, const float2 *__restrict__ tp,
                                           float scale, const uint32_t *__restrict__ atab, float *red)
{
    constexpr bool F16 = Op<MODE>::f16;
    constexpr int NB = L / R;               // butterflies
    constexpr int TPW = NB / 64;            // n8-tiles per warp (8 warps)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane & 3, g = lane >> 2;
    float out[TPW][8];
    if constexpr (R == 16) {
        uint32_t frh[4], frl[4], fih[4], fil[4];
        load_frag(atab, 0, lane, frh);
        load_frag(atab, 1, lane, frl);
        load_frag(atab, 2, lane, fih);
        load_frag(atab, 3, lane, fil);
#pragma unroll
        for (int u = 0; u < TPW; ++u) {
            const int j = (warp + 8 * u) * 8 + g, k = j & (Ns - 1);
            float2 x[4];
            const int in[4] = {2 * q, 2 * q + 1, 2 * q + 8, 2 * q + 9};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                float2 v = buf[mpad<L>(j + NB * in[s])];
                if (Ns > 1 && in[s] > 0) v = twmul<FWD>(v, __ldg(&tp[(in[s] - 1) * Ns + k]));
                x[s] = make_float2(v.x * scale, v.y * scale);
            }
            uint32_t rh0, rl0, rh1, rl1, ih0, il0, ih1, il1;
            split2<F16>(x[0].x, x[1].x, rh0, rl0);     // rows 2q, 2q+1 (real parts)
            split2<F16>(x[2].x, x[3].x, rh1, rl1);     // rows 2q+8, 2q+9
            split2<F16>(x[0].y, x[1].y, ih0, il0);     // imaginary parts
            split2<F16>(x[2].y, x[3].y, ih1, il1);
            float dre[4] = {0.f, 0.f, 0.f, 0.f}, dim[4] = {0.f, 0.f, 0.f, 0.f};
            if constexpr (FWD) {
                // re = Fr xr - Fi xi, im = Fi xr + Fr xi
                mma_split<MODE>(dre, frh, frl, rh0, rh1, rl0, rl1);
                mma_split<MODE>(dre, fih, fil, neg2(ih0), neg2(ih1), neg2(il0), neg2(il1));
                mma_split<MODE>(dim, fih, fil, rh0, rh1, rl0, rl1);
                mma_split<MODE>(dim, frh, frl, ih0, ih1, il0, il1);
            } else {
                // conj(F): re = Fr xr + Fi xi, im = -Fi xr + Fr xi
                mma_split<MODE>(dre, frh, frl, rh0, rh1, rl0, rl1);
                mma_split<MODE>(dre, fih, fil, ih0, ih1, il0, il1);
                mma_split<MODE>(dim, fih, fil, neg2(rh0), neg2(rh1), neg2(rl0), neg2(rl1));
                mma_split<MODE>(dim, frh, frl, ih0, ih1, il0, il1);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                out[u][c] = dre[c];
                out[u][4 + c] = dim[c];
            }
        }
    } else {
        static_assert(R == 8, "final radix 8 or 16");
        uint32_t bh[4], bl[4];
        load_frag(atab, FWD ? 4 : 6, lane, bh);
        load_frag(atab, FWD ? 5 : 7, lane, bl);
#pragma unroll
        for (int u = 0; u < TPW; ++u) {
            const int j = (warp + 8 * u) * 8 + g, k = j & (Ns - 1);
            float2 x[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int r = 2 * q + s;
                float2 v = buf[mpad<L>(j + NB * r)];
                if (Ns > 1 && r > 0) v = twmul<FWD>(v, __ldg(&tp[(r - 1) * Ns + k]));
                x[s] = make_float2(v.x * scale, v.y * scale);
            }
            uint32_t h0, l0, h1, l1;
            split2<F16>(x[0].x, x[1].x, h0, l0);       // rows 2q, 2q+1: real parts
            split2<F16>(x[0].y, x[1].y, h1, l1);       // rows 2q+8, 2q+9: imaginary parts
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            mma_split<MODE>(d, bh, bl, h0, h1, l0, l1);
            // d0, d1: real part of output g for butterflies 2q, 2q+1; d2, d3: imaginary parts
            out[u][0] = d[0];
            out[u][1] = d[1];
            out[u][4] = d[2];
            out[u][5] = d[3];
        }
    }
    float mx = 0.f;
#pragma unroll
    for (int u = 0; u < TPW; ++u)
#pragma unroll
        for (int c = 0; c < 8; ++c) mx = fmaxf(mx, fabsf(out[u][c]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();                               // every gather of the stage precedes the scatter
    mx = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
#pragma unroll
    for (int u = 0; u < TPW; ++u) {
        const int jb = (warp + 8 * u) * 8 + 2 * q;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int j = jb + c, k = j & (Ns - 1);
            const int base = (j - k) * R + k;
            if constexpr (R == 16) {
                dst[mpad<L>(base + g * Ns)] = make_float2(out[u][c], out[u][4 + c]);
                dst[mpad<L>(base + (g + 8) * Ns)] = make_float2(out[u][2 + c], out[u][6 + c]);
            } else {
                dst[mpad<L>(base + g * Ns)] = make_float2(out[u][c], out[u][4 + c]);
            }
        }
    }
    __syncthreads();
    return mx;
}

// Power of two p with max_abs * p in (1/2, 1] (1 for a zero block).
__device__ __forceinline__ float pow2_scale(float max_abs)
{
    if (!(max_abs > 0.f)) return 1.f;
    int e;
    frexpf(max_abs, &e);                            // max_abs = f 2^e, f in [1/2, 1)
    return ldexpf(1.f, -e);
}

// Full transform of buf (in place; the last stage writes dst).  Every stage
// scales its inputs by the power of two that brings the largest of them to
// (1/2, 1] (scale0 for the first stage), so the operands' low parts stay
// clear of FP16 underflow; returns the product of the scales applied.
template <int MODE, bool FWD, int L>
__device__ float mma_transform(float2 *buf, float2 *dst, const float2 *__restrict__ twp, float scale0,
                               const uint32_t *__restrict__ atab, float *red)
{
    float m = mma_stage<MODE, FWD, L, 16>(buf, buf, 1, twp, scale0, atab, red);
    const float s1 = pow2_scale(m);
    m = mma_stage<MODE, FWD, L, 16>(buf, buf, 16, twp, s1, atab, red);
    const float s2 = pow2_scale(m);
    if constexpr (L == 4096) {
        mma_stage<MODE, FWD, L, 16>(buf, dst, 256, twp + 15 * 16, s2, atab, red);
    } else {
        static_assert(L == 2048, "column length 2048 or 4096");
        mma_stage<MODE, FWD, L, 8>(buf, dst, 256, twp + 15 * 16, s2, atab, red);
    }
    return scale0 * s1 * s2;
}

__device__ float block_max(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
    return m;
}

template <int MODE, int L>
__global__ void __launch_bounds__(256, 2)
k_cols_mma(const float2 *__restrict__ sh, const float2 *__restrict__ tab, float2 *__restrict__ oh, int nr, int N,
           uint32_t outmask, const float2 *__restrict__ twp, const uint32_t *__restrict__ atab, unsigned int *flag)
{
    constexpr int PL = mpad_len<L>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    float *red = reinterpret_cast<float *>(smem_raw + 16);
    float2 *Z = reinterpret_cast<float2 *>(smem_raw + 64);
    float2 *W = Z + ((PL + 1) & ~1);
    float2 *tb = W + ((PL + 1) & ~1);
    const int H = nr, P = tab_pitch(nr);
    const int m = blockIdx.x + 1;                  // column 0 runs on the FP32 column pass
    const bool leader = threadIdx.x == 0;
    auto issue = [&](int c) {
        if (leader) {
            mbar_expect_tx(bar, P * sizeof(float2));
            tma_load_1d(tb, tab + ((size_t)c * (N + 1) + m) * P, P * sizeof(float2), bar, l2_evict_first());
        }
    };
    int first = 0;
    while (first < 3 && !((outmask >> first) & 1u)) ++first;
    if (leader) mbar_init(bar, 1);
    __syncthreads();
    if (first < 3) issue(first);
    // the column, zero-padded to L, into W
    float mx = 0.f;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const float2 v = i < nr ? ld_hint(sh + blk(m, i, nr), l2_evict_first()) : make_float2(0.f, 0.f);
        W[mpad<L>(i)] = v;
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    const float s0 = pow2_scale(block_max(mx, red));
    const float sf = mma_transform<MODE, true, L>(W, Z, twp, s0, atab, red);   // Z = FFT(x) sf
    unsigned ph = 0;
    for (int c = first; c < 3; ++c) {
        if (!((outmask >> c) & 1u)) continue;
        const bool ok = mbar_wait_bounded(bar, ph & 1u, flag);
        ++ph;
        if (__syncthreads_or(!ok)) return;
        // products with the kernel spectrum (K_phi stored as i K-hat: times -i)
        float pm = 0.f;
        for (int k = threadIdx.x; k < L; k += blockDim.x) {
            float2 S = k <= H ? tb[k] : cconj(tb[2 * H - k]);
            if (c == 2) S = cmul_mi(S);
            const float2 p = cmul(Z[mpad<L>(k)], S);
            W[mpad<L>(k)] = p;
            pm = fmaxf(pm, fmaxf(fabsf(p.x), fabsf(p.y)));
        }
        const float s1 = pow2_scale(block_max(pm, red));   // block_max synchronises: tb is free
        int next = c + 1;
        while (next < 3 && !((outmask >> next) & 1u)) ++next;
        if (next < 3) {
            if (leader) fence_proxy_async();
            issue(next);
        }
        const float si = mma_transform<MODE, false, L>(W, W, twp, s1, atab, red);
        // y = IFFT(Z S) = W / (sf si): powers of two, exact
        const float un = 1.f / (sf * si);
        float2 *o = oh + (size_t)c * N * nr;
        for (int i = threadIdx.x; i < nr; i += blockDim.x) {
            const float2 v = W[mpad<L>(i)];
            st_hint(o + blk(m, i, nr), make_float2(v.x * un, v.y * un), l2_evict_last());
        }
        __syncthreads();                           // W is rewritten by the next product
    }
    if (leader) mbar_inval(bar);
}

template <int MODE, int L>
cudaError_t go_mma(const void *sh, const void *tab, void *oh, int nr, int nphi, uint32_t outmask, const void *tw_col,
                   const uint32_t *atab, unsigned int *flag, cudaStream_t s)
{
    const int N = nphi / 2;
    constexpr int PL2 = (mpad_len<L>() + 1) & ~1;
    const size_t smem = 64 + (size_t)2 * PL2 * sizeof(float2) + (size_t)tab_pitch(L / 2) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute((const void *)k_cols_mma<MODE, L>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_cols_mma<MODE, L><<<N - 1, 256, smem, s>>>((const float2 *)sh, (const float2 *)tab, (float2 *)oh, nr, N, outmask,
                                                (const float2 *)tw_col, atab, flag);
    return cudaGetLastError();
}

}  // namespace

size_t cols_mma_smem(int nr)
{
    const int L = 2 * nr;
    const int PL = L == 4096 ? mpad_len<4096>() : mpad_len<2048>();
    return 64 + (size_t)2 * ((PL + 1) & ~1) * sizeof(float2) + (size_t)tab_pitch(nr) * sizeof(float2);
}

cudaError_t launch_cols_mma(int engine, const void *sh, const void *tab, void *oh, int nr, int nphi, uint32_t outmask,
                            const void *tw_col, const uint32_t *atab, unsigned int *flag, cudaStream_t s)
{
    // column 0 on the FP32 column pass (one block)
    cudaError_t e = launch_cols<float>(sh, tab, oh, nr, nphi, 1, outmask, tw_col, flag, s, 1);
    if (e != cudaSuccess || nphi / 2 < 2) return e;
    const int L = 2 * nr;
#define SG_GO(M)                                                                                              \
    return L == 4096 ? go_mma<M, 4096>(sh, tab, oh, nr, nphi, outmask, tw_col, atab, flag, s)                 \
                     : go_mma<M, 2048>(sh, tab, oh, nr, nphi, outmask, tw_col, atab, flag, s)
    switch (engine) {
    case 1: SG_GO(1);
    case 2: SG_GO(2);
    case 3: SG_GO(3);
    default: SG_GO(4);
    }
#undef SG_GO
}

}  // namespace sg

// ------------------------------------------------------------------ host
namespace sg {

namespace {

// Round-to-nearest-even conversions of a float to IEEE binary16 and to
// bfloat16 (bit patterns), from the formats' definitions.
uint16_t to_bf16(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
uint16_t to_f16(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    const uint32_t sign = (u >> 16) & 0x8000u;
    const int e = (int)((u >> 23) & 0xFF) - 127;    // unbiased exponent
    uint32_t mant = u & 0x7FFFFFu;
    if (e > 15) return (uint16_t)(sign | 0x7C00u);   // overflow (never for |f| <= 1)
    if (e >= -14) {                                   // normal: 10 mantissa bits
        uint32_t h = ((uint32_t)(e + 15) << 10) | (mant >> 13);
        const uint32_t rem = mant & 0x1FFFu;
        if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;   // carries into the exponent correctly
        return (uint16_t)(sign | h);
    }
    if (e < -25) return (uint16_t)sign;               // below half the smallest subnormal
    mant |= 0x800000u;                                // subnormal: f = mant 2^(e - 23) = (mant 2^(e + 1)) 2^-24
    const int sh = -e - 1;                            // 14 .. 24
    uint32_t h = mant >> sh;
    const uint32_t rem = mant & ((1u << sh) - 1u), half = 1u << (sh - 1);
    if (rem > half || (rem == half && (h & 1u))) ++h;
    return (uint16_t)(sign | h);
}

}  // namespace

void dftmma_frag_table(bool f16, uint32_t *out)
{
    auto cvt = [&](float v) -> uint32_t { return f16 ? to_f16(v) : to_bf16(v); };
    auto back = [&](uint32_t b) -> float {
        if (!f16) {
            const uint32_t u = b << 16;
            float f;
            memcpy(&f, &u, 4);
            return f;
        }
        const uint32_t s = (b & 0x8000u) << 16, e = (b >> 10) & 0x1F, m = b & 0x3FF;
        if (e == 0) return (s ? -1.f : 1.f) * ldexpf((float)m, -24);
        const uint32_t u = s | ((e - 15 + 127) << 23) | (m << 13);
        float f;
        memcpy(&f, &u, 4);
        return f;
    };
    // tile(set, row, col) in FP64
    auto tile = [&](int set, int r, int c) -> double {
        const double tau = 6.283185307179586476925286766559;
        if (set < 2) return cos(tau * r * c / 16.0);            // Fr16
        if (set < 4) return -sin(tau * r * c / 16.0);           // Fi16 (forward sign)
        const bool fwd = set < 6;
        const int m = r & 7, k = c & 7;
        const double cs = cos(tau * m * k / 8.0), fi = (fwd ? -1.0 : 1.0) * sin(tau * m * k / 8.0);
        const bool ro = r >= 8, co = c >= 8;
        if (!ro && !co) return cs;
        if (!ro && co) return -fi;
        if (ro && !co) return fi;
        return cs;
    };
    for (int set = 0; set < 8; ++set) {
        const bool lo = set & 1;
        for (int lane = 0; lane < 32; ++lane) {
            const int g = lane >> 2, q = lane & 3;
            const int rows[4] = {g, g + 8, g, g + 8}, cols[4] = {2 * q, 2 * q, 2 * q + 8, 2 * q + 8};
            for (int w = 0; w < 4; ++w) {
                uint32_t word = 0;
                for (int h = 0; h < 2; ++h) {
                    const double v = tile(set, rows[w], cols[w] + h);
                    const float vf = (float)v;
                    const uint32_t hb = cvt(vf);
                    const uint32_t bits = lo ? cvt((float)(v - (double)back(hb))) : hb;
                    word |= bits << (16 * h);
                }
                out[(set * 32 + lane) * 4 + w] = word;
            }
        }
    }
}

}  // namespace sg
