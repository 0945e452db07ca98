// Column pass with the radix-16 DFTs on the fifth-generation tensor cores
// (tcgen05), for the precision study of the FFT path (Sec. 5.2 FFT
// convolution evaluated with its DFT stages as matrix products; FP32
// gas-only plans, 2 nr in {2048, 4096}).
//
// The column transforms are the register Stockham FFT of sg_fft.cuh (same
// passes, twiddles, exchanges and index maps) and the column loop is the
// FP32 pass's (sg_cols.cuh); only each pass's 16-point DFTs move.  In a
// radix-16 pass thread j holds butterfly j's 16 twiddled inputs.  That
// butterfly is row j of a 128-row operand A (32 reals: re and im of each
// input), and the 16-point DFT is the real 32 x 32 block matrix B with
//     B[2n][2k] = c, B[2n + 1][2k] = -s, B[2n][2k + 1] = s, B[2n + 1][2k + 1] = c,
//     c + i s = exp(-+ 2 pi i n k / 16),
// so row j of D = A B holds the 16 outputs in natural order.
//   A: tensor memory, lane j of the thread's 128-butterfly tile, written by
//      thread j (tcgen05.st);
//   B: shared memory, built once per CTA for both signs (no swizzle, K-major
//      8 x 16-byte core matrices);
//   D: tensor memory, FP32, read back by thread j (tcgen05.ld).
// The first thread of each tile issues that tile's products and commits them
// to the tile's mbarrier; the tile's threads wait on it (bounded), then read
// their rows of D.
//
// Operands are split x = hi + lo and three products are summed in FP32:
//   MODE 1 (BF16 x3): hi = bf16(x), lo = bf16(x - hi); kind::f16, BF16 A and B,
//          hi hi + hi lo + lo hi;
//   MODE 2 (TF32 x3): hi = x with its 13 low mantissa bits cleared (a TF32
//          value), lo = the same of x - hi; kind::tf32; the same three
//          products;
//   MODE 3 (BF16 x1): bf16(x) bf16(B), one product.
//   MODE 4 (FP16 x3): as MODE 1 in FP16 (11 significand bits per part, so
//          22 in all), kind::f16 with F16 A and B.  FP16's 5-bit exponent
//          needs the operands scaled: each 128-butterfly tile multiplies its
//          inputs by the power of two that brings the tile's largest
//          magnitude into (1/2, 1] (a tile-wide max through the tile's
//          named barrier) and divides the products by it, exactly.
// BF16 and TF32 keep FP32's 8-bit exponent, so those need no scaling.
// The length-2048 transform's final radix-8 pass stays on the CUDA cores.
// Column 0 (the packed real pair) stays on the FP32 column pass.
#include <cuda_fp16.h>
#include <stdint.h>

#include "sg_cols.cuh"
#include "sg_fft.cuh"
#include "sg_internal.h"
#include "sg_mem.cuh"

namespace sg {

namespace {

// cos(2 pi q / 16), q = 0..15
__device__ constexpr double kCos16[16] = {1.0,
                                          0.92387953251128675613,
                                          0.70710678118654752440,
                                          0.38268343236508977173,
                                          0.0,
                                          -0.38268343236508977173,
                                          -0.70710678118654752440,
                                          -0.92387953251128675613,
                                          -1.0,
                                          -0.92387953251128675613,
                                          -0.70710678118654752440,
                                          -0.38268343236508977173,
                                          0.0,
                                          0.38268343236508977173,
                                          0.70710678118654752440,
                                          0.92387953251128675613};

template <int MODE> struct TcMode {
    static constexpr bool tf32 = MODE == 2;
    static constexpr bool f16 = MODE == 4;
    static constexpr bool split = MODE != 3;
    static constexpr int esz = tf32 ? 4 : 2;          // operand bytes
    static constexpr int aw = 32 * esz / 4;           // tensor-memory columns of one 32-wide operand row
    static constexpr int ks = tf32 ? 4 : 2;           // K steps of 8 (TF32) or 16 (16-bit) per product
    static constexpr int tile_cols = 2 * aw + 32;     // A hi, A lo, D (FP32)
    static constexpr int bbytes = 32 * 32 * esz;      // one B matrix
    static constexpr unsigned lbo = 128, sbo = 4 * 128 * (esz == 2 ? 1 : 2);
    static constexpr uint32_t idesc = umma_idesc(128, 32, tf32 ? 2u : f16 ? 0u : 1u);
};

__host__ __device__ constexpr int tc_tiles(int L) { return L / 16 / 128; }
__host__ __device__ constexpr int pow2_at_least(int x, int p = 32) { return p >= x ? p : pow2_at_least(x, 2 * p); }
template <int L, int MODE> __host__ __device__ constexpr int tc_tmem_cols()
{
    return pow2_at_least(tc_tiles(L) * TcMode<MODE>::tile_cols);
}

// round-to-nearest-even BF16 bit pattern of a float (finite values)
__device__ __forceinline__ uint32_t bf16_bits(float f)
{
    uint32_t u = __float_as_uint(f);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return u >> 16;
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo16, float hi16)   // lo16 in the low half
{
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi16), "f"(lo16));
    return d;
}

// Per-CTA state of the tensor-core butterflies.
struct TcState {
    uint32_t a_hi, a_lo, d;      // this thread's lane: A hi / lo and D columns
    uint32_t tbase;              // the CTA's tensor-memory allocation
    unsigned bsm;                // shared-memory address of the B matrices
    uint64_t *bar;               // product-completion mbarriers, one per tile
    unsigned phase;              // its next phase parity
    unsigned int *flag;
    int failed;                  // a completion wait gave up (uniform across the CTA)
    float *wmax;                 // FP16 mode: the warps' largest magnitudes, 4 per tile
    float unscale;               // FP16 mode: this transform stage's inverse scale
};

template <int L, int MODE, bool FWD> struct TcDft16 {
    TcState *st;
    // a zero upper half saves nothing in a dense product
    __device__ __forceinline__ void half(float2 (&v)[16]) const { (*this)(v); }
    __device__ __forceinline__ void operator()(float2 (&v)[16]) const
    {
        using M = TcMode<MODE>;
        TcState &s = *st;
        const int t = threadIdx.x;
        // split this thread's row into tensor memory
        if constexpr (M::tf32) {
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float2 x = v[8 * h + j];
                    const uint32_t hr = __float_as_uint(x.x) & 0xFFFFE000u, hm = __float_as_uint(x.y) & 0xFFFFE000u;
                    hi[2 * j] = hr;
                    hi[2 * j + 1] = hm;
                    lo[2 * j] = __float_as_uint(x.x - __uint_as_float(hr)) & 0xFFFFE000u;
                    lo[2 * j + 1] = __float_as_uint(x.y - __uint_as_float(hm)) & 0xFFFFE000u;
                }
                tmem_st16u(s.a_hi + 16 * h, hi);
                tmem_st16u(s.a_lo + 16 * h, lo);
            }
        } else if constexpr (M::f16) {
            // the tile's power-of-two scale: its largest magnitude into (1/2, 1]
            float mx = 0.f;
#pragma unroll
            for (int j = 0; j < 16; ++j) mx = fmaxf(mx, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const int tl = t >> 7, w4 = (t >> 5) & 3;
            if ((t & 31) == 0) s.wmax[4 * tl + w4] = mx;
            asm volatile("bar.sync %0, 128;" ::"r"(1 + tl) : "memory");
            mx = fmaxf(fmaxf(s.wmax[4 * tl], s.wmax[4 * tl + 1]), fmaxf(s.wmax[4 * tl + 2], s.wmax[4 * tl + 3]));
            int ex = 0;
            if (mx > 0.f && isfinite(mx)) frexpf(mx, &ex);   // mx = f 2^ex, f in [1/2, 1)
            const float sc = ldexpf(1.f, -ex), isc = ldexpf(1.f, ex);
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float xr = v[j].x * sc, xi = v[j].y * sc;
                const __half2 h = __floats2half2_rn(xr, xi);
                const __half2 l = __floats2half2_rn(xr - __low2float(h), xi - __high2float(h));
                hi[j] = *reinterpret_cast<const uint32_t *>(&h);
                lo[j] = *reinterpret_cast<const uint32_t *>(&l);
            }
            tmem_st16u(s.a_hi, hi);
            tmem_st16u(s.a_lo, lo);
            s.unscale = isc;
        } else {
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float2 x = v[j];
                const uint32_t h = pack_bf16x2(x.x, x.y);
                hi[j] = h;
                if constexpr (M::split)
                    lo[j] = pack_bf16x2(x.x - __uint_as_float(h << 16), x.y - __uint_as_float(h & 0xFFFF0000u));
            }
            tmem_st16u(s.a_hi, hi);
            if constexpr (M::split) tmem_st16u(s.a_lo, lo);
        }
        tmem_wait_st();
        // each 128-butterfly tile (4 warps) goes on its own: its rows are
        // written, its first thread issues and commits its products, and its
        // threads wait on its own mbarrier
        const int tile = t >> 7;
        tmem_fence_before();
        asm volatile("bar.sync %0, 128;" ::"r"(1 + tile) : "memory");
        tmem_fence_after();
        if ((t & 127) == 0 && !s.failed) {
            const unsigned b0 = s.bsm + (FWD ? 0u : 2u * M::bbytes);        // hi, then lo
            {
                const uint32_t tb = s.tbase + tile * M::tile_cols;
                const uint32_t ah = tb, al = tb + M::aw, d = tb + 2 * M::aw;
#pragma unroll
                for (int k = 0; k < M::ks; ++k)
                    umma_tmem_a<M::tf32>(d, ah + 8 * k, umma_sdesc(b0 + 256 * k, M::lbo, M::sbo), M::idesc, k > 0);
                if constexpr (M::split) {
#pragma unroll
                    for (int k = 0; k < M::ks; ++k)
                        umma_tmem_a<M::tf32>(d, ah + 8 * k, umma_sdesc(b0 + M::bbytes + 256 * k, M::lbo, M::sbo),
                                             M::idesc, 1u);
#pragma unroll
                    for (int k = 0; k < M::ks; ++k)
                        umma_tmem_a<M::tf32>(d, al + 8 * k, umma_sdesc(b0 + 256 * k, M::lbo, M::sbo), M::idesc, 1u);
                }
            }
            umma_commit(s.bar + tile);
        }
        bool ok = true;
        if (!s.failed) ok = mbar_wait_bounded(s.bar + tile, s.phase, s.flag);
        s.phase ^= 1u;
        s.failed = __syncthreads_or(!ok) || s.failed;
        tmem_fence_after();
        if (!s.failed) tmem_ld16c(s.d, v);
        if constexpr (M::f16) {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = make_float2(v[j].x * s.unscale, v[j].y * s.unscale);
        }
    }
};

template <int L, int MODE> struct TcEngine {
    TcState *st;
    template <bool FWD> __device__ __forceinline__ TcDft16<L, MODE, FWD> d16() const { return {st}; }
};

template <int L, int MODE> constexpr size_t tc_smem_bytes()
{
    // header, B matrices (forward hi / lo, inverse hi / lo), exchange buffer,
    // one step of staged kernel spectra
    return 1024 + 4 * (size_t)TcMode<MODE>::bbytes + (((size_t)padded_len(L) * 8 + 15) & ~(size_t)15) +
           (size_t)tab_pitch(L / 2) * 8;
}
// Shared memory a launch asks for: at least enough that no more CTAs fit on
// an SM than its 512 tensor-memory columns serve (228 KB per SM, 1 KB of it
// reserved per CTA), so no CTA's allocation has to wait for another's release.
template <int L, int MODE> constexpr size_t tc_smem_request()
{
    constexpr int ctas = 512 / tc_tmem_cols<L, MODE>();
    constexpr size_t floor_bytes = (size_t)(228 * 1024) / (ctas + 1) - 1024 + 16;
    return tc_smem_bytes<L, MODE>() > floor_bytes ? tc_smem_bytes<L, MODE>() : floor_bytes;
}

// Per-CTA set-up of the tensor-core butterflies: the tensor-memory
// allocation, the B matrices in shared memory (from smem_tc + 1024), the
// product-completion mbarriers and the state of each thread's tile.
template <int L, int MODE>
__device__ __forceinline__ void tc_setup(unsigned char *smem_tc, TcState &st, unsigned int *flag)
{
    using M = TcMode<MODE>;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_tc + 16);    // product completion, one per tile
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem_tc + 48);
    unsigned char *bmat = smem_tc + 1024;
    constexpr int T = L / 16, NCOLS = tc_tmem_cols<L, MODE>();
    const int t = threadIdx.x;
    if (t < 32) {
        tmem_alloc(tslot, NCOLS);
        tmem_relinquish();
    }
    // B matrices: element (n, k) of a K-major 32 x 32 operand at
    // (n / 8) sbo + (k / per) lbo + (n % 8) 16 + (k % per) esz, per = 16 / esz
    constexpr int per = 16 / M::esz;
    for (int idx = t; idx < 4 * 1024; idx += T) {
        const int mat = idx >> 10, e = idx & 1023, n = e >> 5, k = e & 31;   // mat: fwd hi, fwd lo, inv hi, inv lo
        const bool fwd = mat < 2, lo = mat & 1;
        const int i = n >> 1, j = k >> 1, q = (i * j) & 15;
        const double c = kCos16[q], sn = (fwd ? -1.0 : 1.0) * kCos16[(q + 12) & 15];
        // B[2j][2i] = c, B[2j + 1][2i] = -s, B[2j][2i + 1] = s, B[2j + 1][2i + 1] = c
        const double val = (n & 1) ? ((k & 1) ? c : sn) : ((k & 1) ? -sn : c);
        unsigned char *dst = bmat + mat * M::bbytes + (n >> 3) * M::sbo + (k / per) * M::lbo + (n & 7) * 16 +
                             (k % per) * M::esz;
        if constexpr (M::tf32) {
            const uint32_t h = __float_as_uint((float)val) & 0xFFFFE000u;
            const uint32_t l = __float_as_uint((float)(val - (double)__uint_as_float(h))) & 0xFFFFE000u;
            *reinterpret_cast<uint32_t *>(dst) = lo ? l : h;
        } else if constexpr (M::f16) {
            const __half h = __double2half(val);
            const __half l = __double2half(val - (double)__half2float(h));
            *reinterpret_cast<__half *>(dst) = lo ? l : h;
        } else {
            const uint32_t h = bf16_bits((float)val);
            const uint32_t l = bf16_bits((float)(val - (double)__uint_as_float(h << 16)));
            *reinterpret_cast<uint16_t *>(dst) = (uint16_t)(lo ? l : h);
        }
    }
    if (t < tc_tiles(L)) mbar_init(mbar + t, 1);
    fence_proxy_async();                   // the B matrices are read by the tensor cores
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    st.tbase = *tslot;
    const int tile = t >> 7;
    const uint32_t lane = (uint32_t)(32 * ((t >> 5) & 3)) << 16;
    st.a_hi = st.tbase + lane + tile * M::tile_cols;
    st.a_lo = st.a_hi + M::aw;
    st.d = st.a_hi + 2 * M::aw;
    st.bsm = smem_u32(bmat);
    st.bar = mbar;
    st.phase = 0;
    st.flag = flag;
    st.failed = 0;
    st.wmax = reinterpret_cast<float *>(smem_tc + 64);   // 4 per tile, in the header
    st.unscale = 1.f;
}

// Release the CTA's tensor memory once every thread's accesses are done.
template <int L, int MODE> __device__ __forceinline__ void tc_teardown(const TcState &st)
{
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(st.tbase, tc_tmem_cols<L, MODE>());
}

template <int L, int MODE>
__global__ void __launch_bounds__(L / 16, L == 4096 ? 2 : 3)
k_cols_tc(const float2 *__restrict__ sh, const float2 *__restrict__ tab, float2 *__restrict__ oh, int N,
          uint32_t outmask, const float2 *__restrict__ tw, unsigned int *flag)
{
    using M = TcMode<MODE>;
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_tc);          // staged kernel spectra
    float2 *xb = reinterpret_cast<float2 *>(smem_tc + 1024 + 4 * M::bbytes);
    float2 *tb = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(xb) +
                                            ((((size_t)padded_len(L) * 8) + 15) & ~(size_t)15));
    const int m = blockIdx.x + 1;
    TcState st;
    tc_setup<L, MODE>(smem_tc, st, flag);
    cols_pair_steps<float, L, 1>(sh, tab, oh, L / 2, N, outmask, tw, flag, xb, tb, bar, m, 0,
                                 TcEngine<L, MODE>{&st});
    tc_teardown<L, MODE>(st);
}

// One radix-16 stage alone: 256 threads per CTA each run one 16-point DFT of
// in[16 (256 blockIdx.x + t) ..] (natural order) on the tensor cores into out.
template <int MODE>
__global__ void __launch_bounds__(256, 2)
k_tc_stage(const float2 *__restrict__ in, float2 *__restrict__ out, int inverse, unsigned int *flag)
{
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    TcState st;
    tc_setup<4096, MODE>(smem_tc, st, flag);
    const size_t base = ((size_t)blockIdx.x * 256 + threadIdx.x) * 16;
    float2 v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = in[base + j];
    if (inverse) TcDft16<4096, MODE, false>{&st}(v);
    else TcDft16<4096, MODE, true>{&st}(v);
#pragma unroll
    for (int j = 0; j < 16; ++j) out[base + j] = v[j];
    tc_teardown<4096, MODE>(st);
}

template <int L, int MODE>
cudaError_t go_tc(const void *sh, const void *tab, void *oh, int nphi, uint32_t outmask, const void *tw_col,
                  unsigned int *flag, cudaStream_t s)
{
    static_assert(tc_tmem_cols<L, MODE>() <= 256, "tensor-memory budget");
    const size_t smem = tc_smem_request<L, MODE>();
    cudaError_t e = cudaFuncSetAttribute(k_cols_tc<L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_cols_tc<L, MODE><<<nphi / 2 - 1, L / 16, smem, s>>>((const float2 *)sh, (const float2 *)tab, (float2 *)oh,
                                                            nphi / 2, outmask, (const float2 *)tw_col, flag);
    return cudaGetLastError();
}

template <int MODE> cudaError_t go_stage(const void *in, void *out, long long count, int inverse, cudaStream_t s)
{
    const size_t smem = tc_smem_request<4096, MODE>();
    cudaError_t e = cudaFuncSetAttribute(k_tc_stage<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_stage<MODE><<<(unsigned)(count / 256), 256, smem, s>>>((const float2 *)in, (float2 *)out, inverse, nullptr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_stage(int engine, const void *in, void *out, long long count, int inverse, cudaStream_t s)
{
    switch (engine) {
    case SG_ENGINE_TC_BF16X3: return go_stage<1>(in, out, count, inverse, s);
    case SG_ENGINE_TC_TF32X3: return go_stage<2>(in, out, count, inverse, s);
    case SG_ENGINE_TC_FP16X3: return go_stage<4>(in, out, count, inverse, s);
    default: return go_stage<3>(in, out, count, inverse, s);
    }
}

cudaError_t launch_cols_tc(int engine, const void *sh, const void *tab, void *oh, int nr, int nphi, uint32_t outmask,
                           const void *tw_col, unsigned int *flag, cudaStream_t s)
{
    // column 0 on the FP32 column pass (one block)
    cudaError_t e = launch_cols<float>(sh, tab, oh, nr, nphi, 1, outmask, tw_col, flag, s, 1);
    if (e != cudaSuccess || nphi / 2 < 2) return e;
    const int L = 2 * nr;
#define SG_GO(M) \
    return L == 4096 ? go_tc<4096, M>(sh, tab, oh, nphi, outmask, tw_col, flag, s) \
                     : go_tc<2048, M>(sh, tab, oh, nphi, outmask, tw_col, flag, s)
    switch (engine) {
    case SG_ENGINE_TC_BF16X3: SG_GO(1);
    case SG_ENGINE_TC_TF32X3: SG_GO(2);
    case SG_ENGINE_TC_FP16X3: SG_GO(4);
    default: SG_GO(3);
    }
#undef SG_GO
}

}  // namespace sg
