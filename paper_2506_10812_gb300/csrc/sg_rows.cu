// Row transforms of the FFT-convolution path (Sec. 5.2 and App. C of Rendon
// Restrepo et al. 2025) for sm_103a: the forward R2C of every source row
// (radially scaled by r_i, row mean removed; packed spectra stored
// column-major) and the inverse C2R of every output row with its epilogue
// (accelerations / r_i, finite flag).  The FP32 rows of the hot lengths move
// their column-major side by tensor copies; other lengths and FP64 use the
// load/store-unit transpose kernels.
#include <math.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <type_traits>
#include <utility>

#include "sg_fft.cuh"
#include "sg_internal.h"
#include "sg_launch.h"
#include "sg_mem.cuh"

namespace sg {

// ----------------------------------------------------------------- sizes
// Rows per CTA of the transpose row kernels: up to SG_ROW_RPC (4; 8 measured
// slower: 1024-thread CTAs with 139 KB of shared memory), at most 1024
// threads (nphi / 32 per row) and 160 KB of shared memory.
#ifndef SG_ROW_RPC
#define SG_ROW_RPC 4
#endif
__host__ __device__ constexpr int row_rpc_of(int nphi, int esz)
{
    int rpc = SG_ROW_RPC;
    while (rpc > 1 && ((nphi / 32) * rpc > 1024 || (long long)rpc * padded_len(nphi / 2) * esz > 160 * 1024))
        rpc >>= 1;
    return rpc;
}
__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

int row_rpc(int nphi, bool f64) { return row_rpc_of(nphi, f64 ? 16 : 8); }

size_t row_smem_bytes(int nphi, int rpc, bool f64)
{
    return (size_t)rpc * padded_len(nphi / 2) * (f64 ? 16 : 8) + 64 * sizeof(double);
}

// ------------------------------------------- tensor-copy row transforms
// FP32 row transforms of the compiled lengths (nphi = 2 NC, NC = 256 .. 2048),
// NR rows per CTA, whose [N][rows] side moves by 2-D tensor
// copies: the forward transform leaves its [N][NR] spectrum tile with bulk
// tensor stores, the inverse transform receives its tile by bulk tensor
// loads, so neither spends load/store-unit instructions on the column slices.
// The tile is dense, (k, g) at NR k + g; lane l of warp w owns row g = l mod
// NR and transform thread t = w 32 / NR + l / NR, so each half-warp (the unit
// in which shared memory serves 8-byte accesses) touches 16 consecutive tile
// slots.  Row g's exchange buffer starts at g * row_pitch_tma(N) elements.
// The forward kernel also stages its input rows by 1-D bulk copies (so
// it needs 16-byte aligned inputs; the launch falls back to the transpose
// kernel otherwise).  On the 2048 x 4096 disc the pair takes 28.0 + 52.5 us
// per solve against 30.5 + 64.0 us for the load/store-unit transpose
// kernels; computing tw(t + T e) from tw(t) measured faster than loading it.
#ifndef SG_ROWS_FWD_TMA
#define SG_ROWS_FWD_TMA 1          // 0: forward rows by the load/store-unit transpose kernel
#endif
// The inverse rows store the solve's outputs as streaming (evict-first)
// writes: nothing here reads them again, and they would otherwise push out of
// L2 the column output that later CTAs still read.  Gas + dust 2048 x 4096
// (six outputs, 201 MB of column output): inverse rows 92.4 -> 81.0 us,
// solve 291 -> 277 us; the gas solve (three outputs) is unchanged.
#ifndef SG_ROWS_INV_STREAM
#define SG_ROWS_INV_STREAM 1
#endif
// Rows per CTA (NR, 2 or 4) is a per-plan choice (sg_set_tiles); the default
// is 4 for the forward transform and 2 for the inverse (2048 x 4096 disc: the
// inverse 51.0 -> 45.3 us with 2, the forward 27.2 -> 30.6 us; a shared-memory
// floor holding the 2-row inverse to 3 CTAs per SM, 49.0 us).
constexpr int kRowHdr = 1024;                     // mbarrier + partial sums; the tile starts 1024-aligned
// row pitch = 16 / NR (mod 16): a half-warp's NR rows x 16 / NR consecutive
// indices fall in 16 distinct bank pairs
__host__ __device__ constexpr int row_pitch_tma(int N, int NR) { return padded_len(N) + 16 / NR - 1; }
// The 2-row inverse fits 48 registers without spills at 1280 threads per SM
// (5 CTAs): 46.9 -> 45.4 us; at 1536 (40 registers) it spills and takes 56 us.
#ifndef SG_ROWS_INV_SM_THREADS
#define SG_ROWS_INV_SM_THREADS 1280  // resident threads per SM the inverse kernel is compiled for
#endif
// threads of an NR-row CTA of length-2 NC rows, and the CTAs per SM that keep
// `sm_threads` threads resident (1024: 64 registers each)
constexpr int rows_tma_threads(int NC, int NR) { return NR * NC / 16; }
constexpr int rows_tma_min_blocks(int NC, int NR, int sm_threads)
{
    return sm_threads / rows_tma_threads(NC, NR) < 32 ? sm_threads / rows_tma_threads(NC, NR) : 32;
}
size_t row_tma_smem_bytes(int N, int NR)
{
    const size_t tile = (size_t)N * NR * 8, xb = (size_t)NR * row_pitch_tma(N, NR) * 8;
    return kRowHdr + (tile > xb ? tile : xb);
}

// cos(2 pi e / 32), e = 0..8
__device__ constexpr double kCos32[9] = {1.0,
                                         0.98078528040323044913,
                                         0.92387953251128675613,
                                         0.83146961230254523708,
                                         0.70710678118654752440,
                                         0.55557023301960222474,
                                         0.38268343236508977173,
                                         0.19509032201612826785,
                                         0.0};
// exp(-2 pi i e / 32), e = 0..15
template <int E> __device__ __forceinline__ float2 root32()
{
    constexpr double c = E <= 8 ? kCos32[E] : -kCos32[16 - E];
    constexpr double s = E <= 8 ? kCos32[8 - E] : kCos32[E - 8];
    return make_float2((float)c, (float)-s);
}
// tw(t + T e) = exp(-2 pi i (t + T e) / nphi) with T / nphi = 1 / 32: the
// loaded tw(t) times a compile-time root (one extra rounding)
template <int E> __device__ __forceinline__ float2 tw_step(float2 w0)
{
    if constexpr (E == 0) return w0;
    else return cmul(w0, root32<E>());
}
template <int E, typename F> __device__ __forceinline__ void unroll16(F &&f)
{
    if constexpr (E < 16) {
        f(std::integral_constant<int, E>{});
        unroll16<E + 1>(f);
    }
}

template <int NC, int NR>
__global__ void __launch_bounds__(rows_tma_threads(NC, NR), rows_tma_min_blocks(NC, NR, 1024))
k_rows_fwd_tma(const float *__restrict__ x0, const float *__restrict__ x1, const __grid_constant__ CUtensorMap tm,
               const float2 *__restrict__ tw, const float2 *__restrict__ twp, const float *__restrict__ rscale,
               int dc, unsigned int *tflag, int row0, int ahead)
{
    static_assert(NR == 2 || NR == 4, "the tensor-copy row transforms take 2 or 4 rows per CTA");
    constexpr int N = NC, T = N / 16, NW = NR * T / 32, PLS = row_pitch_tma(N, NR), XS = T + T / 16;
    extern __shared__ __align__(1024) unsigned char smem_tma[];
    griddep_launch();                     // the column pass may set up once every row CTA runs
    float *red = reinterpret_cast<float *>(smem_tma + 64);              // NW x NR partial sums
    float2 *reg = reinterpret_cast<float2 *>(smem_tma + kRowHdr);
    if (smem_u32(reg) & 127u) {                                         // TMA alignment (never expected)
        if (threadIdx.x == 0 && tflag) atomicOr(tflag, 2u);
        return;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane & (NR - 1), t = w * (32 / NR) + lane / NR;
    const int a = blockIdx.y, i0 = row0 + blockIdx.x * NR, i = i0 + g;
    const float *xa = a == 0 ? x0 : x1;
    const float sc = rscale ? rscale[i] : 1.f;
    const float2 w0 = __ldg(&tw[t]);                     // R2C twiddle base, used after the transform
    float2 v[16];
    {
        // the NR rows (contiguous) land at a pitch of N + 16 / NR complex,
        // which keeps the half-warp reads conflict-free; the staging overlays
        // the exchange buffers (the transform synchronises first)
        constexpr int IPS = N + 16 / NR;
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem_tma);
        if (threadIdx.x == 0) mbar_init(bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint64_t pf = l2_evict_first();
            mbar_expect_tx(bar, (unsigned)N * 8u * NR);
#pragma unroll
            for (int r = 0; r < NR; ++r) tma_load_1d(reg + r * IPS, xa + (size_t)(i0 + r) * 2 * N, N * 8, bar, pf);
        }
        if (!__syncthreads_and(mbar_wait_bounded(bar, 0, tflag))) return;
        // the CTA `ahead` places on (one wave of resident CTAs later): its input rows
        // go to L2 while this wave transforms, so the next wave does not start on DRAM
        if (threadIdx.x == 0 && ahead > 0 && blockIdx.x + ahead < gridDim.x)
            prefetch_l2_bulk(xa + (size_t)(i0 + ahead * NR) * 2 * N, (unsigned)(N * 8 * NR));
        const float2 *xs = reg + g * IPS + t;
#pragma unroll
        for (int e = 0; e < 16; ++e) {                    // z[n] = x[2n] + i x[2n+1]
            const float2 z = xs[T * e];
            v[e] = make_float2(z.x * sc, z.y * sc);
        }
    }
    float mean = 0.f;
    if (dc) {
        float s = 0.f;
#pragma unroll
        for (int e = 0; e < 16; ++e) s += v[e].x + v[e].y;
        // lanes of one row differ in the bits above log2(NR)
#pragma unroll
        for (int m = NR; m < 32; m <<= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
        if (lane < NR) red[w * NR + lane] = s;
        __syncthreads();
        s = 0.f;
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) s += red[ww * NR + g];
        mean = s / (float)(2 * N);
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = make_float2(v[e].x - mean, v[e].y - mean);
    }
    float2 *xb = reg + g * PLS;
    fft_ct<true, N>(v, t, xb, twp);
    // X[k] = E[k] + W^k O[k], E = (Z[k] + Z*[N-k]) / 2, O = (Z[k] - Z*[N-k]) / 2i
    __syncthreads();
    float2 *zs = xb + t + (t >> 4);                       // pidx(t + T e) = t + (t >> 4) + e XS
#pragma unroll
    for (int e = 0; e < 16; ++e) zs[e * XS] = v[e];
    __syncthreads();
    const float2 *zc = xb + (N - t) + (N >> 4) + ((-t) >> 4);   // pidx(N - k) = zc - e XS
    unroll16<0>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        const float2 Z = v[e];
        if (e == 0 && t == 0) {
            // (X[0], X[nphi/2]) packed; the mean only enters X[0]
            v[e] = make_float2(Z.x + Z.y + mean * (float)(2 * N), Z.x - Z.y);
        } else {
            const float2 Zc = cconj(zc[-e * XS]);
            const float2 E = cscale(cadd(Z, Zc), 0.5f);
            const float2 O = cscale(cmul_mi(csub(Z, Zc)), 0.5f);
            v[e] = cadd(E, cmul(O, tw_step<e>(w0)));
        }
    });
    __syncthreads();                                      // the tile overwrites the exchange buffers
    float2 *tl = reg + NR * t + g;
#pragma unroll
    for (int e = 0; e < 16; ++e) tl[NR * T * e] = v[e];
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t pl = l2_evict_last();
#pragma unroll
        for (int b = 0; b < N / 256; ++b) tma_store_2d(&tm, 2 * i0, a * N + 256 * b, reg + NR * 256 * b, pl);
        bulk_commit();
        bulk_wait_read_all();
    }
}

// CTAs of a tensor-copy forward instance resident at once on the current
// device (CTAs per SM x SMs), queried once per device, row length and rows
// per CTA; 0 when the query fails (no prefetch then).  The forward rows of
// the 2048 x 4096 disc run 512 CTAs in two waves of 304: each first-wave
// CTA prefetches the input rows of the CTA that takes its place, 25.6 against
// 26.7 us (step 132.0 against 133.4 us).
template <int NC, int NR> int fwd_resident_ctas()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    int per = 0, nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rows_fwd_tma<NC, NR>, rows_tma_threads(NC, NR),
                                                      row_tma_smem_bytes(NC, NR)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    v = per * nsm;
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

// ------------------------------------------------------------ row R2C
// rscale: optional per-row multiplier (the radial scaling r_i); dc: remove
// the row mean before the transform.
// NC > 0: compile-time row transform length (nphi / 2).
template <typename R, int NC>
__global__ void __launch_bounds__(1024, 1)
k_rows_fwd(const R *__restrict__ x0, const R *__restrict__ x1, cplx<R> *__restrict__ xh, int nrows,
           int nphi_rt, int rpc, const cplx<R> *__restrict__ tw, const cplx<R> *__restrict__ twp,
           const R *__restrict__ rscale, int dc, int row0)
{
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *red = reinterpret_cast<R *>(smem_raw);                 // 64 reals: per-warp partial sums
    C *sm = reinterpret_cast<C *>(smem_raw + 64 * sizeof(double));
    griddep_launch();
    const int nphi = NC > 0 ? 2 * NC : nphi_rt;
    const int N = nphi >> 1, T = N >> 4;
    if (NC > 0) rpc = row_rpc_of(2 * NC, sizeof(C));           // compile-time for the hot lengths
    const int lg = ilog2(rpc);
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    const int a = blockIdx.y;
    const int i0 = row0 + blockIdx.x * rpc;
    const C *xr = reinterpret_cast<const C *>((a == 0 ? x0 : x1) + (size_t)(i0 + g) * nphi);
    C *xb = sm + g * padded_len(N);
    C v[16];
    const R sc = rscale ? rscale[i0 + g] : (R)1;
#pragma unroll
    for (int e = 0; e < 16; ++e) {                        // z[n] = x[2n] + i x[2n+1]
        const C z = xr[t + T * e];
        v[e] = mkc<C>(z.x * sc, z.y * sc);
    }
    R mean = 0;
    if (dc) {
        R s = 0;
#pragma unroll
        for (int e = 0; e < 16; ++e) s += v[e].x + v[e].y;
        // reduce over the T threads of this row (aligned power-of-two segment)
        const int seg = T < 32 ? T : 32;
        const unsigned lanes = blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u);
        for (int o = seg >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(lanes, s, o);
        if (T > 32) {
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
            __syncthreads();
            s = 0;
            const int w0 = (g * T) >> 5, nw = T >> 5;
            for (int w = 0; w < nw; ++w) s += red[w0 + w];
        }
        mean = s / (R)nphi;
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = mkc<C>(v[e].x - mean, v[e].y - mean);
    }
    fft_any<true, NC>(v, N, T, t, xb, twp);
    // X[k] = E[k] + W^k O[k], E = (Z[k] + Z*[N-k]) / 2, O = (Z[k] - Z*[N-k]) / 2i
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) xb[pidx(t + T * e)] = v[e];
    __syncthreads();
    // FAST: compile-time length, 4 rows, column-major output (T % 16 == 0):
    // every shared-memory and global index below is a per-thread base plus a
    // compile-time multiple of e (or of the copy step).
    constexpr bool FAST = NC >= 256 && BW == 1 && row_rpc_of(2 * NC, sizeof(C)) == 4;
    // pidx(N - k) = zc0 - e (T + T/16) for k = t + T e (N, T e multiples of 16)
    const int zc0 = (N - t) + (N >> 4) + ((-t) >> 4);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int k = t + T * e;
        const C Z = v[e];
        if (e == 0 && t == 0) {
            // (X[0], X[nphi/2]) packed; the mean only enters X[0]
            v[e] = mkc<C>(Z.x + Z.y + mean * (R)nphi, Z.x - Z.y);
        } else {
            const C Zc = cconj(xb[FAST ? zc0 - e * (T + T / 16) : pidx(N - k)]);
            const C E = cscale(cadd(Z, Zc), (R)0.5);
            const C O = cscale(cmul_mi(csub(Z, Zc)), (R)0.5);
            v[e] = cadd(E, cmul(O, __ldg(&tw[k])));
        }
    }
    // write through a [N][rpc] tile: rpc consecutive rows of each column (x BW columns)
    __syncthreads();
    C *out = xh + (size_t)a * N * nrows;
    const uint64_t pl = l2_evict_last();
    if constexpr (FAST) {
        // tile_idx_g(t + T e, g, 2) = 4 (t + T e) + (g ^ ((t >> 2) & 3))
        const int tb0 = 4 * t + (g ^ ((t >> 2) & 3));
#pragma unroll
        for (int e = 0; e < 16; ++e) sm[tb0 + 4 * T * e] = v[e];
        __syncthreads();
        // copy step j: column m = (x >> 2) + j nthr / 4, row gg = x & 3 (x = threadIdx.x)
        constexpr int nthr = (NC / 16) * 4;
        const int x = threadIdx.x, gg = x & 3, m0 = x >> 2;
        const int sb0 = 4 * m0 + (gg ^ ((m0 >> 2) & 3));          // (m >> 2) & 3 is the same for every j
        C *o0 = out + (size_t)m0 * nrows + i0 + gg;
#pragma unroll
        for (int j = 0; j < 16; ++j) st_hint(o0 + (size_t)j * (nthr / 4) * nrows, sm[sb0 + j * nthr], pl);
    } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) sm[tile_idx_g<C>(t + T * e, g, lg)] = v[e];
        __syncthreads();
        const int per = rpc * BW;
        for (int idx = threadIdx.x; idx < N * rpc; idx += blockDim.x) {
            const int bb = idx / per, rem = idx - bb * per;
            const int gg = rem / BW, c = rem - gg * BW;
            st_hint(out + ((size_t)bb * nrows + i0 + gg) * BW + c, sm[tile_idx_g<C>(bb * BW + c, gg, lg)], pl);
        }
    }
}

template <typename R>
cudaError_t launch_rows_fwd(const R *x0, const R *x1, int nsrc, void *xh, int nrows, int nphi,
                            const void *tw_row, const void *twp_row, const R *rscale, bool dc, cudaStream_t s,
                            int row0, int nrows_run, const CUtensorMap *tm, unsigned int *tflag, int tile_rows)
{
    const bool f64 = sizeof(R) == 8;
    const int rpc = row_rpc(nphi, f64);
    if (nrows_run < 0) nrows_run = nrows - row0;
    dim3 grid(nrows_run / rpc, nsrc);
    if constexpr (sizeof(R) == 4 && SG_ROWS_FWD_TMA) {
        const bool aligned = ((uintptr_t)x0 & 15u) == 0 && ((uintptr_t)x1 & 15u) == 0;
        const int NR = tile_rows == 2 ? 2 : 4;
        // whole tiles, each starting on a 16-byte boundary of the map's rows
        if (tm && aligned && rows_tma_eligible(nrows, nphi, false) && nrows_run % NR == 0 && row0 % NR == 0) {
            const dim3 gt(nrows_run / NR, nsrc);
            auto go = [&](auto kern, int N, int ahead) {
                kern<<<gt, NR * N / 16, row_tma_smem_bytes(N, NR), s>>>(x0, x1, *tm, (const float2 *)tw_row,
                                                                        (const float2 *)twp_row, rscale, dc ? 1 : 0,
                                                                        tflag, row0, ahead);
            };
            if (NR == 2) {
                if (nphi == 4096) go(k_rows_fwd_tma<2048, 2>, 2048, fwd_resident_ctas<2048, 2>());
                else if (nphi == 2048) go(k_rows_fwd_tma<1024, 2>, 1024, fwd_resident_ctas<1024, 2>());
                else if (nphi == 1024) go(k_rows_fwd_tma<512, 2>, 512, fwd_resident_ctas<512, 2>());
                else go(k_rows_fwd_tma<256, 2>, 256, fwd_resident_ctas<256, 2>());
            } else {
                if (nphi == 4096) go(k_rows_fwd_tma<2048, 4>, 2048, fwd_resident_ctas<2048, 4>());
                else if (nphi == 2048) go(k_rows_fwd_tma<1024, 4>, 1024, fwd_resident_ctas<1024, 4>());
                else if (nphi == 1024) go(k_rows_fwd_tma<512, 4>, 512, fwd_resident_ctas<512, 4>());
                else go(k_rows_fwd_tma<256, 4>, 256, fwd_resident_ctas<256, 4>());
            }
            return cudaGetLastError();
        }
    }
    auto go = [&](auto kern) {
        kern<<<grid, (nphi / 32) * rpc, row_smem_bytes(nphi, rpc, f64), s>>>(
            x0, x1, (cplx<R> *)xh, nrows, nphi, rpc, (const cplx<R> *)tw_row, (const cplx<R> *)twp_row, rscale,
            dc ? 1 : 0, row0);
    };
    if (!f64 && nphi == 4096) go(k_rows_fwd<R, 2048>);
    else if (!f64 && nphi == 2048) go(k_rows_fwd<R, 1024>);
    else go(k_rows_fwd<R, 0>);
    return cudaGetLastError();
}


// ------------------------------------------------------- row C2R + epilogue
template <typename R, int NC>
__global__ void __launch_bounds__(1024, 1)
k_rows_inv(const cplx<R> *__restrict__ oh, const __grid_constant__ RowOut o, int nrows, int nphi_rt, int rpc,
           const cplx<R> *__restrict__ tw, const cplx<R> *__restrict__ twp, const R *__restrict__ rcen,
           unsigned int *flag, int row0)
{
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw + 64 * sizeof(double));
    const int nphi = NC > 0 ? 2 * NC : nphi_rt;
    const int N = nphi >> 1, T = N >> 4;
    if (NC > 0) rpc = row_rpc_of(2 * NC, sizeof(C));           // compile-time for the hot lengths
    const int lg = ilog2(rpc);
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    const int q = blockIdx.y;
    const int i0 = row0 + blockIdx.x * rpc;
    const C *src = oh + (size_t)o.src[q] * N * nrows;
    griddep_wait();                       // the column pass's output is complete from here on
    // FAST: as in k_rows_fwd, per-thread bases plus compile-time offsets
    constexpr bool FAST = NC >= 256 && BW == 1 && row_rpc_of(2 * NC, sizeof(C)) == 4;
    const uint64_t pf = l2_evict_first();
    if constexpr (FAST) {
        // copy step j: column m = (x >> 2) + j nthr / 4, row gg = x & 3; all 16 loads first
        constexpr int nthr = (NC / 16) * 4;
        const int x = threadIdx.x, gg = x & 3, m0 = x >> 2;
        const C *s0 = src + (size_t)m0 * nrows + i0 + gg;
        C tmp[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) tmp[j] = ld_cg_hint(s0 + (size_t)j * (nthr / 4) * nrows, pf);
        const int sb0 = 4 * m0 + (gg ^ ((m0 >> 2) & 3));
#pragma unroll
        for (int j = 0; j < 16; ++j) sm[sb0 + j * nthr] = tmp[j];
    } else {
        // every thread copies exactly N rpc / blockDim = 16 elements: issue
        // all 16 loads before the first shared-memory store
        const int per = rpc * BW;
        C tmp[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int idx = threadIdx.x + j * blockDim.x;
            const int bb = idx / per, rem = idx - bb * per;
            const int gg = rem / BW, c = rem - gg * BW;
            tmp[j] = ld_cg_hint(src + ((size_t)bb * nrows + i0 + gg) * BW + c, pf);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int idx = threadIdx.x + j * blockDim.x;
            const int bb = idx / per, rem = idx - bb * per;
            const int gg = rem / BW, c = rem - gg * BW;
            sm[tile_idx_g<C>(bb * BW + c, gg, lg)] = tmp[j];
        }
    }
    __syncthreads();
    // Z'[k] = (X[k] + X*[N-k]) + i (X[k] - X*[N-k]) W^-k  (= 2 Z[k])
    // FAST: tile_idx_g(k, g, 2) = 4 k + (g ^ ((t >> 2) & 3)) and
    // tile_idx_g(N - k, g, 2) = 4 (N - k) + (g ^ (((-t) >> 2) & 3)) for k = t + T e
    const int xa0 = 4 * t + (g ^ ((t >> 2) & 3));
    const int xc0 = 4 * (N - t) + (g ^ (((-t) >> 2) & 3));
    C v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int k = t + T * e;
        const C X = sm[FAST ? xa0 + 4 * T * e : tile_idx_g<C>(k, g, lg)];
        if (e == 0 && t == 0) {
            v[e] = mkc<C>(X.x + X.y, X.x - X.y);
        } else {
            const C Xc = cconj(sm[FAST ? xc0 - 4 * T * e : tile_idx_g<C>(N - k, g, lg)]);
            v[e] = cadd(cadd(X, Xc), cmul_i(cmulc(csub(X, Xc), __ldg(&tw[k]))));
        }
    }
    // the transform's exchange buffer overlays the tile; fft_reg
    // synchronises before its first shared-memory write
    fft_any<false, NC>(v, N, T, t, sm + g * padded_len(N), twp);
    const int i = i0 + g;
    // undo the radial source scaling: accelerations / r_i; the potential's
    // own r_i prefactor cancels it
    const R sc = o.is_phi[q] ? (R)1 : (R)1 / rcen[i];
    C *out = reinterpret_cast<C *>(reinterpret_cast<R *>(o.ptr[q]) + (size_t)i * nphi);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        v[e] = mkc<C>(v[e].x * sc, v[e].y * sc);   // (y[2n], y[2n+1])
#if SG_ROWS_INV_STREAM
        __stcs(&out[t + T * e], v[e]);
#else
        out[t + T * e] = v[e];
#endif
    }
    if (flag) {
        bool bad = false;
#pragma unroll
        for (int e = 0; e < 16; ++e) bad |= !(isfinite(v[e].x) && isfinite(v[e].y));
        if (bad) atomicOr(flag, 1u);
    }
}

template <int NC, int NR>
__global__ void __launch_bounds__(rows_tma_threads(NC, NR), rows_tma_min_blocks(NC, NR, SG_ROWS_INV_SM_THREADS))
k_rows_inv_tma(const __grid_constant__ CUtensorMap tm, const __grid_constant__ RowOut o, const float2 *__restrict__ tw,
               const float2 *__restrict__ twp, const float *__restrict__ rcen, unsigned int *flag,
               unsigned int *tflag, int row0)
{
    static_assert(NR == 2 || NR == 4, "the tensor-copy row transforms take 2 or 4 rows per CTA");
    constexpr int N = NC, T = N / 16, PLS = row_pitch_tma(N, NR);
    extern __shared__ __align__(1024) unsigned char smem_tma[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_tma);
    float2 *reg = reinterpret_cast<float2 *>(smem_tma + kRowHdr);
    if (smem_u32(reg) & 127u) {                                         // TMA alignment (never expected)
        if (threadIdx.x == 0 && tflag) atomicOr(tflag, 2u);
        return;
    }
    const int q = blockIdx.y, i0 = row0 + blockIdx.x * NR;
    const int lane = threadIdx.x & 31, g = lane & (NR - 1), t = (threadIdx.x >> 5) * (32 / NR) + lane / NR;
    // plan constants, loaded while the tile is in flight
    const float2 w0 = __ldg(&tw[t]);
    const float sc = o.is_phi[q] ? 1.f : 1.f / __ldg(&rcen[i0 + g]);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    griddep_wait();                       // the column pass's output is complete from here on
    if (threadIdx.x == 0) {
        // the column pass's output is read for the last time
        const uint64_t pf = l2_evict_first();
        mbar_expect_tx(bar, (unsigned)N * 8u * NR);
#pragma unroll
        for (int b = 0; b < N / 256; ++b) tma_load_2d(reg + NR * 256 * b, &tm, 2 * i0, o.src[q] * N + 256 * b, bar, pf);
    }
    if (!__syncthreads_and(mbar_wait_bounded(bar, 0, tflag))) return;
    // Z'[k] = (X[k] + X*[N-k]) + i (X[k] - X*[N-k]) W^-k  (= 2 Z[k])
    const float2 *xa = reg + NR * t + g, *xc = reg + NR * (N - t) + g;
    float2 v[16];
    unroll16<0>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        const float2 X = xa[NR * T * e];
        if (e == 0 && t == 0) {
            v[e] = make_float2(X.x + X.y, X.x - X.y);
        } else {
            const float2 Xc = cconj(xc[-NR * T * e]);
            v[e] = cadd(cadd(X, Xc), cmul_i(cmulc(csub(X, Xc), tw_step<e>(w0))));
        }
    });
    // the exchange buffers overlay the tile; the transform synchronises
    // before its first shared-memory write
    fft_ct<false, N>(v, t, reg + g * PLS, twp);
    const int i = i0 + g;
    float2 *out = reinterpret_cast<float2 *>(reinterpret_cast<float *>(o.ptr[q]) + (size_t)i * 2 * N);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        v[e] = make_float2(v[e].x * sc, v[e].y * sc);     // (y[2n], y[2n+1])
#if SG_ROWS_INV_STREAM
        __stcs(&out[t + T * e], v[e]);
#else
        out[t + T * e] = v[e];
#endif
    }
    if (flag) {
        bool bad = false;
#pragma unroll
        for (int e = 0; e < 16; ++e) bad |= !(isfinite(v[e].x) && isfinite(v[e].y));
        if (bad) atomicOr(flag, 1u);
    }
}

// Tensor map of a [ncols][nr] complex FP32 intermediate (element (m, i) at
// m nr + i) as a 2-D FP32 array [ncols][2 nr], box 2 rows x 256: a row
// transform CTA's `rows` rows of 256 columns.  The driver's encoder is reached through the runtime's entry-point
// query, so the library needs no link against the driver library.
cudaError_t encode_row_map(CUtensorMap *m, void *base, int nr, long long ncols, int rows)
{
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Encode>(p);
    });
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)2 * nr, (cuuint64_t)ncols};
    const cuuint64_t strides[1] = {(cuuint64_t)nr * 8};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * rows), 256}, es[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool rows_tma_eligible(int nr, int nphi, bool f64)
{
    return !f64 && BW == 1 && (nphi == 512 || nphi == 1024 || nphi == 2048 || nphi == 4096) && nr % 4 == 0;
}

template <typename R>
cudaError_t launch_rows_inv(const void *oh, const RowOut &o, int nr, int nphi, const void *tw_row,
                            const void *twp_row, const R *rcen, unsigned int *flag, cudaStream_t s, int row0,
                            int nrows_run, const CUtensorMap *tm, unsigned int *tflag, bool pdl, int tile_rows)
{
    cudaError_t err = cudaSuccess;
    const bool f64 = sizeof(R) == 8;
    const int rpc = row_rpc(nphi, f64);
    if (nrows_run < 0) nrows_run = nr - row0;
    dim3 grid(nrows_run / rpc, o.n);
    if constexpr (sizeof(R) == 4) {
        const int NR = tile_rows == 4 ? 4 : 2;
        if (tm && rows_tma_eligible(nr, nphi, false) && nrows_run % NR == 0 && row0 % NR == 0) {
            const dim3 gt(nrows_run / NR, o.n);
            auto go = [&](auto kern, int N) {
                err = launch_ex(kern, gt, dim3(NR * N / 16), row_tma_smem_bytes(N, NR), s, pdl, *tm, o,
                                (const float2 *)tw_row, (const float2 *)twp_row, rcen, flag, tflag, row0);
            };
            if (NR == 2) {
                if (nphi == 4096) go(k_rows_inv_tma<2048, 2>, 2048);
                else if (nphi == 2048) go(k_rows_inv_tma<1024, 2>, 1024);
                else if (nphi == 1024) go(k_rows_inv_tma<512, 2>, 512);
                else go(k_rows_inv_tma<256, 2>, 256);
            } else {
                if (nphi == 4096) go(k_rows_inv_tma<2048, 4>, 2048);
                else if (nphi == 2048) go(k_rows_inv_tma<1024, 4>, 1024);
                else if (nphi == 1024) go(k_rows_inv_tma<512, 4>, 512);
                else go(k_rows_inv_tma<256, 4>, 256);
            }
            return err != cudaSuccess ? err : cudaGetLastError();
        }
    }
    auto go = [&](auto kern) {
        err = launch_ex(kern, grid, dim3((nphi / 32) * rpc), row_smem_bytes(nphi, rpc, f64), s, pdl,
                        (const cplx<R> *)oh, o, nr, nphi, rpc, (const cplx<R> *)tw_row, (const cplx<R> *)twp_row, rcen,
                        flag, row0);
    };
    if (!f64 && nphi == 4096) go(k_rows_inv<R, 2048>);
    else if (!f64 && nphi == 2048) go(k_rows_inv<R, 1024>);
    else go(k_rows_inv<R, 0>);
    return err != cudaSuccess ? err : cudaGetLastError();
}

cudaError_t set_row_smem_limits(int max_optin)
{
    const void *fns[] = {(const void *)k_rows_fwd<float, 0>,      (const void *)k_rows_fwd<float, 2048>,
                         (const void *)k_rows_fwd<float, 1024>,   (const void *)k_rows_fwd<double, 0>,
                         (const void *)k_rows_inv<float, 0>,      (const void *)k_rows_inv<float, 2048>,
                         (const void *)k_rows_inv<float, 1024>,   (const void *)k_rows_inv<double, 0>,
                         (const void *)k_rows_fwd_tma<2048, 4>,   (const void *)k_rows_fwd_tma<1024, 4>,
                         (const void *)k_rows_fwd_tma<512, 4>,    (const void *)k_rows_fwd_tma<256, 4>,
                         (const void *)k_rows_fwd_tma<2048, 2>,   (const void *)k_rows_fwd_tma<1024, 2>,
                         (const void *)k_rows_fwd_tma<512, 2>,    (const void *)k_rows_fwd_tma<256, 2>,
                         (const void *)k_rows_inv_tma<2048, 2>,   (const void *)k_rows_inv_tma<1024, 2>,
                         (const void *)k_rows_inv_tma<512, 2>,    (const void *)k_rows_inv_tma<256, 2>,
                         (const void *)k_rows_inv_tma<2048, 4>,   (const void *)k_rows_inv_tma<1024, 4>,
                         (const void *)k_rows_inv_tma<512, 4>,    (const void *)k_rows_inv_tma<256, 4>};
    for (const void *fn : fns) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t launch_rows_fwd<float>(const float *, const float *, int, void *, int, int, const void *,
                                            const void *, const float *, bool, cudaStream_t, int, int,
                                            const CUtensorMap *, unsigned int *, int);
template cudaError_t launch_rows_fwd<double>(const double *, const double *, int, void *, int, int, const void *,
                                             const void *, const double *, bool, cudaStream_t, int, int,
                                             const CUtensorMap *, unsigned int *, int);
template cudaError_t launch_rows_inv<float>(const void *, const RowOut &, int, int, const void *, const void *,
                                            const float *, unsigned int *, cudaStream_t, int, int,
                                            const CUtensorMap *, unsigned int *, bool, int);
template cudaError_t launch_rows_inv<double>(const void *, const RowOut &, int, int, const void *, const void *,
                                             const double *, unsigned int *, cudaStream_t, int, int,
                                             const CUtensorMap *, unsigned int *, bool, int);

}  // namespace sg
