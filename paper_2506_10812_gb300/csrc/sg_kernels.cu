// FFT-convolution path of the thin-disc self-gravity solver (Sec. 5.2 and
// App. C of Rendon Restrepo et al. 2025) for sm_103a.
//
// Data flow of one solve (constant aspect ratios, nr x nphi grid, L = 2 nr,
// N = nphi / 2, H = nr):
//   rows_fwd  each source Sigma_a [nr][nphi], scaled by r_i (see below) and
//             with its row mean removed -> row R2C (length nphi) -> packed
//             spectra (column m = 0 holds the real m = 0 and m = nphi/2
//             coefficients as re + i im) stored column-major;
//   cols      per column m: zero-padded length-L forward FFT of every
//             source, products with the kernel spectra (staged in shared
//             memory by TMA bulk copies, all at kernel start or one
//             (target, component) step at a time) summed over sources (Sec.
//             5.2 multi-fluid sums), inverse FFT of every requested (target,
//             component), rows 0..nr-1 written back;
//   rows_inv  per output row: packed C2R (length nphi) and the epilogue.
// The column pass and the inverse rows launch as programmatic dependents of
// the kernel before them (launch_ex; griddep_wait before reading its output).
//
// Layout of the [N][rows] intermediates (sg_mem.cuh, BW = 1): column-major,
// element (m, i) at m rows + i, so the column pass moves contiguous columns
// and a row transform that owns 2 or 4 consecutive rows moves a 16- or
// 32-byte slice of every column.  (The column-blocked variant BW = 4, element (m, i) at
// ((m / 4) rows + i) 4 + m % 4, gives the row transforms whole 128-byte
// lines but makes every column access a stride-4 vector; on the 2048 x 4096
// disc it makes the column pass 44 % slower and the row transforms 14 %
// faster.)
//
// Radial scaling: the lattice kernels carry e^{-3 Delta / 2}, which makes
// the convolution output span (r_out / r_in)^{3/2} across the grid while
// FP32 FFT rounding is uniform in absolute terms.  With
// e^{-alpha Delta} = (r' / r)^alpha the convolution is rewritten exactly as
//     sum_i' Sigma(i') K(i - i') = r_i^-alpha sum_i' [Sigma(i') r_i'^alpha] [e^{alpha Delta} K](i - i'),
// alpha = 1: the sources are multiplied by r_i' in rows_fwd, the kernel
// tables by e^Delta, and the accelerations by 1/r_i in rows_inv (the
// potential's own r_i prefactor cancels the 1/r_i).  Removing each row's
// mean before the row FFT (and adding nphi * mean back to the m = 0
// coefficient) is exact by linearity and keeps the small m != 0 modes of a
// nearly axisymmetric disc from inheriting the rounding of the mean.
//
// The kernel spectra (built once per plan by tab_eval -> rows_fwd<double>
// -> tabcols) already carry -G du dphi / (L nphi), the FFT normalisation.
#include <math.h>
#include <stdint.h>

#include <mutex>
#include <type_traits>
#include <utility>

#include "sg_bessel.cuh"
#include "sg_cols.cuh"
#include "sg_fft.cuh"
#include "sg_internal.h"
#include "sg_mem.cuh"

namespace sg {


// Launch with the programmatic-stream-serialization attribute when pdl:
// the kernel may then start before its predecessor on the stream finishes,
// and must call griddep_wait before reading anything that predecessor
// writes, and read it coherently (ld_cg_hint or TMA, never the
// non-coherent path, which presumes data fixed for the kernel's lifetime).
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                      Args &&...args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

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

__host__ __device__ static inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Kernel spectra staged one (target, component) step at a time (cols_pair_steps):
// every FP32 gas + dust plan, and FP32 gas-only columns of length 4096, which
// then fit 80 registers and run 3 CTAs of 256 threads per SM instead of 2
// (column pass 74.4 -> 70.2 us on the 2048 x 4096 disc).  At length 2048 (1.1
// waves of 6 CTAs per SM) the exposed per-step copy waits made it slower
// (22.3 -> 28.7 us), so those columns keep all three tables staged at once.
#ifndef SG_COLS_GAS_STEPS
#define SG_COLS_GAS_STEPS 1
#endif
__host__ __device__ constexpr bool cols_steps(int nsrc, bool f64, int L)
{
    return !f64 && (nsrc == 2 || (SG_COLS_GAS_STEPS && nsrc == 1 && L == 4096));
}
// launch bounds of k_cols<R, NS, LC>: 768 threads per SM for the staged
// gas-only lengths, otherwise up to 512 threads (128 registers each)
constexpr int cols_max_threads(int ns, bool f64, int lc)
{
    return ns == 1 && cols_steps(1, f64, lc) ? lc / 16 : 512;
}
constexpr int cols_min_blocks(int ns, bool f64, int lc)
{
    return ns == 1 && cols_steps(1, f64, lc) ? 768 / (lc / 16) : 1;
}

size_t col_smem_bytes(int nr, int nsrc, bool f64)
{
    const size_t esz = f64 ? 16 : 8;
    const int L = 2 * nr;
    const size_t xb = align16((size_t)padded_len(L) * esz);
    // FP32 gas + dust: one (target, component) step of kernel spectra staged
    // at a time, source spectra in registers, column 0 recomputed per step
    if (cols_steps(nsrc, f64, L)) return 16 + xb + (size_t)nsrc * tab_pitch(nr) * esz;
    const size_t tb = (size_t)nsrc * 3 * tab_pitch(nr) * esz;
    const size_t spec = nsrc == 2 ? (size_t)2 * L * esz : 0;   // gas + dust spectra live in shared memory
    // column 0 keeps its source spectra in the table area instead
    const size_t col0 = (size_t)nsrc * L * esz;
    return 16 + xb + (tb > col0 ? tb : col0) + spec;
}

size_t tabcol_smem_bytes(int L, bool) { return (size_t)padded_len(L) * 16; }

// ----------------------------------------------------------- kernel table
__global__ void __launch_bounds__(256)
k_tab_eval(int nr, int nphi, double du, double ha, double hb, double scale, double alpha, int mixed,
           double *p0, double *p1, double *p2, float *q0, float *q1, float *q2)
{
    __shared__ BesselWeights bw;
    bessel_weights_init(bw);
    __syncthreads();
    const int L = 2 * nr;
    const size_t n = (size_t)L * nphi;
    const double inv_sqrt_pi = 0.56418958354775628695;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx / nphi), j = (int)(idx - (size_t)k * nphi);
        const int di = (k < nr) ? k : k - L;
        // exact evenness / oddness in psi: evaluate at min(j, nphi - j)
        const int jj = (2 * j <= nphi) ? j : nphi - j;
        const double sgn = (2 * j <= nphi) ? 1.0 : -1.0;
        double vP = 0.0, vR = 0.0, vA = 0.0;
        if (k != nr && !(di == 0 && j == 0)) {
            const double Dl = di * du;                       // Delta = u - u'
            const double sh = sinh(0.5 * Dl);
            const double sp = sinpi((double)jj / nphi);       // sin(psi / 2)
            const double sp2 = sp * sp;
            const double hab2 = 0.5 * (ha * ha * exp(-Dl) + hb * hb * exp(Dl));
            const double X = 0.5 * (sh * sh + sp2) / hab2;    // d^2 / 8
            double k0e, Dx;
            const bool near = (di >= -1 && di <= 1 && jj <= 1);
            if (!mixed || X < 1.0 || near) {
                k0e_D_f64(X, bw, k0e, Dx);
            } else {
                float a, b;
                k0e_D_f32((float)X, bw, a, b);
                k0e = a;
                Dx = b;
            }
            const double hab = sqrt(hab2);
            const double e32 = scale * exp((alpha - 1.5) * Dl);
            vP = e32 * k0e * (0.5 * inv_sqrt_pi) / hab;
            const double c = e32 * Dx * (0.125 * inv_sqrt_pi) / (hab2 * hab);
            vR = c * (expm1(Dl) + 2.0 * sp2);
            vA = c * sgn * sinpi(2.0 * jj / nphi);
        }
        if (p0) p0[idx] = vP;
        if (p1) p1[idx] = vR;
        if (p2) p2[idx] = vA;
        if (q0) q0[idx] = (float)vP;
        if (q1) q1[idx] = (float)vR;
        if (q2) q2[idx] = (float)vA;
    }
}

cudaError_t launch_tab_eval(int nr, int nphi, double du, double ha, double hb, double scale,
                            double alpha, bool mixed, double *o64[3], float *o32[3], cudaStream_t s)
{
    const size_t n = (size_t)2 * nr * nphi;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_tab_eval<<<blocks, 256, 0, s>>>(nr, nphi, du, ha, hb, scale, alpha, mixed ? 1 : 0, o64[0], o64[1],
                                      o64[2], o32[0], o32[1], o32[2]);
    return cudaGetLastError();
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
// Rows per CTA: 4 for the forward transform, 2 for the inverse (2048 x 4096
// disc: the inverse 51.0 -> 45.3 us with 2, the forward 27.2 -> 30.6 us; a
// shared-memory floor holding the 2-row inverse to 3 CTAs per SM, 49.0 us).
#ifndef SG_ROWS_FWD_NR
#define SG_ROWS_FWD_NR 4
#endif
#ifndef SG_ROWS_INV_NR
#define SG_ROWS_INV_NR 2
#endif
constexpr int kRowsFwdNR = SG_ROWS_FWD_NR, kRowsInvNR = SG_ROWS_INV_NR;
static_assert((kRowsFwdNR == 2 || kRowsFwdNR == 4) && (kRowsInvNR == 2 || kRowsInvNR == 4),
              "the tensor-copy row transforms take 2 or 4 rows per CTA");
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
int rows_tma_fwd_rows() { return kRowsFwdNR; }
int rows_tma_inv_rows() { return kRowsInvNR; }
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

template <int NC>
__global__ void __launch_bounds__(rows_tma_threads(NC, kRowsFwdNR), rows_tma_min_blocks(NC, kRowsFwdNR, 1024))
k_rows_fwd_tma(const float *__restrict__ x0, const float *__restrict__ x1, const __grid_constant__ CUtensorMap tm,
               const float2 *__restrict__ tw, const float2 *__restrict__ twp, const float *__restrict__ rscale,
               int dc, unsigned int *tflag, int row0)
{
    constexpr int NR = kRowsFwdNR, N = NC, T = N / 16, NW = NR * T / 32, PLS = row_pitch_tma(N, NR), XS = T + T / 16;
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
                            int row0, int nrows_run, const CUtensorMap *tm, unsigned int *tflag)
{
    const bool f64 = sizeof(R) == 8;
    const int rpc = row_rpc(nphi, f64);
    if (nrows_run < 0) nrows_run = nrows - row0;
    dim3 grid(nrows_run / rpc, nsrc);
    if constexpr (sizeof(R) == 4 && SG_ROWS_FWD_TMA) {
        const bool aligned = ((uintptr_t)x0 & 15u) == 0 && ((uintptr_t)x1 & 15u) == 0;
        if (tm && aligned && rows_tma_eligible(nrows, nphi, false)) {
            const dim3 gt(nrows_run / kRowsFwdNR, nsrc);
            auto go = [&](auto kern, int N) {
                kern<<<gt, kRowsFwdNR * N / 16, row_tma_smem_bytes(N, kRowsFwdNR), s>>>(x0, x1, *tm, (const float2 *)tw_row,
                                                               (const float2 *)twp_row, rscale, dc ? 1 : 0, tflag,
                                                               row0);
            };
            if (nphi == 4096) go(k_rows_fwd_tma<2048>, 2048);
            else if (nphi == 2048) go(k_rows_fwd_tma<1024>, 1024);
            else if (nphi == 1024) go(k_rows_fwd_tma<512>, 512);
            else go(k_rows_fwd_tma<256>, 256);
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


// ---------------------------------------------------------- column pass
template <typename R, int NS, int LC>
__global__ void __launch_bounds__(cols_max_threads(NS, sizeof(R) == 8, LC), cols_min_blocks(NS, sizeof(R) == 8, LC))
k_cols(const cplx<R> *__restrict__ sh, const cplx<R> *__restrict__ tab, cplx<R> *__restrict__ oh, int nr_rt,
       int N, uint32_t outmask, const cplx<R> *__restrict__ tw, unsigned int *flag, int discard)
{
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    const int nr = LC > 0 ? LC / 2 : nr_rt;
    const int L = 2 * nr, T = L >> 4, H = nr, P = tab_pitch(nr);
    C *xb = reinterpret_cast<C *>(smem_raw + 16);
    C *tb = reinterpret_cast<C *>(smem_raw + 16 + align16((size_t)padded_len(L) * sizeof(C)));
    const int t = threadIdx.x, m = blockIdx.x;
    griddep_launch();                     // the inverse rows may set up once every column CTA runs
    constexpr bool PAIR = NS == 2 ? sizeof(R) == 4 : cols_steps(1, sizeof(R) == 8, LC);
    if (m == 0) {
        // column 0 keeps its source spectra in the table area (recomputed
        // per step for FP32 gas + dust)
        griddep_wait();
        if constexpr (PAIR) col0_recompute<R, NS>(sh, tab, oh, nr, N, outmask, tw, xb);
        else col0_path<R, NS>(sh, tab, oh, nr, N, outmask, tw, xb, tb);
        return;
    }
    if constexpr (PAIR) {
        cols_pair_steps<R, LC, NS>(sh, tab, oh, nr, N, outmask, tw, flag, xb, tb, bar, m, discard, RegEngine{});
        return;
    }
    C *sspec = tb + (size_t)NS * 3 * P;           // NS == 2: source spectra in shared memory

    // Stage the kernel spectra of target b (requested components only).
    auto issue = [&](int b) {
        if (t == 0) {
            const uint64_t pol = l2_evict_first();
            unsigned bytes = 0;
            for (int c = 0; c < 3; ++c)
                if ((outmask >> (3 * b + c)) & 1u) bytes += NS * P * sizeof(C);
            mbar_expect_tx(bar, bytes);
            int slot = 0;
            for (int c = 0; c < 3; ++c) {
                if (!((outmask >> (3 * b + c)) & 1u)) continue;
                for (int a = 0; a < NS; ++a, ++slot)
                    tma_load_1d(tb + (size_t)slot * P,
                                tab + ((size_t)((a * NS + b) * 3 + c) * (N + 1) + m) * P, P * sizeof(C), bar, pol);
            }
        }
    };
    if (t == 0) mbar_init(bar, 1);
    __syncthreads();
    issue(0);                                      // lands while the forward FFTs run
    griddep_wait();                                // the row spectra are complete from here on

    C v[16];
    C spec[NS == 1 ? 16 : 1];                      // NS == 1: source spectrum in registers
#pragma unroll 1
    for (int a = 0; a < NS; ++a) {
        const uint64_t pf = l2_evict_first();
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = ld_cg_hint(sh + (size_t)a * N * nr + blk(m, t + T * e, nr), pf);
#pragma unroll
        for (int e = 8; e < 16; ++e) v[e] = mkc<C>(0, 0);   // radial zero padding
        fft_any<true, LC>(v, L, T, t, xb, tw);
        // every thread's loads of this column were consumed before the
        // transform's first barrier: the column is dead
        if (discard) l2_discard_range(sh + (size_t)a * N * nr + blk(m, 0, nr), (size_t)nr * sizeof(C), t, T);
        if constexpr (NS == 1) {
#pragma unroll
            for (int e = 0; e < 16; ++e) spec[e] = v[e];
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) sspec[a * L + t + T * e] = v[e];
        }
    }
#pragma unroll 1
    for (int b = 0; b < NS; ++b) {
        if (b > 0) {
            // every read of the previous stage precedes the TMA rewrite
            __syncthreads();
            fence_proxy_async();
            issue(b);
        }
        const bool ok = mbar_wait_bounded(bar, (unsigned)(b & 1), flag);
        if (__syncthreads_or(!ok)) return;          // the copy never completed: give up on this column
        int slot = 0;
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            if (!((outmask >> (3 * b + c)) & 1u)) continue;
            const C *tcol = tb + (size_t)slot * NS * P;
            slot++;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int k = t + T * e;
                C acc = mkc<C>(0, 0);
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    C S = spec_at(tcol + a * P, k, H, e >= 8);
                    if (c == 2) S = cmul_mi(S);                   // K_phi spectrum = -i S
                    C Z;
                    if constexpr (NS == 1) Z = spec[e];
                    else Z = sspec[a * L + k];
                    acc = cfma(Z, S, acc);
                }
                v[e] = acc;
            }
            fft_any<false, LC>(v, L, T, t, xb, tw);
            C *o = oh + (size_t)(b * 3 + c) * N * nr;
            const uint64_t pl = l2_evict_last();
#pragma unroll
            for (int e = 0; e < 8; ++e) st_hint(o + blk(m, t + T * e, nr), v[e], pl);   // rows 0..nr-1 only
        }
    }
}

template <typename R>
cudaError_t launch_cols(const void *sh, const void *tab, void *oh, int nr, int nphi, int nsrc,
                        uint32_t outmask, const void *tw_col, unsigned int *flag, cudaStream_t s, int ncols, bool pdl,
                        bool discard)
{
    const bool f64 = sizeof(R) == 8;
    const int N = nphi / 2, T = (2 * nr) / 16;
    const size_t smem = col_smem_bytes(nr, nsrc, f64);
    const int grid = ncols > 0 && ncols < N ? ncols : N;
    // whole 128-byte lines per source column (column 0 is read more than once
    // by its CTA and never discarded)
    const bool dc = discard && BW == 1 && ((size_t)nr * 2 * sizeof(R)) % 128 == 0 && ((uintptr_t)sh & 127u) == 0;
    cudaError_t err = cudaSuccess;
    auto go = [&](auto kern) {
        err = launch_ex(kern, dim3(grid), dim3(T), smem, s, pdl, (const cplx<R> *)sh, (const cplx<R> *)tab,
                        (cplx<R> *)oh, nr, N, outmask, (const cplx<R> *)tw_col, flag, dc ? 1 : 0);
    };
    const int L = 2 * nr;
    if (nsrc == 1) {
        if (!f64 && L == 4096) go(k_cols<R, 1, 4096>);
        else if (!f64 && L == 2048) go(k_cols<R, 1, 2048>);
        else if (!f64 && L == 1024) go(k_cols<R, 1, 1024>);
        else if (!f64 && L == 512) go(k_cols<R, 1, 512>);
        else if (!f64 && L == 256) go(k_cols<R, 1, 256>);
        else go(k_cols<R, 1, 0>);
    } else {
        if (!f64 && L == 4096) go(k_cols<R, 2, 4096>);
        else if (!f64 && L == 2048) go(k_cols<R, 2, 2048>);
        else if (!f64 && L == 1024) go(k_cols<R, 2, 1024>);
        else if (!f64 && L == 512) go(k_cols<R, 2, 512>);
        else if (!f64 && L == 256) go(k_cols<R, 2, 256>);
        else go(k_cols<R, 2, 0>);
    }
    return err != cudaSuccess ? err : cudaGetLastError();
}

// ------------------------------------------- table column FFT + packing
// spec: [nphi/2][L] row spectra of one real table (FP64, sg_mem.cuh layout);
// tab: [nphi/2 + 1][P] kernel spectrum columns (slot k = S(k), 0 <= k <= H).
template <typename R>
__global__ void __launch_bounds__(512)
k_tabcols(const double2 *__restrict__ spec, cplx<R> *__restrict__ tab, int L, int N, int odd,
          const double2 *__restrict__ tw)
{
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *xb = reinterpret_cast<double2 *>(smem_raw);
    const int T = L >> 4, H = L >> 1, t = threadIdx.x, m = blockIdx.x;
    const int P = H + 2;
    double2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = spec[blk(m, t + T * e, L)];
    fft_reg<true>(v, L, T, t, xb, tw);
    // the spectrum goes back to the (now free) exchange buffer, padded index
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) xb[pidx(t + T * e)] = v[e];
    __syncthreads();
    auto sp = [&](int k) { return xb[pidx(k & (L - 1))]; };
    // stored spectrum S = i T for the odd (sin psi) component, T otherwise;
    // S(0) and S(H) are real by symmetry and stored with a zero imaginary part
    auto S = [&](double2 x) { return odd ? cmul_i(x) : x; };
    auto put = [&](C *col, int k, double2 x) {
        if (k == 0 || k == H) x.y = 0.0;
        col[k] = mkc<C>((R)x.x, (R)x.y);
    };
    for (int k = t; k <= H; k += T) {
        if (m != 0) {
            put(tab + (size_t)m * P, k, S(sp(k)));
        } else {
            // unpack columns 0 and nphi/2 from the packed column
            const double2 X = sp(k), Xn = cconj(sp(L - k));
            put(tab, k, S(cscale(cadd(X, Xn), 0.5)));
            put(tab + (size_t)N * P, k, S(cscale(cmul_mi(csub(X, Xn)), 0.5)));
        }
    }
    if (t == 0) {
        tab[(size_t)m * P + H + 1] = mkc<C>(0, 0);
        if (m == 0) tab[(size_t)N * P + H + 1] = mkc<C>(0, 0);
    }
}

template <typename R>
cudaError_t launch_tabcols(const void *spec, void *tab, int L, int nphi, bool odd,
                           const void *tw_col64, cudaStream_t s)
{
    const int N = nphi / 2;
    k_tabcols<R><<<N, L / 16, tabcol_smem_bytes(L, true), s>>>(
        (const double2 *)spec, (cplx<R> *)tab, L, N, odd ? 1 : 0, (const double2 *)tw_col64);
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
        out[t + T * e] = v[e];
    }
    if (flag) {
        bool bad = false;
#pragma unroll
        for (int e = 0; e < 16; ++e) bad |= !(isfinite(v[e].x) && isfinite(v[e].y));
        if (bad) atomicOr(flag, 1u);
    }
}

template <int NC>
__global__ void __launch_bounds__(rows_tma_threads(NC, kRowsInvNR),
                                  rows_tma_min_blocks(NC, kRowsInvNR, SG_ROWS_INV_SM_THREADS))
k_rows_inv_tma(const __grid_constant__ CUtensorMap tm, const __grid_constant__ RowOut o, const float2 *__restrict__ tw,
               const float2 *__restrict__ twp, const float *__restrict__ rcen, unsigned int *flag,
               unsigned int *tflag, int row0)
{
    constexpr int NR = kRowsInvNR, N = NC, T = N / 16, PLS = row_pitch_tma(N, NR);
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
        out[t + T * e] = v[e];
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
                            int nrows_run, const CUtensorMap *tm, unsigned int *tflag, bool pdl)
{
    cudaError_t err = cudaSuccess;
    const bool f64 = sizeof(R) == 8;
    const int rpc = row_rpc(nphi, f64);
    if (nrows_run < 0) nrows_run = nr - row0;
    dim3 grid(nrows_run / rpc, o.n);
    if constexpr (sizeof(R) == 4) {
        if (tm && rows_tma_eligible(nr, nphi, false)) {
            const dim3 gt(nrows_run / kRowsInvNR, o.n);
            auto go = [&](auto kern, int N) {
                err = launch_ex(kern, gt, dim3(kRowsInvNR * N / 16), row_tma_smem_bytes(N, kRowsInvNR), s, pdl, *tm,
                                o, (const float2 *)tw_row, (const float2 *)twp_row, rcen, flag, tflag, row0);
            };
            if (nphi == 4096) go(k_rows_inv_tma<2048>, 2048);
            else if (nphi == 2048) go(k_rows_inv_tma<1024>, 1024);
            else if (nphi == 1024) go(k_rows_inv_tma<512>, 512);
            else go(k_rows_inv_tma<256>, 256);
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

// Raise every kernel's dynamic shared-memory limit to the device maximum
// (the launch's own request still sets the occupancy), so plans of any size
// can share the kernels.
cudaError_t set_smem_limits(int max_optin)
{
    const void *fns[] = {(const void *)k_rows_fwd<float, 0>,      (const void *)k_rows_fwd<float, 2048>,
                         (const void *)k_rows_fwd<float, 1024>,   (const void *)k_rows_fwd<double, 0>,
                         (const void *)k_rows_inv<float, 0>,      (const void *)k_rows_inv<float, 2048>,
                         (const void *)k_rows_inv<float, 1024>,   (const void *)k_rows_inv<double, 0>,
                         (const void *)k_cols<float, 1, 0>,       (const void *)k_cols<float, 1, 4096>,
                         (const void *)k_cols<float, 1, 2048>,    (const void *)k_cols<float, 2, 0>,
                         (const void *)k_cols<float, 2, 4096>,    (const void *)k_cols<float, 2, 2048>,
                         (const void *)k_cols<double, 1, 0>,      (const void *)k_cols<double, 2, 0>,
                         (const void *)k_tabcols<float>,          (const void *)k_tabcols<double>,
                         (const void *)k_rows_fwd_tma<2048>,      (const void *)k_rows_fwd_tma<1024>,
                         (const void *)k_rows_inv_tma<2048>,      (const void *)k_rows_inv_tma<1024>,
                         (const void *)k_rows_fwd_tma<512>,       (const void *)k_rows_fwd_tma<256>,
                         (const void *)k_rows_inv_tma<512>,       (const void *)k_rows_inv_tma<256>,
                         (const void *)k_cols<float, 1, 1024>,    (const void *)k_cols<float, 1, 512>,
                         (const void *)k_cols<float, 1, 256>,     (const void *)k_cols<float, 2, 1024>,
                         (const void *)k_cols<float, 2, 512>,     (const void *)k_cols<float, 2, 256>};
    for (const void *fn : fns) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t launch_rows_fwd<float>(const float *, const float *, int, void *, int, int, const void *,
                                            const void *, const float *, bool, cudaStream_t, int, int,
                                            const CUtensorMap *, unsigned int *);
template cudaError_t launch_rows_fwd<double>(const double *, const double *, int, void *, int, int, const void *,
                                             const void *, const double *, bool, cudaStream_t, int, int,
                                             const CUtensorMap *, unsigned int *);
template cudaError_t launch_cols<float>(const void *, const void *, void *, int, int, int, uint32_t, const void *,
                                        unsigned int *, cudaStream_t, int, bool, bool);
template cudaError_t launch_cols<double>(const void *, const void *, void *, int, int, int, uint32_t, const void *,
                                         unsigned int *, cudaStream_t, int, bool, bool);
template cudaError_t launch_tabcols<float>(const void *, void *, int, int, bool, const void *, cudaStream_t);
template cudaError_t launch_tabcols<double>(const void *, void *, int, int, bool, const void *, cudaStream_t);
template cudaError_t launch_rows_inv<float>(const void *, const RowOut &, int, int, const void *, const void *,
                                            const float *, unsigned int *, cudaStream_t, int, int,
                                            const CUtensorMap *, unsigned int *, bool);
template cudaError_t launch_rows_inv<double>(const void *, const RowOut &, int, int, const void *, const void *,
                                             const double *, unsigned int *, cudaStream_t, int, int,
                                             const CUtensorMap *, unsigned int *, bool);

}  // namespace sg
