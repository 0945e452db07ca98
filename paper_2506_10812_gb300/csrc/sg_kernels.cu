// FFT-convolution path of the thin-disc self-gravity solver (Sec. 5.2 and
// App. C of Rendon Restrepo et al. 2025) for sm_103a.
//
// Data flow of one solve (constant aspect ratios, nr x nphi grid, L = 2 nr):
//   rows_fwd  each source Sigma_a [nr][nphi] -> row R2C (length nphi) ->
//             packed spectra written transposed, [nphi/2][nr] complex
//             (column m = 0 holds the real m = 0 and m = nphi/2 rows as
//             re + i im);
//   cols      per column m: zero-padded length-L forward FFT of every
//             source, products with the packed kernel spectra summed over
//             sources (Sec. 5.2 multi-fluid sums), inverse FFT of every
//             requested (target, component), rows 0..nr-1 written
//             [nphi/2][nr];
//   rows_inv  per output row: packed C2R (length nphi) and the epilogue
//             (Phi times r_i), written [nr][nphi].
// The kernel spectra (built once per plan by tab_eval -> rows_fwd<double>
// -> tabcols) already carry -G du dphi / (L nphi), the FFT normalisation.
#include <math.h>

#include "sg_bessel.cuh"
#include "sg_fft.cuh"
#include "sg_internal.h"

namespace sg {

// ----------------------------------------------------------------- sizes
int row_rpc(int nphi, bool f64)
{
    const int T = nphi / 32;                  // threads per row transform
    const size_t esz = f64 ? 16 : 8;
    int rpc = 4;
    while (rpc > 1 && (T * rpc > 512 || (size_t)rpc * padded_len(nphi / 2) * esz > 160 * 1024)) rpc >>= 1;
    return rpc;
}

size_t row_smem_bytes(int nphi, int rpc, bool f64)
{
    return (size_t)rpc * padded_len(nphi / 2) * (f64 ? 16 : 8);
}

size_t col_smem_bytes(int nr, int nsrc, bool f64)
{
    const int L = 2 * nr;
    return ((size_t)padded_len(L) + (size_t)nsrc * L) * (f64 ? 16 : 8);
}

size_t tabcol_smem_bytes(int L, bool) { return (size_t)padded_len(L) * 16; }

// Swizzled [N][rpc] transpose tile: conflict-free for both the per-row
// strided access (consecutive k, fixed row) and the chunked copy.
template <typename C>
__device__ __forceinline__ int tile_idx(int k, int g, int rpc)
{
    constexpr int per_wavefront = 128 / sizeof(C);       // 16 (float2) or 8 (double2)
    const int sh = __ffs(per_wavefront / rpc) - 1;        // log2(per_wavefront / rpc)
    return k * rpc + (g ^ ((k >> sh) & (rpc - 1)));
}

// ----------------------------------------------------------- kernel table
__global__ void __launch_bounds__(256)
k_tab_eval(int nr, int nphi, double du, double ha, double hb, double scale, int mixed,
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
            const double e32 = scale * exp(-1.5 * Dl);
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
                            bool mixed, double *o64[3], float *o32[3], cudaStream_t s)
{
    const size_t n = (size_t)2 * nr * nphi;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_tab_eval<<<blocks, 256, 0, s>>>(nr, nphi, du, ha, hb, scale, mixed ? 1 : 0, o64[0], o64[1],
                                      o64[2], o32[0], o32[1], o32[2]);
    return cudaGetLastError();
}

// ------------------------------------------------------------ row R2C
template <typename R>
__global__ void __launch_bounds__(512)
k_rows_fwd(const R *__restrict__ x0, const R *__restrict__ x1, cplx<R> *__restrict__ xh, int nrows,
           int nphi, int rpc, const cplx<R> *__restrict__ tw)
{
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    const int N = nphi >> 1, T = N >> 4;
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    const int a = blockIdx.y;
    const int i0 = blockIdx.x * rpc;
    const C *xr = reinterpret_cast<const C *>((a == 0 ? x0 : x1) + (size_t)(i0 + g) * nphi);
    C *xb = sm + g * padded_len(N);
    C v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = xr[t + T * e];    // z[n] = x[2n] + i x[2n+1]
    fft_reg<true>(v, N, T, t, xb, tw, 2);
    // X[k] = E[k] + W^k O[k], E = (Z[k] + Z*[N-k]) / 2, O = (Z[k] - Z*[N-k]) / 2i
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) xb[pidx(t + T * e)] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int k = t + T * e;
        const C Z = v[e];
        if (k == 0) {
            v[e] = mkc<C>(Z.x + Z.y, Z.x - Z.y);          // (X[0], X[nphi/2]) packed
        } else {
            const C Zc = cconj(xb[pidx(N - k)]);
            const C E = cscale(cadd(Z, Zc), (R)0.5);
            const C O = cscale(cmul_mi(csub(Z, Zc)), (R)0.5);
            v[e] = cadd(E, cmul(O, __ldg(&tw[k])));
        }
    }
    // transposed write through a [N][rpc] tile: rpc consecutive rows per m
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) sm[tile_idx<C>(t + T * e, g, rpc)] = v[e];
    __syncthreads();
    C *out = xh + (size_t)a * N * nrows + i0;
    for (int idx = threadIdx.x; idx < N * rpc; idx += blockDim.x) {
        const int k = idx / rpc, gg = idx - k * rpc;
        out[(size_t)k * nrows + gg] = sm[tile_idx<C>(k, gg, rpc)];
    }
}

template <typename R>
cudaError_t launch_rows_fwd(const R *x0, const R *x1, int nsrc, void *xh, int nrows, int nphi,
                            const void *tw_row, cudaStream_t s)
{
    const bool f64 = sizeof(R) == 8;
    const int rpc = row_rpc(nphi, f64);
    dim3 grid(nrows / rpc, nsrc);
    k_rows_fwd<R><<<grid, (nphi / 32) * rpc, row_smem_bytes(nphi, rpc, f64), s>>>(
        x0, x1, (cplx<R> *)xh, nrows, nphi, rpc, (const cplx<R> *)tw_row);
    return cudaGetLastError();
}

// ---------------------------------------------------- packed table access
// Packed Hermitian column: slot 0 = (S(0), S(H)), slot k = S(k) for 0<k<H;
// S(k) for k > H is conj(S(L - k)).  `upper`: k >= H.
template <typename C>
__device__ __forceinline__ C tab_at(const C *__restrict__ col, int k, int H, bool upper)
{
    const int idx = upper ? (2 * H - k) : k;
    const int id = idx & (H - 1);
    const C v = __ldg(&col[id]);
    if (id == 0) return mkc<C>(upper ? v.y : v.x, 0);
    return upper ? cconj(v) : v;
}

// --------------------------------------------------------- column pass
template <typename R, int NS>
__global__ void __launch_bounds__(512)
k_cols(const cplx<R> *__restrict__ sh, const cplx<R> *__restrict__ tab, cplx<R> *__restrict__ oh,
       int nr, int N, uint32_t outmask, const cplx<R> *__restrict__ tw)
{
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *xb = reinterpret_cast<C *>(smem_raw);
    const int L = 2 * nr, T = L >> 4, H = nr;
    const int t = threadIdx.x, m = blockIdx.x;
    C *spec = xb + padded_len(L);
    C v[16];
#pragma unroll 1
    for (int a = 0; a < NS; ++a) {
        const C *col = sh + ((size_t)a * N + m) * nr;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = col[t + T * e];
#pragma unroll
        for (int e = 8; e < 16; ++e) v[e] = mkc<C>(0, 0);   // radial zero padding
        fft_reg<true>(v, L, T, t, xb, tw, 1);
#pragma unroll
        for (int e = 0; e < 16; ++e) spec[a * L + t + T * e] = v[e];
    }
    __syncthreads();
#pragma unroll 1
    for (int b = 0; b < NS; ++b) {
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            if (!((outmask >> (3 * b + c)) & 1u)) continue;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int k = t + T * e;
                C acc = mkc<C>(0, 0);
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    const C *tc = tab + ((size_t)((a * NS + b) * 3 + c) * (N + 1)) * nr;
                    const C Z = spec[a * L + k];
                    if (m != 0) {
                        C S = tab_at(tc + (size_t)m * nr, k, H, e >= 8);
                        if (c == 2) S = cmul_mi(S);               // K_phi spectrum = -i S
                        acc = cfma(Z, S, acc);
                    } else {
                        // packed column: Z = A + iB with A, B the spectra of the
                        // real m = 0 and m = nphi/2 columns
                        const C Zm = cconj(spec[a * L + ((L - k) & (L - 1))]);
                        C S0 = tab_at(tc, k, H, e >= 8);
                        C SN = tab_at(tc + (size_t)N * nr, k, H, e >= 8);
                        if (c == 2) {
                            S0 = cmul_mi(S0);
                            SN = cmul_mi(SN);
                        }
                        acc = cadd(acc, cscale(cadd(cmul(cadd(Z, Zm), S0), cmul(csub(Z, Zm), SN)), (R)0.5));
                    }
                }
                v[e] = acc;
            }
            fft_reg<false>(v, L, T, t, xb, tw, 1);
            C *o = oh + ((size_t)(b * 3 + c) * N + m) * nr;
#pragma unroll
            for (int e = 0; e < 8; ++e) o[t + T * e] = v[e];       // rows 0..nr-1 only
        }
    }
}

template <typename R>
cudaError_t launch_cols(const void *sh, const void *tab, void *oh, int nr, int nphi, int nsrc,
                        uint32_t outmask, const void *tw_col, cudaStream_t s)
{
    const bool f64 = sizeof(R) == 8;
    const int N = nphi / 2, T = (2 * nr) / 16;
    const size_t smem = col_smem_bytes(nr, nsrc, f64);
    if (nsrc == 1)
        k_cols<R, 1><<<N, T, smem, s>>>((const cplx<R> *)sh, (const cplx<R> *)tab, (cplx<R> *)oh, nr, N,
                                       outmask, (const cplx<R> *)tw_col);
    else
        k_cols<R, 2><<<N, T, smem, s>>>((const cplx<R> *)sh, (const cplx<R> *)tab, (cplx<R> *)oh, nr, N,
                                       outmask, (const cplx<R> *)tw_col);
    return cudaGetLastError();
}

// ------------------------------------------- table column FFT + packing
template <typename R>
__global__ void __launch_bounds__(512)
k_tabcols(const double2 *__restrict__ spec, cplx<R> *__restrict__ tab, int L, int N, int odd,
          const double2 *__restrict__ tw)
{
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *xb = reinterpret_cast<double2 *>(smem_raw);
    const int T = L >> 4, H = L >> 1, t = threadIdx.x, m = blockIdx.x;
    double2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = spec[(size_t)m * L + t + T * e];
    fft_reg<true>(v, L, T, t, xb, tw, 1);
    // the spectrum goes back to the (now free) exchange buffer, padded index
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) xb[pidx(t + T * e)] = v[e];
    __syncthreads();
    auto sp = [&](int k) { return xb[pidx(k)]; };
    // stored spectrum S = i T for the odd (sin psi) component, T otherwise
    auto S = [&](double2 x) { return odd ? cmul_i(x) : x; };
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = t + T * e;
        if (m != 0) {
            double2 out = S(sp(k));
            if (k == 0) out = make_double2(out.x, S(sp(H)).x);
            tab[(size_t)m * H + k] = mkc<C>((R)out.x, (R)out.y);
        } else {
            // unpack columns 0 and nphi/2 from the packed column
            auto A = [&](int kk) {
                const double2 X = sp(kk), Xn = cconj(sp((L - kk) & (L - 1)));
                return cscale(cadd(X, Xn), 0.5);
            };
            auto B = [&](int kk) {
                const double2 X = sp(kk), Xn = cconj(sp((L - kk) & (L - 1)));
                return cscale(cmul_mi(csub(X, Xn)), 0.5);
            };
            double2 a = S(A(k)), b = S(B(k));
            if (k == 0) {
                a = make_double2(a.x, S(A(H)).x);
                b = make_double2(b.x, S(B(H)).x);
            }
            tab[k] = mkc<C>((R)a.x, (R)a.y);
            tab[(size_t)N * H + k] = mkc<C>((R)b.x, (R)b.y);
        }
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
template <typename R>
__global__ void __launch_bounds__(512)
k_rows_inv(const cplx<R> *__restrict__ oh, RowOut o, int nrows, int nphi, int rpc,
           const cplx<R> *__restrict__ tw, const R *__restrict__ rcen, unsigned int *flag)
{
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    const int N = nphi >> 1, T = N >> 4;
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    const int q = blockIdx.y;
    const int i0 = blockIdx.x * rpc;
    const C *src = oh + (size_t)o.src[q] * N * nrows + i0;
    for (int idx = threadIdx.x; idx < N * rpc; idx += blockDim.x) {
        const int k = idx / rpc, gg = idx - k * rpc;
        sm[tile_idx<C>(k, gg, rpc)] = src[(size_t)k * nrows + gg];
    }
    __syncthreads();
    // Z'[k] = (X[k] + X*[N-k]) + i (X[k] - X*[N-k]) W^-k  (= 2 Z[k])
    C v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int k = t + T * e;
        const C X = sm[tile_idx<C>(k, g, rpc)];
        if (k == 0) {
            v[e] = mkc<C>(X.x + X.y, X.x - X.y);
        } else {
            const C Xc = cconj(sm[tile_idx<C>(N - k, g, rpc)]);
            v[e] = cadd(cadd(X, Xc), cmul_i(cmulc(csub(X, Xc), __ldg(&tw[k]))));
        }
    }
    // the transform's exchange buffer overlays the tile; fft_reg
    // synchronises before its first shared-memory write
    fft_reg<false>(v, N, T, t, sm + g * padded_len(N), tw, 2);
    const int i = i0 + g;
    const R sc = o.is_phi[q] ? rcen[i] : (R)1;
    C *out = reinterpret_cast<C *>(reinterpret_cast<R *>(o.ptr[q]) + (size_t)i * nphi);
    bool bad = false;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const C y = mkc<C>(v[e].x * sc, v[e].y * sc);   // (y[2n], y[2n+1])
        bad |= !(isfinite(y.x) && isfinite(y.y));
        out[t + T * e] = y;
    }
    if (flag && bad) atomicOr(flag, 1u);
}

template <typename R>
cudaError_t launch_rows_inv(const void *oh, const RowOut &o, int nr, int nphi, const void *tw_row,
                            const R *rcen, unsigned int *flag, cudaStream_t s)
{
    const bool f64 = sizeof(R) == 8;
    const int rpc = row_rpc(nphi, f64);
    dim3 grid(nr / rpc, o.n);
    k_rows_inv<R><<<grid, (nphi / 32) * rpc, row_smem_bytes(nphi, rpc, f64), s>>>(
        (const cplx<R> *)oh, o, nr, nphi, rpc, (const cplx<R> *)tw_row, rcen, flag);
    return cudaGetLastError();
}

// Raise every kernel's dynamic shared-memory limit to the device maximum
// (the launch's own request still sets the occupancy), so plans of any size
// can share the kernels.
cudaError_t set_smem_limits(int max_optin)
{
    const void *fns[] = {(const void *)k_rows_fwd<float>,  (const void *)k_rows_fwd<double>,
                         (const void *)k_rows_inv<float>,  (const void *)k_rows_inv<double>,
                         (const void *)k_cols<float, 1>,   (const void *)k_cols<float, 2>,
                         (const void *)k_cols<double, 1>,  (const void *)k_cols<double, 2>,
                         (const void *)k_tabcols<float>,   (const void *)k_tabcols<double>};
    for (const void *fn : fns) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t launch_rows_fwd<float>(const float *, const float *, int, void *, int, int, const void *, cudaStream_t);
template cudaError_t launch_rows_fwd<double>(const double *, const double *, int, void *, int, int, const void *, cudaStream_t);
template cudaError_t launch_cols<float>(const void *, const void *, void *, int, int, int, uint32_t, const void *, cudaStream_t);
template cudaError_t launch_cols<double>(const void *, const void *, void *, int, int, int, uint32_t, const void *, cudaStream_t);
template cudaError_t launch_tabcols<float>(const void *, void *, int, int, bool, const void *, cudaStream_t);
template cudaError_t launch_tabcols<double>(const void *, void *, int, int, bool, const void *, cudaStream_t);
template cudaError_t launch_rows_inv<float>(const void *, const RowOut &, int, int, const void *, const float *, unsigned int *, cudaStream_t);
template cudaError_t launch_rows_inv<double>(const void *, const RowOut &, int, int, const void *, const double *, unsigned int *, cudaStream_t);

}  // namespace sg
