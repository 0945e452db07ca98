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
#include "sg_launch.h"
#include "sg_mem.cuh"

namespace sg {



bool cols_staging_steps(int nr, int nsrc, bool f64, int staging)
{
    return staging < 0 ? cols_steps_default(nsrc, f64, 2 * nr) : staging != 0 && !f64;
}

size_t col_smem_bytes(int nr, int nsrc, bool f64, int staging)
{
    const size_t esz = f64 ? 16 : 8;
    const int L = 2 * nr;
    const size_t xb = align16((size_t)padded_len(L) * esz);
    // per step: one (target, component) step of kernel spectra staged at a
    // time, source spectra in registers, column 0 recomputed per step
    if (cols_staging_steps(nr, nsrc, f64, staging)) return 16 + xb + (size_t)nsrc * tab_pitch(nr) * esz;
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

// All-at-once column kernel of a plan shape (ST = 0; per-step kernels in
// sg_cols_steps.cu).
template <typename R>
using ColsKernel = void (*)(const cplx<R> *, const cplx<R> *, cplx<R> *, int, int, uint32_t, const cplx<R> *,
                            unsigned int *, int);
template <typename R>
ColsKernel<R> cols_kernel_all(int nsrc, int L)
{
    const bool f64 = sizeof(R) == 8;
    if (nsrc == 1) {
        if (!f64 && L == 4096) return k_cols<R, 1, 4096, false>;
        if (!f64 && L == 2048) return k_cols<R, 1, 2048, false>;
        if (!f64 && L == 1024) return k_cols<R, 1, 1024, false>;
        if (!f64 && L == 512) return k_cols<R, 1, 512, false>;
        if (!f64 && L == 256) return k_cols<R, 1, 256, false>;
        return k_cols<R, 1, 0, false>;
    }
    if (!f64 && L == 4096) return k_cols<R, 2, 4096, false>;
    if (!f64 && L == 2048) return k_cols<R, 2, 2048, false>;
    if (!f64 && L == 1024) return k_cols<R, 2, 1024, false>;
    if (!f64 && L == 512) return k_cols<R, 2, 512, false>;
    if (!f64 && L == 256) return k_cols<R, 2, 256, false>;
    return k_cols<R, 2, 0, false>;
}

template <typename R>
cudaError_t launch_cols(const void *sh, const void *tab, void *oh, int nr, int nphi, int nsrc,
                        uint32_t outmask, const void *tw_col, unsigned int *flag, cudaStream_t s, int ncols, bool pdl,
                        bool discard, int staging)
{
    const bool f64 = sizeof(R) == 8;
    const int N = nphi / 2, T = (2 * nr) / 16;
    const bool steps = cols_staging_steps(nr, nsrc, f64, staging);
    const size_t smem = col_smem_bytes(nr, nsrc, f64, steps ? 1 : 0);
    const int grid = ncols > 0 && ncols < N ? ncols : N;
    // whole 128-byte lines per source column (column 0 is read more than once
    // by its CTA and never discarded)
    const bool dc = discard && BW == 1 && ((size_t)nr * 2 * sizeof(R)) % 128 == 0 && ((uintptr_t)sh & 127u) == 0;
    ColsKernel<R> kern;
    if constexpr (sizeof(R) == 4) kern = steps ? cols_kernel_steps(nsrc, 2 * nr) : cols_kernel_all<R>(nsrc, 2 * nr);
    else kern = cols_kernel_all<R>(nsrc, 2 * nr);
    const cudaError_t err = launch_ex(kern, dim3(grid), dim3(T), smem, s, pdl, (const cplx<R> *)sh,
                                      (const cplx<R> *)tab, (cplx<R> *)oh, nr, N, outmask,
                                      (const cplx<R> *)tw_col, flag, dc ? 1 : 0);
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

// Raise every kernel's dynamic shared-memory limit to the device maximum
// (the launch's own request still sets the occupancy), so plans of any size
// can share the kernels.
cudaError_t set_smem_limits(int max_optin)
{
    const void *fns[] = {(const void *)k_cols<float, 1, 0, false>,    (const void *)k_cols<float, 1, 4096, false>,
                         (const void *)k_cols<float, 1, 2048, false>, (const void *)k_cols<float, 1, 1024, false>,
                         (const void *)k_cols<float, 1, 512, false>,  (const void *)k_cols<float, 1, 256, false>,
                         (const void *)k_cols<float, 2, 0, false>,    (const void *)k_cols<float, 2, 4096, false>,
                         (const void *)k_cols<float, 2, 2048, false>, (const void *)k_cols<float, 2, 1024, false>,
                         (const void *)k_cols<float, 2, 512, false>,  (const void *)k_cols<float, 2, 256, false>,
                         (const void *)k_cols<double, 1, 0, false>,   (const void *)k_cols<double, 2, 0, false>,
                         (const void *)k_tabcols<float>,              (const void *)k_tabcols<double>};
    for (const void *fn : fns) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = set_cols_steps_smem_limits(max_optin);
    return e != cudaSuccess ? e : set_row_smem_limits(max_optin);
}

template cudaError_t launch_cols<float>(const void *, const void *, void *, int, int, int, uint32_t, const void *,
                                        unsigned int *, cudaStream_t, int, bool, bool, int);
template cudaError_t launch_cols<double>(const void *, const void *, void *, int, int, int, uint32_t, const void *,
                                         unsigned int *, cudaStream_t, int, bool, bool, int);
template cudaError_t launch_tabcols<float>(const void *, void *, int, int, bool, const void *, cudaStream_t);
template cudaError_t launch_tabcols<double>(const void *, void *, int, int, bool, const void *, cudaStream_t);
}  // namespace sg
