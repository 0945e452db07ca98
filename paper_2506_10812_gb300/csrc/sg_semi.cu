// Semi-spectral solve for axisymmetric scale heights: the route Sec. 5.2
// gives for a non-constant H/r, a Fourier transform along phi and a direct
// sum along r (cost n_r n_phi log n_phi + n_phi n_r^2).
//
// With H_a = H_a(r) the pair kernel of Sec. 2.2 (Eq. "SG force kernel
// exact", Eq. "mean root square height", Eq. "grav. potential 2D") depends on
// the two radii and on the angle difference only.  The direct sum
//     f_c(i, j) = sum_a sum_{i', j'} W^{ab}_c(i, i', j - j') Sigma_a(i', j')
// is then a circular convolution in phi for every radial pair, and with the
// phi-DFT (hats) it becomes one complex n_r x n_r matrix-vector product per
// azimuthal mode m:
//     f^_c(i, m) = sum_a sum_{i'} W^^{ab}_c(i, i', m) Sigma^_a(i', m).
// Per unit surface density (m_u = r'^2 du dphi, H^2 = (H_a(r')^2 + H_b(r)^2)/2,
// X = s^2 / (8 H^2), Delta = (i - i') du, psi = (j - j') dphi):
//     W_Phi = -G m_u e^X K0(X) / (2 sqrt(pi) H),
//     W_r   = -G m_u D(X) r' (expm1(Delta) + 2 sin^2(psi/2)) / (8 sqrt(pi) H^3),
//     W_phi = -G m_u D(X) r' sin psi / (8 sqrt(pi) H^3),
// and 0 for the self cell; the direct path's pair terms, so the result is
// the direct sum's.
//
// The plan stores W^ (FP64 kernel samples, FP64 row FFTs, rounded to the plan
// dtype) as [pair][component][n_phi/2][n_r][n_r] complex, slot m = 0 packing
// the real m = 0 and m = n_phi/2 matrices as re + i im like the row spectra.
// The entries carry the conventions of the row transforms around them: the
// forward rows multiply each source row by r_i', the inverse rows divide the
// accelerations by r_i, and the inverse is unnormalised (1 / n_phi).  A solve
// is rows_fwd, k_semi_mv (the tables streamed from HBM once), rows_inv.
#include <math.h>
#include <stdint.h>

#include <vector>

#include "sg_bessel.cuh"
#include "sg_fft.cuh"
#include "sg_internal.h"
#include "sg_mem.cuh"

namespace sg {

namespace {

// Kernel samples of target rows i0 .. i0 + ci - 1 against every source row,
// every lag: o_c[(il nr + i') nphi + dj], FP64.
__global__ void __launch_bounds__(256)
k_semi_eval(int nr, int nphi, int i0, int ci, const double *__restrict__ rc, const double *__restrict__ Ha,
            const double *__restrict__ Hb, double du, double dphi, double G, double *__restrict__ o_phi,
            double *__restrict__ o_r, double *__restrict__ o_a)
{
    __shared__ BesselWeights bw;
    bessel_weights_init(bw);
    __syncthreads();
    const double inv_sqrt_pi = 0.56418958354775628695;
    const size_t n = (size_t)ci * nr * nphi;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)(idx / nphi), dj = (int)(idx - (size_t)row * nphi);
        const int il = row / nr, ip = row - il * nr, i = i0 + il;
        double vP = 0.0, vR = 0.0, vA = 0.0;
        if (!(i == ip && dj == 0)) {
            const double r = rc[i], rp = rc[ip];
            const double Dl = (i - ip) * du;
            const double sh = sinh(0.5 * Dl);
            const double sp = sinpi((double)dj / nphi);               // sin(psi / 2)
            const double sp2 = sp * sp;
            const double s2 = 4.0 * r * rp * (sh * sh + sp2);
            const double H2 = 0.5 * (Ha[ip] * Ha[ip] + Hb[i] * Hb[i]);
            const double X = s2 / (8.0 * H2);
            double k0e, Dx;
            k0e_D_f64(X, bw, k0e, Dx);
            const double invH = 1.0 / sqrt(H2);
            const double mu = G * rp * rp * du * dphi;
            const double f = -mu * Dx * (0.125 * inv_sqrt_pi) * invH * invH * invH;
            // row transforms: sources enter times r_i', accelerations leave divided by
            // r_i, the inverse is unnormalised
            const double acc = r / (rp * nphi), pot = 1.0 / (rp * nphi);
            vR = f * rp * (expm1(Dl) + 2.0 * sp2) * acc;
            vA = f * rp * sinpi(2.0 * dj / nphi) * acc;
            vP = -mu * k0e * (0.5 * inv_sqrt_pi) * invH * pot;
        }
        o_phi[idx] = vP;
        o_r[idx] = vR;
        o_a[idx] = vA;
    }
}

// Packed row spectra of the chunk ([nphi/2][ci nr], FP64) -> the table rows
// i0 .. i0 + ci - 1 of one (pair, component): tab[(m nr + i) nr + i'].
template <typename R>
__global__ void __launch_bounds__(256)
k_semi_pack(const double2 *__restrict__ spec, cplx<R> *__restrict__ tab, int nr, int N, int i0, int ci)
{
    const size_t rows = (size_t)ci * nr, n = (size_t)N * rows;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t m = idx / rows, k = idx - m * rows;
        const double2 v = spec[blk(m, k, rows)];
        tab[(m * nr + i0) * nr + k] = mkc<cplx<R>>((R)v.x, (R)v.y);
    }
}

struct SemiOut {
    int b[6], c[6];   // target fluid and component of each requested output (grid z)
};

// One CTA: mode m, 32 target rows, one requested output.  The source spectra
// of column m wait in shared memory; each warp runs 4 target rows, its lanes
// striding the source rows of each table row (each table entry is read once,
// streaming).  Slot m = 0 multiplies re by re and im by im (two real
// matrices, the m = 0 and m = nphi/2 modes).
template <typename R, int NS>
__global__ void __launch_bounds__(256)
k_semi_mv(const cplx<R> *__restrict__ sh, const cplx<R> *__restrict__ tab, cplx<R> *__restrict__ oh, int nr,
          int N, const __grid_constant__ SemiOut q)
{
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *ss = reinterpret_cast<C *>(smem_raw);
    const int m = blockIdx.x, z = blockIdx.z, b = q.b[z], c = q.c[z];
    for (int k = threadIdx.x; k < NS * nr; k += blockDim.x) {
        const int a = k / nr, ip = k - a * nr;
        ss[k] = sh[(size_t)a * N * nr + blk(m, ip, nr)];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ib = blockIdx.y * 32 + w * 4;
    const bool packed0 = m == 0;
    R ar[4] = {0, 0, 0, 0}, ai[4] = {0, 0, 0, 0};
#pragma unroll 1
    for (int a = 0; a < NS; ++a) {
        const C *T = tab + ((size_t)((a * NS + b) * 3 + c) * N + m) * nr * nr;
        const C *sa = ss + a * nr;
        if constexpr (sizeof(R) == 4) {
            // two complex per lane per step (16-byte loads; nr is even); four
            // steps of four rows in flight per thread
#pragma unroll 4
            for (int ip = 2 * lane; ip < nr; ip += 64) {
                const float4 s = *reinterpret_cast<const float4 *>(sa + ip);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (ib + k >= nr) break;
                    const float4 t = __ldcs(reinterpret_cast<const float4 *>(T + (size_t)(ib + k) * nr + ip));
                    if (packed0) {
                        ar[k] = fmaf(t.x, s.x, fmaf(t.z, s.z, ar[k]));
                        ai[k] = fmaf(t.y, s.y, fmaf(t.w, s.w, ai[k]));
                    } else {
                        ar[k] = fmaf(t.x, s.x, fmaf(-t.y, s.y, fmaf(t.z, s.z, fmaf(-t.w, s.w, ar[k]))));
                        ai[k] = fmaf(t.x, s.y, fmaf(t.y, s.x, fmaf(t.z, s.w, fmaf(t.w, s.z, ai[k]))));
                    }
                }
            }
        } else {
#pragma unroll 2
            for (int ip = lane; ip < nr; ip += 32) {
                const C s = sa[ip];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (ib + k >= nr) break;
                    const C t = T[(size_t)(ib + k) * nr + ip];
                    if (packed0) {
                        ar[k] = fma(t.x, s.x, ar[k]);
                        ai[k] = fma(t.y, s.y, ai[k]);
                    } else {
                        ar[k] = fma(t.x, s.x, fma(-t.y, s.y, ar[k]));
                        ai[k] = fma(t.x, s.y, fma(t.y, s.x, ai[k]));
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ar[k] += __shfl_xor_sync(0xffffffffu, ar[k], o);
            ai[k] += __shfl_xor_sync(0xffffffffu, ai[k], o);
        }
    }
    if (lane < 4 && ib + lane < nr) {
        R xr = ar[0], xi = ai[0];
#pragma unroll
        for (int k = 1; k < 4; ++k)
            if (lane == k) {
                xr = ar[k];
                xi = ai[k];
            }
        oh[(size_t)(b * 3 + c) * N * nr + blk(m, ib + lane, nr)] = mkc<C>(xr, xi);
    }
}

int grid_for(size_t n) { return (int)((n + 255) / 256 < 152 * 32 ? (n + 255) / 256 : 152 * 32); }

}  // namespace

size_t semi_table_bytes(int nr, int nphi, int nsrc, bool f64)
{
    return (size_t)nsrc * nsrc * 3 * (nphi / 2) * (size_t)nr * nr * (f64 ? 16 : 8);
}

template <typename R>
cudaError_t build_semi_tables(int nr, int nphi, int nsrc, double du, double dphi, double G, const double *rc_h,
                              const double *H_h[2], void *tab, const void *tw_row64, const void *twp_row64,
                              cudaStream_t s)
{
    const int N = nphi / 2;
    // chunk of target rows: 3 component samples + one spectrum, ~512 MB of FP64 scratch
    const size_t per_row = (size_t)nr * nphi * 8 * 4;
    int ci = 1;
    while (ci < nr && (size_t)(2 * ci) * per_row <= ((size_t)512 << 20)) ci *= 2;
    double *rc = nullptr, *H = nullptr, *eval = nullptr;
    void *spec = nullptr;
    const size_t chunk = (size_t)ci * nr * nphi;
    cudaError_t e = cudaMalloc((void **)&rc, nr * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&H, 2 * (size_t)nr * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&eval, 3 * chunk * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&spec, chunk * sizeof(double));   // [N][ci nr] complex
    if (e == cudaSuccess) e = cudaMemcpyAsync(rc, rc_h, nr * sizeof(double), cudaMemcpyHostToDevice, s);
    for (int a = 0; a < nsrc && e == cudaSuccess; ++a)
        e = cudaMemcpyAsync(H + (size_t)a * nr, H_h[a], nr * sizeof(double), cudaMemcpyHostToDevice, s);
    const size_t one = (size_t)N * nr * nr;   // entries of one (pair, component) table
    for (int a = 0; a < nsrc && e == cudaSuccess; ++a)
        for (int b = 0; b < nsrc && e == cudaSuccess; ++b)
            for (int i0 = 0; i0 < nr && e == cudaSuccess; i0 += ci) {
                double *o[3] = {eval, eval + chunk, eval + 2 * chunk};
                k_semi_eval<<<grid_for(chunk), 256, 0, s>>>(nr, nphi, i0, ci, rc, H + (size_t)a * nr,
                                                           H + (size_t)b * nr, du, dphi, G, o[0], o[1], o[2]);
                e = cudaGetLastError();
                for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
                    e = launch_rows_fwd<double>(o[c], nullptr, 1, spec, ci * nr, nphi, tw_row64, twp_row64, nullptr,
                                                false, s);
                    if (e != cudaSuccess) break;
                    cplx<R> *dst = reinterpret_cast<cplx<R> *>(tab) + (size_t)((a * nsrc + b) * 3 + c) * one;
                    k_semi_pack<R><<<grid_for((size_t)N * ci * nr), 256, 0, s>>>((const double2 *)spec, dst, nr, N,
                                                                                 i0, ci);
                    e = cudaGetLastError();
                }
            }
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    cudaFree(rc);
    cudaFree(H);
    cudaFree(eval);
    cudaFree(spec);
    return e;
}

size_t semi_mv_smem(int nr, int nsrc, bool f64) { return (size_t)nsrc * nr * (f64 ? 16 : 8); }

template <typename R>
cudaError_t launch_semi_mv(const void *sh, const void *tab, void *oh, int nr, int nphi, int nsrc, uint32_t outmask,
                           cudaStream_t s)
{
    SemiOut q{};
    int nz = 0;
    for (int k = 0; k < 6; ++k)
        if ((outmask >> k) & 1u) {
            q.b[nz] = k / 3;
            q.c[nz] = k % 3;
            ++nz;
        }
    if (!nz) return cudaSuccess;
    const int N = nphi / 2;
    const dim3 grid(N, (nr + 31) / 32, nz);
    const size_t smem = semi_mv_smem(nr, nsrc, sizeof(R) == 8);
    using C = cplx<R>;
    if (nsrc == 1)
        k_semi_mv<R, 1><<<grid, 256, smem, s>>>((const C *)sh, (const C *)tab, (C *)oh, nr, N, q);
    else
        k_semi_mv<R, 2><<<grid, 256, smem, s>>>((const C *)sh, (const C *)tab, (C *)oh, nr, N, q);
    return cudaGetLastError();
}

cudaError_t set_semi_smem_limits(int max_optin)
{
    const void *fns[] = {(const void *)k_semi_mv<float, 1>, (const void *)k_semi_mv<float, 2>,
                         (const void *)k_semi_mv<double, 1>, (const void *)k_semi_mv<double, 2>};
    for (const void *f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t build_semi_tables<float>(int, int, int, double, double, double, const double *,
                                              const double *[2], void *, const void *, const void *, cudaStream_t);
template cudaError_t build_semi_tables<double>(int, int, int, double, double, double, const double *,
                                               const double *[2], void *, const void *, const void *, cudaStream_t);
template cudaError_t launch_semi_mv<float>(const void *, const void *, void *, int, int, int, uint32_t, cudaStream_t);
template cudaError_t launch_semi_mv<double>(const void *, const void *, void *, int, int, int, uint32_t, cudaStream_t);

}  // namespace sg
