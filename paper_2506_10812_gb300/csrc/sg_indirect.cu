// Indirect term (Sec. 5.4, App. E of Rendon Restrepo et al. 2025): the
// star's pull by each source fluid a reduces to two global sums,
//     A_a = sqrt(2) G sum_cells m_a K_a cos phi',   B_a = the same with sin phi',
//     K_a = (1/sqrt(pi)) H_a^-2 (d_a/4) e^{d_a^2/4} [K1 - K0](d_a^2/4),  d_a = r'/H_a,
// m_a = Sigma_a r'^2 du dphi, and the indirect potential's gradient is
// (A cos phi + B sin phi) e_r + (-A sin phi + B cos phi) e_phi.
//
// For a constant aspect ratio h_a, K_a r'^2 = D(1/(4 h_a^2)) / (4 sqrt(pi) h_a^3)
// is one number, so the per-cell work is a weighted sum of Sigma; with a
// scale-height field the factor is evaluated per cell (FP64 Bessel).  The
// reduction is FP64 and deterministic: per-block partial sums, then one
// block adds them in a fixed order.
#include <math.h>

#include "sg_bessel.cuh"
#include "sg_internal.h"

namespace sg {

constexpr int IB = 256;   // threads per block

int indirect_blocks(int nphi)
{
    // when nphi divides the thread count every thread keeps one phi column
    int per = (nphi % IB == 0) ? nphi / IB : 1;
    int nb = per * ((304 + per - 1) / per);
    return nb;
}

template <typename R>
__global__ void __launch_bounds__(IB)
k_indirect_partial(int nr, int nphi, int nsrc, const R *__restrict__ s0, const R *__restrict__ s1,
                   const R *__restrict__ H0, const R *__restrict__ H1, const R *__restrict__ rcen, int fixed_j,
                   double *partial)
{
    __shared__ BesselWeights bw;
    __shared__ double red[IB / 32][4];
    bessel_weights_init(bw);
    __syncthreads();
    const long tid = (long)blockIdx.x * IB + threadIdx.x;
    const long nthr = (long)gridDim.x * IB;
    const long ncell = (long)nr * nphi;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};   // [fluid][cos, sin]
    double cj = 0.0, sj = 0.0;
    if (fixed_j) sincospi(2.0 * ((double)(tid % nphi) + 0.5) / nphi, &sj, &cj);
    for (long c = tid; c < ncell; c += nthr) {
        const int i = (int)(c / nphi);
        const int j = (int)(c - (long)i * nphi);
        if (!fixed_j) sincospi(2.0 * ((double)j + 0.5) / nphi, &sj, &cj);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (a >= nsrc) break;
            const R *sig = a ? s1 : s0;
            const R *Hf = a ? H1 : H0;
            double q = (double)sig[c];
            if (Hf) {
                // per-cell factor r'^2 K_a
                const double r = (double)rcen[i], H = (double)Hf[c];
                double k0e, D;
                k0e_D_f64(0.25 * r * r / (H * H), bw, k0e, D);
                q *= r * r * (0.56418958354775628695 / (H * H)) * (0.25 * r / H) * D;
            }
            if (fixed_j) {
                acc[2 * a] += q;
            } else {
                acc[2 * a] += q * cj;
                acc[2 * a + 1] += q * sj;
            }
        }
    }
    if (fixed_j)
        for (int a = 0; a < 2; ++a) {
            acc[2 * a + 1] = acc[2 * a] * sj;
            acc[2 * a] *= cj;
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[w][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int ww = 0; ww < IB / 32; ++ww) v += red[ww][threadIdx.x];
        partial[(size_t)blockIdx.x * 4 + threadIdx.x] = v;
    }
}

// out[2 a + k] = sqrt(2) G du dphi C_a sum_blocks partial; C_a = 1 with a
// scale-height field (already in the partials), else D(1/(4 h_a^2)) / (4 sqrt(pi) h_a^3).
__global__ void __launch_bounds__(32)
k_indirect_final(int nblocks, int nsrc, const double *__restrict__ partial, double h0, double h1, int field0,
                 int field1, double scale, double *out)
{
    __shared__ BesselWeights bw;
    bessel_weights_init(bw);
    __syncthreads();
    const int k = threadIdx.x;
    if (k >= 2 * nsrc) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * 4 + k];
    const int a = k >> 1;
    double C = 1.0;
    if (!(a ? field1 : field0)) {
        const double h = a ? h1 : h0;
        double k0e, D;
        k0e_D_f64(0.25 / (h * h), bw, k0e, D);
        C = D * 0.56418958354775628695 / (4.0 * h * h * h);
    }
    out[k] = scale * C * s;
}

template <typename R>
cudaError_t launch_indirect(int nr, int nphi, int nsrc, const R *s0, const R *s1, const R *H0, const R *H1,
                            double h0, double h1, const R *rcen, double G, double du, double dphi, double *partial,
                            double *out, cudaStream_t s)
{
    const int nb = indirect_blocks(nphi);
    const int fixed_j = ((long)nb * IB) % nphi == 0 ? 1 : 0;
    k_indirect_partial<R><<<nb, IB, 0, s>>>(nr, nphi, nsrc, s0, s1, H0, H1, rcen, fixed_j, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_indirect_final<<<1, 32, 0, s>>>(nb, nsrc, partial, h0, h1, H0 != nullptr, H1 != nullptr,
                                      1.4142135623730950488 * G * du * dphi, out);
    return cudaGetLastError();
}

template cudaError_t launch_indirect<float>(int, int, int, const float *, const float *, const float *, const float *,
                                            double, double, const float *, double, double, double, double *,
                                            double *, cudaStream_t);
template cudaError_t launch_indirect<double>(int, int, int, const double *, const double *, const double *,
                                             const double *, double, double, const double *, double, double, double,
                                             double *, double *, cudaStream_t);

}  // namespace sg
