// Direct O(N^2) pair sum with position-dependent scale heights (Sec. 2.2):
//     g_b(r) = -G sum_a sum_{cells r' != r} m_a(r') K_ab(r, r') e_s,
//     Phi_b(r) = -G sum_a sum_{cells r' != r} m_a(r') e^X K0(X) / (2 sqrt(pi) H_ab),
// m_a = Sigma_a r'^2 du dphi, H_ab^2 = (H_a(r')^2 + H_b(r)^2) / 2 (Eq. "mean
// root square height"), X = s^2 / (8 H_ab^2).  This is the parity path of
// the library and the only one valid for non-constant H/r.
//
// The pair geometry is taken from the integer index differences
// (di, dj) = (i - i', j - j'), with Delta = di du and psi = dj dphi:
//     s^2            = 4 r r' [sinh^2(Delta/2) + sin^2(psi/2)],
//     e_r . (r - r') = r' [expm1(Delta) + 2 sin^2(psi/2)],
//     e_phi . (r - r') = r' sin psi,
// using per-lag tables built in FP64, so FP32 keeps full relative precision
// for the nearest neighbours (no cancellation in r - r').
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "sg.h"
#include "sg_bessel.cuh"
#include "sg_internal.h"

namespace sg {

template <typename R> struct pair_of;
template <> struct pair_of<float> { using type = float2; };
template <> struct pair_of<double> { using type = double2; };

template <typename R> struct Acc {
    R s = 0, c = 0;
    __device__ __forceinline__ void add(R v)   // Kahan-compensated sum
    {
        R y = v - c;
        R t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

template <typename R>
__device__ __forceinline__ void k0e_D_any(R x, const BesselWeights &bw, R &k0e, R &D);
template <>
__device__ __forceinline__ void k0e_D_any<double>(double x, const BesselWeights &bw, double &k0e, double &D)
{
    k0e_D_f64(x, bw, k0e, D);
}
template <>
__device__ __forceinline__ void k0e_D_any<float>(float x, const BesselWeights &bw, float &k0e, float &D)
{
    if (x < 1.0f) {   // log singularity region: FP64
        double a, b;
        k0e_D_f64((double)x, bw, a, b);
        k0e = (float)a;
        D = (float)b;
    } else {
        k0e_D_f32(x, bw, k0e, D);
    }
}

constexpr int DT = 256;   // targets per CTA and sources per shared-memory tile
// FP32: compiled for 4 resident CTAs per SM (64 registers, a few spilled):
// 256 x 512 gas + dust solve 708 -> 641 ms against the unbounded 94-register
// build at 2 CTAs per SM (2 and 3 CTAs per SM: 754 and 751 ms); bit-identical.
#ifndef SG_DIRECT_MINB
#define SG_DIRECT_MINB 4
#endif

template <typename R>
__global__ void __launch_bounds__(DT, sizeof(R) == 4 ? SG_DIRECT_MINB : 1)
k_direct(int nr, int nphi, R G, const R *__restrict__ sig_g, const R *__restrict__ sig_d,
         const R *__restrict__ Hg, const R *__restrict__ Hd, R h_g, R h_d, int tgt, R *phi, R *gr,
         R *gphi, const typename pair_of<R>::type *__restrict__ geo_i,
         const typename pair_of<R>::type *__restrict__ geo_j, const R *__restrict__ rcen, R dudphi,
         unsigned int *flag)
{
    using P2 = typename pair_of<R>::type;
    __shared__ BesselWeights bw;
    __shared__ R s_r[DT], s_m[DT], s_H2[DT];
    __shared__ int s_i[DT], s_j[DT];
    bessel_weights_init(bw);
    const int ncell = nr * nphi;
    const int tid = blockIdx.x * DT + threadIdx.x;
    const bool valid = tid < ncell;
    const int i = valid ? tid / nphi : 0;
    const int j = valid ? tid - i * nphi : 0;
    const R r = rcen[i];
    const R *Hb_f = tgt == 0 ? Hg : Hd;
    const R hb = tgt == 0 ? h_g : h_d;
    const R Hb = valid ? (Hb_f ? Hb_f[tid] : hb * r) : (R)1;
    const R Hb2 = Hb * Hb;
    const R c_force = (R)(0.125 * 0.56418958354775628695);   // 1 / (8 sqrt(pi))
    const R c_pot = (R)(0.5 * 0.56418958354775628695);       // 1 / (2 sqrt(pi))
    Acc<R> agr, agp, aph;
    const int nsrc_fluids = sig_d ? 2 : 1;
    for (int a = 0; a < nsrc_fluids; ++a) {
        const R *sig = a == 0 ? sig_g : sig_d;
        const R *Ha_f = a == 0 ? Hg : Hd;
        const R ha = a == 0 ? h_g : h_d;
        for (int s0 = 0; s0 < ncell; s0 += DT) {
            __syncthreads();
            const int src = s0 + threadIdx.x;
            if (src < ncell) {
                const int ii = src / nphi, jj = src - (src / nphi) * nphi;
                const R rr = rcen[ii];
                const R Ha = Ha_f ? Ha_f[src] : ha * rr;
                s_r[threadIdx.x] = rr;
                s_m[threadIdx.x] = G * sig[src] * rr * rr * dudphi;
                s_H2[threadIdx.x] = Ha * Ha;
                s_i[threadIdx.x] = ii;
                s_j[threadIdx.x] = jj;
            }
            __syncthreads();
            const int cnt = min(DT, ncell - s0);
            if (!valid) continue;
            for (int q = 0; q < cnt; ++q) {
                if (s0 + q == tid) continue;                 // self cell excluded
                const int di = i - s_i[q];
                int dj = j - s_j[q];
                if (dj < 0) dj += nphi;
                const P2 gi = geo_i[di + nr - 1];            // (sinh^2(D/2), expm1(D))
                const P2 gj = geo_j[dj];                     // (sin^2(psi/2), sin psi)
                const R rr = s_r[q];
                const R s2 = (R)4 * r * rr * (gi.x + gj.x);
                const R H2 = (R)0.5 * (s_H2[q] + Hb2);
                const R X = s2 / ((R)8 * H2);
                R k0e, D;
                k0e_D_any<R>(X, bw, k0e, D);
                const R invH = (R)1 / sqrt(H2);
                const R f = -s_m[q] * D * c_force * invH * invH * invH;   // -G m K / s
                agr.add(f * rr * (gi.y + (R)2 * gj.x));
                agp.add(f * rr * gj.y);
                aph.add(-s_m[q] * k0e * c_pot * invH);
            }
        }
    }
    if (!valid) return;
    if (phi) phi[tid] = aph.s;
    if (gr) gr[tid] = agr.s;
    if (gphi) gphi[tid] = agp.s;
    if (flag && !(isfinite(aph.s) && isfinite(agr.s) && isfinite(agp.s))) atomicOr(flag, 1u);
}

template <typename R>
cudaError_t launch_direct(int nr, int nphi, double r_in, double du, double G, const R *sig_g,
                          const R *sig_d, const R *Hg, const R *Hd, double h_g, double h_d, int tgt,
                          R *phi, R *gr, R *gphi, const R *geo_i, const R *geo_j, const R *rcen,
                          unsigned int *flag, cudaStream_t s)
{
    (void)r_in;
    using P2 = typename pair_of<R>::type;
    const int ncell = nr * nphi;
    const double dphi = 2.0 * M_PI / nphi;
    k_direct<R><<<(ncell + DT - 1) / DT, DT, 0, s>>>(
        nr, nphi, (R)G, sig_g, sig_d, Hg, Hd, (R)h_g, (R)h_d, tgt, phi, gr, gphi, (const P2 *)geo_i,
        (const P2 *)geo_j, rcen, (R)(du * dphi), flag);
    return cudaGetLastError();
}

template cudaError_t launch_direct<float>(int, int, double, double, double, const float *, const float *,
                                          const float *, const float *, double, double, int, float *,
                                          float *, float *, const float *, const float *, const float *,
                                          unsigned int *, cudaStream_t);
template cudaError_t launch_direct<double>(int, int, double, double, double, const double *, const double *,
                                           const double *, const double *, double, double, int, double *,
                                           double *, double *, const double *, const double *,
                                           const double *, unsigned int *, cudaStream_t);

}  // namespace sg

// ---------------------------------------------------------------------------
// Allocation-free direct sum (sg_direct_noalloc in sg.h).
//
// Some callers cannot let a library allocate device memory: host codes whose
// device memory is owned by their own allocator or a fixed pool (a library
// cudaMalloc would bypass their accounting or fragment the pool), and time
// loops that must never enter the CUDA allocator.  sg_direct_noalloc serves
// them with the direct pair sum of a plan of the DIRECT method, without a
// plan: the per-lag geometry tables that a plan keeps in its own device
// memory live instead in the fixed array below, compiled into this library.
// Every GPU that loads the library holds the array until the process exits.

namespace {

constexpr int kNoAllocMaxNr = 1024;     // largest nr the array can serve
constexpr int kNoAllocMaxNphi = 4096;   // largest nphi
// FP64 layout (FP32 uses the first half of each part):
//   [0, 32768)       lag table over di: (sinh^2(D/2), expm1(D)), 2 (2 nr - 1) reals
//   [32768, 98304)   lag table over dj: (sin^2(psi/2), sin psi), 2 nphi reals
//   [98304, 106496)  cell-centre radii, nr reals
constexpr size_t kNoAllocGeoJ = 32768, kNoAllocRcen = 98304, kNoAllocBytes = 106496;
static_assert(2 * (2 * kNoAllocMaxNr - 1) * sizeof(double) <= kNoAllocGeoJ, "geo_i part too small");
static_assert(2 * kNoAllocMaxNphi * sizeof(double) <= kNoAllocRcen - kNoAllocGeoJ, "geo_j part too small");
static_assert(kNoAllocMaxNr * sizeof(double) <= kNoAllocBytes - kNoAllocRcen, "rcen part too small");

}  // namespace

static __device__ __align__(256) unsigned char g_sg_noalloc_scratch[kNoAllocBytes];

namespace sg {

// Fill the three geometry tables for one grid (FP64 arithmetic).
template <typename R>
__global__ void k_direct_geometry(int nr, int nphi, double r_in, double du, R *geo_i, R *geo_j, R *rcen)
{
    const int n = max(2 * nr - 1, max(nphi, nr));
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        if (q < 2 * nr - 1) {
            const double D = (q - (nr - 1)) * du, sh = sinh(0.5 * D);
            geo_i[2 * q] = (R)(sh * sh);
            geo_i[2 * q + 1] = (R)expm1(D);
        }
        if (q < nphi) {
            const int jj = (2 * q <= nphi) ? q : nphi - q;
            const double sg = (2 * q <= nphi) ? 1.0 : -1.0;
            const double sp = sinpi((double)jj / nphi);
            geo_j[2 * q] = (R)(sp * sp);
            geo_j[2 * q + 1] = (R)(sg * sinpi(2.0 * jj / nphi));
        }
        if (q < nr) rcen[q] = (R)(r_in * exp((q + 0.5) * du));
    }
}

}  // namespace sg

namespace {

// The array's device address, looked up once per CUDA context.  A context is
// identified by its unique id (cuCtxGetId: never reused within a process), so
// a primary context that cudaDeviceReset tore down and the runtime created
// again gets a fresh lookup instead of the old, dangling address.
struct NoAllocSlot {
    unsigned long long ctx_id;
    void *ptr;
};
std::mutex g_noalloc_mutex;
NoAllocSlot g_noalloc[64] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context; 0 when none is current.
unsigned long long current_ctx_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the array in the current context: the lookup runs on the
// first call in each context (it also makes the device's primary context
// current when none is), later calls reuse it.
cudaError_t noalloc_scratch(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocSlot &slot = g_noalloc[dev];
    const unsigned long long id = current_ctx_id();
    if (id == 0 || id != slot.ctx_id || !slot.ptr) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_sg_noalloc_scratch);
        if (e != cudaSuccess) return e;
        slot.ptr = ptr;
        slot.ctx_id = current_ctx_id();            // nonzero once the lookup made a context current
    }
    *out = slot.ptr;
    return cudaSuccess;
}

template <typename R>
sg_status direct_noalloc_t(const sg_params *p, void *scratch, const void *sg_, const void *sd_,
                           void *const outs[6], int nsrc, cudaStream_t s)
{
    const double du = std::log(p->r_out / p->r_in) / p->nr;
    R *geo_i = (R *)scratch;
    R *geo_j = (R *)((char *)scratch + kNoAllocGeoJ);
    R *rcen = (R *)((char *)scratch + kNoAllocRcen);
    // every entry the sum reads is rewritten here first, so nothing from an
    // earlier call is used
    const int n = std::max(2 * p->nr - 1, std::max(p->nphi, p->nr));
    sg::k_direct_geometry<R><<<(n + 255) / 256, 256, 0, s>>>(p->nr, p->nphi, p->r_in, du, geo_i, geo_j, rcen);
    cudaError_t e = cudaGetLastError();
    for (int b = 0; b < nsrc && e == cudaSuccess; ++b) {
        if (!(outs[3 * b] || outs[3 * b + 1] || outs[3 * b + 2])) continue;
        e = sg::launch_direct<R>(p->nr, p->nphi, p->r_in, du, p->G, (const R *)sg_, nsrc == 2 ? (const R *)sd_ : nullptr,
                                 (const R *)p->H_g_field, (const R *)p->H_d_field, p->h_g, p->h_d, b, (R *)outs[3 * b],
                                 (R *)outs[3 * b + 1], (R *)outs[3 * b + 2], geo_i, geo_j, rcen, nullptr, s);
    }
    if (e != cudaSuccess) {
        fprintf(stderr, "sg_direct_noalloc: %s\n", cudaGetErrorString(e));
        return SG_ERR_CUDA;
    }
    return SG_OK;
}

}  // namespace

extern "C" sg_status sg_direct_noalloc(const sg_params *p, const void *sigma_g, const void *sigma_d, void *phi_g,
                                       void *gr_g, void *gphi_g, void *phi_d, void *gr_d, void *gphi_d, void *stream)
{
    if (!p || !sigma_g) return SG_ERR_ARG;
    if (p->method != SG_METHOD_DIRECT || (p->dtype != SG_F32 && p->dtype != SG_F64)) return SG_ERR_ARG;
    if (!(std::isfinite(p->r_in) && std::isfinite(p->r_out) && p->r_in > 0 && p->r_out > p->r_in) ||
        !std::isfinite(p->G) || p->nr < 1 || p->nphi < 1)
        return SG_ERR_ARG;
    if (p->nr > kNoAllocMaxNr || p->nphi > kNoAllocMaxNphi) {
        fprintf(stderr, "sg_direct_noalloc: grid %d x %d exceeds the fixed scratch (nr <= %d, nphi <= %d)\n", p->nr,
                p->nphi, kNoAllocMaxNr, kNoAllocMaxNphi);
        return SG_ERR_UNSUPPORTED;
    }
    // the parameter sets sg_plan_create accepts for a DIRECT plan
    if (!(std::isfinite(p->h_g) && (p->h_g > 0 || p->H_g_field))) return SG_ERR_ARG;
    const int nsrc = (p->h_d > 0 || p->H_d_field) ? 2 : 1;
    if (nsrc == 2 && (!std::isfinite(p->h_d) || !sigma_d)) return SG_ERR_ARG;
    // an error left pending by the caller's own work is theirs: report it
    // without consuming it, and launch nothing
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) {
        fprintf(stderr, "sg_direct_noalloc: a CUDA error is already pending (%s); nothing launched\n",
                cudaGetErrorString(pending));
        return SG_ERR_CUDA;
    }
    void *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) {
        fprintf(stderr, "sg_direct_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
        return SG_ERR_CUDA;
    }
    void *outs[6] = {phi_g, gr_g, gphi_g, phi_d, gr_d, gphi_d};
    cudaStream_t s = (cudaStream_t)stream;
    return p->dtype == SG_F64 ? direct_noalloc_t<double>(p, scratch, sigma_g, sigma_d, outs, nsrc, s)
                              : direct_noalloc_t<float>(p, scratch, sigma_g, sigma_d, outs, nsrc, s);
}

