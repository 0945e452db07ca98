// C ABI of the self-gravity library: plan lifetime, argument checks and the
// launch sequence of each entry point (declared and documented in sg.h).
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sg.h"
#include "sg_internal.h"

using namespace sg;

namespace {

sg_status fail(sg_plan *pl, sg_status s, const char *fmt, ...)
{
    if (pl) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(pl->err, sizeof(pl->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

sg_status cuda_fail(sg_plan *pl, cudaError_t e, const char *what)
{
    return fail(pl, e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

void free_all(sg_plan *pl)
{
    // FP64 plans share one twiddle table between the solve and the table build
    if (pl->tw_row == pl->tw_row64) pl->tw_row = nullptr;
    if (pl->twp_row == pl->twp_row64) pl->twp_row = nullptr;
    if (pl->twp_col == pl->twp_col64) pl->twp_col = nullptr;
    void *ptrs[] = {pl->tw_row, pl->tw_row64, pl->twp_row, pl->twp_row64, pl->twp_col, pl->twp_col64,
                    pl->tab, pl->sh, pl->oh, pl->rcen, pl->geo_i, pl->geo_j, pl->Hg, pl->Hd, pl->flag,
                    pl->stage, pl->ipart, pl->atab};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (cudaEvent_t ev : pl->cev)
        if (ev) cudaEventDestroy(ev);
    if (pl->cstream) cudaStreamDestroy(pl->cstream);
    // leave no error state behind for the next call's launch check
    cudaGetLastError();
}

template <typename R>
std::vector<R> twiddles(int M)
{
    // exp(-2 pi i m / M), m = 0..M-1, from FP64 sin/cos of the exact angle
    std::vector<R> v(2 * (size_t)M);
    for (int m = 0; m < M; ++m) {
        const double a = 2.0 * M_PI * (double)m / (double)M;
        v[2 * (size_t)m] = (R)std::cos(a);
        v[2 * (size_t)m + 1] = (R)(-std::sin(a));
    }
    return v;
}

// Per-pass Stockham twiddles of a length-L transform (layout in sg_fft.cuh):
// for the pass with stride Ns and radix R, W_{Ns R}^{r k} at (r - 1) Ns + k.
template <typename R>
std::vector<R> pass_twiddles(int L)
{
    std::vector<R> v;
    auto put = [&](int Ns, int Rad) {
        for (int r = 1; r < Rad; ++r)
            for (int k = 0; k < Ns; ++k) {
                const double a = 2.0 * M_PI * (double)r * (double)k / ((double)Ns * Rad);
                v.push_back((R)std::cos(a));
                v.push_back((R)(-std::sin(a)));
            }
    };
    int Ns = 16;
    while (Ns * 16 <= L) {
        put(Ns, 16);
        Ns *= 16;
    }
    if (Ns < L) put(Ns, L / Ns);
    if (v.empty()) v.assign(2, (R)0);
    return v;
}

template <typename R>
cudaError_t upload(void **dst, const std::vector<R> &h, cudaStream_t s)
{
    cudaError_t e = cudaMalloc(dst, h.size() * sizeof(R));
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(*dst, h.data(), h.size() * sizeof(R), cudaMemcpyHostToDevice, s);
}

std::mutex g_dev_mutex;
bool g_dev_ready[64] = {false};

cudaError_t device_setup(int dev)
{
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_dev_ready[dev]) return cudaSuccess;
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = set_smem_limits(optin);
    if (e == cudaSuccess) e = set_semi_smem_limits(optin);
    if (e == cudaSuccess) g_dev_ready[dev] = true;
    return e;
}

template <typename R>
std::vector<R> geometry_i(int nr, double du)
{
    // lag table over di = -(nr-1)..nr-1: (sinh^2(Delta/2), expm1(Delta))
    std::vector<R> v(2 * (size_t)(2 * nr - 1));
    for (int di = -(nr - 1); di <= nr - 1; ++di) {
        const double D = di * du, sh = std::sinh(0.5 * D);
        v[2 * (size_t)(di + nr - 1)] = (R)(sh * sh);
        v[2 * (size_t)(di + nr - 1) + 1] = (R)std::expm1(D);
    }
    return v;
}

template <typename R>
std::vector<R> geometry_j(int nphi)
{
    // lag table over dj = 0..nphi-1: (sin^2(psi/2), sin psi), exactly even/odd
    std::vector<R> v(2 * (size_t)nphi);
    for (int dj = 0; dj < nphi; ++dj) {
        const int jj = (2 * dj <= nphi) ? dj : nphi - dj;
        const double sg = (2 * dj <= nphi) ? 1.0 : -1.0;
        const double sp = std::sin(M_PI * jj / nphi);
        v[2 * (size_t)dj] = (R)(sp * sp);
        v[2 * (size_t)dj + 1] = (R)(sg * std::sin(2.0 * M_PI * jj / nphi));
    }
    return v;
}

template <typename R>
std::vector<R> centres(int nr, double r_in, double du)
{
    std::vector<R> v(nr);
    for (int i = 0; i < nr; ++i) v[i] = (R)(r_in * std::exp((i + 0.5) * du));
    return v;
}

sg_status check_device(sg_plan *pl)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != pl->device)
        return fail(pl, SG_ERR_ARG, "plan belongs to device %d but device %d is current", pl->device, dev);
    return SG_OK;
}

// Radial scaling exponent of the FFT path (see sg_kernels.cu): sources times
// r, kernel tables times e^{Delta}, accelerations divided by r.
constexpr double kAlpha = 1.0;

// Build the packed kernel spectra of every ordered fluid pair (App. C
// lattice kernels, Sec. 5.2 precomputation).
// The row transforms' tensor maps of sh and oh, boxes of the plan's tiles.
void encode_maps(sg_plan *pl)
{
    pl->tm_rows = rows_tma_eligible(pl->p.nr, pl->p.nphi, pl->f64) &&
                  encode_row_map(&pl->tm_sh, pl->sh, pl->p.nr, (long long)pl->nsrc * pl->N, pl->rows_fwd) ==
                      cudaSuccess &&
                  encode_row_map(&pl->tm_oh, pl->oh, pl->p.nr, (long long)pl->nsrc * 3 * pl->N, pl->rows_inv) ==
                      cudaSuccess;
}

sg_status build_tables(sg_plan *pl, cudaStream_t s)
{
    const int nr = pl->p.nr, nphi = pl->p.nphi, L = pl->L, N = pl->N;
    const size_t lat = (size_t)L * nphi;
    double *eval = nullptr;
    void *spec = nullptr;
    cudaError_t e = cudaMalloc((void **)&eval, 3 * lat * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(pl, e, "table scratch");
    e = cudaMalloc(&spec, (size_t)N * L * 2 * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(eval);
        return cuda_fail(pl, e, "table scratch");
    }
    // -G du dphi from the cell measure, 1/(L nphi) from the unnormalised
    // forward and inverse transforms
    const double scale = -pl->p.G * pl->du * pl->dphi / ((double)L * nphi);
    const size_t tab_one = (size_t)(N + 1) * tab_pitch(nr) * 2 * pl->esz;
    sg_status st = SG_OK;
    for (int a = 0; a < pl->nsrc && st == SG_OK; ++a) {
        for (int b = 0; b < pl->nsrc && st == SG_OK; ++b) {
            const double ha = a == 0 ? pl->p.h_g : pl->p.h_d;
            const double hb = b == 0 ? pl->p.h_g : pl->p.h_d;
            double *o64[3] = {eval, eval + lat, eval + 2 * lat};
            float *o32[3] = {nullptr, nullptr, nullptr};
            e = launch_tab_eval(nr, nphi, pl->du, ha, hb, scale, kAlpha, !pl->f64, o64, o32, s);
            for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
                e = launch_rows_fwd<double>(o64[c], nullptr, 1, spec, L, nphi, pl->tw_row64, pl->twp_row64,
                                            nullptr, false, s);
                if (e != cudaSuccess) break;
                char *dst = (char *)pl->tab + (size_t)((a * pl->nsrc + b) * 3 + c) * tab_one;
                e = pl->f64 ? launch_tabcols<double>(spec, dst, L, nphi, c == 2, pl->twp_col64, s)
                            : launch_tabcols<float>(spec, dst, L, nphi, c == 2, pl->twp_col64, s);
            }
            if (e != cudaSuccess) st = cuda_fail(pl, e, "kernel table build");
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (st == SG_OK && e2 != cudaSuccess) st = cuda_fail(pl, e2, "kernel table build");
    cudaFree(eval);
    cudaFree(spec);
    return st;
}

uint32_t outmask_of(const sg_plan *pl, void *const outs[6])
{
    uint32_t m = 0;
    for (int q = 0; q < 6; ++q)
        if (outs[q] && (q < 3 || pl->nsrc == 2)) m |= 1u << q;
    return m;
}

template <typename R>
sg_status solve_t(sg_plan *pl, const void *sg_, const void *sd_, void *const outs[6], cudaStream_t s,
                  unsigned int *sflag, bool check_finite)
{
    const uint32_t mask = outmask_of(pl, outs);
    if (!mask) return SG_OK;
    const int nr = pl->p.nr, nphi = pl->p.nphi;
    unsigned int *flag = check_finite ? sflag : nullptr;
    cudaError_t e;
    const bool ev = pl->ev[0] != nullptr;
    if (ev) cudaEventRecord(pl->ev[0], s);
    // The column pass and the inverse rows start as programmatic dependents
    // of the kernel before them (set-up and kernel-spectrum staging overlap
    // its last CTAs); a stage-timed solve keeps plain stream order so that
    // each stage's events bracket its own kernel only.
    if (pl->p.method == SG_METHOD_FFT) {
        e = launch_rows_fwd<R>((const R *)sg_, (const R *)sd_, pl->nsrc, pl->sh, nr, nphi, pl->tw_row,
                               pl->twp_row, (const R *)pl->rcen, true, s, 0, -1, pl->tm_rows ? &pl->tm_sh : nullptr,
                               sflag, pl->rows_fwd);
        if (e != cudaSuccess) return cuda_fail(pl, e, "row transform");
        if (ev) cudaEventRecord(pl->ev[1], s);
        e = pl->engine >= SG_ENGINE_TC_BF16X3
                ? launch_cols_tc(pl->engine, pl->sh, pl->tab, pl->oh, nr, nphi, mask, pl->twp_col, sflag, s)
            : pl->engine ? launch_cols_mma(pl->engine, pl->sh, pl->tab, pl->oh, nr, nphi, mask, pl->twp_col, pl->atab,
                                           sflag, s)
                         : launch_cols<R>(pl->sh, pl->tab, pl->oh, nr, nphi, pl->nsrc, mask, pl->twp_col, sflag, s,
                                          0, !ev, true, pl->cols_staging);
        if (e != cudaSuccess) return cuda_fail(pl, e, "column pass");
        if (ev) cudaEventRecord(pl->ev[2], s);
        RowOut ro{};
        for (int q = 0; q < 6; ++q) {
            if (!((mask >> q) & 1u)) continue;
            ro.ptr[ro.n] = outs[q];
            ro.src[ro.n] = q;
            ro.is_phi[ro.n] = (q % 3) == SG_COMP_PHI;
            ++ro.n;
        }
        e = launch_rows_inv<R>(pl->oh, ro, nr, nphi, pl->tw_row, pl->twp_row, (const R *)pl->rcen, flag, s, 0, -1,
                               pl->tm_rows ? &pl->tm_oh : nullptr, sflag, !ev, pl->rows_inv);
        if (e != cudaSuccess) return cuda_fail(pl, e, "inverse row transform");
        if (ev) cudaEventRecord(pl->ev[3], s);
    } else if (pl->p.method == SG_METHOD_SEMISPECTRAL) {
        // the FFT path's row transforms around the per-mode radial products
        e = launch_rows_fwd<R>((const R *)sg_, (const R *)sd_, pl->nsrc, pl->sh, nr, nphi, pl->tw_row,
                               pl->twp_row, (const R *)pl->rcen, true, s, 0, -1, pl->tm_rows ? &pl->tm_sh : nullptr,
                               sflag, pl->rows_fwd);
        if (e != cudaSuccess) return cuda_fail(pl, e, "row transform");
        if (ev) cudaEventRecord(pl->ev[1], s);
        e = launch_semi_mv<R>(pl->sh, pl->tab, pl->oh, nr, nphi, pl->nsrc, mask, s);
        if (e != cudaSuccess) return cuda_fail(pl, e, "radial products");
        if (ev) cudaEventRecord(pl->ev[2], s);
        RowOut ro{};
        for (int q = 0; q < 6; ++q) {
            if (!((mask >> q) & 1u)) continue;
            ro.ptr[ro.n] = outs[q];
            ro.src[ro.n] = q;
            ro.is_phi[ro.n] = (q % 3) == SG_COMP_PHI;
            ++ro.n;
        }
        e = launch_rows_inv<R>(pl->oh, ro, nr, nphi, pl->tw_row, pl->twp_row, (const R *)pl->rcen, flag, s, 0, -1,
                               pl->tm_rows ? &pl->tm_oh : nullptr, sflag, false, pl->rows_inv);
        if (e != cudaSuccess) return cuda_fail(pl, e, "inverse row transform");
        if (ev) cudaEventRecord(pl->ev[3], s);
    } else {
        for (int b = 0; b < pl->nsrc; ++b) {
            if (!((mask >> (3 * b)) & 7u)) continue;
            e = launch_direct<R>(nr, nphi, pl->p.r_in, pl->du, pl->p.G, (const R *)sg_,
                                 pl->nsrc == 2 ? (const R *)sd_ : nullptr, (const R *)pl->Hg,
                                 (const R *)pl->Hd, pl->p.h_g, pl->p.h_d, b, (R *)outs[3 * b],
                                 (R *)outs[3 * b + 1], (R *)outs[3 * b + 2], (const R *)pl->geo_i,
                                 (const R *)pl->geo_j, (const R *)pl->rcen, flag, s);
            if (e != cudaSuccess) return cuda_fail(pl, e, "direct sum");
        }
        if (ev)
            for (int q = 1; q < 4; ++q) cudaEventRecord(pl->ev[q], s);
    }
    return SG_OK;
}

sg_status solve_any(sg_plan *pl, const void *sg_, const void *sd_, void *const outs[6], void *stream)
{
    if (!pl) return SG_ERR_ARG;
    return solve_into(pl, sg_, sd_, outs, (cudaStream_t)stream, pl->flag, (pl->p.flags & SG_CHECK_FINITE) != 0);
}

}  // namespace

// Declared in sg_internal.h.
sg_status solve_into(sg_plan *pl, const void *sg_, const void *sd_, void *const outs[6], cudaStream_t s,
                     unsigned int *sflag, bool check_finite)
{
    if (!pl) return SG_ERR_ARG;
    sg_status st = check_device(pl);
    if (st != SG_OK) return st;
    if (!sg_) return fail(pl, SG_ERR_ARG, "sigma_g is NULL");
    if (pl->nsrc == 2 && !sd_) return fail(pl, SG_ERR_ARG, "bi-fluid plan needs sigma_d");
    // the row transforms move element pairs
    const uintptr_t amask = 2 * pl->esz - 1;
    bool misaligned = ((uintptr_t)sg_ & amask) || (pl->nsrc == 2 && ((uintptr_t)sd_ & amask));
    for (int q = 0; q < 6; ++q) misaligned |= ((uintptr_t)outs[q] & amask) != 0;
    if (misaligned) return fail(pl, SG_ERR_ARG, "device buffers must be aligned to %d bytes", (int)(amask + 1));
    return pl->f64 ? solve_t<double>(pl, sg_, sd_, outs, s, sflag, check_finite)
                   : solve_t<float>(pl, sg_, sd_, outs, s, sflag, check_finite);
}

namespace {

// Pipelined host-buffer FFT solve: row chunks of the inputs are copied on the
// plan's copy stream while the previous chunk's row transforms run on `s`;
// after the column pass, each chunk's inverse row transforms are followed on
// the copy stream by that chunk's output copies, overlapping the next
// chunk's transforms.
template <typename R>
sg_status solve_host_fft(sg_plan *pl, const void *hsg, const void *hsd, void *const host_out[6], cudaStream_t s)
{
    const int nr = pl->p.nr, nphi = pl->p.nphi;
    const size_t row_b = (size_t)nphi * pl->esz, bytes = (size_t)nr * row_b;
    char *stg = (char *)pl->stage;
    R *dsg = (R *)stg, *dsd = pl->nsrc == 2 ? (R *)(stg + bytes) : nullptr;
    void *dev_out[6];
    for (int q = 0; q < 6; ++q) dev_out[q] = host_out[q] ? stg + (2 + q) * bytes : nullptr;
    const uint32_t mask = outmask_of(pl, dev_out);
    // Inputs go up in nin chunks, each chunk's row transforms starting as it
    // lands; outputs come down in two copies per output: inverse-row chunk 0
    // alone (the copies start early) and chunks 1 .. nch-1 together, which
    // finish on the GPU while the first copy is still running (each copy call
    // costs ~2.5 us on the host link, so fewer and larger copies save time).
    const int rpc = row_rpc(nphi, pl->f64);
    const int nin = nr / rpc < 4 ? nr / rpc : 4, rows_in = nr / nin;
    const int nch = nr / rpc < 8 ? nr / rpc : 8, rows = nr / nch;
    cudaStream_t c = pl->cstream;
    cudaEvent_t *ein = pl->cev, *eout = pl->cev + 8, start = pl->cev[16];
    unsigned int *flag = (pl->p.flags & SG_CHECK_FINITE) ? pl->flag : nullptr;
    cudaError_t e = cudaEventRecord(start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c, start, 0);
    for (int k = 0; k < nin && e == cudaSuccess; ++k) {
        const size_t off = (size_t)k * rows_in * row_b, len = (size_t)rows_in * row_b;
        e = cudaMemcpyAsync((char *)dsg + off, (const char *)hsg + off, len, cudaMemcpyHostToDevice, c);
        if (e == cudaSuccess && dsd)
            e = cudaMemcpyAsync((char *)dsd + off, (const char *)hsd + off, len, cudaMemcpyHostToDevice, c);
        if (e == cudaSuccess) e = cudaEventRecord(ein[k], c);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ein[k], 0);
        if (e == cudaSuccess)
            e = launch_rows_fwd<R>(dsg, dsd, pl->nsrc, pl->sh, nr, nphi, pl->tw_row, pl->twp_row, (const R *)pl->rcen,
                                   true, s, k * rows_in, rows_in, pl->tm_rows ? &pl->tm_sh : nullptr, pl->flag,
                                   pl->rows_fwd);
    }
    if (e != cudaSuccess) return cuda_fail(pl, e, "pipelined input and row transform");
    if (!mask) return cuda_fail(pl, cudaStreamSynchronize(s), "solve");
    e = pl->engine >= SG_ENGINE_TC_BF16X3
            ? launch_cols_tc(pl->engine, pl->sh, pl->tab, pl->oh, nr, nphi, mask, pl->twp_col, pl->flag, s)
        : pl->engine ? launch_cols_mma(pl->engine, pl->sh, pl->tab, pl->oh, nr, nphi, mask, pl->twp_col, pl->atab,
                                       pl->flag, s)
                     : launch_cols<R>(pl->sh, pl->tab, pl->oh, nr, nphi, pl->nsrc, mask, pl->twp_col, pl->flag, s, 0,
                                      true, true, pl->cols_staging);
    if (e != cudaSuccess) return cuda_fail(pl, e, "column pass");
    RowOut ro{};
    for (int q = 0; q < 6; ++q) {
        if (!((mask >> q) & 1u)) continue;
        ro.ptr[ro.n] = dev_out[q];
        ro.src[ro.n] = q;
        ro.is_phi[ro.n] = (q % 3) == SG_COMP_PHI;
        ++ro.n;
    }
    for (int k = 0; k < nch && e == cudaSuccess; ++k) {
        // chunk 0 follows the column pass directly: a programmatic dependent of it
        e = launch_rows_inv<R>(pl->oh, ro, nr, nphi, pl->tw_row, pl->twp_row, (const R *)pl->rcen, flag, s, k * rows,
                               rows, pl->tm_rows ? &pl->tm_oh : nullptr, pl->flag, k == 0, pl->rows_inv);
        if (k != 0 && k != nch - 1) continue;
        // copy group: chunk 0, then chunks 1 .. nch-1
        const int k0 = k == 0 ? 0 : 1;
        if (e == cudaSuccess) e = cudaEventRecord(eout[k], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c, eout[k], 0);
        const size_t off = (size_t)k0 * rows * row_b, len = (size_t)(k - k0 + 1) * rows * row_b;
        for (int q = 0; q < 6 && e == cudaSuccess; ++q)
            if ((mask >> q) & 1u)
                e = cudaMemcpyAsync((char *)host_out[q] + off, (const char *)dev_out[q] + off, len,
                                    cudaMemcpyDeviceToHost, c);
    }
    if (e != cudaSuccess) return cuda_fail(pl, e, "pipelined inverse transform and output");
    e = cudaStreamSynchronize(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(pl, e, "solve");
    return SG_OK;
}

}  // namespace

extern "C" {

sg_status sg_plan_create(sg_plan **out, const sg_params *p, void *stream)
{
    if (!out) return SG_ERR_ARG;
    *out = nullptr;
    if (!p) return SG_ERR_ARG;
    sg_plan *pl = new (std::nothrow) sg_plan();
    if (!pl) return SG_ERR_OOM;
    pl->p = *p;
    auto reject = [&](sg_status s, const char *msg) {
        fprintf(stderr, "sg_plan_create: %s\n", msg);
        delete pl;
        return s;
    };
    const bool fft = p->method == SG_METHOD_FFT, semi = p->method == SG_METHOD_SEMISPECTRAL;
    if (p->method != SG_METHOD_FFT && p->method != SG_METHOD_DIRECT && !semi)
        return reject(SG_ERR_ARG, "unknown method");
    if (p->dtype != SG_F32 && p->dtype != SG_F64) return reject(SG_ERR_ARG, "unknown dtype");
    if (!(std::isfinite(p->r_in) && std::isfinite(p->r_out) && p->r_in > 0 && p->r_out > p->r_in))
        return reject(SG_ERR_ARG, "need 0 < r_in < r_out");
    if (!std::isfinite(p->G)) return reject(SG_ERR_ARG, "G must be finite");
    if (p->nr < 1 || p->nphi < 1) return reject(SG_ERR_ARG, "nr and nphi must be positive");
    if (!(std::isfinite(p->h_g) && (p->h_g > 0 || (!fft && p->H_g_field))))
        return reject(SG_ERR_ARG, "h_g must be > 0");
    pl->nsrc = (p->h_d > 0 || (!fft && p->H_d_field)) ? 2 : 1;
    if (fft) {
        if (p->H_g_field || p->H_d_field)
            return reject(SG_ERR_NOT_FFT_COMPATIBLE, "the FFT method needs constant aspect ratios (no H fields)");
        if (!is_pow2(p->nr) || !is_pow2(p->nphi) || p->nr < 8 || p->nr > 4096 || p->nphi < 32 || p->nphi > 8192)
            return reject(SG_ERR_UNSUPPORTED, "FFT method: nr, nphi powers of two, 8<=nr<=4096, 32<=nphi<=8192");
    } else if (semi) {
        if (!is_pow2(p->nr) || !is_pow2(p->nphi) || p->nr < 8 || p->nr > 4096 || p->nphi < 32 || p->nphi > 8192)
            return reject(SG_ERR_UNSUPPORTED,
                          "semi-spectral method: nr, nphi powers of two, 8<=nr<=4096, 32<=nphi<=8192");
    } else if ((long long)p->nr * p->nphi > (1LL << 24)) {
        return reject(SG_ERR_UNSUPPORTED, "direct method limited to 2^24 cells");
    }
    if (pl->nsrc == 2 && !std::isfinite(p->h_d)) return reject(SG_ERR_ARG, "h_d must be finite");
    pl->f64 = p->dtype == SG_F64;
    pl->esz = pl->f64 ? 8 : 4;
    pl->L = 2 * p->nr;
    pl->N = p->nphi / 2;
    pl->du = std::log(p->r_out / p->r_in) / p->nr;
    pl->dphi = 2.0 * M_PI / p->nphi;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&pl->device);
    if (e == cudaSuccess) e = device_setup(pl->device);
    if (e != cudaSuccess) {
        fprintf(stderr, "sg_plan_create: %s\n", cudaGetErrorString(e));
        delete pl;
        return SG_ERR_CUDA;
    }
    if (fft || semi) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device);
        const size_t need[] = {row_smem_bytes(p->nphi, row_rpc(p->nphi, pl->f64), pl->f64),
                               row_smem_bytes(p->nphi, row_rpc(p->nphi, true), true),
                               fft ? col_smem_bytes(p->nr, pl->nsrc, pl->f64) : semi_mv_smem(p->nr, pl->nsrc, pl->f64),
                               fft ? tabcol_smem_bytes(pl->L, true) : 0};
        for (size_t b : need)
            if (b > (size_t)optin) return reject(SG_ERR_UNSUPPORTED, "grid too large for shared memory in this dtype");
    }
    // semi-spectral: H fields must not depend on phi; their radial profiles build the tables
    std::vector<double> Hprof[2];
    if (semi) {
        const size_t cells_h = (size_t)p->nr * p->nphi;
        for (int a = 0; a < pl->nsrc; ++a) {
            const void *fld = a == 0 ? p->H_g_field : p->H_d_field;
            const double h = a == 0 ? p->h_g : p->h_d;
            Hprof[a].resize(p->nr);
            if (!fld) {
                for (int i = 0; i < p->nr; ++i) Hprof[a][i] = h * p->r_in * std::exp((i + 0.5) * pl->du);
                continue;
            }
            std::vector<double> hv(cells_h);
            cudaError_t ce;
            if (pl->f64) {
                ce = cudaMemcpy(hv.data(), fld, cells_h * sizeof(double), cudaMemcpyDeviceToHost);
            } else {
                std::vector<float> hf(cells_h);
                ce = cudaMemcpy(hf.data(), fld, cells_h * sizeof(float), cudaMemcpyDeviceToHost);
                for (size_t k = 0; k < cells_h; ++k) hv[k] = hf[k];
            }
            if (ce != cudaSuccess) {
                cudaGetLastError();
                return reject(SG_ERR_ARG, "could not read an H field (device pointer of the plan dtype expected)");
            }
            for (int i = 0; i < p->nr; ++i) {
                const double v = hv[(size_t)i * p->nphi];
                if (!(std::isfinite(v) && v > 0))
                    return reject(SG_ERR_ARG, "H fields must be finite and positive");
                for (int j = 1; j < p->nphi; ++j)
                    if (hv[(size_t)i * p->nphi + j] != v)
                        return reject(SG_ERR_ARG, "the semi-spectral method needs H fields independent of phi");
                Hprof[a][i] = v;
            }
        }
    }
    const size_t cells = (size_t)p->nr * p->nphi;
    std::vector<float> f;
    std::vector<double> d;
#define SG_TRY(call, what)                                       \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) {                                 \
            fprintf(stderr, "sg_plan_create: %s: %s\n", what, cudaGetErrorString(e_)); \
            free_all(pl);                                        \
            sg_status st_ = e_ == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA; \
            delete pl;                                           \
            return st_;                                          \
        }                                                        \
    } while (0)
    if (pl->f64) SG_TRY(upload(&pl->rcen, centres<double>(p->nr, p->r_in, pl->du), s), "centres");
    else SG_TRY(upload(&pl->rcen, centres<float>(p->nr, p->r_in, pl->du), s), "centres");
    SG_TRY(cudaMalloc((void **)&pl->flag, sizeof(unsigned int)), "flag");
    SG_TRY(cudaMalloc((void **)&pl->ipart, (size_t)indirect_blocks(p->nphi) * 4 * sizeof(double)), "indirect sums");
    SG_TRY(cudaMemsetAsync(pl->flag, 0, sizeof(unsigned int), s), "flag");
    if (semi) {
        SG_TRY(upload(&pl->tw_row64, twiddles<double>(p->nphi), s), "twiddles");
        SG_TRY(upload(&pl->twp_row64, pass_twiddles<double>(p->nphi / 2), s), "twiddles");
        if (pl->f64) {
            pl->tw_row = pl->tw_row64;
            pl->twp_row = pl->twp_row64;
        } else {
            SG_TRY(upload(&pl->tw_row, twiddles<float>(p->nphi), s), "twiddles");
            SG_TRY(upload(&pl->twp_row, pass_twiddles<float>(p->nphi / 2), s), "twiddles");
        }
        const size_t cbytes = 2 * pl->esz;
        SG_TRY(cudaMalloc(&pl->tab, semi_table_bytes(p->nr, p->nphi, pl->nsrc, pl->f64)), "semi-spectral tables");
        SG_TRY(cudaMalloc(&pl->sh, (size_t)pl->nsrc * pl->N * p->nr * cbytes), "scratch");
        SG_TRY(cudaMalloc(&pl->oh, (size_t)pl->nsrc * 3 * pl->N * p->nr * cbytes), "scratch");
        encode_maps(pl);
        if (p->H_g_field) {
            SG_TRY(cudaMalloc(&pl->Hg, cells * pl->esz), "H_g copy");
            SG_TRY(cudaMemcpyAsync(pl->Hg, p->H_g_field, cells * pl->esz, cudaMemcpyDeviceToDevice, s), "H_g copy");
        }
        if (p->H_d_field && pl->nsrc == 2) {
            SG_TRY(cudaMalloc(&pl->Hd, cells * pl->esz), "H_d copy");
            SG_TRY(cudaMemcpyAsync(pl->Hd, p->H_d_field, cells * pl->esz, cudaMemcpyDeviceToDevice, s), "H_d copy");
        }
        std::vector<double> rc(p->nr);
        for (int i = 0; i < p->nr; ++i) rc[i] = p->r_in * std::exp((i + 0.5) * pl->du);
        const double *hp[2] = {Hprof[0].data(), pl->nsrc == 2 ? Hprof[1].data() : nullptr};
        SG_TRY(pl->f64 ? build_semi_tables<double>(p->nr, p->nphi, pl->nsrc, pl->du, pl->dphi, p->G, rc.data(), hp,
                                                   pl->tab, pl->tw_row64, pl->twp_row64, s)
                       : build_semi_tables<float>(p->nr, p->nphi, pl->nsrc, pl->du, pl->dphi, p->G, rc.data(), hp,
                                                  pl->tab, pl->tw_row64, pl->twp_row64, s),
               "semi-spectral table build");
    } else if (fft) {
        SG_TRY(upload(&pl->tw_row64, twiddles<double>(p->nphi), s), "twiddles");
        SG_TRY(upload(&pl->twp_row64, pass_twiddles<double>(p->nphi / 2), s), "twiddles");
        SG_TRY(upload(&pl->twp_col64, pass_twiddles<double>(pl->L), s), "twiddles");
        if (pl->f64) {
            pl->tw_row = pl->tw_row64;
            pl->twp_row = pl->twp_row64;
            pl->twp_col = pl->twp_col64;
        } else {
            SG_TRY(upload(&pl->tw_row, twiddles<float>(p->nphi), s), "twiddles");
            SG_TRY(upload(&pl->twp_row, pass_twiddles<float>(p->nphi / 2), s), "twiddles");
            SG_TRY(upload(&pl->twp_col, pass_twiddles<float>(pl->L), s), "twiddles");
        }
        const size_t cbytes = 2 * pl->esz;
        SG_TRY(cudaMalloc(&pl->tab, (size_t)pl->nsrc * pl->nsrc * 3 * (pl->N + 1) * tab_pitch(p->nr) * cbytes),
               "kernel spectra");
        SG_TRY(cudaMalloc(&pl->sh, (size_t)pl->nsrc * pl->N * p->nr * cbytes), "scratch");
        SG_TRY(cudaMalloc(&pl->oh, (size_t)pl->nsrc * 3 * pl->N * p->nr * cbytes), "scratch");
        encode_maps(pl);
        sg_status st = build_tables(pl, s);
        if (st != SG_OK) {
            fprintf(stderr, "sg_plan_create: %s\n", pl->err);
            free_all(pl);
            delete pl;
            return st;
        }
    } else {
        if (pl->f64) {
            SG_TRY(upload(&pl->geo_i, geometry_i<double>(p->nr, pl->du), s), "geometry");
            SG_TRY(upload(&pl->geo_j, geometry_j<double>(p->nphi), s), "geometry");
        } else {
            SG_TRY(upload(&pl->geo_i, geometry_i<float>(p->nr, pl->du), s), "geometry");
            SG_TRY(upload(&pl->geo_j, geometry_j<float>(p->nphi), s), "geometry");
        }
        if (p->H_g_field) {
            SG_TRY(cudaMalloc(&pl->Hg, cells * pl->esz), "H_g copy");
            SG_TRY(cudaMemcpyAsync(pl->Hg, p->H_g_field, cells * pl->esz, cudaMemcpyDeviceToDevice, s), "H_g copy");
        }
        if (p->H_d_field && pl->nsrc == 2) {
            SG_TRY(cudaMalloc(&pl->Hd, cells * pl->esz), "H_d copy");
            SG_TRY(cudaMemcpyAsync(pl->Hd, p->H_d_field, cells * pl->esz, cudaMemcpyDeviceToDevice, s), "H_d copy");
        }
        if (pl->nsrc == 2 && !p->H_d_field && !(p->h_d > 0)) {
            free_all(pl);
            return reject(SG_ERR_ARG, "dust needs h_d > 0 or H_d_field");
        }
    }
    SG_TRY(cudaStreamSynchronize(s), "plan build");
#undef SG_TRY
    pl->p.H_g_field = pl->Hg;
    pl->p.H_d_field = pl->Hd;
    *out = pl;
    return SG_OK;
}

sg_status sg_kernel_table(sg_plan *pl, int pair, int comp, void *out_dev, void *stream)
{
    if (!pl) return SG_ERR_ARG;
    sg_status st = check_device(pl);
    if (st != SG_OK) return st;
    if (pl->p.method != SG_METHOD_FFT) return fail(pl, SG_ERR_UNSUPPORTED, "kernel tables exist for the FFT method only");
    if (pair < 0 || pair >= pl->nsrc * pl->nsrc) return fail(pl, SG_ERR_ARG, "pair %d not in this plan", pair);
    if (comp < 0 || comp > 2) return fail(pl, SG_ERR_ARG, "component %d out of range", comp);
    if (!out_dev) return fail(pl, SG_ERR_ARG, "out_dev is NULL");
    const int a = pair / pl->nsrc, b = pair % pl->nsrc;   // SG_PAIR_*: source * 2 + target
    const double ha = a == 0 ? pl->p.h_g : pl->p.h_d;
    const double hb = b == 0 ? pl->p.h_g : pl->p.h_d;
    double *o64[3] = {nullptr, nullptr, nullptr};
    float *o32[3] = {nullptr, nullptr, nullptr};
    if (pl->f64) o64[comp] = (double *)out_dev;
    else o32[comp] = (float *)out_dev;
    cudaError_t e = launch_tab_eval(pl->p.nr, pl->p.nphi, pl->du, ha, hb, 1.0, 0.0, !pl->f64, o64, o32,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(pl, e, "kernel table");
    return SG_OK;
}

sg_status sg_potential(sg_plan *pl, const void *sigma_g, const void *sigma_d, void *phi_g, void *phi_d,
                       void *stream)
{
    void *outs[6] = {phi_g, nullptr, nullptr, phi_d, nullptr, nullptr};
    return solve_any(pl, sigma_g, sigma_d, outs, stream);
}

sg_status sg_accel(sg_plan *pl, const void *sigma_g, const void *sigma_d, void *gr_g, void *gphi_g,
                   void *gr_d, void *gphi_d, void *stream)
{
    void *outs[6] = {nullptr, gr_g, gphi_g, nullptr, gr_d, gphi_d};
    return solve_any(pl, sigma_g, sigma_d, outs, stream);
}

sg_status sg_solve(sg_plan *pl, const void *sigma_g, const void *sigma_d, void *phi_g, void *gr_g,
                   void *gphi_g, void *phi_d, void *gr_d, void *gphi_d, void *stream)
{
    void *outs[6] = {phi_g, gr_g, gphi_g, phi_d, gr_d, gphi_d};
    return solve_any(pl, sigma_g, sigma_d, outs, stream);
}

sg_status sg_solve_host(sg_plan *pl, const void *sigma_g, const void *sigma_d, void *phi_g, void *gr_g,
                        void *gphi_g, void *phi_d, void *gr_d, void *gphi_d, void *stream)
{
    if (!pl) return SG_ERR_ARG;
    sg_status st = check_device(pl);
    if (st != SG_OK) return st;
    if (!sigma_g || (pl->nsrc == 2 && !sigma_d)) return fail(pl, SG_ERR_ARG, "missing input");
    const size_t bytes = (size_t)pl->p.nr * pl->p.nphi * pl->esz;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (!pl->stage) {
        e = cudaMalloc(&pl->stage, 8 * bytes);
        if (e != cudaSuccess) {
            pl->stage = nullptr;
            return cuda_fail(pl, e, "staging buffers");
        }
    }
    if (!pl->cstream) {
        e = cudaStreamCreateWithFlags(&pl->cstream, cudaStreamNonBlocking);
        for (int i = 0; i < 17 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&pl->cev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            // leave nothing half made: the next call creates the stream and all its events again
            for (int i = 0; i < 17; ++i)
                if (pl->cev[i]) {
                    cudaEventDestroy(pl->cev[i]);
                    pl->cev[i] = nullptr;
                }
            if (pl->cstream) cudaStreamDestroy(pl->cstream);
            pl->cstream = nullptr;
            return cuda_fail(pl, e, "copy stream");
        }
    }
    char *stg = (char *)pl->stage;
    void *host_out[6] = {phi_g, gr_g, gphi_g, phi_d, gr_d, gphi_d};
    if (pl->p.method == SG_METHOD_FFT)
        return pl->f64 ? solve_host_fft<double>(pl, sigma_g, sigma_d, host_out, s)
                       : solve_host_fft<float>(pl, sigma_g, sigma_d, host_out, s);
    void *dev_out[6];
    for (int q = 0; q < 6; ++q) dev_out[q] = host_out[q] ? stg + (2 + q) * bytes : nullptr;
    e = cudaMemcpyAsync(stg, sigma_g, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && pl->nsrc == 2) e = cudaMemcpyAsync(stg + bytes, sigma_d, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(pl, e, "host to device copy");
    st = solve_any(pl, stg, pl->nsrc == 2 ? stg + bytes : nullptr, dev_out, stream);
    if (st != SG_OK) return st;
    const uint32_t mask = outmask_of(pl, dev_out);
    for (int q = 0; q < 6; ++q) {
        if (!((mask >> q) & 1u)) continue;
        e = cudaMemcpyAsync(host_out[q], dev_out[q], bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(pl, e, "device to host copy");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(pl, e, "solve");
    return SG_OK;
}

sg_status sg_indirect(sg_plan *pl, const void *sigma_g, const void *sigma_d, double *ab_dev, void *stream)
{
    if (!pl) return SG_ERR_ARG;
    sg_status st = check_device(pl);
    if (st != SG_OK) return st;
    if (!sigma_g || !ab_dev) return fail(pl, SG_ERR_ARG, "sigma_g and ab_dev are required");
    if (pl->nsrc == 2 && !sigma_d) return fail(pl, SG_ERR_ARG, "bi-fluid plan needs sigma_d");
    const int nr = pl->p.nr, nphi = pl->p.nphi;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e =
        pl->f64 ? launch_indirect<double>(nr, nphi, pl->nsrc, (const double *)sigma_g, (const double *)sigma_d,
                                          (const double *)pl->Hg, (const double *)pl->Hd, pl->p.h_g, pl->p.h_d,
                                          (const double *)pl->rcen, pl->p.G, pl->du, pl->dphi, pl->ipart, ab_dev, s)
                : launch_indirect<float>(nr, nphi, pl->nsrc, (const float *)sigma_g, (const float *)sigma_d,
                                         (const float *)pl->Hg, (const float *)pl->Hd, pl->p.h_g, pl->p.h_d,
                                         (const float *)pl->rcen, pl->p.G, pl->du, pl->dphi, pl->ipart, ab_dev, s);
    if (e != cudaSuccess) return cuda_fail(pl, e, "indirect term");
    return SG_OK;
}

sg_status sg_sync(sg_plan *pl, void *stream)
{
    if (!pl) return SG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, pl->flag, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->flag, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(pl, e, "sg_sync");
    if (h & 2u) return fail(pl, SG_ERR_TIMEOUT, "a staged bulk copy did not complete");
    if (h & 1u) return fail(pl, SG_ERR_NONFINITE, "non-finite value in an output");
    return SG_OK;
}

sg_status sg_set_stage_events(sg_plan *pl, void *const *events)
{
    if (!pl) return SG_ERR_ARG;
    for (int q = 0; q < 4; ++q) {
        if (events && !events[q]) return fail(pl, SG_ERR_ARG, "stage event %d is NULL", q);
        pl->ev[q] = events ? (cudaEvent_t)events[q] : nullptr;
    }
    return SG_OK;
}

sg_status sg_stage_times(void *const *events, float *ms)
{
    if (!events || !ms) return SG_ERR_ARG;
    for (int q = 0; q < 4; ++q)
        if (!events[q]) return SG_ERR_ARG;
    if (cudaEventSynchronize((cudaEvent_t)events[3]) != cudaSuccess) return SG_ERR_CUDA;
    for (int q = 0; q < 3; ++q)
        if (cudaEventElapsedTime(&ms[q], (cudaEvent_t)events[q], (cudaEvent_t)events[q + 1]) != cudaSuccess) {
            cudaGetLastError();
            return SG_ERR_CUDA;
        }
    return SG_OK;
}

int32_t sg_launches_per_solve(const sg_plan *pl, uint32_t outmask)
{
    if (!pl) return 0;
    const uint32_t allowed = pl->nsrc == 2 ? 0x3Fu : 0x7u;
    outmask &= allowed;
    if (!outmask) return 0;
    if (pl->p.method == SG_METHOD_FFT) return pl->engine ? 4 : 3;   // tensor-core engines: column 0 apart
    if (pl->p.method == SG_METHOD_SEMISPECTRAL) return 3;
    return ((outmask & 7u) ? 1 : 0) + ((outmask & 0x38u) ? 1 : 0);
}

sg_status sg_set_column_engine(sg_plan *pl, int32_t engine)
{
    if (!pl) return SG_ERR_ARG;
    if (engine < SG_ENGINE_FFT32 || engine > SG_ENGINE_TC_FP16X3)
        return fail(pl, SG_ERR_ARG, "unknown engine %d", engine);
    if (engine == SG_ENGINE_FFT32) {
        pl->engine = 0;
        return SG_OK;
    }
    if (pl->p.method != SG_METHOD_FFT || pl->f64 || pl->nsrc != 1 || (pl->p.nr != 1024 && pl->p.nr != 2048))
        return fail(pl, SG_ERR_UNSUPPORTED,
                    "tensor-core column engines need an FP32 gas-only FFT plan with nr = 1024 or 2048");
    sg_status st = check_device(pl);
    if (st != SG_OK) return st;
    if (engine >= SG_ENGINE_TC_BF16X3) {
        pl->engine = engine;
        return SG_OK;
    }
    uint32_t h[8 * 32 * 4];
    dftmma_frag_table(engine == SG_ENGINE_DFT_FP16X3 || engine == SG_ENGINE_DFT_FP16, h);
    cudaError_t e = cudaSuccess;
    if (!pl->atab) e = cudaMalloc((void **)&pl->atab, sizeof(h));
    if (e == cudaSuccess) e = cudaMemcpy(pl->atab, h, sizeof(h), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(pl, e, "fragment table");
    pl->engine = engine;
    return SG_OK;
}

sg_status sg_get_tiles(const sg_plan *pl, sg_tiles *t)
{
    if (!pl || !t) return SG_ERR_ARG;
    t->rows_fwd = pl->rows_fwd;
    t->rows_inv = pl->rows_inv;
    t->cols_staging = cols_staging_steps(pl->p.nr, pl->nsrc, pl->f64, pl->cols_staging) ? SG_COLS_STAGE_STEP
                                                                                          : SG_COLS_STAGE_ALL;
    return SG_OK;
}

sg_status sg_set_tiles(sg_plan *pl, const sg_tiles *t)
{
    if (!pl) return SG_ERR_ARG;
    if (!t) return fail(pl, SG_ERR_ARG, "tiles is NULL");
    if ((t->rows_fwd != 2 && t->rows_fwd != 4) || (t->rows_inv != 2 && t->rows_inv != 4))
        return fail(pl, SG_ERR_ARG, "rows per CTA must be 2 or 4");
    if (t->cols_staging != SG_COLS_STAGE_ALL && t->cols_staging != SG_COLS_STAGE_STEP)
        return fail(pl, SG_ERR_ARG, "unknown column staging %d", t->cols_staging);
    if (pl->p.method == SG_METHOD_DIRECT) return fail(pl, SG_ERR_UNSUPPORTED, "tiles apply to FFT and semi-spectral plans");
    if (pl->f64 && t->cols_staging == SG_COLS_STAGE_STEP)
        return fail(pl, SG_ERR_UNSUPPORTED, "per-step column staging is FP32 only");
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device);
    if (e != cudaSuccess) return cuda_fail(pl, e, "device attribute");
    if (col_smem_bytes(pl->p.nr, pl->nsrc, pl->f64, t->cols_staging) > (size_t)optin)
        return fail(pl, SG_ERR_UNSUPPORTED, "this column staging needs %zu bytes of shared memory per block",
                    col_smem_bytes(pl->p.nr, pl->nsrc, pl->f64, t->cols_staging));
    pl->rows_fwd = t->rows_fwd;
    pl->rows_inv = t->rows_inv;
    pl->cols_staging = t->cols_staging;
    encode_maps(pl);
    return SG_OK;
}

sg_status sg_tc_dft16(int32_t engine, int64_t count, const void *in, void *out, int32_t inverse, void *stream)
{
    if (engine < SG_ENGINE_TC_BF16X3 || engine > SG_ENGINE_TC_FP16X3 || count < 256 || count % 256 ||
        count / 256 > 0x7FFFFFFF || !in || !out)
        return SG_ERR_ARG;
    // complex FP32 elements (8-byte loads and stores); the kernel reads and
    // writes through restrict pointers, so the two ranges must not overlap
    const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out, bytes = (uintptr_t)count * 16 * 8;
    if (((a | b) & 7u) || (a < b + bytes && b < a + bytes)) return SG_ERR_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = launch_tc_stage(engine, in, out, count, inverse ? 1 : 0, (cudaStream_t)stream);
    return e == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

void sg_destroy(sg_plan *pl)
{
    if (!pl) return;
    cudaDeviceSynchronize();
    free_all(pl);
    delete pl;
}

const char *sg_status_string(sg_status s)
{
    switch (s) {
    case SG_OK: return "ok";
    case SG_ERR_ARG: return "invalid argument";
    case SG_ERR_UNSUPPORTED: return "unsupported configuration";
    case SG_ERR_NOT_FFT_COMPATIBLE: return "FFT method needs constant aspect ratios";
    case SG_ERR_CUDA: return "CUDA error";
    case SG_ERR_OOM: return "device out of memory";
    case SG_ERR_NONFINITE: return "non-finite output";
    case SG_ERR_TIMEOUT: return "timeout";
    }
    return "unknown status";
}

const char *sg_last_error(const sg_plan *pl) { return pl ? pl->err : ""; }

}  // extern "C"
