// The column pass's per-column work shared by its engines (sg_kernels.cu:
// radix-16 butterflies in registers; sg_tcdft.cu: on the tensor cores): the
// packed kernel-spectrum access and the staged-spectrum column loop.
#pragma once

#include <stdint.h>

#include "sg_fft.cuh"
#include "sg_internal.h"
#include "sg_mem.cuh"

namespace sg {

// Kernel spectrum of one (pair, component, column m): P = H + 2 complex,
// slot k = S(k) for 0 <= k <= H (S(0), S(H) real); S(k > H) = conj(S(L - k)).
template <typename C>
__device__ __forceinline__ C spec_at(const C *col, int k, int H, bool upper)
{
    return upper ? cconj(col[2 * H - k]) : col[k];
}

// Column m = 0 holds the packed (m = 0, m = nphi/2) pair of real columns:
// Z = A + i B, so P = A S0 + i B SN = ((Z + Z*(-k)) S0 + (Z - Z*(-k)) SN) / 2.
template <typename R, int NS>
__device__ __noinline__ void col0_path(const cplx<R> *__restrict__ sh, const cplx<R> *__restrict__ tab,
                                       cplx<R> *__restrict__ oh, int nr, int N, uint32_t outmask,
                                       const cplx<R> *__restrict__ tw, cplx<R> *xb, cplx<R> *spec)
{
    using C = cplx<R>;
    const int L = 2 * nr, T = L >> 4, H = nr, P = tab_pitch(nr);
    const int t = threadIdx.x;
    C v[16];
    for (int a = 0; a < NS; ++a) {
        const C *col = sh + (size_t)a * N * nr;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = ld_cg_hint(col + blk(0, t + T * e, nr), l2_evict_first());
#pragma unroll
        for (int e = 8; e < 16; ++e) v[e] = mkc<C>(0, 0);
        fft_reg<true>(v, L, T, t, xb, tw);
#pragma unroll
        for (int e = 0; e < 16; ++e) spec[a * L + t + T * e] = v[e];
    }
    __syncthreads();
    for (int b = 0; b < NS; ++b) {
        for (int c = 0; c < 3; ++c) {
            if (!((outmask >> (3 * b + c)) & 1u)) continue;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int k = t + T * e;
                C acc = mkc<C>(0, 0);
                for (int a = 0; a < NS; ++a) {
                    const C *t0 = tab + ((size_t)((a * NS + b) * 3 + c) * (N + 1)) * P;
                    const C *tn = t0 + (size_t)N * P;
                    const C Z = spec[a * L + k];
                    const C Zm = cconj(spec[a * L + ((L - k) & (L - 1))]);
                    C S0 = spec_at(t0, k, H, e >= 8), SN = spec_at(tn, k, H, e >= 8);
                    if (c == 2) {
                        S0 = cmul_mi(S0);
                        SN = cmul_mi(SN);
                    }
                    acc = cadd(acc, cscale(cadd(cmul(cadd(Z, Zm), S0), cmul(csub(Z, Zm), SN)), (R)0.5));
                }
                v[e] = acc;
            }
            fft_reg<false>(v, L, T, t, xb, tw);
            C *o = oh + (size_t)(b * 3 + c) * N * nr;
#pragma unroll
            for (int e = 0; e < 8; ++e) o[blk(0, t + T * e, nr)] = v[e];
        }
    }
}

// LC > 0: compile-time column length (2 nr).
// Column 0 of a plan that stages kernel spectra per step (no shared-memory
// source spectra): each requested (target, component) step transforms the
// packed source columns again and pairs Z(k) with Z*(L - k) through the
// exchange buffer.  The same terms in the same order as col0_path, so the
// same result; for gas + dust 18 transforms instead of 8, in one CTA of the
// first wave.
template <typename R, int NS>
__device__ __noinline__ void col0_recompute(const cplx<R> *__restrict__ sh, const cplx<R> *__restrict__ tab,
                                            cplx<R> *__restrict__ oh, int nr, int N, uint32_t outmask,
                                            const cplx<R> *__restrict__ tw, cplx<R> *xb)
{
    using C = cplx<R>;
    const int L = 2 * nr, T = L >> 4, H = nr, P = tab_pitch(nr);
    const int t = threadIdx.x;
    for (int q = 0; q < 3 * NS; ++q) {
        if (!((outmask >> q) & 1u)) continue;
        const int b = q / 3, c = q % 3;
        C acc[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = mkc<C>(0, 0);
        for (int a = 0; a < NS; ++a) {
            C v[16];
            const C *col = sh + (size_t)a * N * nr;
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = ld_cg_hint(col + blk(0, t + T * e, nr), l2_evict_first());
#pragma unroll
            for (int e = 8; e < 16; ++e) v[e] = mkc<C>(0, 0);
            fft_reg<true>(v, L, T, t, xb, tw);
            __syncthreads();                   // the transform's last exchange reads are done
#pragma unroll
            for (int e = 0; e < 16; ++e) xb[pidx(t + T * e)] = v[e];
            __syncthreads();
            const C *t0 = tab + ((size_t)((a * NS + b) * 3 + c) * (N + 1)) * P;
            const C *tn = t0 + (size_t)N * P;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int k = t + T * e;
                const C Z = v[e];
                const C Zm = cconj(xb[pidx((L - k) & (L - 1))]);
                C S0 = spec_at(t0, k, H, e >= 8), SN = spec_at(tn, k, H, e >= 8);
                if (c == 2) {
                    S0 = cmul_mi(S0);
                    SN = cmul_mi(SN);
                }
                acc[e] = cadd(acc[e], cscale(cadd(cmul(cadd(Z, Zm), S0), cmul(csub(Z, Zm), SN)), (R)0.5));
            }
            __syncthreads();                   // before the next transform rewrites the buffer
        }
        fft_reg<false>(acc, L, T, t, xb, tw);
        C *o = oh + (size_t)(b * 3 + c) * N * nr;
#pragma unroll
        for (int e = 0; e < 8; ++e) o[blk(0, t + T * e, nr)] = acc[e];
    }
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Column-pass staging of the kernel spectra (a per-plan choice, sg_set_tiles):
// ST = 0 stages every requested table of a target at once (gas + dust: the
// source spectra in shared memory); ST = 1 stages one (target, component)
// step at a time (cols_pair_steps, source spectra in registers), FP32 only.
// Default: per step for every FP32 gas + dust plan and for FP32 gas-only
// columns of length 4096, which then fit 80 registers and run 3 CTAs of 256
// threads per SM instead of 2 (column pass 74.4 -> 70.2 us on the 2048 x 4096
// disc).  At length 2048 (1.1 waves of 6 CTAs per SM) the exposed per-step
// copy waits made it slower (22.3 -> 28.7 us), so those columns default to all
// tables at once.
__host__ __device__ constexpr bool cols_steps_default(int nsrc, bool f64, int L)
{
    return !f64 && (nsrc == 2 || (nsrc == 1 && L == 4096));
}
// launch bounds of k_cols<R, NS, LC, ST>: 768 threads per SM for the staged
// gas-only FP32 lengths >= 1024, otherwise up to 512 threads (128 registers)
constexpr bool cols_tight(int ns, bool f64, int lc, bool st) { return ns == 1 && st && !f64 && lc >= 1024; }
constexpr int cols_max_threads(int ns, bool f64, int lc, bool st) { return cols_tight(ns, f64, lc, st) ? lc / 16 : 512; }
constexpr int cols_min_blocks(int ns, bool f64, int lc, bool st)
{
    return cols_tight(ns, f64, lc, st) ? 768 / (lc / 16) : 1;
}

// Columns m >= 1 of a plan that stages kernel spectra per step (ST = 1):
// the source spectra stay in registers, and the kernel spectra of one
// (target, component) step (one table per source) are staged at a time; the
// next step's copy is issued once the products have read the buffer, so it
// lands during the inverse transform.  Gas + dust at 2 nr = 4096: 66 KB of
// shared memory and 2 CTAs per SM instead of 197 KB and 1; gas only: 51 KB,
// 80 registers and 3 CTAs per SM instead of 2.
template <typename R, int LC, int NS, typename Eng>
__device__ __forceinline__ void cols_pair_steps(const cplx<R> *__restrict__ sh, const cplx<R> *__restrict__ tab,
                                                cplx<R> *__restrict__ oh, int nr, int N, uint32_t outmask,
                                                const cplx<R> *__restrict__ tw, unsigned int *flag, cplx<R> *xb,
                                                cplx<R> *tb, uint64_t *bar, int m, int discard, const Eng &eng)
{
    using C = cplx<R>;
    const int L = 2 * nr, T = L >> 4, H = nr, P = tab_pitch(nr);
    const int t = threadIdx.x;
    auto next_q = [&](int q) {
        for (++q; q < 3 * NS; ++q)
            if ((outmask >> q) & 1u) return q;
        return -1;
    };
    auto issue = [&](int q) {
        if (t == 0) {
            const int b = q / 3, c = q % 3;
            const uint64_t pol = l2_evict_first();
            mbar_expect_tx(bar, (unsigned)(NS * P * sizeof(C)));
#pragma unroll
            for (int a = 0; a < NS; ++a)
                tma_load_1d(tb + (size_t)a * P, tab + ((size_t)((a * NS + b) * 3 + c) * (N + 1) + m) * P,
                            P * sizeof(C), bar, pol);
        }
    };
    int q = next_q(-1);
    if (t == 0) mbar_init(bar, 1);
    __syncthreads();
    if (q >= 0) issue(q);                          // lands while the forward FFTs run
    griddep_wait();                                // the row spectra are complete from here on
    C spec[NS][16];
#pragma unroll
    for (int a = 0; a < NS; ++a) {
        C v[16];
        const uint64_t pf = l2_evict_first();
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = ld_cg_hint(sh + (size_t)a * N * nr + blk(m, t + T * e, nr), pf);
#pragma unroll
        for (int e = 8; e < 16; ++e) v[e] = mkc<C>(0, 0);   // radial zero padding
        fft_any<true, LC, true>(v, L, T, t, xb, tw, eng.template d16<true>());
        // every thread's loads of this column were consumed before the
        // transform's first barrier: the column is dead
        if (discard) l2_discard_range(sh + (size_t)a * N * nr + blk(m, 0, nr), (size_t)nr * sizeof(C), t, T);
#pragma unroll
        for (int e = 0; e < 16; ++e) spec[a][e] = v[e];
    }
    for (int s = 0; q >= 0; ++s) {
        const int b = q / 3, c = q % 3;
        if (__syncthreads_or(!mbar_wait_bounded(bar, (unsigned)(s & 1), flag))) return;
        C v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int k = t + T * e;
            C acc = mkc<C>(0, 0);
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                C S = spec_at(tb + (size_t)a * P, k, H, e >= 8);
                if (c == 2) S = cmul_mi(S);                   // K_phi spectrum = -i S
                acc = cfma(spec[a][e], S, acc);
            }
            v[e] = acc;
        }
        const int qn = next_q(q);
        if (qn >= 0) {
            // every read of this step's spectra precedes the TMA rewrite
            __syncthreads();
            fence_proxy_async();
            issue(qn);
        }
        fft_any<false, LC>(v, L, T, t, xb, tw, eng.template d16<false>());
        C *o = oh + (size_t)(b * 3 + c) * N * nr;
        const uint64_t pl = l2_evict_last();
#pragma unroll
        for (int e = 0; e < 8; ++e) st_hint(o + blk(m, t + T * e, nr), v[e], pl);   // rows 0..nr-1 only
        q = qn;
    }
}

// Column pass, one CTA per column m (LC: compile-time column length, 0 for
// any; ST: staging as above).
template <typename R, int NS, int LC, bool ST>
__global__ void __launch_bounds__(cols_max_threads(NS, sizeof(R) == 8, LC, ST),
                                  cols_min_blocks(NS, sizeof(R) == 8, LC, ST))
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
    static_assert(!ST || sizeof(R) == 4, "per-step staging is FP32 only");
    constexpr bool PAIR = ST;
    if (m == 0) {
        // column 0 keeps its source spectra in the table area (recomputed
        // per step when staging per step)
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
        fft_any<true, LC, true>(v, L, T, t, xb, tw);
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

}  // namespace sg
