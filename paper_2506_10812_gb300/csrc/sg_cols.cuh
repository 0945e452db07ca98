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

// Columns m >= 1 of a plan that stages kernel spectra per step (cols_steps):
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
        fft_any<true, LC>(v, L, T, t, xb, tw, eng.template d16<true>());
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

}  // namespace sg
