// Many independent discs in one persistent launch (the paper evolves one
// disc per run and precomputes its kernel once, Sec. 5.2; here a batch of
// FFT plans, uneven grids, gas-only or gas + dust, is solved together).
// The batch's other engine (configure_streams, host side at the end) does not
// use this kernel: it captures every disc's sg_solve launch chain on forked
// streams of the batch's graph; the autotuner times both engines.
//
// Work decomposition.  A disc's FFT solve has three stages (the arithmetic is
// that of sg_kernels.cu, see its header): row R2C of every source, the
// column pass (forward padded FFT, products with the kernel spectra, inverse
// FFT of every requested output), and the row C2R + epilogue of every
// output.  Each stage is cut into tasks that fill one block: a block of
// `threads` threads runs G = threads / T transforms side by side, T = n / 16
// threads per length-n transform, so a task is G rows (or G columns) of one
// disc.  The host writes the task list once; blocks of the persistent grid
// take tasks in list order from a device counter.  A column task of disc d
// waits until every row task of d has finished; an inverse-row task waits for
// every column task of d.  The list puts every task after the tasks it waits
// for, and a block takes a task only after it has finished its previous one,
// so every awaited task is held by a running block: the waits cannot form a
// cycle, whatever the number of resident blocks.  Each wait is bounded
// (%globaltimer), sets bit 2 of the batch flag and aborts the launch when it
// gives up.
//
// Memory ordering: a finished task's threads fence (gpu scope), the block
// synchronises, and one thread increments the disc's stage counter; the
// waiting thread reads the counter with ld.acquire.gpu and its block
// synchronises before reading.  Data written during the launch (the spectral
// intermediates) is read with ld.global.cg, never through the non-coherent
// path; the kernel spectra, twiddles and inputs are read-only.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sg.h"
#include "sg_fft.cuh"
#include "sg_internal.h"
#include "sg_mem.cuh"

namespace sg {

enum { TASK_FWD = 0, TASK_COL0 = 1, TASK_COL = 2, TASK_INV = 3 };

template <typename R>
struct BatchDisc {
    const R *s[2];                 // sources [nr][nphi]
    cplx<R> *sh;                   // row spectra, [nsrc][N][nr] (sg_mem.cuh layout)
    const cplx<R> *tab;            // kernel spectra of the plan
    cplx<R> *oh;                   // column-pass output, [6][N][nr] (sg_mem.cuh layout)
    R *out[6];                     // outputs by slot 3 b + c (NULL: not requested)
    const R *rcen;                 // r_i
    const cplx<R> *tw_row, *twp_row, *twp_col;
    int nr, nphi, nsrc;
    uint32_t outmask;
    unsigned n_fwd, n_col;         // tasks of stage 0 and 1 (the wait targets)
};

struct BatchArgs {
    const int4 *tasks;             // {type, disc, a (source) or q (slot), tile}
    int ntasks;
    int ndisc;
    unsigned *ctl;                 // [0] next task, [1] abort, [2..] fwd_done[ndisc], col_done[ndisc]
    unsigned *flag;                // bit 1: non-finite output, bit 2: a wait gave up
    int check_finite;
    const unsigned *gate;          // mapped host word, or NULL
    unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_acquire_sys(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait (one thread) until *p >= target.  Gives up after timeout_ns
// of %globaltimer time or 2^25 polls, or when another block has aborted;
// the first to give up sets flag bit 2 and the abort word.
__device__ bool wait_at_least(const unsigned *p, unsigned target, bool sys, const BatchArgs &a)
{
    auto rd = [&]() { return sys ? ld_acquire_sys(p) : ld_acquire_gpu(p); };
    if (rd() >= target) return true;
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    for (int it = 0; it < (1 << 25); ++it) {
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
        if (rd() >= target) return true;
        if (ld_acquire_gpu(a.ctl + 1)) return false;
        if (global_ns() - t0 > a.timeout_ns) break;
    }
    atomicOr(a.flag, 4u);
    atomicExch(a.ctl + 1, 1u);
    return false;
}

// ------------------------------------------------------------ row R2C task
// Rows rb G .. rb G + G - 1 of source `a` (rows past nr recompute row nr - 1
// and store nothing).  Same arithmetic as k_rows_fwd.
template <typename R, int NC>
__device__ void task_fwd(const BatchDisc<R> &D, int a, int rb, unsigned char *smem)
{
    using C = cplx<R>;
    R *red = reinterpret_cast<R *>(smem);
    C *sm = reinterpret_cast<C *>(smem + 64 * sizeof(double));
    const int nr = D.nr, nphi = D.nphi, N = nphi >> 1, T = N >> 4;
    const int G = blockDim.x / T, lg = __ffs(G) - 1;
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    const int i0 = rb * G, iv = min(i0 + g, nr - 1);
    const C *xr = reinterpret_cast<const C *>(D.s[a] + (size_t)iv * nphi);
    C *xb = sm + g * padded_len(N);
    C v[16];
    const R sc = D.rcen[iv];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const C z = __ldg(xr + t + T * e);
        v[e] = mkc<C>(z.x * sc, z.y * sc);
    }
    R s = 0;
#pragma unroll
    for (int e = 0; e < 16; ++e) s += v[e].x + v[e].y;
    const int seg = T < 32 ? T : 32;
    for (int o = seg >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (T > 32) {
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        s = 0;
        const int w0 = (g * T) >> 5, nw = T >> 5;
        for (int w = 0; w < nw; ++w) s += red[w0 + w];
    }
    const R mean = s / (R)nphi;
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = mkc<C>(v[e].x - mean, v[e].y - mean);
    fft_any<true, NC>(v, N, T, t, xb, D.twp_row);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) xb[pidx(t + T * e)] = v[e];
    __syncthreads();
    // fast: T a multiple of 16 and at most 16 rows (column-major layout): the
    // mirrored index, the tile swizzle and the copy addresses are per-thread
    // bases plus multiples of e or of the copy step (as in k_rows_fwd)
    const bool fast = BW == 1 && (T & 15) == 0 && lg <= 4;
    const int sh = lg < 4 ? 4 - lg : 0;
    const int zc0 = (N - t) + (N >> 4) + ((-t) >> 4);             // pidx(N - k) = zc0 - e (T + T/16)
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int k = t + T * e;
        const C Z = v[e];
        if (e == 0 && t == 0) {
            v[e] = mkc<C>(Z.x + Z.y + mean * (R)nphi, Z.x - Z.y);
        } else {
            const C Zc = cconj(xb[fast ? zc0 - e * (T + T / 16) : pidx(N - k)]);
            const C E = cscale(cadd(Z, Zc), (R)0.5);
            const C O = cscale(cmul_mi(csub(Z, Zc)), (R)0.5);
            v[e] = cadd(E, cmul(O, __ldg(&D.tw_row[k])));
        }
    }
    __syncthreads();
    C *out = D.sh + (size_t)a * N * nr;
    const uint64_t pl = l2_evict_last();
    if (fast) {
        const int tb0 = (t << lg) + (g ^ ((t >> sh) & (G - 1)));
#pragma unroll
        for (int e = 0; e < 16; ++e) sm[tb0 + ((T * e) << lg)] = v[e];
        __syncthreads();
        // copy step j: column m0 + j T, row gg (N G = 16 blockDim elements)
        const int x = threadIdx.x, gg = x & (G - 1), m0 = x >> lg;
        const int sb0 = (m0 << lg) + (gg ^ ((m0 >> sh) & (G - 1)));
        if (i0 + gg < nr) {
            C *o0 = out + (size_t)m0 * nr + i0 + gg;
#pragma unroll
            for (int j = 0; j < 16; ++j) st_hint(o0 + (size_t)j * T * nr, sm[sb0 + j * (int)blockDim.x], pl);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) sm[tile_idx_g<C>(t + T * e, g, lg)] = v[e];
        __syncthreads();
        const int per = G * BW;
        for (int idx = threadIdx.x; idx < N * G; idx += blockDim.x) {
            const int bb = idx / per, rem = idx - bb * per;
            const int gg = rem / BW, c = rem - gg * BW;
            if (i0 + gg < nr)
                st_hint(out + ((size_t)bb * nr + i0 + gg) * BW + c, sm[tile_idx_g<C>(bb * BW + c, gg, lg)], pl);
        }
    }
}

// ----------------------------------------------------------- column tasks
template <typename C>
__device__ __forceinline__ C tab_at(const C *col, int k, int H, bool upper, uint64_t pol)
{
    return upper ? cconj(ld_hint(col + 2 * H - k, pol)) : ld_hint(col + k, pol);
}

// Columns cb G + g (1 <= m < N; other groups recompute column N - 1 or 1 and
// store nothing).  Same arithmetic as k_cols.
template <typename R, int NS, int LC>
__device__ void task_col(const BatchDisc<R> &D, int cb, unsigned char *smem)
{
    using C = cplx<R>;
    const int nr = D.nr, N = D.nphi >> 1, L = 2 * nr, T = L >> 4, H = nr, P = tab_pitch(nr);
    const int G = blockDim.x / T;
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    const int m = cb * G + g;
    const bool valid = m >= 1 && m < N;
    const int mv = min(max(m, 1), N - 1);
    C *xb = reinterpret_cast<C *>(smem) + (size_t)g * (padded_len(L) + (NS - 1) * 2 * L);
    C *sspec = xb + padded_len(L);                 // NS == 2: both spectra, own entries only
    const uint64_t pf = l2_evict_first();
    C v[16];
    C spec[NS == 1 ? 16 : 1];
#pragma unroll 1
    for (int a = 0; a < NS; ++a) {
        const C *src = D.sh + (size_t)a * N * nr;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = ld_cg_hint(src + blk(mv, t + T * e, nr), pf);
#pragma unroll
        for (int e = 8; e < 16; ++e) v[e] = mkc<C>(0, 0);
        fft_any<true, LC>(v, L, T, t, xb, D.twp_col);
        if constexpr (NS == 1) {
#pragma unroll
            for (int e = 0; e < 16; ++e) spec[e] = v[e];
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) sspec[a * L + t + T * e] = v[e];
        }
    }
    const uint64_t pl = l2_evict_last();
#pragma unroll 1
    for (int q = 0; q < 3 * NS; ++q) {
        if (!((D.outmask >> q) & 1u)) continue;
        const int b = q / 3, c = q - 3 * b;
        const C *tc[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) tc[a] = D.tab + ((size_t)((a * NS + b) * 3 + c) * (N + 1) + mv) * P;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int k = t + T * e;
            C acc = mkc<C>(0, 0);
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                C S = tab_at(tc[a], k, H, e >= 8, pf);
                if (c == 2) S = cmul_mi(S);
                C Z;
                if constexpr (NS == 1) Z = spec[e];
                else Z = sspec[a * L + k];
                acc = cfma(Z, S, acc);
            }
            v[e] = acc;
        }
        fft_any<false, LC>(v, L, T, t, xb, D.twp_col);
        if (valid) {
            C *o = D.oh + (size_t)q * N * nr;
#pragma unroll
            for (int e = 0; e < 8; ++e) st_hint(o + blk(m, t + T * e, nr), v[e], pl);
        }
    }
}

// Gas + dust column task with two groups per column (G = threads / T >= 2):
// groups 2j and 2j + 1 share column m = cb G/2 + j.  Group 2j + r runs the
// forward transform of source r into the column's shared spectrum buffer,
// then the three outputs of target b = r.  While one output's inverse
// transform runs, the kernel-spectrum columns of its next output (the two
// sources' columns of pair (a, b), component c) are staged into the group's
// shared buffer by 1-D bulk copies on the group's mbarrier.  Same products,
// summation order and transforms as task_col.
//
// Shared memory per column, in complex elements (every region 16-byte
// aligned): 2 (two mbarriers) | 2 x align2(padded_len(L)) (exchange buffers)
// | 2 L (both spectra) | 2 x 2 P (staged kernel spectra).
__host__ __device__ inline size_t col2_elems(int L, int P)
{
    const size_t xbn = (size_t)(padded_len(L) + 1) & ~(size_t)1;
    return 2 + 2 * xbn + 2 * (size_t)L + 4 * (size_t)P;
}

template <typename R, int LC>
__device__ void task_col2(const BatchDisc<R> &D, int cb, unsigned char *smem, unsigned *flag, bool &failed)
{
    using C = cplx<R>;
    const int nr = D.nr, N = D.nphi >> 1, L = 2 * nr, T = L >> 4, H = nr, P = tab_pitch(nr);
    const int G = blockDim.x / T, cpt = G >> 1;
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    const int j = g >> 1, r = g & 1;
    const int m = cb * cpt + j;
    const bool valid = m >= 1 && m < N;
    const int mv = min(max(m, 1), N - 1);
    const size_t xbn = (size_t)(padded_len(L) + 1) & ~(size_t)1;
    C *col = reinterpret_cast<C *>(smem) + (size_t)j * col2_elems(L, P);
    uint64_t *bar = reinterpret_cast<uint64_t *>(col) + r;
    C *xb = col + 2 + r * xbn;
    C *spec = col + 2 + 2 * xbn;
    C *stage = spec + 2 * L + 2 * (size_t)r * P;
    const bool leader = t == 0;
    auto issue = [&](int c) {
        if (leader && ((D.outmask >> (3 * r + c)) & 1u)) {
            const uint64_t pol = l2_evict_first();
            mbar_expect_tx(bar, 2u * P * sizeof(C));
#pragma unroll
            for (int a = 0; a < 2; ++a)
                tma_load_1d(stage + (size_t)a * P, D.tab + ((size_t)((a * 2 + r) * 3 + c) * (N + 1) + mv) * P,
                            P * sizeof(C), bar, pol);
        }
    };
    if (leader) {
        mbar_init(bar, 1);
        fence_proxy_async();                        // the stage held another task's data
    }
    __syncthreads();
    issue(0);                                       // lands during the forward transform
    const uint64_t pf = l2_evict_first();
    C v[16];
    {
        const C *src = D.sh + (size_t)r * N * nr;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = ld_cg_hint(src + blk(mv, t + T * e, nr), pf);
#pragma unroll
        for (int e = 8; e < 16; ++e) v[e] = mkc<C>(0, 0);
    }
    fft_any<true, LC>(v, L, T, t, xb, D.twp_col);
#pragma unroll
    for (int e = 0; e < 16; ++e) spec[(size_t)r * L + t + T * e] = v[e];
    __syncthreads();                                // both spectra complete
    const uint64_t pl = l2_evict_last();
    unsigned ph = 0;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        const int q = 3 * r + c;
        const bool req = (D.outmask >> q) & 1u;
        bool ok = true;
        if (req) ok = mbar_wait_bounded(bar, ph & 1u, flag, 4u);
        if (__syncthreads_or(!ok)) {
            failed = true;                          // a staged copy never landed: give up on this task
            return;
        }
        if (req) ++ph;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int k = t + T * e;
            C acc = mkc<C>(0, 0);
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                C S = e >= 8 ? cconj(stage[(size_t)a * P + 2 * H - k]) : stage[(size_t)a * P + k];
                if (c == 2) S = cmul_mi(S);
                acc = cfma(spec[(size_t)a * L + k], S, acc);
            }
            v[e] = acc;
        }
        __syncthreads();                            // every read of the stage precedes its rewrite
        if (c < 2) {
            if (leader) fence_proxy_async();
            issue(c + 1);
        }
        fft_any<false, LC>(v, L, T, t, xb, D.twp_col);
        if (valid && req) {
            C *o = D.oh + (size_t)q * N * nr;
#pragma unroll
            for (int e = 0; e < 8; ++e) st_hint(o + blk(m, t + T * e, nr), v[e], pl);
        }
    }
    if (leader) mbar_inval(bar);                    // every wait on it has returned
}

// Column m = 0 (the packed m = 0 and m = nphi/2 real columns).  Every group
// computes it; group 0 stores.  Same arithmetic as col0_path.
template <typename R, int NS>
__device__ void task_col0(const BatchDisc<R> &D, unsigned char *smem)
{
    using C = cplx<R>;
    const int nr = D.nr, N = D.nphi >> 1, L = 2 * nr, T = L >> 4, H = nr, P = tab_pitch(nr);
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    C *xb = reinterpret_cast<C *>(smem) + (size_t)g * (padded_len(L) + 2 * L);
    C *spec = xb + padded_len(L);
    C v[16];
    for (int a = 0; a < NS; ++a) {
        const C *col = D.sh + (size_t)a * N * nr;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = ld_cg_hint(col + blk(0, t + T * e, nr), l2_evict_first());
#pragma unroll
        for (int e = 8; e < 16; ++e) v[e] = mkc<C>(0, 0);
        fft_reg<true>(v, L, T, t, xb, D.twp_col);
#pragma unroll
        for (int e = 0; e < 16; ++e) spec[a * L + t + T * e] = v[e];
    }
    __syncthreads();
    for (int q = 0; q < 3 * NS; ++q) {
        if (!((D.outmask >> q) & 1u)) continue;
        const int b = q / 3, c = q - 3 * b;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int k = t + T * e;
            C acc = mkc<C>(0, 0);
            for (int a = 0; a < NS; ++a) {
                const C *t0 = D.tab + ((size_t)((a * NS + b) * 3 + c) * (N + 1)) * P;
                const C *tn = t0 + (size_t)N * P;
                const C Z = spec[a * L + k];
                const C Zm = cconj(spec[a * L + ((L - k) & (L - 1))]);
                C S0 = e >= 8 ? cconj(t0[2 * H - k]) : t0[k];
                C SN = e >= 8 ? cconj(tn[2 * H - k]) : tn[k];
                if (c == 2) {
                    S0 = cmul_mi(S0);
                    SN = cmul_mi(SN);
                }
                acc = cadd(acc, cscale(cadd(cmul(cadd(Z, Zm), S0), cmul(csub(Z, Zm), SN)), (R)0.5));
            }
            v[e] = acc;
        }
        fft_reg<false>(v, L, T, t, xb, D.twp_col);
        if (g == 0) {
            C *o = D.oh + (size_t)q * N * nr;
#pragma unroll
            for (int e = 0; e < 8; ++e) o[blk(0, t + T * e, nr)] = v[e];
        }
    }
}

// ------------------------------------------------- row C2R + epilogue task
// Rows rb G .. of output slot q.  Same arithmetic as k_rows_inv.
template <typename R, int NC>
__device__ void task_inv(const BatchDisc<R> &D, int q, int rb, const BatchArgs &A, unsigned char *smem)
{
    using C = cplx<R>;
    C *sm = reinterpret_cast<C *>(smem + 64 * sizeof(double));
    const int nr = D.nr, nphi = D.nphi, N = nphi >> 1, T = N >> 4;
    const int G = blockDim.x / T, lg = __ffs(G) - 1;
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    const int i0 = rb * G;
    const C *src = D.oh + (size_t)q * N * nr;
    const int per = G * BW;
    // fast: as in task_fwd (per-thread bases)
    const bool fast = BW == 1 && (T & 15) == 0 && lg <= 4;
    const int sh = lg < 4 ? 4 - lg : 0;
    {
        // N G = 16 blockDim elements: 16 loads per thread, all issued first
        const uint64_t pf = l2_evict_first();
        C tmp[16];
        if (fast) {
            const int x = threadIdx.x, gg = x & (G - 1), m0 = x >> lg;
            const C *s0 = src + (size_t)m0 * nr + min(i0 + gg, nr - 1);
#pragma unroll
            for (int j = 0; j < 16; ++j) tmp[j] = ld_cg_hint(s0 + (size_t)j * T * nr, pf);
            const int sb0 = (m0 << lg) + (gg ^ ((m0 >> sh) & (G - 1)));
#pragma unroll
            for (int j = 0; j < 16; ++j) sm[sb0 + j * (int)blockDim.x] = tmp[j];
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int idx = threadIdx.x + j * blockDim.x;
                const int bb = idx / per, rem = idx - bb * per;
                const int gg = rem / BW, c = rem - gg * BW;
                const int row = min(i0 + gg, nr - 1);
                tmp[j] = ld_cg_hint(src + ((size_t)bb * nr + row) * BW + c, pf);
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int idx = threadIdx.x + j * blockDim.x;
                const int bb = idx / per, rem = idx - bb * per;
                const int gg = rem / BW, c = rem - gg * BW;
                sm[tile_idx_g<C>(bb * BW + c, gg, lg)] = tmp[j];
            }
        }
    }
    __syncthreads();
    const int xa0 = (t << lg) + (g ^ ((t >> sh) & (G - 1)));
    const int xc0 = ((N - t) << lg) + (g ^ (((-t) >> sh) & (G - 1)));
    C v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int k = t + T * e;
        const C X = sm[fast ? xa0 + ((T * e) << lg) : tile_idx_g<C>(k, g, lg)];
        if (e == 0 && t == 0) {
            v[e] = mkc<C>(X.x + X.y, X.x - X.y);
        } else {
            const C Xc = cconj(sm[fast ? xc0 - ((T * e) << lg) : tile_idx_g<C>(N - k, g, lg)]);
            v[e] = cadd(cadd(X, Xc), cmul_i(cmulc(csub(X, Xc), __ldg(&D.tw_row[k]))));
        }
    }
    fft_any<false, NC>(v, N, T, t, sm + g * padded_len(N), D.twp_row);
    const int i = i0 + g;
    if (i < nr) {
        const R sc = (q % 3) == 0 ? (R)1 : (R)1 / D.rcen[i];
        C *out = reinterpret_cast<C *>(D.out[q] + (size_t)i * nphi);
        bool bad = false;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const C y = mkc<C>(v[e].x * sc, v[e].y * sc);
            bad |= !(isfinite(y.x) && isfinite(y.y));
            out[t + T * e] = y;
        }
        if (A.check_finite && bad) atomicOr(A.flag, 1u);
    }
}

// ------------------------------------------------------------ L2 prefetch
// One bulk prefetch into L2 (address and size multiples of 16 bytes).
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The read-only data a task reads first: the input rows of a row task; the
// kernel-spectrum columns and the column blocks of the row spectra of a
// column task.  Every range lies inside its buffer; (nr + 2) complex per
// spectrum column, nphi reals per row and nr x 4 complex per column block
// are multiples of 16 bytes.
template <typename R>
__device__ void prefetch_task(const BatchDisc<R> &D, int4 tk, int threads)
{
    using C = cplx<R>;
    const int nr = D.nr, nphi = D.nphi, N = nphi >> 1, L = 2 * nr, P = tab_pitch(nr), ns = D.nsrc;
    if (tk.x == TASK_FWD) {
        const int G = threads / (N >> 4);
        const int i0 = tk.w * G, rows = min(G, nr - i0);
        prefetch_l2(D.s[tk.z] + (size_t)i0 * nphi, (unsigned)((size_t)rows * nphi * sizeof(R)));
    } else if (tk.x == TASK_COL || tk.x == TASK_COL0) {
        const int G0 = threads / (L >> 4);
        const int G = (ns == 2 && G0 >= 2) ? G0 / 2 : G0;             // columns per task
        const int m0 = tk.x == TASK_COL ? tk.w * G : 0;
        const int cols = tk.x == TASK_COL ? min(G, N - m0) : 1;
        for (int q = 0; q < 3 * ns; ++q) {
            if (!((D.outmask >> q) & 1u)) continue;
            const int b = q / 3, c = q - 3 * b;
            for (int a = 0; a < ns; ++a) {
                const C *t0 = D.tab + (size_t)((a * ns + b) * 3 + c) * (N + 1) * P;
                prefetch_l2(t0 + (size_t)m0 * P, (unsigned)((size_t)cols * P * sizeof(C)));
                if (tk.x == TASK_COL0) prefetch_l2(t0 + (size_t)N * P, (unsigned)(P * sizeof(C)));
            }
        }
        const int b0 = m0 / BW, b1 = (m0 + cols - 1) / BW;
        for (int a = 0; a < ns; ++a)
            prefetch_l2(D.sh + (size_t)a * N * nr + (size_t)b0 * nr * BW,
                        (unsigned)((size_t)(b1 - b0 + 1) * nr * BW * sizeof(C)));
    }
}

// ------------------------------------------------------- persistent kernel
// SPEC: the row transforms of nphi = 2048, 4096 and the column transforms of
// length 1024, 2048, 4096 use the compile-time variant of sg_fft.cuh (FP32).
template <typename R, bool SPEC>
__global__ void __launch_bounds__(512) k_batch(const BatchDisc<R> *__restrict__ discs, const __grid_constant__ BatchArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int4 s_task, s_ahead;          // s_ahead: thread 0 only
    unsigned *next = A.ctl, *fwd_done = A.ctl + 2, *col_done = A.ctl + 2 + A.ndisc;
    if (A.gate) {
        if (threadIdx.x == 0) s_task.x = wait_at_least(A.gate, 1u, true, A) ? 0 : -1;
        __syncthreads();
        if (s_task.x < 0) return;
    }
    // Thread 0 holds the next task while the block runs the current one and
    // prefetches its read-only data into L2.  A held task only waits on tasks
    // earlier in the list, and its holder finishes its current (earlier) task
    // first, so holding one task ahead keeps the waits acyclic.
    auto dequeue = [&]() {
        int4 tk = make_int4(-1, 0, 0, 0);
        if (!ld_acquire_gpu(A.ctl + 1)) {
            const unsigned i = atomicAdd(next, 1u);
            if (i < (unsigned)A.ntasks) tk = A.tasks[i];
        }
        return tk;
    };
    if (threadIdx.x == 0) s_ahead = dequeue();
    for (;;) {
        __syncthreads();                        // every thread has read the previous s_task
        if (threadIdx.x == 0) {
            int4 tk = s_ahead;
            const int4 ahead = tk.x >= 0 ? dequeue() : make_int4(-1, 0, 0, 0);
            s_ahead = ahead;
            if (ahead.x >= 0) prefetch_task<R>(discs[ahead.y], ahead, blockDim.x);
            if (tk.x == TASK_COL0 || tk.x == TASK_COL) {
                if (!wait_at_least(fwd_done + tk.y, discs[tk.y].n_fwd, false, A)) tk.x = -1;
            } else if (tk.x == TASK_INV) {
                if (!wait_at_least(col_done + tk.y, discs[tk.y].n_col, false, A)) tk.x = -1;
            }
            s_task = tk;
        }
        __syncthreads();
        const int4 tk = s_task;
        if (tk.x < 0) break;
        const BatchDisc<R> &D = discs[tk.y];
        switch (tk.x) {
        case TASK_FWD:
            if (SPEC && D.nphi == 4096) task_fwd<R, SPEC ? 2048 : 0>(D, tk.z, tk.w, smem_raw);
            else if (SPEC && D.nphi == 2048) task_fwd<R, SPEC ? 1024 : 0>(D, tk.z, tk.w, smem_raw);
            else task_fwd<R, 0>(D, tk.z, tk.w, smem_raw);
            break;
        case TASK_COL0:
            if (D.nsrc == 1) task_col0<R, 1>(D, smem_raw);
            else task_col0<R, 2>(D, smem_raw);
            break;
        case TASK_COL:
            if (D.nsrc == 1) {
                if (SPEC && D.nr == 2048) task_col<R, 1, SPEC ? 4096 : 0>(D, tk.w, smem_raw);
                else if (SPEC && D.nr == 1024) task_col<R, 1, SPEC ? 2048 : 0>(D, tk.w, smem_raw);
                else if (SPEC && D.nr == 512) task_col<R, 1, SPEC ? 1024 : 0>(D, tk.w, smem_raw);
                else task_col<R, 1, 0>(D, tk.w, smem_raw);
            } else if ((int)blockDim.x >= D.nr / 4) {      // two groups per column
                bool failed = false;
                if (SPEC && D.nr == 2048) task_col2<R, SPEC ? 4096 : 0>(D, tk.w, smem_raw, A.flag, failed);
                else if (SPEC && D.nr == 1024) task_col2<R, SPEC ? 2048 : 0>(D, tk.w, smem_raw, A.flag, failed);
                else if (SPEC && D.nr == 512) task_col2<R, SPEC ? 1024 : 0>(D, tk.w, smem_raw, A.flag, failed);
                else task_col2<R, 0>(D, tk.w, smem_raw, A.flag, failed);
                if (failed) {
                    if (threadIdx.x == 0) atomicExch(A.ctl + 1, 1u);
                    return;
                }
            } else {
                if (SPEC && D.nr == 2048) task_col<R, 2, SPEC ? 4096 : 0>(D, tk.w, smem_raw);
                else if (SPEC && D.nr == 1024) task_col<R, 2, SPEC ? 2048 : 0>(D, tk.w, smem_raw);
                else if (SPEC && D.nr == 512) task_col<R, 2, SPEC ? 1024 : 0>(D, tk.w, smem_raw);
                else task_col<R, 2, 0>(D, tk.w, smem_raw);
            }
            break;
        default:
            if (SPEC && D.nphi == 4096) task_inv<R, SPEC ? 2048 : 0>(D, tk.z, tk.w, A, smem_raw);
            else if (SPEC && D.nphi == 2048) task_inv<R, SPEC ? 1024 : 0>(D, tk.z, tk.w, A, smem_raw);
            else task_inv<R, 0>(D, tk.z, tk.w, A, smem_raw);
            break;
        }
        if (tk.x != TASK_INV) {
            __threadfence();                    // this thread's stores, before the count
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(tk.x == TASK_FWD ? fwd_done + tk.y : col_done + tk.y, 1u);
        }
    }
}

}  // namespace sg

// ======================================================================
// Host side
// ======================================================================
using namespace sg;

struct sg_batch {
    int n = 0;
    bool f64 = false;
    int device = 0, sms = 0, max_smem = 0;
    std::vector<sg_plan *> plans;
    std::vector<const void *> sg, sd;
    std::vector<void *> outs;            // 6 per disc
    uint32_t flags = 0;
    unsigned long long timeout_ns = 0;
    sg_batch_opts cfg{};                 // in use
    int grid = 0, ntasks = 0;
    float tuned_ms = 0.f;
    std::vector<sg_batch_opts> tried;    // autotune candidates and their times
    std::vector<float> tried_ms;
    std::vector<sg_tile_trial> tile_trials;   // autotune: launch tiles timed per plan shape
    void *discs = nullptr;               // BatchDisc<R>[n]
    int4 *tasks = nullptr;
    size_t tasks_cap = 0;
    unsigned *ctl = nullptr, *flag = nullptr;
    unsigned *gate_h = nullptr, *gate_d = nullptr;
    cudaStream_t cs = nullptr;           // capture stream
    std::vector<cudaStream_t> ss;        // stream engine: the forked streams
    std::vector<cudaEvent_t> sev;        // ... and their join events (+ the fork event last)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    char err[256] = {0};
};

namespace {

sg_status bfail(sg_batch *b, sg_status s, const char *fmt, ...)
{
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

sg_status bcuda(sg_batch *b, cudaError_t e, const char *what)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

uint32_t batch_outmask(const sg_batch *b, int k)
{
    uint32_t m = 0;
    for (int q = 0; q < 6; ++q)
        if (b->outs[6 * (size_t)k + q]) m |= 1u << q;
    return m;
}

// Columns per column task: one per group, or one per two groups for gas +
// dust when a block holds at least two transforms (task_col2).
int cols_per_task(const sg_plan *pl, int threads)
{
    const int G = threads / (2 * pl->p.nr / 16);
    return (pl->nsrc == 2 && G >= 2) ? G / 2 : G;
}

// Dynamic shared memory of one task of disc k with `threads` threads.
size_t task_smem(const sg_plan *pl, int threads)
{
    const size_t esz = pl->f64 ? 16 : 8;
    const int N = pl->p.nphi / 2, L = 2 * pl->p.nr;
    const int Gr = threads / (N / 16), Gc = threads / (L / 16);
    const size_t rows = 64 * sizeof(double) + (size_t)Gr * padded_len(N) * esz;
    const size_t col = (pl->nsrc == 2 && Gc >= 2)
                           ? (size_t)(Gc / 2) * col2_elems(L, tab_pitch(pl->p.nr)) * esz
                           : (size_t)Gc * (padded_len(L) + (pl->nsrc - 1) * 2 * L) * esz;
    const size_t col0 = (size_t)Gc * (padded_len(L) + 2 * L) * esz;
    return std::max(rows, std::max(col, col0));
}

struct TaskCounts {
    unsigned fwd, col;
};

// Task list of one configuration; descriptors' wait targets filled in.
template <typename R>
void build_tasks(sg_batch *b, int threads, int order, std::vector<BatchDisc<R>> &dd, std::vector<int4> &tasks)
{
    const int n = b->n;
    dd.assign(n, BatchDisc<R>{});
    std::vector<std::vector<int4>> st[3];
    for (auto &v : st) v.assign(n, {});
    for (int k = 0; k < n; ++k) {
        const sg_plan *pl = b->plans[k];
        BatchDisc<R> &D = dd[k];
        const int nr = pl->p.nr, nphi = pl->p.nphi, N = nphi / 2, L = 2 * nr;
        D.s[0] = (const R *)b->sg[k];
        D.s[1] = (const R *)b->sd[k];
        D.sh = (cplx<R> *)pl->sh;
        D.tab = (const cplx<R> *)pl->tab;
        D.oh = (cplx<R> *)pl->oh;
        for (int q = 0; q < 6; ++q) D.out[q] = (R *)b->outs[6 * (size_t)k + q];
        D.rcen = (const R *)pl->rcen;
        D.tw_row = (const cplx<R> *)pl->tw_row;
        D.twp_row = (const cplx<R> *)pl->twp_row;
        D.twp_col = (const cplx<R> *)pl->twp_col;
        D.nr = nr;
        D.nphi = nphi;
        D.nsrc = pl->nsrc;
        D.outmask = batch_outmask(b, k);
        const int Gr = threads / (N / 16), Gc = cols_per_task(pl, threads);
        const int rblocks = (nr + Gr - 1) / Gr;
        const int cblocks = (N + Gc - 1) / Gc;       // tile 0 holds column 0's group (idle) and 1..Gc-1
        for (int a = 0; a < pl->nsrc; ++a)
            for (int r = 0; r < rblocks; ++r) st[0][k].push_back(make_int4(TASK_FWD, k, a, r));
        st[1][k].push_back(make_int4(TASK_COL0, k, 0, 0));
        for (int c = 0; c < cblocks; ++c)
            if (c * Gc + Gc > 1) st[1][k].push_back(make_int4(TASK_COL, k, 0, c));
        for (int q = 0; q < 6; ++q)
            if ((D.outmask >> q) & 1u)
                for (int r = 0; r < rblocks; ++r) st[2][k].push_back(make_int4(TASK_INV, k, q, r));
        D.n_fwd = (unsigned)st[0][k].size();
        D.n_col = (unsigned)st[1][k].size();
    }
    // largest discs first, so that small ones fill the tail
    std::vector<int> ordk(n);
    for (int k = 0; k < n; ++k) ordk[k] = k;
    std::stable_sort(ordk.begin(), ordk.end(), [&](int x, int y) {
        return (long)dd[x].nr * dd[x].nphi * dd[x].nsrc > (long)dd[y].nr * dd[y].nphi * dd[y].nsrc;
    });
    tasks.clear();
    auto put = [&](int s, int k) { tasks.insert(tasks.end(), st[s][k].begin(), st[s][k].end()); };
    if (order == SG_BATCH_ORDER_STAGED) {
        for (int s = 0; s < 3; ++s)
            for (int k : ordk) put(s, k);
    } else {
        for (int j = 0; j < n + 2; ++j) {
            if (j < n) put(0, ordk[j]);
            if (j >= 1 && j - 1 < n) put(1, ordk[j - 1]);
            if (j >= 2) put(2, ordk[j - 2]);
        }
    }
}

template <typename R, bool SPEC>
sg_status configure_k(sg_batch *b, int threads, int ctas_per_sm, int order);

template <typename R>
sg_status configure(sg_batch *b, int threads, int ctas_per_sm, int order, bool spec)
{
    if constexpr (sizeof(R) == 4) {
        if (spec) return configure_k<R, true>(b, threads, ctas_per_sm, order);
    }
    return configure_k<R, false>(b, threads, ctas_per_sm, order);
}

template <typename R, bool SPEC>
sg_status configure_k(sg_batch *b, int threads, int ctas_per_sm, int order)
{
    std::vector<BatchDisc<R>> dd;
    std::vector<int4> tasks;
    build_tasks<R>(b, threads, order, dd, tasks);
    size_t smem = 0;
    for (int k = 0; k < b->n; ++k) smem = std::max(smem, task_smem(b->plans[k], threads));
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, (const void *)k_batch<R, SPEC>);
    if (e != cudaSuccess) return bcuda(b, e, "kernel attributes");
    const int dyn_max = b->max_smem - (int)fa.sharedSizeBytes;     // the kernel's static words come first
    if (smem > (size_t)dyn_max) return bfail(b, SG_ERR_UNSUPPORTED, "batch needs %zu B of shared memory", smem);
    // the device maximum, so that graphs of batches with other sizes stay launchable
    e = cudaFuncSetAttribute((const void *)k_batch<R, SPEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    if (e != cudaSuccess) return bcuda(b, e, "shared-memory limit");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<R, SPEC>, threads, smem);
    if (e != cudaSuccess) return bcuda(b, e, "occupancy");
    if (occ < 1) return bfail(b, SG_ERR_UNSUPPORTED, "batch kernel does not fit on an SM (%zu B)", smem);
    const int cps = (ctas_per_sm <= 0 || ctas_per_sm > occ) ? occ : ctas_per_sm;
    const int grid = std::min((int)tasks.size(), cps * b->sms);

    if (tasks.size() > b->tasks_cap) {
        if (b->tasks) cudaFree(b->tasks);
        b->tasks = nullptr;
        b->tasks_cap = 0;
        e = cudaMalloc((void **)&b->tasks, tasks.size() * sizeof(int4));
        if (e != cudaSuccess) return bcuda(b, e, "task list");
        b->tasks_cap = tasks.size();
    }
    e = cudaMemcpy(b->tasks, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->discs, dd.data(), dd.size() * sizeof(BatchDisc<R>), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(b, e, "task upload");

    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    BatchArgs A{};
    A.tasks = b->tasks;
    A.ntasks = (int)tasks.size();
    A.ndisc = b->n;
    A.ctl = b->ctl;
    A.flag = b->flag;
    A.check_finite = (b->flags & SG_CHECK_FINITE) ? 1 : 0;
    A.gate = (b->flags & SG_BATCH_HOST_GATE) ? b->gate_d : nullptr;
    A.timeout_ns = b->timeout_ns;
    e = cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "graph capture");
    cudaMemsetAsync(b->ctl, 0, (2 + 2 * (size_t)b->n) * sizeof(unsigned), b->cs);
    k_batch<R, SPEC><<<grid, threads, smem, b->cs>>>((const BatchDisc<R> *)b->discs, A);
    cudaError_t le = cudaGetLastError();
    e = cudaStreamEndCapture(b->cs, &b->graph);
    if (le != cudaSuccess) return bcuda(b, le, "batch launch");
    if (e != cudaSuccess) return bcuda(b, e, "graph capture");
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return bcuda(b, e, "graph instantiate");
    b->cfg.threads = threads;
    b->cfg.ctas_per_sm = cps;
    b->cfg.order = order;
    b->cfg.specialize = SPEC ? 1 : 0;
    b->cfg.streams = 0;
    b->grid = grid;
    b->ntasks = (int)tasks.size();
    return SG_OK;
}

// The stream engine: every disc's sg_solve launch chain captured in one graph
// on K forked streams, discs assigned largest first to the least loaded
// stream (load = the disc's model traffic in 4-byte units per cell: sources
// nsrc, row spectra written and read 2 nsrc, kernel spectra nsrc nout,
// column output written and read 2 nout, outputs nout), status words in
// b->flag.
sg_status configure_streams(sg_batch *b, int K)
{
    cudaError_t e = cudaSuccess;
    while ((int)b->ss.size() < K && e == cudaSuccess) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->ss.push_back(st);
    }
    while ((int)b->sev.size() < 65 && e == cudaSuccess) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->sev.push_back(ev);
    }
    if (e != cudaSuccess) return bcuda(b, e, "batch streams");
    std::vector<double> cost(b->n);
    int launches = 0;
    for (int k = 0; k < b->n; ++k) {
        const sg_plan *pl = b->plans[k];
        const uint32_t m = batch_outmask(b, k);
        const int nout = __builtin_popcount(m);
        cost[k] = (double)pl->p.nr * pl->p.nphi * (3 * pl->nsrc + pl->nsrc * nout + 3 * nout);
        launches += m ? 3 : 0;
    }
    std::vector<int> order(b->n);
    for (int k = 0; k < b->n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<std::vector<int>> assign(K);
    std::vector<double> load(K, 0.0);
    for (int k : order) {
        const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        assign[j].push_back(k);
        load[j] += cost[k];
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    const bool finite = (b->flags & SG_CHECK_FINITE) != 0;
    cudaEvent_t fork = b->sev[64];
    e = cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "graph capture");
    sg_status st = SG_OK;
    e = cudaEventRecord(fork, b->cs);
    for (int j = 0; j < K && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(b->ss[j], fork, 0);
    for (int j = 0; j < K && e == cudaSuccess && st == SG_OK; ++j)
        for (int k : assign[j]) {
            st = solve_into(b->plans[k], b->sg[k], b->sd[k], b->outs.data() + 6 * (size_t)k, b->ss[j], b->flag,
                            finite);
            if (st != SG_OK) {
                bfail(b, st, "disc %d: %s", k, sg_last_error(b->plans[k]));
                break;
            }
        }
    for (int j = 0; j < K && e == cudaSuccess; ++j) {
        e = cudaEventRecord(b->sev[j], b->ss[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cs, b->sev[j], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->cs, &g);
    if (st != SG_OK || e != cudaSuccess || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (st != SG_OK) return st;
        return bcuda(b, e != cudaSuccess ? e : ce, "stream-engine capture");
    }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return bcuda(b, e, "graph instantiate");
    b->cfg.threads = b->cfg.ctas_per_sm = b->cfg.order = b->cfg.specialize = 0;
    b->cfg.streams = K;
    b->grid = 0;
    b->ntasks = launches;
    return SG_OK;
}

sg_status configure_any(sg_batch *b, int threads, int cps, int order, bool spec)
{
    return b->f64 ? configure<double>(b, threads, cps, order, false) : configure<float>(b, threads, cps, order, spec);
}

bool threads_fit(const sg_batch *b, int threads)
{
    for (const sg_plan *pl : b->plans)
        if (pl->p.nphi / 32 > threads || 2 * pl->p.nr / 16 > threads) return false;
    return true;
}

// Time the current configuration: median of `reps` solves after 2 warm-ups.
sg_status time_config(sg_batch *b, cudaStream_t s, int reps, float *ms)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> t;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps + 2 && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, s);
        e = cudaGraphLaunch(b->exec, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float x = 0.f;
        if (e == cudaSuccess && r >= 2) {
            cudaEventElapsedTime(&x, e0, e1);
            t.push_back(x);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return bcuda(b, e, "autotune run");
    unsigned f = 0;
    cudaMemcpy(&f, b->flag, sizeof(f), cudaMemcpyDeviceToHost);
    if (f & 6u) return bfail(b, SG_ERR_TIMEOUT, "a device wait gave up while tuning");
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return SG_OK;
}

// Launch tiles per plan shape (nr, nphi, nsrc): every candidate (rows per CTA
// of the tensor-copy row transforms, column staging) timed on the first disc
// of the shape with sg_solve's launch chain alone, median of `reps` solves
// after 2 warm-ups; every disc of the shape then takes the fastest.  Shapes
// whose row transforms do not use tensor copies vary the staging only.
sg_status tune_tiles(sg_batch *b, cudaStream_t s, int reps)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return bcuda(b, e, "tile trials");
    }
    const bool finite = (b->flags & SG_CHECK_FINITE) != 0;
    sg_status st = SG_OK;
    for (int k = 0; k < b->n && st == SG_OK; ++k) {
        sg_plan *pl = b->plans[k];
        auto same = [&](const sg_plan *q) {
            return q->p.nr == pl->p.nr && q->p.nphi == pl->p.nphi && q->nsrc == pl->nsrc;
        };
        bool seen = false;
        for (int j = 0; j < k && !seen; ++j) seen = same(b->plans[j]);
        if (seen) continue;
        sg_tiles t0{};
        sg_get_tiles(pl, &t0);
        const bool rows = rows_tma_eligible(pl->p.nr, pl->p.nphi, pl->f64);
        const size_t first = b->tile_trials.size();
        float best = 0.f;
        sg_tiles bt = t0;
        for (int stg = 0; stg <= (pl->f64 ? 0 : 1) && st == SG_OK; ++stg)
            for (int rf : {2, 4})
                for (int ri : {2, 4}) {
                    if (st != SG_OK) break;
                    if (!rows && (rf != t0.rows_fwd || ri != t0.rows_inv)) continue;
                    const sg_tiles t{rf, ri, stg};
                    const sg_status ts = sg_set_tiles(pl, &t);
                    if (ts == SG_ERR_UNSUPPORTED) continue;   // staging over the shared-memory limit
                    if (ts != SG_OK) {
                        st = bfail(b, ts, "disc %d: %s", k, sg_last_error(pl));
                        break;
                    }
                    std::vector<float> ms;
                    for (int r = 0; r < reps + 2 && st == SG_OK; ++r) {
                        e = cudaEventRecord(e0, s);
                        if (e == cudaSuccess) {
                            st = solve_into(pl, b->sg[k], b->sd[k], b->outs.data() + 6 * (size_t)k, s, b->flag,
                                            finite);
                            if (st != SG_OK) st = bfail(b, st, "disc %d: %s", k, sg_last_error(pl));
                        }
                        if (st == SG_OK && e == cudaSuccess) e = cudaEventRecord(e1, s);
                        if (st == SG_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
                        float x = 0.f;
                        if (st == SG_OK && e == cudaSuccess && r >= 2 && cudaEventElapsedTime(&x, e0, e1) == cudaSuccess)
                            ms.push_back(x);
                        if (e != cudaSuccess) st = bcuda(b, e, "tile trial");
                    }
                    if (st != SG_OK) break;
                    std::sort(ms.begin(), ms.end());
                    const float med = ms.empty() ? 0.f : ms[ms.size() / 2];
                    b->tile_trials.push_back(sg_tile_trial{k, pl->p.nr, pl->p.nphi, pl->nsrc, t, med, 0});
                    if (b->tile_trials.size() == first + 1 || med < best) {
                        best = med;
                        bt = t;
                    }
                }
        if (st != SG_OK) {
            sg_set_tiles(pl, &t0);   // the plan keeps its own tiles when a trial fails
            break;
        }
        for (size_t i = first; i < b->tile_trials.size(); ++i) {
            const sg_tiles &t = b->tile_trials[i].tiles;
            b->tile_trials[i].chosen = t.rows_fwd == bt.rows_fwd && t.rows_inv == bt.rows_inv &&
                                       t.cols_staging == bt.cols_staging;
        }
        for (int j = k; j < b->n && st == SG_OK; ++j)
            if (same(b->plans[j])) {
                const sg_status ts = sg_set_tiles(b->plans[j], &bt);
                if (ts != SG_OK) st = bfail(b, ts, "disc %d: %s", j, sg_last_error(b->plans[j]));
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SG_OK) return st;
    unsigned f = 0;
    e = cudaMemcpy(&f, b->flag, sizeof(f), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "tile trials");
    if (f & 6u) return bfail(b, SG_ERR_TIMEOUT, "a device wait gave up while timing tiles");
    return SG_OK;
}

void batch_free(sg_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cs) cudaStreamDestroy(b->cs);
    for (cudaStream_t st : b->ss) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->sev) cudaEventDestroy(ev);
    void *ptrs[] = {b->discs, b->tasks, b->ctl, b->flag};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (b->gate_h) cudaFreeHost(b->gate_h);
    cudaGetLastError();
}

}  // namespace

extern "C" {

sg_status sg_batch_create(sg_batch **out, sg_plan *const *plans, int32_t n, const void *const *sigma_g,
                          const void *const *sigma_d, void *const *outs, const sg_batch_opts *opts, void *stream)
{
    if (!out) return SG_ERR_ARG;
    *out = nullptr;
    if (!plans || n < 1 || !sigma_g || !outs) return SG_ERR_ARG;
    sg_batch_opts o{};
    if (opts) o = *opts;
    auto reject = [&](sg_status s, const char *msg, int k) {
        fprintf(stderr, "sg_batch_create: disc %d: %s\n", k, msg);
        return s;
    };
    for (int k = 0; k < n; ++k) {
        const sg_plan *pl = plans[k];
        if (!pl) return reject(SG_ERR_ARG, "NULL plan", k);
        if (pl->p.method != SG_METHOD_FFT) return reject(SG_ERR_ARG, "batches take FFT plans only", k);
        if (pl->f64 != plans[0]->f64) return reject(SG_ERR_ARG, "mixed dtypes", k);
        if (pl->device != plans[0]->device) return reject(SG_ERR_ARG, "plans on different devices", k);
        if (!sigma_g[k]) return reject(SG_ERR_ARG, "sigma_g is NULL", k);
        if (pl->nsrc == 2 && (!sigma_d || !sigma_d[k])) return reject(SG_ERR_ARG, "bi-fluid plan needs sigma_d", k);
        if (pl->nsrc == 1)
            for (int q = 3; q < 6; ++q)
                if (outs[6 * (size_t)k + q]) return reject(SG_ERR_ARG, "dust output of a gas-only plan", k);
        // the transforms move element pairs: every buffer aligned to two elements
        const uintptr_t amask = 2 * pl->esz - 1;
        bool mis = ((uintptr_t)sigma_g[k] & amask) || (pl->nsrc == 2 && ((uintptr_t)sigma_d[k] & amask));
        for (int q = 0; q < 6; ++q) mis |= ((uintptr_t)outs[6 * (size_t)k + q] & amask) != 0;
        if (mis) return reject(SG_ERR_ARG, "a buffer is not aligned to two elements", k);
    }
    if (o.threads != 0 && o.threads != 256 && o.threads != 512) return reject(SG_ERR_ARG, "threads must be 256 or 512", -1);
    if (o.order != SG_BATCH_ORDER_PIPELINED && o.order != SG_BATCH_ORDER_STAGED)
        return reject(SG_ERR_ARG, "unknown order", -1);
    if (!(o.timeout_ms >= 0) || o.timeout_ms > 600000) return reject(SG_ERR_ARG, "timeout_ms out of range", -1);
    if (o.streams < 0 || o.streams > 64) return reject(SG_ERR_ARG, "streams must be 0..64", -1);
    if (o.streams > 0 && (o.flags & SG_BATCH_HOST_GATE))
        return reject(SG_ERR_ARG, "the host gate needs the persistent engine (streams = 0)", -1);

    sg_batch *b = new (std::nothrow) sg_batch();
    if (!b) return SG_ERR_OOM;
    b->n = n;
    b->f64 = plans[0]->f64;
    b->device = plans[0]->device;
    b->plans.assign(plans, plans + n);
    b->sg.assign(sigma_g, sigma_g + n);
    b->sd.assign(n, nullptr);
    for (int k = 0; k < n; ++k)
        if (plans[k]->nsrc == 2) b->sd[k] = sigma_d[k];
    b->outs.assign(outs, outs + 6 * (size_t)n);
    b->flags = o.flags;
    b->timeout_ns = (unsigned long long)((o.timeout_ms > 0 ? o.timeout_ms : 2000.0) * 1e6);
    auto bad = [&](sg_status st) {
        fprintf(stderr, "sg_batch_create: %s\n", b->err);
        batch_free(b);
        delete b;
        return st;
    };
    cudaError_t e = cudaSetDevice(b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    if (e != cudaSuccess) return bad(bcuda(b, e, "device query"));
    const size_t dsz = b->f64 ? sizeof(BatchDisc<double>) : sizeof(BatchDisc<float>);
    e = cudaMalloc(&b->discs, dsz * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->ctl, (2 + 2 * (size_t)n) * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->flag, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->flag, 0, sizeof(unsigned));
    if (e == cudaSuccess && (o.flags & SG_BATCH_HOST_GATE)) {
        e = cudaHostAlloc((void **)&b->gate_h, sizeof(unsigned), cudaHostAllocMapped);
        if (e == cudaSuccess) {
            *(volatile unsigned *)b->gate_h = 0u;
            e = cudaHostGetDevicePointer((void **)&b->gate_d, b->gate_h, 0);
        }
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bad(bcuda(b, e, "batch allocation"));
    // the plans' tables were built on their own streams; the batch reads them
    e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return bad(bcuda(b, e, "stream sync"));

    sg_status st;
    if (o.autotune && !(o.flags & SG_BATCH_HOST_GATE)) {
        // the plans' launch tiles first: the stream engine's chains use them
        st = tune_tiles(b, (cudaStream_t)stream, 5);
        if (st != SG_OK) return bad(st);
        float best = 0.f;
        sg_batch_opts bc{};
        bool have = false;
        for (int spec = 0; spec <= (b->f64 ? 0 : 1); ++spec)
        for (int threads : {256, 512}) {
            if (!threads_fit(b, threads)) continue;
            for (int order : {SG_BATCH_ORDER_PIPELINED, SG_BATCH_ORDER_STAGED}) {
                for (int cps = 1; cps <= 8; ++cps) {
                    st = configure_any(b, threads, cps, order, spec != 0);
                    if (st == SG_ERR_UNSUPPORTED) break;
                    if (st != SG_OK) return bad(st);
                    if (b->cfg.ctas_per_sm < cps) break;     // past the occupancy maximum
                    float ms = 0.f;
                    st = time_config(b, (cudaStream_t)stream, 5, &ms);
                    if (st != SG_OK) return bad(st);
                    b->tried.push_back(b->cfg);
                    b->tried_ms.push_back(ms);
                    if (!have || ms < best) {
                        best = ms;
                        bc = b->cfg;
                        have = true;
                    }
                }
            }
        }
        for (int K : {2, 4, 8, 16, 32}) {
            if (K > 2 * b->n) break;
            st = configure_streams(b, std::min(K, b->n));
            if (st != SG_OK) return bad(st);
            float ms = 0.f;
            st = time_config(b, (cudaStream_t)stream, 5, &ms);
            if (st != SG_OK) return bad(st);
            b->tried.push_back(b->cfg);
            b->tried_ms.push_back(ms);
            if (!have || ms < best) {
                best = ms;
                bc = b->cfg;
                have = true;
            }
            if (K >= b->n) break;
        }
        if (!have) return bad(bfail(b, SG_ERR_UNSUPPORTED, "no batch configuration fits (transforms too long)"));
        st = bc.streams ? configure_streams(b, bc.streams)
                        : configure_any(b, bc.threads, bc.ctas_per_sm, bc.order, bc.specialize != 0);
        if (st != SG_OK) return bad(st);
        b->cfg.autotune = 1;
        b->tuned_ms = best;
    } else if (o.streams > 0) {
        st = configure_streams(b, o.streams);
        if (st != SG_OK) return bad(st);
    } else {
        const int threads = o.threads ? o.threads : 256;
        if (!threads_fit(b, threads))
            return bad(bfail(b, SG_ERR_UNSUPPORTED, "a transform is longer than 16 x %d threads", threads));
        st = configure_any(b, threads, o.ctas_per_sm, o.order, o.specialize != 0);
        if (st != SG_OK) return bad(st);
    }
    b->cfg.flags = b->flags;
    b->cfg.timeout_ms = (double)b->timeout_ns * 1e-6;
    e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemset(b->flag, 0, sizeof(unsigned));
    if (e != cudaSuccess) return bad(bcuda(b, e, "batch setup"));
    *out = b;
    return SG_OK;
}

sg_status sg_batch_solve(sg_batch *b, void *stream)
{
    if (!b) return SG_ERR_ARG;
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bcuda(b, e, "set device");
    if (b->gate_h) *(volatile unsigned *)b->gate_h = 0u;
    e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return bcuda(b, e, "graph launch");
    return SG_OK;
}

sg_status sg_batch_solve_loop(sg_batch *b, void *stream)
{
    if (!b) return SG_ERR_ARG;
    for (int k = 0; k < b->n; ++k) {
        void *const *o = b->outs.data() + 6 * (size_t)k;
        sg_status st = sg_solve(b->plans[k], b->sg[k], b->sd[k], o[0], o[1], o[2], o[3], o[4], o[5], stream);
        if (st != SG_OK) return bfail(b, st, "disc %d: %s", k, sg_last_error(b->plans[k]));
    }
    return SG_OK;
}

sg_status sg_batch_release(sg_batch *b)
{
    if (!b) return SG_ERR_ARG;
    if (!b->gate_h) return bfail(b, SG_ERR_ARG, "batch was created without SG_BATCH_HOST_GATE");
    __atomic_store_n(b->gate_h, 1u, __ATOMIC_SEQ_CST);
    return SG_OK;
}

sg_status sg_batch_sync(sg_batch *b, void *stream)
{
    if (!b) return SG_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return bcuda(b, e, "stream sync");
    unsigned f = 0;
    e = cudaMemcpy(&f, b->flag, sizeof(f), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && f) e = cudaMemset(b->flag, 0, sizeof(unsigned));
    if (e != cudaSuccess) return bcuda(b, e, "flag read");
    // bit 4: a wait of the persistent kernel; bit 2: a staged copy of a per-disc chain
    if (f & 6u) return bfail(b, SG_ERR_TIMEOUT, "a device-side wait gave up (outputs incomplete)");
    if (f & 1u) return bfail(b, SG_ERR_NONFINITE, "non-finite output");
    return SG_OK;
}

sg_status sg_batch_config(const sg_batch *b, sg_batch_opts *opts, int32_t *grid, int32_t *ntasks, float *tuned_ms)
{
    if (!b) return SG_ERR_ARG;
    if (opts) *opts = b->cfg;
    if (grid) *grid = b->grid;
    if (ntasks) *ntasks = b->ntasks;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    return SG_OK;
}

int32_t sg_batch_tune_results(const sg_batch *b, int32_t max, sg_batch_opts *cfgs, float *ms)
{
    if (!b) return -1;
    const int n = (int)b->tried.size();
    for (int i = 0; i < n && i < max; ++i) {
        if (cfgs) cfgs[i] = b->tried[i];
        if (ms) ms[i] = b->tried_ms[i];
    }
    return n;
}

int32_t sg_batch_tile_trials(const sg_batch *b, int32_t max, sg_tile_trial *out)
{
    if (!b) return -1;
    const int n = (int)b->tile_trials.size();
    for (int i = 0; i < n && i < max && out; ++i) out[i] = b->tile_trials[i];
    return n;
}

void sg_batch_destroy(sg_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    batch_free(b);
    delete b;
}

const char *sg_batch_last_error(const sg_batch *b) { return b ? b->err : ""; }

}  // extern "C"
