// Kernels of the spectral neural-operator surrogate (the learned form of the
// Sec. 5.2 field solve): a batched BF16 tensor-core GEMM with FP32
// accumulation, the per-mode complex channel mixing of the spectral
// convolutions, and the elementwise pieces of training (GELU, casts, bias
// gradients, relative-L2 loss, Adam).  All device buffers are caller-owned;
// shapes and layouts are stated per entry point in sg.h.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <atomic>
#include <type_traits>

#include "sg.h"
#include "sg_mem.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 32;   // CTA tile; 4 warps of 32 x 32
constexpr int SK = BK + 8;                 // padded row of the K-contiguous shared tiles (bf16)

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C[z] = alpha op(A[z]) B[z] + beta C[z] (+ bias[n]); op(A) = A ([M][K]) or
// A^T (A stored [K][M]); B [K][N]; all row-major with leading dimensions lda,
// ldb, ldc; batch strides sa, sb, sc (elements; 0 broadcasts).  Shared tiles
// hold A as [m][k] and B as [n][k] (K contiguous) so every fragment register
// is one 32-bit load.
template <bool TA>
__global__ void __launch_bounds__(128)
k_gemm(int M, int N, int K, float alpha, const __nv_bfloat16 *__restrict__ A, int lda, long long sa,
       const __nv_bfloat16 *__restrict__ B, int ldb, long long sb, float beta, float *__restrict__ C, int ldc,
       long long sc, __nv_bfloat16 *__restrict__ Cb, const float *__restrict__ bias, int vecA, int vecB)
{
    __shared__ __align__(16) __nv_bfloat16 As[BM][SK];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][SK];
    const int z = blockIdx.z;
    A += z * sa;
    B += z * sb;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, q = lane & 3;
    float acc[2][4][4] = {};
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += BK) {
        // A tile: BM x BK.  vecA: 8 consecutive elements along the stored
        // row (k for A, m for A^T) per 16-byte load where fully in range.
        if (vecA) {
            for (int i = tid; i < BM * BK / 8; i += 128) {
                int m, k;
                if (TA) {
                    m = (i % (BM / 8)) * 8;
                    k = i / (BM / 8);
                } else {
                    k = (i % (BK / 8)) * 8;
                    m = i / (BK / 8);
                }
                const int gm = m0 + m, gk = k0 + k;
                if (TA) {
                    if (gk < K && gm + 8 <= M) {
                        const uint4 u = *reinterpret_cast<const uint4 *>(A + (size_t)gk * lda + gm);
                        const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&u);
#pragma unroll
                        for (int j = 0; j < 8; ++j) As[m + j][k] = e[j];
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) As[m + j][k] = (gk < K && gm + j < M) ? A[(size_t)gk * lda + gm + j] : zero;
                    }
                } else {
                    if (gm < M && gk + 8 <= K) {
                        *reinterpret_cast<uint4 *>(&As[m][k]) = *reinterpret_cast<const uint4 *>(A + (size_t)gm * lda + gk);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) As[m][k + j] = (gm < M && gk + j < K) ? A[(size_t)gm * lda + gk + j] : zero;
                    }
                }
            }
        } else {
            for (int i = tid; i < BM * BK; i += 128) {
                int m, k;
                if (TA) {                   // A stored [K][M]: m fastest for coalescing
                    m = i % BM;
                    k = i / BM;
                } else {
                    k = i % BK;
                    m = i / BK;
                }
                const int gm = m0 + m, gk = k0 + k;
                __nv_bfloat16 v = zero;
                if (gm < M && gk < K) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
                As[m][k] = v;
            }
        }
        // B tile: BK x BN stored [n][k]
        if (vecB) {
            for (int i = tid; i < BK * BN / 8; i += 128) {
                const int n = (i % (BN / 8)) * 8, k = i / (BN / 8);
                const int gn = n0 + n, gk = k0 + k;
                if (gk < K && gn + 8 <= N) {
                    const uint4 u = *reinterpret_cast<const uint4 *>(B + (size_t)gk * ldb + gn);
                    const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&u);
#pragma unroll
                    for (int j = 0; j < 8; ++j) Bs[n + j][k] = e[j];
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) Bs[n + j][k] = (gk < K && gn + j < N) ? B[(size_t)gk * ldb + gn + j] : zero;
                }
            }
        } else {
            for (int i = tid; i < BK * BN; i += 128) {
                const int n = i % BN, k = i / BN;
                const int gn = n0 + n, gk = k0 + k;
                Bs[n][k] = (gn < N && gk < K) ? B[(size_t)gk * ldb + gn] : zero;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + g;
                af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * q]);
                af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * q]);
                af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * q + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * q + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + g;
                bf[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 2 * q]);
                bf[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 2 * q + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    mma_bf16(acc[i][j], af[i][0], af[i][1], af[i][2], af[i][3], bf[j][0], bf[j][1]);
        }
        __syncthreads();
    }
    if (C) C += z * sc;
    if (Cb) Cb += z * sc;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int m = m0 + wm + i * 16 + g + (h >= 2 ? 8 : 0);
                const int n = n0 + wn + j * 8 + 2 * q + (h & 1);
                if (m < M && n < N) {
                    float v = alpha * acc[i][j][h];
                    if (bias) v += bias[n];
                    if (C) {
                        float *p = C + (size_t)m * ldc + n;
                        if (beta != 0.f) v += beta * *p;
                        *p = v;
                    }
                    if (Cb) Cb[(size_t)m * ldc + n] = __float2bfloat16(v);
                }
            }
}

// ----------------------------------------------------------------------
// The same GEMM on the tcgen05 tensor cores.  One CTA of 128 threads owns a
// 128 x BN tile of C (BN = 32, 64 or 128) and walks K in steps of 64: every
// thread loads part of the A and B tiles into registers, stores them into
// shared memory in the K-major core-matrix layout the tensor core reads
// (transposing B, and A^T, 8 x 8 blocks in registers), and one thread issues
// four 128 x BN x 16 BF16 products accumulating in FP32 in tensor memory and
// commits them to the stage's mbarrier.  Two shared-memory stages: the loads
// of step s + 1 run while the products of step s do.  The epilogue reads
// each thread's row of the accumulator (warp w: rows 32 w .. 32 w + 31)
// and applies alpha, bias and beta.
//
// Tile layout: row r, K chunk c (8 elements, 16 bytes) at
//   (r / 8) SBO + c LBO + (r % 8) 16 bytes,  LBO = 144, SBO = 8 LBO + 16,
// i.e. core matrices of 8 rows x 16 bytes, padded so that the row-per-lane
// stores of A and the block-per-thread stores of B are free of bank
// conflicts.
constexpr int TC_BM = 128, TC_BK = 64, TC_LBO = 144, TC_SBO = 8 * TC_LBO + 16;

__device__ unsigned g_nn_flag;   // bit 0: a tensor-core wait gave up

__host__ __device__ constexpr unsigned tc_tile_bytes(int rows) { return (unsigned)(rows / 8) * TC_SBO; }
__host__ __device__ constexpr unsigned tc_stage_bytes(int bn) { return tc_tile_bytes(TC_BM) + tc_tile_bytes(bn); }
// NST stages, or the epilogue's FP32 tile (row stride bn + 4) if larger;
// then two mbarriers and the tensor-memory address
__host__ __device__ constexpr unsigned tc_data_bytes(int bn, int nst)
{
    return nst * tc_stage_bytes(bn) > (unsigned)TC_BM * (bn + 4) * 4 ? nst * tc_stage_bytes(bn)
                                                                     : (unsigned)TC_BM * (bn + 4) * 4;
}
__host__ __device__ constexpr unsigned tc_smem_bytes(int bn, int nst) { return tc_data_bytes(bn, nst) + 32; }
// resident CTAs per SM the launch bounds aim at (shared memory allows them;
// tensor memory: at most 512 columns in all)
__host__ __device__ constexpr int tc_min_blocks(int bn, int nst)
{
    return nst == 1 ? (bn == 32 ? 6 : bn == 64 ? 5 : 3) : (bn == 128 ? 3 : 4);
}
__device__ __forceinline__ unsigned tc_off(int r, int c) { return (r >> 3) * TC_SBO + c * TC_LBO + (r & 7) * 16; }

__device__ __forceinline__ uint32_t word_of(const uint4 &u, int w)
{
    return w == 0 ? u.x : w == 1 ? u.y : w == 2 ? u.z : u.w;
}
__device__ __forceinline__ void set_word(uint4 &u, int w, uint32_t v)
{
    if (w == 0) u.x = v;
    else if (w == 1) u.y = v;
    else if (w == 2) u.z = v;
    else u.w = v;
}
// 8 x 8 transpose of 16-bit elements: r[i] holds elements 0..7 of row i,
// o[j] receives element j of rows 0..7 (lower address first).
__device__ __forceinline__ void transpose8x8(const uint4 (&r)[8], uint4 (&o)[8])
{
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint32_t a = word_of(r[2 * p], w), b = word_of(r[2 * p + 1], w);
            set_word(o[2 * w], p, __byte_perm(a, b, 0x5410));
            set_word(o[2 * w + 1], p, __byte_perm(a, b, 0x7632));
        }
}

// 8 consecutive bf16 of a row at (row, col) of a row-major matrix with
// leading dimension ld, zero outside rows < nrow, cols < ncol; vec: 16-byte
// loads allowed where the 8 are in range.
__device__ __forceinline__ uint4 ld8(const __nv_bfloat16 *__restrict__ X, int ld, int row, int col, int nrow,
                                     int ncol, int vec)
{
    uint4 u = make_uint4(0, 0, 0, 0);
    if (row >= nrow || col >= ncol) return u;
    const __nv_bfloat16 *p = X + (size_t)row * ld + col;
    if (vec && col + 8 <= ncol) return __ldg(reinterpret_cast<const uint4 *>(p));
    unsigned short e[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) e[j] = col + j < ncol ? __bfloat16_as_ushort(p[j]) : (unsigned short)0;
    u.x = e[0] | ((uint32_t)e[1] << 16);
    u.y = e[2] | ((uint32_t)e[3] << 16);
    u.z = e[4] | ((uint32_t)e[5] << 16);
    u.w = e[6] | ((uint32_t)e[7] << 16);
    return u;
}

template <bool TA, int BN, int NST, bool FOLD = false>
__global__ void __launch_bounds__(128, tc_min_blocks(BN, NST))
k_gemm_tc(int M, int N, int K, float alpha, const __nv_bfloat16 *__restrict__ A, int lda, long long sa,
          const __nv_bfloat16 *__restrict__ B, int ldb, long long sb, float beta, float *__restrict__ C, int ldc,
          long long sc, __nv_bfloat16 *__restrict__ Cb, const float *__restrict__ bias, int vecA, int vecB,
          int batch, int fold)
{
    using namespace sg;
    extern __shared__ __align__(128) unsigned char sm[];
    constexpr unsigned AB = tc_tile_bytes(TC_BM), ST = tc_stage_bytes(BN);
    constexpr uint32_t IDESC = umma_idesc(TC_BM, BN, 1);
    static_assert(NST == 1 || NST == 2, "one or two shared-memory stages");
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + tc_data_bytes(BN, NST));
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + tc_data_bytes(BN, NST) + 16);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // fold > 1 (A shared by the batch, N % 8 == 0): the tile's columns are
    // `fold` consecutive batch entries side by side, column nn = (nn / N)-th
    // entry, its column nn % N; otherwise one batch entry per CTA.
    static_assert(!FOLD || BN == 128, "folded tiles are 128 columns wide");
    const int m0 = blockIdx.x * TC_BM;
    const int z0 = FOLD ? blockIdx.z * fold : blockIdx.z, n0 = FOLD ? 0 : blockIdx.y * BN;
    A += z0 * sa;
    if (warp == 0) {
        tmem_alloc(tslot, BN);
        tmem_relinquish();
    }
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = *tslot;
    const unsigned sbase = smem_u32(sm);

    // Per-thread share of a stage.  A ([M][K]): the thread's row 32 warp +
    // lane, its 8 chunks of 8 k.  A^T ([K][M]) and B ([K][N]): one 8 k x 8
    // m (or n) block, transposed; thread (blk, kc) = (t / 8, t % 8).
    constexpr int NBB = BN;                 // B blocks per stage: BN / 8 n-blocks x 8 k-chunks
    uint4 ra[8], rb[8];
    const int kc = t & 7, blk = t >> 3;
    auto load = [&](int s) {
        const int k0 = s * TC_BK;
        if constexpr (!TA) {
            const int r = m0 + 32 * warp + lane;
#pragma unroll
            for (int c = 0; c < 8; ++c) ra[c] = ld8(A, lda, r, k0 + 8 * c, M, K, vecA);
        } else {
            // A^T block: rows k0 + 8 kc .. + 7 of the stored [K][M], columns m0 + 8 blk .. + 7
#pragma unroll
            for (int i = 0; i < 8; ++i) ra[i] = ld8(A, lda, k0 + 8 * kc + i, m0 + 8 * blk, K, M, vecA);
        }
        if (t < NBB) {
            int zb = z0, col = n0 + 8 * blk;
            if constexpr (FOLD) {
                zb = z0 + (8 * blk) / N;
                col = (8 * blk) % N;
            }
            const bool live = !FOLD || (8 * blk < fold * N && zb < batch);
            const __nv_bfloat16 *Bz = B + zb * sb;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                rb[i] = live ? ld8(Bz, ldb, k0 + 8 * kc + i, col, K, N, vecB) : make_uint4(0, 0, 0, 0);
        }
    };
    auto store = [&](int b) {
        unsigned char *sa_ = sm + b * ST, *sb_ = sa_ + AB;
        if constexpr (!TA) {
            const int r = 32 * warp + lane;
#pragma unroll
            for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4 *>(sa_ + tc_off(r, c)) = ra[c];
        } else {
            uint4 o[8];
            transpose8x8(ra, o);
#pragma unroll
            for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4 *>(sa_ + tc_off(8 * blk + j, kc)) = o[j];
        }
        if (t < NBB) {
            uint4 o[8];
            transpose8x8(rb, o);
#pragma unroll
            for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4 *>(sb_ + tc_off(8 * blk + j, kc)) = o[j];
        }
    };

    const int S = (K + TC_BK - 1) / TC_BK;
    bool ok = true;
    load(0);
    for (int s = 0; s < S; ++s) {
        const int b = s % NST;
        // the products of step s - NST read this buffer
        if (s >= NST) ok = mbar_wait_bounded(&bar[b], (unsigned)(((s - NST) / NST) & 1), &g_nn_flag, 1u);
        if (__syncthreads_or(!ok)) break;
        store(b);
        fence_proxy_async();               // generic-proxy stores, visible to the tensor core
        __syncthreads();
        if (t == 0) {
            tmem_fence_after();
            const unsigned a0 = sbase + b * ST, b0 = a0 + AB;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk)
                umma_ss(tmem, umma_sdesc(a0 + 2 * kk * TC_LBO, TC_LBO, TC_SBO),
                        umma_sdesc(b0 + 2 * kk * TC_LBO, TC_LBO, TC_SBO), IDESC, (s > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&bar[b]);
        }
        if (s + 1 < S) load(s + 1);
    }
    // every product of the tile (the last commit covers all earlier ones)
    if (ok) ok = mbar_wait_bounded(&bar[(S - 1) % NST], (unsigned)(((S - 1) / NST) & 1), &g_nn_flag, 1u);
    if (!ok && NST == 2 && S >= 2)   // let the other stage's products finish before the memory is released
        mbar_wait_bounded(&bar[(S - 2) % NST], (unsigned)(((S - 2) / NST) & 1), &g_nn_flag, 1u);
    ok = !__syncthreads_or(!ok);
    tmem_fence_after();
    if (ok) {
        // The products are complete, so the stage buffers are free: each
        // warp moves its 32 accumulator rows there (row stride BN + 4 floats,
        // conflict-free), then the CTA writes the tile out row by row with
        // consecutive threads on consecutive columns.
        constexpr int PS = BN + 4, CPR = BN / 4;
        float *stg = reinterpret_cast<float *>(sm);
        const int r = 32 * warp + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            float v[32];
            tmem_ld32f(tmem + ((uint32_t)(32 * warp) << 16) + c0, v);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<float4 *>(stg + r * PS + c0 + 4 * j) =
                    make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
        __syncthreads();
        const bool vc = (ldc & 3) == 0 && (!C || ((uintptr_t)C & 15) == 0) && (!Cb || ((uintptr_t)Cb & 7) == 0) &&
                        (sc & 3) == 0;
        // output column nn of the tile -> (batch entry, column)
        auto where = [&](int nn, int &zz, int &n) {
            if constexpr (FOLD) {
                zz = nn < fold * N ? z0 + nn / N : batch;
                n = nn % N;
            } else {
                zz = z0;
                n = n0 + nn;
            }
        };
        // groups of G float4 per thread: the old C values of a group are
        // loaded first, so that their loads are in flight together
        constexpr int G = BN == 32 ? 4 : 8;
#pragma unroll 1
        for (int g0 = 0; g0 < CPR; g0 += G) {
            float4 old[G];
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int i = t + 128 * (g0 + u), rr = i / CPR, c4 = i - rr * CPR;
                int zz, n;
                where(4 * c4, zz, n);
                const int m = m0 + rr;
                old[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (C && beta != 0.f && vc && g0 + u < CPR && m < M && n + 4 <= N && zz < batch)
                    old[u] = *reinterpret_cast<const float4 *>(C + zz * sc + (size_t)m * ldc + n);
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
                if (g0 + u >= CPR) break;
                const int i = t + 128 * (g0 + u), rr = i / CPR, c4 = i - rr * CPR;
                int zz, n;
                where(4 * c4, zz, n);
                const int m = m0 + rr;
                if (m >= M || n >= N || zz >= batch) continue;
                float *Cz = C ? C + zz * sc : nullptr;
                __nv_bfloat16 *Cbz = Cb ? Cb + zz * sc : nullptr;
                const float4 a = *reinterpret_cast<const float4 *>(stg + rr * PS + 4 * c4);
                float x[4] = {alpha * a.x, alpha * a.y, alpha * a.z, alpha * a.w};
                if (vc && n + 4 <= N) {
                    if (bias) {
                        if (((uintptr_t)bias & 15) == 0) {   // n is a multiple of 4
                            const float4 bv = __ldg(reinterpret_cast<const float4 *>(bias + n));
                            x[0] += bv.x;
                            x[1] += bv.y;
                            x[2] += bv.z;
                            x[3] += bv.w;
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j) x[j] += __ldg(bias + n + j);
                        }
                    }
                    if (Cz) {
                        if (beta != 0.f) {
                            x[0] += beta * old[u].x;
                            x[1] += beta * old[u].y;
                            x[2] += beta * old[u].z;
                            x[3] += beta * old[u].w;
                        }
                        *reinterpret_cast<float4 *>(Cz + (size_t)m * ldc + n) = make_float4(x[0], x[1], x[2], x[3]);
                    }
                    if (Cbz) {
                        __nv_bfloat162 lo = __floats2bfloat162_rn(x[0], x[1]), hi = __floats2bfloat162_rn(x[2], x[3]);
                        uint2 w;
                        w.x = *reinterpret_cast<uint32_t *>(&lo);
                        w.y = *reinterpret_cast<uint32_t *>(&hi);
                        *reinterpret_cast<uint2 *>(Cbz + (size_t)m * ldc + n) = w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (n + j >= N) break;
                        float y = x[j];
                        if (bias) y += __ldg(bias + n + j);
                        if (Cz) {
                            float *p = Cz + (size_t)m * ldc + n + j;
                            if (beta != 0.f) y += beta * *p;
                            *p = y;
                        }
                        if (Cbz) Cbz[(size_t)m * ldc + n + j] = __float2bfloat16(y);
                    }
                }
            }
        }
    }
    tmem_fence_before();
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after();
        tmem_dealloc(tmem, BN);
    }
}

int g_gemm_engine = SG_NN_GEMM_TCGEN05;

}  // namespace

extern "C" sg_status sg_nn_set_gemm_engine(int32_t engine)
{
    if (engine != SG_NN_GEMM_TCGEN05 && engine != SG_NN_GEMM_MMA_SYNC) return SG_ERR_ARG;
    g_gemm_engine = engine;
    return SG_OK;
}

extern "C" sg_status sg_nn_check(void *stream)
{
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    unsigned f = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&f, g_nn_flag, sizeof(f));
    const unsigned zero = 0;
    if (e == cudaSuccess && f) e = cudaMemcpyToSymbol(g_nn_flag, &zero, sizeof(zero));
    if (e != cudaSuccess) return SG_ERR_CUDA;
    return f ? SG_ERR_TIMEOUT : SG_OK;
}

extern "C" sg_status sg_nn_gemm(int32_t batch, int32_t M, int32_t N, int32_t K, float alpha, const void *A,
                                int32_t lda, int64_t stride_a, int32_t trans_a, const void *B, int32_t ldb,
                                int64_t stride_b, float beta, float *C, int32_t ldc, int64_t stride_c, void *C_bf16,
                                const float *bias, void *stream)
{
    if (batch < 1 || M < 1 || N < 1 || K < 1 || !A || !B || (!C && !C_bf16)) return SG_ERR_ARG;
    if (batch > 65535) return SG_ERR_UNSUPPORTED;
    if (!C && beta != 0.f) return SG_ERR_ARG;
    // rows at least as long as the operands' (op(A) is M x K); elements
    // naturally aligned (bf16 2 bytes, float 4 bytes)
    if (lda < (trans_a ? M : K) || ldb < N || ldc < N || stride_a < 0 || stride_b < 0 || stride_c < 0)
        return SG_ERR_ARG;
    if ((((uintptr_t)A | (uintptr_t)B | (uintptr_t)C_bf16) & 1u) || (((uintptr_t)C | (uintptr_t)bias) & 3u))
        return SG_ERR_ARG;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
    cudaStream_t s = (cudaStream_t)stream;
    auto a = (const __nv_bfloat16 *)A;
    auto b = (const __nv_bfloat16 *)B;
    // 16-byte loads need 16-byte aligned rows in every batch entry
    const int vecA = (lda % 8 == 0) && (stride_a % 8 == 0) && ((uintptr_t)A % 16 == 0);
    const int vecB = (ldb % 8 == 0) && (stride_b % 8 == 0) && ((uintptr_t)B % 16 == 0);
    if (g_gemm_engine == SG_NN_GEMM_TCGEN05) {
        // the kernels' shared-memory limit, once per device
        static std::atomic<unsigned long long> done{0};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SG_ERR_CUDA;
        if (!((done.load() >> dev) & 1ull)) {
            const void *fns[] = {
                (const void *)k_gemm_tc<false, 32, 1>,  (const void *)k_gemm_tc<false, 64, 1>,
                (const void *)k_gemm_tc<false, 128, 1>, (const void *)k_gemm_tc<true, 32, 1>,
                (const void *)k_gemm_tc<true, 64, 1>,   (const void *)k_gemm_tc<true, 128, 1>,
                (const void *)k_gemm_tc<false, 32, 2>,  (const void *)k_gemm_tc<false, 64, 2>,
                (const void *)k_gemm_tc<false, 128, 2>, (const void *)k_gemm_tc<true, 32, 2>,
                (const void *)k_gemm_tc<true, 64, 2>,   (const void *)k_gemm_tc<true, 128, 2>,
                (const void *)k_gemm_tc<false, 128, 2, true>};
            for (const void *f : fns)
                if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes(128, 2)) !=
                    cudaSuccess)
                    return SG_ERR_CUDA;
            done.fetch_or(1ull << dev);
        }
        // A shared by a batch of narrow products with K > 64 (the azimuthal
        // DFTs): fold batch entries side by side into 128-column tiles, so a
        // CTA reads each A step once for all of them
        const int fold =
            (!trans_a && stride_a == 0 && K > TC_BK && N % 8 == 0 && N <= 64 && batch > 1) ? TC_BM / N : 1;
        const int bn = fold > 1 ? 128 : N <= 32 ? 32 : N <= 64 ? 64 : 128, nst = K <= TC_BK ? 1 : 2;
        const dim3 gt((M + TC_BM - 1) / TC_BM, fold > 1 ? 1 : (N + bn - 1) / bn, (batch + fold - 1) / fold);
        if (gt.y > 65535) return SG_ERR_UNSUPPORTED;
        auto go = [&](auto kern) {
            kern<<<gt, 128, tc_smem_bytes(bn, nst), s>>>(M, N, K, alpha, a, lda, stride_a, b, ldb, stride_b, beta, C,
                                                         ldc, stride_c, (__nv_bfloat16 *)C_bf16, bias, vecA, vecB,
                                                         batch, fold);
        };
        auto pick = [&](auto ta) {
            constexpr bool TA = decltype(ta)::value;
            if (fold > 1 && !TA) {
                go(k_gemm_tc<false, 128, 2, true>);
            } else if (nst == 1) {
                if (bn == 32) go(k_gemm_tc<TA, 32, 1>);
                else if (bn == 64) go(k_gemm_tc<TA, 64, 1>);
                else go(k_gemm_tc<TA, 128, 1>);
            } else {
                if (bn == 32) go(k_gemm_tc<TA, 32, 2>);
                else if (bn == 64) go(k_gemm_tc<TA, 64, 2>);
                else go(k_gemm_tc<TA, 128, 2>);
            }
        };
        if (trans_a) pick(std::true_type{});
        else pick(std::false_type{});
    } else if (trans_a) {
        k_gemm<true><<<grid, 128, 0, s>>>(M, N, K, alpha, a, lda, stride_a, b, ldb, stride_b, beta, C, ldc, stride_c,
                                          (__nv_bfloat16 *)C_bf16, bias, vecA, vecB);
    } else {
        k_gemm<false><<<grid, 128, 0, s>>>(M, N, K, alpha, a, lda, stride_a, b, ldb, stride_b, beta, C, ldc, stride_c,
                                           (__nv_bfloat16 *)C_bf16, bias, vecA, vecB);
    }
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

// ----------------------------------------------------------------------
// Spectral-convolution pieces (per sample b; C channels; K1 radial modes;
// M1 azimuthal modes).  T = [Gc; Gs] V1 from the radial DFT GEMM, laid out
// [b][2 K1][2 M1][C] (row kk < K1: Gc rows, kk >= K1: Gs rows; column j =
// 2 m + {0: re, 1: im}); V2 complex [b][K1][M1][C] as float2.
namespace {

__global__ void k_spec_combine(int n, int K1, int M1, int C, const float *__restrict__ T, float2 *__restrict__ V2)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // over b K1 M1 C
    if (idx >= n) return;
    const int c = idx % C, m = (idx / C) % M1, k = (idx / (C * M1)) % K1, b = idx / (C * M1 * K1);
    const size_t row = (size_t)2 * M1 * C;
    const float *tc = T + ((size_t)b * 2 * K1 + k) * row, *ts = tc + (size_t)K1 * row;
    const float cr = tc[(2 * m) * C + c], ci = tc[(2 * m + 1) * C + c];
    const float sr = ts[(2 * m) * C + c], si = ts[(2 * m + 1) * C + c];
    V2[idx] = make_float2(cr - si, ci + sr);                // (Gc + i Gs)(V1r + i V1i)
}

// backward: dT from dV2 (complex gradient g = dL/dRe + i dL/dIm), written as BF16
__global__ void k_spec_combine_bwd(int n, int K1, int M1, int C, const float2 *__restrict__ dV2,
                                   __nv_bfloat16 *__restrict__ dT)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int c = idx % C, m = (idx / C) % M1, k = (idx / (C * M1)) % K1, b = idx / (C * M1 * K1);
    const size_t row = (size_t)2 * M1 * C;
    __nv_bfloat16 *tc = dT + ((size_t)b * 2 * K1 + k) * row, *ts = tc + (size_t)K1 * row;
    const float2 g = dV2[idx];
    tc[(2 * m) * C + c] = __float2bfloat16(g.x);
    tc[(2 * m + 1) * C + c] = __float2bfloat16(g.y);
    ts[(2 * m) * C + c] = __float2bfloat16(g.y);
    ts[(2 * m + 1) * C + c] = __float2bfloat16(-g.x);
}

// O[b][kk][m][o] = sum_i V2[b][kk][m][i] W[kk][m][i][o]; written as BF16
// planes O_out[b][ri][kk][m][o] (ri 0: re, 1: im) for the inverse radial GEMM.
__global__ void k_modemix(int B, int K1, int M1, int C, const float2 *__restrict__ V2, const float2 *__restrict__ W,
                          __nv_bfloat16 *__restrict__ Oout)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // over b K1 M1 C(o)
    const int n = B * K1 * M1 * C;
    if (idx >= n) return;
    const int o = idx % C, km = (idx / C) % (K1 * M1), b = idx / (C * K1 * M1);
    const float2 *x = V2 + ((size_t)b * K1 * M1 + km) * C;
    const float2 *w = W + (size_t)km * C * C + o;
    float re = 0.f, im = 0.f;
    for (int i = 0; i < C; ++i) {
        const float2 a = x[i], ww = w[(size_t)i * C];
        re += a.x * ww.x - a.y * ww.y;
        im += a.x * ww.y + a.y * ww.x;
    }
    const size_t plane = (size_t)K1 * M1 * C;
    Oout[(size_t)b * 2 * plane + (size_t)km * C + o] = __float2bfloat16(re);
    Oout[(size_t)b * 2 * plane + plane + (size_t)km * C + o] = __float2bfloat16(im);
}

// backward of the mode mixing: dO given as FP32 planes [b][ri][kk][m][o];
// dV2[b][kk][m][i] = sum_o dO conj(W[i][o]); dW[kk][m][i][o] = sum_b conj(V2) dO.
__global__ void k_modemix_bwd_x(int B, int K1, int M1, int C, const float *__restrict__ dO,
                                const float2 *__restrict__ W, float2 *__restrict__ dV2)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // over b K1 M1 C(i)
    const int n = B * K1 * M1 * C;
    if (idx >= n) return;
    const int i = idx % C, km = (idx / C) % (K1 * M1), b = idx / (C * K1 * M1);
    const size_t plane = (size_t)K1 * M1 * C;
    const float *gr = dO + (size_t)b * 2 * plane + (size_t)km * C, *gi = gr + plane;
    const float2 *w = W + ((size_t)km * C + i) * C;
    float re = 0.f, im = 0.f;
    for (int o = 0; o < C; ++o) {
        const float2 ww = w[o];
        re += gr[o] * ww.x + gi[o] * ww.y;                  // g conj(w)
        im += gi[o] * ww.x - gr[o] * ww.y;
    }
    dV2[idx] = make_float2(re, im);
}

__global__ void k_modemix_bwd_w(int B, int K1, int M1, int C, const float2 *__restrict__ V2,
                                const float *__restrict__ dO, float2 *__restrict__ dW)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // over K1 M1 C(i) C(o)
    const int n = K1 * M1 * C * C;
    if (idx >= n) return;
    const int o = idx % C, i = (idx / C) % C, km = idx / (C * C);
    const size_t plane = (size_t)K1 * M1 * C;
    float re = 0.f, im = 0.f;
    for (int b = 0; b < B; ++b) {
        const float2 x = V2[((size_t)b * K1 * M1 + km) * C + i];
        const float gr = dO[(size_t)b * 2 * plane + (size_t)km * C + o], gi = dO[(size_t)b * 2 * plane + plane + (size_t)km * C + o];
        re += x.x * gr + x.y * gi;                          // conj(x) g
        im += x.x * gi - x.y * gr;
    }
    dW[idx] = make_float2(re, im);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x)
{
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void k_act(long long n, const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, int apply)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(apply ? gelu(x[i]) : x[i]);
}

// dpre = dy gelu'(pre) (or dy), as FP32 and BF16
__global__ void k_act_bwd(long long n, const float *__restrict__ pre, const float *__restrict__ dy,
                          float *__restrict__ dpre, __nv_bfloat16 *__restrict__ dpre_b, int apply)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float g = apply ? dy[i] * gelu_d(pre[i]) : dy[i];
        if (dpre) dpre[i] = g;
        if (dpre_b) dpre_b[i] = __float2bfloat16(g);
    }
}

// out[c] += sum over a chunk of rows of x[rows][C] (blockIdx.y: row chunk);
// out is zeroed (or kept) by the caller before the launch.
__global__ void k_colsum(long long rows, int C, long long chunk, const float *__restrict__ x, float *__restrict__ out)
{
    __shared__ float red[256];
    const int c = blockIdx.x;
    const long long r0 = blockIdx.y * chunk, r1 = r0 + chunk < rows ? r0 + chunk : rows;
    float s = 0.f;
    for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) s += x[r * C + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&out[c], red[0]);
}

// Relative-L2 loss per (sample, channel): pred, target [B][npix][2];
// stats[b * 2 + ch] = (|pred - t|^2, |t|^2) accumulated with atomics.
__global__ void k_rel_l2(int B, long long npix, int CH, const float *__restrict__ pred, const float *__restrict__ tgt,
                         float *__restrict__ stats)
{
    const int b = blockIdx.y;
    __shared__ float red[2][8][256];
    float e[8] = {}, t[8] = {};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x)
        for (int c = 0; c < CH; ++c) {
            const float y = tgt[((size_t)b * npix + p) * CH + c], d = pred[((size_t)b * npix + p) * CH + c] - y;
            e[c] += d * d;
            t[c] += y * y;
        }
    for (int c = 0; c < CH; ++c) {
        red[0][c][threadIdx.x] = e[c];
        red[1][c][threadIdx.x] = t[c];
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int c = 0; c < CH; ++c) {
                red[0][c][threadIdx.x] += red[0][c][threadIdx.x + w];
                red[1][c][threadIdx.x] += red[1][c][threadIdx.x + w];
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < CH; ++c) {
            atomicAdd(&stats[(b * CH + c) * 2], red[0][c][0]);
            atomicAdd(&stats[(b * CH + c) * 2 + 1], red[1][c][0]);
        }
}

// gradient of L = mean over (b, ch) of |pred - t|^2 / |t|^2
__global__ void k_rel_l2_grad(int B, long long npix, int CH, const float *__restrict__ pred,
                              const float *__restrict__ tgt, const float *__restrict__ stats, float *__restrict__ dpred)
{
    const long long n = (long long)B * npix * CH;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % CH);
        const int b = (int)(i / (npix * CH));
        const float tt = stats[(b * CH + c) * 2 + 1];
        dpred[i] = 2.f * (pred[i] - tgt[i]) / (tt * (float)(B * CH));
    }
}

__global__ void k_adam(long long n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16 *__restrict__ wb)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gg = g[i];
        const float mm = b1 * m[i] + (1.f - b1) * gg, vv = b2 * v[i] + (1.f - b2) * gg * gg;
        m[i] = mm;
        v[i] = vv;
        const float ww = w[i] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        w[i] = ww;
        if (wb) wb[i] = __float2bfloat16(ww);
    }
}

__global__ void k_cast(long long n, const float *__restrict__ x, __nv_bfloat16 *__restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

int blocks_for(long long n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

}  // namespace

namespace {
// element pointers aligned to their type (NULL passes); element counts the
// kernels index with int
inline bool al(const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }
inline bool fits(long long n) { return n > 0 && n <= 0x7FFFFFFFLL; }
}  // namespace

extern "C" {

sg_status sg_nn_spec_combine(int32_t B, int32_t K1, int32_t M1, int32_t C, const float *T, void *V2, void *stream)
{
    if (!T || !V2 || B < 1 || K1 < 1 || M1 < 1 || C < 1) return SG_ERR_ARG;
    if (!al(T, 4) || !al(V2, 8) || !fits((long long)B * K1 * M1 * C)) return SG_ERR_ARG;
    const int n = B * K1 * M1 * C;
    k_spec_combine<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, K1, M1, C, T, (float2 *)V2);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_nn_spec_combine_bwd(int32_t B, int32_t K1, int32_t M1, int32_t C, const void *dV2, void *dT_bf16,
                                 void *stream)
{
    if (!dV2 || !dT_bf16 || B < 1 || K1 < 1 || M1 < 1 || C < 1) return SG_ERR_ARG;
    if (!al(dV2, 8) || !al(dT_bf16, 2) || !fits((long long)B * K1 * M1 * C)) return SG_ERR_ARG;
    const int n = B * K1 * M1 * C;
    k_spec_combine_bwd<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, K1, M1, C, (const float2 *)dV2,
                                                                        (__nv_bfloat16 *)dT_bf16);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_nn_modemix(int32_t B, int32_t K1, int32_t M1, int32_t C, const void *V2, const void *W, void *O_bf16,
                        void *stream)
{
    if (!V2 || !W || !O_bf16 || B < 1 || K1 < 1 || M1 < 1 || C < 1) return SG_ERR_ARG;
    if (!al(V2, 8) || !al(W, 8) || !al(O_bf16, 2) || !fits((long long)B * K1 * M1 * C) ||
        !fits((long long)K1 * M1 * C * C))
        return SG_ERR_ARG;
    const int n = B * K1 * M1 * C;
    k_modemix<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(B, K1, M1, C, (const float2 *)V2, (const float2 *)W,
                                                               (__nv_bfloat16 *)O_bf16);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_nn_modemix_bwd(int32_t B, int32_t K1, int32_t M1, int32_t C, const void *V2, const void *W,
                            const float *dO, void *dV2, void *dW, void *stream)
{
    if (!V2 || !W || !dO || (!dV2 && !dW) || B < 1 || K1 < 1 || M1 < 1 || C < 1) return SG_ERR_ARG;
    if (!al(V2, 8) || !al(W, 8) || !al(dO, 4) || !al(dV2, 8) || !al(dW, 8) || !fits((long long)B * K1 * M1 * C) ||
        !fits((long long)K1 * M1 * C * C))
        return SG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (dV2) {
        const int n = B * K1 * M1 * C;
        k_modemix_bwd_x<<<(n + 255) / 256, 256, 0, s>>>(B, K1, M1, C, dO, (const float2 *)W, (float2 *)dV2);
    }
    if (dW) {
        const int n = K1 * M1 * C * C;
        k_modemix_bwd_w<<<(n + 255) / 256, 256, 0, s>>>(B, K1, M1, C, (const float2 *)V2, dO, (float2 *)dW);
    }
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_nn_act(int64_t n, const float *x, void *y_bf16, int32_t gelu_on, void *stream)
{
    if (!x || !y_bf16 || n < 1) return SG_ERR_ARG;
    if (!al(x, 4) || !al(y_bf16, 2)) return SG_ERR_ARG;
    k_act<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, x, (__nv_bfloat16 *)y_bf16, gelu_on);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_nn_act_bwd(int64_t n, const float *pre, const float *dy, float *dpre, void *dpre_bf16, int32_t gelu_on,
                        void *stream)
{
    if (!pre || !dy || (!dpre && !dpre_bf16) || n < 1) return SG_ERR_ARG;
    if (!al(pre, 4) || !al(dy, 4) || !al(dpre, 4) || !al(dpre_bf16, 2)) return SG_ERR_ARG;
    k_act_bwd<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, pre, dy, dpre, (__nv_bfloat16 *)dpre_bf16, gelu_on);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_nn_colsum(int64_t rows, int32_t C, const float *x, float *out, int32_t accumulate, void *stream)
{
    if (!x || !out || rows < 1 || C < 1) return SG_ERR_ARG;
    if (!al(x, 4) || !al(out, 4)) return SG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!accumulate) cudaMemsetAsync(out, 0, sizeof(float) * C, s);
    // enough row chunks to fill the GPU (about 2048 blocks), at least 4096 rows each
    long long chunks = 2048 / C + 1;
    if (rows / chunks < 4096) chunks = rows / 4096 + 1;
    if (chunks > 65535) chunks = 65535;
    const long long chunk = (rows + chunks - 1) / chunks;
    dim3 grid(C, (unsigned)chunks);
    k_colsum<<<grid, 256, 0, s>>>(rows, C, chunk, x, out);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_nn_rel_l2(int32_t B, int64_t npix, int32_t CH, const float *pred, const float *tgt, float *stats,
                       float *dpred, void *stream)
{
    if (!pred || !tgt || !stats || B < 1 || npix < 1 || CH < 1 || CH > 8) return SG_ERR_ARG;
    if (!al(pred, 4) || !al(tgt, 4) || !al(stats, 4) || !al(dpred, 4)) return SG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(stats, 0, sizeof(float) * 2 * B * CH, s);
    dim3 grid(256, B);
    k_rel_l2<<<grid, 256, 0, s>>>(B, npix, CH, pred, tgt, stats);
    if (dpred) k_rel_l2_grad<<<blocks_for((long long)B * npix * CH), 256, 0, s>>>(B, npix, CH, pred, tgt, stats, dpred);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_nn_adam(int64_t n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                     int32_t step, void *w_bf16, void *stream)
{
    if (!w || !g || !m || !v || n < 1 || step < 1) return SG_ERR_ARG;
    if (!al(w, 4) || !al(g, 4) || !al(m, 4) || !al(v, 4) || !al(w_bf16, 2)) return SG_ERR_ARG;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, w, g, m, v, lr, b1, b2, eps, c1, c2,
                                                            (__nv_bfloat16 *)w_bf16);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_nn_cast(int64_t n, const float *x, void *y_bf16, void *stream)
{
    if (!x || !y_bf16 || n < 1) return SG_ERR_ARG;
    if (!al(x, 4) || !al(y_bf16, 2)) return SG_ERR_ARG;
    k_cast<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, x, (__nv_bfloat16 *)y_bf16);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

}  // extern "C"

// ----------------------------------------------------------------------
// Training fields of the surrogate (log-normal-like background from random
// Fourier features, m = 1..6 spirals, Gaussian clumps of the Sec. 4.4 form,
// dust as a noisy fraction of the gas), evaluated cell by cell on the
// log-polar grid from per-sample parameters drawn on the host.
//
// params[b] (floats): [0] ln r_in, [1] du, [2] dphi, [3] sigma_ln, [4] eps
// (dust fraction), [5] noise seed (as float bits), [6] cot(pitch),
// [8 .. 8 + 4 NF) features (kr, km, amp, phase), then 6 x (A_m, psi_m) for
// the spirals, then 3 x (x_c, y_c, A, R) for the clumps.
namespace {

constexpr int NF = 32;
constexpr int NPAR = 8 + 4 * NF + 12 + 12;

__device__ __forceinline__ float hash_unit(uint32_t seed, uint32_t i)
{
    // splitmix-style integer hash of (seed, i) to [0, 1)
    uint32_t x = seed * 0x9E3779B9u ^ (i + 0x7F4A7C15u);
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return (float)(x >> 8) * (1.f / 16777216.f);
}

__global__ void k_fields(int R, int P, const float *__restrict__ params, float *__restrict__ sg, float *__restrict__ sd)
{
    const int b = blockIdx.y;
    const float *q = params + (size_t)b * NPAR;
    const long long n = (long long)R * P;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / P), j = (int)(idx - (long long)i * P);
        const float u = (i + 0.5f) * q[1], lr = q[0] + u, r = expf(lr), phi = (j + 0.5f) * q[2];
        float gsum = 0.f;
        for (int f = 0; f < NF; ++f) {
            const float *w = q + 8 + 4 * f;
            gsum += w[2] * cosf(w[0] * u + w[1] * phi + w[3]);
        }
        float s = expf(q[3] * gsum - 0.5f * q[3] * q[3]) / r;
        float sp = 1.f;
        const float *spr = q + 8 + 4 * NF;
        for (int m = 1; m <= 6; ++m) sp += spr[2 * (m - 1)] * cosf(m * (phi - q[6] * u) + spr[2 * (m - 1) + 1]);
        s *= sp;
        const float *cl = spr + 12;
        const float x = r * cosf(phi), y = r * sinf(phi);
        for (int c = 0; c < 3; ++c) {
            const float dx = x - cl[4 * c], dy = y - cl[4 * c + 1], R2 = cl[4 * c + 3] * cl[4 * c + 3];
            s *= 1.f + cl[4 * c + 2] * expf(-(dx * dx + dy * dy) / (2.f * R2));
        }
        sg[(size_t)b * n + idx] = s;
        if (sd) {
            const uint32_t seed = __float_as_uint(q[5]);
            sd[(size_t)b * n + idx] = q[4] * s * (1.f + 0.02f * (hash_unit(seed, (uint32_t)idx) - 0.5f));
        }
    }
}

}  // namespace

extern "C" sg_status sg_nn_fields(int32_t B, int32_t nr, int32_t nphi, const float *params, float *sigma_g,
                                  float *sigma_d, void *stream)
{
    if (B < 1 || nr < 1 || nphi < 1 || !params || !sigma_g) return SG_ERR_ARG;
    if (B > 65535 || !al(params, 4) || !al(sigma_g, 4) || !al(sigma_d, 4)) return SG_ERR_ARG;
    dim3 grid(256, B);
    k_fields<<<grid, 256, 0, (cudaStream_t)stream>>>(nr, nphi, params, sigma_g, sigma_d);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

namespace {
__global__ void k_transpose(int rows, int cols, const float *__restrict__ x, __nv_bfloat16 *__restrict__ y)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int r = idx / cols, c = idx - r * cols;
    y[(size_t)c * rows + r] = __float2bfloat16(x[idx]);
}
}  // namespace

extern "C" sg_status sg_nn_transpose(int32_t rows, int32_t cols, const float *x, void *y_bf16, void *stream)
{
    if (rows < 1 || cols < 1 || !x || !y_bf16) return SG_ERR_ARG;
    if (!al(x, 4) || !al(y_bf16, 2) || !fits((long long)rows * cols)) return SG_ERR_ARG;
    const int n = rows * cols;
    k_transpose<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(rows, cols, x, (__nv_bfloat16 *)y_bf16);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

namespace {
// x[b][i][j][0..6] = (sg s_g[b], sd s_d[b], hg[b] / 0.05, hd[b] / 0.05, u / u_max, cos phi, sin phi)
__global__ void k_pack_in(int B, int R, int P, const float *__restrict__ sg, const float *__restrict__ sd,
                          const float *__restrict__ per, float du, __nv_bfloat16 *__restrict__ x)
{
    const long long n = (long long)B * R * P;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(idx / ((long long)R * P));
        const long long cell = idx - (long long)b * R * P;
        const int i = (int)(cell / P), j = (int)(cell - (long long)i * P);
        const float *q = per + 4 * b;
        float s, c;
        sincospif(2.f * (j + 0.5f) / P, &s, &c);
        __nv_bfloat16 *o = x + idx * 7;
        o[0] = __float2bfloat16(sg[idx] * q[0]);
        o[1] = __float2bfloat16(sd ? sd[idx] * q[1] : 0.f);
        o[2] = __float2bfloat16(q[2]);
        o[3] = __float2bfloat16(q[3]);
        o[4] = __float2bfloat16((i + 0.5f) / R);
        o[5] = __float2bfloat16(c);
        o[6] = __float2bfloat16(s);
    }
}
// t[b][cell][0..1] = (a[b][cell], c[b][cell]) * scale[b]
__global__ void k_pack_out(int B, long long npix, const float *__restrict__ a, const float *__restrict__ c,
                           const float *__restrict__ scale, float *__restrict__ t)
{
    const long long n = (long long)B * npix;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
        const float s = scale[idx / npix];
        t[2 * idx] = a[idx] * s;
        t[2 * idx + 1] = c[idx] * s;
    }
}
// the inverse: a = t[..][0] / scale, c = t[..][1] / scale
__global__ void k_unpack_out(int B, long long npix, const float *__restrict__ t, const float *__restrict__ scale,
                             float *__restrict__ a, float *__restrict__ c)
{
    const long long n = (long long)B * npix;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
        const float s = 1.f / scale[idx / npix];
        a[idx] = t[2 * idx] * s;
        c[idx] = t[2 * idx + 1] * s;
    }
}
}  // namespace

extern "C" {
sg_status sg_nn_pack_inputs(int32_t B, int32_t nr, int32_t nphi, const float *sigma_g, const float *sigma_d,
                            const float *per_sample, void *x_bf16, void *stream)
{
    if (B < 1 || nr < 1 || nphi < 1 || !sigma_g || !per_sample || !x_bf16) return SG_ERR_ARG;
    if (!al(sigma_g, 4) || !al(sigma_d, 4) || !al(per_sample, 4) || !al(x_bf16, 2)) return SG_ERR_ARG;
    k_pack_in<<<1024, 256, 0, (cudaStream_t)stream>>>(B, nr, nphi, sigma_g, sigma_d, per_sample, 0.f,
                                                     (__nv_bfloat16 *)x_bf16);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}
sg_status sg_nn_pack_targets(int32_t B, int64_t npix, const float *a, const float *c, const float *scale, float *t,
                             int32_t unpack, void *stream)
{
    if (B < 1 || npix < 1 || !a || !c || !scale || !t) return SG_ERR_ARG;
    if (!al(a, 4) || !al(c, 4) || !al(scale, 4) || !al(t, 4)) return SG_ERR_ARG;
    if (unpack)
        k_unpack_out<<<1024, 256, 0, (cudaStream_t)stream>>>(B, npix, t, scale, (float *)a, (float *)c);
    else
        k_pack_out<<<1024, 256, 0, (cudaStream_t)stream>>>(B, npix, a, c, scale, t);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}
}
