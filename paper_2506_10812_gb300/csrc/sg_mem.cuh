// Shared device helpers of the FFT path: the layout of the [N][rows]
// spectral intermediates, the swizzled transpose tile of the row
// transforms, and L2 cache-policy loads and stores.
#pragma once

#include <stdint.h>

#include "sg_fft.cuh"

namespace sg {

// Columns per block of the [N][rows] intermediates: element (m, i) at
// ((m / BW) rows + i) BW + m % BW.  BW = 1 is plain column-major.
#ifndef SG_BW
#define SG_BW 1
#endif
constexpr int BW = SG_BW;

// Swizzled [N][rpc] transpose tile: conflict-free for both the per-row
// strided access (consecutive k, fixed row) and the blocked copy.
template <typename C>
__device__ __forceinline__ int tile_idx(int k, int g, int rpc)
{
    constexpr int lg_wf = sizeof(C) == 8 ? 4 : 3;         // log2(128 / sizeof(C))
    const int lg_rpc = rpc == 4 ? 2 : (rpc == 2 ? 1 : 0);
    return k * rpc + (g ^ ((k >> (lg_wf - lg_rpc)) & (rpc - 1)));
}

// The same swizzle for any power-of-two number of rows 2^lg (equal to
// tile_idx for rpc = 1, 2, 4); for more than 16 rows (8-byte elements) the
// XOR takes the low bits of k.
template <typename C>
__device__ __forceinline__ int tile_idx_g(int k, int g, int lg)
{
    constexpr int lg_wf = sizeof(C) == 8 ? 4 : 3;
    const int sh = lg_wf > lg ? lg_wf - lg : 0;
    return (k << lg) + (g ^ ((k >> sh) & ((1 << lg) - 1)));
}

// index of element (m, i) in a [N][nrows] intermediate
__device__ __forceinline__ size_t blk(int m, int i, int nrows)
{
    return ((size_t)(m / BW) * nrows + i) * BW + (m & (BW - 1));
}

// ------------------------------------------------ L2 eviction policies
// Per-instruction L2 cache hints (createpolicy): the kernel spectra stream
// through L2 once per solve (evict-first); the column pass's output is read
// again by the inverse row transforms right after (evict-last), so it should
// stay in L2 instead of the streamed spectra.
__device__ __forceinline__ uint64_t l2_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void st_hint(float2 *p, float2 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_hint(double2 *p, double2 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.x), "d"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ float2 ld_hint(const float2 *p, uint64_t pol)
{
    float2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double2 ld_hint(const double2 *p, uint64_t pol)
{
    double2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
    return v;
}

// Coherent load (L2 only, no L1 allocation, no non-coherent path) for data
// that other blocks of the same launch wrote.
__device__ __forceinline__ float2 ld_cg_hint(const float2 *p, uint64_t pol)
{
    float2 v;
    asm volatile("ld.global.cg.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol)
                 : "memory");
    return v;
}
__device__ __forceinline__ double2 ld_cg_hint(const double2 *p, uint64_t pol)
{
    double2 v;
    asm volatile("ld.global.cg.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol)
                 : "memory");
    return v;
}

// ------------------------------------------ programmatic dependent launch
// griddep_wait: until the grids this launch depends on programmatically have
// completed and their memory is visible (returns at once for an ordinary
// launch); every thread that reads their output calls it first.
// griddep_launch: this CTA lets the dependent grid start launching.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------- TMA bulk copy + mbarrier
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16)
// with an L2 cache policy
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, uint64_t *bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after 2^22 polls (far beyond any copy time),
// ORs `bit` (default 2: a plan's timeout bit) into *flag and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned int *flag,
                                                  unsigned bit = 2u)
{
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    if (flag) atomicOr(flag, bit);
    return false;
}
// 2-D tensor copies (cp.async.bulk.tensor) through a CUtensorMap kernel
// parameter: coordinates (x, y) in elements, x innermost; the box lands in
// (or leaves) shared memory densely, x fastest.  The shared-memory address
// must be 128-byte aligned and x times the element size a multiple of 16.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const void *tmap, int x, int y, const void *src, uint64_t pol)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%1, %2}], [%3], %4;" ::"l"(
                     tmap),
                 "r"(x), "r"(y), "r"(smem_u32(src)), "l"(pol)
                 : "memory");
}
// L2 prefetch hint for a contiguous range (16-byte aligned, multiple of 16 bytes)
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Until every committed bulk store has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Before the barrier's shared memory is used for anything else.
__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------- dead-data L2 discards
// The spectral intermediates are written into L2 by one kernel and read once
// by the next.  Once read they are dead, but L2 is write-back: left alone,
// every such line is written to DRAM when it is evicted (and, under pressure,
// lines not yet read are evicted and fetched again).  discard.global.L2
// invalidates a 128-byte line without writing it back; it is issued only for
// lines every reader has finished with, and nothing reads them again before
// the next solve rewrites them.
__device__ __forceinline__ void l2_discard(const void *p)
{
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}
// Discard the `bytes` (a multiple of 128, 128-byte aligned) at p, the lines
// spread over the `nthr` threads of the caller (thread index `tid`).
__device__ __forceinline__ void l2_discard_range(const void *p, size_t bytes, int tid, int nthr)
{
    const char *c = reinterpret_cast<const char *>(p);
    for (size_t off = (size_t)tid * 128; off < bytes; off += (size_t)nthr * 128) l2_discard(c + off);
}


// ------------------------------------------------- tensor memory (TMEM)
// Each SM's tensor memory is 128 lanes x 512 columns of 32-bit cells.  With
// the 32x32b shapes a warp reaches the 32 lanes 32 (warp % 4) .. + 31 only:
// thread l of the warp is lane 32 (warp % 4) + l, and register j of a
// transfer is column col + j.  An address is (lane << 16) | column.
// Allocation (a power of two >= 32 columns) and release are whole-warp
// operations of one warp; a CTA must release what it allocated before it exits.
__device__ __forceinline__ void tmem_alloc(uint32_t *smem_dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// around a CTA barrier that orders tensor-memory accesses
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 8 complex FP32 values (16 cells) of this thread's lane, from column col of
// taddr on; each call waits for its own transfer, so the registers are
// written (load) or free (store) when it returns.
__device__ __forceinline__ void tmem_st8c(uint32_t taddr, const float2 (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16};\n\ttcgen05.wait::st.sync.aligned;" ::"r"(taddr),
                 "f"(v[0].x), "f"(v[0].y), "f"(v[1].x), "f"(v[1].y), "f"(v[2].x), "f"(v[2].y), "f"(v[3].x),
                 "f"(v[3].y), "f"(v[4].x), "f"(v[4].y), "f"(v[5].x), "f"(v[5].y), "f"(v[6].x), "f"(v[6].y),
                 "f"(v[7].x), "f"(v[7].y)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld8c(uint32_t taddr, float2 (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%16];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y), "=f"(v[2].x), "=f"(v[2].y), "=f"(v[3].x),
                   "=f"(v[3].y), "=f"(v[4].x), "=f"(v[4].y), "=f"(v[5].x), "=f"(v[5].y), "=f"(v[6].x),
                   "=f"(v[6].y), "=f"(v[7].x), "=f"(v[7].y)
                 : "r"(taddr)
                 : "memory");
}

// ----------------------------------------------- tcgen05 matrix products
// Shared-memory matrix descriptor (no swizzle): start address, the byte
// offset between core matrices adjacent along K (lbo) and along M / N (sbo),
// each encoded >> 4; bits 46..48 hold the fixed value 0b001.  A core matrix is
// 8 rows of 16 bytes stored contiguously (rows 16 bytes apart).
__device__ __forceinline__ uint64_t umma_sdesc(unsigned smem_addr, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((smem_addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of a dense kind::f16 / kind::tf32 product with an
// FP32 accumulator, A and B K-major: ab = 0 F16, 1 BF16 (kind::f16), 2 TF32.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N, uint32_t ab)
{
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D[tmem] (+)= A[tmem] B[smem]; issued by one thread.
template <bool TF32>
__device__ __forceinline__ void umma_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate)
{
    if constexpr (TF32)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
                     "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
                     : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
                     "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
                     : "memory");
}
// D[tmem] (+)= A[smem] B[smem] (kind::f16, both operands K-major through
// shared-memory descriptors); issued by one thread.
__device__ __forceinline__ void umma_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
                 : "memory");
}
// One arrive on the mbarrier once every product this thread issued before
// it has completed.
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 16 32-bit cells of this thread's lane to / from columns col .. col + 15.
__device__ __forceinline__ void tmem_st16u(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
                 "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 32 cells (16 complex FP32 values) of this thread's lane, waited for.
__device__ __forceinline__ void tmem_ld16c(uint32_t taddr, float2 (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                 "[%32];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y), "=f"(v[2].x), "=f"(v[2].y),
                   "=f"(v[3].x), "=f"(v[3].y), "=f"(v[4].x), "=f"(v[4].y), "=f"(v[5].x), "=f"(v[5].y),
                   "=f"(v[6].x), "=f"(v[6].y), "=f"(v[7].x), "=f"(v[7].y), "=f"(v[8].x), "=f"(v[8].y),
                   "=f"(v[9].x), "=f"(v[9].y), "=f"(v[10].x), "=f"(v[10].y), "=f"(v[11].x), "=f"(v[11].y),
                   "=f"(v[12].x), "=f"(v[12].y), "=f"(v[13].x), "=f"(v[13].y), "=f"(v[14].x), "=f"(v[14].y),
                   "=f"(v[15].x), "=f"(v[15].y)
                 : "r"(taddr)
                 : "memory");
}

// 32 FP32 cells of this thread's lane, columns col .. col + 31, waited for.
__device__ __forceinline__ void tmem_ld32f(uint32_t taddr, float (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                 "[%32];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
                   "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]),
                   "=f"(v[15]), "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]),
                   "=f"(v[22]), "=f"(v[23]), "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]),
                   "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
                 : "r"(taddr)
                 : "memory");
}

}  // namespace sg
