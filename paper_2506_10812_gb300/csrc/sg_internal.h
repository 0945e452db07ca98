// Internal launch interface between the C ABI (sg_api.cu) and the kernels
// (sg_kernels.cu, sg_direct.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sg.h"

namespace sg {

// Twiddle tables: tw_row[k] = exp(-2 pi i k / nphi), k < nphi (the R2C /
// C2R pre- and post-processing); twp_row / twp_col / twp_col64: per-pass
// tables (sg_fft.cuh) of the length-nphi/2 row and length-2nr column
// transforms.  Every launch below that transforms takes the per-pass table
// of its own length.
//
// Row transforms process RPC rows per CTA (one group of nphi/32 threads per
// row) so that the transposed [m][row] intermediates move in RPC-element
// chunks; both the forward and the inverse use the same shared-memory size.
int row_rpc(int nphi, bool f64);
size_t row_smem_bytes(int nphi, int rpc, bool f64);
// Column pass: shared memory per CTA and whether kernel spectra are staged
// per (target, component) step; staging < 0 is the plan default, 0 all
// tables at once, 1 per step (FP32 only; FP64 always all at once).
size_t col_smem_bytes(int nr, int nsrc, bool f64, int staging = -1);
bool cols_staging_steps(int nr, int nsrc, bool f64, int staging);
size_t tabcol_smem_bytes(int L, bool f64);
// complex slots per stored kernel-spectrum column
__host__ __device__ inline int tab_pitch(int nr) { return nr + 2; }
cudaError_t set_cols_steps_smem_limits(int max_optin);   // the per-step column kernels
cudaError_t set_smem_limits(int max_optin);       // every kernel (calls set_row_smem_limits)
cudaError_t set_row_smem_limits(int max_optin);   // the row transforms (sg_rows.cu)

// Kernel-table evaluation (App. C lattice), one ordered pair (source aspect
// ratio ha, target hb), all three components times scale * e^{alpha Delta},
// written as [2 nr][nphi] arrays of type double (out64) or float (out32);
// NULL skips.  mixed: evaluate the Bessel functions in FP32 where X >= 1
// outside the nearest-neighbour stencil, FP64 elsewhere; otherwise FP64.
cudaError_t launch_tab_eval(int nr, int nphi, double du, double ha, double hb, double scale,
                            double alpha, bool mixed, double *o64[3], float *o32[3], cudaStream_t s);

// Row R2C of `nsrc` real [nrows][nphi] arrays x[a] (each row times
// rscale[row] when rscale != NULL; row mean removed when dc) into packed
// spectra xh + a * (nphi/2) * nrows, [nphi/2][nrows] in the layout of sg_mem.cuh
// (slot m = 0 packs the real m = 0 and m = nphi/2 coefficients).
// row0, nrows_run: transform only rows row0 .. row0 + nrows_run - 1 (multiples
// of row_rpc; nrows_run < 0: to the end); nrows stays the row stride.
// tm: the tensor map of xh (encode_row_map over nsrc nphi/2 columns, box of
// tile_rows rows); with it, FP32 rows of the hot lengths (rows_tma_eligible)
// store their spectrum tiles by bulk tensor copies, tile_rows (2 or 4) rows
// per CTA (bit 2 of *tflag when a staged copy never completed).
template <typename R>
cudaError_t launch_rows_fwd(const R *x0, const R *x1, int nsrc, void *xh, int nrows, int nphi,
                            const void *tw_row, const void *twp_row, const R *rscale, bool dc, cudaStream_t s,
                            int row0 = 0, int nrows_run = -1, const CUtensorMap *tm = nullptr,
                            unsigned int *tflag = nullptr, int tile_rows = 4);

// 2-D tensor map of a [ncols][nr] complex FP32 intermediate for the
// tensor-copy row transforms; rows_tma_eligible: the sizes they take.
// `rows`: rows per CTA of the kernel that uses the map (the plan's tiles).
cudaError_t encode_row_map(CUtensorMap *m, void *base, int nr, long long ncols, int rows);
bool rows_tma_eligible(int nr, int nphi, bool f64);

// Column pass of the solve: forward padded FFT of every source column,
// products with the packed kernel spectra, inverse FFT of every requested
// (target, component), rows 0..nr-1 kept.
// flag: bit 2 set when a staged copy never completed (bounded wait).
// ncols > 0: only columns 0 .. ncols - 1.  pdl: programmatic dependent
// launch on the row transform before it (the set-up and the first kernel-
// spectrum copies overlap that kernel's last CTAs).  discard: the row spectra
// are dead once read, so each column's L2 lines are discarded after its
// forward transform (never written back; the caller reads sh no more).
// staging: kernel-spectrum staging (col_smem_bytes).
template <typename R>
cudaError_t launch_cols(const void *sh, const void *tab, void *oh, int nr, int nphi, int nsrc,
                        uint32_t outmask, const void *tw_col, unsigned int *flag, cudaStream_t s, int ncols = 0,
                        bool pdl = false, bool discard = false, int staging = -1);
// the per-step (FP32) column kernel of a plan shape, L = 2 nr
using ColsKernelF32 = void (*)(const float2 *, const float2 *, float2 *, int, int, uint32_t, const float2 *,
                               unsigned int *, int);
ColsKernelF32 cols_kernel_steps(int nsrc, int L);

// Column pass with tensor-core DFT stages (sg_dftmma.cu): FP32 gas-only
// plans with 2 nr in {2048, 4096}; engine 1..4 as SG_ENGINE_DFT_*; atab
// the A-fragment table of the engine's precision (dftmma_frag_table).
cudaError_t launch_cols_mma(int engine, const void *sh, const void *tab, void *oh, int nr, int nphi, uint32_t outmask,
                            const void *tw_col, const uint32_t *atab, unsigned int *flag, cudaStream_t s);
size_t cols_mma_smem(int nr);

// Column pass with tcgen05 DFT stages (sg_tcdft.cu): FP32 gas-only plans with
// 2 nr in {2048, 4096}; engine SG_ENGINE_TC_*.
cudaError_t launch_cols_tc(int engine, const void *sh, const void *tab, void *oh, int nr, int nphi, uint32_t outmask,
                           const void *tw_col, unsigned int *flag, cudaStream_t s);
// One radix-16 stage alone on the tcgen05 engine `engine`: count 16-point
// DFTs (a multiple of 256) of in -> out, natural order (sg_tc_dft16).
cudaError_t launch_tc_stage(int engine, const void *in, void *out, long long count, int inverse, cudaStream_t s);
// Host: the 8 x 32 x 4 A-fragment words (FP16 if f16, else BF16).
void dftmma_frag_table(bool f16, uint32_t *out);

// Column FFT of a table's row spectra ([nphi/2][L] complex, sg_mem.cuh layout,
// double) and packing into [nphi/2 + 1][tab_pitch(L/2)] complex of type R;
// `odd` for the sin(psi) component (stored multiplied by i).
template <typename R>
cudaError_t launch_tabcols(const void *spec, void *tab, int L, int nphi, bool odd,
                           const void *tw_col64, cudaStream_t s);

struct RowOut {
    void *ptr[6];     // output arrays [nr][nphi]
    int src[6];       // index of the [nphi/2][nr] spectrum in the column output
    int is_phi[6];    // multiply by r_i (potential)
    int n;
};

// Inverse row transforms (C2R) of the column-pass output and the epilogue
// (accelerations divided by r_i, undoing the radial source scaling; finite
// check into *flag bit 1 when flag != NULL).
// tm: the tensor map of oh (all nsrc * 3 spectra); with it, FP32 rows of the
// hot lengths load their tiles by bulk tensor copies, tile_rows (2 or 4) rows
// per CTA, the map's box (bit 2 of *tflag when a copy never completed).
// pdl: programmatic dependent launch on the column pass before it.
template <typename R>
cudaError_t launch_rows_inv(const void *oh, const RowOut &o, int nr, int nphi, const void *tw_row,
                            const void *twp_row, const R *rcen, unsigned int *flag, cudaStream_t s, int row0 = 0,
                            int nrows_run = -1, const CUtensorMap *tm = nullptr, unsigned int *tflag = nullptr,
                            bool pdl = false, int tile_rows = 2);

// Indirect term (App. E): out[2 a + {0, 1}] = (A_a, B_a) in FP64; partial
// holds indirect_blocks(nphi) x 4 doubles.
int indirect_blocks(int nphi);
template <typename R>
cudaError_t launch_indirect(int nr, int nphi, int nsrc, const R *s0, const R *s1, const R *H0, const R *H1,
                            double h0, double h1, const R *rcen, double G, double du, double dphi, double *partial,
                            double *out, cudaStream_t s);

// Semi-spectral method (sg_semi.cu): tables of the phi-DFT of the exact pair
// kernel for axisymmetric scale heights, [pair][component][nphi/2][nr][nr]
// complex of type R (semi_table_bytes); rc_h, H_h[a]: host radial centres
// and the source fluids' H profiles (FP64, nr each).  Synchronises `s`.
size_t semi_table_bytes(int nr, int nphi, int nsrc, bool f64);
template <typename R>
cudaError_t build_semi_tables(int nr, int nphi, int nsrc, double du, double dphi, double G, const double *rc_h,
                              const double *H_h[2], void *tab, const void *tw_row64, const void *twp_row64,
                              cudaStream_t s);
// The per-mode matrix-vector products: row spectra sh ([nsrc][nphi/2][nr])
// -> column output oh ([nsrc * 3][nphi/2][nr]) for the outputs in outmask.
template <typename R>
cudaError_t launch_semi_mv(const void *sh, const void *tab, void *oh, int nr, int nphi, int nsrc, uint32_t outmask,
                           cudaStream_t s);
size_t semi_mv_smem(int nr, int nsrc, bool f64);
cudaError_t set_semi_smem_limits(int max_optin);

// Direct pair sum (general scale heights) for one target fluid.
template <typename R>
cudaError_t launch_direct(int nr, int nphi, double r_in, double du, double G, const R *sig_g,
                          const R *sig_d, const R *Hg, const R *Hd, double h_g, double h_d, int tgt,
                          R *phi, R *gr, R *gphi, const R *geo_i, const R *geo_j, const R *rcen,
                          unsigned int *flag, cudaStream_t s);

}  // namespace sg

// Plan state (sg_api.cu owns its lifetime; sg_batch_api.cu reads the buffers).
struct sg_plan {
    sg_params p{};
    int nsrc = 1;
    bool f64 = false;
    int L = 0, N = 0;
    double du = 0, dphi = 0;
    int device = 0;
    size_t esz = 4;                       // bytes per real element
    void *tw_row = nullptr, *tw_row64 = nullptr;     // exp(-2 pi i k / nphi), k < nphi
    void *twp_row = nullptr, *twp_row64 = nullptr;   // per-pass tables, length nphi / 2
    void *twp_col = nullptr, *twp_col64 = nullptr;   // per-pass tables, length 2 nr
    void *tab = nullptr, *sh = nullptr, *oh = nullptr;
    void *rcen = nullptr, *geo_i = nullptr, *geo_j = nullptr;
    void *Hg = nullptr, *Hd = nullptr;
    unsigned int *flag = nullptr;         // bit 1: non-finite output, bit 2: staging timeout
    double *ipart = nullptr;              // indirect-term partial sums
    void *stage = nullptr;                // sg_solve_host: [2 inputs + 6 outputs][cells]
    int engine = 0;                       // column-pass engine (SG_ENGINE_*)
    uint32_t *atab = nullptr;             // its A-fragment table (tensor-core engines)
    cudaStream_t cstream = nullptr;       // sg_solve_host: copy stream of the pipelined solve
    cudaEvent_t cev[2 * 16] = {};         // sg_solve_host: per-chunk copy / compute events
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};   // sg_set_stage_events
    int rows_fwd = 4, rows_inv = 2;       // launch tiles (sg_set_tiles): rows per CTA of the row transforms
    int cols_staging = -1;                // column-pass staging (-1: default, 0 all at once, 1 per step)
    bool tm_rows = false;                 // tensor maps below are valid (rows_tma_eligible)
    CUtensorMap tm_sh{}, tm_oh{};         // the row transforms' views of sh and oh
    char err[256] = {0};
};

// sg_solve's argument checks and launch chain on `s`, with the status word
// `sflag` (bit 1: non-finite output when check_finite; bit 2: a staged copy
// that never completed) in place of the plan's own (sg_api.cu).
sg_status solve_into(sg_plan *pl, const void *sigma_g, const void *sigma_d, void *const outs[6], cudaStream_t s,
                     unsigned int *sflag, bool check_finite);
