/*
 * sg.h -- C ABI of the GB300 (sm_103a) thin-disc self-gravity library.
 *
 * The library computes the 2-D self-gravity potential Phi and the radial and
 * azimuthal accelerations g_r, g_phi of a Gaussian-stratified thin disc made
 * of gas and an optional dust fluid, on a log-polar grid, with the exact
 * Bessel kernel of Rendon Restrepo et al. (2025), "Self-gravity in thin
 * protoplanetary discs 1":
 *
 *   kernel            Sec. 2.2, Eq. "SG force kernel exact"
 *                     K_ab = (1/sqrt(pi)) H_ab^-2 (d/8) e^X [K1(X) - K0(X)],
 *                     X = d^2/8, d = s/H_ab,
 *   scale height      Sec. 2.2, Eq. "mean root square height"
 *                     H_ab^2 = (H_a(r')^2 + H_b(r)^2) / 2,
 *   acceleration      Sec. 2.2, Eq. "volume force 2D" divided by Sigma_b:
 *                     g_b(r) = -G sum_a int Sigma_a(r') K_ab e_s d^2r',
 *   potential         Sec. 5.6, Eq. "grav. potential 2D":
 *                     Phi_b(r) = -G sum_a int Sigma_a(r') e^X K0(X) / (2 sqrt(pi) H_ab) d^2r',
 *   fast method       Sec. 5.2 and App. C: for constant aspect ratios h_a, h_b
 *                     the sums are convolutions on the log-polar lattice,
 *                     evaluated by a 2-D FFT with the radial direction
 *                     zero-padded to 2 nr; the kernel spectra are built once
 *                     per plan (Sec. 5.2: precomputed for the whole run).
 *
 * Discretisation: nr cells log-spaced between the radial EDGES r_in and
 * r_out, centres r_i = r_in exp((i + 1/2) du), du = ln(r_out/r_in)/nr;
 * nphi cells, centres phi_j = (j + 1/2) 2 pi / nphi.  Cell mass
 * Sigma r_i^2 du dphi (midpoint rule).  The self cell is excluded for every
 * fluid pair.  The paper states no discretisation; this one makes the FFT
 * convolution and the direct pair sum the same finite sum.
 *
 * Memory: every field argument is a caller-owned DEVICE buffer, contiguous
 * row-major [nr][nphi] (phi fastest), in the plan's dtype (float for SG_F32,
 * double for SG_F64), unless a function says otherwise.  The plan owns its
 * kernel spectra and scratch, allocated by sg_plan_create and released by
 * sg_destroy.  sg_solve / sg_potential / sg_accel allocate nothing, never
 * synchronise the host, and enqueue their work on `stream` (a cudaStream_t;
 * NULL is the legacy default stream).  A plan must not be used by two
 * streams at once (its scratch is shared).
 *
 * Errors: arguments are checked on the host before anything is enqueued;
 * a failed check returns SG_ERR_ARG (or SG_ERR_UNSUPPORTED /
 * SG_ERR_NOT_FFT_COMPATIBLE) and enqueues nothing.  A CUDA launch error
 * returns SG_ERR_CUDA.  sg_last_error() gives a one-line description of the
 * plan's most recent failure.
 */
#ifndef SG_H
#define SG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_plan sg_plan;
typedef struct sg_batch sg_batch;

typedef enum {
    SG_OK = 0,
    SG_ERR_ARG = 1,                /* invalid argument (NULL, size, range)          */
    SG_ERR_UNSUPPORTED = 2,        /* valid but not implemented (size, dtype combo) */
    SG_ERR_NOT_FFT_COMPATIBLE = 3, /* FFT method asked with non-constant H          */
    SG_ERR_CUDA = 4,               /* a CUDA runtime call or launch failed          */
    SG_ERR_OOM = 5,                /* device allocation failed                      */
    SG_ERR_NONFINITE = 6,          /* SG_CHECK_FINITE found a NaN/Inf output         */
    SG_ERR_TIMEOUT = 7             /* a bounded device-side wait gave up            */
} sg_status;

enum { SG_F32 = 0, SG_F64 = 1 };                  /* plan dtype                        */
/* App. C convolution / direct sum / semi-spectral (FFT in phi, direct in r) */
enum { SG_METHOD_FFT = 0, SG_METHOD_DIRECT = 1, SG_METHOD_SEMISPECTRAL = 2 };
/* Ordered fluid pairs, source -> target (Sec. 2.2 names the four
 * combinations; pointwise K_gd = K_dg, but the lattice tables differ). */
enum { SG_PAIR_GG = 0, SG_PAIR_GD = 1, SG_PAIR_DG = 2, SG_PAIR_DD = 3 };
enum { SG_COMP_PHI = 0, SG_COMP_R = 1, SG_COMP_AZ = 2 };

#define SG_CHECK_FINITE 2u  /* flag: record NaN/Inf outputs, reported by sg_sync */

typedef struct {
    int32_t nr, nphi;        /* cells.  FFT and SEMISPECTRAL: powers of two,
                                8 <= nr <= 4096, 32 <= nphi <= 8192; FP64 FFT
                                plans stage a column's three kernel spectra in
                                shared memory, so nr <= 2048 gas-only and
                                nr <= 1024 gas + dust (SG_ERR_UNSUPPORTED above).
                                DIRECT: nr >= 1, nphi >= 1                          */
    double r_in, r_out;      /* radial cell edges, 0 < r_in < r_out                 */
    double h_g, h_d;         /* aspect ratios H^sg/r of gas and dust (> 0);
                                h_d <= 0 means a gas-only disc                      */
    const void *H_g_field;   /* DIRECT and SEMISPECTRAL, optional: device [nr][nphi]
                                H_g^sg(r,phi) in the plan dtype (copied at create);
                                NULL = h_g r.  SEMISPECTRAL: every row constant    */
    const void *H_d_field;   /* optional, as above for dust                         */
    double G;                /* gravitational constant (the paper's tests use 1)   */
    int32_t dtype;           /* SG_F32 or SG_F64                                    */
    int32_t method;          /* SG_METHOD_FFT, _DIRECT or _SEMISPECTRAL              */
    uint32_t flags;          /* SG_CHECK_FINITE                                     */
} sg_params;

/* Create a plan: validate `p`, allocate the plan's device memory and, for the
 * FFT method, build the kernel spectra of every fluid pair (Sec. 5.2: the
 * kernel depends on the grid and the aspect ratios only, so it is computed
 * once).  The build runs on `stream`; the call synchronises `stream` before
 * returning.  On success *out holds the plan (owned by the caller, release
 * with sg_destroy); on failure *out is NULL and nothing stays allocated.
 *
 * SG_METHOD_SEMISPECTRAL (Sec. 5.2's route for a non-constant H/r: Fourier
 * transform in phi, direct sum in r) takes scale heights that depend on r
 * only, H_a(r) = h_a r or any positive field whose rows are constant
 * (SG_ERR_ARG otherwise).  The pair kernel then depends on (r, r', phi - phi')
 * and the direct sum is, per azimuthal mode m, one complex nr x nr matrix
 * product.  The plan holds the phi-DFT of the exact pair kernel for every
 * (fluid pair, component, m, r, r'): semi_table size = nsrc^2 x 3 x nphi/2 x
 * nr^2 x (8 FP32 / 16 FP64), 25.8 GB for a 1024 x 2048 gas disc in FP32
 * (SG_ERR_OOM when it does not fit), built from FP64 kernel samples and row
 * transforms.  A solve is the FFT path's row transforms around one pass
 * that streams the tables; its result is the direct sum's (the same finite
 * sum, to the plan dtype's rounding).  sg_kernel_table is FFT only.        */
sg_status sg_plan_create(sg_plan **out, const sg_params *p, void *stream);

/* Write the real-space lattice kernel of one ordered fluid pair and one
 * component (App. C), K_c(Delta_i du, Delta_j dphi) for Delta_i in
 * [-nr, nr) stored circularly in 2 nr rows (row k <-> Delta_i = k for
 * k < nr, k - 2 nr otherwise; row nr, the lag never used, is 0) and Delta_j
 * in [0, nphi):
 *     COMP_PHI: e^{-3D/2} e^X K0(X) / (2 sqrt(pi) h_ab)
 *     COMP_R  : e^{-3D/2} (e^D - cos psi) D(X) / (8 sqrt(pi) h_ab^3)
 *     COMP_AZ : e^{-3D/2} sin psi D(X) / (8 sqrt(pi) h_ab^3)
 * with D = Delta_i du, psi = Delta_j dphi, h_ab^2 = (h_a^2 e^-D + h_b^2 e^D)/2,
 * d^2 = 4 [sinh^2(D/2) + sin^2(psi/2)] / h_ab^2, X = d^2/8, D(X) =
 * e^X [K1(X) - K0(X)] and the self entry (0, 0) = 0.  `out_dev` is a device
 * buffer of 2 nr * nphi elements of the plan dtype.  FFT method only
 * (SG_ERR_UNSUPPORTED otherwise); a dust pair needs a bi-fluid plan.
 * Asynchronous on `stream`.                                                */
sg_status sg_kernel_table(sg_plan *plan, int pair, int comp, void *out_dev, void *stream);

/* Potential of each target fluid, Phi_b = sum over source fluids a of
 * Phi^{ab} (Sec. 5.6, Eq. "grav. potential 2D").  sigma_g: Sigma_g [nr][nphi];
 * sigma_d: Sigma_d, required for a bi-fluid plan and ignored otherwise.
 * phi_g / phi_d: outputs for the gas / dust targets; either may be NULL to
 * skip it (phi_d is ignored for a gas-only plan).  Asynchronous.           */
sg_status sg_potential(sg_plan *plan, const void *sigma_g, const void *sigma_d,
                       void *phi_g, void *phi_d, void *stream);

/* Accelerations g_r, g_phi (force per unit mass, Sec. 2.2 Eq. "volume force
 * 2D" divided by Sigma_b) of each target fluid, summed over the source
 * fluids.  Any output pointer may be NULL to skip it.  Asynchronous.       */
sg_status sg_accel(sg_plan *plan, const void *sigma_g, const void *sigma_d,
                   void *gr_g, void *gphi_g, void *gr_d, void *gphi_d, void *stream);

/* sg_potential and sg_accel fused: one forward transform of each source
 * serves every requested output.  Any output pointer may be NULL.
 * For these three entry points every input and output is a device buffer
 * of nr * nphi elements of the plan dtype, aligned to two elements (8 bytes
 * for SG_F32, 16 for SG_F64; any cudaMalloc or torch allocation is); a
 * misaligned buffer is rejected with SG_ERR_ARG.                           */
sg_status sg_solve(sg_plan *plan, const void *sigma_g, const void *sigma_d,
                   void *phi_g, void *gr_g, void *gphi_g,
                   void *phi_d, void *gr_d, void *gphi_d, void *stream);

/* Indirect term (Sec. 5.4, App. E): the pull of each source fluid a on the
 * central star, as the two sums
 *     A_a = sqrt(2) G sum_cells m_a K_a cos phi',  B_a = sqrt(2) G sum_cells m_a K_a sin phi',
 *     K_a = (1/sqrt(pi)) H_a^-2 (d_a/4) e^{d_a^2/4} [K1 - K0](d_a^2/4),  d_a = r'/H_a,
 * with m_a = Sigma_a r'^2 du dphi and H_a = h_a r' (or the plan's
 * scale-height field).  The indirect potential is
 * Phi_ind = r (A cos phi + B sin phi) with A = sum_a A_a, B = sum_a B_a, and
 * every fluid feels -grad Phi_ind = -(A cos phi + B sin phi) e_r +
 * (A sin phi - B cos phi) e_phi.  ab_dev: device buffer of 2 nsrc doubles
 * receiving (A_g, B_g[, A_d, B_d]), accumulated in FP64 in a fixed order
 * (deterministic).  Both methods; asynchronous on `stream`.              */
sg_status sg_indirect(sg_plan *plan, const void *sigma_g, const void *sigma_d, double *ab_dev, void *stream);

/* sg_solve with HOST buffers: inputs and outputs are host memory (pinned
 * memory gives full copy bandwidth).  The call copies the inputs to
 * plan-owned device buffers, solves, copies the requested outputs back and
 * synchronises `stream` before returning.  The first call allocates the
 * plan's staging buffers.                                                  */
sg_status sg_solve_host(sg_plan *plan, const void *sigma_g, const void *sigma_d,
                        void *phi_g, void *gr_g, void *gphi_g,
                        void *phi_d, void *gr_d, void *gphi_d, void *stream);

/* Synchronise `stream` and report the plan's finite check: SG_ERR_NONFINITE
 * if an output written since the previous sg_sync held a NaN or Inf (plans
 * created with SG_CHECK_FINITE), SG_ERR_CUDA on an asynchronous CUDA error,
 * SG_OK otherwise.  Clears the flag.                                       */
sg_status sg_sync(sg_plan *plan, void *stream);

/* Number of kernel launches one sg_solve call enqueues for the outputs
 * selected by `outmask` (bit 3 b + c for target b in {gas, dust} and
 * component c in SG_COMP_*).                                               */
int32_t sg_launches_per_solve(const sg_plan *plan, uint32_t outmask);

/* Stage timing: with `events` pointing at four cudaEvent_t handles (created
 * by the caller), every following solve records events[0] before its first
 * launch, events[1] after the row transforms, events[2] after the column
 * pass and events[3] after the last launch, on the solve's stream (direct
 * method: events[1..3] after the pair sum).  NULL stops the recording.    */
sg_status sg_set_stage_events(sg_plan *plan, void *const *events);

/* Durations in milliseconds of the three stages of one solve recorded with
 * sg_set_stage_events: ms[0] row transforms, ms[1] column pass, ms[2]
 * inverse row transforms (events[0..3] as recorded; waits for events[3]). */
sg_status sg_stage_times(void *const *events, float *ms);

/* Direct pair sum without a plan and without any device allocation.  (The
 * paper has no counterpart: this serves callers that cannot let a library
 * allocate device memory, such as host codes whose device memory is owned
 * by their own allocator or a fixed pool, and time loops that must never
 * enter the CUDA allocator.)
 *
 * Computes what sg_solve computes for a plan created from `p` with
 * method = SG_METHOD_DIRECT (p->method must say so): Phi, g_r, g_phi of each
 * target fluid; any output may be NULL.  The scale-height fields
 * p->H_g_field / p->H_d_field, when given, are read in place (device
 * buffers in the dtype, kept alive by the caller until the work is done).
 * SG_CHECK_FINITE is ignored.  Inputs and outputs are caller-owned device
 * buffers as for sg_solve; the work is enqueued on `stream`.
 *
 * Scratch: the geometry tables live in one fixed 104 KiB array inside this
 * library (every GPU that loads the library keeps it until the process
 * exits), so grids are limited to nr <= 1024 and nphi <= 4096; larger grids
 * return SG_ERR_UNSUPPORTED with a message on stderr.  The call allocates
 * and frees nothing.  Its first call in a CUDA context looks up the array's
 * device address (cudaGetSymbolAddress) for that context, so make that first
 * call before any stream capture; after cudaDeviceReset the next call looks
 * it up again in the new context.  Every call shares the array and rewrites
 * the part it reads before reading it; calls whose GPU work overlaps (two
 * streams, two host threads) race on it, so serialise them.
 *
 * Errors: SG_ERR_ARG for the parameter sets sg_plan_create rejects (h_g,
 * h_d not finite, h_g <= 0 without H_g_field, a second fluid without
 * sigma_d ...); SG_ERR_CUDA, with nothing launched, when a CUDA error is
 * already pending on the calling thread (left unconsumed for the caller to
 * read), or when a launch of this call fails.                              */
sg_status sg_direct_noalloc(const sg_params *p, const void *sigma_g, const void *sigma_d,
                            void *phi_g, void *gr_g, void *gphi_g,
                            void *phi_d, void *gr_d, void *gphi_d, void *stream);

/* ------------------------------------------------------------------------
 * Launch tiles of an FFT plan's kernels.  The paper fixes no GPU work
 * decomposition (its FFT convolution, Sec. 5.2, runs on CPU cores); these
 * choose how the solve's three kernels split the grid, and do not change
 * what is computed:
 *   rows_fwd, rows_inv  grid rows per CTA (2 or 4) of the forward and the
 *                       inverse row transforms where those move their tiles
 *                       by tensor copies (FP32 plans with nphi in
 *                       {512, 1024, 2048, 4096} and nr % 4 == 0); other plans
 *                       record the value and run their own row kernels.
 *   cols_staging        SG_COLS_STAGE_ALL: the column pass stages every
 *                       requested kernel-spectrum table of a target in shared
 *                       memory at once; SG_COLS_STAGE_STEP: one (target,
 *                       component) step at a time while the source spectra
 *                       stay in registers (FP32 plans only).
 * Defaults: rows_fwd 4, rows_inv 2; per-step staging for FP32 gas + dust and
 * FP32 gas-only plans with nr = 2048, all at once otherwise.  Every tile
 * set performs the same operations on every element, but each kernel
 * variant is compiled separately and fuses multiply-adds in its own way, so
 * solves with different tiles agree to FP32 rounding (relative L2 ~1e-7),
 * not bit for bit; equal tiles give equal bits.  sg_set_tiles re-encodes the
 * plan's tensor maps on the host (no device work, no allocation); solves
 * already enqueued keep the tiles they were launched with.  Errors:
 * SG_ERR_ARG (NULL, a value outside the lists above), SG_ERR_UNSUPPORTED
 * (a direct-method plan, per-step staging of an FP64 plan, a staging whose
 * shared memory exceeds the device's per-block limit).  Batches' stream
 * engine and sg_batch_solve_loop launch with each plan's tiles; a batch's
 * captured graph keeps the tiles its plans had when it was created.       */
enum { SG_COLS_STAGE_ALL = 0, SG_COLS_STAGE_STEP = 1 };
typedef struct {
    int32_t rows_fwd;
    int32_t rows_inv;
    int32_t cols_staging;
} sg_tiles;
sg_status sg_get_tiles(const sg_plan *plan, sg_tiles *tiles);
sg_status sg_set_tiles(sg_plan *plan, const sg_tiles *tiles);

/* ------------------------------------------------------------------------
 * Batches of independent discs.  The paper evolves one disc per run and
 * builds its kernel once per run (Sec. 5.2); a batch binds many FFT plans
 * (uneven grids, gas-only or gas + dust, one dtype, one device) and their
 * device buffers, and solves all of them with ONE persistent kernel launch.
 * That launch works through a task list: for every disc the row transforms of
 * each source, the column pass, and the inverse row transforms of each output.
 * Blocks take tasks in list order from a device counter.  A task that depends
 * on a disc's earlier stage waits, on the device, for that stage's
 * completion count.  The list is ordered so that every wait is on tasks
 * taken before it, and each wait is bounded in time.  The
 * counter reset and the launch are captured once in a CUDA graph, so
 * sg_batch_solve is one graph launch.
 *
 * A second engine (opts.streams > 0) captures instead, in that one graph,
 * every disc's sg_solve launch chain on `streams` forked streams (discs
 * assigned largest first to the least loaded stream), so that the small
 * discs' kernels overlap the large ones'.  Its results are sg_solve's, bit
 * for bit.  The persistent engine's results are sg_solve's to FP32 rounding
 * (its row transforms reduce the row mean and form twiddles in another
 * order) and do not depend on its launch configuration (threads, blocks,
 * task order).  With autotune both engines' candidates are timed.
 * ---------------------------------------------------------------------- */
#define SG_BATCH_HOST_GATE 4u   /* opts flag: blocks wait for sg_batch_release      */

enum { SG_BATCH_ORDER_PIPELINED = 0, SG_BATCH_ORDER_STAGED = 1 };

typedef struct {
    int32_t threads;       /* threads per block, 256 or 512 (0: 256)                 */
    int32_t ctas_per_sm;   /* resident blocks per SM of the persistent grid
                              (0: the occupancy maximum; larger values are capped)   */
    int32_t order;         /* task order: SG_BATCH_ORDER_PIPELINED interleaves the
                              stages of consecutive discs (disc k's rows, k-1's
                              columns, k-2's inverse rows); _STAGED runs every
                              disc's stage s before any stage s+1               */
    int32_t specialize;    /* 1: FP32 transforms of the lengths sg_solve compiles
                              for (rows of nphi 2048 and 4096, columns of 2 nr =
                              1024, 2048, 4096) use compile-time kernels; other
                              lengths and FP64 stay generic                      */
    int32_t autotune;      /* 1: at create, on the bound buffers, first give each
                              plan shape its fastest launch tiles
                              (sg_batch_tile_trials), then time every
                              (specialize, threads, ctas_per_sm, order)
                              candidate of the persistent engine and every
                              stream count of the stream engine, and keep the
                              fastest; those five fields are ignored          */
    uint32_t flags;        /* SG_CHECK_FINITE, SG_BATCH_HOST_GATE                   */
    double timeout_ms;     /* bound of each device-side wait (0: 2000 ms)          */
    int32_t streams;       /* 0: the persistent kernel; 1..64: the per-disc launch
                              chains on this many streams of one graph (threads,
                              ctas_per_sm, order, specialize and timeout_ms are
                              then unused; no SG_BATCH_HOST_GATE)               */
} sg_batch_opts;

/* Bind `n` FFT plans and their buffers into a batch.  For disc k:
 * sigma_g[k], sigma_d[k] (NULL for a gas-only plan) are its inputs and
 * outs[6 k + q] its outputs in sg_solve order (phi_g, gr_g, gphi_g, phi_d,
 * gr_d, gphi_d; NULL skips one; the dust outputs of a gas-only plan must be
 * NULL), all caller-owned device buffers that must stay valid, at the same
 * addresses, for the batch's lifetime (the graph holds the addresses; write
 * each step's inputs into the same buffers).  Every plan keeps owning its
 * kernel spectra and scratch, and must outlive the batch and not be solved on
 * another stream while a batch solve runs.  opts may be NULL (defaults).
 * With opts->autotune the call runs the batch several times on `stream`
 * (outputs are overwritten).  Synchronises `stream`.  Errors: SG_ERR_ARG
 * (NULL, n < 1, mixed dtypes or devices, a direct-method plan, missing
 * sigma_d, a buffer not aligned to two elements), SG_ERR_UNSUPPORTED (a
 * transform longer than 16 x threads:
 * nphi > 8192 or nr > 2048 with 256 threads), SG_ERR_OOM, SG_ERR_CUDA.    */
sg_status sg_batch_create(sg_batch **out, sg_plan *const *plans, int32_t n,
                          const void *const *sigma_g, const void *const *sigma_d,
                          void *const *outs, const sg_batch_opts *opts, void *stream);

/* Solve every disc of the batch: one graph launch (a 4-byte-per-disc
 * counter reset and the persistent kernel, or the per-disc launch chains on
 * forked streams) on `stream`.  Never synchronises the host.  With SG_BATCH_HOST_GATE every block first waits (bounded by
 * timeout_ms) until sg_batch_release is called; each gated solve must then
 * be followed by sg_batch_release and sg_batch_sync before the next.      */
sg_status sg_batch_solve(sg_batch *batch, void *stream);

/* The per-disc baseline: sg_solve on every plan in turn (three launches per
 * disc), same buffers, same results.                                     */
sg_status sg_batch_solve_loop(sg_batch *batch, void *stream);

/* Open the host gate of a SG_BATCH_HOST_GATE batch (a store to mapped host
 * memory that the blocks poll); SG_ERR_ARG for a batch without the gate.  */
sg_status sg_batch_release(sg_batch *batch);

/* Synchronise `stream` and report: SG_ERR_TIMEOUT if a device-side wait of
 * a solve since the last sg_batch_sync gave up (its outputs are incomplete;
 * the context stays usable), SG_ERR_NONFINITE (SG_CHECK_FINITE) if an output
 * held a NaN or Inf, SG_ERR_CUDA on an asynchronous error.  Clears the
 * flags.                                                                 */
sg_status sg_batch_sync(sg_batch *batch, void *stream);

/* The configuration in use (streams, or threads, ctas_per_sm, order;
 * autotune = 1 if it was tuned), the persistent grid size (0 for the stream
 * engine), the number of tasks (kernel launches for the stream engine) and
 * the tuned time per solve in ms (0 when not tuned); any pointer may be
 * NULL.                                                                   */
sg_status sg_batch_config(const sg_batch *batch, sg_batch_opts *opts, int32_t *grid,
                          int32_t *ntasks, float *tuned_ms);

/* The autotuner's engine candidates in the order they were timed (the tile
 * trials before them: sg_batch_tile_trials): writes up to `max`
 * configurations to cfgs and their median times per solve (ms) to ms
 * (either may be NULL) and returns how many were timed (0 without
 * autotune; -1 for a NULL batch).                                         */
int32_t sg_batch_tune_results(const sg_batch *batch, int32_t max, sg_batch_opts *cfgs, float *ms);

/* The autotuner's launch-tile trials (sg_tiles), in the order they were
 * timed: per plan shape (nr, nphi, nsrc), every candidate tile set timed on
 * the first disc of that shape with sg_solve alone (median ms of 5 solves
 * after 2 warm-ups); `chosen` marks the set every disc of the shape was then
 * given (sg_set_tiles on the caller's plans, kept after the batch is
 * destroyed).  The stream engine and sg_batch_solve_loop launch with those
 * tiles; the persistent kernel has its own decomposition (threads,
 * ctas_per_sm).  Writes up to `max` trials to `out` (may be NULL) and returns
 * how many were timed (0 without autotune; -1 for a NULL batch).          */
typedef struct {
    int32_t disc;
    int32_t nr, nphi, nsrc;
    sg_tiles tiles;
    float ms;
    int32_t chosen;
} sg_tile_trial;
int32_t sg_batch_tile_trials(const sg_batch *batch, int32_t max, sg_tile_trial *out);

/* Release the batch (not its plans or buffers).  Synchronises the device. */
void sg_batch_destroy(sg_batch *batch);
const char *sg_batch_last_error(const sg_batch *batch);

/* Column-pass engine of an FFT plan, for the precision study of the DFT
 * stages (Sec. 5.2 FFT convolution evaluated with the DFTs on tensor cores).
 * SG_ENGINE_FFT32 (default): the FP32 register FFT.
 * SG_ENGINE_DFT_*: every radix-16 / radix-8 stage of the column transforms
 * as a block-matrix product on warp-level mma.sync (m16n8k16, FP32
 * accumulate), with FP16 or BF16 operands split into high and low parts and
 * three products summed (..._X3), or a single product.
 * SG_ENGINE_TC_*: the radix-16 stages on the tcgen05 tensor cores (operands
 * in tensor and shared memory, FP32 accumulators in tensor memory): BF16,
 * TF32 or FP16 hi + lo operands with three products (FP16: each tile's
 * operands scaled by a power of two into FP16's range), or one BF16 product;
 * the length-2048 transforms' final radix-8 pass stays on CUDA cores.
 * All need an FP32 gas-only FFT plan with nr = 1024 or 2048
 * (SG_ERR_UNSUPPORTED otherwise); column 0 stays on the FP32 path.  The call
 * allocates a 4 KiB table on the first mma.sync engine and synchronises the
 * device; set it before capturing solves in a graph.  Batches ignore it.  */
enum { SG_ENGINE_FFT32 = 0, SG_ENGINE_DFT_FP16X3 = 1, SG_ENGINE_DFT_BF16X3 = 2, SG_ENGINE_DFT_FP16 = 3,
       SG_ENGINE_DFT_BF16 = 4, SG_ENGINE_TC_BF16X3 = 5, SG_ENGINE_TC_TF32X3 = 6, SG_ENGINE_TC_BF16 = 7,
       SG_ENGINE_TC_FP16X3 = 8 };
sg_status sg_set_column_engine(sg_plan *plan, int32_t engine);

/* One radix-16 stage of a tcgen05 engine alone, for testing it against a
 * plain DFT: `count` independent 16-point DFTs (a positive multiple of 256)
 * of the complex FP32 sequences in[16 q .. 16 q + 15] (interleaved re, im;
 * caller-owned device memory, 8-byte aligned) into out (same layout,
 * natural order; a separate buffer that does not overlap in),
 * X[k] = sum_n x[n] exp(-+ 2 pi i n k / 16) (inverse: +, unnormalised).
 * engine: SG_ENGINE_TC_*.  A CTA runs 256 DFTs (two tensor-core tiles) with
 * the column engine's own operand split, scaling, products and bounded
 * waits.  Errors: SG_ERR_ARG (engine, count, NULL, alignment, overlap),
 * SG_ERR_CUDA.  Async.                                                     */
sg_status sg_tc_dft16(int32_t engine, int64_t count, const void *in, void *out, int32_t inverse, void *stream);

/* ------------------------------------------------------------------------
 * Kernels of the spectral neural-operator surrogate of the field solve
 * (paper_2506_10812_gb300/surrogate.py builds a 4-layer, width-32 spectral
 * neural operator from them, trains it on fields the FFT solve labels and
 * gates it against that exact path).  Every pointer is a caller-owned
 * device buffer, row-major; "bf16" buffers hold bfloat16, the others float.
 * Each call enqueues on `stream` and returns SG_ERR_ARG for NULL,
 * non-positive sizes, a pointer not aligned to its element (float 4 bytes,
 * bf16 2, complex float2 8) or an element count beyond 2^31 - 1 where the
 * kernels index with int, SG_ERR_CUDA for a launch error.
 * ---------------------------------------------------------------------- */

/* Batched GEMM on the tensor cores (bf16 in, FP32 accumulate): for
 * z < batch,
 *   C[z] = alpha op(A[z]) B[z] + beta C[z] (+ bias[n]),
 * op(A) = A ([M][K], leading dim lda) or, with trans_a, A^T (A stored [K][M]);
 * B [K][N] (ldb); C [M][N] (ldc) float and/or C_bf16 (same layout, bf16);
 * stride_* are batch strides in elements (0 broadcasts); bias float [N] or
 * NULL; beta != 0 needs C.  batch <= 65535, N <= 65535 x 128.  lda >= K
 * (M with trans_a), ldb >= N, ldc >= N, strides >= 0, and every pointer
 * aligned to its element (bf16 2 bytes, float 4), else SG_ERR_ARG.
 * Engine (sg_nn_set_gemm_engine, process-wide, read at each call; set it
 * before calls are issued from several host threads): SG_NN_GEMM_TCGEN05 (default)
 * runs 128 x {32, 64, 128} tiles of tcgen05.mma with the accumulator in
 * tensor memory; SG_NN_GEMM_MMA_SYNC the warp-level m16n8k16 kernel, kept
 * for comparison.  Both sum K in the same 16-element groups but in a
 * different order, so they agree to FP32 rounding.  A tensor-core wait that
 * gives up (bounded; never expected) leaves that tile unwritten and is
 * reported by sg_nn_check.                                                */
enum { SG_NN_GEMM_TCGEN05 = 0, SG_NN_GEMM_MMA_SYNC = 1 };
sg_status sg_nn_set_gemm_engine(int32_t engine);
/* Synchronise `stream`; SG_ERR_TIMEOUT if a tensor-core wait of an
 * sg_nn_gemm on this device gave up since the last check (clears it).   */
sg_status sg_nn_check(void *stream);
sg_status sg_nn_gemm(int32_t batch, int32_t M, int32_t N, int32_t K, float alpha, const void *A, int32_t lda,
                     int64_t stride_a, int32_t trans_a, const void *B, int32_t ldb, int64_t stride_b, float beta,
                     float *C, int32_t ldc, int64_t stride_c, void *C_bf16, const float *bias, void *stream);

/* Radial-DFT combine of a spectral convolution: T [B][2 K1][2 M1][C] float
 * (rows < K1: cosine rows, >= K1: minus-sine rows; column 2m + {re, im}) ->
 * V2 [B][K1][M1][C] complex (float2) = (Gc + i Gs)(V1r + i V1i).  _bwd maps
 * the complex gradient dV2 to dT (bf16, same layout as T).              */
sg_status sg_nn_spec_combine(int32_t B, int32_t K1, int32_t M1, int32_t C, const float *T, void *V2, void *stream);
sg_status sg_nn_spec_combine_bwd(int32_t B, int32_t K1, int32_t M1, int32_t C, const void *dV2, void *dT_bf16,
                                 void *stream);

/* Per-mode complex channel mixing: O[b][kk][m][o] = sum_i V2[b][kk][m][i]
 * W[kk][m][i][o] (float2), written as bf16 planes O[b][re, im][kk][m][o].
 * _bwd: from dO (float planes, same layout) the gradients dV2 = dO conj(W)
 * and dW = sum_b conj(V2) dO (either output may be NULL).                */
sg_status sg_nn_modemix(int32_t B, int32_t K1, int32_t M1, int32_t C, const void *V2, const void *W, void *O_bf16,
                        void *stream);
sg_status sg_nn_modemix_bwd(int32_t B, int32_t K1, int32_t M1, int32_t C, const void *V2, const void *W,
                            const float *dO, void *dV2, void *dW, void *stream);

/* y = GELU(x) (gelu_on) or x, float -> bf16; _bwd: dpre = dy GELU'(pre) (or
 * dy) as float and/or bf16.                                             */
sg_status sg_nn_act(int64_t n, const float *x, void *y_bf16, int32_t gelu_on, void *stream);
sg_status sg_nn_act_bwd(int64_t n, const float *pre, const float *dy, float *dpre, void *dpre_bf16, int32_t gelu_on,
                        void *stream);
/* out[c] (+)= sum_r x[r][c] for x [rows][C].                            */
sg_status sg_nn_colsum(int64_t rows, int32_t C, const float *x, float *out, int32_t accumulate, void *stream);
/* Relative L2 of pred against tgt ([B][npix][CH], CH <= 8): stats[(b CH + c)
 * 2 + {0, 1}] = (|pred - tgt|^2, |tgt|^2) per sample and channel; with dpred
 * also the gradient of the mean over (b, c) of their ratio.             */
sg_status sg_nn_rel_l2(int32_t B, int64_t npix, int32_t CH, const float *pred, const float *tgt, float *stats,
                       float *dpred, void *stream);
/* Adam step (bias-corrected for `step` >= 1) on float weights w with
 * moments m, v; also refreshes the bf16 copy w_bf16 when non-NULL.       */
sg_status sg_nn_adam(int64_t n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                     int32_t step, void *w_bf16, void *stream);
/* float -> bf16 copy; transpose of a float [rows][cols] matrix to bf16
 * [cols][rows].                                                          */
sg_status sg_nn_cast(int64_t n, const float *x, void *y_bf16, void *stream);
sg_status sg_nn_transpose(int32_t rows, int32_t cols, const float *x, void *y_bf16, void *stream);
/* Seeded training fields on an nr x nphi log-polar grid for B samples from
 * per-sample parameters (float [B][NPAR], layout in surrogate.py): gas
 * Sigma_g (log-normal-like background, m = 1..6 spirals, Gaussian clumps) and,
 * when sigma_d is non-NULL, dust as a noisy fraction of it; [B][nr][nphi]. */
sg_status sg_nn_fields(int32_t B, int32_t nr, int32_t nphi, const float *params, float *sigma_g, float *sigma_d,
                       void *stream);

/* Network input x [B][nr][nphi][7] (bf16) = (Sigma_g s_g, Sigma_d s_d, h_g / 0.05,
 * h_d / 0.05, (i + 1/2) / nr, cos phi_j, sin phi_j) with per_sample [B][4]
 * = (s_g, s_d, h_g, h_d); sigma_d may be NULL (channel 1 = 0).  Targets:
 * t [B][npix][2] = (a, c) scale[b]; with unpack the inverse (a, c written). */
sg_status sg_nn_pack_inputs(int32_t B, int32_t nr, int32_t nphi, const float *sigma_g, const float *sigma_d,
                            const float *per_sample, void *x_bf16, void *stream);
sg_status sg_nn_pack_targets(int32_t B, int64_t npix, const float *a, const float *c, const float *scale, float *t,
                             int32_t unpack, void *stream);

/* Release a plan and all its device memory (NULL is a no-op).  Synchronises
 * the device before freeing.                                               */
void sg_destroy(sg_plan *plan);

const char *sg_status_string(sg_status s);
const char *sg_last_error(const sg_plan *plan);

#ifdef __cplusplus
}
#endif

#endif /* SG_H */
