/*
 * rg.h -- C ABI of the GB300 GEMM landscape-smoothing library ("rg" = rugged
 * GEMM).  The operations follow the problem statement of "From Roofline to
 * Ruggedness: Decomposing and Smoothing the GEMM Performance Landscape"
 * (arXiv 2605.29752):
 *
 *   C = A * B, A is M x K, B is K x N, C is M x N, all row-major ("NN"),
 *   BF16 operands, FP32 accumulation and output            (Sec. 2.2, Sec. 7.1)
 *   achieved TFLOP/s = 2 M N K / (t 1e12)                   (Sec. 2, definitions)
 *   roughness = mean |T_{i+1} - T_i| along one axis         (Sec. 2, definitions)
 *   T0 -> T1 (padding) -> T2 (splitting) plan table, O(1) lookup   (Sec. 7.1)
 *   dynamic best-of-tiles selection                          (Sec. 6.4)
 *
 * Conventions shared by every call:
 *   - Every call returns an int status (RG_OK or a negative RG_ERR_*); no call
 *     aborts the process.  rg_strerror() names a code; rg_last_error() gives
 *     the calling thread's last detailed message.
 *   - Device pointers are plain CUDA device addresses (for example
 *     torch.Tensor.data_ptr()); the caller owns them and keeps them valid
 *     until the stream work that uses them has finished.
 *   - Calls that take a stream enqueue on it and return without waiting
 *     (stream = NULL means the legacy default stream).  rg_sweep,
 *     rg_plan_build and rg_check synchronise.
 *   - Alignment (TMA): A, B and C must be 16-byte aligned, lda and ldb
 *     multiples of 8 elements, ldc a multiple of 4 elements; otherwise
 *     RG_ERR_ALIGN.  lda >= K, ldb >= N, ldc >= N.
 *   - The library owns rg_ctx (device workspace for split-K partials, tile
 *     tickets, the device error word) and rg_plan objects.
 *   - One rg_ctx serves one device.  Calls that use split-K (split > 1) share
 *     the context's workspace: enqueue them on one stream (or otherwise order
 *     them); overlapping split-K launches on one context race.
 */
#ifndef RG_H
#define RG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
enum {
  RG_OK = 0,
  RG_ERR_INVALID = -1,        /* bad argument (null pointer, negative size, bad id)  */
  RG_ERR_ALIGN = -2,          /* pointer or leading dimension violates TMA alignment */
  RG_ERR_SHAPE = -3,          /* shape outside the plan grid / workspace capacity    */
  RG_ERR_OOM = -4,            /* device or host allocation failed                    */
  RG_ERR_CUDA = -5,           /* a CUDA runtime or driver call failed                */
  RG_ERR_TIMEOUT = -6,        /* a bounded device wait expired (kernel returned)     */
  RG_ERR_PLAN_MISMATCH = -7,  /* plan file header does not match                     */
  RG_ERR_ADMISSION = -8,      /* serving: request can never fit the HBM budget       */
  RG_ERR_NO_DEVICE = -9       /* no usable sm_103 device                             */
};

/* ---- kernel variants ----
 * Eight output tiles (BM x BN): the paper's six (tiles 0..5, RG_NUM_PAPER_TILES,
 * the best-of-6 of Sec. 6.4) and two 192-wide ones, 128 x 192 and 256 x 192,
 * whose 1.5x-wider column tiles fill the 152 SMs where the 128- and 256-wide
 * tiles leave a partial wave.  Each tile has an in-kernel split-K factor S in
 * {1, 2, 4, 8} (id = tile * RG_NUM_SPLITS + log2(S)) and a stream-K schedule
 * (id = RG_VARIANT_SK(tile)); the three 256-row tiles with BN >= 128 (the pair
 * tiles 256x128, 256x256, 256x192, in that order) also run as tcgen05
 * cta_group::2 pairs (RG_VARIANT_2SM).  Ties in best-of selection go to the
 * lowest id.                                                  (Sec. 6.1, 6.4) */
enum {
  RG_TILE_128x64 = 0, RG_TILE_128x128 = 1, RG_TILE_128x256 = 2,
  RG_TILE_256x64 = 3, RG_TILE_256x128 = 4, RG_TILE_256x256 = 5,
  RG_TILE_128x192 = 6, RG_TILE_256x192 = 7,
  RG_NUM_TILES = 8,
  RG_NUM_PAPER_TILES = 6,
  RG_NUM_PAIR_TILES = 3
};
#define RG_NUM_SPLITS 4
#define RG_VARIANT(tile, log2_split) ((tile) * RG_NUM_SPLITS + (log2_split))
/* Stream-K variant of a tile (ids 32..39, after the split-K ids): with T = wP + r
 * tiles on P SMs (0 < r < P), either all whole waves but the last run
 * data-parallel and the K iterations of the last whole wave and the remainder
 * are divided evenly among the P CTAs (w >= 1 and r <= P/4 or r >= P/2; each CTA
 * gets at least one tile's worth, so at most 2 CTAs share a tile), or all whole
 * waves run data-parallel and the r remainder tiles' iterations are divided
 * evenly among up to min(2r, P) CTAs (each at least 4 K blocks).  A tile whose
 * iterations span several CTAs is summed by its last arriving piece in the
 * fixed order of their K ranges. */
#define RG_VARIANT_SK(tile) (RG_NUM_TILES * RG_NUM_SPLITS + (tile))
/* Index of a pair tile among the pair tiles (256x128 -> 0, 256x256 -> 1, 256x192 -> 2). */
#define RG_PAIR_INDEX(tile) ((tile) == RG_TILE_256x192 ? 2 : (tile) - RG_TILE_256x128)
/* 2-SM variant of a 256-row tile (ids 40..43 for 256x128, 44..47 for 256x256,
 * 48..51 for 256x192, split-K 1/2/4/8): a 2-CTA cluster computes one 256 x BN
 * tile as a single tcgen05 cta_group::2 MMA unit; each CTA loads 128 rows of A
 * and BN/2 columns of B (256x192: two 64-column boxes, of which its MMAs read
 * 96) and holds its 128 output rows in its own TMEM, so each SM moves about
 * 128 x BK + BN/2 x BK operand elements per K block instead of 256 x BK + BN x BK.
 * With split-K each CTA publishes and reduces its own 128 rows as in the 1-CTA
 * kernels (same workspace, tickets and fixed summation order).  No kernel of
 * this library uses TMA multicast. */
#define RG_VARIANT_2SM(tile, log2_split) \
  (RG_NUM_TILES * RG_NUM_SPLITS + RG_NUM_TILES + RG_PAIR_INDEX(tile) * RG_NUM_SPLITS + (log2_split))
/* cta_group::2 stream-K variant of a 256-row tile (ids 52, 53, 54 for 256x128,
 * 256x256, 256x192): the stream-K schedule above over 256 x BN pair tiles and
 * the 2-CTA clusters (one per SM pair); each CTA of a cluster sums its own 128
 * rows of a shared tile in the fixed order of the pieces' K ranges.  It removes
 * the partial last wave that quantises the large cells (Sec. 9.4 names split-K
 * as the remedy). */
#define RG_VARIANT_2SM_SK(tile) (RG_NUM_TILES * RG_NUM_SPLITS + RG_NUM_TILES + \
                                 RG_NUM_PAIR_TILES * RG_NUM_SPLITS + RG_PAIR_INDEX(tile))
#define RG_NUM_VARIANTS (RG_NUM_TILES * RG_NUM_SPLITS + RG_NUM_TILES + RG_NUM_PAIR_TILES * RG_NUM_SPLITS + \
                         RG_NUM_PAIR_TILES)

typedef struct rg_ctx rg_ctx;
typedef struct rg_plan rg_plan;

/* One grid axis: sizes start, start + step, ..., start + (count-1) * step. */
typedef struct { int32_t start, step, count; } rg_axis;
/* The (M, N, K) grid.  Cell (a, b, c) has linear index (a * n.count + b) * k.count + c. */
typedef struct { rg_axis m, n, k; } rg_grid;

/* One leaf of a plan: run the box [m0, m0+m) x [n0, n0+n) x [k0, k0+k) of the
 * problem as if it were the padded problem pm x pn x pk (pm >= m, ...), with
 * kernel variant `variant`.  beta = 0 writes C, beta = 1 adds into C.  A leaf
 * may start once every leaf with a lower phase has finished.    (Sec. 7.1) */
typedef struct {
  int32_t variant;
  int32_t beta;
  int32_t phase;
  int32_t reserved;
  int64_t m0, n0, k0;
  int64_t m, n, k;
  int64_t pm, pn, pk;
} rg_leaf;

/* Sweep options (Sec. 3: each configuration's time is the mean of 5 timed
 * launches after one discarded warm-up launch; Sec. 5.4: randomised order). */
typedef struct {
  int32_t reps;               /* timed launches per (variant, cell); default 5       */
  int32_t warmup;             /* untimed launches before them; default 1             */
  int32_t global_warmup;      /* launches before the whole sweep; default 5          */
  int32_t shuffle;            /* 1: randomised (variant, cell) order; default 1      */
  uint64_t seed;              /* shuffle seed; default 0                             */
  int64_t spin_ns;            /* device spin before each timed group, per queued launch,
                                 so the launches queue behind it; default 4000       */
  int32_t prune_splits;       /* 1: skip variants that cannot help on a cell, their
                                 entries set to RG_T_UNMEASURED; default 1:
                                 split-K (S > 1, also cta_group::2) where the unsplit
                                 CTA count already fills the SMs or a split would get
                                 fewer than 2 K blocks; stream-K (also cta_group::2)
                                 where the tiles fill no whole wave or no tile is
                                 split;
                                 cta_group::2 pairs with M <= 128                     */
  int32_t shard_index;        /* with shard_count > 1: this call times only the items at
                                 positions shard_index, shard_index + shard_count, ... of
                                 the randomised, pruned order (identical on identical GPUs
                                 with the same seed) and sets every other measured entry
                                 to RG_T_OTHER_SHARD, so the shards of several GPUs merge
                                 into the whole table (Sec. 3 sweep split over GPUs);
                                 default 0                                             */
  int32_t shard_count;        /* default 1 (no sharding)                             */
  int32_t reserved;
} rg_sweep_opts;
/* Entry of a (variant, cell) pair another shard of a sharded sweep times. */
#define RG_T_OTHER_SHARD ((int64_t)0)
/* Time entry of a (variant, cell) pair the sweep did not measure: larger than
 * any real time, so best-of selection never picks it. */
#define RG_T_UNMEASURED ((int64_t)1 << 60)

/* ---- library / context ---- */
const char* rg_version(void);
const char* rg_strerror(int status);
/* Last detailed error message of the calling thread ("" if none). */
const char* rg_last_error(void);
void rg_sweep_opts_default(rg_sweep_opts* opts);

/* Create a context on CUDA device `device`.  workspace_bytes sizes the split-K
 * partial buffer (0 = default 512 MiB, enough for S = 8 at 4096 x 4096).
 * Fails with RG_ERR_NO_DEVICE unless the device is compute capability 10.3. */
int rg_init(int device, int64_t workspace_bytes, rg_ctx** out);
void rg_destroy(rg_ctx* ctx);
/* Number of SMs of the context's device. */
int rg_sm_count(const rg_ctx* ctx, int32_t* out);
/* Synchronise the stream, then read and clear the device error word.
 * Returns RG_ERR_TIMEOUT if a kernel gave up a bounded wait since the last check. */
int rg_check(rg_ctx* ctx, void* stream);
/* Set the bounded-wait budget in GPU clock cycles for later launches
 * (default 2e9, about a second).  A test may set it tiny to force the timeout path. */
int rg_set_timeout_cycles(rg_ctx* ctx, int64_t cycles);
/* Declare (enable = 1) that A and B of the GEMMs this context launches from now
 * on are not written by any work enqueued before them on their stream (static
 * operands, such as weights).  The kernels then start loading A and B and
 * running their MMAs before the preceding grid in the stream has completed
 * (programmatic dependent launch); only the epilogue, which writes C and the
 * split-K workspace, waits for it, so independent GEMMs on static operands
 * overlap on idle SMs.  Default 0: every global access waits.  rg_sweep and
 * rg_sweep_memtwin always time with it off (a timed launch must not overlap the
 * previous one's work) and restore the setting afterwards.  Enabling it while a
 * preceding kernel writes A or B is a data race.  Errors: RG_ERR_INVALID for a
 * null context. */
int rg_set_static_operands(rg_ctx* ctx, int32_t enable);
/* Failure-path testing: while enabled, every GEMM launch of this context first
 * makes its MMA warp wait on a barrier that nothing arrives on, so that bounded
 * wait expires after the timeout budget; the kernel then records the error,
 * lets its in-flight copies land, releases TMEM and returns, and rg_check
 * reports RG_ERR_TIMEOUT.  Off by default. */
int rg_set_test_stall(rg_ctx* ctx, int32_t enable);
/* Phase timers, a compile-time option of the library (built with RG_PHASE_TIMERS=1,
 * e.g. `python -m paper_2605_29752_gb300.build --phase-timers`): while enabled,
 * every BF16 GEMM launch of this context writes per-CTA stamps into a buffer the
 * context owns (each launch overwrites it), kTraceFields = 12 uint64 per CTA:
 *   0 globaltimer at entry (ns), 1 globaltimer at exit (ns), 2 SM clock at exit,
 *   3 dependency wait done, 4 first operand stage landed, 5 last MMA commit,
 *   6 first accumulator ready in the epilogue, 7 epilogue done,
 *   8 first split-K fixup start, 9 split-K fixup end, 10 work units of the CTA,
 * SM-clock fields counted in cycles from the CTA's entry (0 = not reached).
 * rg_phase_trace_read synchronises the device, copies the records of up to
 * max_ctas CTAs (the SM count at most) to `out` and clears the buffer.  In a
 * library built without the option both return RG_ERR_INVALID. */
#define RG_TRACE_FIELDS 12
int rg_phase_trace(rg_ctx* ctx, int32_t enable);
int rg_phase_trace_read(rg_ctx* ctx, uint64_t* out, int32_t max_ctas, int32_t* n_ctas);
/* Number of kernel launches this context has enqueued so far (GEMM kernels and
 * the sweep's spin kernels). */
int rg_launch_count(const rg_ctx* ctx, int64_t* out);

/* ---- GEMM (Sec. 2.2; variants Sec. 6.1; fused padding / split-K Sec. 7.1) ----
 * C = A * B (beta = 0) or C += A * B (beta = 1).  variant in [0, RG_NUM_VARIANTS).
 * A: M x K BF16 (lda), B: K x N BF16 (ldb), C: M x N FP32 (ldc), device memory.
 * (pm, pn, pk) >= (M, N, K) run the launch as the zero-padded problem of that
 * size (pass 0 for "same as M, N, K"); the padding is never materialised:
 * out-of-range operand reads are zero-filled and out-of-range outputs dropped.
 * M, N or K == 0: nothing to compute (C untouched if M or N is 0; C = 0 for
 * K == 0 with beta = 0).  Split-K (S > 1) of the 128x256, 256x128, 256x256 and
 * 256x192 1-CTA tiles (not 256x256 with S = 8) runs as clusters of S CTAs that sum the
 * S partials through distributed shared memory; the other split variants sum
 * them through the context's workspace.  Both sum in the order 0..S-1, so the
 * two forms give the same bits. */
int rg_gemm(rg_ctx* ctx, int64_t M, int64_t N, int64_t K,
            const void* A, int64_t lda, const void* B, int64_t ldb,
            float* C, int64_t ldc, int32_t variant, int32_t beta,
            int64_t pm, int64_t pn, int64_t pk, void* stream);

/* ---- plan table (Sec. 7.1, host) ----
 * T0_ns: [n_variants][cells] int64 nanoseconds (cells in the grid's linear
 * order), variant_ids[v] the library variant measured in row v: BF16 ids
 * (0..RG_NUM_VARIANTS-1) or FP8 ids (RG_FP8_VARIANT_BASE..), not both.  Builds
 * best-of selection, T1 (padding), T2 (splitting) and every cell's leaf list.
 * The grid must have start == step on every axis (whole multiples of the step),
 * except with RG_PLAN_PAD_ONLY, where any grid is accepted (padding moves to a
 * larger grid cell; nothing is split). */
int rg_plan_build(const rg_grid* grid, const int64_t* T0_ns, int32_t n_variants,
                  const int32_t* variant_ids, rg_plan** out);
/* As rg_plan_build with flags: RG_PLAN_PAD_ONLY stops after T1 (padding only:
 * T2 = T1, every action "keep"), the "DP pad" stage of the paper's ladder
 * (Sec. 7.5, Table 10).  flags = 0 is rg_plan_build. */
#define RG_PLAN_PAD_ONLY 1
int rg_plan_build_ex(const rg_grid* grid, const int64_t* T0_ns, int32_t n_variants,
                     const int32_t* variant_ids, int32_t flags, rg_plan** out);
void rg_plan_free(rg_plan* plan);
int rg_plan_grid(const rg_plan* plan, rg_grid* out);
/* Copy out the plan's tables (any pointer may be NULL), each [cells] in the
 * grid's linear order: T0* (best-of time), vstar (its variant id), T1, the pad
 * target cell (3 ints per cell), T2, action (0 keep, 1 split M, 2 split N,
 * 3 split K) and q (second piece size in steps). */
int rg_plan_tables(const rg_plan* plan, int64_t* T0s, int32_t* vstar, int64_t* T1,
                   int32_t* target3, int64_t* T2, int32_t* action, int32_t* q);
/* O(1) lookup: the cell that covers (M, N, K) (each size rounded up to the
 * grid) and its leaves (a pointer into the plan, valid until rg_plan_free).
 * RG_ERR_SHAPE if a size exceeds the grid.  t2_ns may be NULL. */
int rg_plan_lookup(const rg_plan* plan, int64_t M, int64_t N, int64_t K,
                   const rg_leaf** leaves, int32_t* n_leaves, int64_t* t2_ns);
/* Execute the plan for C = A * B: lookup, then the cell's leaves in order on
 * `stream`, each clipped to (M, N, K).  Operand conventions as rg_gemm. */
int rg_gemm_plan(rg_ctx* ctx, const rg_plan* plan, int64_t M, int64_t N, int64_t K,
                 const void* A, int64_t lda, const void* B, int64_t ldb,
                 float* C, int64_t ldc, void* stream);
/* rg_gemm_plan on HOST buffers, for callers whose operands live in host memory:
 * copies A (M x K, lda) and B (K x N, ldb) from the host into device staging
 * buffers the context owns (allocated on first use and grown when a larger
 * problem comes; leading dimensions rounded up to the TMA alignment there),
 * executes the plan on `stream`, copies C (M x N, ldc) back and synchronises
 * the stream, so C holds the result on return.  Host buffers may be pageable
 * or pinned (pinned memory makes the copies asynchronous DMA).  M, N, K > 0.
 * Errors: those of rg_gemm_plan, RG_ERR_OOM for a staging buffer,
 * RG_ERR_TIMEOUT as rg_check.  Not for concurrent use of one context. */
int rg_gemm_plan_host(rg_ctx* ctx, const rg_plan* plan, int64_t M, int64_t N, int64_t K,
                      const void* A, int64_t lda, const void* B, int64_t ldb,
                      float* C, int64_t ldc, void* stream);
/* Binary plan file with a header (magic, version, grid, variant set, device
 * name, SM count) and an FNV-1a checksum of the body.  rg_plan_load checks
 * the header against `ctx`'s device (ctx may be NULL to skip the device check). */
int rg_plan_save(const rg_plan* plan, const rg_ctx* ctx, const char* path);
int rg_plan_load(const char* path, const rg_ctx* ctx, rg_plan** out);

/* ---- variant and schedule queries (host; no device needed) ----
 * rg_variant_desc: out = {tile, split factor (1 for stream-K), stream-K (0/1),
 * cta_group::2 (0/1), BM, BN} of BF16 variant `v` in [0, RG_NUM_VARIANTS); the
 * pair forms report their 256-row tile.  RG_ERR_INVALID for another id.
 * rg_streamk_geometry: the stream-K schedule of `tiles` output tiles (pair tiles
 * for a cta_group::2 variant) of `kblocks` 64-deep K blocks on `units` CTAs
 * (clusters): out = {CTAs (clusters) launched, tiles run whole data-parallel,
 * CTAs (clusters) sharing the remaining tiles' K iterations, most CTAs sharing
 * one tile}, as the stream-K variants' launcher and kernel use it.  tiles,
 * kblocks, units > 0, else RG_ERR_INVALID. */
int rg_variant_desc(int32_t v, int32_t out[6]);
int rg_streamk_geometry(int64_t tiles, int64_t kblocks, int64_t units, int64_t out[4]);

/* ---- surface statistics (Sec. 2 definitions; Sec. 8.6 conventions; host) ----
 * tflops_out[c] = (2.0*M*N*K) / (t_ns[c] * 1e3) per cell (may be NULL);
 * rough_out = {R_M, R_N, R_K, R_3D = (R_M+R_N+R_K)/3, R_N on the largest-K slice};
 * mean_out = mean TFLOP/s.  Sums are correctly rounded, so the results do not
 * depend on summation order.  t_ns must be > 0. */
int rg_surface_stats(const rg_grid* grid, const int64_t* t_ns, double* tflops_out,
                     double rough_out[5], double* mean_out);

/* ---- grouped GEMM under CUDA graphs (many problems, one persistent launch per kernel family) ----
 * A group runs a list of independent NN GEMMs.  Each problem names the kernel
 * variant the autotuner chose for it: a 1-CTA tile with in-kernel split-K
 * (S = 1/2/4/8) or a cta_group::2 pair tile with split-K; a stream-K variant
 * runs as its tile with split 1; variant = -1 means the group's tile, split 1.
 * The problems are sorted into eleven kernel families (the eight 1-CTA tiles, the
 * three cta_group::2 tiles); each family present becomes one persistent launch
 * over all SMs whose work units are the concatenation of its problems'
 * (tile, K split) units.  Each problem has its own sizes, operands, leading
 * dimensions, beta and padded launch extents (pm, pn, pk as in rg_gemm;
 * 0 = no padding).  The split-K partials and tickets live in a workspace the
 * group owns (workspace_bytes, at least 1 MiB); when a family's problems need
 * more than it holds at once, the family runs as several launches in turn.
 * The launches of one call run one after another on `stream`; problems of one
 * call must not write overlapping parts of C (they may run concurrently).
 * A result is bitwise that of rg_gemm with the same variant (same split
 * boundaries and summation order), whatever else the call contains.
 * rg_group_create allocates the workspace and tickets and, for each family,
 * kGroupSlots = 4 slots of work lists (pinned host + device, for max_items
 * problems each), instantiating one CUDA graph per slot: [copy the host list
 * to the device list, grouped kernel].  rg_gemm_grouped allocates nothing: it
 * fills the next slot of each family it uses (waiting first until that slot's
 * replay from 4 launches ago has finished), then replays its graph on `stream`;
 * the call returns without waiting for the GEMMs.  Operand conventions and
 * alignment are those of rg_gemm; every problem is checked before anything is
 * enqueued (RG_ERR_SHAPE for one whose partials alone exceed the workspace);
 * K == 0 problems are rejected.  One group serves one stream at a time. */
typedef struct {
  int64_t M, N, K;
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  float* C;
  int64_t ldc;
  int64_t pm, pn, pk;
  int32_t beta;
  int32_t variant;            /* kernel variant, or -1 for the group's tile with split 1 */
} rg_group_problem;
typedef struct rg_group rg_group;
int rg_group_create(rg_ctx* ctx, int32_t tile, int32_t max_items, int64_t workspace_bytes, rg_group** out);
void rg_group_destroy(rg_group* group);
int rg_gemm_grouped(rg_group* group, const rg_group_problem* problems, int32_t n, void* stream);

/* ---- serving: continuous batching over the grouped GEMM ----
 * One engine serves GEMM requests of arbitrary shape with operands resident in
 * device memory.  Requests are admitted in arrival order once arrived and once
 * their operand bytes (2MK + 2KN + 4MN) fit under hbm_budget_bytes next to the
 * admitted, unfinished requests; one that can never fit is rejected with
 * RG_ERR_ADMISSION in its result.  Each request goes through rg_plan_lookup
 * (plan may be NULL) and becomes its plan cell's leaves (Sec. 7.1): sub-boxes
 * of the problem, each with the variant the autotuner chose for it (tile,
 * split factor, cta_group::2; a stream-K choice runs as its tile, split 1),
 * its padded launch extents, beta and phase; without a plan a request is one
 * leaf on opts->tile.  Whenever one of max_inflight slots is free, up to
 * max_batch admitted requests form one batch on that slot's stream: for each
 * phase in order, one rg_gemm_grouped call over that phase's leaves of the
 * whole batch, so batches formed while others run overlap them on the device;
 * finished batches release budget and admit waiting requests.  A request's
 * result is bitwise the same alone and in any mix.  A request with C == NULL
 * gets its output (ldc = N) from an arena of hbm_budget_bytes allocated by the
 * engine and released when it stops (its values are then gone: for load
 * tests).  Times in results are nanoseconds on the host's steady clock from
 * the engine's start.  A, B and (non-NULL) C are device memory the caller keeps
 * valid until the request has finished.
 *
 * rg_serve replays a trace on the calling thread and returns when every
 * request has finished or been rejected; arrival_ns (non-decreasing) are the
 * trace's arrival times.  The online form runs the same engine on a worker
 * thread: rg_serve_start creates it, rg_serve_submit enqueues one request (its
 * arrival is the submission; arrival_ns is ignored) and returns its id (0, 1,
 * ... in submission order), rg_serve_poll reports without blocking whether a
 * request has finished (done = 1 and its result), rg_serve_wait blocks until it
 * has, and rg_serve_stop waits for every submitted request, stops the worker,
 * frees the engine and fills the statistics.  Submit, poll and wait may be
 * called from any thread; a server uses its context's device on its own
 * streams.  A CUDA failure stops the worker; later calls return its status. */
typedef struct {
  int64_t hbm_budget_bytes;   /* default 64 GiB */
  int32_t max_batch;          /* requests per batch; default 64 */
  int32_t max_inflight;       /* batches on the GPU at once, 1..16; default 2 */
  int32_t tile;               /* tile for requests without a plan; default RG_TILE_128x128 */
  int32_t workspace_mib;      /* split-K workspace of each in-flight slot, MiB; default 256 */
  const rg_plan* fp8_plan;    /* plan for FP8 requests (FP8 variant ids), or NULL: one 128x256 leaf */
} rg_serve_opts;
/* Request precision: BF16 operands A, B (the default), or FP8 e4m3 operands with
 * per-128x128-block FP32 scales (A = qA, B = qB; sA, sB and their leading
 * dimensions as rg_gemm_fp8_ex).  An FP8 request goes through opts->fp8_plan and
 * its leaves run on the batch's stream after that phase's grouped BF16 launch;
 * its operand bytes are MK + KN + 4MN plus the scales. */
#define RG_DTYPE_BF16 0
#define RG_DTYPE_FP8 1
typedef struct {
  int64_t M, N, K;
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  float* C;
  int64_t ldc;
  int64_t arrival_ns;
  int32_t dtype;              /* RG_DTYPE_BF16 or RG_DTYPE_FP8 */
  int32_t reserved;
  const float* sA;            /* FP8 only */
  int64_t lds_a;
  const float* sB;            /* FP8 only */
  int64_t lds_b;
} rg_serve_request;
typedef struct {
  int64_t admitted_ns, launched_ns, done_ns;
  int32_t batch;              /* index of the batch that ran it, -1 if none */
  int32_t status;             /* RG_OK; RG_ERR_ADMISSION (never fits the budget); RG_ERR_SHAPE (beyond the
                                 plan grid); or, from the checks of rg_gemm made at admission,
                                 RG_ERR_INVALID / RG_ERR_ALIGN / RG_ERR_SHAPE */
} rg_serve_result;
typedef struct {
  int64_t requests, batches, admission_stalls;
  double wall_s, p50_latency_us, p99_latency_us, mean_latency_us;
  double tflops;              /* useful 2MNK of served requests / (last completion - first arrival) */
} rg_serve_stats;
void rg_serve_opts_default(rg_serve_opts* opts);
int rg_serve(rg_ctx* ctx, const rg_plan* plan, const rg_serve_opts* opts, const rg_serve_request* requests,
             int32_t n, rg_serve_result* results, rg_serve_stats* stats);
typedef struct rg_server rg_server;
int rg_serve_start(rg_ctx* ctx, const rg_plan* plan, const rg_serve_opts* opts, rg_server** out);
int rg_serve_submit(rg_server* server, const rg_serve_request* request, int64_t* id_out);
int rg_serve_poll(rg_server* server, int64_t id, rg_serve_result* result, int32_t* done);
int rg_serve_wait(rg_server* server, int64_t id, rg_serve_result* result);
int rg_serve_stop(rg_server* server, rg_serve_stats* stats);

/* ---- FP8 e4m3 with FP32 scales per 128 x 128 block (precision variant of the GEMM) ----
 * rg_fp8_quantize: X (rows x cols FP32, ldx) -> Q (e4m3 bytes, ldq) and scales
 * [ceil(rows/128)][ceil(cols/128)] (row-major, FP32): per block amax, s = amax / 448
 * (IEEE division; s = 1 for an all-zero block), Q = e4m3(x / s) rounded to nearest
 * even with saturation to +-448.
 * FP8 GEMM: C (M x N FP32, ldc) = sum over 128-deep K blocks kb of
 * sA[i/128][kb] * sB[kb][j/128] * (qA * qB restricted to kb), FP32 accumulation;
 * qA M x K e4m3 (lda), sA [ceil(M/128)] rows of lds_a >= ceil(K/128) scales,
 * qB K x N e4m3 (ldb), sB [ceil(K/128)] rows of lds_b >= ceil(N/128) scales, as
 * produced by rg_fp8_quantize.  qA, qB, C 16-byte aligned; lda, ldb multiples of
 * 16; ldc a multiple of 4.  Device pointers, stream-ordered.
 * FP8 kernel variants (ids in their own range, RG_FP8_VARIANT_BASE + ...): the
 * 128 x 256 and 128 x 128 output tiles (FP8 tile 0 and 1) and the 256 x 256 tile
 * as a tcgen05 cta_group::2 pair on a 2-CTA cluster (FP8 tile 2: each CTA loads
 * its 128 rows of A and 128 columns of B, and promotes and stores its own 128
 * output rows), each with in-kernel split-K S = 1/2/4/8, id =
 * RG_FP8_VARIANT(tile, log2(S)).  Split-K partials go through the context's
 * workspace and are summed by the last arriving split in the fixed order
 * 0..S-1, so results are deterministic.
 * rg_gemm_fp8_ex: one launch of `variant`, beta = 0 writes C, beta = 1 adds into
 * it; (pm, pn, pk) >= (M, N, K) run it as the zero-padded problem of that size (0
 * = same), never materialised (zero-filled reads, clipped stores, scales of
 * padding blocks read as 0).  Errors as rg_gemm (RG_ERR_SHAPE when split-K
 * partials exceed the workspace), and RG_ERR_CUDA, before any launch, when the
 * library's FP8 kernels were not built with the 168 registers per thread that
 * their in-kernel register split (setmaxnreg) adds up to.  rg_gemm_fp8 = rg_gemm_fp8_ex with variant
 * RG_FP8_VARIANT(0, 0), compact scales (lds_a = ceil(K/128), lds_b = ceil(N/128)),
 * beta 0 and no padding.
 * rg_gemm_fp8_plan: the O(1) plan lookup (Sec. 7.1) of an FP8 plan (a plan built
 * by rg_plan_build from FP8 variant ids), then the cell's leaves in order, each
 * on the sub-views of qA, sA, qB, sB and C its box selects; the boxes' offsets
 * must be multiples of 128 (grid steps that are), else RG_ERR_SHAPE.  A BF16
 * plan is refused (RG_ERR_INVALID), as rg_gemm_plan refuses an FP8 plan. */
#define RG_FP8_VARIANT_BASE 64
#define RG_FP8_NUM_TILES 3
#define RG_FP8_VARIANT(tile, log2_split) (RG_FP8_VARIANT_BASE + (tile) * RG_NUM_SPLITS + (log2_split))
#define RG_FP8_NUM_VARIANTS (RG_FP8_NUM_TILES * RG_NUM_SPLITS)
int rg_fp8_quantize(rg_ctx* ctx, const float* X, int64_t rows, int64_t cols, int64_t ldx, uint8_t* Q,
                    int64_t ldq, float* scales, void* stream);
int rg_gemm_fp8(rg_ctx* ctx, int64_t M, int64_t N, int64_t K, const uint8_t* qA, int64_t lda, const float* sA,
                const uint8_t* qB, int64_t ldb, const float* sB, float* C, int64_t ldc, void* stream);
int rg_gemm_fp8_ex(rg_ctx* ctx, int64_t M, int64_t N, int64_t K, const uint8_t* qA, int64_t lda, const float* sA,
                   int64_t lds_a, const uint8_t* qB, int64_t ldb, const float* sB, int64_t lds_b, float* C,
                   int64_t ldc, int32_t variant, int32_t beta, int64_t pm, int64_t pn, int64_t pk, void* stream);
int rg_gemm_fp8_plan(rg_ctx* ctx, const rg_plan* plan, int64_t M, int64_t N, int64_t K, const uint8_t* qA,
                     int64_t lda, const float* sA, int64_t lds_a, const uint8_t* qB, int64_t ldb, const float* sB,
                     int64_t lds_b, float* C, int64_t ldc, void* stream);
/* Times FP8 GEMMs on every cell of `grid` with the sweep protocol and outputs of
 * rg_sweep (same options; split pruning as rg_sweep's for split-K, and the pair
 * tile pruned where M <= 128): n_variants
 * FP8 variant ids, or a plan (n_variants = 1, ids ignored).  Cell (M, N, K) uses
 * the contiguous prefixes qA[0 : M*K] (lda = K) and qB[0 : K*N] (ldb = N) with
 * compact scale arrays read from sA and sB (they must hold the largest cell's
 * blocks); C holds max M * max N floats.  Grid sizes must be multiples of 16.
 * t_ns_out[v][cell], tflops_out[v][cell] and stats_out[v][6] as in rg_sweep. */
int rg_sweep_fp8(rg_ctx* ctx, const rg_grid* grid, int32_t n_variants, const int32_t* variant_ids,
                 const rg_plan* plan, const uint8_t* qA, const float* sA, const uint8_t* qB, const float* sB,
                 float* C, const rg_sweep_opts* opts, int64_t* t_ns_out, double* tflops_out, double* stats_out,
                 void* stream);

/* ---- first-principles landscapes (Sec. 9.1, 9.2) and kernel grading (Sec. 10; host) ----
 * out[cell] = achieved TFLOP/s of the analytic landscape on `grid`:
 *   RG_LANDSCAPE_IDEAL:   P * min(1, W / C), W = ceil(M/BM) ceil(N/BN) for tiles[0]
 *                         (the compute ceiling with its partial-wave ramp, Sec. 9.1);
 *   RG_LANDSCAPE_OPTIMAL: 2MNK / min over the n_tiles tiles of max(t_compute, t_memory),
 *                         t_compute = 2MNK / (P * eta_wave), eta_wave = W / (ceil(W/C) C),
 *                         t_memory = 2MK/(BW eta_A) + 2KN/(BW eta_B) + 4MN/(BW eta_D)  (Sec. 9.2).
 * P = p_tflops (TFLOP/s), C = c_units (SMs, or SM pairs for 2-CTA tiles), BW = bw_gbs (GB/s),
 * tiles = n_tiles (BM, BN) pairs.  channels > 0 selects the paper's interleaved-channel model
 * for eta (channels, interleave bytes); channels = 0 sets every eta to 1 (HBM, no disclosed hash). */
#define RG_LANDSCAPE_IDEAL 0
#define RG_LANDSCAPE_OPTIMAL 1
int rg_landscape(const rg_grid* grid, int32_t mode, double p_tflops, int32_t c_units, double bw_gbs,
                 int32_t n_tiles, const int32_t* tiles, int32_t channels, int32_t interleave, double* out);
/* Kernel Optimality Level (Sec. 10.2-10.3, Table 19): tau = mean_a / mean_o, rho = r_a / r_o;
 * T band 0..3 at tau 0.50 / 0.75 / 0.95; S band 3 for rho <= 1.25, 2 up to 2, 1 up to 3, else 0;
 * level = min(T, S).  out = {tau, rho}, bands = {T, S, L}. */
int rg_kol(double mean_a, double mean_o, double r_a, double r_o, double out[2], int32_t bands[3]);

/* ---- sweep (Sec. 3, Sec. 5.4; surface and roughness, Sec. 2 and Sec. 8.6) ----
 * Times every (variant, cell) pair: for each, `warmup` untimed launches, a
 * short device spin, then `reps` launches between two CUDA events;
 * t_ns_out[v][cell] = round(elapsed / reps) in ns.  Operands of cell (M, N, K)
 * are the contiguous prefixes A[0 : M*K] (lda = K) and B[0 : K*N] (ldb = N);
 * C must hold max M * max N floats.  If plan != NULL the single timed item per
 * cell is the plan's execution (n_variants must be 1, variant ids ignored).
 * Besides the times it returns, per timed row v, the throughput surface
 * tflops_out[v][cell] and stats_out[v][6] = {R_M, R_N, R_K, R_3D, R_N on the
 * largest-K slice, mean TFLOP/s}, exactly as rg_surface_stats computes them
 * from t_ns_out (correctly rounded sums).  A row with cells the pruning left
 * unmeasured (or another shard times) has TFLOP/s 0 there and NaN statistics.  Either pointer may be
 * NULL.  Synchronises; returns RG_ERR_TIMEOUT if a kernel gave up a wait. */
int rg_sweep(rg_ctx* ctx, const rg_grid* grid, int32_t n_variants, const int32_t* variant_ids,
             const rg_plan* plan, const void* A, const void* B, float* C,
             const rg_sweep_opts* opts, int64_t* t_ns_out, double* tflops_out, double* stats_out, void* stream);

/* ---- four-surface decomposition (Sec. 4, Figs. 5-6, Table 3) ----
 * The memory twin of a tile runs the tile's GEMM kernel (split 1, beta 0) with
 * every MMA replaced by a no-op: the same TMA loads of A and B, the same
 * pipeline, TMEM read-back and TMA stores of C.  C receives whatever the
 * accumulators held (undefined values): the twin exists to be timed.
 * rg_gemm_memtwin: one launch, arguments and errors as rg_gemm with variant
 * RG_VARIANT(tile, 0).  rg_sweep_memtwin: rg_sweep's protocol and operand
 * conventions over the n_tiles tile ids (0..RG_NUM_TILES-1); nothing is pruned;
 * t_ns_out[t][cell]. */
int rg_gemm_memtwin(rg_ctx* ctx, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B,
                    int64_t ldb, float* C, int64_t ldc, int32_t tile, void* stream);
int rg_sweep_memtwin(rg_ctx* ctx, const rg_grid* grid, int32_t n_tiles, const int32_t* tile_ids, const void* A,
                     const void* B, float* C, const rg_sweep_opts* opts, int64_t* t_ns_out, void* stream);
/* Host.  Per cell of `grid` (times in ns, all > 0; P = p_tflops > 0):
 *   compute_ns_out[cell]  = (2.0 * M * N * K) / (P * 1e3)          (useful flops at peak)
 *   overhead_ns_out[cell] = t_gemm - max(compute, t_mem)            (may be negative)
 * stats_out = {share of cells with compute > t_mem (compute-bound),
 *              mean over cells of overhead / t_gemm,
 *              sum overhead / sum t_gemm,
 *              mean over cells of t_mem / t_gemm}.
 * Any output may be NULL.  Sums are correctly rounded.  Errors: RG_ERR_INVALID. */
int rg_decompose(const rg_grid* grid, const int64_t* t_gemm_ns, const int64_t* t_mem_ns, double p_tflops,
                 double* compute_ns_out, double* overhead_ns_out, double stats_out[4]);

/* ---- GEMM without device allocation ----
 * The paper has no counterpart to this entry point.  It is for callers that
 * must not allocate device memory on their call path (a host framework whose
 * own allocator owns the device memory budget, or code that cannot afford the
 * implicit device synchronisation cudaMalloc may cause).  It computes exactly
 * what rg_gemm computes (same kernel, same summation order) but needs no
 * rg_ctx: its split-K scratch -- partial sums, tile tickets and the
 * bounded-wait error word -- lives in one fixed device array inside the
 * library, RG_NOALLOC_PARTIAL_BYTES of partials plus tickets for
 * RG_NOALLOC_MAX_TILES output tiles (about 16.3 MiB), which every GPU that
 * loads the library holds until the process exits.
 *   - Runs on the calling thread's current device, on `stream`.  The caller
 *     still owns and passes A, B and C (device memory, rg_gemm conventions).
 *   - The first call on a device does a one-time set-up on that device (device
 *     check, kernel attributes, the scratch array's device address); make that
 *     first call before any stream capture.
 *   - Split-K launches (variant with S > 1) whose partials would exceed the
 *     scratch (S * tiles * BM * BN * 4 > RG_NOALLOC_PARTIAL_BYTES, or more than
 *     RG_NOALLOC_MAX_TILES tiles) are rejected with RG_ERR_SHAPE before any
 *     work is enqueued; split 1 has no size limit beyond rg_gemm's.
 *   - Every call shares the one scratch array and it keeps the previous call's
 *     contents; each call clears the tickets and error word it uses (an async
 *     memset on `stream`).  Calls whose work overlaps on the GPU (other streams,
 *     other threads) race on the scratch: order them.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 *   - RG_OK means the launch was enqueued, not that it finished.  A bounded
 *     wait that expires inside the kernel (which then returns with C partly
 *     written) is recorded in the scratch's error word; rg_noalloc_check reads
 *     it.  The next rg_gemm_noalloc call clears that word, so check before it.
 *   - With the tiles of this library the ticket limit never binds before the
 *     partial-byte limit (a launch whose partials fit has at most 256 tiles);
 *     it guards the array's bounds. */
#define RG_NOALLOC_PARTIAL_BYTES ((int64_t)16 << 20)
#define RG_NOALLOC_MAX_TILES 4096
int rg_gemm_noalloc(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B, int64_t ldb,
                    float* C, int64_t ldc, int32_t variant, int32_t beta, void* stream);
/* The status of the rg_gemm_noalloc work enqueued so far on the calling thread's
 * current device: synchronises `stream`, then reads the scratch array's error
 * word (a device-to-host copy; nothing is allocated).  RG_OK if no bounded wait
 * expired (also when no rg_gemm_noalloc call has run on this device yet);
 * RG_ERR_TIMEOUT if one did, in which case the error word and every ticket are
 * cleared (synchronously) so the next call starts clean; RG_ERR_CUDA if a CUDA
 * call fails.  Like rg_gemm_noalloc, it races with calls still running on other
 * streams.  The paper has no counterpart to it. */
int rg_noalloc_check(void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RG_H */
