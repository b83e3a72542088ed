// BF16 NN GEMM for sm_103a (C = A * B, A M x K row-major, B K x N row-major,
// C M x N FP32; Sec. 2.2 of "From Roofline to Ruggedness") in the paper's six
// tiles (Sec. 6.1) and a 128 x 192 one, with the padding and split-K of Sec. 7.1 fused in, plus
// the sweep (Sec. 3, Sec. 5.4) and plan execution (Sec. 7.1) that drive it.
//
// Kernel structure (one CTA per SM, persistent over output tiles x K splits):
//   warp 0     TMA producer: A tile (BM x 64, K-major, 128B swizzle) and B tile
//              (64 x BN, N-major, 128B swizzle, 64-column boxes) into an
//              mbarrier-guarded ring of STAGES shared-memory stages of one K
//              block, or two for 128x64, 128x128 and the 256x128 pair.
//   warp 1     allocates TMEM; one thread issues tcgen05.mma (M = 128, N = BN,
//              K = 16) into a TMEM accumulator, double-buffered when it fits,
//              and commits stage releases / accumulator-full to mbarriers.
//   warps 2-5  epilogue: tcgen05.ld of their 32 TMEM lanes, 128B-swizzled
//              staging, TMA store (beta = 0) or TMA reduce-add (beta = 1).
// Padding is never materialised: tensor maps carry the logical extents, so
// TMA zero-fills reads past them and clips writes; the launch itself uses the
// padded extents (tile counts and K blocks).
// Split-K (S > 1): split s runs K blocks [s*kb/S, (s+1)*kb/S); each epilogue
// warp writes its FP32 partial rows to the workspace, fences and takes a
// ticket; the last arriver of a (tile, warp) row block sums the S partials in
// the fixed order 0..S-1 (so results are deterministic), stores C and resets
// the ticket.  No CTA waits for another CTA outside its own cluster (a
// cta_group::2 pair, or the S CTAs of a cluster split-K tile, which the
// hardware schedules together).
// Every mbarrier wait is bounded; on expiry the kernel records an error code
// in a device word, releases its TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <type_traits>
#include <type_traits>
#include <vector>

#include "ptx.cuh"
#include "rg_internal.h"

namespace rg {

constexpr int kThreads = 192;
constexpr int kBK = 64;                       // K per block: one 128-byte swizzle row of BF16
constexpr int kStagingPerWarp = 2 * 32 * 32 * 4;  // two 32x32 FP32 staging tiles per epilogue warp
constexpr int kMaxTickets = 1 << 18;
constexpr uint32_t FULL = 0xffffffffu;
// Bound for the waits that let this CTA's own in-flight TMA copies and MMAs
// land before it exits (independent of the per-wait budget, which a caller
// may set tiny): about half a second.
constexpr long long kDrainCycles = 1LL << 30;

enum : int { kErrProducer = 1, kErrMma = 2, kErrEpilogue = 3 };

// Phase stamps, a compile-time option (RG_PHASE_TIMERS=1): per CTA, fields
//   0 globaltimer at entry (ns)     1 globaltimer at exit (ns)     2 clock64 at exit
//   3 dependency wait done          4 first operand stage landed   5 last MMA commit
//   6 first accumulator ready       7 epilogue done                8 first split-K fixup start
//   9 last split-K fixup end        10 work units of the CTA
// with every clock64 field counted from the CTA's entry.  Without the option the
// stamps compile to nothing.
constexpr int kTraceFields = 12;
#ifndef RG_PHASE_TIMERS
#define RG_PHASE_TIMERS 0
#endif
#if RG_PHASE_TIMERS
#define RG_STAMP(f)                                                                       \
  do {                                                                                    \
    if (trace_row) trace_row[f] = static_cast<unsigned long long>(clock64() - t_entry);   \
  } while (0)
#else
#define RG_STAMP(f) \
  do {              \
  } while (0)
#endif
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct GemmArgs {
  int32_t M, N;             // logical output extents
  int32_t tiles_m, tiles_n; // tiles of the (padded) launch
  int32_t splits;
  int32_t kblocks;          // ceil(padded K / 64)
  int32_t beta;
  int32_t stall;            // test hook: the MMA warp first waits on a barrier nothing arrives on
  int32_t dp_tiles;         // stream-K: tiles run whole before the shared tail
  int32_t panel;            // tile order: column panels of this many tiles (pairs: tile columns)
  int32_t early;            // 1: A and B are static, so loads may start before the preceding grid completes
  int32_t reserved_;
  float* ws;                // split-K partials [split][tile][BM][BN]
  int32_t* tickets;         // [tile][4], zero between launches
  int32_t* err;
  long long timeout;        // cycles per wait
  unsigned long long* trace;  // phase stamps [CTA][kTraceFields] (RG_PHASE_TIMERS builds), or null
};

// CTAS = 2: one CTA of a cta_group::2 pair (BM = 128 rows of its own, BN / 2
// columns of B in its shared memory, M = 256 per MMA instruction).
template <int BM, int BN, int STAGES, int CTAS = 1>
struct KCfg {
  // K blocks per ring stage.  Every stage costs one full/empty barrier round, and a stage
  // of one 64-deep K block of a 128-row tile with N <= 128 holds less MMA work than that
  // round takes; those tiles (128x64, 128x128 and the 256x128 pair's CTAs) put two K
  // blocks in a stage, with half as many stages in the same bytes.
  static constexpr int SUB = (BM == 128 && BN <= 128) ? 2 : 1;
  static constexpr int A_BYTES = BM * kBK * 2;
  // B columns a CTA loads: its BN / CTAS rounded up to whole 64-column (128-byte) boxes
  // (a 256x192 pair's CTA loads 128 columns, of which its MMAs read 96)
  static constexpr int BN_LOAD = (BN / CTAS + 63) / 64 * 64;
  static constexpr int B_BYTES = kBK * BN_LOAD * 2;
  static constexpr int SUB_BYTES = A_BYTES + B_BYTES;  // one K block: A, then B
  static constexpr int STAGE_BYTES = SUB * SUB_BYTES;
  static constexpr int HALVES = BM / 128;
  static constexpr int ACC_COLS = HALVES * BN;
  static constexpr int NBUF = (2 * ACC_COLS <= 512) ? 2 : 1;
  static constexpr int USED_COLS = NBUF * ACC_COLS;
  static constexpr int TMEM_COLS = USED_COLS <= 32 ? 32 : USED_COLS <= 64 ? 64 : USED_COLS <= 128 ? 128
                                   : USED_COLS <= 256 ? 256 : 512;
  static constexpr int STAGING_OFF = STAGES * STAGE_BYTES;
  static constexpr int BAR_OFF = STAGING_OFF + 4 * kStagingPerWarp;
  static constexpr int SMEM_BYTES = 1024 + BAR_OFF + 256;
  static_assert((2 * STAGES + 9) * 8 <= 256, "barrier block");
  static constexpr uint32_t IDESC = instr_desc(1, 1, 0, 1, 128 * CTAS, BN);
  static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "stages must keep 1024-byte alignment");
  static_assert(SMEM_BYTES <= 232448, "shared memory budget");
  static_assert(BN % 64 == 0 && BN <= 256 && (BM == 128 || BM == 256), "tile shape");
  static_assert(CTAS == 1 || (CTAS == 2 && BM == 128 && BN % 64 == 0), "pair tile shape");
};

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Distributed shared memory (split-K clusters): a 16-byte store into another CTA's
// shared memory (shared::cluster address), a fence ordering this thread's earlier
// accesses at cluster scope, and a bounded wait that acquires at cluster scope what
// other CTAs released by arriving on a barrier of this CTA.
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}
__device__ __forceinline__ void fence_acq_rel_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, long long budget,
                                                  volatile int* abort) {
  const long long t0 = clock64();
  while (!mbar_try_wait_cluster(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

__device__ __forceinline__ void load_acc(uint32_t taddr, bool have, float (&v)[32]) {
  if (have) {
    uint32_t r[32];
    tmem_ld_32x32b_x32(taddr, r);
    tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = 0.f;
  }
}

// One warp stores a 32 x 32 FP32 block (lane = row) through a swizzled staging
// buffer with a TMA store, or a TMA reduce-add when beta = 1.
__device__ __forceinline__ void store_block(const CUtensorMap* tmC, const float (&v)[32], int row0, int col0,
                                            int M, int N, int beta, uint32_t stg0, int& sbuf, int lane) {
  if (row0 >= M || col0 >= N) return;  // wholly outside the logical C (padding)
  if (lane == 0) bulk_wait_read<1>();  // the buffer about to be reused has been read
  __syncwarp();
  const uint32_t buf = stg0 + sbuf * 4096;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    st_shared_v4(buf + lane * 128 + ((j ^ (lane & 7)) << 4), v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
  fence_proxy_async_smem();
  __syncwarp();
  if (lane == 0) {
    if (beta)
      tma_reduce_add_2d(tmC, buf, col0, row0);
    else
      tma_store_2d(tmC, buf, col0, row0);
    bulk_commit();
  }
  sbuf ^= 1;
}

// One work unit: which output tile of which problem, which K blocks, and where
// its operands and output live.
struct Unit {
  const CUtensorMap* a;
  const CUtensorMap* b;
  const CUtensorMap* c;
  const CUtensorMap* w;  // split-K workspace [split][tile][BM rows] x BN, FP32 (split-K only)
  int tm, tn;     // tile coordinates in the problem
  int s, splits;  // K split index and count
  int kb0, kb1;   // K blocks [kb0, kb1) of this unit
  int M, N;       // logical output extents of the problem
  int beta;
  int tile, ntiles;  // tile id / tile count of the problem (split-K workspace and tickets)
  int ws_row0 = 0;   // first workspace row of the problem's partials (grouped launches)
  int tk0 = 0;       // first ticket of the problem (grouped launches)
};

// Tile order: the tile grid is cut into column panels `panel` tiles wide and
// walked row by row inside each panel, so the tiles resident at one time share a
// panel of B that stays in L2 while A streams past.  panel >= tiles_n is plain
// row-major order.
__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int panel, int& tm, int& tn) {
  if (panel >= tiles_n) {
    tm = tile / tiles_n;
    tn = tile % tiles_n;
    return;
  }
  const int per = panel * tiles_m;
  const int p = tile / per;
  const int w = min(panel, tiles_n - p * panel);
  const int r = tile - p * per;
  tm = r / w;
  tn = p * panel + r % w;
}

__device__ __forceinline__ Unit split_unit(const CUtensorMap* a, const CUtensorMap* b, const CUtensorMap* c,
                                           const CUtensorMap* w, int u, int tiles_m, int tiles_n, int splits,
                                           int kblocks, int M, int N, int beta, int panel) {
  Unit x;
  x.a = a;
  x.b = b;
  x.c = c;
  x.w = w;
  x.tile = u / splits;
  x.s = u % splits;
  x.splits = splits;
  tile_coords(x.tile, tiles_m, tiles_n, panel, x.tm, x.tn);
  // 32-bit: splits <= 8 and kblocks <= 2^24, so (s + 1) * kblocks < 2^27
  x.kb0 = splits == 1 ? 0 : x.s * kblocks / splits;
  x.kb1 = splits == 1 ? kblocks : (x.s + 1) * kblocks / splits;
  x.M = M;
  x.N = N;
  x.beta = beta;
  x.ntiles = tiles_m * tiles_n;
  return x;
}

// One problem whose tensor maps are kernel parameters (rg_gemm).  SPLIT: the
// instance for split-K launches (S > 1); without it the kernel carries no
// reduction path (and none of its register pressure).
template <bool SPLIT>
struct SingleSched {
  static constexpr bool kMapsInGlobal = false;
  static constexpr bool kMemOnly = false;
  static constexpr bool k2Sm = false;
  static constexpr bool kSplit = SPLIT;
  static constexpr int rank = 0;
  const CUtensorMap* a;
  const CUtensorMap* b;
  const CUtensorMap* c;
  const CUtensorMap* w;
  int tiles_m, tiles_n, splits, kblocks, M, N, beta;
  int panel = 1 << 30;
  __device__ __forceinline__ void prefetch() const {
    prefetch_tmap(a);
    prefetch_tmap(b);
    prefetch_tmap(c);
  }
  __device__ __forceinline__ void init() {}
  // units u = blockIdx.x + i * gridDim.x of the (tile, split) space
  __device__ __forceinline__ int count() const {
    const int t = tiles_m * tiles_n * splits;
    return static_cast<int>(blockIdx.x) < t ? (t - 1 - static_cast<int>(blockIdx.x)) / static_cast<int>(gridDim.x) + 1
                                            : 0;
  }
  __device__ __forceinline__ Unit unit(int i) const {
    return split_unit(a, b, c, w, static_cast<int>(blockIdx.x) + i * static_cast<int>(gridDim.x), tiles_m, tiles_n,
                      splits, kblocks, M, N, beta, panel);
  }
};

// The memory twin of SingleSched: the same units, loads and stores, with the
// MMAs replaced by no-ops (the memory surface of the four-surface decomposition,
// Sec. 4).  Its output is whatever the accumulators held: timing only.
struct MemTwinSched : SingleSched<false> {
  static constexpr bool kMemOnly = true;
};

// Split-K inside a cluster: a cluster of S CTAs (S = splits, consecutive blockIdx.x)
// computes one output tile, CTA rank s the K blocks [s kblocks / S, (s+1) kblocks / S),
// one unit per CTA (no persistence).  The S partials never leave the chip: the
// epilogue's cluster branch sums them through distributed shared memory in the
// fixed order 0..S-1, the same sums as the workspace path's last arriver.
struct ClusterSplitSched : SingleSched<false> {
  static constexpr bool kClusterSplit = true;
  __device__ __forceinline__ int count() const {
    return static_cast<int>(blockIdx.x) < tiles_m * tiles_n * splits ? 1 : 0;
  }
  __device__ __forceinline__ Unit unit(int) const {
    return split_unit(a, b, c, w, static_cast<int>(blockIdx.x), tiles_m, tiles_n, splits, kblocks, M, N, beta, panel);
  }
};
template <class S, class = void>
struct IsClusterSplit : std::false_type {};
template <class S>
struct IsClusterSplit<S, std::void_t<decltype(S::kClusterSplit)>> : std::bool_constant<S::kClusterSplit> {};

// Stream-K (hybrid): whole waves of tiles run data-parallel, one tile per CTA
// per wave (tile g + i * G on CTA g, for tiles below dp_tiles: all whole waves,
// or all but the last in sk_geometry's balanced form); the remaining tiles' K
// iterations are divided evenly among the first tail CTAs:
// CTA h owns tail iterations [h I / tail, (h+1) I / tail), processed as one
// segment per tile it touches.  A tail tile covered by one segment is stored
// directly; one split over several CTAs is summed by its last arriving segment
// in the fixed order of the segments' K ranges (through the split-K workspace,
// slot = segment * ntiles + tile).  So no wave is left partly idle.
// TWO_SM: the same schedule over 2-CTA clusters and 256-row pair tiles (G =
// clusters, tile = pair tile); each CTA of a cluster computes, publishes and
// reduces its own 128 rows, as in the cta_group::2 split-K form (tiles_m counts
// 128-row tiles and is even).
template <bool TWO_SM>
struct StreamKSched {
  static constexpr bool kMapsInGlobal = false;
  static constexpr bool kMemOnly = false;
  static constexpr bool k2Sm = TWO_SM;
  static constexpr bool kSplit = true;
  const CUtensorMap* a;
  const CUtensorMap* b;
  const CUtensorMap* c;
  const CUtensorMap* w;
  int tiles_m, tiles_n, kblocks, M, N, beta;
  int tail = 0;      // CTAs (clusters) sharing the tail tiles (from the launcher)
  int dp_tiles = 0;  // tiles run whole (from the launcher)
  int panel = 1 << 30;
  int rank = 0;
  long long iters = 0, begin = 0, end = 0;
  int G = 1, g = 0, T = 0, n_dp = 0, t0 = 0, n_sk = 0;
  __device__ __forceinline__ void prefetch() const {
    prefetch_tmap(a);
    prefetch_tmap(b);
    prefetch_tmap(c);
  }
  __device__ __forceinline__ long long cta_begin(int h) const { return static_cast<long long>(h) * iters / tail; }
  // the tail CTA whose range holds tail iteration x
  __device__ __forceinline__ int cta_of(long long x) const {
    int h = static_cast<int>((x * tail) / iters);
    while (h + 1 < tail && cta_begin(h + 1) <= x) ++h;
    while (h > 0 && cta_begin(h) > x) --h;
    return h;
  }
  __device__ __forceinline__ void init() {
    if constexpr (TWO_SM) {
      rank = static_cast<int>(cluster_ctarank());
      G = static_cast<int>(gridDim.x) / 2;
      g = static_cast<int>(blockIdx.x) / 2;
      T = (tiles_m / 2) * tiles_n;
    } else {
      G = static_cast<int>(gridDim.x);
      g = static_cast<int>(blockIdx.x);
      T = tiles_m * tiles_n;
    }
    n_dp = g < dp_tiles ? (dp_tiles - 1 - g) / G + 1 : 0;
    iters = static_cast<long long>(T - dp_tiles) * kblocks;
    if (tail > 0 && g < tail && iters > 0) {
      begin = cta_begin(g);
      end = cta_begin(g + 1);
      if (end > begin) {
        t0 = static_cast<int>(begin / kblocks);
        n_sk = static_cast<int>((end - 1) / kblocks) - t0 + 1;
      }
    }
  }
  __device__ __forceinline__ int count() const { return n_dp + n_sk; }
  __device__ __forceinline__ Unit unit(int i) const {
    Unit x;
    x.a = a;
    x.b = b;
    x.c = c;
    x.w = w;
    x.M = M;
    x.N = N;
    x.beta = beta;
    if (i < n_dp) {  // a whole tile of the data-parallel waves
      x.tile = g + i * G;
      x.kb0 = 0;
      x.kb1 = kblocks;
      x.splits = 1;
      x.s = 0;
    } else {  // a segment of a tail tile
      const int j = i - n_dp;
      const int lt = t0 + j;  // index among the tail tiles
      x.tile = dp_tiles + lt;
      const long long tb = static_cast<long long>(lt) * kblocks;
      const long long lo = begin > tb ? begin : tb;
      const long long hi = end < tb + kblocks ? end : tb + kblocks;
      x.kb0 = static_cast<int>(lo - tb);
      x.kb1 = static_cast<int>(hi - tb);
      const int first = cta_of(tb), last = cta_of(tb + kblocks - 1);
      x.splits = last - first + 1;
      x.s = g - first;
    }
    if constexpr (TWO_SM) {
      int pr, pc;
      tile_coords(x.tile, tiles_m / 2, tiles_n, panel, pr, pc);
      x.tm = 2 * pr + rank;
      x.tn = pc;
      x.tile = x.tm * tiles_n + x.tn;
      x.ntiles = tiles_m * tiles_n;
    } else {
      tile_coords(x.tile, tiles_m, tiles_n, panel, x.tm, x.tn);
      x.ntiles = T;
    }
    return x;
  }
};

// cta_group::2: 2-CTA clusters, each cluster one 256-row output tile run as a
// single tcgen05 MMA unit.  Tile (m, n) of 128-row tiles pairs (2p, n) with
// (2p+1, n): CTA rank r of cluster p computes 128-row tile 2p + r, loads its own
// 128 rows of A and its half (BN / 2 columns) of the B tile into its own shared
// memory, and the even CTA issues the MMAs for both.  A CTA whose rows fall
// outside the problem still loads (zero-filled reads) so that the pair's MMAs
// are fed; its stores are dropped.  Units are (pair tile, K split).
template <bool SPLIT>
struct TwoSmSched {
  static constexpr bool kMapsInGlobal = false;
  static constexpr bool kMemOnly = false;
  static constexpr bool k2Sm = true;
  static constexpr bool kSplit = SPLIT;
  const CUtensorMap* a;
  const CUtensorMap* b;
  const CUtensorMap* c;
  const CUtensorMap* w;
  int tiles_m, tiles_n, kblocks, M, N, beta;  // tiles_m counts 128-row tiles
  int rank = 0, cid = 0, ncl = 1, pairs = 0;
  int splits = 1;
  int panel = 1 << 30;
  __device__ __forceinline__ void prefetch() const {
    prefetch_tmap(a);
    prefetch_tmap(b);
    prefetch_tmap(c);
  }
  __device__ __forceinline__ void init() {
    rank = static_cast<int>(cluster_ctarank());
    cid = static_cast<int>(blockIdx.x) / 2;
    ncl = static_cast<int>(gridDim.x) / 2;
    pairs = ((tiles_m + 1) / 2) * tiles_n;
  }
  __device__ __forceinline__ int count() const {
    const int units = pairs * splits;
    return cid < units ? (units - 1 - cid) / ncl + 1 : 0;
  }
  __device__ __forceinline__ Unit unit(int i) const {
    const int u = cid + i * ncl;
    const int p = u / splits;
    Unit x;
    x.a = a;
    x.b = b;
    x.c = c;
    x.w = w;
    int pr, pc;
    tile_coords(p, (tiles_m + 1) / 2, tiles_n, panel, pr, pc);
    x.tm = 2 * pr + rank;
    x.tn = pc;
    x.s = u % splits;
    x.splits = splits;
    x.kb0 = splits == 1 ? 0 : x.s * kblocks / splits;
    x.kb1 = splits == 1 ? kblocks : (x.s + 1) * kblocks / splits;
    x.M = M;
    x.N = N;
    x.beta = beta;
    x.ntiles = tiles_m * tiles_n;
    x.tile = x.tm * tiles_n + x.tn;
    return x;
  }
};

// Many problems in one launch (rg_gemm_grouped): a device-resident work list
// whose header gives the item count and the total unit count; the units are the
// concatenation of every item's (tile, K split) units (item i owns units
// [unit_start, unit_start + tiles * splits)).  Each item carries its own tensor
// maps (in global memory), launch extents, beta, split factor and the offsets of
// its split-K partials and tickets in the launch's workspace.  TWO_SM: units are
// (256-row pair tile, split) and every 2-CTA cluster runs one at a time as a
// tcgen05 cta_group::2 unit (tiles_m counts 128-row tiles).
// Work-list records keep CUtensorMap's 128-byte alignment: a 128-byte header,
// then 512-byte items (three maps and the sizes).
struct alignas(128) GroupItem {
  CUtensorMap a, b, c;
  int32_t M, N, beta, tiles_m;
  int32_t tiles_n, kblocks, unit_start, splits;
  int32_t ws_row0, tk0, reserved[2];
};
struct alignas(128) GroupHeader {
  int32_t n_items;
  int32_t total_units;
  int32_t reserved[30];
};

template <bool TWO_SM>
struct GroupSched {
  static constexpr bool kMapsInGlobal = true;
  static constexpr bool kMemOnly = false;
  static constexpr bool k2Sm = TWO_SM;
  static constexpr bool kSplit = true;
  const GroupHeader* h;
  const GroupItem* items;
  const CUtensorMap* w;      // the launch's split-K workspace
  int n_items = 0, total_units = 0;  // read after the grid dependency wait
  int rank = 0, cid = 0, ncl = 1;
  __device__ __forceinline__ void prefetch() const {}
  __device__ __forceinline__ void init() {
    n_items = h->n_items;
    total_units = h->total_units;
    if constexpr (TWO_SM) {
      rank = static_cast<int>(cluster_ctarank());
      cid = static_cast<int>(blockIdx.x) / 2;
      ncl = static_cast<int>(gridDim.x) / 2;
    } else {
      cid = static_cast<int>(blockIdx.x);
      ncl = static_cast<int>(gridDim.x);
    }
  }
  __device__ __forceinline__ int count() const {
    return cid < total_units ? (total_units - 1 - cid) / ncl + 1 : 0;
  }
  __device__ __forceinline__ Unit unit(int i) const {
    const int u = cid + i * ncl;
    int lo = 0, hi = n_items - 1;  // last item whose unit_start <= u
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].unit_start <= u) lo = mid; else hi = mid - 1;
    }
    const GroupItem& it = items[lo];
    Unit x;
    if constexpr (TWO_SM) {
      const int v = u - it.unit_start;
      const int p = v / it.splits;
      x.a = &it.a;
      x.b = &it.b;
      x.c = &it.c;
      x.w = w;
      x.tm = 2 * (p / it.tiles_n) + rank;  // tiles_m (128-row tiles) is even: pairs never overhang
      x.tn = p % it.tiles_n;
      x.s = v % it.splits;
      x.splits = it.splits;
      x.kb0 = it.splits == 1 ? 0 : x.s * it.kblocks / it.splits;
      x.kb1 = it.splits == 1 ? it.kblocks : (x.s + 1) * it.kblocks / it.splits;
      x.M = it.M;
      x.N = it.N;
      x.beta = it.beta;
      x.ntiles = it.tiles_m * it.tiles_n;
      x.tile = x.tm * it.tiles_n + x.tn;
    } else {
      x = split_unit(&it.a, &it.b, &it.c, w, u - it.unit_start, it.tiles_m, it.tiles_n, it.splits, it.kblocks, it.M,
                     it.N, it.beta, it.tiles_n);
    }
    x.ws_row0 = it.ws_row0;
    x.tk0 = it.tk0;
    return x;
  }
};

template <int BM, int BN, int STAGES, class Sched>
__device__ __forceinline__ void gemm_body(Sched& sched, float* ws, int32_t* tickets, int32_t* err, long long timeout,
                                          int stall, int early, unsigned long long* trace = nullptr) {
#if RG_PHASE_TIMERS
  const long long t_entry = clock64();
  unsigned long long* trace_row = trace ? trace + static_cast<size_t>(blockIdx.x) * kTraceFields : nullptr;
  if (trace_row && threadIdx.x == 0) {
    trace_row[0] = global_ns();
    for (int f = 3; f < kTraceFields; ++f) trace_row[f] = 0;  // stamps this launch may not reach
  }
  __syncthreads();
#else
  (void)trace;
#endif
  constexpr bool P2 = Sched::k2Sm;  // one CTA of a cta_group::2 pair
  constexpr bool CS = IsClusterSplit<Sched>::value;  // one K slice of a cluster split-K tile
  using C = KCfg<BM, BN, STAGES, P2 ? 2 : 1>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_s = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (raw_s & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int i) { return bar0 + 8u * i; };
  auto empty_bar = [&](int i) { return bar0 + 8u * (STAGES + i); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // cluster split-K: the other CTAs' operand rings are free / their blocks for this CTA have landed
  const uint32_t go_bar = bar0 + 8u * (2 * STAGES + 6);
  const uint32_t recv_bar = bar0 + 8u * (2 * STAGES + 7);
  const uint32_t ready_bar = bar0 + 8u * (2 * STAGES + 8);  // this CTA's four epilogue warps saw the sum final
  int never = 0;
  volatile int* no_abort = &never;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    sched.prefetch();
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(full_bar(i), 1);
      mbar_init(empty_bar(i), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      // pair: the even CTA's accumulator is free once both CTAs' epilogue warps drained it
      mbar_init(tempty_bar(b), P2 ? 8 : 4);
    }
    mbar_init(drain_bar, 1);
    if constexpr (CS) {
      mbar_init(go_bar, sched.splits - 1);             // one arrival per other CTA
      mbar_init(recv_bar, 4 * (sched.splits - 1));     // one per epilogue warp of every other CTA
      mbar_init(ready_bar, 4);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    if constexpr (P2) {  // collective with the partner's warp 1: the same columns in both CTAs
      tmem_alloc_pair(smem_u32(tmem_slot), C::TMEM_COLS);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (P2 || CS) cluster_sync();  // the other CTAs' barriers are initialised
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // Everything above overlaps the previous grid in the stream; nothing below
  // touches global memory before that grid has completed -- except, when A and
  // B are declared static (early), the operand loads and the MMAs, which touch
  // only A, B, shared memory and TMEM: then only the epilogue, which writes C
  // and the split-K workspace, waits for the previous grid.
  // The schedule of a single problem depends only on kernel parameters, so it,
  // and the producer's first unit, are worked out while the previous grid may
  // still be running (a grouped work list is read after the wait).
  Unit first{};
  if constexpr (!Sched::kMapsInGlobal) {
    sched.init();
    if (warp == 0 && lane == 0 && sched.count() > 0) first = sched.unit(0);
  }
  if (!early) grid_dependency_wait();
  grid_launch_dependents();
  if constexpr (Sched::kMapsInGlobal) sched.init();
  const int nunits = sched.count();
  if (threadIdx.x == 0) {
    RG_STAMP(3);
#if RG_PHASE_TIMERS
    if (trace_row) trace_row[10] = static_cast<unsigned long long>(nunits);
#endif
  }

  if (warp == 0) {
    // ------------------------------------------------ TMA producer (one thread)
    if (lane == 0) {
      int stage = 0, fills = 0;
      uint32_t ph = 0;
      uint32_t issued_mask = 0, issued_ph = 0;
      bool ok = true;
      for (int i = 0; ok && i < nunits; ++i) {
        const Unit w = (!Sched::kMapsInGlobal && i == 0) ? first : sched.unit(i);
        if constexpr (Sched::kMapsInGlobal) {
          tensormap_fence_acquire(w.a);
          tensormap_fence_acquire(w.b);
        }
        for (int kbs = w.kb0; kbs < w.kb1; kbs += C::SUB) {
          const int nsub = w.kb1 - kbs < C::SUB ? w.kb1 - kbs : C::SUB;  // K blocks in this stage
          // a stage's first fill needs no wait: nothing has used it yet
          if (fills >= STAGES && !mbar_wait(empty_bar(stage), ph ^ 1u, timeout, abort_flag)) {
            ok = false;
            break;
          }
          ++fills;
          if constexpr (P2) {
            // Both CTAs' loads complete on the even CTA's full barrier, which expects both halves.
            if (sched.rank == 0) mbar_arrive_expect_tx(full_bar(stage), 2 * nsub * C::SUB_BYTES);
            const uint32_t fb = mapa_shared(full_bar(stage), 0);
            for (int u = 0; u < nsub; ++u) {
              const int kb = kbs + u;
              const uint32_t sa = sbase + stage * C::STAGE_BYTES + u * C::SUB_BYTES;
              const uint32_t sb = sa + C::A_BYTES;
              tma_load_2d_pair(sa, w.a, fb, kb * kBK, w.tm * BM);
#pragma unroll
              for (int j = 0; j < C::BN_LOAD / 64; ++j)
                tma_load_2d_pair(sb + j * (kBK * 128), w.b, fb, w.tn * BN + sched.rank * (BN / 2) + j * 64, kb * kBK);
            }
          } else {
            mbar_arrive_expect_tx(full_bar(stage), nsub * C::SUB_BYTES);
            for (int u = 0; u < nsub; ++u) {
              const int kb = kbs + u;
              const uint32_t sa = sbase + stage * C::STAGE_BYTES + u * C::SUB_BYTES;
              const uint32_t sb = sa + C::A_BYTES;
              tma_load_2d(sa, w.a, full_bar(stage), kb * kBK, w.tm * BM);
#pragma unroll
              for (int j = 0; j < BN / 64; ++j)
                tma_load_2d(sb + j * (kBK * 128), w.b, full_bar(stage), w.tn * BN + j * 64, kb * kBK);
            }
          }
          issued_mask |= 1u << stage;
          issued_ph = (issued_ph & ~(1u << stage)) | (ph << stage);
          if (++stage == STAGES) {
            stage = 0;
            ph ^= 1u;
          }
        }
      }
      if (!ok) {
        atomicExch(err, kErrProducer);
        *abort_flag = 1;
      }
      // no TMA write may still be landing when the CTA exits
      if (!P2 || sched.rank == 0) {
        for (int i = 0; i < STAGES; ++i)
          if (issued_mask & (1u << i)) mbar_wait(full_bar(i), (issued_ph >> i) & 1u, kDrainCycles, no_abort);
      } else if (!ok) {
        // The odd CTA's loads complete on its partner's barriers; after an abort it
        // gives them a bounded time to land (normally every one of them was consumed).
        const long long t0 = clock64();
        while (clock64() - t0 < (kDrainCycles >> 6)) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer (one thread)
    // Lane 0 alone runs the loop: tcgen05.mma and tcgen05.commit are issued by a
    // single thread, and keeping the other 31 lanes out of the loop saves a warp
    // vote and a warp reconvergence per stage (about 200 of the 550 cycles a stage
    // cost when the whole warp stepped through it).
    if (lane == 0) {
      int stage = 0, acc = 0;
      uint32_t ph = 0, aph = 0;
      bool ok = true;
      if (stall) ok = mbar_wait(drain_bar, 0, timeout, abort_flag);
      // a pair's odd CTA issues nothing: the even CTA's MMAs read and write both
      const int issue_units = (!P2 || sched.rank == 0) ? nunits : 0;
      for (int i = 0; ok && i < issue_units; ++i) {
        const Unit w = sched.unit(i);
        const int kb0 = w.kb0, kb1 = w.kb1;
        ok = mbar_wait(tempty_bar(acc), aph ^ 1u, timeout, abort_flag);
        if (!ok) break;
        tc_fence_after();
        const uint32_t d0 = tmem_base + static_cast<uint32_t>(acc * C::ACC_COLS);
        for (int kbs = kb0; kbs < kb1; kbs += C::SUB) {
          const int nsub = kb1 - kbs < C::SUB ? kb1 - kbs : C::SUB;  // K blocks in this stage
          ok = mbar_wait(full_bar(stage), ph, timeout, abort_flag);
          if (!ok) break;
          if (i == 0 && kbs == kb0) RG_STAMP(4);
          tc_fence_after();
          if constexpr (Sched::kMemOnly) {
            mbar_arrive(empty_bar(stage));  // no MMA reads the stage: it is free once its bytes have landed
          } else {
            for (int u = 0; u < nsub; ++u) {
              const uint32_t sa = sbase + stage * C::STAGE_BYTES + u * C::SUB_BYTES;
              const uint32_t sb = sa + C::A_BYTES;
              // The descriptors of the block's K steps differ only in their start
              // address field (bits 0-13, address >> 4; no carry: shared addresses
              // stay below 2^18), so they are the block's base descriptors plus constants.
              const uint64_t adesc0 = smem_desc_sw128(sa, 16, 1024);
              const uint64_t bdesc0 = smem_desc_sw128(sb, kBK * 128, 1024);
              const uint32_t first = kbs + u > kb0 ? 1u : 0u;
#pragma unroll
              for (int k = 0; k < kBK / 16; ++k) {
                const uint64_t bdesc = bdesc0 + static_cast<uint64_t>((k * 2048) >> 4);
#pragma unroll
                for (int h = 0; h < C::HALVES; ++h) {
                  const uint64_t adesc = adesc0 + static_cast<uint64_t>((h * (128 * 128) + k * 32) >> 4);
                  if constexpr (P2)
                    mma_f16_pair(d0, adesc, bdesc, C::IDESC, k > 0 ? 1u : first);
                  else
                    mma_f16(d0 + h * BN, adesc, bdesc, C::IDESC, k > 0 ? 1u : first);
                }
              }
            }
            if constexpr (P2)
              mma_commit_pair_multicast(empty_bar(stage), 3);  // the stage is free in both CTAs
            else
              mma_commit(empty_bar(stage));
          }
          if (++stage == STAGES) {
            stage = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        if constexpr (Sched::kMemOnly)
          mbar_arrive(tfull_bar(acc));
        else if constexpr (P2)
          mma_commit_pair_multicast(tfull_bar(acc), 3);  // both CTAs' halves of the accumulator are final
        else
          mma_commit(tfull_bar(acc));
        if (++acc == C::NBUF) {
          acc = 0;
          aph ^= 1u;
        }
        if (i + 1 == issue_units) RG_STAMP(5);
      }
      if (!ok) {
        atomicExch(err, kErrMma);
        *abort_flag = 1;
        if constexpr (P2)
          mma_commit_pair(drain_bar);
        else
          mma_commit(drain_bar);  // completes once every issued MMA has finished
        mbar_wait(drain_bar, 0, kDrainCycles, no_abort);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ epilogue (warps 2-5)
    if (early) grid_dependency_wait();
    const int q = warp & 3;  // TMEM lanes 32q..32q+31 are the ones this warp may read
    const uint32_t stg0 = sbase + C::STAGING_OFF + (warp - 2) * kStagingPerWarp;
#if RG_PHASE_TIMERS
    bool fixup_seen = false;  // this launch has stamped its first split-K fixup
#endif
    int acc = 0, sbuf = 0;
    uint32_t aph = 0;
    bool ok = true;
    for (int i = 0; i < nunits; ++i) {
      const Unit w = sched.unit(i);
      const int tile = w.tile, s = w.s, tm = w.tm, tn = w.tn, kb0 = w.kb0, kb1 = w.kb1, ntiles = w.ntiles;
      if constexpr (Sched::kMapsInGlobal) {
        if (lane == 0) tensormap_fence_acquire(w.c);
      }
      ok = __all_sync(FULL, mbar_wait(tfull_bar(acc), aph, timeout, abort_flag));
      if (!ok) break;
      if (i == 0 && warp == 2 && lane == 0) RG_STAMP(6);
      tc_fence_after();
      const bool have = kb1 > kb0;
      const uint32_t tacc = tmem_base + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(acc * C::ACC_COLS);
      if constexpr (CS) {
        // Split-K inside the cluster, through distributed shared memory.  Block b = q kPerWarp + j
        // (32 x 32, j = h kCols + c) of the tile is reduced by CTA b % S; the other CTAs write their
        // partial of it into that CTA's operand ring, free once its MMAs have all completed.
        const int S = w.splits, r = w.s;
        constexpr int kCols = BN / 32, kPerWarp = C::HALVES * kCols;
        const int nown = 4 * kPerWarp / S;  // blocks each CTA reduces (S divides 4 kPerWarp)
        // 1. this CTA's ring is free once all four epilogue warps have seen the sum final
        if (lane == 0) mbar_arrive(ready_bar);
        if (warp == 2 && lane == 0 && mbar_wait(ready_bar, 0, timeout, abort_flag))
          for (int o = 0; o < S; ++o)
            if (o != r) mbar_arrive_cluster(mapa_shared(go_bar, static_cast<uint32_t>(o)));
        // 2. every CTA's ring is free: send the blocks other CTAs reduce (slot = the source's rank
        //    among that CTA's sources), then release them with one arrival per warp and CTA
        ok = __all_sync(FULL, mbar_wait_cluster(go_bar, 0, timeout, abort_flag));
        if (!ok) break;
#pragma unroll 1
        for (int j = 0; j < kPerWarp; ++j) {
          const int b = q * kPerWarp + j, o = b % S;
          if (o == r) continue;
          float v[32];
          load_acc(tacc + (j / kCols) * BN + (j % kCols) * 32, have, v);
          const int slot = r < o ? r : r - 1;
          const uint32_t dst =
              mapa_shared(sbase + static_cast<uint32_t>(slot * nown + b / S) * 4096u, static_cast<uint32_t>(o));
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
            st_cluster_v4(dst + lane * 128 + ((jj ^ (lane & 7)) << 4), v[4 * jj], v[4 * jj + 1], v[4 * jj + 2],
                          v[4 * jj + 3]);
        }
        fence_acq_rel_cluster();
        __syncwarp();
        if (lane == 0)
          for (int o = 0; o < S; ++o)
            if (o != r) mbar_arrive_cluster(mapa_shared(recv_bar, static_cast<uint32_t>(o)));
        // 3. every other CTA's partials of this CTA's blocks have landed: sum each in the fixed
        //    order 0..S-1 (this CTA's own partial, from TMEM, at position r) and store it
        ok = __all_sync(FULL, mbar_wait_cluster(recv_bar, 0, timeout, abort_flag));
        if (!ok) break;
#pragma unroll 1
        for (int j = 0; j < kPerWarp; ++j) {
          const int b = q * kPerWarp + j;
          if (b % S != r) continue;
          float own[32], sum[32];
          load_acc(tacc + (j / kCols) * BN + (j % kCols) * 32, have, own);
#pragma unroll 1
          for (int src = 0; src < S; ++src) {
            float p[32];
            if (src == r) {
#pragma unroll
              for (int e = 0; e < 32; ++e) p[e] = own[e];
            } else {
              const uint32_t from =
                  sbase + static_cast<uint32_t>((src < r ? src : src - 1) * nown + b / S) * 4096u + lane * 128;
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                const float4 x = ld_shared_v4(from + ((jj ^ (lane & 7)) << 4));
                p[4 * jj] = x.x;
                p[4 * jj + 1] = x.y;
                p[4 * jj + 2] = x.z;
                p[4 * jj + 3] = x.w;
              }
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) sum[e] = src == 0 ? p[e] : sum[e] + p[e];
          }
          store_block(w.c, sum, tm * BM + (j / kCols) * 128 + q * 32, tn * BN + (j % kCols) * 32, w.M, w.N, w.beta,
                      stg0, sbuf, lane);
        }
      } else if (!Sched::kSplit || w.splits == 1) {
#pragma unroll 1
        for (int h = 0; h < C::HALVES; ++h)
#pragma unroll 1
          for (int c = 0; c < BN / 32; ++c) {
            float v[32];
            load_acc(tacc + h * BN + c * 32, have, v);
            store_block(w.c, v, tm * BM + h * 128 + q * 32, tn * BN + c * 32, w.M, w.N, w.beta, stg0, sbuf,
                        lane);
          }
      } else if constexpr (Sched::kSplit) {
        // Split-K.  Publish this split's FP32 partial tile: TMEM -> swizzled staging ->
        // TMA store into the workspace (rows (s * ntiles + tile) * BM ..), then wait
        // for the stores, fence them against the generic proxy and take the ticket
        // of this (tile, warp) row block with an acquire-release atomic.
        const int wrow = w.ws_row0 + (s * ntiles + tile) * BM;
#pragma unroll 1
        for (int h = 0; h < C::HALVES; ++h)
#pragma unroll 1
          for (int c = 0; c < BN / 32; ++c) {
            float v[32];
            load_acc(tacc + h * BN + c * 32, have, v);
            store_block(w.w, v, wrow + h * 128 + q * 32, c * 32, INT_MAX, INT_MAX, 0, stg0, sbuf, lane);
          }
        if (lane == 0) {
          bulk_wait<0>();
          fence_proxy_async_global();
        }
        __syncwarp();
        int last = 0;
        if (lane == 0) {
          int32_t* t = tickets + w.tk0 + static_cast<size_t>(tile) * 4 + q;
          const int old = atom_add_acq_rel_gpu(t, 1);
          last = (old == w.splits - 1);
          if (last) *t = 0;
        }
        last = __shfl_sync(FULL, last, 0);
#if RG_PHASE_TIMERS
        if (last && warp == 2 && lane == 0 && !fixup_seen) {
          RG_STAMP(8);
          fixup_seen = true;
        }
#endif
        if (last) {
          // The last arriver sums the S partials of each 32 x 32 block in the fixed
          // order 0..S-1.  Lane l holds block rows 4j + l/8 (j = 0..7), columns
          // 4(l%8)..4(l%8)+3, so each warp load reads four whole 128-byte rows;
          // partials are loaded kBatch at a time.  Its own partial (still in TMEM,
          // one row per lane) is brought into that layout through the staging buffer.
          constexpr int kBatch = 3;
          const int rsub = lane >> 3, g = lane & 7;
          if (w.splits == 2) {
            // Two pieces (split 2, every stream-K tail tile): the other piece's partial of the
            // next 32 x 32 block is loaded while this block is reduced, hiding the load latency;
            // own + other is the same sum in either order, so the result is that of the fixed order.
            const int other = 1 - s;
            constexpr int kChunks = C::HALVES * (BN / 32);
            auto src_of = [&](int ch) {
              return ws + static_cast<size_t>(w.ws_row0 + (other * ntiles + tile) * BM + (ch / (BN / 32)) * 128 +
                                              q * 32) * BN + (ch % (BN / 32)) * 32 + 4 * g;
            };
            float4 nxt[8];
            {
              const float* src = src_of(0);
#pragma unroll
              for (int j = 0; j < 8; ++j)
                nxt[j] = __ldcg(reinterpret_cast<const float4*>(src + static_cast<size_t>(4 * j + rsub) * BN));
            }
#pragma unroll 1
            for (int ch = 0; ch < kChunks; ++ch) {
              const int h = ch / (BN / 32), c = ch % (BN / 32);
              float4 cur[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) cur[j] = nxt[j];
              if (ch + 1 < kChunks) {
                const float* src = src_of(ch + 1);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                  nxt[j] = __ldcg(reinterpret_cast<const float4*>(src + static_cast<size_t>(4 * j + rsub) * BN));
              }
              float own[32];
              load_acc(tacc + h * BN + c * 32, have, own);
              if (lane == 0) bulk_wait_read<1>();
              __syncwarp();
              const uint32_t buf = stg0 + sbuf * 4096;
#pragma unroll
              for (int j = 0; j < 8; ++j)
                st_shared_v4(buf + lane * 128 + ((j ^ (lane & 7)) << 4), own[4 * j], own[4 * j + 1], own[4 * j + 2],
                             own[4 * j + 3]);
              __syncwarp();
              float4 sum[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int r = 4 * j + rsub;
                const float4 o = ld_shared_v4(buf + r * 128 + ((g ^ (r & 7)) << 4));
                sum[j] = make_float4(o.x + cur[j].x, o.y + cur[j].y, o.z + cur[j].z, o.w + cur[j].w);
              }
              __syncwarp();
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int r = 4 * j + rsub;
                st_shared_v4(buf + r * 128 + ((g ^ (r & 7)) << 4), sum[j].x, sum[j].y, sum[j].z, sum[j].w);
              }
              fence_proxy_async_smem();
              __syncwarp();
              const int row0 = tm * BM + h * 128 + q * 32, col0 = tn * BN + c * 32;
              if (row0 < w.M && col0 < w.N) {
                if (lane == 0) {
                  if (w.beta)
                    tma_reduce_add_2d(w.c, buf, col0, row0);
                  else
                    tma_store_2d(w.c, buf, col0, row0);
                  bulk_commit();
                }
                sbuf ^= 1;
              }
            }
          } else
#pragma unroll 1
          for (int h = 0; h < C::HALVES; ++h)
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
              float own[32];
              load_acc(tacc + h * BN + c * 32, have, own);
              if (lane == 0) bulk_wait_read<1>();
              __syncwarp();
              const uint32_t buf = stg0 + sbuf * 4096;
#pragma unroll
              for (int j = 0; j < 8; ++j)
                st_shared_v4(buf + lane * 128 + ((j ^ (lane & 7)) << 4), own[4 * j], own[4 * j + 1], own[4 * j + 2],
                             own[4 * j + 3]);
              __syncwarp();
              float4 o[8], sum[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int r = 4 * j + rsub;
                o[j] = ld_shared_v4(buf + r * 128 + ((g ^ (r & 7)) << 4));
              }
              int t = 0;
              for (int base = 0; base < w.splits; base += kBatch) {
                float4 x[kBatch][8];
#pragma unroll
                for (int b = 0; b < kBatch; ++b) {
                  const int tb = base + b;
                  if (tb < w.splits && tb != s) {
                    const float* src = ws + static_cast<size_t>(w.ws_row0 + (tb * ntiles + tile) * BM + h * 128 +
                                                                q * 32) * BN + c * 32 + 4 * g;
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                      x[b][j] = __ldcg(reinterpret_cast<const float4*>(src + static_cast<size_t>(4 * j + rsub) * BN));
                  }
                }
#pragma unroll
                for (int b = 0; b < kBatch; ++b) {
                  const int tb = base + b;
                  if (tb < w.splits) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                      const float4 p = (tb == s) ? o[j] : x[b][j];
                      if (t == 0) {
                        sum[j] = p;
                      } else {
                        sum[j].x += p.x; sum[j].y += p.y; sum[j].z += p.z; sum[j].w += p.w;
                      }
                    }
                    ++t;
                  }
                }
              }
              __syncwarp();
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int r = 4 * j + rsub;
                st_shared_v4(buf + r * 128 + ((g ^ (r & 7)) << 4), sum[j].x, sum[j].y, sum[j].z, sum[j].w);
              }
              fence_proxy_async_smem();
              __syncwarp();
              const int row0 = tm * BM + h * 128 + q * 32, col0 = tn * BN + c * 32;
              if (row0 < w.M && col0 < w.N) {
                if (lane == 0) {
                  if (w.beta)
                    tma_reduce_add_2d(w.c, buf, col0, row0);
                  else
                    tma_store_2d(w.c, buf, col0, row0);
                  bulk_commit();
                }
                sbuf ^= 1;
              }
            }
        }
      }
#if RG_PHASE_TIMERS
      if (w.splits > 1 && warp == 2 && lane == 0 && fixup_seen) RG_STAMP(9);
#endif
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if constexpr (P2)
          mbar_arrive_cluster(mapa_shared(tempty_bar(acc), 0));  // the even CTA's MMA reuses it
        else
          mbar_arrive(tempty_bar(acc));
      }
      if (++acc == C::NBUF) {
        acc = 0;
        aph ^= 1u;
      }
    }
    if (!ok && lane == 0) {
      atomicExch(err, kErrEpilogue);
      *abort_flag = 1;
    }
    // the staging buffers must have been read before the CTA exits; the global writes
    // themselves complete with the grid (a dependent grid's griddepcontrol.wait sees them)
    if (lane == 0) bulk_wait_read<0>();
    __syncwarp();
    if (warp == 2 && lane == 0) RG_STAMP(7);
  }

  __syncthreads();
#if RG_PHASE_TIMERS
  if (trace_row && threadIdx.x == 0) {
    trace_row[1] = global_ns();
    RG_STAMP(2);
  }
#endif
  // no CTA of a pair exits while its partner may still arrive on its barriers or
  // run MMAs on its shared memory and TMEM (nor one of a split-K cluster while the
  // others may still write its shared memory)
  if constexpr (P2 || CS) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    if constexpr (P2)
      tmem_dealloc_pair(tmem_base, C::TMEM_COLS);
    else
      tmem_dealloc(tmem_base, C::TMEM_COLS);
  }
}


template <int BM, int BN, int STAGES, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmW,
                     const GemmArgs args) {
  SingleSched<SPLIT> sched{&tmA,        &tmB,          &tmC,   &tmW,  args.tiles_m, args.tiles_n,
                           args.splits, args.kblocks, args.M, args.N, args.beta};
  sched.panel = args.panel;
  gemm_body<BM, BN, STAGES>(sched, args.ws, args.tickets, args.err, args.timeout, args.stall, args.early, args.trace);
}

// Split-K through distributed shared memory: launched as clusters of S CTAs (a
// launch attribute), one output tile per cluster.
template <int BM, int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_csplit_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                            const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmW,
                            const GemmArgs args) {
  ClusterSplitSched sched{{&tmA,        &tmB,          &tmC,   &tmW,  args.tiles_m, args.tiles_n,
                           args.splits, args.kblocks, args.M, args.N, args.beta}};
  sched.panel = args.panel;
  gemm_body<BM, BN, STAGES>(sched, args.ws, args.tickets, args.err, args.timeout, args.stall, args.early, args.trace);
}

template <int BM, int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_memtwin_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                             const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmW,
                             const GemmArgs args) {
  MemTwinSched sched{{&tmA,        &tmB,          &tmC,   &tmW,  args.tiles_m, args.tiles_n,
                      args.splits, args.kblocks, args.M, args.N, args.beta}};
  sched.panel = args.panel;
  gemm_body<BM, BN, STAGES>(sched, args.ws, args.tickets, args.err, args.timeout, args.stall, args.early, args.trace);
}

template <int BM, int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_streamk_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                             const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmW,
                             const GemmArgs args) {
  StreamKSched<false> sched{&tmA,   &tmB,   &tmC,      &tmW,        args.tiles_m, args.tiles_n, args.kblocks,
                            args.M, args.N, args.beta, args.splits /* CTAs sharing the tail */, args.dp_tiles};
  sched.panel = args.panel;
  gemm_body<BM, BN, STAGES>(sched, args.ws, args.tickets, args.err, args.timeout, args.stall, args.early, args.trace);
}

// cta_group::2 stream-K: whole waves of 256 x BN pair tiles on the 2-CTA clusters,
// the remainder tiles' K iterations spread over the clusters.
template <int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_2sm_streamk_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                                 const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmW,
                                 const GemmArgs args) {
  StreamKSched<true> sched{&tmA,   &tmB,   &tmC,      &tmW,        args.tiles_m, args.tiles_n, args.kblocks,
                           args.M, args.N, args.beta, args.splits /* clusters sharing the tail */, args.dp_tiles};
  sched.panel = args.panel;
  gemm_body<128, BN, STAGES>(sched, args.ws, args.tickets, args.err, args.timeout, args.stall, args.early, args.trace);
}

// cta_group::2: 2-CTA clusters, each pair one 256 x BN output tile (128 rows per CTA).
template <int BN, int STAGES, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_2sm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                         const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmW,
                         const GemmArgs args) {
  TwoSmSched<SPLIT> sched{&tmA, &tmB, &tmC, &tmW, args.tiles_m, args.tiles_n, args.kblocks, args.M, args.N, args.beta};
  sched.splits = args.splits;
  sched.panel = args.panel;
  gemm_body<128, BN, STAGES>(sched, args.ws, args.tickets, args.err, args.timeout, args.stall, args.early, args.trace);
}

template <int BM, int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_grouped_kernel(const GroupHeader* __restrict__ hdr, const GroupItem* __restrict__ items,
                             const __grid_constant__ CUtensorMap tmW, float* ws, int32_t* tickets, int32_t* err,
                             long long timeout) {
  GroupSched<false> sched{hdr, items, &tmW};
  gemm_body<BM, BN, STAGES>(sched, ws, tickets, err, timeout, 0, 0);
}

// The grouped launch of the cta_group::2 form: compiled with a cluster shape of
// two CTAs, so a graph kernel node launches it as pairs without a launch attribute.
template <int BN, int STAGES>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    gemm_bf16_grouped_2sm_kernel(const GroupHeader* __restrict__ hdr, const GroupItem* __restrict__ items,
                                 const __grid_constant__ CUtensorMap tmW, float* ws, int32_t* tickets, int32_t* err,
                                 long long timeout) {
  GroupSched<true> sched{hdr, items, &tmW};
  gemm_body<128, BN, STAGES>(sched, ws, tickets, err, timeout, 0, 0);
}

// Device-side spin of about `ns` nanoseconds (global timer), so that launches
// enqueued behind it start back to back.  Bounded by a cycle cap as well.
__global__ void spin_kernel(long long ns) {
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  const long long c0 = clock64();
  do {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  } while (static_cast<long long>(t - t0) < ns && clock64() - c0 < 4LL * ns + 100000LL);
}

// ------------------------------------------------------------------ host side

using KernFn = void (*)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap, const GemmArgs);

struct TileKernel {
  KernFn fn;        // split 1
  KernFn fn_split;  // split-K (S > 1)
  KernFn sk;        // stream-K instance of the same tile
  int bm, bn, smem;
  KernFn mem;           // memory twin (loads and stores, no MMA)
  KernFn two_sm;        // cta_group::2 instance (256-row tiles with BN >= 128), split 1, else null
  KernFn two_sm_split;  // cta_group::2 split-K instance, else null
  int smem2;
  KernFn two_sm_sk;     // cta_group::2 stream-K instance, else null
  KernFn csplit;        // split-K through distributed shared memory (clusters of S CTAs)
  int ring;             // bytes of the operand ring (the cluster split-K receive space)
};

// Stages of the cta_group::2 instances, per CTA: 16 KB of A + BN/2 x 64 of B per K block;
// the 256x128 pair's stages hold two K blocks.
template <int BN>
constexpr int kStages2Sm = BN == 128 ? 4 : 6;

template <int BM, int BN, int ST>
TileKernel make_tile_kernel() {
  TileKernel t{gemm_bf16_kernel<BM, BN, ST, false>, gemm_bf16_kernel<BM, BN, ST, true>,
               gemm_bf16_streamk_kernel<BM, BN, ST>, BM, BN, KCfg<BM, BN, ST>::SMEM_BYTES,
               gemm_bf16_memtwin_kernel<BM, BN, ST>, nullptr, nullptr, 0, nullptr,
               gemm_bf16_csplit_kernel<BM, BN, ST>, KCfg<BM, BN, ST>::STAGING_OFF};
  if constexpr (BM == 256 && BN >= 128) {
    t.two_sm = gemm_bf16_2sm_kernel<BN, kStages2Sm<BN>, false>;
    t.two_sm_split = gemm_bf16_2sm_kernel<BN, kStages2Sm<BN>, true>;
    t.smem2 = KCfg<128, BN, kStages2Sm<BN>, 2>::SMEM_BYTES;
    t.two_sm_sk = gemm_bf16_2sm_streamk_kernel<BN, kStages2Sm<BN>>;
  }
  return t;
}

static const TileKernel& tile_kernel(int tile) {
  static const TileKernel table[RG_NUM_TILES] = {
      make_tile_kernel<128, 64, 4>(),  make_tile_kernel<128, 128, 3>(), make_tile_kernel<128, 256, 4>(),
      make_tile_kernel<256, 64, 4>(),  make_tile_kernel<256, 128, 4>(), make_tile_kernel<256, 256, 3>(),
      make_tile_kernel<128, 192, 4>(), make_tile_kernel<256, 192, 3>(),
  };
  return table[tile];
}

// Grouped launches come in eleven kernel families: the eight 1-CTA tiles, then the
// cta_group::2 forms of the pair tiles (256x128, 256x256, 256x192).
constexpr int kGroupFamilies = RG_NUM_TILES + RG_NUM_PAIR_TILES;
using GroupedFn = void (*)(const GroupHeader*, const GroupItem*, const CUtensorMap, float*, int32_t*, int32_t*,
                           long long);
static const void* grouped_kernel(int family) {
  static const GroupedFn table[kGroupFamilies] = {
      gemm_bf16_grouped_kernel<128, 64, 4>,  gemm_bf16_grouped_kernel<128, 128, 3>,
      gemm_bf16_grouped_kernel<128, 256, 4>, gemm_bf16_grouped_kernel<256, 64, 4>,
      gemm_bf16_grouped_kernel<256, 128, 4>, gemm_bf16_grouped_kernel<256, 256, 3>,
      gemm_bf16_grouped_kernel<128, 192, 4>, gemm_bf16_grouped_kernel<256, 192, 3>,
      gemm_bf16_grouped_2sm_kernel<128, kStages2Sm<128>>, gemm_bf16_grouped_2sm_kernel<256, kStages2Sm<256>>,
      gemm_bf16_grouped_2sm_kernel<192, kStages2Sm<192>>,
  };
  return reinterpret_cast<const void*>(table[family]);
}
static int family_smem(int family) {
  return family < RG_NUM_TILES ? tile_kernel(family).smem : tile_kernel(pair_tile(family - RG_NUM_TILES)).smem2;
}
static int family_bn(int family) {
  return family < RG_NUM_TILES ? tile_kernel(family).bn : tile_kernel(pair_tile(family - RG_NUM_TILES)).bn;
}
// The family and the variant a grouped problem runs: stream-K variants run as
// their tile with split 1 (the grouped scheduler has no stream-K form).
static int grouped_variant(int v) {
  if (!variant_streamk(v)) return v;
  return variant_2sm(v) ? RG_VARIANT_2SM(variant_tile(v), 0) : RG_VARIANT(variant_tile(v), 0);
}
static int family_of(int v) {
  return variant_2sm(v) ? RG_NUM_TILES + RG_PAIR_INDEX(variant_tile(v)) : variant_tile(v);
}

}  // namespace rg

struct rg_ctx {
  int device = 0;
  int sm_count = 0;
  char name[64] = {0};
  float* ws = nullptr;
  int64_t ws_bytes = 0;
  int32_t* tickets = nullptr;
  int32_t* err = nullptr;
  long long timeout = 2000000000LL;
  int32_t stall = 0;
  int32_t static_operands = 0;  // rg_set_static_operands
  int64_t launches = 0;
  std::vector<cudaEvent_t> events;
  unsigned long long* trace = nullptr;  // phase stamps of the last traced launch (RG_PHASE_TIMERS builds)
  int32_t trace_on = 0;
  // device staging of rg_gemm_plan_host (grown on demand)
  void* stage_a = nullptr;
  void* stage_b = nullptr;
  float* stage_c = nullptr;
  int64_t stage_a_bytes = 0, stage_b_bytes = 0, stage_c_bytes = 0;
};

namespace rg {

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_mu;

static int cuda_fail(cudaError_t e, const char* what) {
  return fail(RG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static int get_encode() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_encode) return RG_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    return fail(RG_ERR_CUDA, "cannot resolve cuTensorMapEncodeTiled from the driver");
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return RG_OK;
}

// 2D row-major tensor map: `inner` contiguous elements per row, `outer` rows,
// rows `row_bytes` apart; box `box_inner` x `box_outer`; 128-byte swizzle;
// out-of-range elements read as zero.
static int make_map(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
                    uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(RG_ERR_INVALID, "cuTensorMapEncodeTiled rejected a tensor map (code " +
                                                         std::to_string(static_cast<int>(r)) + ")");
  return RG_OK;
}

struct Launch {
  KernFn fn = nullptr;
  CUtensorMap a, b, c, w;
  GemmArgs args{};
  dim3 grid;
  int smem = 0;
  bool zero_only = false;  // K == 0 with beta == 0: C = 0
  bool noop = false;
  int64_t ws_slots = 1;  // > 1: the launch uses the split-K workspace and tickets
  int cluster = 1;       // 2: launched as 2-CTA clusters
  float* C = nullptr;
  int64_t M = 0, N = 0, ldc = 0;
};

static int prepare(rg_ctx* ctx, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B,
                   int64_t ldb, float* C, int64_t ldc, int32_t variant, int32_t beta, int64_t pm, int64_t pn,
                   int64_t pk, Launch* L) {
  if (!ctx) return fail(RG_ERR_INVALID, "null context");
  if (M < 0 || N < 0 || K < 0) return fail(RG_ERR_INVALID, "negative size");
  if (variant < 0 || variant >= RG_NUM_VARIANTS) return fail(RG_ERR_INVALID, "variant id out of range");
  if (beta != 0 && beta != 1) return fail(RG_ERR_INVALID, "beta must be 0 or 1");
  if (pm == 0) pm = M;
  if (pn == 0) pn = N;
  if (pk == 0) pk = K;
  if (pm < M || pn < N || pk < K) return fail(RG_ERR_INVALID, "padded extents smaller than the problem");
  if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30) || pm > (1 << 30) || pn > (1 << 30) || pk > (1 << 30))
    return fail(RG_ERR_SHAPE, "size beyond 2^30");
  *L = Launch{};
  if (M == 0 || N == 0) {
    L->noop = true;
    return RG_OK;
  }
  if (!C) return fail(RG_ERR_INVALID, "null C");
  if (ldc < N) return fail(RG_ERR_INVALID, "ldc < N");
  if ((reinterpret_cast<uintptr_t>(C) & 15) || (ldc % 4)) return fail(RG_ERR_ALIGN, "C must be 16-byte aligned, ldc % 4 == 0");
  if (K == 0) {
    L->zero_only = (beta == 0);
    L->noop = (beta != 0);
    L->C = C;
    L->M = M;
    L->N = N;
    L->ldc = ldc;
    return RG_OK;
  }
  if (!A || !B) return fail(RG_ERR_INVALID, "null operand");
  if (lda < K || ldb < N) return fail(RG_ERR_INVALID, "lda < K or ldb < N");
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) || (lda % 8) || (ldb % 8))
    return fail(RG_ERR_ALIGN, "A and B must be 16-byte aligned with lda, ldb multiples of 8");
  int rc = get_encode();
  if (rc != RG_OK) return rc;
  const int tile = variant_tile(variant);
  const bool sk = variant_streamk(variant);
  const bool two = variant_2sm(variant);
  const int splits = variant_split(variant);
  const TileKernel& tk = tile_kernel(tile);
  const int64_t tiles_m = (pm + tk.bm - 1) / tk.bm;
  const int64_t tiles_n = (pn + tk.bn - 1) / tk.bn;
  const int64_t kblocks = (pk + kBK - 1) / kBK;
  // Split-K of a 1-CTA tile of at least 128 x 256 outputs runs as clusters of S CTAs reducing
  // through distributed shared memory, when the other S - 1 partials of a CTA's 1/S of the tile
  // fit its operand ring (not 256 x 256 with S = 8); otherwise through the workspace.  Measured
  // under the sweep protocol, the cluster form is 2-9 % faster than the workspace for these
  // tiles (768^2 x 2048 on 128 x 256, S = 2: 15.6 against 15.9 us; 256 x 512 x 4096 on 256 x 128,
  // S = 4: 19.6 against 21.4 us) but 3-21 % slower for the smaller ones (128^2 x 4096 on 128 x 64,
  // S = 8: 13.4 against 10.6 us), where its cluster launch and handshakes cost more than the
  // workspace round trip of their small partials.
  const bool csplit = splits > 1 && !two && !sk && tk.bm * tk.bn >= 128 * 256 &&
                      static_cast<int64_t>(splits - 1) * tk.bm * tk.bn * 4 / splits <= tk.ring;
  // workspace slots per tile: the split count, or stream-K's most segments on one tile
  int64_t slots = csplit ? 1 : splits;
  SkGeometry skg{};
  if (sk) {  // cta_group::2: the schedule runs over pair tiles and clusters
    skg = two ? sk_geometry(tiles_m * tiles_n, kblocks, ctx->sm_count / 2)
              : sk_geometry(tiles_m * tiles_n, kblocks, ctx->sm_count);
    slots = skg.max_pieces;
  }
  const bool uses_ws = slots > 1;
  if (uses_ws) {
    const int64_t need = slots * tiles_m * tiles_n * tk.bm * tk.bn * 4;
    if (need > ctx->ws_bytes || (two ? 2 : 1) * tiles_m * tiles_n * 4 > kMaxTickets)
      return fail(RG_ERR_SHAPE, "split-K workspace too small for this shape");
  }
  // cta_group::2: each CTA loads its own 128 rows of A (and 64-column boxes of B)
  rc = make_map(&L->a, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, A, K, M, lda * 2, kBK, two ? tk.bm / 2 : tk.bm);
  if (rc == RG_OK) rc = make_map(&L->b, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B, N, K, ldb * 2, 64, kBK);
  if (rc == RG_OK) rc = make_map(&L->c, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, C, N, M, ldc * 4, 32, 32);
  if (rc == RG_OK) {
    if (uses_ws)  // workspace rows: [slot][tile][BM], BN floats each
      rc = make_map(&L->w, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, ctx->ws, tk.bn,
                    static_cast<uint64_t>(slots) * tiles_m * tiles_n * tk.bm, static_cast<uint64_t>(tk.bn) * 4, 32, 32);
    else
      L->w = L->c;  // unused without split-K
  }
  if (rc != RG_OK) return rc;
  L->fn = (sk && two) ? tk.two_sm_sk
          : sk        ? tk.sk
          : csplit    ? tk.csplit
          : two       ? (splits > 1 ? tk.two_sm_split : tk.two_sm)
                      : (splits > 1 ? tk.fn_split : tk.fn);
  L->cluster = two ? 2 : csplit ? splits : 1;
  L->smem = two ? tk.smem2 : tk.smem;
  L->ws_slots = slots;
  GemmArgs& g = L->args;
  g.M = static_cast<int32_t>(M);
  g.N = static_cast<int32_t>(N);
  g.tiles_m = static_cast<int32_t>(two ? 2 * tiles_m : tiles_m);  // cta_group::2: 128-row tiles
  g.tiles_n = static_cast<int32_t>(tiles_n);
  g.splits = sk ? static_cast<int32_t>(skg.tail_ctas) : splits;  // stream-K: CTAs sharing the tail tiles
  g.dp_tiles = sk ? static_cast<int32_t>(skg.dp_tiles) : 0;
  g.kblocks = static_cast<int32_t>(kblocks);
  {
    // column panels whose B slice (panel tiles x padded K, BF16) is at most 32 MiB
    const int64_t bcol = std::max<int64_t>(1, kblocks * kBK * tk.bn * 2);
    g.panel = static_cast<int32_t>(std::max<int64_t>(1, std::min<int64_t>(tiles_n, (32LL << 20) / bcol)));
  }
  g.beta = beta;
  g.ws = ctx->ws;
  g.tickets = ctx->tickets;
  g.err = ctx->err;
  g.timeout = ctx->timeout;
  g.stall = ctx->stall;
  g.early = ctx->static_operands;
  g.trace = ctx->trace_on ? ctx->trace : nullptr;
  const int64_t units = tiles_m * tiles_n * splits;
  if (two && sk) {  // stream-K over 2-CTA clusters
    L->grid = dim3(static_cast<unsigned>(2 * skg.grid));
  } else if (two) {  // one 2-CTA cluster per (256-row tile, split), at most one CTA per SM
    L->grid = dim3(static_cast<unsigned>(2 * std::min<int64_t>(tiles_m * tiles_n * splits, ctx->sm_count / 2)));
  } else if (csplit) {  // one cluster of S CTAs per tile, not persistent
    L->grid = dim3(static_cast<unsigned>(units));
  } else {
    L->grid = dim3(static_cast<unsigned>(sk ? skg.grid : std::min<int64_t>(units, ctx->sm_count)));
  }
  return RG_OK;
}

static cudaError_t launch(rg_ctx* ctx, const Launch& L, cudaStream_t st) {
  if (L.noop) return cudaSuccess;
  if (L.zero_only) return cudaMemset2DAsync(L.C, L.ldc * 4, 0, L.N * 4, L.M, st);
  ++ctx->launches;
  void* params[5] = {const_cast<CUtensorMap*>(&L.a), const_cast<CUtensorMap*>(&L.b), const_cast<CUtensorMap*>(&L.c),
                     const_cast<CUtensorMap*>(&L.w), const_cast<GemmArgs*>(&L.args)};
  // Programmatic dependent launch: the grid may be scheduled while the previous
  // grid in the stream finishes; the kernel waits (griddepcontrol.wait) before
  // its first global memory access.
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = static_cast<unsigned>(L.cluster);
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = L.grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = static_cast<size_t>(L.smem);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = L.cluster > 1 ? 2 : 1;
  return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(L.fn), params);
}

int ctx_device(const rg_ctx* ctx) { return ctx ? ctx->device : 0; }

void ctx_identity(const rg_ctx* ctx, char name[64], int32_t* sms) {
  std::memset(name, 0, 64);
  *sms = 0;
  if (!ctx) return;
  std::memcpy(name, ctx->name, 64);
  *sms = ctx->sm_count;
}

// Leaves of the plan cell covering (M, N, K), clipped to the problem.
static int plan_launches(rg_ctx* ctx, const rg_plan* plan, int64_t M, int64_t N, int64_t K, const void* A,
                         int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, std::vector<Launch>& out) {
  out.clear();
  if (!plan) return fail(RG_ERR_INVALID, "null plan");
  if (M <= 0 || N <= 0 || K <= 0) return fail(RG_ERR_INVALID, "plan execution needs positive sizes");
  int64_t cell = 0;
  if (plan_cell(plan->p, M, N, K, &cell) != RG_OK) return fail(RG_ERR_SHAPE, "shape beyond the plan grid");
  const Plan& P = plan->p;
  if (!P.variant_ids.empty() && variant_fp8(P.variant_ids[0]))
    return fail(RG_ERR_INVALID, "an FP8 plan runs through rg_gemm_fp8_plan");
  for (int64_t i = P.leaf_off[cell]; i < P.leaf_off[cell + 1]; ++i) {
    const rg_leaf& lf = P.leaves[i];
    if (lf.m0 >= M || lf.n0 >= N || lf.k0 >= K) continue;  // wholly in the padding
    const int64_t m = std::min(lf.m, M - lf.m0), n = std::min(lf.n, N - lf.n0), k = std::min(lf.k, K - lf.k0);
    const auto* a = static_cast<const uint16_t*>(A) + lf.m0 * lda + lf.k0;
    const auto* b = static_cast<const uint16_t*>(B) + lf.k0 * ldb + lf.n0;
    float* c = C + lf.m0 * ldc + lf.n0;
    Launch L;
    const int rc = prepare(ctx, m, n, k, a, lda, b, ldb, c, ldc, lf.variant, lf.beta, lf.pm, lf.pn, lf.pk, &L);
    if (rc != RG_OK) return rc;
    out.push_back(L);
  }
  return RG_OK;
}

}  // namespace rg

// ------------------------------------------------------------------ shared with the FP8 and grouped kernels
namespace rg {

int fp8_make_map(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
                 uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  const int rc = get_encode();
  if (rc != RG_OK) return rc;
  return make_map(m, dt, base, inner, outer, row_bytes, box_inner, box_outer);
}

// Launch with programmatic dependent launch allowed (the kernel waits on
// griddepcontrol before touching global memory).
cudaError_t fp8_launch_pdl(const void* fn, dim3 grid, int threads, int smem, cudaStream_t st, void** params) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, params);
}

// The sweep protocol (Sec. 3: one discarded warm-up launch, then the mean of
// `reps` launches; Sec. 5.4: items in the given, randomised order): for each
// item, `prep` readies its launches and reports how many one repetition makes,
// `run` enqueues one repetition.  A device spin before the timed group lets the
// host enqueue the whole group, so the events time back-to-back device work.
// Events are recorded in batches of 256 items and read after one synchronise.
int timed_sweep(rg_ctx* ctx, const std::vector<int64_t>& order, const rg_sweep_opts& o, cudaStream_t st,
                int64_t* t_ns_out, const std::function<int(int64_t, int*)>& prep,
                const std::function<cudaError_t()>& run) {
  const int kBatch = 256;
  while (ctx->events.size() < 2 * kBatch) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return cuda_fail(e, "sweep: event");
    ctx->events.push_back(ev);
  }
  int nl = 1;
  if (!order.empty() && o.global_warmup > 0) {
    int rc = prep(order[0], &nl);
    if (rc != RG_OK) return rc;
    for (int i = 0; i < o.global_warmup; ++i)
      if (cudaError_t e = run(); e != cudaSuccess) return cuda_fail(e, "sweep: warm-up");
  }
  for (size_t base = 0; base < order.size(); base += kBatch) {
    const size_t nb = std::min<size_t>(kBatch, order.size() - base);
    for (size_t i = 0; i < nb; ++i) {
      int rc = prep(order[base + i], &nl);
      if (rc != RG_OK) return rc;
      cudaError_t e = cudaSuccess;
      for (int w = 0; w < o.warmup && e == cudaSuccess; ++w) e = run();
      if (e == cudaSuccess && o.spin_ns > 0) {
        spin_kernel<<<1, 1, 0, st>>>(o.spin_ns * o.reps * static_cast<long long>(nl));
        ++ctx->launches;
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaEventRecord(ctx->events[2 * i], st);
      for (int r = 0; r < o.reps && e == cudaSuccess; ++r) e = run();
      if (e == cudaSuccess) e = cudaEventRecord(ctx->events[2 * i + 1], st);
      if (e != cudaSuccess) return cuda_fail(e, "sweep: launch");
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "sweep: synchronize");
    for (size_t i = 0; i < nb; ++i) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ctx->events[2 * i], ctx->events[2 * i + 1]);
      if (e != cudaSuccess) return cuda_fail(e, "sweep: event time");
      const int64_t t = std::llround(static_cast<double>(ms) * 1e6 / o.reps);
      t_ns_out[order[base + i]] = t > 0 ? t : 1;
    }
  }
  return RG_OK;
}

// The context's error word, wait budget, SM count and split-K workspace for the
// kernels of other translation units.
int ctx_fp8_info(rg_ctx* ctx, Fp8CtxInfo* out) {
  if (!ctx) return fail(RG_ERR_INVALID, "null context");
  out->err = ctx->err;
  out->timeout = ctx->timeout;
  out->sms = ctx->sm_count;
  out->ws = ctx->ws;
  out->ws_bytes = ctx->ws_bytes;
  out->tickets = ctx->tickets;
  out->max_tickets = kMaxTickets;
  return RG_OK;
}

void ctx_count_launches(rg_ctx* ctx, int64_t n) {
  if (ctx) ctx->launches += n;
}

}  // namespace rg

// ------------------------------------------------------------------ C ABI

extern "C" int rg_init(int device, int64_t workspace_bytes, rg_ctx** out) {
  rg::clear_error();
  if (!out) return rg::fail(RG_ERR_INVALID, "rg_init: null out");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return rg::fail(RG_ERR_NO_DEVICE, "rg_init: no CUDA device");
  }
  if (device < 0 || device >= n) return rg::fail(RG_ERR_INVALID, "rg_init: device index out of range");
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) return rg::cuda_fail(e, "rg_init");
  if (prop.major != 10 || prop.minor != 3)
    return rg::fail(RG_ERR_NO_DEVICE, "rg_init: needs a compute capability 10.3 device (GB300), found " +
                                          std::to_string(prop.major) + "." + std::to_string(prop.minor));
  if ((e = cudaSetDevice(device)) != cudaSuccess) return rg::cuda_fail(e, "rg_init: cudaSetDevice");
  int rc = rg::get_encode();
  if (rc != RG_OK) return rc;
  auto* ctx = new (std::nothrow) rg_ctx();
  if (!ctx) return rg::fail(RG_ERR_OOM, "rg_init: host allocation");
  ctx->device = device;
  ctx->sm_count = prop.multiProcessorCount;
  std::strncpy(ctx->name, prop.name, 63);
  ctx->ws_bytes = workspace_bytes > 0 ? workspace_bytes : (512LL << 20);
  for (int t = 0; t < RG_NUM_TILES; ++t) {
    const rg::TileKernel& tk = rg::tile_kernel(t);
    if ((e = cudaFuncSetAttribute(reinterpret_cast<const void*>(tk.fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tk.smem)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(reinterpret_cast<const void*>(tk.fn_split),
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, tk.smem)) != cudaSuccess ||
        (tk.two_sm_split && (e = cudaFuncSetAttribute(reinterpret_cast<const void*>(tk.two_sm_split),
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, tk.smem2)) !=
                                cudaSuccess) ||
        (e = cudaFuncSetAttribute(reinterpret_cast<const void*>(tk.sk), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tk.smem)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(reinterpret_cast<const void*>(tk.csplit),
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, tk.smem)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(reinterpret_cast<const void*>(tk.mem), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tk.smem)) != cudaSuccess ||
        (tk.two_sm && (e = cudaFuncSetAttribute(reinterpret_cast<const void*>(tk.two_sm),
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, tk.smem2)) != cudaSuccess) ||
        (tk.two_sm_sk && (e = cudaFuncSetAttribute(reinterpret_cast<const void*>(tk.two_sm_sk),
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, tk.smem2)) !=
                             cudaSuccess)) {
      delete ctx;
      return rg::cuda_fail(e, "rg_init: shared-memory attribute");
    }
  }
  for (int f = 0; f < rg::kGroupFamilies; ++f)
    if ((e = cudaFuncSetAttribute(rg::grouped_kernel(f), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  rg::family_smem(f))) != cudaSuccess) {
      delete ctx;
      return rg::cuda_fail(e, "rg_init: shared-memory attribute (grouped)");
    }
  if ((e = cudaMalloc(&ctx->ws, ctx->ws_bytes)) != cudaSuccess ||
      (e = cudaMalloc(&ctx->tickets, sizeof(int32_t) * rg::kMaxTickets)) != cudaSuccess ||
      (e = cudaMalloc(&ctx->err, sizeof(int32_t))) != cudaSuccess) {
    cudaFree(ctx->ws);
    cudaFree(ctx->tickets);
    cudaFree(ctx->err);
    delete ctx;
    cudaGetLastError();
    return rg::fail(RG_ERR_OOM, std::string("rg_init: device allocation: ") + cudaGetErrorString(e));
  }
  cudaMemset(ctx->tickets, 0, sizeof(int32_t) * rg::kMaxTickets);
  cudaMemset(ctx->err, 0, sizeof(int32_t));
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
    rg_destroy(ctx);
    return rg::cuda_fail(e, "rg_init");
  }
  *out = ctx;
  return RG_OK;
}

extern "C" void rg_destroy(rg_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  for (auto ev : ctx->events) cudaEventDestroy(ev);
  cudaFree(ctx->trace);
  cudaFree(ctx->stage_a);
  cudaFree(ctx->stage_b);
  cudaFree(ctx->stage_c);
  cudaFree(ctx->ws);
  cudaFree(ctx->tickets);
  cudaFree(ctx->err);
  delete ctx;
}

extern "C" int rg_sm_count(const rg_ctx* ctx, int32_t* out) {
  if (!ctx || !out) return rg::fail(RG_ERR_INVALID, "rg_sm_count: null argument");
  *out = ctx->sm_count;
  return RG_OK;
}

extern "C" int rg_set_test_stall(rg_ctx* ctx, int32_t enable) {
  if (!ctx) return rg::fail(RG_ERR_INVALID, "rg_set_test_stall: null context");
  ctx->stall = enable ? 1 : 0;
  return RG_OK;
}

extern "C" int rg_launch_count(const rg_ctx* ctx, int64_t* out) {
  if (!ctx || !out) return rg::fail(RG_ERR_INVALID, "rg_launch_count: null argument");
  *out = ctx->launches;
  return RG_OK;
}

extern "C" int rg_phase_trace(rg_ctx* ctx, int32_t enable) {
  rg::clear_error();
  if (!ctx) return rg::fail(RG_ERR_INVALID, "rg_phase_trace: null context");
  if (!RG_PHASE_TIMERS)
    return rg::fail(RG_ERR_INVALID, "rg_phase_trace: this library was built without phase timers "
                                    "(build with RG_PHASE_TIMERS=1)");
  if (enable && !ctx->trace) {
    const size_t bytes = sizeof(unsigned long long) * rg::kTraceFields * static_cast<size_t>(ctx->sm_count);
    cudaError_t e = cudaMalloc(&ctx->trace, bytes);
    if (e == cudaSuccess) e = cudaMemset(ctx->trace, 0, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->trace = nullptr;
      return rg::fail(RG_ERR_OOM, "rg_phase_trace: trace buffer");
    }
  }
  ctx->trace_on = enable ? 1 : 0;
  return RG_OK;
}

extern "C" int rg_phase_trace_read(rg_ctx* ctx, uint64_t* out, int32_t max_ctas, int32_t* n_ctas) {
  rg::clear_error();
  if (!ctx || !out || !n_ctas || max_ctas <= 0) return rg::fail(RG_ERR_INVALID, "rg_phase_trace_read: bad argument");
  if (!ctx->trace) return rg::fail(RG_ERR_INVALID, "rg_phase_trace_read: tracing was never enabled");
  const int32_t n = std::min(max_ctas, ctx->sm_count);
  const size_t bytes = sizeof(unsigned long long) * rg::kTraceFields * static_cast<size_t>(n);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(out, ctx->trace, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemset(ctx->trace, 0, sizeof(unsigned long long) * rg::kTraceFields * static_cast<size_t>(ctx->sm_count));
  if (e != cudaSuccess) return rg::cuda_fail(e, "rg_phase_trace_read");
  *n_ctas = n;
  return RG_OK;
}

extern "C" int rg_set_static_operands(rg_ctx* ctx, int32_t enable) {
  if (!ctx) return rg::fail(RG_ERR_INVALID, "rg_set_static_operands: null context");
  ctx->static_operands = enable ? 1 : 0;
  return RG_OK;
}

extern "C" int rg_set_timeout_cycles(rg_ctx* ctx, int64_t cycles) {
  if (!ctx || cycles <= 0) return rg::fail(RG_ERR_INVALID, "rg_set_timeout_cycles: bad argument");
  ctx->timeout = cycles;
  return RG_OK;
}

extern "C" int rg_check(rg_ctx* ctx, void* stream) {
  if (!ctx) return rg::fail(RG_ERR_INVALID, "rg_check: null context");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return rg::cuda_fail(e, "rg_check: stream");
  int32_t code = 0;
  if ((e = cudaMemcpy(&code, ctx->err, sizeof(code), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return rg::cuda_fail(e, "rg_check: read error word");
  if (code != 0) {
    cudaMemset(ctx->err, 0, sizeof(int32_t));
    cudaMemset(ctx->tickets, 0, sizeof(int32_t) * rg::kMaxTickets);  // a kernel may have stopped mid-reduction
    cudaDeviceSynchronize();
    static const char* role[] = {"", "TMA producer", "MMA issuer", "epilogue"};
    return rg::fail(RG_ERR_TIMEOUT, std::string("rg_check: a bounded wait expired in the ") +
                                        (code >= 1 && code <= 3 ? role[code] : "kernel"));
  }
  return RG_OK;
}

extern "C" int rg_gemm(rg_ctx* ctx, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B,
                       int64_t ldb, float* C, int64_t ldc, int32_t variant, int32_t beta, int64_t pm, int64_t pn,
                       int64_t pk, void* stream) {
  rg::clear_error();
  rg::Launch L;
  int rc = rg::prepare(ctx, M, N, K, A, lda, B, ldb, C, ldc, variant, beta, pm, pn, pk, &L);
  if (rc != RG_OK) return rc;
  cudaError_t e = rg::launch(ctx, L, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RG_OK : rg::cuda_fail(e, "rg_gemm: launch");
}

extern "C" int rg_gemm_plan(rg_ctx* ctx, const rg_plan* plan, int64_t M, int64_t N, int64_t K, const void* A,
                            int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, void* stream) {
  rg::clear_error();
  std::vector<rg::Launch> ls;
  int rc = rg::plan_launches(ctx, plan, M, N, K, A, lda, B, ldb, C, ldc, ls);
  if (rc != RG_OK) return rc;
  for (const auto& L : ls) {
    cudaError_t e = rg::launch(ctx, L, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return rg::cuda_fail(e, "rg_gemm_plan: launch");
  }
  return RG_OK;
}

namespace {
// Grow a device staging buffer to at least `bytes` (the old contents are not kept).
int grow_stage(void** buf, int64_t* cap, int64_t bytes, cudaStream_t st) {
  if (bytes <= *cap) return RG_OK;
  cudaError_t e = cudaStreamSynchronize(st);  // work on the stream may still read the old buffer
  if (e == cudaSuccess && *buf) e = cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  if (e == cudaSuccess) e = cudaMalloc(buf, static_cast<size_t>(bytes));
  if (e != cudaSuccess) {
    *buf = nullptr;
    cudaGetLastError();
    return rg::fail(RG_ERR_OOM, std::string("rg_gemm_plan_host: staging buffer: ") + cudaGetErrorString(e));
  }
  *cap = bytes;
  return RG_OK;
}
}  // namespace

extern "C" int rg_gemm_plan_host(rg_ctx* ctx, const rg_plan* plan, int64_t M, int64_t N, int64_t K, const void* A,
                                 int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, void* stream) {
  rg::clear_error();
  if (!ctx || !plan || !A || !B || !C) return rg::fail(RG_ERR_INVALID, "rg_gemm_plan_host: null argument");
  if (M <= 0 || N <= 0 || K <= 0) return rg::fail(RG_ERR_INVALID, "rg_gemm_plan_host: sizes must be positive");
  if (lda < K || ldb < N || ldc < N) return rg::fail(RG_ERR_INVALID, "rg_gemm_plan_host: leading dimensions");
  if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30)) return rg::fail(RG_ERR_SHAPE, "rg_gemm_plan_host: size");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // device copies with leading dimensions rounded up to the TMA alignment
  const int64_t dlda = (K + 7) / 8 * 8, dldb = (N + 7) / 8 * 8, dldc = (N + 3) / 4 * 4;
  int rc = grow_stage(&ctx->stage_a, &ctx->stage_a_bytes, 2 * M * dlda, st);
  if (rc == RG_OK) rc = grow_stage(&ctx->stage_b, &ctx->stage_b_bytes, 2 * K * dldb, st);
  if (rc == RG_OK)
    rc = grow_stage(reinterpret_cast<void**>(&ctx->stage_c), &ctx->stage_c_bytes, 4 * M * dldc, st);
  if (rc != RG_OK) return rc;
  cudaError_t e = cudaMemcpy2DAsync(ctx->stage_a, dlda * 2, A, lda * 2, K * 2, M, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(ctx->stage_b, dldb * 2, B, ldb * 2, N * 2, K, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return rg::cuda_fail(e, "rg_gemm_plan_host: copy in");
  rc = rg_gemm_plan(ctx, plan, M, N, K, ctx->stage_a, dlda, ctx->stage_b, dldb, ctx->stage_c, dldc, stream);
  if (rc != RG_OK) return rc;
  e = cudaMemcpy2DAsync(C, ldc * 4, ctx->stage_c, dldc * 4, N * 4, M, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return rg::cuda_fail(e, "rg_gemm_plan_host: copy out");
  return rg_check(ctx, stream);
}

namespace {
uint64_t splitmix_next(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
}  // namespace

// The sweep behind rg_sweep and rg_sweep_memtwin.  memtwin: the ids are tile
// ids and every cell runs that tile's memory twin (never pruned).
static int sweep_impl(rg_ctx* ctx, const rg_grid* grid, int32_t n_variants, const int32_t* variant_ids,
                      const rg_plan* plan, const void* A, const void* B, float* C, const rg_sweep_opts* opts,
                      int64_t* t_ns_out, double* tflops_out, double* stats_out, void* stream, bool memtwin) {
  rg::clear_error();
  if (!ctx || !grid || !A || !B || !C || !t_ns_out) return rg::fail(RG_ERR_INVALID, "rg_sweep: null argument");
  if (!rg::grid_valid(*grid)) return rg::fail(RG_ERR_INVALID, "rg_sweep: invalid grid");
  if (plan ? n_variants != 1 : (n_variants <= 0 || !variant_ids))
    return rg::fail(RG_ERR_INVALID, "rg_sweep: variants");
  if (memtwin)
    for (int32_t i = 0; i < n_variants; ++i)
      if (variant_ids[i] < 0 || variant_ids[i] >= RG_NUM_TILES)
        return rg::fail(RG_ERR_INVALID, "rg_sweep_memtwin: tile id out of range");
  rg_sweep_opts o;
  rg_sweep_opts_default(&o);
  if (opts) o = *opts;
  if (o.reps <= 0 || o.warmup < 0 || o.global_warmup < 0 || o.spin_ns < 0 || o.shard_count < 1 ||
      o.shard_index < 0 || o.shard_index >= o.shard_count)
    return rg::fail(RG_ERR_INVALID, "rg_sweep: options");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t cells = rg::cells_of(*grid);
  const int64_t nk = grid->k.count, nn = grid->n.count;
  std::vector<int64_t> order(static_cast<size_t>(cells) * n_variants);
  for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int64_t>(i);
  if (o.shuffle) {
    uint64_t s = o.seed;
    for (size_t i = order.size() - 1; i > 0; --i) {
      const size_t j = static_cast<size_t>(splitmix_next(s) % (i + 1));
      std::swap(order[i], order[j]);
    }
  }
  std::vector<rg::Launch> ls;
  auto dims = [&](int64_t item, int64_t* M, int64_t* N, int64_t* K) {
    const int64_t cell = item % cells;
    const int64_t a = cell / (nn * nk), b = (cell / nk) % nn, c = cell % nk;
    *M = rg::axis_value(grid->m, a);
    *N = rg::axis_value(grid->n, b);
    *K = rg::axis_value(grid->k, c);
  };
  // A split-K variant is worth timing only where the unsplit tile count leaves
  // SMs idle and every split keeps at least two K blocks.
  auto pruned = [&](int64_t item) -> bool {
    if (plan || memtwin || !o.prune_splits) return false;
    const int32_t v = variant_ids[item / cells];
    const int S = rg::variant_split(v);
    const bool sk = rg::variant_streamk(v);
    if (rg::variant_2sm(v)) {  // a 256-row pair tile is worth it only beyond 128 rows
      int64_t M, N, K;
      dims(item, &M, &N, &K);
      if (M <= 128) return true;
      const rg::TileShape ts = rg::tile_shape(rg::variant_tile(v));
      const int64_t pairs = ((M + ts.bm - 1) / ts.bm) * ((N + ts.bn - 1) / ts.bn);
      if (sk) {  // as the 1-CTA stream-K rule, over clusters
        const int64_t clusters = ctx->sm_count / 2;
        return pairs < clusters ||
               rg::sk_geometry(pairs, (K + rg::kBK - 1) / rg::kBK, clusters).max_pieces == 1;
      }
      if (S == 1) return false;
      return 2 * pairs >= ctx->sm_count || (K + rg::kBK - 1) / rg::kBK < 2 * S;
    }
    if (S == 1 && !sk) return false;
    int64_t M, N, K;
    dims(item, &M, &N, &K);
    const rg::TileShape ts = rg::tile_shape(rg::variant_tile(v));
    const int64_t tiles = ((M + ts.bm - 1) / ts.bm) * ((N + ts.bn - 1) / ts.bn);
    const int64_t kblocks = (K + rg::kBK - 1) / rg::kBK;
    if (sk) {  // stream-K is timed where the tiles fill a wave (split-K covers fewer) and it splits some tile
      return tiles < ctx->sm_count || rg::sk_geometry(tiles, kblocks, ctx->sm_count).max_pieces == 1;
    }
    return tiles >= ctx->sm_count || kblocks < 2 * S;
  };
  if (o.prune_splits && !plan) {  // timed items first, pruned ones marked
    std::vector<int64_t> keep;
    keep.reserve(order.size());
    for (int64_t it : order) {
      if (pruned(it))
        t_ns_out[it] = RG_T_UNMEASURED;
      else
        keep.push_back(it);
    }
    order.swap(keep);
  }
  if (o.shard_count > 1) {  // this shard's share of the common order; the others' entries marked
    std::vector<int64_t> mine;
    mine.reserve(order.size() / o.shard_count + 1);
    for (size_t p = 0; p < order.size(); ++p) {
      if (static_cast<int32_t>(p % o.shard_count) == o.shard_index)
        mine.push_back(order[p]);
      else
        t_ns_out[order[p]] = RG_T_OTHER_SHARD;
    }
    order.swap(mine);
  }
  auto prep = [&](int64_t item, int* launches) -> int {
    int64_t M, N, K;
    dims(item, &M, &N, &K);
    int rc;
    if (plan) {
      rc = rg::plan_launches(ctx, plan, M, N, K, A, K, B, N, C, N, ls);
    } else {
      ls.resize(1);
      const int32_t v = variant_ids[item / cells];
      rc = rg::prepare(ctx, M, N, K, A, K, B, N, C, N, memtwin ? RG_VARIANT(v, 0) : v, 0, 0, 0, 0, &ls[0]);
      if (rc == RG_OK && memtwin) ls[0].fn = rg::tile_kernel(v).mem;
    }
    *launches = static_cast<int>(ls.size());
    return rc;
  };
  auto run = [&]() -> cudaError_t {
    for (const auto& L : ls) {
      cudaError_t e = rg::launch(ctx, L, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  // The sweep times one GEMM at a time: the static-operand mode stays off even
  // though the operands are constant, because it would let a launch's loads and
  // MMAs run on idle SMs while the launch ahead of it is still running, so the
  // per-launch time would measure several overlapped GEMMs.
  const int32_t saved_static = ctx->static_operands;
  ctx->static_operands = 0;
  int rc = rg::timed_sweep(ctx, order, o, st, t_ns_out, prep, run);
  ctx->static_operands = saved_static;
  if (rc != RG_OK) return rc;
  rc = rg_check(ctx, stream);
  if (rc != RG_OK) return rc;
  return rg::sweep_surfaces(grid, plan ? 1 : n_variants, t_ns_out, tflops_out, stats_out);
}

extern "C" int rg_sweep(rg_ctx* ctx, const rg_grid* grid, int32_t n_variants, const int32_t* variant_ids,
                        const rg_plan* plan, const void* A, const void* B, float* C, const rg_sweep_opts* opts,
                        int64_t* t_ns_out, double* tflops_out, double* stats_out, void* stream) {
  return sweep_impl(ctx, grid, n_variants, variant_ids, plan, A, B, C, opts, t_ns_out, tflops_out, stats_out, stream,
                    false);
}

extern "C" int rg_sweep_memtwin(rg_ctx* ctx, const rg_grid* grid, int32_t n_tiles, const int32_t* tile_ids,
                                const void* A, const void* B, float* C, const rg_sweep_opts* opts, int64_t* t_ns_out,
                                void* stream) {
  return sweep_impl(ctx, grid, n_tiles, tile_ids, nullptr, A, B, C, opts, t_ns_out, nullptr, nullptr, stream, true);
}

extern "C" int rg_gemm_memtwin(rg_ctx* ctx, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                               const void* B, int64_t ldb, float* C, int64_t ldc, int32_t tile, void* stream) {
  rg::clear_error();
  if (tile < 0 || tile >= RG_NUM_TILES) return rg::fail(RG_ERR_INVALID, "rg_gemm_memtwin: tile id out of range");
  rg::Launch L;
  int rc = rg::prepare(ctx, M, N, K, A, lda, B, ldb, C, ldc, RG_VARIANT(tile, 0), 0, 0, 0, 0, &L);
  if (rc != RG_OK) return rc;
  if (L.fn) L.fn = rg::tile_kernel(tile).mem;
  cudaError_t e = rg::launch(ctx, L, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RG_OK : rg::cuda_fail(e, "rg_gemm_memtwin: launch");
}

// ------------------------------------------------------------------ grouped GEMM under CUDA graphs
//
// A group object owns, per kernel family, kGroupSlots slots (built on the
// family's first use).  Each slot: a pinned host work list, a device work list
// (header + items), a CUDA graph [copy host list -> device list, persistent
// grouped kernel over all SMs] instantiated once, and an event marking the
// slot's last replay.  A call sorts its problems by family; for each family
// present it fills work lists -- starting a further list whenever the next item's
// split-K partials or tickets would not fit the group's workspace, or the list is
// full -- and replays one graph per list on the caller's stream, so the lists of
// one call run one after another and each may reuse the whole workspace.  The
// graph's topology never changes; only the list contents do.
namespace rg {
constexpr int kGroupSlots = 4;
constexpr int64_t kGroupMinWorkspace = 1 << 20;
}

struct rg_group {
  rg_ctx* ctx = nullptr;
  int tile = 0;
  int max_items = 0;
  float* ws = nullptr;
  int64_t ws_bytes = 0;
  int32_t* tickets = nullptr;
  struct Slot {
    unsigned char* host = nullptr;  // pinned: header + items
    unsigned char* dev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t copy_node = nullptr;
    cudaEvent_t done = nullptr;
    bool used = false;
  };
  struct Family {
    Slot slot[rg::kGroupSlots];
    int next = 0;
    bool ready = false;
    CUtensorMap tmW;
  } fam[rg::kGroupFamilies];
};

namespace rg {
static_assert(sizeof(GroupHeader) == 128 && sizeof(GroupItem) == 512, "work-list record sizes");
static size_t group_bytes(int n) { return sizeof(GroupHeader) + static_cast<size_t>(n) * sizeof(GroupItem); }

static void group_free(rg_group* g) {
  if (!g) return;
  for (auto& f : g->fam)
    for (auto& sl : f.slot) {
      if (sl.used) cudaEventSynchronize(sl.done);
      if (sl.exec) cudaGraphExecDestroy(sl.exec);
      if (sl.graph) cudaGraphDestroy(sl.graph);
      if (sl.done) cudaEventDestroy(sl.done);
      if (sl.host) cudaFreeHost(sl.host);
      if (sl.dev) cudaFree(sl.dev);
    }
  cudaFree(g->ws);
  cudaFree(g->tickets);
  delete g;
}

static int group_build_graph(rg_group* g, int family, rg_group::Slot& sl) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e != cudaSuccess) return cuda_fail(e, "rg_group: graph");
  cudaGraphNode_t copy = nullptr, kern = nullptr;
  e = cudaGraphAddMemcpyNode1D(&copy, graph, nullptr, 0, sl.dev, sl.host, group_bytes(g->max_items),
                               cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const GroupHeader* hdr = reinterpret_cast<const GroupHeader*>(sl.dev);
    const GroupItem* items = reinterpret_cast<const GroupItem*>(sl.dev + sizeof(GroupHeader));
    CUtensorMap tmW = g->fam[family].tmW;
    float* ws = g->ws;
    int32_t* tickets = g->tickets;
    int32_t* err = g->ctx->err;
    long long timeout = g->ctx->timeout;
    void* params[7] = {&hdr, &items, &tmW, &ws, &tickets, &err, &timeout};
    const bool two = family >= RG_NUM_TILES;
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(grouped_kernel(family));
    kp.gridDim = dim3(static_cast<unsigned>(two ? g->ctx->sm_count / 2 * 2 : g->ctx->sm_count));
    kp.blockDim = dim3(kThreads);
    kp.sharedMemBytes = static_cast<unsigned>(family_smem(family));
    kp.kernelParams = params;
    e = cudaGraphAddKernelNode(&kern, graph, &copy, 1, &kp);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(e, "rg_group: build graph");
  }
  sl.graph = graph;
  sl.copy_node = copy;
  return RG_OK;
}

// Slots, graphs and the workspace tensor map of one family, on its first use.
static int group_family_ready(rg_group* g, int family) {
  rg_group::Family& f = g->fam[family];
  if (f.ready) return RG_OK;
  const int bn = family_bn(family);
  int rc = make_map(&f.tmW, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g->ws, static_cast<uint64_t>(bn),
                    static_cast<uint64_t>(g->ws_bytes / (4 * bn)), static_cast<uint64_t>(bn) * 4, 32, 32);
  if (rc != RG_OK) return rc;
  const size_t bytes = group_bytes(g->max_items);
  for (auto& sl : f.slot) {
    cudaError_t e = cudaMallocHost(&sl.host, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&sl.dev, bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(RG_ERR_OOM, std::string("rg_gemm_grouped: work lists: ") + cudaGetErrorString(e));
    }
    std::memset(sl.host, 0, bytes);
    rc = group_build_graph(g, family, sl);
    if (rc != RG_OK) return rc;
  }
  f.ready = true;
  return RG_OK;
}

// Replays the next slot of `family` with the list in `items` (count items, units units).
static int group_flush(rg_group* g, int family, const std::vector<GroupItem>& items, int64_t units,
                       cudaStream_t st) {
  if (items.empty()) return RG_OK;
  rg_group::Family& f = g->fam[family];
  rg_group::Slot& sl = f.slot[f.next];
  f.next = (f.next + 1) % kGroupSlots;
  cudaError_t e;
  if (sl.used && (e = cudaEventSynchronize(sl.done)) != cudaSuccess) return cuda_fail(e, "rg_gemm_grouped: slot");
  auto* hdr = reinterpret_cast<GroupHeader*>(sl.host);
  hdr->n_items = static_cast<int32_t>(items.size());
  hdr->total_units = static_cast<int32_t>(units);
  std::memcpy(sl.host + sizeof(GroupHeader), items.data(), items.size() * sizeof(GroupItem));
  const int n = static_cast<int>(items.size());
  e = cudaGraphExecMemcpyNodeSetParams1D(sl.exec, sl.copy_node, sl.dev, sl.host, group_bytes(n),
                                         cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaGraphLaunch(sl.exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
  if (e != cudaSuccess) return cuda_fail(e, "rg_gemm_grouped: replay");
  sl.used = true;
  g->ctx->launches += 1;
  return RG_OK;
}
}  // namespace rg

extern "C" int rg_group_create(rg_ctx* ctx, int32_t tile, int32_t max_items, int64_t workspace_bytes,
                               rg_group** out) {
  rg::clear_error();
  if (!ctx || !out || tile < 0 || tile >= RG_NUM_TILES || max_items <= 0 || max_items > (1 << 20) ||
      workspace_bytes < 0)
    return rg::fail(RG_ERR_INVALID, "rg_group_create: bad argument");
  *out = nullptr;
  auto* g = new (std::nothrow) rg_group();
  if (!g) return rg::fail(RG_ERR_OOM, "rg_group_create: host allocation");
  g->ctx = ctx;
  g->tile = tile;
  g->max_items = max_items;
  g->ws_bytes = std::max<int64_t>(workspace_bytes, rg::kGroupMinWorkspace) / 1024 * 1024;
  cudaError_t e = cudaMalloc(&g->ws, static_cast<size_t>(g->ws_bytes));
  if (e == cudaSuccess) e = cudaMalloc(&g->tickets, sizeof(int32_t) * rg::kMaxTickets);
  if (e == cudaSuccess) e = cudaMemset(g->tickets, 0, sizeof(int32_t) * rg::kMaxTickets);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    rg::group_free(g);
    return rg::fail(RG_ERR_OOM, std::string("rg_group_create: ") + cudaGetErrorString(e));
  }
  // every family's work lists and graphs now, so that no call allocates or
  // instantiates on the serving path
  for (int f = 0; f < rg::kGroupFamilies; ++f) {
    const int rc = rg::group_family_ready(g, f);
    if (rc != RG_OK) {
      rg::group_free(g);
      return rc;
    }
  }
  *out = g;
  return RG_OK;
}

extern "C" void rg_group_destroy(rg_group* g) { rg::group_free(g); }

namespace rg {
void group_workspace(rg_group* g, float** ws, int64_t* ws_bytes, int32_t** tickets, int64_t* max_tickets) {
  *ws = g->ws;
  *ws_bytes = g->ws_bytes;
  *tickets = g->tickets;
  *max_tickets = kMaxTickets;
}
}  // namespace rg

extern "C" int rg_gemm_grouped(rg_group* g, const rg_group_problem* probs, int32_t n, void* stream) {
  rg::clear_error();
  if (!g || (n > 0 && !probs) || n < 0) return rg::fail(RG_ERR_INVALID, "rg_gemm_grouped: bad argument");
  if (n == 0) return RG_OK;
  // A view of the context whose split-K workspace and tickets are the group's.
  rg_ctx view;
  view.device = g->ctx->device;
  view.sm_count = g->ctx->sm_count;
  view.ws = g->ws;
  view.ws_bytes = g->ws_bytes;
  view.tickets = g->tickets;
  view.err = g->ctx->err;
  view.timeout = g->ctx->timeout;
  struct Prepared {
    int family;
    rg::Launch L;
  };
  std::vector<Prepared> prep;
  prep.reserve(static_cast<size_t>(n));
  for (int32_t i = 0; i < n; ++i) {  // every problem is checked before anything is enqueued
    const rg_group_problem& p = probs[i];
    if (p.variant >= RG_NUM_VARIANTS) return rg::fail(RG_ERR_INVALID, "rg_gemm_grouped: variant id out of range");
    const int v = p.variant < 0 ? RG_VARIANT(g->tile, 0) : rg::grouped_variant(p.variant);
    Prepared q;
    q.family = rg::family_of(v);
    const int rc = rg::prepare(&view, p.M, p.N, p.K, p.A, p.lda, p.B, p.ldb, p.C, p.ldc, v, p.beta, p.pm, p.pn, p.pk,
                               &q.L);
    if (rc != RG_OK) return rc;
    if (q.L.noop) continue;
    if (q.L.zero_only) return rg::fail(RG_ERR_INVALID, "rg_gemm_grouped: K == 0 problems are not grouped");
    prep.push_back(q);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<rg::GroupItem> items;
  items.reserve(static_cast<size_t>(g->max_items));
  for (int f = 0; f < rg::kGroupFamilies; ++f) {
    bool any = false;
    for (const auto& q : prep) any = any || q.family == f;
    if (!any) continue;
    int rc = rg::group_family_ready(g, f);
    if (rc != RG_OK) return rc;
    const bool two = f >= RG_NUM_TILES;
    const int bm = two ? 128 : rg::tile_kernel(f).bm;
    const int64_t ws_rows = g->ws_bytes / (4 * rg::family_bn(f));
    items.clear();
    int64_t units = 0, rows = 0, tks = 0;
    for (const auto& q : prep) {
      if (q.family != f) continue;
      const rg::GemmArgs& a = q.L.args;
      const int64_t ntiles = static_cast<int64_t>(a.tiles_m) * a.tiles_n;
      const int64_t my_units = (two ? ntiles / 2 : ntiles) * a.splits;
      const int64_t my_rows = a.splits > 1 ? a.splits * ntiles * bm : 0;
      const int64_t my_tks = a.splits > 1 ? 4 * ntiles : 0;
      if (my_rows > ws_rows || my_tks > rg::kMaxTickets)
        return rg::fail(RG_ERR_SHAPE, "rg_gemm_grouped: a problem's split-K partials exceed the group's workspace");
      if (static_cast<int>(items.size()) == g->max_items || rows + my_rows > ws_rows || tks + my_tks > rg::kMaxTickets ||
          units + my_units > (1LL << 30)) {
        if ((rc = rg::group_flush(g, f, items, units, st)) != RG_OK) return rc;
        items.clear();
        units = rows = tks = 0;
      }
      rg::GroupItem it;
      std::memset(&it, 0, sizeof(it));
      it.a = q.L.a;
      it.b = q.L.b;
      it.c = q.L.c;
      it.M = a.M;
      it.N = a.N;
      it.beta = a.beta;
      it.tiles_m = a.tiles_m;
      it.tiles_n = a.tiles_n;
      it.kblocks = a.kblocks;
      it.unit_start = static_cast<int32_t>(units);
      it.splits = a.splits;
      it.ws_row0 = static_cast<int32_t>(rows);
      it.tk0 = static_cast<int32_t>(tks);
      items.push_back(it);
      units += my_units;
      rows += my_rows;
      tks += my_tks;
    }
    if ((rc = rg::group_flush(g, f, items, units, st)) != RG_OK) return rc;
  }
  return RG_OK;
}

// ------------------------------------------------------------------ entry point without allocation
//
// rg_gemm_noalloc runs the same kernel as rg_gemm, but its split-K scratch
// (partial sums, tile tickets, the bounded-wait error word) lives in one
// file-scope device array instead of memory from cudaMalloc.  It is for
// callers that must not allocate device memory on their call path: a host
// framework whose own allocator owns the device memory budget, or code that
// cannot afford the implicit device synchronisation cudaMalloc may cause.
// The array is part of the library image: every GPU that loads the library
// holds it until the process exits.
namespace rg {

constexpr int64_t kNoallocPartialBytes = RG_NOALLOC_PARTIAL_BYTES;
constexpr int64_t kNoallocTickets = 4 * RG_NOALLOC_MAX_TILES;
// layout: [partials | error word, padded to 256 B | tickets]
constexpr int64_t kNoallocErrOff = kNoallocPartialBytes;
constexpr int64_t kNoallocTicketOff = kNoallocErrOff + 256;
constexpr int64_t kNoallocBytes = kNoallocTicketOff + kNoallocTickets * 4;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

struct NoallocDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int sm_count = 0;
};
constexpr int kNoallocMaxDevices = 64;
static NoallocDevice g_noalloc_dev[kNoallocMaxDevices];
static std::mutex g_noalloc_mu;

// One-time set-up per device, run by the first call on that device with the
// device current: checks the device, resolves the tensor-map encoder, sets the
// kernels' shared-memory limit and looks up the array's device address.
static int noalloc_setup(int dev, NoallocDevice** out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(RG_ERR_INVALID, "rg_gemm_noalloc: device index too large");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoallocDevice& d = g_noalloc_dev[dev];
  if (!d.ready) {
    int major = 0, minor = 0, sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "rg_gemm_noalloc: device attributes");
    if (major != 10 || minor != 3) return fail(RG_ERR_NO_DEVICE, "rg_gemm_noalloc: needs a compute capability 10.3 device");
    int rc = get_encode();
    if (rc != RG_OK) return rc;
    for (int t = 0; t < RG_NUM_TILES; ++t) {
      const TileKernel& tk = tile_kernel(t);
      for (KernFn fn : {tk.fn, tk.fn_split, tk.sk, tk.csplit}) {
        e = cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize, tk.smem);
        if (e != cudaSuccess) return cuda_fail(e, "rg_gemm_noalloc: shared-memory attribute");
      }
      for (KernFn fn : {tk.two_sm, tk.two_sm_split, tk.two_sm_sk}) {
        if (!fn) continue;
        e = cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tk.smem2);
        if (e != cudaSuccess) return cuda_fail(e, "rg_gemm_noalloc: shared-memory attribute");
      }
    }
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) return cuda_fail(e, "rg_gemm_noalloc: cudaGetSymbolAddress of the scratch array");
    d.scratch = static_cast<unsigned char*>(ptr);
    d.sm_count = sms;
    d.ready = true;
  }
  *out = &d;
  return RG_OK;
}

}  // namespace rg

extern "C" int rg_gemm_noalloc(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B,
                               int64_t ldb, float* C, int64_t ldc, int32_t variant, int32_t beta, void* stream) {
  rg::clear_error();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rg::cuda_fail(e, "rg_gemm_noalloc: cudaGetDevice");
  rg::NoallocDevice* d = nullptr;
  int rc = rg::noalloc_setup(dev, &d);
  if (rc != RG_OK) return rc;
  if (variant < 0 || variant >= RG_NUM_VARIANTS) return rg::fail(RG_ERR_INVALID, "rg_gemm_noalloc: variant id out of range");
  const int splits = rg::variant_split(variant);
  if ((splits > 1 || rg::variant_streamk(variant)) && M > 0 && N > 0 && K > 0) {
    const rg::TileShape ts = rg::tile_shape(rg::variant_tile(variant));
    const int64_t tiles = ((M + ts.bm - 1) / ts.bm) * ((N + ts.bn - 1) / ts.bn);
    int64_t slots = splits;
    if (rg::variant_streamk(variant)) {
      const int64_t kb = (K + rg::kBK - 1) / rg::kBK;
      slots = rg::sk_geometry(tiles, kb, rg::variant_2sm(variant) ? d->sm_count / 2 : d->sm_count).max_pieces;
    }
    const int64_t need = slots > 1 ? slots * tiles * ts.bm * ts.bn * 4 : 0;
    const int64_t ticket_tiles = rg::variant_2sm(variant) ? 2 * tiles : tiles;  // cta_group::2: 128-row tiles
    if (need > rg::kNoallocPartialBytes || (slots > 1 && ticket_tiles > RG_NOALLOC_MAX_TILES))
      return rg::fail(RG_ERR_SHAPE, "rg_gemm_noalloc: split-K needs " + std::to_string(need) +
                                        " scratch bytes and " + std::to_string(tiles) + " tiles; the fixed scratch holds " +
                                        std::to_string(rg::kNoallocPartialBytes) + " bytes and " +
                                        std::to_string(RG_NOALLOC_MAX_TILES) + " tiles");
  }
  // A context whose workspace, tickets and error word are views of the scratch
  // array; constructing it allocates nothing on the device.
  rg_ctx view;
  view.device = dev;
  view.sm_count = d->sm_count;
  view.ws = reinterpret_cast<float*>(d->scratch);
  view.ws_bytes = rg::kNoallocPartialBytes;
  view.err = reinterpret_cast<int32_t*>(d->scratch + rg::kNoallocErrOff);
  view.tickets = reinterpret_cast<int32_t*>(d->scratch + rg::kNoallocTicketOff);
  rg::Launch L;
  rc = rg::prepare(&view, M, N, K, A, lda, B, ldb, C, ldc, variant, beta, 0, 0, 0, &L);
  if (rc != RG_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!L.noop && !L.zero_only) {
    // the error word and the tickets this launch uses must start at zero
    const int64_t clear = rg::kNoallocTicketOff - rg::kNoallocErrOff +
                          (L.ws_slots > 1 ? static_cast<int64_t>(L.args.tiles_m) * L.args.tiles_n * 4 * 4 : 0);
    e = cudaMemsetAsync(d->scratch + rg::kNoallocErrOff, 0, static_cast<size_t>(clear), st);
    if (e != cudaSuccess) return rg::cuda_fail(e, "rg_gemm_noalloc: clear tickets");
  }
  e = rg::launch(&view, L, st);
  return e == cudaSuccess ? RG_OK : rg::cuda_fail(e, "rg_gemm_noalloc: launch");
}

extern "C" int rg_noalloc_check(void* stream) {
  rg::clear_error();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rg::cuda_fail(e, "rg_noalloc_check: cudaGetDevice");
  if (dev < 0 || dev >= rg::kNoallocMaxDevices) return rg::fail(RG_ERR_INVALID, "rg_noalloc_check: device index too large");
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(rg::g_noalloc_mu);
    if (rg::g_noalloc_dev[dev].ready) scratch = rg::g_noalloc_dev[dev].scratch;
  }
  if (!scratch) return RG_OK;  // no rg_gemm_noalloc call has run on this device
  if ((e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream))) != cudaSuccess)
    return rg::cuda_fail(e, "rg_noalloc_check: stream");
  int32_t code = 0;
  if ((e = cudaMemcpy(&code, scratch + rg::kNoallocErrOff, sizeof(code), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return rg::cuda_fail(e, "rg_noalloc_check: read error word");
  if (code == 0) return RG_OK;
  // a kernel that gave up a wait may have stopped mid-reduction: clear the error
  // word and every ticket so the next call starts clean
  e = cudaMemset(scratch + rg::kNoallocErrOff, 0, static_cast<size_t>(rg::kNoallocBytes - rg::kNoallocErrOff));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return rg::cuda_fail(e, "rg_noalloc_check: clear scratch");
  static const char* role[] = {"", "TMA producer", "MMA issuer", "epilogue"};
  return rg::fail(RG_ERR_TIMEOUT, std::string("rg_noalloc_check: a bounded wait expired in the ") +
                                      (code >= 1 && code <= 3 ? role[code] : "kernel"));
}
