// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "rg.h"

namespace rg {

// Record a message for rg_last_error() on this thread and return `code`.
int fail(int code, const std::string& msg);
void clear_error();

inline int64_t cells_of(const rg_grid& g) {
  return static_cast<int64_t>(g.m.count) * g.n.count * g.k.count;
}
inline bool grid_valid(const rg_grid& g) {
  const rg_axis* ax[3] = {&g.m, &g.n, &g.k};
  for (auto* a : ax)
    if (a->count <= 0 || a->step <= 0 || a->start <= 0) return false;
  return true;
}
inline int64_t axis_value(const rg_axis& a, int64_t i) { return a.start + i * a.step; }

struct Plan {
  rg_grid grid{};
  std::vector<int32_t> variant_ids;
  std::vector<int64_t> T0s, T1, T2;
  std::vector<int32_t> vstar, target3, action, q;
  std::vector<int64_t> leaf_off;  // cells + 1 offsets into leaves
  std::vector<rg_leaf> leaves;
};

// Tile geometry of a variant id.
struct TileShape {
  int bm, bn;
};
TileShape tile_shape(int tile);
// Variant ids: tile * RG_NUM_SPLITS + log2(split) for the split-K variants, then
// RG_VARIANT_SK(tile) (stream-K), RG_VARIANT_2SM(tile, log2(split)) (cta_group::2,
// the pair tiles 256x128, 256x256, 256x192) and RG_VARIANT_2SM_SK(tile)
// (cta_group::2 stream-K).
constexpr int kClassicVariants = RG_NUM_TILES * RG_NUM_SPLITS;
constexpr int k2SmVariants = kClassicVariants + RG_NUM_TILES;
constexpr int k2SmSkVariants = k2SmVariants + RG_NUM_PAIR_TILES * RG_NUM_SPLITS;
// The tile of the i-th pair tile (RG_PAIR_INDEX inverted).
constexpr int pair_tile(int i) { return i == 2 ? RG_TILE_256x192 : RG_TILE_256x128 + i; }
constexpr bool is_pair_tile(int t) {
  return t == RG_TILE_256x128 || t == RG_TILE_256x256 || t == RG_TILE_256x192;
}
inline bool variant_2sm(int v) { return v >= k2SmVariants; }
inline bool variant_streamk(int v) { return (v >= kClassicVariants && v < k2SmVariants) || v >= k2SmSkVariants; }
inline int variant_tile(int v) {
  return v >= k2SmSkVariants     ? pair_tile(v - k2SmSkVariants)
         : v >= k2SmVariants     ? pair_tile((v - k2SmVariants) / RG_NUM_SPLITS)
         : v >= kClassicVariants ? v - kClassicVariants
                                 : v / RG_NUM_SPLITS;
}
inline bool variant_fp8(int v) { return v >= RG_FP8_VARIANT_BASE && v < RG_FP8_VARIANT_BASE + RG_FP8_NUM_VARIANTS; }
inline bool variant_valid(int v) { return (v >= 0 && v < RG_NUM_VARIANTS) || variant_fp8(v); }
inline int variant_split(int v) {
  return variant_streamk(v)      ? 1
         : v >= k2SmVariants     ? 1 << ((v - k2SmVariants) % RG_NUM_SPLITS)
                                 : 1 << (v % RG_NUM_SPLITS);
}
// Stream-K geometry shared by the launcher, the sweep's pruning and the kernel,
// for T tiles on P CTAs with T = w P + r, 0 < r < P (whole waves with no
// remainder run data-parallel).
//  - Balanced form (w >= 1 and r <= P/4 or r >= P/2): all whole waves but the
//    last run data-parallel (one tile per CTA per wave), and the K iterations of
//    the last whole wave plus the remainder are divided evenly among all P CTAs.
//    Each gets at least one tile's worth, so no tile spans more than 2 CTAs, and
//    the partial wave costs 1 + r/P tiles of time per CTA instead of 2, at the
//    price of one published partial per CTA.
//  - Remainder form (w = 0, or P/4 < r < P/2): all whole waves run data-parallel
//    and only the r remainder tiles' iterations are divided, among up to
//    min(kSkMaxPieces r, P) CTAs (each at least kSkMinIters K blocks); the tail
//    costs about half a tile and 2r partials.  With w = 0 a tile can span one
//    more CTA than kSkMaxPieces; max_pieces counts it.
// Measured on GB300 (sweep protocol, 9 shapes): the balanced form wins where r is
// small (4096 x 1280 x 4096 on 256 x 256 pairs, r/P = 4/76: 36.9 against 41.0 us)
// and where r >= P/2 (2176 x 1920 x 1152 on 128 x 128, r/P = 103/152: 18.7 against
// 21.8 us); the remainder form where P/4 < r < P/2 (2560 x 2560 x 2048 on pairs,
// 24/76: 28.2 against 31.5 us), since its 2r partials cost less than P of them.
constexpr int64_t kSkMinIters = 4;
// About 2 pieces per tail tile: the last arriving piece then reads one other
// partial, and that fixup, not the K loop, bounds the tail (phase timers: each
// further partial adds about 0.3 us per 32-column chunk of a CTA's rows).
constexpr int64_t kSkMaxPieces = 2;
struct SkGeometry {
  int64_t grid;       // CTAs launched
  int64_t dp_tiles;   // tiles [0, dp_tiles) run whole, tile g + i * grid on CTA g
  int64_t tail_ctas;  // CTAs 0..tail_ctas-1 share the iterations of tiles [dp_tiles, tiles)
  int64_t max_pieces; // most CTAs touching one tail tile (workspace slots per tile)
};
inline SkGeometry sk_geometry(int64_t tiles, int64_t kblocks, int64_t sms) {
  SkGeometry g{};
  const int64_t waves = tiles / sms, rem = tiles % sms;
  g.grid = waves > 0 ? sms : 1;
  g.max_pieces = 1;
  g.tail_ctas = 0;
  if (rem == 0) {
    g.dp_tiles = tiles;
    return g;
  }
  const bool balanced = waves > 0 && (4 * rem <= sms || 2 * rem >= sms);
  g.dp_tiles = balanced ? (waves - 1) * sms : waves * sms;
  const int64_t tail = tiles - g.dp_tiles;
  const int64_t iters = tail * kblocks;
  int64_t c = sms;
  if (!balanced) {
    c = iters / kSkMinIters;
    if (c > tail * kSkMaxPieces) c = tail * kSkMaxPieces;
    if (c > sms) c = sms;
    if (c < 1) c = 1;
  }
  g.tail_ctas = c;
  if (g.grid < c) g.grid = c;
  auto begin = [&](int64_t h) { return h * iters / c; };
  auto cta_of = [&](int64_t x) {
    int64_t h = (x * c) / iters;
    while (h + 1 < c && begin(h + 1) <= x) ++h;
    while (h > 0 && begin(h) > x) --h;
    return h;
  };
  for (int64_t t = 0; t < tail; ++t) {
    const int64_t p = cta_of((t + 1) * kblocks - 1) - cta_of(t * kblocks) + 1;
    if (p > g.max_pieces) g.max_pieces = p;
  }
  return g;
}

}  // namespace rg

#ifdef __CUDACC__
#include <cuda_runtime.h>

#include <functional>
namespace rg {
int timed_sweep(rg_ctx* ctx, const std::vector<int64_t>& order, const rg_sweep_opts& o, cudaStream_t st,
                int64_t* t_ns_out, const std::function<int(int64_t, int*)>& prep,
                const std::function<cudaError_t()>& run);
}
#endif

namespace rg {
int plan_cell(const Plan& P, int64_t M, int64_t N, int64_t K, int64_t* cell);
struct Fp8CtxInfo {
  int32_t* err;
  long long timeout;
  int sms;
  float* ws;
  int64_t ws_bytes;
  int32_t* tickets;
  int64_t max_tickets;
};
int ctx_fp8_info(rg_ctx* ctx, Fp8CtxInfo* out);
void ctx_count_launches(rg_ctx* ctx, int64_t n);
// An FP8 GEMM request of the serving engine (operands as rg_gemm_fp8_ex).
struct Fp8Request {
  int64_t M, N, K;
  const uint8_t* qA;
  int64_t lda;
  const float* sA;
  int64_t lds_a;
  const uint8_t* qB;
  int64_t ldb;
  const float* sB;
  int64_t lds_b;
  float* C;
  int64_t ldc;
};
// The argument checks of rg_gemm_fp8_ex for a request (RG_OK or the status it would return).
int fp8_request_status(const Fp8Request& r);
// Enqueues on `st` the leaves of phase `phase` of the request's FP8 plan cell (without a plan:
// one leaf, RG_FP8_VARIANT(0, 0), phase 0), with the given split-K workspace and tickets;
// *max_phase receives the cell's largest phase.
int fp8_enqueue_phase(rg_ctx* ctx, const rg_plan* plan, const Fp8Request& r, int32_t phase, float* ws,
                      int64_t ws_bytes, int32_t* tickets, int64_t max_tickets, void* stream, int32_t* max_phase);
// The split-K workspace and tickets of a group (for work enqueued on the group's stream).
void group_workspace(rg_group* g, float** ws, int64_t* ws_bytes, int32_t** tickets, int64_t* max_tickets);
// The CUDA device of a context (for threads the library starts).
int ctx_device(const rg_ctx* ctx);
int sweep_surfaces(const rg_grid* grid, int32_t rows, const int64_t* t_ns, double* tflops_out, double* stats_out);
}

struct rg_plan {
  rg::Plan p;
};
