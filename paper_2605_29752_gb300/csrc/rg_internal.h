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
inline int variant_tile(int v) { return v / RG_NUM_SPLITS; }
inline int variant_split(int v) { return 1 << (v % RG_NUM_SPLITS); }

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

struct rg_plan {
  rg::Plan p;
};
