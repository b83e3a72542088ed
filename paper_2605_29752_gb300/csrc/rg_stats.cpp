// Surface statistics (Sec. 2 definitions of achieved TFLOPs and roughness;
// Sec. 8.6 / Table 17 slice and 3D conventions) and the library's error
// plumbing.  Compiled without floating-point contraction so every operation
// is one IEEE double operation in the stated order.
#include <algorithm>
#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "rg_internal.h"

namespace rg {

static thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
void clear_error() { g_last_error.clear(); }

TileShape tile_shape(int tile) {
  static const TileShape shapes[RG_NUM_TILES] = {{128, 64}, {128, 128}, {128, 256}, {256, 64},
                                                 {256, 128}, {256, 256}, {128, 192}, {256, 192}};
  return shapes[tile];
}

// Correctly rounded sum of doubles.  Partials form a non-overlapping expansion
// grown with error-free two-sums (Shewchuk, "Adaptive Precision Floating-Point
// Arithmetic and Fast Robust Geometric Predicates", 1997); the result is the
// expansion rounded to the nearest double, ties to even, with the correction
// for a half-way top partial whose remainder lies beyond it.  This is the
// published scheme of R. Hettinger's "msum" recipe (Python Cookbook, recipe
// 393090), on which Python's math.fsum is built; following the same steps is
// what makes these sums equal the oracle's math.fsum results bit for bit.
class ExactSum {
 public:
  void add(double x) {
    size_t i = 0;
    for (size_t j = 0; j < p_.size(); ++j) {
      double y = p_[j];
      if (std::fabs(x) < std::fabs(y)) std::swap(x, y);
      const double hi = x + y;
      const double lo = y - (hi - x);
      if (lo != 0.0) p_[i++] = lo;
      x = hi;
    }
    p_.resize(i);
    if (x != 0.0) p_.push_back(x);
  }
  double value() const {
    size_t n = p_.size();
    if (n == 0) return 0.0;
    double hi = p_[--n];
    double lo = 0.0;
    while (n > 0) {
      const double x = hi;
      const double y = p_[--n];
      hi = x + y;
      const double yr = hi - x;
      lo = y - yr;
      if (lo != 0.0) break;
    }
    if (n > 0 && ((lo < 0.0 && p_[n - 1] < 0.0) || (lo > 0.0 && p_[n - 1] > 0.0))) {
      const double y = lo * 2.0;
      const double x = hi + y;
      const double yr = x - hi;
      if (y == yr) hi = x;
    }
    return hi;
  }

 private:
  std::vector<double> p_;
};

double exact_mean(const double* v, int64_t n) {
  if (n <= 0) return 0.0;
  ExactSum s;
  for (int64_t i = 0; i < n; ++i) s.add(v[i]);
  return s.value() / static_cast<double>(n);
}

}  // namespace rg

extern "C" const char* rg_version(void) { return "rg 0.1 (sm_103a tcgen05 BF16 NN GEMM, landscape smoothing)"; }

extern "C" const char* rg_last_error(void) { return rg::g_last_error.c_str(); }

extern "C" const char* rg_strerror(int status) {
  switch (status) {
    case RG_OK: return "ok";
    case RG_ERR_INVALID: return "invalid argument";
    case RG_ERR_ALIGN: return "pointer or leading dimension violates TMA alignment";
    case RG_ERR_SHAPE: return "shape outside the plan grid or workspace capacity";
    case RG_ERR_OOM: return "out of memory";
    case RG_ERR_CUDA: return "CUDA error";
    case RG_ERR_TIMEOUT: return "a bounded device wait expired";
    case RG_ERR_PLAN_MISMATCH: return "plan file does not match";
    case RG_ERR_ADMISSION: return "request exceeds the serving memory budget";
    case RG_ERR_NO_DEVICE: return "no usable sm_103 device";
    default: return "unknown status";
  }
}

extern "C" void rg_sweep_opts_default(rg_sweep_opts* o) {
  if (!o) return;
  o->reps = 5;
  o->warmup = 1;
  o->global_warmup = 5;
  o->shuffle = 1;
  o->seed = 0;
  o->spin_ns = 4000;
  o->prune_splits = 1;
  o->shard_index = 0;
  o->shard_count = 1;
  o->reserved = 0;
}

extern "C" int rg_variant_desc(int32_t v, int32_t out[6]) {
  rg::clear_error();
  if (!out || v < 0 || v >= RG_NUM_VARIANTS) return rg::fail(RG_ERR_INVALID, "rg_variant_desc: variant id out of range");
  const int tile = rg::variant_tile(v);
  const rg::TileShape ts = rg::tile_shape(tile);
  out[0] = tile;
  out[1] = rg::variant_split(v);
  out[2] = rg::variant_streamk(v) ? 1 : 0;
  out[3] = rg::variant_2sm(v) ? 1 : 0;
  out[4] = ts.bm;
  out[5] = ts.bn;
  return RG_OK;
}

extern "C" int rg_streamk_geometry(int64_t tiles, int64_t kblocks, int64_t units, int64_t out[4]) {
  rg::clear_error();
  if (!out || tiles <= 0 || kblocks <= 0 || units <= 0 || tiles > (1LL << 30) || kblocks > (1LL << 24))
    return rg::fail(RG_ERR_INVALID, "rg_streamk_geometry: sizes");
  const rg::SkGeometry g = rg::sk_geometry(tiles, kblocks, units);
  out[0] = g.grid;
  out[1] = g.dp_tiles;
  out[2] = g.tail_ctas;
  out[3] = g.max_pieces;
  return RG_OK;
}

extern "C" int rg_surface_stats(const rg_grid* grid, const int64_t* t_ns, double* tflops_out,
                                double rough_out[5], double* mean_out) {
  rg::clear_error();
  if (!grid || !t_ns) return rg::fail(RG_ERR_INVALID, "rg_surface_stats: null argument");
  if (!rg::grid_valid(*grid)) return rg::fail(RG_ERR_INVALID, "rg_surface_stats: invalid grid");
  const int64_t nm = grid->m.count, nn = grid->n.count, nk = grid->k.count;
  const int64_t cells = nm * nn * nk;
  std::vector<double> S(cells);
  for (int64_t a = 0; a < nm; ++a)
    for (int64_t b = 0; b < nn; ++b)
      for (int64_t c = 0; c < nk; ++c) {
        const int64_t i = (a * nn + b) * nk + c;
        if (t_ns[i] <= 0) return rg::fail(RG_ERR_INVALID, "rg_surface_stats: times must be positive");
        const double M = static_cast<double>(rg::axis_value(grid->m, a));
        const double N = static_cast<double>(rg::axis_value(grid->n, b));
        const double K = static_cast<double>(rg::axis_value(grid->k, c));
        const double flops = 2.0 * M * N * K;
        const double den = static_cast<double>(t_ns[i]) * 1e3;
        S[i] = flops / den;
      }
  if (tflops_out)
    for (int64_t i = 0; i < cells; ++i) tflops_out[i] = S[i];
  if (mean_out) *mean_out = rg::exact_mean(S.data(), cells);
  if (rough_out) {
    auto at = [&](int64_t a, int64_t b, int64_t c) { return S[(a * nn + b) * nk + c]; };
    rg::ExactSum sm, sn, sk, ss;
    for (int64_t a = 0; a + 1 < nm; ++a)
      for (int64_t b = 0; b < nn; ++b)
        for (int64_t c = 0; c < nk; ++c) sm.add(std::fabs(at(a + 1, b, c) - at(a, b, c)));
    for (int64_t a = 0; a < nm; ++a)
      for (int64_t b = 0; b + 1 < nn; ++b)
        for (int64_t c = 0; c < nk; ++c) sn.add(std::fabs(at(a, b + 1, c) - at(a, b, c)));
    for (int64_t a = 0; a < nm; ++a)
      for (int64_t b = 0; b < nn; ++b)
        for (int64_t c = 0; c + 1 < nk; ++c) sk.add(std::fabs(at(a, b, c + 1) - at(a, b, c)));
    for (int64_t a = 0; a < nm; ++a)
      for (int64_t b = 0; b + 1 < nn; ++b) ss.add(std::fabs(at(a, b + 1, nk - 1) - at(a, b, nk - 1)));
    const double pm = static_cast<double>((nm - 1) * nn * nk);
    const double pn = static_cast<double>(nm * (nn - 1) * nk);
    const double pk = static_cast<double>(nm * nn * (nk - 1));
    const double ps = static_cast<double>(nm * (nn - 1));
    const double rM = nm > 1 ? sm.value() / pm : 0.0;
    const double rN = nn > 1 ? sn.value() / pn : 0.0;
    const double rK = nk > 1 ? sk.value() / pk : 0.0;
    rough_out[0] = rM;
    rough_out[1] = rN;
    rough_out[2] = rK;
    rough_out[3] = (rM + rN + rK) / 3.0;
    rough_out[4] = nn > 1 ? ss.value() / ps : 0.0;
  }
  return RG_OK;
}

namespace rg {
// The sweep's surfaces: per timed row, rg_surface_stats' TFLOP/s surface and
// {R_M, R_N, R_K, R_3D, R_N on the largest-K slice, mean}.  A row with cells the
// sweep did not measure (RG_T_UNMEASURED) gets TFLOP/s 0 there, the same
// expression as rg_surface_stats elsewhere, and NaN statistics: a surface with
// holes has no roughness.
int sweep_surfaces(const rg_grid* grid, int32_t rows, const int64_t* t_ns, double* tflops_out, double* stats_out) {
  if (!tflops_out && !stats_out) return RG_OK;
  const int64_t cells = cells_of(*grid);
  const int64_t nn = grid->n.count, nk = grid->k.count;
  for (int32_t v = 0; v < rows; ++v) {
    const int64_t* t = t_ns + static_cast<int64_t>(v) * cells;
    double* tf = tflops_out ? tflops_out + static_cast<int64_t>(v) * cells : nullptr;
    double* st = stats_out ? stats_out + 6 * static_cast<int64_t>(v) : nullptr;
    bool full = true;
    for (int64_t i = 0; i < cells && full; ++i) full = t[i] != RG_T_UNMEASURED && t[i] != RG_T_OTHER_SHARD;
    if (full) {
      double rough[5], mean = 0.0;
      const int rc = rg_surface_stats(grid, t, tf, rough, &mean);
      if (rc != RG_OK) return rc;
      if (st) {
        for (int j = 0; j < 5; ++j) st[j] = rough[j];
        st[5] = mean;
      }
      continue;
    }
    if (tf)
      for (int64_t i = 0; i < cells; ++i) {
        if (t[i] == RG_T_UNMEASURED || t[i] == RG_T_OTHER_SHARD) {
          tf[i] = 0.0;
          continue;
        }
        const double M = static_cast<double>(axis_value(grid->m, i / (nn * nk)));
        const double N = static_cast<double>(axis_value(grid->n, (i / nk) % nn));
        const double K = static_cast<double>(axis_value(grid->k, i % nk));
        tf[i] = (2.0 * M * N * K) / (static_cast<double>(t[i]) * 1e3);
      }
    if (st)
      for (int j = 0; j < 6; ++j) st[j] = std::numeric_limits<double>::quiet_NaN();
  }
  return RG_OK;
}
}  // namespace rg

// ---------------------------------------------------------------- first-principles landscapes
namespace {
int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}
int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Channel utilisation of one tensor under the interleave model of Sec. 9.2.
double eta_channel(int64_t L, int64_t e, int64_t channels, int64_t interleave) {
  const int64_t w = std::min(channels, e);
  const int64_t s = ((L * e) / interleave) % channels;
  const int64_t g = gcd64(s, channels);
  const double reach = static_cast<double>(w * channels) / static_cast<double>(g);
  return std::min(static_cast<double>(channels), reach) / static_cast<double>(channels);
}
}  // namespace

extern "C" int rg_landscape(const rg_grid* grid, int32_t mode, double p_tflops, int32_t c_units, double bw_gbs,
                            int32_t n_tiles, const int32_t* tiles, int32_t channels, int32_t interleave,
                            double* out) {
  rg::clear_error();
  if (!grid || !tiles || !out || n_tiles <= 0 || c_units <= 0 || !(p_tflops > 0.0))
    return rg::fail(RG_ERR_INVALID, "rg_landscape: bad argument");
  if (!rg::grid_valid(*grid)) return rg::fail(RG_ERR_INVALID, "rg_landscape: invalid grid");
  if (mode != RG_LANDSCAPE_IDEAL && mode != RG_LANDSCAPE_OPTIMAL) return rg::fail(RG_ERR_INVALID, "rg_landscape: mode");
  if (mode == RG_LANDSCAPE_OPTIMAL && !(bw_gbs > 0.0)) return rg::fail(RG_ERR_INVALID, "rg_landscape: bandwidth");
  if (channels < 0 || (channels > 0 && interleave <= 0)) return rg::fail(RG_ERR_INVALID, "rg_landscape: channels");
  for (int t = 0; t < n_tiles; ++t)
    if (tiles[2 * t] <= 0 || tiles[2 * t + 1] <= 0) return rg::fail(RG_ERR_INVALID, "rg_landscape: tile");
  const int64_t nm = grid->m.count, nn = grid->n.count, nk = grid->k.count;
  const double C = static_cast<double>(c_units);
  for (int64_t a = 0; a < nm; ++a)
    for (int64_t b = 0; b < nn; ++b)
      for (int64_t c = 0; c < nk; ++c) {
        const int64_t Mi = rg::axis_value(grid->m, a), Ni = rg::axis_value(grid->n, b), Ki = rg::axis_value(grid->k, c);
        const double M = static_cast<double>(Mi), N = static_cast<double>(Ni), K = static_cast<double>(Ki);
        double v;
        if (mode == RG_LANDSCAPE_IDEAL) {
          const int64_t W = ceil_div(Mi, tiles[0]) * ceil_div(Ni, tiles[1]);
          v = p_tflops * std::min(1.0, static_cast<double>(W) / C);
        } else {
          const double fl = 2.0 * M * N * K;
          double eA = 1.0, eB = 1.0, eD = 1.0;
          if (channels > 0) {
            eA = eta_channel(Ki, 2, channels, interleave);
            eB = eta_channel(Ni, 2, channels, interleave);
            eD = eta_channel(Ni, 4, channels, interleave);
          }
          const double bw = bw_gbs * 1e9;
          const double t_mem = 2.0 * M * K / (bw * eA) + 2.0 * K * N / (bw * eB) + 4.0 * M * N / (bw * eD);
          double best = INFINITY;
          for (int t = 0; t < n_tiles; ++t) {
            const int64_t W = ceil_div(Mi, tiles[2 * t]) * ceil_div(Ni, tiles[2 * t + 1]);
            const double eta = static_cast<double>(W) / (static_cast<double>(ceil_div(W, c_units)) * C);
            const double t_comp = fl / (p_tflops * 1e12 * eta);
            best = std::min(best, std::max(t_comp, t_mem));
          }
          v = fl / best / 1e12;
        }
        out[(a * nn + b) * nk + c] = v;
      }
  return RG_OK;
}

extern "C" int rg_kol(double mean_a, double mean_o, double r_a, double r_o, double out[2], int32_t bands[3]) {
  if (!out || !bands || !(mean_o > 0.0) || !(r_o > 0.0)) return rg::fail(RG_ERR_INVALID, "rg_kol: bad argument");
  const double tau = mean_a / mean_o;
  const double rho = r_a / r_o;
  const int32_t T = tau < 0.50 ? 0 : tau < 0.75 ? 1 : tau < 0.95 ? 2 : 3;
  const int32_t S = rho > 3.0 ? 0 : rho > 2.0 ? 1 : rho > 1.25 ? 2 : 3;
  out[0] = tau;
  out[1] = rho;
  bands[0] = T;
  bands[1] = S;
  bands[2] = std::min(T, S);
  return RG_OK;
}

// Four-surface decomposition (Sec. 4): the compute surface is the useful-flop
// time at peak, the memory surface the measured memory twin, the overhead
// surface what the GEMM takes beyond the larger of the two; a cell is
// compute-bound when even a zero-waste kernel would be limited by compute
// (t_compute > t_memory, Table 3).
extern "C" int rg_decompose(const rg_grid* grid, const int64_t* t_gemm_ns, const int64_t* t_mem_ns, double p_tflops,
                            double* compute_ns_out, double* overhead_ns_out, double stats_out[4]) {
  rg::clear_error();
  if (!grid || !t_gemm_ns || !t_mem_ns) return rg::fail(RG_ERR_INVALID, "rg_decompose: null argument");
  if (!rg::grid_valid(*grid)) return rg::fail(RG_ERR_INVALID, "rg_decompose: invalid grid");
  if (!(p_tflops > 0.0)) return rg::fail(RG_ERR_INVALID, "rg_decompose: peak must be positive");
  const int64_t nm = grid->m.count, nn = grid->n.count, nk = grid->k.count;
  const int64_t cells = nm * nn * nk;
  for (int64_t i = 0; i < cells; ++i)
    if (t_gemm_ns[i] <= 0 || t_mem_ns[i] <= 0) return rg::fail(RG_ERR_INVALID, "rg_decompose: times must be positive");
  int64_t compute_bound = 0;
  rg::ExactSum share_o, share_m, sum_o, sum_g;
  for (int64_t a = 0; a < nm; ++a)
    for (int64_t b = 0; b < nn; ++b)
      for (int64_t c = 0; c < nk; ++c) {
        const int64_t i = (a * nn + b) * nk + c;
        const double M = static_cast<double>(rg::axis_value(grid->m, a));
        const double N = static_cast<double>(rg::axis_value(grid->n, b));
        const double K = static_cast<double>(rg::axis_value(grid->k, c));
        const double flops = 2.0 * M * N * K;
        const double tc = flops / (p_tflops * 1e3);
        const double tg = static_cast<double>(t_gemm_ns[i]);
        const double tm = static_cast<double>(t_mem_ns[i]);
        const double to = tg - std::max(tc, tm);
        if (compute_ns_out) compute_ns_out[i] = tc;
        if (overhead_ns_out) overhead_ns_out[i] = to;
        if (tc > tm) ++compute_bound;
        share_o.add(to / tg);
        share_m.add(tm / tg);
        sum_o.add(to);
        sum_g.add(tg);
      }
  if (stats_out) {
    stats_out[0] = static_cast<double>(compute_bound) / static_cast<double>(cells);
    stats_out[1] = share_o.value() / static_cast<double>(cells);
    stats_out[2] = sum_o.value() / sum_g.value();
    stats_out[3] = share_m.value() / static_cast<double>(cells);
  }
  return RG_OK;
}
