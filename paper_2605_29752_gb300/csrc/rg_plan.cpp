// Plan table: dynamic best-of selection (Sec. 6.4) and the padding-and-splitting
// dynamic programme T0 -> T1 -> T2 (Sec. 7.1), built once offline and used at
// run time as an O(1) lookup.
//
// Readings where the paper is silent (each a total order, so the tables are
// unique and bit-exact across implementations):
//   - times are integer nanoseconds;
//   - best-of ties go to the lowest variant id;
//   - T1's pad target is the cell c' >= c minimising (T0*, M'N'K', M', N', K');
//   - T2 takes a split only when strictly faster, candidates ranked keep < split M
//     < split N < split K (the order of the recurrence's terms), then by the
//     second piece's size q, smallest first;
//   - piece 1 of a split is the first p - q steps, piece 2 the last q steps; a K
//     split's piece 2 accumulates (beta = 1) after piece 1.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <tuple>

#include "rg_internal.h"

namespace {

using rg::Plan;

struct Key {  // (T0*, volume, M, N, K), compared lexicographically
  int64_t t, vol, m, n, k;
  bool operator<(const Key& o) const {
    return std::tie(t, vol, m, n, k) < std::tie(o.t, o.vol, o.m, o.n, o.k);
  }
};

struct Dims {
  int64_t nm, nn, nk;
  int64_t idx(int64_t a, int64_t b, int64_t c) const { return (a * nn + b) * nk + c; }
};

// Expand one cell into leaves; returns the dependency depth (number of phases).
int64_t expand(const Plan& P, const Dims& d, int64_t a, int64_t b, int64_t c, int64_t m0, int64_t n0,
               int64_t k0, int32_t beta, int32_t phase0, std::vector<rg_leaf>& out) {
  const rg_grid& g = P.grid;
  const int64_t i = d.idx(a, b, c);
  const int32_t act = P.action[i];
  const int64_t q = P.q[i];
  if (act == 0) {
    const int32_t ta = P.target3[3 * i], tb = P.target3[3 * i + 1], tc = P.target3[3 * i + 2];
    rg_leaf L{};
    L.variant = P.vstar[d.idx(ta, tb, tc)];
    L.beta = beta;
    L.phase = phase0;
    L.m0 = m0; L.n0 = n0; L.k0 = k0;
    L.m = rg::axis_value(g.m, a); L.n = rg::axis_value(g.n, b); L.k = rg::axis_value(g.k, c);
    L.pm = rg::axis_value(g.m, ta); L.pn = rg::axis_value(g.n, tb); L.pk = rg::axis_value(g.k, tc);
    out.push_back(L);
    return 1;
  }
  if (act == 1) {
    const int64_t p = a + 1;
    const int64_t d1 = expand(P, d, p - q - 1, b, c, m0, n0, k0, beta, phase0, out);
    const int64_t d2 = expand(P, d, q - 1, b, c, m0 + (p - q) * g.m.step, n0, k0, beta, phase0, out);
    return std::max(d1, d2);
  }
  if (act == 2) {
    const int64_t p = b + 1;
    const int64_t d1 = expand(P, d, a, p - q - 1, c, m0, n0, k0, beta, phase0, out);
    const int64_t d2 = expand(P, d, a, q - 1, c, m0, n0 + (p - q) * g.n.step, k0, beta, phase0, out);
    return std::max(d1, d2);
  }
  const int64_t p = c + 1;  // split K: piece 2 runs after every leaf of piece 1
  const int64_t d1 = expand(P, d, a, b, p - q - 1, m0, n0, k0, beta, phase0, out);
  const int64_t d2 =
      expand(P, d, a, b, q - 1, m0, n0, k0 + (p - q) * g.k.step, 1, static_cast<int32_t>(phase0 + d1), out);
  return d1 + d2;
}

uint64_t fnv1a(const uint8_t* p, size_t n, uint64_t h = 1469598103934665603ull) {
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

extern "C" int rg_plan_build(const rg_grid* grid, const int64_t* T0_ns, int32_t n_variants,
                             const int32_t* variant_ids, rg_plan** out) {
  return rg_plan_build_ex(grid, T0_ns, n_variants, variant_ids, 0, out);
}

extern "C" int rg_plan_build_ex(const rg_grid* grid, const int64_t* T0_ns, int32_t n_variants,
                                const int32_t* variant_ids, int32_t flags, rg_plan** out) {
  rg::clear_error();
  if (!grid || !T0_ns || !variant_ids || !out || n_variants <= 0)
    return rg::fail(RG_ERR_INVALID, "rg_plan_build: null argument or n_variants <= 0");
  if (flags & ~RG_PLAN_PAD_ONLY) return rg::fail(RG_ERR_INVALID, "rg_plan_build: unknown flags");
  if (!rg::grid_valid(*grid)) return rg::fail(RG_ERR_INVALID, "rg_plan_build: invalid grid");
  if (!(flags & RG_PLAN_PAD_ONLY) &&
      (grid->m.start != grid->m.step || grid->n.start != grid->n.step || grid->k.start != grid->k.step))
    return rg::fail(RG_ERR_INVALID, "rg_plan_build: splitting needs start == step on every axis");
  for (int v = 0; v < n_variants; ++v) {
    if (!rg::variant_valid(variant_ids[v])) return rg::fail(RG_ERR_INVALID, "rg_plan_build: variant id out of range");
    if (v > 0 && variant_ids[v] <= variant_ids[v - 1])
      return rg::fail(RG_ERR_INVALID, "rg_plan_build: variant ids must be strictly increasing");
    if (rg::variant_fp8(variant_ids[v]) != rg::variant_fp8(variant_ids[0]))
      return rg::fail(RG_ERR_INVALID, "rg_plan_build: BF16 and FP8 variant ids cannot share a plan");
  }
  const Dims d{grid->m.count, grid->n.count, grid->k.count};
  const int64_t cells = rg::cells_of(*grid);
  for (int64_t i = 0; i < cells * n_variants; ++i)
    if (T0_ns[i] <= 0) return rg::fail(RG_ERR_INVALID, "rg_plan_build: times must be positive");

  auto* plan = new (std::nothrow) rg_plan();
  if (!plan) return rg::fail(RG_ERR_OOM, "rg_plan_build: out of host memory");
  Plan& P = plan->p;
  P.grid = *grid;
  P.variant_ids.assign(variant_ids, variant_ids + n_variants);
  P.T0s.resize(cells);
  P.vstar.resize(cells);
  P.T1.resize(cells);
  P.target3.resize(3 * cells);
  P.T2.resize(cells);
  P.action.resize(cells);
  P.q.resize(cells);

  // best-of: min over variants, lowest id on ties (Sec. 6.4)
  std::vector<int32_t> vrow(cells, 0);
  for (int64_t i = 0; i < cells; ++i) {
    int64_t best = T0_ns[i];
    int32_t arg = 0;
    for (int v = 1; v < n_variants; ++v) {
      const int64_t t = T0_ns[static_cast<int64_t>(v) * cells + i];
      if (t < best) { best = t; arg = v; }
    }
    P.T0s[i] = best;
    vrow[i] = arg;
    P.vstar[i] = variant_ids[arg];
  }

  // T1: sweep from the last cell to the first, min over the 2x2x2 neighbourhood
  std::vector<Key> key(cells);
  for (int64_t a = d.nm - 1; a >= 0; --a)
    for (int64_t b = d.nn - 1; b >= 0; --b)
      for (int64_t c = d.nk - 1; c >= 0; --c) {
        const int64_t i = d.idx(a, b, c);
        const int64_t M = rg::axis_value(grid->m, a), N = rg::axis_value(grid->n, b),
                      K = rg::axis_value(grid->k, c);
        Key cur{P.T0s[i], M * N * K, M, N, K};
        int32_t ta = static_cast<int32_t>(a), tb = static_cast<int32_t>(b), tc = static_cast<int32_t>(c);
        for (int di = 0; di <= 1; ++di)
          for (int dj = 0; dj <= 1; ++dj)
            for (int dl = 0; dl <= 1; ++dl) {
              if (!di && !dj && !dl) continue;
              const int64_t na = a + di, nb = b + dj, nc = c + dl;
              if (na >= d.nm || nb >= d.nn || nc >= d.nk) continue;
              const int64_t j = d.idx(na, nb, nc);
              if (key[j] < cur) {
                cur = key[j];
                ta = P.target3[3 * j]; tb = P.target3[3 * j + 1]; tc = P.target3[3 * j + 2];
              }
            }
        key[i] = cur;
        P.T1[i] = cur.t;
        P.target3[3 * i] = ta; P.target3[3 * i + 1] = tb; P.target3[3 * i + 2] = tc;
      }

  // T2: sweep from the first cell to the last, starting from T1
  P.T2 = P.T1;
  const int64_t split_rows = (flags & RG_PLAN_PAD_ONLY) ? 0 : d.nm;
  for (int64_t a = 0; a < split_rows; ++a)
    for (int64_t b = 0; b < d.nn; ++b)
      for (int64_t c = 0; c < d.nk; ++c) {
        const int64_t i = d.idx(a, b, c);
        int64_t best = P.T2[i];
        int32_t act = 0, qq = 0;
        int64_t p = a + 1;
        for (int64_t q = 1; q < p; ++q) {
          const int64_t v = P.T2[d.idx(p - q - 1, b, c)] + P.T2[d.idx(q - 1, b, c)];
          if (v < best) { best = v; act = 1; qq = static_cast<int32_t>(q); }
        }
        p = b + 1;
        for (int64_t q = 1; q < p; ++q) {
          const int64_t v = P.T2[d.idx(a, p - q - 1, c)] + P.T2[d.idx(a, q - 1, c)];
          if (v < best) { best = v; act = 2; qq = static_cast<int32_t>(q); }
        }
        p = c + 1;
        for (int64_t q = 1; q < p; ++q) {
          const int64_t v = P.T2[d.idx(a, b, p - q - 1)] + P.T2[d.idx(a, b, q - 1)];
          if (v < best) { best = v; act = 3; qq = static_cast<int32_t>(q); }
        }
        P.T2[i] = best;
        P.action[i] = act;
        P.q[i] = qq;
      }

  // flatten every cell's leaves
  P.leaf_off.assign(cells + 1, 0);
  P.leaves.reserve(cells * 2);
  for (int64_t a = 0; a < d.nm; ++a)
    for (int64_t b = 0; b < d.nn; ++b)
      for (int64_t c = 0; c < d.nk; ++c) {
        const int64_t i = d.idx(a, b, c);
        P.leaf_off[i] = static_cast<int64_t>(P.leaves.size());
        expand(P, d, a, b, c, 0, 0, 0, 0, 0, P.leaves);
      }
  P.leaf_off[cells] = static_cast<int64_t>(P.leaves.size());
  *out = plan;
  return RG_OK;
}

extern "C" void rg_plan_free(rg_plan* plan) { delete plan; }

extern "C" int rg_plan_grid(const rg_plan* plan, rg_grid* out) {
  if (!plan || !out) return rg::fail(RG_ERR_INVALID, "rg_plan_grid: null argument");
  *out = plan->p.grid;
  return RG_OK;
}

extern "C" int rg_plan_tables(const rg_plan* plan, int64_t* T0s, int32_t* vstar, int64_t* T1,
                              int32_t* target3, int64_t* T2, int32_t* action, int32_t* q) {
  if (!plan) return rg::fail(RG_ERR_INVALID, "rg_plan_tables: null plan");
  const Plan& P = plan->p;
  const size_t n = P.T0s.size();
  if (T0s) std::memcpy(T0s, P.T0s.data(), n * sizeof(int64_t));
  if (vstar) std::memcpy(vstar, P.vstar.data(), n * sizeof(int32_t));
  if (T1) std::memcpy(T1, P.T1.data(), n * sizeof(int64_t));
  if (target3) std::memcpy(target3, P.target3.data(), 3 * n * sizeof(int32_t));
  if (T2) std::memcpy(T2, P.T2.data(), n * sizeof(int64_t));
  if (action) std::memcpy(action, P.action.data(), n * sizeof(int32_t));
  if (q) std::memcpy(q, P.q.data(), n * sizeof(int32_t));
  return RG_OK;
}

namespace rg {
// Cell index covering a size on one axis (rounded up to the grid), or -1.
static int64_t cover_index(const rg_axis& ax, int64_t v) {
  if (v <= ax.start) return 0;
  const int64_t i = (v - ax.start + ax.step - 1) / ax.step;
  return i < ax.count ? i : -1;
}
int plan_cell(const Plan& P, int64_t M, int64_t N, int64_t K, int64_t* cell) {
  const int64_t a = cover_index(P.grid.m, M), b = cover_index(P.grid.n, N), c = cover_index(P.grid.k, K);
  if (a < 0 || b < 0 || c < 0) return RG_ERR_SHAPE;
  *cell = (a * P.grid.n.count + b) * P.grid.k.count + c;
  return RG_OK;
}
}  // namespace rg

extern "C" int rg_plan_lookup(const rg_plan* plan, int64_t M, int64_t N, int64_t K, const rg_leaf** leaves,
                              int32_t* n_leaves, int64_t* t2_ns) {
  if (!plan || !leaves || !n_leaves) return rg::fail(RG_ERR_INVALID, "rg_plan_lookup: null argument");
  if (M <= 0 || N <= 0 || K <= 0) return rg::fail(RG_ERR_INVALID, "rg_plan_lookup: sizes must be positive");
  int64_t cell = 0;
  if (rg::plan_cell(plan->p, M, N, K, &cell) != RG_OK)
    return rg::fail(RG_ERR_SHAPE, "rg_plan_lookup: shape beyond the plan grid");
  const Plan& P = plan->p;
  *leaves = P.leaves.data() + P.leaf_off[cell];
  *n_leaves = static_cast<int32_t>(P.leaf_off[cell + 1] - P.leaf_off[cell]);
  if (t2_ns) *t2_ns = P.T2[cell];
  return RG_OK;
}

// ---------------------------------------------------------------- file format
namespace {
const char kMagic[8] = {'R', 'G', 'P', 'L', 'A', 'N', '0', '1'};
// 2: the variant numbering without the multicast pairs, with cta_group::2 stream-K and FP8 ids;
// 3: seven tiles (128 x 192 added), which renumbers every id from 24 on;
// 4: eight tiles and three pair tiles (256 x 192 added), which renumbers every id from 28 on
const uint32_t kPlanFileVersion = 4;

template <class T>
void put(std::vector<uint8_t>& b, const T* p, size_t n) {
  const uint8_t* s = reinterpret_cast<const uint8_t*>(p);
  b.insert(b.end(), s, s + n * sizeof(T));
}
template <class T>
bool get(const std::vector<uint8_t>& b, size_t& off, T* p, size_t n) {
  if (off + n * sizeof(T) > b.size()) return false;
  std::memcpy(p, b.data() + off, n * sizeof(T));
  off += n * sizeof(T);
  return true;
}
}  // namespace

namespace rg {
// Device identity recorded in plan files: name and SM count of a context (empty if none).
void ctx_identity(const rg_ctx* ctx, char name[64], int32_t* sms);
}

extern "C" int rg_plan_save(const rg_plan* plan, const rg_ctx* ctx, const char* path) {
  if (!plan || !path) return rg::fail(RG_ERR_INVALID, "rg_plan_save: null argument");
  const Plan& P = plan->p;
  std::vector<uint8_t> body;
  char name[64] = {0};
  int32_t sms = 0;
  rg::ctx_identity(ctx, name, &sms);
  put(body, name, 64);
  put(body, &sms, 1);
  put(body, &P.grid, 1);
  const int64_t nv = static_cast<int64_t>(P.variant_ids.size());
  const int64_t cells = static_cast<int64_t>(P.T0s.size());
  const int64_t nl = static_cast<int64_t>(P.leaves.size());
  put(body, &nv, 1);
  put(body, &cells, 1);
  put(body, &nl, 1);
  put(body, P.variant_ids.data(), nv);
  put(body, P.T0s.data(), cells);
  put(body, P.vstar.data(), cells);
  put(body, P.T1.data(), cells);
  put(body, P.target3.data(), 3 * cells);
  put(body, P.T2.data(), cells);
  put(body, P.action.data(), cells);
  put(body, P.q.data(), cells);
  put(body, P.leaf_off.data(), cells + 1);
  put(body, P.leaves.data(), nl);
  const uint64_t sum = fnv1a(body.data(), body.size());
  FILE* f = std::fopen(path, "wb");
  if (!f) return rg::fail(RG_ERR_INVALID, std::string("rg_plan_save: cannot open ") + path);
  const uint32_t version = kPlanFileVersion;
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&version, 4, 1, f) == 1 &&
            std::fwrite(&sum, 8, 1, f) == 1 && std::fwrite(body.data(), 1, body.size(), f) == body.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? RG_OK : rg::fail(RG_ERR_INVALID, "rg_plan_save: write failed");
}

extern "C" int rg_plan_load(const char* path, const rg_ctx* ctx, rg_plan** out) {
  if (!path || !out) return rg::fail(RG_ERR_INVALID, "rg_plan_load: null argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return rg::fail(RG_ERR_INVALID, std::string("rg_plan_load: cannot open ") + path);
  char magic[8];
  uint32_t version = 0;
  uint64_t sum = 0;
  std::vector<uint8_t> body;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::fread(&version, 4, 1, f) == 1 && std::fread(&sum, 8, 1, f) == 1;
  if (ok) {
    uint8_t buf[1 << 16];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) body.insert(body.end(), buf, buf + n);
  }
  std::fclose(f);
  if (!ok || std::memcmp(magic, kMagic, 8) != 0 || version != kPlanFileVersion)
    return rg::fail(RG_ERR_PLAN_MISMATCH, "rg_plan_load: not a plan file of this version");
  if (fnv1a(body.data(), body.size()) != sum)
    return rg::fail(RG_ERR_PLAN_MISMATCH, "rg_plan_load: checksum mismatch");
  size_t off = 0;
  char name[64];
  int32_t sms = 0;
  auto* plan = new (std::nothrow) rg_plan();
  if (!plan) return rg::fail(RG_ERR_OOM, "rg_plan_load: out of host memory");
  Plan& P = plan->p;
  int64_t nv = 0, cells = 0, nl = 0;
  ok = get(body, off, name, 64) && get(body, off, &sms, 1) && get(body, off, &P.grid, 1) &&
       get(body, off, &nv, 1) && get(body, off, &cells, 1) && get(body, off, &nl, 1) && nv > 0 &&
       nv <= RG_NUM_VARIANTS + RG_FP8_NUM_VARIANTS && cells == rg::cells_of(P.grid) && nl >= cells;
  if (ok) {
    P.variant_ids.resize(nv);
    P.T0s.resize(cells); P.vstar.resize(cells); P.T1.resize(cells); P.target3.resize(3 * cells);
    P.T2.resize(cells); P.action.resize(cells); P.q.resize(cells); P.leaf_off.resize(cells + 1);
    P.leaves.resize(nl);
    ok = get(body, off, P.variant_ids.data(), nv) && get(body, off, P.T0s.data(), cells) &&
         get(body, off, P.vstar.data(), cells) && get(body, off, P.T1.data(), cells) &&
         get(body, off, P.target3.data(), 3 * cells) && get(body, off, P.T2.data(), cells) &&
         get(body, off, P.action.data(), cells) && get(body, off, P.q.data(), cells) &&
         get(body, off, P.leaf_off.data(), cells + 1) && get(body, off, P.leaves.data(), nl) &&
         off == body.size();
  }
  if (!ok) {
    delete plan;
    return rg::fail(RG_ERR_PLAN_MISMATCH, "rg_plan_load: malformed body");
  }
  if (ctx) {
    char cname[64] = {0};
    int32_t csms = 0;
    rg::ctx_identity(ctx, cname, &csms);
    if (std::strncmp(cname, name, 64) != 0 || csms != sms) {
      delete plan;
      return rg::fail(RG_ERR_PLAN_MISMATCH, std::string("rg_plan_load: plan was built on '") + name +
                                                "', this device is '" + cname + "'");
    }
  }
  *out = plan;
  return RG_OK;
}
