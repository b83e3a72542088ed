// Serving: a request loop with continuous batching on top of the grouped GEMM.
//
// rg_serve runs one trace of GEMM requests, each with an arrival time, on the
// calling thread:
//   - admission: requests are admitted in arrival order once they have arrived
//     and their operand bytes (2MK + 2KN + 4MN) fit under the HBM budget next to
//     the requests already admitted and not yet finished; a request that can
//     never fit is rejected (RG_ERR_ADMISSION); an admitted request whose C is
//     NULL gets its output from an arena of budget bytes owned by the run;
//   - routing: each request goes through the plan's O(1) lookup; a single-leaf
//     cell contributes its autotuned tile shape and its padded launch extents (the
//     DP's padding), a split cell runs as-is on the default tile (its pieces would
//     need ordered launches);
//   - batching: whenever an in-flight slot is free and admitted requests are
//     waiting, up to max_batch of them become one grouped launch per tile shape
//     among them (a CUDA graph
//     replay) on that slot's stream; up to max_inflight launches are on the GPU at
//     once, so a batch admitted while another runs overlaps it on the device;
//   - completion: slots are polled with events; a finished batch releases its
//     requests' budget and arena space, so waiting requests are admitted.
// Latency = completion observed on the host - arrival, both on the host's
// steady clock measured from the start of the run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "rg_internal.h"

namespace {

struct Arena {  // first-fit allocator over one device allocation, 256-byte granules
  unsigned char* base = nullptr;
  int64_t size = 0;
  std::map<int64_t, int64_t> free_;  // offset -> length
  bool init(int64_t bytes) {
    if (bytes <= 0) return true;
    if (cudaMalloc(&base, static_cast<size_t>(bytes)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    size = bytes;
    free_[0] = bytes;
    return true;
  }
  void release_all() {
    if (base) cudaFree(base);
    base = nullptr;
  }
  int64_t alloc(int64_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const int64_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        return off;
      }
    }
    return -1;
  }
  void free(int64_t off, int64_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

int64_t request_bytes(const rg_serve_request& r) { return 2 * r.M * r.K + 2 * r.K * r.N + 4 * r.M * r.N; }

// The per-request checks of rg_gemm (sizes, leading dimensions, TMA alignment),
// made at admission so that one malformed request is rejected alone instead of
// failing the grouped launch it would join.
int request_status(const rg_serve_request& r) {
  if (r.M <= 0 || r.N <= 0 || r.K <= 0 || !r.A || !r.B) return RG_ERR_INVALID;
  if (r.lda < r.K || r.ldb < r.N || (r.C && r.ldc < r.N)) return RG_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(r.A) & 15) || (reinterpret_cast<uintptr_t>(r.B) & 15) || (r.lda % 8) ||
      (r.ldb % 8))
    return RG_ERR_ALIGN;
  if (r.C && ((reinterpret_cast<uintptr_t>(r.C) & 15) || (r.ldc % 4))) return RG_ERR_ALIGN;
  if (r.M > (1 << 30) || r.N > (1 << 30) || r.K > (1 << 30)) return RG_ERR_SHAPE;
  return RG_OK;
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = p / 100.0 * static_cast<double>(v.size() - 1);
  const size_t lo = static_cast<size_t>(std::floor(pos));
  const size_t hi = std::min(v.size() - 1, lo + 1);
  return v[lo] + (v[hi] - v[lo]) * (pos - static_cast<double>(lo));
}

}  // namespace

extern "C" void rg_serve_opts_default(rg_serve_opts* o) {
  if (!o) return;
  o->hbm_budget_bytes = 64LL << 30;
  o->max_batch = 64;
  o->max_inflight = 2;
  o->tile = RG_TILE_128x128;
}

extern "C" int rg_serve(rg_ctx* ctx, const rg_plan* plan, const rg_serve_opts* opts, const rg_serve_request* reqs,
                        int32_t n, rg_serve_result* results, rg_serve_stats* stats) {
  rg::clear_error();
  if (!ctx || !opts || (n > 0 && (!reqs || !results)) || n < 0)
    return rg::fail(RG_ERR_INVALID, "rg_serve: bad argument");
  if (opts->max_batch <= 0 || opts->max_inflight <= 0 || opts->max_inflight > 16 || opts->tile < 0 ||
      opts->tile >= RG_NUM_TILES || opts->hbm_budget_bytes <= 0)
    return rg::fail(RG_ERR_INVALID, "rg_serve: options");
  for (int32_t i = 1; i < n; ++i)
    if (reqs[i].arrival_ns < reqs[i - 1].arrival_ns) return rg::fail(RG_ERR_INVALID, "rg_serve: arrivals not sorted");
  bool need_arena = false;
  for (int32_t i = 0; i < n; ++i) need_arena = need_arena || reqs[i].C == nullptr;

  struct Slot {
    rg_group* group[RG_NUM_TILES] = {};  // one grouped kernel per tile shape
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<int32_t> members;
    bool busy = false;
  };
  std::vector<Slot> slots(static_cast<size_t>(opts->max_inflight));
  Arena arena;
  auto cleanup = [&]() {
    for (auto& s : slots) {
      if (s.stream) cudaStreamSynchronize(s.stream);
      for (rg_group* g : s.group)
        if (g) rg_group_destroy(g);
      if (s.done) cudaEventDestroy(s.done);
      if (s.stream) cudaStreamDestroy(s.stream);
    }
    arena.release_all();
  };
  for (auto& s : slots) {
    for (int t = 0; t < RG_NUM_TILES; ++t) {
      const int rc = rg_group_create(ctx, t, opts->max_batch, &s.group[t]);
      if (rc != RG_OK) {
        cleanup();
        return rc;
      }
    }
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
      cleanup();
      return rg::fail(RG_ERR_CUDA, "rg_serve: stream or event");
    }
  }
  if (need_arena && !arena.init(opts->hbm_budget_bytes)) {
    cleanup();
    return rg::fail(RG_ERR_OOM, "rg_serve: output arena of the budget size");
  }

  std::vector<int64_t> c_off(static_cast<size_t>(n), -1);
  std::vector<float*> c_ptr(static_cast<size_t>(n), nullptr);
  for (int32_t i = 0; i < n; ++i) {
    results[i] = rg_serve_result{};
    results[i].status = RG_OK;
    results[i].batch = -1;
  }
  std::deque<int32_t> ready;
  std::vector<rg_group_problem> probs[RG_NUM_TILES];
  int64_t resident = 0, stalls = 0, batches = 0, done_count = 0;
  int32_t next = 0;
  bool stalled_head = false;
  const auto t0 = std::chrono::steady_clock::now();
  auto now_ns = [&]() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
  };
  int rc = RG_OK;
  while (done_count < n && rc == RG_OK) {
    const int64_t now = now_ns();
    // completions
    for (auto& s : slots) {
      if (!s.busy) continue;
      const cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        rc = rg::fail(RG_ERR_CUDA, std::string("rg_serve: batch failed: ") + cudaGetErrorString(q));
        break;
      }
      const int64_t t = now_ns();
      for (int32_t r : s.members) {
        results[r].done_ns = t;
        resident -= request_bytes(reqs[r]);
        if (c_off[r] >= 0) arena.free(c_off[r], 4 * reqs[r].M * reqs[r].N);
        ++done_count;
      }
      s.members.clear();
      s.busy = false;
    }
    if (rc != RG_OK) break;
    // admission, in arrival order
    while (next < n && reqs[next].arrival_ns <= now) {
      const rg_serve_request& r = reqs[next];
      const int st = request_status(r);
      const int64_t bytes = st == RG_OK ? request_bytes(r) : 0;
      if (st != RG_OK || bytes > opts->hbm_budget_bytes || (r.C == nullptr && 4 * r.M * r.N > arena.size)) {
        results[next].status = st != RG_OK ? st : RG_ERR_ADMISSION;
        results[next].done_ns = now;
        ++done_count;
        ++next;
        stalled_head = false;
        continue;
      }
      if (resident + bytes > opts->hbm_budget_bytes) {
        if (!stalled_head) ++stalls;
        stalled_head = true;
        break;
      }
      int64_t off = -1;
      if (r.C == nullptr) {
        off = arena.alloc(4 * r.M * r.N);
        if (off < 0) {
          if (!stalled_head) ++stalls;
          stalled_head = true;
          break;
        }
      }
      stalled_head = false;
      c_off[next] = off;
      c_ptr[next] = r.C ? r.C : reinterpret_cast<float*>(arena.base + off);
      resident += bytes;
      results[next].admitted_ns = now;
      ready.push_back(next);
      ++next;
    }
    // launch a batch on a free slot
    if (!ready.empty()) {
      for (auto& s : slots) {
        if (s.busy || ready.empty()) continue;
        for (auto& pv : probs) pv.clear();
        s.members.clear();
        while (!ready.empty() && static_cast<int32_t>(s.members.size()) < opts->max_batch) {
          const int32_t i = ready.front();
          ready.pop_front();
          const rg_serve_request& r = reqs[i];
          rg_group_problem p{};
          p.M = r.M; p.N = r.N; p.K = r.K;
          p.A = r.A; p.lda = r.lda; p.B = r.B; p.ldb = r.ldb;
          p.C = c_ptr[i]; p.ldc = r.C ? r.ldc : r.N;
          int tile = opts->tile;
          if (plan) {  // a single-leaf cell lends its autotuned tile and its padded extents
            const rg_leaf* lv = nullptr;
            int32_t nl = 0;
            if (rg_plan_lookup(plan, r.M, r.N, r.K, &lv, &nl, nullptr) == RG_OK && nl == 1) {
              tile = rg::variant_tile(lv[0].variant);
              p.pm = std::max(lv[0].pm, r.M);
              p.pn = std::max(lv[0].pn, r.N);
              p.pk = std::max(lv[0].pk, r.K);
            }
          }
          probs[tile].push_back(p);
          s.members.push_back(i);
        }
        const int64_t t = now_ns();
        for (int tl = 0; tl < RG_NUM_TILES && rc == RG_OK; ++tl)  // one grouped launch per tile shape present
          if (!probs[tl].empty())
            rc = rg_gemm_grouped(s.group[tl], probs[tl].data(), static_cast<int32_t>(probs[tl].size()), s.stream);
        if (rc == RG_OK && cudaEventRecord(s.done, s.stream) != cudaSuccess)
          rc = rg::fail(RG_ERR_CUDA, "rg_serve: event record");
        if (rc != RG_OK) break;
        for (int32_t i : s.members) {
          results[i].launched_ns = t;
          results[i].batch = static_cast<int32_t>(batches);
        }
        ++batches;
        s.busy = true;
      }
    }
  }
  const int64_t end = now_ns();
  cleanup();
  if (rc != RG_OK) return rc;
  if (stats) {
    std::vector<double> lat;
    double flops = 0.0;
    int64_t first = -1, last = 0;
    for (int32_t i = 0; i < n; ++i) {
      if (results[i].status != RG_OK) continue;
      lat.push_back(static_cast<double>(results[i].done_ns - reqs[i].arrival_ns) * 1e-3);
      flops += 2.0 * static_cast<double>(reqs[i].M) * static_cast<double>(reqs[i].N) * static_cast<double>(reqs[i].K);
      if (first < 0) first = reqs[i].arrival_ns;
      last = std::max(last, results[i].done_ns);
    }
    stats->requests = static_cast<int64_t>(lat.size());
    stats->batches = batches;
    stats->admission_stalls = stalls;
    stats->wall_s = static_cast<double>(end) * 1e-9;
    stats->p50_latency_us = percentile(lat, 50.0);
    stats->p99_latency_us = percentile(lat, 99.0);
    double sum = 0.0;
    for (double x : lat) sum += x;
    stats->mean_latency_us = lat.empty() ? 0.0 : sum / static_cast<double>(lat.size());
    const double span = first >= 0 ? static_cast<double>(last - first) * 1e-9 : 0.0;
    stats->tflops = span > 0.0 ? flops / span / 1e12 : 0.0;
  }
  return RG_OK;
}
