// Serving: continuous batching of GEMM requests on top of the grouped GEMM.
//
// One engine drives both entry points:
//   - rg_serve replays a trace of requests with arrival times on the calling
//     thread (a load generator with a known arrival process);
//   - rg_serve_start / rg_serve_submit / rg_serve_poll / rg_serve_stop run the
//     same engine on a worker thread that takes requests as callers submit them.
// Per engine step:
//   - completion: in-flight slots are polled with events; a finished batch
//     releases its requests' budget and arena space;
//   - admission: arrived requests are admitted in arrival order once their
//     operand bytes (2MK + 2KN + 4MN) fit under the HBM budget next to the
//     admitted, unfinished requests; a request that can never fit is rejected
//     (RG_ERR_ADMISSION); one whose C is NULL gets its output from an arena of
//     budget bytes owned by the engine;
//   - routing: every request goes through the plan's O(1) lookup (Sec. 7.1) and
//     becomes its cell's leaves -- each a sub-box of the problem with the variant
//     the autotuner chose for it (tile, split factor, cta_group::2), its padded
//     launch extents, beta and phase; without a plan a request is one leaf on the
//     default tile;
//   - batching: whenever an in-flight slot is free and admitted requests wait,
//     up to max_batch of them form one batch: for each phase in order, one
//     rg_gemm_grouped call over that phase's leaves of every request in the
//     batch (one persistent launch per kernel family present, replayed from CUDA
//     graphs) on the slot's stream, so a K split's beta = 1 leaves follow their
//     first piece, and batches formed while others run overlap them on the GPU.
// A request's leaves and their variants depend only on its shape, and a grouped
// result is bitwise rg_gemm's for the same variant, so a request's result is the
// same alone and in any mix.
// Latency = completion observed on the host - arrival, both on the host's
// steady clock measured from the engine's start.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
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

int64_t request_bytes(const rg_serve_request& r) {
  if (r.dtype == RG_DTYPE_FP8)
    return r.M * r.K + r.K * r.N + 4 * r.M * r.N + 4 * (((r.M + 127) / 128) * r.lds_a + ((r.K + 127) / 128) * r.lds_b);
  return 2 * r.M * r.K + 2 * r.K * r.N + 4 * r.M * r.N;
}

rg::Fp8Request fp8_request(const rg_serve_request& r, float* C, int64_t ldc) {
  return rg::Fp8Request{r.M,  r.N,  r.K,   static_cast<const uint8_t*>(r.A), r.lda, r.sA, r.lds_a,
                        static_cast<const uint8_t*>(r.B), r.ldb, r.sB, r.lds_b, C, ldc};
}

// The per-request checks of rg_gemm (sizes, leading dimensions, TMA alignment),
// made at admission so that one malformed request is rejected alone instead of
// failing the grouped launch it would join.
int request_status(const rg_serve_request& r) {
  if (r.dtype == RG_DTYPE_FP8) return rg::fp8_request_status(fp8_request(r, r.C, r.ldc));
  if (r.dtype != RG_DTYPE_BF16) return RG_ERR_INVALID;
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

int validate_opts(const rg_serve_opts* o) {
  if (!o || o->max_batch <= 0 || o->max_inflight <= 0 || o->max_inflight > 16 || o->tile < 0 ||
      o->tile >= RG_NUM_TILES || o->hbm_budget_bytes <= 0 || o->workspace_mib < 0)
    return RG_ERR_INVALID;
  return RG_OK;
}

class Engine {
 public:
  struct Record {
    rg_serve_request req{};
    rg_serve_result res{};
    int64_t c_off = -1;
    float* c_ptr = nullptr;
    bool done = false;
  };

  Engine(rg_ctx* ctx, const rg_plan* plan, const rg_serve_opts& o) : ctx_(ctx), plan_(plan), o_(o) {}
  ~Engine() { release(); }

  int init(bool need_arena) {
    slots_.resize(static_cast<size_t>(o_.max_inflight));
    const int64_t ws = static_cast<int64_t>(o_.workspace_mib > 0 ? o_.workspace_mib : 256) << 20;
    for (auto& s : slots_) {
      const int rc = rg_group_create(ctx_, o_.tile, std::max(o_.max_batch, 16), ws, &s.group);
      if (rc != RG_OK) return rc;
      if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess)
        return rg::fail(RG_ERR_CUDA, "rg_serve: stream or event");
    }
    if (need_arena && !arena_.init(o_.hbm_budget_bytes))
      return rg::fail(RG_ERR_OOM, "rg_serve: output arena of the budget size");
    t0_ = std::chrono::steady_clock::now();  // the engine's clock starts once it is set up
    return RG_OK;
  }

  void release() {
    for (auto& s : slots_) {
      if (s.stream) cudaStreamSynchronize(s.stream);
      if (s.group) rg_group_destroy(s.group);
      if (s.done) cudaEventDestroy(s.done);
      if (s.stream) cudaStreamDestroy(s.stream);
      s = Slot{};
    }
    arena_.release_all();
  }

  int64_t now_ns() const {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0_).count();
  }

  // A request has arrived (its arrival_ns is already on the engine's clock).
  int64_t add(const rg_serve_request& r) {
    Record rec;
    rec.req = r;
    rec.res.status = RG_OK;
    rec.res.batch = -1;
    recs_.push_back(rec);
    arrived_.push_back(static_cast<int64_t>(recs_.size()) - 1);
    return static_cast<int64_t>(recs_.size()) - 1;
  }

  // One pass of completion, admission and launching.  Returns RG_OK or the
  // error that stopped the engine.
  int step() {
    int rc = RG_OK;
    for (auto& s : slots_) {  // completions
      if (!s.busy) continue;
      const cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return rg::fail(RG_ERR_CUDA, std::string("rg_serve: batch failed: ") + cudaGetErrorString(q));
      const int64_t t = now_ns();
      for (int64_t r : s.members) finish(r, t);
      s.members.clear();
      s.busy = false;
    }
    const int64_t now = now_ns();
    while (!arrived_.empty()) {  // admission, in arrival order
      const int64_t i = arrived_.front();
      Record& rec = recs_[static_cast<size_t>(i)];
      const rg_serve_request& r = rec.req;
      const int st = request_status(r);
      const int64_t bytes = st == RG_OK ? request_bytes(r) : 0;
      if (st != RG_OK || bytes > o_.hbm_budget_bytes || (r.C == nullptr && 4 * r.M * r.N > arena_.size)) {
        rec.res.status = st != RG_OK ? st : RG_ERR_ADMISSION;
        rec.res.done_ns = now;
        rec.done = true;
        ++done_count_;
        arrived_.pop_front();
        stalled_head_ = false;
        continue;
      }
      if (resident_ + bytes > o_.hbm_budget_bytes) {
        if (!stalled_head_) ++stalls_;
        stalled_head_ = true;
        break;
      }
      int64_t off = -1;
      if (r.C == nullptr) {
        off = arena_.alloc(4 * r.M * r.N);
        if (off < 0) {
          if (!stalled_head_) ++stalls_;
          stalled_head_ = true;
          break;
        }
      }
      stalled_head_ = false;
      rec.c_off = off;
      rec.c_ptr = r.C ? r.C : reinterpret_cast<float*>(arena_.base + off);
      resident_ += bytes;
      rec.res.admitted_ns = now;
      ready_.push_back(i);
      arrived_.pop_front();
    }
    for (auto& s : slots_) {  // launch batches on free slots
      if (s.busy || ready_.empty()) continue;
      if ((rc = launch_batch(s)) != RG_OK) return rc;
    }
    return RG_OK;
  }

  bool idle() const { return arrived_.empty() && ready_.empty() && !any_busy(); }
  int64_t done_count() const { return done_count_; }
  std::vector<Record>& records() { return recs_; }

  void fill_stats(rg_serve_stats* stats, int64_t end) const {
    std::vector<double> lat;
    double flops = 0.0;
    int64_t first = -1, last = 0;
    for (const auto& rec : recs_) {
      if (rec.res.status != RG_OK || !rec.done) continue;
      lat.push_back(static_cast<double>(rec.res.done_ns - rec.req.arrival_ns) * 1e-3);
      flops += 2.0 * static_cast<double>(rec.req.M) * static_cast<double>(rec.req.N) * static_cast<double>(rec.req.K);
      if (first < 0 || rec.req.arrival_ns < first) first = rec.req.arrival_ns;
      last = std::max(last, rec.res.done_ns);
    }
    stats->requests = static_cast<int64_t>(lat.size());
    stats->batches = batches_;
    stats->admission_stalls = stalls_;
    stats->wall_s = static_cast<double>(end) * 1e-9;
    stats->p50_latency_us = percentile(lat, 50.0);
    stats->p99_latency_us = percentile(lat, 99.0);
    double sum = 0.0;
    for (double x : lat) sum += x;
    stats->mean_latency_us = lat.empty() ? 0.0 : sum / static_cast<double>(lat.size());
    const double span = first >= 0 ? static_cast<double>(last - first) * 1e-9 : 0.0;
    stats->tflops = span > 0.0 ? flops / span / 1e12 : 0.0;
  }

 private:
  struct Slot {
    rg_group* group = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<int64_t> members;
    bool busy = false;
  };

  bool any_busy() const {
    for (const auto& s : slots_)
      if (s.busy) return true;
    return false;
  }

  void finish(int64_t r, int64_t t) {
    Record& rec = recs_[static_cast<size_t>(r)];
    rec.res.done_ns = t;
    rec.done = true;
    resident_ -= request_bytes(rec.req);
    if (rec.c_off >= 0) arena_.free(rec.c_off, 4 * rec.req.M * rec.req.N);
    ++done_count_;
  }

  // The leaves of one request: its plan cell's leaves clipped to the problem,
  // or one leaf on the default tile.
  int route(const Record& rec, std::vector<std::pair<int32_t, rg_group_problem>>& out) const {
    const rg_serve_request& r = rec.req;
    const int64_t ldc = r.C ? r.ldc : r.N;
    if (!plan_) {
      rg_group_problem p{};
      p.M = r.M; p.N = r.N; p.K = r.K;
      p.A = r.A; p.lda = r.lda; p.B = r.B; p.ldb = r.ldb;
      p.C = rec.c_ptr; p.ldc = ldc;
      p.variant = RG_VARIANT(o_.tile, 0);
      out.emplace_back(0, p);
      return RG_OK;
    }
    const rg_leaf* lv = nullptr;
    int32_t nl = 0;
    const int rc = rg_plan_lookup(plan_, r.M, r.N, r.K, &lv, &nl, nullptr);
    if (rc != RG_OK) return rc;
    for (int32_t j = 0; j < nl; ++j) {
      const rg_leaf& lf = lv[j];
      if (lf.m0 >= r.M || lf.n0 >= r.N || lf.k0 >= r.K) continue;  // wholly in the padding
      rg_group_problem p{};
      p.M = std::min(lf.m, r.M - lf.m0);
      p.N = std::min(lf.n, r.N - lf.n0);
      p.K = std::min(lf.k, r.K - lf.k0);
      p.A = static_cast<const uint16_t*>(r.A) + lf.m0 * r.lda + lf.k0;
      p.lda = r.lda;
      p.B = static_cast<const uint16_t*>(r.B) + lf.k0 * r.ldb + lf.n0;
      p.ldb = r.ldb;
      p.C = rec.c_ptr + lf.m0 * ldc + lf.n0;
      p.ldc = ldc;
      p.pm = lf.pm;
      p.pn = lf.pn;
      p.pk = lf.pk;
      p.beta = lf.beta;
      p.variant = lf.variant;
      out.emplace_back(lf.phase, p);
    }
    return RG_OK;
  }

  int launch_batch(Slot& s) {
    std::vector<std::pair<int32_t, rg_group_problem>> leaves;
    std::vector<int64_t> fp8;  // FP8 members, run leaf by leaf after each phase's grouped launch
    s.members.clear();
    while (!ready_.empty() && static_cast<int32_t>(s.members.size()) < o_.max_batch) {
      const int64_t i = ready_.front();
      ready_.pop_front();
      if (recs_[static_cast<size_t>(i)].req.dtype == RG_DTYPE_FP8) {
        fp8.push_back(i);
        s.members.push_back(i);
        continue;
      }
      const int rc = route(recs_[static_cast<size_t>(i)], leaves);
      if (rc != RG_OK) {  // a shape beyond the plan grid fails alone
        Record& rec = recs_[static_cast<size_t>(i)];
        rec.res.status = rc;
        finish(i, now_ns());
        continue;
      }
      s.members.push_back(i);
    }
    if (s.members.empty()) return RG_OK;
    const int64_t t = now_ns();
    int32_t max_phase = 0;
    for (const auto& l : leaves) max_phase = std::max(max_phase, l.first);
    float* ws = nullptr;
    int32_t* tickets = nullptr;
    int64_t ws_bytes = 0, max_tickets = 0;
    rg::group_workspace(s.group, &ws, &ws_bytes, &tickets, &max_tickets);
    std::vector<int32_t> fp8_phases(fp8.size(), 0);
    std::vector<rg_group_problem> probs;
    for (int32_t ph = 0; ph <= max_phase; ++ph) {  // a K split's later pieces after the earlier ones
      probs.clear();
      for (const auto& l : leaves)
        if (l.first == ph) probs.push_back(l.second);
      if (!probs.empty()) {
        const int rc = rg_gemm_grouped(s.group, probs.data(), static_cast<int32_t>(probs.size()), s.stream);
        if (rc != RG_OK) return rc;
      }
      for (size_t j = 0; j < fp8.size(); ++j) {  // the same stream, so the group's workspace is free
        if (ph > fp8_phases[j]) continue;
        Record& rec = recs_[static_cast<size_t>(fp8[j])];
        if (rec.done) continue;
        int32_t mp = 0;
        const int rc = rg::fp8_enqueue_phase(ctx_, o_.fp8_plan, fp8_request(rec.req, rec.c_ptr, rec.req.C ? rec.req.ldc : rec.req.N),
                                             ph, ws, ws_bytes, tickets, max_tickets, s.stream, &mp);
        if (rc == RG_ERR_SHAPE && ph == 0) {  // beyond the FP8 plan's grid: fails alone, before any launch
          rec.res.status = rc;
          finish(fp8[j], now_ns());
          s.members.erase(std::find(s.members.begin(), s.members.end(), fp8[j]));
          continue;
        }
        if (rc != RG_OK) return rc;
        if (ph == 0) {
          fp8_phases[j] = mp;
          max_phase = std::max(max_phase, mp);
        }
      }
    }
    if (s.members.empty()) return RG_OK;
    if (cudaEventRecord(s.done, s.stream) != cudaSuccess) return rg::fail(RG_ERR_CUDA, "rg_serve: event record");
    for (int64_t i : s.members) {
      recs_[static_cast<size_t>(i)].res.launched_ns = t;
      recs_[static_cast<size_t>(i)].res.batch = static_cast<int32_t>(batches_);
    }
    ++batches_;
    s.busy = true;
    return RG_OK;
  }

  rg_ctx* ctx_;
  const rg_plan* plan_;
  rg_serve_opts o_;
  std::vector<Slot> slots_;
  Arena arena_;
  std::vector<Record> recs_;
  std::deque<int64_t> arrived_, ready_;
  int64_t resident_ = 0, stalls_ = 0, batches_ = 0, done_count_ = 0;
  bool stalled_head_ = false;
  std::chrono::steady_clock::time_point t0_ = std::chrono::steady_clock::now();
};

}  // namespace

extern "C" void rg_serve_opts_default(rg_serve_opts* o) {
  if (!o) return;
  o->hbm_budget_bytes = 64LL << 30;
  o->max_batch = 64;
  o->max_inflight = 2;
  o->tile = RG_TILE_128x128;
  o->workspace_mib = 256;
  o->fp8_plan = nullptr;
}

extern "C" int rg_serve(rg_ctx* ctx, const rg_plan* plan, const rg_serve_opts* opts, const rg_serve_request* reqs,
                        int32_t n, rg_serve_result* results, rg_serve_stats* stats) {
  rg::clear_error();
  if (!ctx || !opts || (n > 0 && (!reqs || !results)) || n < 0)
    return rg::fail(RG_ERR_INVALID, "rg_serve: bad argument");
  if (validate_opts(opts) != RG_OK) return rg::fail(RG_ERR_INVALID, "rg_serve: options");
  for (int32_t i = 1; i < n; ++i)
    if (reqs[i].arrival_ns < reqs[i - 1].arrival_ns) return rg::fail(RG_ERR_INVALID, "rg_serve: arrivals not sorted");
  bool need_arena = false;
  for (int32_t i = 0; i < n; ++i) need_arena = need_arena || reqs[i].C == nullptr;
  Engine eng(ctx, plan, *opts);
  int rc = eng.init(need_arena);
  if (rc != RG_OK) return rc;
  int32_t next = 0;
  while (eng.done_count() < n && rc == RG_OK) {
    const int64_t now = eng.now_ns();
    while (next < n && reqs[next].arrival_ns <= now) eng.add(reqs[next++]);
    rc = eng.step();
  }
  const int64_t end = eng.now_ns();
  eng.release();
  if (rc != RG_OK) return rc;
  auto& recs = eng.records();
  for (int32_t i = 0; i < n; ++i) results[i] = recs[static_cast<size_t>(i)].res;
  if (stats) eng.fill_stats(stats, end);
  return RG_OK;
}

// ------------------------------------------------------------------ online serving
//
// A worker thread owns the engine (its streams, groups and arena) and runs its
// steps while any request is outstanding; submitted requests wait in a queue
// guarded by a mutex, and results are read back under the same mutex.
struct rg_server {
  rg_ctx* ctx = nullptr;
  Engine* eng = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  std::vector<rg_serve_request> inbox;
  std::vector<rg_serve_result> results;  // by request id, copied from the engine
  std::vector<uint8_t> done;
  int64_t submitted = 0, finished = 0;
  bool stopping = false;
  int status = RG_OK;  // the first error that stopped the worker
  std::string error;
};

namespace {
void server_loop(rg_server* sv) {
  cudaSetDevice(rg::ctx_device(sv->ctx));
  Engine& eng = *sv->eng;
  std::vector<rg_serve_request> batch;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      if (eng.idle() && sv->inbox.empty()) {
        if (sv->stopping) break;
        sv->cv.wait_for(lk, std::chrono::milliseconds(2));
      }
      batch.swap(sv->inbox);
    }
    const int64_t now = eng.now_ns();
    for (auto& r : batch) {
      r.arrival_ns = now;
      eng.add(r);
    }
    batch.clear();
    const int rc = eng.step();
    auto& recs = eng.records();
    std::lock_guard<std::mutex> lk(sv->mu);
    for (size_t i = sv->results.size(); i < recs.size(); ++i) {
      sv->results.push_back(recs[i].res);
      sv->done.push_back(0);
    }
    for (size_t i = 0; i < recs.size(); ++i)
      if (recs[i].done && !sv->done[i]) {
        sv->results[i] = recs[i].res;
        sv->done[i] = 1;
        ++sv->finished;
      }
    if (rc != RG_OK) {
      sv->status = rc;
      sv->error = rg_last_error();
      sv->cv.notify_all();
      return;
    }
    sv->cv.notify_all();
  }
}
}  // namespace

extern "C" int rg_serve_start(rg_ctx* ctx, const rg_plan* plan, const rg_serve_opts* opts, rg_server** out) {
  rg::clear_error();
  if (!ctx || !opts || !out) return rg::fail(RG_ERR_INVALID, "rg_serve_start: bad argument");
  *out = nullptr;
  if (validate_opts(opts) != RG_OK) return rg::fail(RG_ERR_INVALID, "rg_serve_start: options");
  auto* sv = new (std::nothrow) rg_server();
  if (!sv) return rg::fail(RG_ERR_OOM, "rg_serve_start: host allocation");
  sv->ctx = ctx;
  sv->eng = new (std::nothrow) Engine(ctx, plan, *opts);
  if (!sv->eng) {
    delete sv;
    return rg::fail(RG_ERR_OOM, "rg_serve_start: host allocation");
  }
  const int rc = sv->eng->init(true);
  if (rc != RG_OK) {
    delete sv->eng;
    delete sv;
    return rc;
  }
  sv->worker = std::thread(server_loop, sv);
  *out = sv;
  return RG_OK;
}

extern "C" int rg_serve_submit(rg_server* sv, const rg_serve_request* req, int64_t* id_out) {
  rg::clear_error();
  if (!sv || !req || !id_out) return rg::fail(RG_ERR_INVALID, "rg_serve_submit: bad argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->status != RG_OK) return rg::fail(sv->status, "rg_serve_submit: the server stopped: " + sv->error);
  if (sv->stopping) return rg::fail(RG_ERR_INVALID, "rg_serve_submit: the server is stopping");
  sv->inbox.push_back(*req);
  *id_out = sv->submitted++;
  sv->cv.notify_all();
  return RG_OK;
}

extern "C" int rg_serve_poll(rg_server* sv, int64_t id, rg_serve_result* out, int32_t* done) {
  rg::clear_error();
  if (!sv || !out || !done || id < 0) return rg::fail(RG_ERR_INVALID, "rg_serve_poll: bad argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (id >= sv->submitted) return rg::fail(RG_ERR_INVALID, "rg_serve_poll: unknown request id");
  *done = 0;
  if (static_cast<size_t>(id) < sv->done.size() && sv->done[static_cast<size_t>(id)]) {
    *out = sv->results[static_cast<size_t>(id)];
    *done = 1;
  }
  if (sv->status != RG_OK && !*done) return rg::fail(sv->status, "rg_serve_poll: the server stopped: " + sv->error);
  return RG_OK;
}

extern "C" int rg_serve_wait(rg_server* sv, int64_t id, rg_serve_result* out) {
  rg::clear_error();
  if (!sv || !out || id < 0) return rg::fail(RG_ERR_INVALID, "rg_serve_wait: bad argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  if (id >= sv->submitted) return rg::fail(RG_ERR_INVALID, "rg_serve_wait: unknown request id");
  sv->cv.wait(lk, [&] {
    return sv->status != RG_OK || (static_cast<size_t>(id) < sv->done.size() && sv->done[static_cast<size_t>(id)]);
  });
  if (static_cast<size_t>(id) < sv->done.size() && sv->done[static_cast<size_t>(id)]) {
    *out = sv->results[static_cast<size_t>(id)];
    return RG_OK;
  }
  return rg::fail(sv->status, "rg_serve_wait: the server stopped: " + sv->error);
}

extern "C" int rg_serve_stop(rg_server* sv, rg_serve_stats* stats) {
  rg::clear_error();
  if (!sv) return rg::fail(RG_ERR_INVALID, "rg_serve_stop: null server");
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stopping = true;
    sv->cv.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();
  const int64_t end = sv->eng->now_ns();
  if (stats) sv->eng->fill_stats(stats, end);
  const int status = sv->status;
  const std::string error = sv->error;
  delete sv->eng;  // releases streams, groups and the arena
  delete sv;
  if (status != RG_OK) return rg::fail(status, "rg_serve_stop: the server had stopped: " + error);
  return RG_OK;
}
