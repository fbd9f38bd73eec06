// Serving loop of the C ABI (bsrht_server_*, bsrht_submit, bsrht_poll,
// bsrht_wait): continuous batching of sketch / RSVD (Algorithm 1) / Nystrom
// (Algorithm 2) requests on one GPU.
//
// A server holds one device pool (cudaMalloc'ed once, hbm_budget bytes) for
// request scratch, carved by a first-fit allocator, and E executor threads,
// each with its own non-blocking stream.  An idle executor takes the first
// queued request whose scratch fits in the free pool (requests that fit may
// overtake one that does not, at most kMaxSkips times, then the head waits
// for memory alone); when it takes a small sketch it also takes up to
// max_group - 1 further queued small sketches of the same kernel instance and
// runs them as one grouped persistent launch.  Sketch launches (single and
// grouped) are captured into CUDA graphs and replayed from a per-executor
// cache of executable graphs, updated in place for new pointers.  RSVD and
// Nystrom read numerical statuses back during the call (their fallbacks are
// host decisions), so they run eagerly on the executor's stream.  Each
// executor waits for its work with a bounded event poll.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "bsrht.h"
#include "capi_internal.cuh"
#include "common.cuh"
#include "sketch.cuh"

namespace bsrht {
namespace {

constexpr size_t kNone = ~size_t(0);
constexpr int kMaxSkips = 16;

// First-fit allocator over [0, cap) in 256-byte units.  free_ maps offset to
// length of the free ranges (disjoint, never adjacent); live_ the handed-out
// ranges.
class FirstFit {
 public:
  explicit FirstFit(size_t cap = 0) { reset(cap); }
  void reset(size_t cap) {
    cap_ = cap / 256 * 256;
    free_.clear();
    live_.clear();
    if (cap_ > 0) free_[0] = cap_;
    used_ = high_ = 0;
  }
  static size_t round(size_t b) { return (std::max<size_t>(b, 1) + 255) / 256 * 256; }
  size_t alloc(size_t bytes) {
    bytes = round(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > bytes) free_[off + bytes] = len - bytes;
      live_[off] = bytes;
      used_ += bytes;
      high_ = std::max(high_, used_);
      return off;
    }
    return kNone;
  }
  bool release(size_t off) {
    auto lv = live_.find(off);
    if (lv == live_.end()) return false;
    size_t len = lv->second;
    live_.erase(lv);
    used_ -= len;
    auto next = free_.lower_bound(off);
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        off = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    next = free_.lower_bound(off);
    if (next != free_.end() && off + len == next->first) {
      len += next->second;
      free_.erase(next);
    }
    free_[off] = len;
    return true;
  }
  size_t cap() const { return cap_; }
  size_t used() const { return used_; }
  size_t high() const { return high_; }
  // Invariants: ranges inside [0, cap), disjoint, free ranges not adjacent,
  // free + live = cap.  Returns the number of violations.
  int check() const {
    int bad = 0;
    std::map<size_t, std::pair<size_t, int>> all;
    for (auto& f : free_) all[f.first] = {f.second, 0};
    for (auto& l : live_) {
      if (all.count(l.first)) ++bad;
      all[l.first] = {l.second, 1};
    }
    size_t pos = 0, sum = 0, used = 0;
    int prev_kind = -1;
    for (auto& a : all) {
      if (a.first != pos) ++bad;  // gap or overlap
      if (a.second.first == 0 || a.second.first % 256) ++bad;
      if (a.second.second == 0 && prev_kind == 0) ++bad;  // adjacent free ranges
      prev_kind = a.second.second;
      pos = a.first + a.second.first;
      sum += a.second.first;
      if (a.second.second) used += a.second.first;
    }
    if (sum != cap_ || (cap_ > 0 && pos != cap_)) ++bad;
    if (used != used_) ++bad;
    return bad;
  }

 private:
  size_t cap_ = 0, used_ = 0, high_ = 0;
  std::map<size_t, size_t> free_, live_;
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t ticket = 0;
  bsrht_request r{};
  size_t bytes = 0;       // scratch while it runs
  bool grouped = false;   // small sketch: runs inside a grouped launch
  bool tune = false;      // autotune its shape class before running
  SketchPlan gplan;       // plain-kernel plan (grouped sketches)
  size_t off = kNone;
  int skips = 0;
  int status = BSRHT_OK;
  bool done = false;
  double t_submit = 0.0, t_done = 0.0;
};

std::string plan_key(const char* tag, const SketchPlan& pl, int64_t groups) {
  char b[160];
  snprintf(b, sizeof(b), "%s:%d:%d:%d:%lld", tag, pl.dtype, pl.path, pl.inst, (long long)groups);
  return b;
}

int tune_class(const bsrht_request& r, int64_t lda) {
  // Same buckets as the library's tuning table: (dtype, r, ceil log2 m, l > 512, row alignment).
  int64_t rb = (r.n + r.p - 1) / r.p, rr = 1;
  while (rr < rb) rr <<= 1;
  int lr = 0, lm = 0;
  while ((int64_t(1) << (lr + 1)) <= rr) ++lr;
  while ((int64_t(1) << lm) < std::max<int64_t>(r.m, 1)) ++lm;
  const int es = r.dtype == BSRHT_F64 ? 8 : r.dtype == BSRHT_F32 ? 4 : 2;
  const int al = ((lda * es) % 16) == 0 ? 1 : 0;
  return (((r.dtype * 64 + lr) * 64 + lm) * 2 + (r.l > 512 ? 1 : 0)) * 2 + al;
}

}  // namespace
}  // namespace bsrht

using namespace bsrht;

struct bsrht_server {
  int device = 0;
  bsrht_server_opts o{};
  char* pool = nullptr;
  FirstFit alloc;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<std::thread> threads;
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, failed = 0;
  int64_t grouped_launches = 0, grouped_requests = 0, graph_launches = 0;
  std::set<int> tuned;     // shape classes tuned (or being tuned) here
  int64_t tuned_count = 0;

  // Under mu: takes the next admissible work into batch.
  bool pick(std::vector<Req*>& batch) {
    for (size_t idx = 0; idx < queue.size(); ++idx) {
      if (idx > 0 && queue[0]->skips >= kMaxSkips) return false;  // the head waits for memory alone
      Req* q = queue[idx];
      const size_t off = alloc.alloc(q->bytes);
      if (off == kNone) continue;
      q->off = off;
      batch.push_back(q);
      for (size_t j = 0; j < idx; ++j) queue[j]->skips++;
      queue.erase(queue.begin() + (std::ptrdiff_t)idx);
      if (q->grouped) {
        const int cap = std::max(1, std::min<int>(o.max_group, kMaxGroup));
        for (size_t j = idx; j < queue.size() && (int)batch.size() < cap;) {
          Req* c = queue[j];
          if (c->grouped && c->gplan.dtype == q->gplan.dtype && c->gplan.inst == q->gplan.inst &&
              (c->gplan.dtype == BSRHT_F64) == (q->gplan.dtype == BSRHT_F64)) {
            const size_t o2 = alloc.alloc(c->bytes);
            if (o2 != kNone) {
              c->off = o2;
              batch.push_back(c);
              queue.erase(queue.begin() + (std::ptrdiff_t)j);
              continue;
            }
          }
          ++j;
        }
      }
      return true;
    }
    return false;
  }

  void finish(const std::vector<Req*>& batch, const std::vector<int>& st, bool keep_memory) {
    std::lock_guard<std::mutex> lock(mu);
    const double t = now_s();
    for (size_t i = 0; i < batch.size(); ++i) {
      Req* q = batch[i];
      if (!keep_memory) alloc.release(q->off);
      q->status = st[i];
      q->done = true;
      q->t_done = t;
      ++completed;
      if (st[i] != BSRHT_OK) ++failed;
      lat_ms.push_back((t - q->t_submit) * 1e3);
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
};

namespace bsrht {
namespace {

struct GraphCache {
  std::map<std::string, cudaGraphExec_t> execs;
  ~GraphCache() {
    for (auto& e : execs) cudaGraphExecDestroy(e.second);
  }
};

// Captures enqueue(stream) into a graph and launches it, reusing the cached
// executable graph of `key` when cudaGraphExecUpdate accepts the new one.
template <typename F>
int run_graph(cudaStream_t s, GraphCache& cache, const std::string& key, F&& enqueue) {
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return enqueue(s);
  }
  const int st = enqueue(s);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (st != BSRHT_OK || ce != cudaSuccess || g == nullptr) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st != BSRHT_OK ? st : cuda_failure(ce, __FILE__, __LINE__);
  }
  auto it = cache.execs.find(key);
  if (it != cache.execs.end()) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(it->second, g, &info) == cudaSuccess) {
      cudaGraphDestroy(g);
      return cudaGraphLaunch(it->second, s) == cudaSuccess ? BSRHT_OK : BSRHT_ECUDA;
    }
    cudaGetLastError();
    cudaGraphExecDestroy(it->second);
    cache.execs.erase(it);
  }
  if (cache.execs.size() >= 64) {
    for (auto& e : cache.execs) cudaGraphExecDestroy(e.second);
    cache.execs.clear();
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    return cuda_failure(ie, __FILE__, __LINE__);
  }
  cache.execs[key] = ex;
  return cudaGraphLaunch(ex, s) == cudaSuccess ? BSRHT_OK : BSRHT_ECUDA;
}

// Bounded wait for everything enqueued on s so far.
int wait_bounded(cudaStream_t s, cudaEvent_t ev, int64_t timeout_ms) {
  const cudaError_t er = cudaEventRecord(ev, s);
  if (er != cudaSuccess) return cuda_failure(er, __FILE__, __LINE__);
  const double t0 = now_s();
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return BSRHT_OK;
    if (e != cudaErrorNotReady) return cuda_failure(e, __FILE__, __LINE__);
    if ((now_s() - t0) * 1e3 > (double)timeout_ms) return BSRHT_ETIMEDOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

void executor(bsrht_server* sv) {
  cudaSetDevice(sv->device);
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  const bool ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
  GraphCache cache;
  for (;;) {
    std::vector<Req*> batch;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      for (;;) {
        if (sv->pick(batch)) break;
        if (sv->stop && sv->queue.empty()) {
          lock.unlock();
          cache.execs.clear();
          if (ev) cudaEventDestroy(ev);
          if (s) cudaStreamDestroy(s);
          return;
        }
        sv->cv_work.wait(lock);
      }
    }
    std::vector<int> st(batch.size(), BSRHT_OK);
    int common = ok ? BSRHT_OK : BSRHT_ECUDA;
    bool graphs_used = false;
    if (common == BSRHT_OK && batch[0]->grouped) {
      std::vector<const SketchPlan*> plans;
      std::vector<const void*> As;
      std::vector<uint64_t> seeds;
      std::vector<void*> outs, works;
      for (Req* q : batch) {
        plans.push_back(&q->gplan);
        As.push_back(q->r.A);
        seeds.push_back(q->r.seed);
        outs.push_back(q->r.out);
        works.push_back(sv->pool + q->off);
      }
      auto enq = [&](cudaStream_t st_) {
        return sketch_group_run(plans.data(), As.data(), seeds.data(), outs.data(), works.data(), (int)batch.size(),
                                st_);
      };
      if (sv->o.use_graphs) {
        common = run_graph(s, cache, plan_key("group", batch[0]->gplan, 1), enq);
        graphs_used = true;
      } else {
        common = enq(s);
      }
    } else if (common == BSRHT_OK) {
      Req* q = batch[0];
      const bsrht_request& r = q->r;
      bsrht_opts o;
      bsrht_opts_init(&o);
      o.dtype = r.dtype;
      o.lda = r.lda;
      o.stream = s;
      o.workspace = sv->pool + q->off;
      o.workspace_bytes = q->bytes;
      o.precision = r.precision;
      int pdt = r.dtype;  // the sketch plan's element-type code (validated at submit)
      plan_dtype(o, &pdt);
      if (r.kind == BSRHT_REQ_SKETCH) {
        if (q->tune) {
          const size_t wb = sketch_autotune_work_bytes(r.dtype, r.n, r.m, r.lda, r.p, r.l);
          const size_t wpad = (wb + 255) / 256 * 256;
          int c = 0;
          double t = 0.0;
          common = sketch_autotune(r.A, r.dtype, r.n, r.m, r.lda, r.p, r.l, sv->pool + q->off, wb,
                                   sv->pool + q->off + wpad, s, &c, &t);
        }
        SketchPlan pl;
        if (common == BSRHT_OK)
          common = sketch_make_plan(pl, pdt, BSRHT_VARIANT_AUTO, r.n, r.m, r.lda, r.p, r.l, true, r.A);
        if (common == BSRHT_OK && pl.work_bytes > q->bytes) common = BSRHT_ENOMEM;
        if (common == BSRHT_OK) {
          auto enq = [&](cudaStream_t st_) {
            o.stream = st_;
            return bsrht_sketch(r.A, r.n, r.m, r.p, r.l, r.seed, r.out, &o);
          };
          if (sv->o.use_graphs) {
            const int64_t groups = (r.l + std::max<int64_t>(pl.jgroup, 1) - 1) / std::max<int64_t>(pl.jgroup, 1);
            common = run_graph(s, cache, plan_key("one", pl, groups), enq);
            graphs_used = true;
          } else {
            common = enq(s);
          }
        }
      } else if (r.kind == BSRHT_REQ_RSVD) {
        common = bsrht_rsvd(r.A, r.n, r.m, r.k, r.l, r.p, r.seed, r.U, r.S, r.V, &o);
      } else {
        common = bsrht_nystrom(r.A, r.n, r.k, r.l, r.p, r.seed, r.U, r.S, &o);
      }
    }
    bool keep = false;
    if (common == BSRHT_OK || common == BSRHT_ECUDA) {
      const int w = wait_bounded(s, ev, sv->o.exec_timeout_ms);
      if (w == BSRHT_ETIMEDOUT) keep = true;  // the work may still be running on this memory
      if (common == BSRHT_OK) common = w;
    } else {
      // A numerical or argument status: whatever was enqueued must still end
      // before the scratch is reused.
      if (wait_bounded(s, ev, sv->o.exec_timeout_ms) == BSRHT_ETIMEDOUT) keep = true;
    }
    for (auto& x : st) x = common;
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      if (graphs_used && common == BSRHT_OK) sv->graph_launches++;
      if (batch[0]->grouped) {
        sv->grouped_launches++;
        sv->grouped_requests += (int64_t)batch.size();
      }
    }
    sv->finish(batch, st, keep);
  }
}

int validate_and_size(bsrht_server* sv, const bsrht_request& r, Req& q) {
  if (r.kind < BSRHT_REQ_SKETCH || r.kind > BSRHT_REQ_NYSTROM) return BSRHT_EINVAL;
  if (r.dtype < BSRHT_F64 || r.dtype > BSRHT_F16 || !r.A) return BSRHT_EINVAL;
  bsrht_opts o;
  bsrht_opts_init(&o);
  o.dtype = r.dtype;
  o.lda = r.lda;
  o.precision = r.precision;
  size_t bytes = 0;
  if (r.kind == BSRHT_REQ_SKETCH) {
    if (!r.out || r.m < 1) return BSRHT_EINVAL;
    int pdt = r.dtype;
    int st = plan_dtype(o, &pdt);
    if (st != BSRHT_OK) return st;
    SketchPlan pl;
    st = sketch_make_plan(pl, pdt, BSRHT_VARIANT_AUTO, r.n, r.m, r.lda, r.p, r.l, true, r.A);
    if (st != BSRHT_OK) return st;
    const int64_t lda = r.lda == 0 ? r.m : r.lda;
    if (pdt != r.dtype) {
      // FP64 arithmetic on FP32 storage: the TMA-fed integer-transform
      // kernel alone (no grouped launch, no tuning).
      q.bytes = FirstFit::round(pl.work_bytes);
      return q.bytes > sv->alloc.cap() ? BSRHT_ENOMEM : BSRHT_OK;
    }
    SketchPlan gp;
    const int gst = sketch_make_plan_grouped(gp, r.dtype, r.n, r.m, lda, r.p, r.l);
    const int occ_tiles = num_sms() * 2;
    if (sv->o.max_group > 1 && gst == BSRHT_OK && gp.T < occ_tiles) {
      q.grouped = true;
      q.gplan = gp;
      bytes = sketch_group_work_bytes(gp);
    } else {
      // Sized for any instance: the shape class may be tuned before it runs.
      bytes = std::max(pl.work_bytes, sketch_autotune_work_bytes(r.dtype, r.n, r.m, lda, r.p, r.l));
      if (sv->o.autotune && pl.path != 1) {
        std::lock_guard<std::mutex> lock(sv->mu);
        const int cls = tune_class(r, lda);
        if (!sv->tuned.count(cls)) {
          sv->tuned.insert(cls);
          sv->tuned_count++;
          q.tune = true;
        }
      }
      if (q.tune) {
        const size_t wb = sketch_autotune_work_bytes(r.dtype, r.n, r.m, lda, r.p, r.l);
        const size_t ob = (size_t)r.l * (size_t)r.m * (r.dtype == BSRHT_F64 ? 8 : 4);
        bytes = std::max(bytes, (wb + 255) / 256 * 256 + ob);
        // the tuned plan may need more than the built-in one
        bytes = std::max(bytes, wb);
      }
    }
  } else if (r.kind == BSRHT_REQ_RSVD) {
    if (!r.U || !r.S || !r.V) return BSRHT_EINVAL;
    const int st = bsrht_rsvd_workspace(r.n, r.m, r.k, r.l, r.p, &o, &bytes);
    if (st != BSRHT_OK) return st;
  } else {
    if (!r.U || !r.S) return BSRHT_EINVAL;
    const int st = bsrht_nystrom_workspace(r.n, r.k, r.l, r.p, &o, &bytes);
    if (st != BSRHT_OK) return st;
  }
  q.bytes = FirstFit::round(bytes);
  if (q.bytes > sv->alloc.cap()) return BSRHT_ENOMEM;
  return BSRHT_OK;
}

}  // namespace
}  // namespace bsrht

extern "C" {

void bsrht_server_opts_init(bsrht_server_opts* o) {
  if (!o) return;
  o->hbm_budget = size_t(1) << 30;
  o->executors = 4;
  o->max_group = 16;
  o->use_graphs = 1;
  o->autotune = 1;
  o->exec_timeout_ms = 600000;
}

int bsrht_server_create_ex(const bsrht_server_opts* opts, bsrht_server** out) {
  if (!opts || !out) return BSRHT_EINVAL;
  *out = nullptr;
  if (opts->hbm_budget < 256 || opts->executors < 1 || opts->executors > 64 || opts->max_group < 1 ||
      opts->exec_timeout_ms < 1)
    return BSRHT_EINVAL;
  std::unique_ptr<bsrht_server> sv(new bsrht_server());
  sv->o = *opts;
  sv->o.max_group = std::min<int32_t>(sv->o.max_group, kMaxGroup);
  BSRHT_CUDA_TRY(cudaGetDevice(&sv->device));
  void* p = nullptr;
  if (cudaMalloc(&p, opts->hbm_budget) != cudaSuccess) {
    cudaGetLastError();
    return BSRHT_ENOMEM;
  }
  sv->pool = static_cast<char*>(p);
  sv->alloc.reset(opts->hbm_budget);
  for (int i = 0; i < sv->o.executors; ++i) sv->threads.emplace_back(executor, sv.get());
  *out = sv.release();
  return BSRHT_OK;
}

int bsrht_server_create(size_t hbm_budget, bsrht_server** out) {
  bsrht_server_opts o;
  bsrht_server_opts_init(&o);
  o.hbm_budget = hbm_budget;
  return bsrht_server_create_ex(&o, out);
}

int bsrht_submit(bsrht_server* sv, const bsrht_request* r, uint64_t* ticket) {
  if (!sv || !r || !ticket) return BSRHT_EINVAL;
  std::unique_ptr<Req> q(new Req());
  q->r = *r;
  if (q->r.lda == 0) q->r.lda = r->kind == BSRHT_REQ_NYSTROM ? r->n : r->m;
  const int st = validate_and_size(sv, q->r, *q);
  if (st != BSRHT_OK) return st;
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stop) return BSRHT_EINVAL;
  q->ticket = sv->next_ticket++;
  q->t_submit = now_s();
  *ticket = q->ticket;
  sv->queue.push_back(q.get());
  sv->reqs[q->ticket] = std::move(q);
  sv->submitted++;
  sv->cv_work.notify_one();
  return BSRHT_OK;
}

int bsrht_poll(bsrht_server* sv, uint64_t ticket, int* done) {
  if (!sv || !done) return BSRHT_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return BSRHT_EINVAL;
  *done = it->second->done ? 1 : 0;
  return it->second->done ? it->second->status : BSRHT_OK;
}

int bsrht_wait(bsrht_server* sv, uint64_t ticket, int64_t timeout_us) {
  if (!sv || timeout_us < 0) return BSRHT_EINVAL;
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return BSRHT_EINVAL;
  Req* q = it->second.get();
  if (!sv->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), [&] { return q->done; }))
    return BSRHT_ETIMEDOUT;
  return q->status;
}

int bsrht_request_times(bsrht_server* sv, uint64_t ticket, double* submit_s, double* done_s) {
  if (!sv || !submit_s || !done_s) return BSRHT_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return BSRHT_EINVAL;
  *submit_s = it->second->t_submit;
  *done_s = it->second->done ? it->second->t_done : -1.0;
  return BSRHT_OK;
}

int bsrht_server_stats_get(bsrht_server* sv, bsrht_server_stats* out) {
  if (!sv || !out) return BSRHT_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->failed = sv->failed;
  out->pending = sv->submitted - sv->completed;
  out->grouped_launches = sv->grouped_launches;
  out->grouped_requests = sv->grouped_requests;
  out->graph_launches = sv->graph_launches;
  out->tuned_classes = sv->tuned_count;
  out->pool_high_bytes = sv->alloc.high();
  if (!sv->lat_ms.empty()) {
    std::vector<double> v = sv->lat_ms;
    std::sort(v.begin(), v.end());
    // Nearest-rank percentiles.
    auto pct = [&](double p) {
      size_t rank = (size_t)std::ceil(p / 100.0 * (double)v.size());
      rank = std::min(std::max<size_t>(rank, 1), v.size());
      return v[rank - 1];
    };
    out->p50_ms = pct(50.0);
    out->p99_ms = pct(99.0);
    double s = 0.0;
    for (double x : v) s += x;
    out->mean_ms = s / (double)v.size();
    out->max_ms = v.back();
  }
  return BSRHT_OK;
}

int bsrht_server_destroy(bsrht_server* sv) {
  if (!sv) return BSRHT_EINVAL;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->threads) t.join();
  if (sv->pool) cudaFree(sv->pool);
  delete sv;
  return BSRHT_OK;
}

int bsrht_selftest_pool_allocator(uint64_t seed, int32_t steps) {
  // Reference model: a byte map of the pool (0 free, 1 live) checked against
  // the allocator after each step; first fit must return the lowest offset
  // of a free run that is long enough.
  const size_t cap = 256 * 97;
  FirstFit ff(cap);
  std::vector<uint8_t> model(cap / 256, 0);
  std::vector<std::pair<size_t, size_t>> live;
  uint64_t x = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto rnd = [&]() {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    return x;
  };
  int bad = 0;
  for (int it = 0; it < steps; ++it) {
    if (live.empty() || rnd() % 3 != 0) {
      const size_t units = 1 + rnd() % 12;
      const size_t off = ff.alloc(units * 256 - (rnd() % 256));
      size_t expect = kNone;
      for (size_t u = 0; u + units <= model.size() && expect == kNone; ++u) {
        bool fits = true;
        for (size_t k = 0; k < units && fits; ++k) fits = model[u + k] == 0;
        if (fits) expect = u * 256;
      }
      if (off != expect) ++bad;
      if (off != kNone) {
        for (size_t k = 0; k < units; ++k) model[off / 256 + k] = 1;
        live.push_back({off, units});
      }
    } else {
      const size_t i = rnd() % live.size();
      if (!ff.release(live[i].first)) ++bad;
      for (size_t k = 0; k < live[i].second; ++k) model[live[i].first / 256 + k] = 0;
      live.erase(live.begin() + (std::ptrdiff_t)i);
    }
    bad += ff.check();
    size_t used = 0;
    for (uint8_t b : model) used += b;
    if (used * 256 != ff.used()) ++bad;
  }
  if (ff.release(12345)) ++bad;  // unknown offset
  return bad;
}

}  // extern "C"
