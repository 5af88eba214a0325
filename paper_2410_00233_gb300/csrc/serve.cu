// Serving loop: continuous batching of deblur requests on one GPU.
//
// Requests are admitted while device memory (a caller-given budget) and slots allow; a
// builder thread provides their KP factors (TSVD of R(A) + Terms), from a cache keyed by
// the PSF when the same PSF was seen before; a worker thread keeps the split Bregman state
// of every admitted request resident and advances all of them together, a few outer steps
// per round (each (image size, precision) group on its own stream, the groups at the same
// time), so requests that arrive while others run join at the next round and finished
// ones leave.  Each request's arithmetic is exactly that of sb_solve alone: the kernels
// are per problem and their reductions have a fixed order, and splitting the outer steps
// into rounds changes nothing.
#include <stdio.h>
#include <stdlib.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <string>
#include <thread>
#include <unordered_map>

#include "kpsb_internal.cuh"

namespace kpsb {

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Optional event log on stderr (environment variable KPSB_SERVER_LOG=1).
static bool srv_log_on() {
  static int on = -1;
  if (on < 0) {
    const char* v = getenv("KPSB_SERVER_LOG");
    on = (v && v[0] == '1') ? 1 : 0;
  }
  return on == 1;
}
#define SRV_LOG(...)                                               \
  do {                                                             \
    if (srv_log_on()) {                                            \
      fprintf(stderr, "[kpsb server %.3f] ", now_s());             \
      fprintf(stderr, __VA_ARGS__);                                \
      fprintf(stderr, "\n");                                       \
    }                                                              \
  } while (0)

enum { RQ_QUEUED = 0, RQ_BUILDING, RQ_READY, RQ_RUNNING, RQ_DONE, RQ_FAILED };

struct SrvReq {
  uint64_t id = 0;
  kpsb_request r{};
  std::vector<double> psf, b;
  uint64_t key = 0;
  int state = RQ_QUEUED;
  kpsb_status status = KPSB_OK;
  std::string err;
  kpsb_kp* kp = nullptr;
  size_t reserved = 0;      // bytes reserved for the request's device state
  size_t res_factor = 0;    // bytes reserved for factors (until they exist or are found cached)
  double* dev = nullptr;    // device b and x
  SBState sb;
  std::vector<double> x;
  kpsb_sb_stats stats{};
  double t_submit = 0.0, t_done = 0.0;
};

struct CacheEnt {
  kpsb_kp* kp = nullptr;
  size_t bytes = 0;
  int refs = 0;
  uint64_t last_use = 0;
};

}  // namespace kpsb

struct kpsb_server {
  size_t budget = 0;
  int max_active = 0;
  int round_steps = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_build, cv_done;
  bool stop = false;
  uint64_t next_id = 1, use_clock = 0;
  std::deque<kpsb::SrvReq*> queue;
  std::deque<kpsb::SrvReq*> to_build;
  std::vector<kpsb::SrvReq*> ready, active;
  std::unordered_map<uint64_t, kpsb::SrvReq*> all;
  std::unordered_map<uint64_t, kpsb::CacheEnt> cache;
  size_t used = 0, peak = 0;
  int resident = 0;  // admitted and not yet finished
  kpsb_srv_stats st{};
  std::thread worker, builder;
};

namespace kpsb {

static uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

static int est_k(const kpsb_request& r) { return r.rank_or_tol >= 1.0 ? (int)r.rank_or_tol : 30; }

// Device bytes of the factors of a handle (Ax, Ay; tensor-core tables when used).
static size_t factor_bytes(int n, int k, int prec) {
  size_t b = sizeof(float) * (size_t)2 * k * n * n;
  if (tc_supported(n, prec)) b += tc_table_bytes(n, k, prec);
  return b;
}

static size_t state_bytes(const kpsb_request& r) {
  return sb_state_bytes(r.n, est_k(r), r.prec) + sizeof(double) * (size_t)2 * r.n * r.n + 512;
}

static void account(kpsb_server* s, long long delta) {
  s->used = (size_t)((long long)s->used + delta);
  s->peak = std::max(s->peak, s->used);
}

// Evict unreferenced cache entries (least recently used first) until `need` more bytes fit.
static void evict_for(kpsb_server* s, size_t need, std::vector<kpsb_kp*>& freed) {
  while (s->used + need > s->budget) {
    uint64_t best = 0, bl = UINT64_MAX;
    bool found = false;
    for (auto& kv : s->cache)
      if (kv.second.refs == 0 && kv.second.last_use < bl) {
        bl = kv.second.last_use;
        best = kv.first;
        found = true;
      }
    if (!found) return;
    CacheEnt e = s->cache[best];
    s->cache.erase(best);
    account(s, -(long long)e.bytes);
    freed.push_back(e.kp);
  }
}

static void fail(kpsb_server* s, SrvReq* q, kpsb_status code, const std::string& msg) {
  if (q->state != RQ_QUEUED) s->resident--;
  q->state = RQ_FAILED;
  q->status = code;
  q->err = msg;
  q->t_done = now_s();
  s->st.failed++;
  s->cv_done.notify_all();
}

// Builder: factors for admitted requests (cache hit or kp_build).
static void builder_main(kpsb_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    SrvReq* q = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_build.wait(lk, [&] { return s->stop || !s->to_build.empty(); });
      if (s->stop) break;
      q = s->to_build.front();
      s->to_build.pop_front();
      auto it = s->cache.find(q->key);
      if (it != s->cache.end()) {
        it->second.refs++;
        it->second.last_use = ++s->use_clock;
        q->kp = it->second.kp;
        s->st.cache_hits++;
        account(s, -(long long)q->res_factor);  // the factors exist already
        q->res_factor = 0;
        q->state = RQ_READY;
        s->ready.push_back(q);
        s->cv_work.notify_all();
        continue;
      }
    }
    kpsb_build_opts o;
    memset(&o, 0, sizeof(o));
    o.stream = st;
    o.seed = q->key;
    kpsb_kp* kp = nullptr;
    SRV_LOG("build start id=%llu n=%d", (unsigned long long)q->id, q->r.n);
    kpsb_status bs = kp_build(q->psf.data(), q->r.s0, q->r.s1, q->r.n, q->r.bc, q->r.rank_or_tol,
                              q->r.method, &o, &kp);
    std::string msg = bs ? std::string(kpsb_last_error()) : std::string();
    SRV_LOG("build done id=%llu status=%d %s", (unsigned long long)q->id, (int)bs, msg.c_str());
    std::lock_guard<std::mutex> lk(s->mu);
    if (bs != KPSB_OK) {
      account(s, -(long long)(q->reserved + q->res_factor));
      q->reserved = q->res_factor = 0;
      fail(s, q, bs, msg);
      s->cv_work.notify_all();
      continue;
    }
    s->st.cache_misses++;
    const size_t real = factor_bytes(kp->n, kp->k, q->r.prec);
    account(s, (long long)real - (long long)q->res_factor);  // reservation -> actual factor bytes
    q->res_factor = 0;
    CacheEnt& e = s->cache[q->key];
    if (e.kp) {  // another request built the same PSF meanwhile: keep the first
      account(s, -(long long)real);
      kp_free(kp);
    } else {
      e.kp = kp;
      e.bytes = real;
    }
    e.refs++;
    e.last_use = ++s->use_clock;
    q->kp = e.kp;
    q->state = RQ_READY;
    s->ready.push_back(q);
    s->cv_work.notify_all();
  }
  cudaStreamDestroy(st);
}

// Worker: admission, joining, rounds of split Bregman, retirement.
static void worker_main(kpsb_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::vector<cudaStream_t> gstreams;  // one per concurrently advanced (n, precision) group
  cudaEvent_t joined = nullptr;        // the joins of a round, awaited by every group stream
  cudaEventCreateWithFlags(&joined, cudaEventDisableTiming);
  for (;;) {
    std::vector<SrvReq*> joining;
    std::vector<kpsb_kp*> evicted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        return s->stop || !s->ready.empty() || !s->active.empty() ||
               (!s->queue.empty() && s->resident < s->max_active);
      });
      if (s->stop) break;
      // admission: FIFO while slots and memory allow
      while (!s->queue.empty()) {
        SrvReq* q = s->queue.front();
        if (s->resident >= s->max_active) break;
        const size_t sbytes = state_bytes(q->r);
        const size_t fbytes = s->cache.count(q->key) ? 0 : factor_bytes(q->r.n, est_k(q->r), q->r.prec);
        const size_t need = sbytes + fbytes;
        if (need > s->budget) {
          s->queue.pop_front();
          fail(s, q, KPSB_EBUSY, "request needs more device memory than the server budget");
          continue;
        }
        if (s->used + need > s->budget) evict_for(s, need, evicted);
        if (s->used + need > s->budget) break;  // wait for memory to free up
        s->queue.pop_front();
        SRV_LOG("admit id=%llu need=%zu used=%zu", (unsigned long long)q->id, need, s->used);
        q->reserved = sbytes;
        q->res_factor = fbytes;
        account(s, (long long)need);
        s->resident++;
        q->state = RQ_BUILDING;
        s->to_build.push_back(q);
        s->cv_build.notify_all();
      }
      joining.swap(s->ready);
      if (joining.empty() && s->active.empty()) {
        // nothing runnable yet (factors being built or memory held): wait briefly
        s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    for (kpsb_kp* kp : evicted) kp_free(kp);
    // join: device state of newly ready requests
    for (SrvReq* q : joining) {
      const size_t NN = (size_t)q->r.n * q->r.n;
      kpsb_sb_opts o;
      sb_fill_defaults(nullptr, o);
      o.prec = q->r.prec;
      double beta = q->r.beta > 0.0 ? q->r.beta : q->r.lambda * q->r.lambda / 2.0;
      kpsb_status js = KPSB_OK;
      cudaError_t e = cudaMallocAsync((void**)&q->dev, sizeof(double) * 2 * NN, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(q->dev, q->b.data(), sizeof(double) * NN, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) js = KPSB_ECUDA;
      if (js == KPSB_OK)
        js = sb_state_init(&q->sb, q->kp, q->dev, q->dev + NN, q->r.mu, q->r.lambda, beta, q->r.tv,
                           q->r.iters, o, st);
      std::lock_guard<std::mutex> lk(s->mu);
      if (js != KPSB_OK) {
        account(s, -(long long)q->reserved);
        q->reserved = 0;
        auto it = s->cache.find(q->key);
        if (it != s->cache.end() && it->second.kp == q->kp) it->second.refs--;
        fail(s, q, js, kpsb_last_error());
        continue;
      }
      q->state = RQ_RUNNING;
      s->active.push_back(q);
      SRV_LOG("joined id=%llu", (unsigned long long)q->id);
    }
    std::vector<SrvReq*> act;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      act = s->active;
    }
    if (act.empty()) continue;
    // one round: every (n, precision) group advances round_steps outer steps.  The groups
    // run at the same time, each on its own stream from its own host thread (small, latency-
    // bound groups overlap the large ones); they start after the joins queued on st.
    std::map<std::pair<int, int>, std::vector<SBState*>> groups;
    std::map<SBState*, SrvReq*> owner;
    for (SrvReq* q : act) {
      groups[{q->r.n, q->r.prec}].push_back(&q->sb);
      owner[&q->sb] = q;
    }
    std::vector<std::pair<std::pair<int, int>, std::vector<SBState*>>> glist(groups.begin(), groups.end());
    const size_t G = glist.size();
    std::vector<kpsb_status> gstat(G, KPSB_OK);
    std::vector<std::vector<kpsb_sb_stats>> gstats(G);
    std::vector<std::vector<int>> gdone(G);
    std::vector<std::string> gmsg(G);
    while (gstreams.size() < G) {
      cudaStream_t gs = nullptr;
      if (cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) != cudaSuccess) break;
      gstreams.push_back(gs);
    }
    cudaError_t je = cudaEventRecord(joined, st);
    auto run_group = [&](size_t gi) {
      cudaStream_t gs = gstreams.empty() ? st : gstreams[gi % gstreams.size()];
      std::vector<SBState*>& set = glist[gi].second;
      kpsb_sb_opts o;
      sb_fill_defaults(nullptr, o);
      o.prec = glist[gi].first.second;
      SRV_LOG("round start n=%d prec=%d count=%d", glist[gi].first.first, o.prec, (int)set.size());
      kpsb_status rs = je == cudaSuccess && cudaStreamWaitEvent(gs, joined, 0) == cudaSuccess ? KPSB_OK : KPSB_ECUDA;
      if (rs == KPSB_OK) rs = sb_advance(set.data(), (int)set.size(), s->round_steps, o, gs);
      SRV_LOG("round end status=%d %s", (int)rs, rs ? kpsb_last_error() : "");
      if (rs == KPSB_OK) rs = sb_state_read(set.data(), (int)set.size(), gstats[gi], gdone[gi], gs);
      if (rs == KPSB_OK && cudaStreamSynchronize(gs) != cudaSuccess) rs = KPSB_ECUDA;
      if (rs != KPSB_OK) gmsg[gi] = kpsb_last_error();
      gstat[gi] = rs;
    };
    if (G == 1 || gstreams.size() < G) {
      for (size_t gi = 0; gi < G; ++gi) run_group(gi);
    } else {
      std::vector<std::thread> th;
      for (size_t gi = 0; gi < G; ++gi)
        th.emplace_back([&, gi] {
          cudaSetDevice(s->device);
          run_group(gi);
        });
      for (auto& t : th) t.join();
    }
    // retirement (every group's work has completed: each thread synchronised its stream)
    for (size_t gi = 0; gi < G; ++gi) {
      kpsb_status rs = gstat[gi];
      const std::vector<SBState*>& set = glist[gi].second;
      for (size_t i = 0; i < set.size(); ++i) {
        SrvReq* q = owner[set[i]];
        if (rs == KPSB_OK && !gdone[gi][i]) continue;
        kpsb_status qs = rs;
        if (qs == KPSB_OK) {
          const size_t NN = (size_t)q->r.n * q->r.n;
          q->x.resize(NN);
          cudaError_t e = cudaMemcpyAsync(q->x.data(), q->dev + NN, sizeof(double) * NN, cudaMemcpyDeviceToHost, st);
          if (e == cudaSuccess) e = cudaStreamSynchronize(st);
          if (e != cudaSuccess) qs = KPSB_ECUDA;
          q->stats = gstats[gi][i];
        }
        sb_state_free(&q->sb, st);
        cudaFreeAsync(q->dev, st);
        q->dev = nullptr;
        std::lock_guard<std::mutex> lk(s->mu);
        account(s, -(long long)q->reserved);
        q->reserved = 0;
        auto it = s->cache.find(q->key);
        if (it != s->cache.end() && it->second.kp == q->kp) it->second.refs--;
        s->active.erase(std::find(s->active.begin(), s->active.end(), q));
        if (qs != KPSB_OK) {
          fail(s, q, qs, qs == rs ? gmsg[gi] : std::string("copying the result back failed"));
        } else {
          q->state = RQ_DONE;
          q->t_done = now_s();
          s->resident--;
          s->st.completed++;
          s->cv_done.notify_all();
        }
      }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.rounds++;
  }
  cudaStreamSynchronize(st);
  for (cudaStream_t gs : gstreams) cudaStreamDestroy(gs);
  if (joined) cudaEventDestroy(joined);
  cudaStreamDestroy(st);
}

}  // namespace kpsb

using namespace kpsb;

extern "C" kpsb_status srv_create(size_t budget_bytes, int max_active, int round_steps, kpsb_server_t* out) {
  clear_error();
  KPSB_REQUIRE(out, "null pointer");
  KPSB_REQUIRE(budget_bytes > 0 && max_active >= 1, "budget and max_active must be positive");
  kpsb_server* s = new (std::nothrow) kpsb_server();
  if (!s) {
    set_error("out of host memory");
    return KPSB_ENOMEM;
  }
  s->budget = budget_bytes;
  s->max_active = max_active;
  s->round_steps = round_steps > 0 ? round_steps : 5;
  cudaGetDevice(&s->device);
  s->worker = std::thread(worker_main, s);
  s->builder = std::thread(builder_main, s);
  *out = s;
  return KPSB_OK;
}

extern "C" kpsb_status srv_submit(kpsb_server_t s, const kpsb_request* r, unsigned long long* id) {
  clear_error();
  KPSB_REQUIRE(s && r && id && r->psf && r->b, "null pointer");
  KPSB_TRY(ra_check(r->s0, r->s1, r->n, r->bc));
  KPSB_REQUIRE(r->method == KPSB_EGKB || r->method == KPSB_RSVD, "unknown method %d", r->method);
  KPSB_REQUIRE(r->rank_or_tol > 0.0, "rank_or_tol must be > 0");
  KPSB_REQUIRE(r->mu > 0.0 && r->lambda > 0.0 && r->iters >= 1, "mu, lambda > 0 and iters >= 1 required");
  KPSB_REQUIRE(r->tv == KPSB_ANISO || r->tv == KPSB_ISO, "unknown TV type %d", r->tv);
  KPSB_REQUIRE(prec_valid(r->prec), "unknown precision %d", r->prec);
  SrvReq* q = new SrvReq();
  q->r = *r;
  q->psf.assign(r->psf, r->psf + (size_t)r->s0 * r->s1);
  q->b.assign(r->b, r->b + (size_t)r->n * r->n);
  q->r.psf = nullptr;
  q->r.b = nullptr;
  if (r->psf_key) {
    q->key = r->psf_key;
  } else {
    uint64_t h = fnv1a(q->psf.data(), sizeof(double) * q->psf.size());
    int meta[6] = {r->s0, r->s1, r->n, r->bc, r->method, r->prec};
    h = fnv1a(meta, sizeof(meta), h);
    h = fnv1a(&r->rank_or_tol, sizeof(double), h);
    q->key = h ? h : 1;
  }
  q->t_submit = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  q->id = s->next_id++;
  s->all[q->id] = q;
  s->queue.push_back(q);
  s->st.submitted++;
  *id = q->id;
  s->cv_work.notify_all();
  return KPSB_OK;
}

extern "C" kpsb_status srv_poll(kpsb_server_t s, unsigned long long id, long long timeout_us,
                                double* x_out, kpsb_sb_stats* stats, double* latency_s) {
  clear_error();
  KPSB_REQUIRE(s, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) {
    set_error("unknown request id %llu", id);
    return KPSB_ENOTFOUND;
  }
  SrvReq* q = it->second;
  auto pred = [&] { return q->state == RQ_DONE || q->state == RQ_FAILED; };
  if (timeout_us < 0)
    s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred))
    return KPSB_ETIMEOUT;
  kpsb_status code = q->state == RQ_DONE ? KPSB_OK : q->status;
  if (code == KPSB_OK) {
    if (x_out) memcpy(x_out, q->x.data(), sizeof(double) * q->x.size());
    if (stats) *stats = q->stats;
  } else {
    set_error("%s", q->err.c_str());
  }
  if (latency_s) *latency_s = q->t_done - q->t_submit;
  s->all.erase(it);
  delete q;
  return code;
}

extern "C" kpsb_status srv_stats(kpsb_server_t s, kpsb_srv_stats* out) {
  clear_error();
  KPSB_REQUIRE(s && out, "null pointer");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->bytes_in_use = s->used;
  out->peak_bytes = s->peak;
  out->active = (int)s->active.size();
  out->queued = (int)s->queue.size();
  out->cached = (int)s->cache.size();
  return KPSB_OK;
}

extern "C" void srv_destroy(kpsb_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_build.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->builder.joinable()) s->builder.join();
  cudaSetDevice(s->device);
  for (auto& kv : s->all) {
    SrvReq* q = kv.second;
    if (q->sb.mem) sb_state_free(&q->sb, nullptr);
    if (q->dev) cudaFreeAsync(q->dev, nullptr);
    delete q;
  }
  for (auto& kv : s->cache) kp_free(kv.second.kp);
  cudaDeviceSynchronize();
  delete s;
}
