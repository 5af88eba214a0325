// Instrumentation: process-wide kernel-launch counter and CUDA-event timing of the
// Kronecker-sum GEMM applies and of the split Bregman vector kernels (recorded on the
// stream each one runs on, by category).
#include <stdio.h>
#include <stdlib.h>

#include <atomic>
#include <chrono>
#include <mutex>
#include <vector>

#include "kpsb_internal.cuh"

namespace kpsb {

static std::atomic<unsigned long long> g_launches{0};
static thread_local bool t_capturing = false;

void count_launch(long long n) {
  if (t_capturing && n == 1) return;
  g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed);
}

void set_capture_mode(bool on) { t_capturing = on; }

// Host phase trace: with KPSB_TRACE set in the environment, each call prints one stderr line
// "[kpsb trace] <seconds since the first trace> <stream> <phase>".
void trace(cudaStream_t st, const char* phase) {
  static const bool on = getenv("KPSB_TRACE") != nullptr;
  if (!on) return;
  using clk = std::chrono::steady_clock;
  static const clk::time_point t0 = clk::now();
  const double t = std::chrono::duration<double>(clk::now() - t0).count();
  fprintf(stderr, "[kpsb trace] %.6f %p %s\n", t, (void*)st, phase);
}

namespace {
struct TimerRec {
  cudaEvent_t a = nullptr, b = nullptr;
  double flops = 0.0;
  int launches = 0;
  int cat = 0;
  bool used = false;
};
std::mutex g_tm;
bool g_timing = false;
std::vector<TimerRec> g_recs;
size_t g_next = 0;
}  // namespace

bool gemm_timing_enabled() {
  std::lock_guard<std::mutex> lk(g_tm);
  return g_timing;
}

int timer_begin(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_tm);
  if (!g_timing) return -1;
  if (g_next == g_recs.size()) {
    TimerRec r;
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return -1;
    g_recs.push_back(r);
  }
  int slot = (int)g_next++;
  cudaEventRecord(g_recs[slot].a, st);
  return slot;
}

int gemm_timer_begin(cudaStream_t st) { return timer_begin(st); }

void timer_end(int slot, cudaStream_t st, int cat, double flops, int launches) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_tm);
  if (slot >= (int)g_recs.size()) return;
  TimerRec& r = g_recs[slot];
  cudaEventRecord(r.b, st);
  r.flops = flops;
  r.launches = launches;
  r.cat = cat;
  r.used = true;
}

void timer_set_value(int slot, double v) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_tm);
  if (slot < (int)g_recs.size()) g_recs[slot].flops = v;
}

void gemm_timer_end(int slot, cudaStream_t st, double flops, int launches) {
  timer_end(slot, st, TIMER_KP_APPLY, flops, launches);
}

}  // namespace kpsb

using namespace kpsb;

extern "C" unsigned long long kpsb_kernel_launches(void) { return g_launches.load(); }

extern "C" kpsb_status kpsb_gemm_timing(int enable) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_tm);
  g_timing = enable != 0;
  if (g_timing) {
    g_next = 0;
    for (auto& r : g_recs) r.used = false;
    KPSB_TRY(simt_work(nullptr, true));
    KPSB_TRY(tc_work(nullptr, true));
  }
  return KPSB_OK;
}

extern "C" kpsb_status kpsb_apply_counts(unsigned long long* problem_applies, unsigned long long* kn3) {
  clear_error();
  unsigned long long a[2] = {0, 0}, b[2] = {0, 0};
  KPSB_TRY(simt_work(a, false));
  KPSB_TRY(tc_work(b, false));
  if (kn3) *kn3 = a[0] + b[0];
  if (problem_applies) *problem_applies = a[1] + b[1];
  return KPSB_OK;
}

extern "C" kpsb_status kpsb_timer_stats(int category, unsigned long long* launches, double* ms,
                                        double* flops) {
  clear_error();
  KPSB_REQUIRE(category >= 0 && category < TIMER_CATEGORIES, "unknown timer category %d", category);
  std::lock_guard<std::mutex> lk(g_tm);
  unsigned long long L = 0;
  double T = 0.0, F = 0.0;
  for (size_t i = 0; i < g_next && i < g_recs.size(); ++i) {
    TimerRec& r = g_recs[i];
    if (!r.used || r.cat != category) continue;
    KPSB_TRY_CUDA(cudaEventSynchronize(r.b));
    float t = 0.f;
    KPSB_TRY_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    T += t;
    F += r.flops;
    L += r.launches;
  }
  if (category == TIMER_KP_APPLY) {
    // flops the applies performed: 4 k n^3 per active problem (device counters), so
    // problems whose CGLS has stopped count nothing
    unsigned long long a[2] = {0, 0}, b[2] = {0, 0};
    KPSB_TRY(simt_work(a, false));
    KPSB_TRY(tc_work(b, false));
    F = 4.0 * (double)(a[0] + b[0]);
  }
  if (launches) *launches = L;
  if (ms) *ms = T;
  if (flops) *flops = F;
  return KPSB_OK;
}

extern "C" kpsb_status kpsb_gemm_stats(unsigned long long* launches, double* ms, double* flops) {
  return kpsb_timer_stats(TIMER_KP_APPLY, launches, ms, flops);
}
