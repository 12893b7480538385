// Launch counting and optional CUDA-event timing of selected kernel classes.
// Timing is off unless rr_profile_start enables classes; when on, an event
// pair brackets every launch of an enabled class on its own stream.  Safe to
// call from several host threads (independent factors objects driven
// concurrently): the counter is atomic, and an event pair is reserved under
// a lock by the thread that begins it and closed by the same thread.
#include <atomic>
#include <mutex>
#include <vector>

#include "rr_internal.cuh"

namespace {
unsigned g_mask = 0;
std::vector<cudaEvent_t> g_start[PROF_N], g_stop[PROF_N];
size_t g_used[PROF_N] = {0};
long long g_class_launches[PROF_N] = {0};
std::atomic<long long> g_launches{0};
std::mutex g_prof_mu;
thread_local size_t t_open[PROF_N];  // event pair this thread opened, per class

int g_suspended = 0;

// bounded-wait diagnostics (rr_debug_waits)
constexpr uint32_t kDefaultWaitTries = 1u << 22;
uint32_t g_wait_tries = kDefaultWaitTries;
int g_stall_launches = 0;
}  // namespace

uint32_t wait_tries() { return g_wait_tries; }

int take_stall() {
  if (g_stall_launches <= 0) return 0;
  --g_stall_launches;
  return 1;
}

extern "C" rr_status rr_debug_waits(unsigned tries, int stall_launches) {
  if (stall_launches < 0) {
    set_error("rr_debug_waits: stall_launches must be >= 0");
    return RR_ERR_ARG;
  }
  g_wait_tries = tries == 0 ? kDefaultWaitTries : tries;
  g_stall_launches = stall_launches;
  return RR_OK;
}

ProfSuspend::ProfSuspend() { ++g_suspended; }
ProfSuspend::~ProfSuspend() { --g_suspended; }

void prof_count(int n) {
  if (!g_suspended) g_launches += n;
}

void prof_begin(int cls, cudaStream_t st) {
  if (g_suspended) return;
  g_launches += 1;
  if (!(g_mask & (1u << cls))) return;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  g_class_launches[cls] += 1;
  t_open[cls] = static_cast<size_t>(-1);  // no pair unless the events exist
  size_t i = g_used[cls];
  if (i >= g_start[cls].size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
    g_start[cls].push_back(a);
    g_stop[cls].push_back(b);
  }
  cudaEventRecord(g_start[cls][i], st);
  g_used[cls] = i + 1;  // reserved: this thread's prof_end closes pair i
  t_open[cls] = i;
}

void prof_end(int cls, cudaStream_t st) {
  if (g_suspended || !(g_mask & (1u << cls))) return;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  const size_t i = t_open[cls];
  if (i >= g_stop[cls].size()) return;
  cudaEventRecord(g_stop[cls][i], st);
}

extern "C" rr_status rr_profile_start(unsigned mask) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  g_mask = mask;
  for (int c = 0; c < PROF_N; ++c) {
    g_used[c] = 0;
    g_class_launches[c] = 0;
  }
  g_launches = 0;
  return RR_OK;
}

extern "C" rr_status rr_profile_read(int cls, double* ms, long long* launches) {
  if (cls < 0 || cls >= PROF_N) {
    set_error("rr_profile_read: unknown kernel class");
    return RR_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_prof_mu);
  double total = 0.0;
  for (size_t i = 0; i < g_used[cls]; ++i) {
    cudaError_t e = cudaEventSynchronize(g_stop[cls][i]);
    if (e != cudaSuccess) return cuda_status(e, "rr_profile_read");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, g_start[cls][i], g_stop[cls][i]);
    if (e != cudaSuccess) return cuda_status(e, "rr_profile_read");
    total += t;
  }
  if (ms) *ms = total;
  if (launches) *launches = g_class_launches[cls];
  return RR_OK;
}

extern "C" long long rr_launch_count(void) { return g_launches.load(); }
