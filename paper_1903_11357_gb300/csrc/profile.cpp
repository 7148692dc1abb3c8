// Per-kernel timing accumulators (CUDA events on the launching streams).
#include "profile.h"

#include <atomic>
#include <mutex>

#include "common.h"

namespace dgasm {

namespace {
std::atomic<int> g_on{0};
std::mutex g_mu;
double g_ms[PK_NKINDS] = {0};
long long g_n[PK_NKINDS] = {0};
}  // namespace

bool profiling() { return g_on.load() != 0; }
bool profiling(int kind) { return (g_on.load() >> kind) & 1; }

void prof_add(int kind, double ms, long long launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_ms[kind] += ms;
  g_n[kind] += launches;
}

EventPairs::~EventPairs() {
  for (auto e : a) cudaEventDestroy(e);
  for (auto e : b) cudaEventDestroy(e);
}

void EventPairs::reserve(size_t n) {
  while (a.size() < n) {
    cudaEvent_t x, y;
    if (cudaEventCreate(&x) != cudaSuccess) return;
    if (cudaEventCreate(&y) != cudaSuccess) { cudaEventDestroy(x); return; }
    a.push_back(x);
    b.push_back(y);
  }
}

int EventPairs::begin(int k, cudaStream_t s) {
  if (!profiling(k)) return -1;
  if (used == a.size()) {
    cudaEvent_t x, y;
    if (cudaEventCreate(&x) != cudaSuccess) return -1;
    if (cudaEventCreate(&y) != cudaSuccess) { cudaEventDestroy(x); return -1; }
    a.push_back(x);
    b.push_back(y);
  }
  kind.push_back(k);
  record(a[used], s);
  return (int)used++;
}

void EventPairs::end(int idx, cudaStream_t s) {
  if (idx >= 0) record(b[idx], s);
}

// inside a stream capture an event must be recorded as an external node to be timed later
void EventPairs::record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &st);
  if (st == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}

void EventPairs::accumulate() {
  for (size_t i = 0; i < used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a[i], b[i]) == cudaSuccess) prof_add(kind[i], ms, 1);
    else cudaGetLastError();
  }
}

}  // namespace dgasm

extern "C" int dgasm_profile_enable(int mask) {
  dgasm::g_on.store(mask & ((1 << dgasm::PK_NKINDS) - 1));
  return DGASM_OK;
}

extern "C" int dgasm_profile_read(int kind, double* total_ms, int64_t* launches, int reset) {
  using namespace dgasm;
  if (kind < 0 || kind >= PK_NKINDS) return set_error(DGASM_EINVAL, "profile kind %d out of range", kind);
  std::lock_guard<std::mutex> lk(g_mu);
  if (total_ms) *total_ms = g_ms[kind];
  if (launches) *launches = g_n[kind];
  if (reset) { g_ms[kind] = 0; g_n[kind] = 0; }
  return DGASM_OK;
}
