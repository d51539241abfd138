// Kernel-family timing for benchmarks: while enabled, each launch of an
// instrumented kernel family is bracketed by CUDA events on the stream it is
// launched on (inside captured CUDA graphs the events become event-record
// nodes and are read after every replay), and the kernels add the bytes they
// move for active right-hand sides to a device counter per family.
#include <mutex>
#include <vector>

#include "vie_internal.cuh"

namespace {

struct Pair {
  cudaEvent_t a = nullptr, b = nullptr;
  int family = 0;
};

struct Profiler {
  std::mutex mu;
  bool on = false;
  unsigned mask = 0;
  int epoch = 0;
  std::vector<Pair> pool;
  std::vector<Pair> pending;                 // direct launches since the last harvest
  double ms[VIE_PROF_FAMILIES] = {};
  long long launches[VIE_PROF_FAMILIES] = {};
  unsigned long long* d_bytes = nullptr;     // device counters [families]
};

Profiler& prof() {
  static Profiler p;
  return p;
}

thread_local std::vector<Pair>* t_capture_sink = nullptr;

const char* kNames[VIE_PROF_FAMILIES] = {"line_x",    "line_y",   "fused_tucker", "fused_stored",
                                         "line_iy",   "line_ix",  "tucker_rebuild", "arnoldi_dots",
                                         "arnoldi_update", "arnoldi_small", "fp64_vector", "setup",
                                         "matvec_fp64"};

void harvest(std::vector<Pair>& v, Profiler& p, bool recycle) {
  for (Pair& q : v) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess) {
      p.ms[q.family] += t;
      p.launches[q.family] += 1;
    } else {
      cudaGetLastError();
    }
    if (recycle) p.pool.push_back(q);
  }
  if (recycle) v.clear();
}

}  // namespace

unsigned long long* prof_bytes(int family) {
  Profiler& p = prof();
  return (p.on && p.d_bytes) ? p.d_bytes + family : nullptr;
}

int prof_epoch() { return prof().on ? prof().epoch : -1; }

int prof_begin(int family, cudaStream_t s) {
  Profiler& p = prof();
  if (!p.on || !(p.mask & (1u << family))) return -1;
  std::lock_guard<std::mutex> lk(p.mu);
  if (p.pool.empty()) {
    Pair q;
    if (cudaEventCreate(&q.a) != cudaSuccess || cudaEventCreate(&q.b) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    p.pool.push_back(q);
  }
  Pair q = p.pool.back();
  p.pool.pop_back();
  q.family = family;
  // inside a stream capture the record becomes an event node that is visible
  // outside the graph only with cudaEventRecordExternal
  if (t_capture_sink) cudaEventRecordWithFlags(q.a, s, cudaEventRecordExternal);
  else cudaEventRecord(q.a, s);
  std::vector<Pair>& dst = t_capture_sink ? *t_capture_sink : p.pending;
  dst.push_back(q);
  return (int)dst.size() - 1;
}

void prof_end(int handle, cudaStream_t s) {
  if (handle < 0) return;
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  std::vector<Pair>& dst = t_capture_sink ? *t_capture_sink : p.pending;
  if (handle < (int)dst.size()) {
    if (t_capture_sink) cudaEventRecordWithFlags(dst[handle].b, s, cudaEventRecordExternal);
    else cudaEventRecord(dst[handle].b, s);
  }
}

void prof_set_capture_sink(std::vector<ProfEventPair>* sink) {
  t_capture_sink = reinterpret_cast<std::vector<Pair>*>(sink);
}

// read the events of one replay of a captured graph (stream already synchronised)
void prof_harvest_graph(std::vector<ProfEventPair>& pairs) {
  Profiler& p = prof();
  if (!p.on) return;
  std::lock_guard<std::mutex> lk(p.mu);
  harvest(reinterpret_cast<std::vector<Pair>&>(pairs), p, false);
}

void prof_release_pairs(std::vector<ProfEventPair>& pairs) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  for (auto& q : reinterpret_cast<std::vector<Pair>&>(pairs)) p.pool.push_back(q);
  pairs.clear();
}

static_assert(sizeof(Pair) == sizeof(ProfEventPair), "event pair layout");

extern "C" {

int vie_profile_start(unsigned mask) {
  Profiler& p = prof();
  p.mask = mask;
  std::lock_guard<std::mutex> lk(p.mu);
  if (!p.d_bytes) {
    cudaError_t e = cudaMalloc(&p.d_bytes, VIE_PROF_FAMILIES * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_status(e, "profiler counters");
  }
  cudaError_t e = cudaMemset(p.d_bytes, 0, VIE_PROF_FAMILIES * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_status(e, "profiler counters");
  for (int f = 0; f < VIE_PROF_FAMILIES; ++f) {
    p.ms[f] = 0.0;
    p.launches[f] = 0;
  }
  // a graph captured without events must be captured again, and vice versa
  p.epoch += 1;
  p.on = true;
  return VIE_OK;
}

int vie_profile_stop(vie_profile_entry* out, int max_entries, int* count) {
  Profiler& p = prof();
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e, "profile stop");
  std::lock_guard<std::mutex> lk(p.mu);
  harvest(p.pending, p, true);
  unsigned long long bytes[VIE_PROF_FAMILIES] = {};
  if (p.d_bytes) cudaMemcpy(bytes, p.d_bytes, sizeof(bytes), cudaMemcpyDeviceToHost);
  int n = 0;
  for (int f = 0; f < VIE_PROF_FAMILIES && n < max_entries; ++f) {
    if (p.launches[f] == 0) continue;
    vie_profile_entry& r = out[n++];
    snprintf(r.name, sizeof(r.name), "%s", kNames[f]);
    r.launches = p.launches[f];
    r.ms = p.ms[f];
    r.bytes = (double)bytes[f];
  }
  if (count) *count = n;
  p.on = false;
  p.epoch += 1;
  return VIE_OK;
}

}  // extern "C"
