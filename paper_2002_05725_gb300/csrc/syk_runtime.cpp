// Runtime services of the library: work counters, CUDA-event timing of every
// apply_H launch, and a pinned host staging buffer for small device reads.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "syk_krylov.cuh"

namespace syk {
namespace {

std::atomic<int64_t> g_applies{0};
std::atomic<int64_t> g_bases{0};
std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_mv[kMvKinds];

struct Prof {
  std::mutex mtx;
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  std::vector<cudaEvent_t> pool;
  int64_t launches = 0;
  double total_ms = 0.0;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
Prof& prof() {
  static Prof* p = new Prof;  // never destroyed: events may outlive static teardown
  return *p;
}
thread_local cudaEvent_t t_start = nullptr;

}  // namespace

thread_local bool t_capturing = false;
thread_local int64_t t_cap_launches = 0, t_cap_applies = 0;
thread_local int64_t t_cap_mv[kMvKinds] = {};
std::atomic<uint64_t> g_epoch{1};
std::atomic<int> g_graphs{1};  // 0 off, 1 segment graphs, 2 device-driven evolutions

void count_applies(int64_t states) {
  if (t_capturing) t_cap_applies += states;
  else g_applies += states;
}
void count_bases(int64_t n) { g_bases += n; }
void count_launch(int64_t n) {
  if (t_capturing) t_cap_launches += n;
  else g_launches += n;
}
void count_matvec(int kind) {
  if (t_capturing) t_cap_mv[kind] += 1;
  else g_mv[kind] += 1;
}
void count_matvec_replay(const int64_t* kinds) {
  for (int k = 0; k < kMvKinds; ++k) g_mv[k] += kinds[k];
}
void capture_counts_begin() {
  t_capturing = true;
  t_cap_launches = t_cap_applies = 0;
  for (int k = 0; k < kMvKinds; ++k) t_cap_mv[k] = 0;
}
void capture_counts_end(int64_t* launches, int64_t* applies, int64_t* kinds) {
  t_capturing = false;
  *launches = t_cap_launches;
  *applies = t_cap_applies;
  for (int k = 0; k < kMvKinds; ++k) kinds[k] = t_cap_mv[k];
}
uint64_t graph_epoch() { return g_epoch.load(); }
void bump_graph_epoch() { ++g_epoch; }
bool graphs_enabled() { return g_graphs.load() != 0; }
bool device_chains_enabled() { return g_graphs.load() == 2; }

bool prof_enabled() {
  Prof& p = prof();
  std::lock_guard<std::mutex> lk(p.mtx);
  return p.on;
}

void prof_before_apply(cudaStream_t st) {
  Prof& p = prof();
  std::lock_guard<std::mutex> lk(p.mtx);
  if (!p.on) return;
  t_start = p.get();
  cudaEventRecord(t_start, st);
}

void prof_after_apply(cudaStream_t st) {
  Prof& p = prof();
  std::lock_guard<std::mutex> lk(p.mtx);
  if (!p.on || !t_start) return;
  cudaEvent_t e = p.get();
  cudaEventRecord(e, st);
  p.pending.emplace_back(t_start, e);
  t_start = nullptr;
}

// Accumulates every completed event pair (called after a synchronisation).
void prof_collect() {
  Prof& p = prof();
  std::lock_guard<std::mutex> lk(p.mtx);
  size_t keep = 0;
  for (size_t i = 0; i < p.pending.size(); ++i) {
    auto pr = p.pending[i];
    if (cudaEventQuery(pr.second) == cudaSuccess) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      p.total_ms += ms;
      p.launches += 1;
      p.pool.push_back(pr.first);
      p.pool.push_back(pr.second);
    } else {
      p.pending[keep++] = pr;
    }
  }
  p.pending.resize(keep);
}

int ensure_smem_limit(const void* func, int bytes) {
  static std::mutex mtx;
  static std::map<std::pair<const void*, int>, int> done;  // (kernel, device) -> limit set
  int dev = -1;
  SYK_CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mtx);
  int& cur = done[{func, dev}];
  if (bytes <= cur) return SYK_OK;
  SYK_CUDA_CHECK(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  cur = bytes;
  return SYK_OK;
}

int sm_count() {
  static std::atomic<int> cache[128] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return 1;
  int v = cache[dev].load();
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
  cache[dev] = v;
  return v;
}

void* pinned_scratch(size_t bytes) {
  static thread_local void* buf = nullptr;
  static thread_local size_t cap = 0;
  if (bytes > cap) {
    if (buf) cudaFreeHost(buf);
    cap = std::max<size_t>(bytes, 4096);
    if (cudaMallocHost(&buf, cap) != cudaSuccess) {
      buf = nullptr;
      cap = 0;
    }
  }
  return buf;
}

}  // namespace syk

extern "C" int syk_counters(int64_t* h_applies, int64_t* krylov_bases, int64_t* launches, int reset) {
  if (h_applies) *h_applies = syk::g_applies.load();
  if (krylov_bases) *krylov_bases = syk::g_bases.load();
  if (launches) *launches = syk::g_launches.load();
  if (reset) {
    syk::g_applies = 0;
    syk::g_bases = 0;
    syk::g_launches = 0;
  }
  return SYK_OK;
}

extern "C" int syk_matvec_launches(int64_t* rows, int64_t* tiled, int64_t* coset, int reset) {
  if (rows) *rows = syk::g_mv[syk::kMvRows].load();
  if (tiled) *tiled = syk::g_mv[syk::kMvTiled].load();
  if (coset) *coset = syk::g_mv[syk::kMvCoset].load();
  if (reset)
    for (int k = 0; k < syk::kMvKinds; ++k) syk::g_mv[k] = 0;
  return SYK_OK;
}

extern "C" int syk_use_graphs(int on) {
  if (on < 0 || on > 2) {
    syk::set_error("syk_use_graphs: mode must be 0, 1 or 2 (got %d)", on);
    return SYK_EINVAL;
  }
  syk::g_graphs = on;
  syk::bump_graph_epoch();
  return SYK_OK;
}

extern "C" int syk_profile_enable(int on) {
  syk::Prof& p = syk::prof();
  std::lock_guard<std::mutex> lk(p.mtx);
  p.on = on != 0;
  return SYK_OK;
}

extern "C" int syk_profile_read(int64_t* launches, double* total_ms, int reset) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    syk::set_error("syk_profile_read: %s", cudaGetErrorString(e));
    return SYK_ECUDA;
  }
  syk::prof_collect();
  syk::Prof& p = syk::prof();
  std::lock_guard<std::mutex> lk(p.mtx);
  if (launches) *launches = p.launches;
  if (total_ms) *total_ms = p.total_ms;
  if (reset) {
    p.launches = 0;
    p.total_ms = 0.0;
  }
  return SYK_OK;
}
