// Status word, error strings, launch statistics of libtnrsvd.so.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "tnr_internal.cuh"

namespace tnr {

// One device status word per host thread slot: slot 0 serves ordinary callers, the batched
// solver gives each of its workers its own slot, so concurrent solves on different streams never
// see (or clear) one another's errors.
static __device__ int g_status_words[kStatusSlots];
static thread_local int t_status_slot = 0;

void set_status_slot(int slot) { t_status_slot = (slot >= 0 && slot < kStatusSlots) ? slot : 0; }

int *status_ptr() {
  static int *cache[kMaxDevices] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  int *base = nullptr;
  {
    std::lock_guard<std::mutex> g(mu);
    if (!cache[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_status_words) != cudaSuccess) return nullptr;
      cache[dev] = static_cast<int *>(p);
    }
    base = cache[dev];
  }
  return base + t_status_slot;
}

// The dynamic shared-memory limit set by cudaFuncSetAttribute belongs to the kernel, not to a
// launch: every host thread shares it. Lowering it while another thread is about to launch the
// same kernel with more shared memory makes that launch fail, so the limit only ever goes up.
// The default limit is 48 KB minus the kernel's static shared memory, so every size is checked.
int ensure_dynamic_smem(const void *func, size_t bytes) {
  if (bytes == 0) return TNR_OK;
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, size_t> raised;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TNR_ECUDA;
  std::lock_guard<std::mutex> g(mu);
  size_t &cur = raised[{dev, func}];
  if (cur >= bytes) return TNR_OK;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return check_cuda(e);
  cur = bytes;
  return TNR_OK;
}

int check_cuda_at(cudaError_t e, const char *file, int line) {
  if (e == cudaSuccess) return TNR_OK;
  const char *base = strrchr(file, '/');
  fprintf(stderr, "libtnrsvd: CUDA error %d (%s) at %s:%d\n", (int)e, cudaGetErrorString(e), base ? base + 1 : file,
          line);
  return TNR_ECUDA;
}

int check_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TNR_OK;
  fprintf(stderr, "libtnrsvd: CUDA error %d (%s)\n", (int)e, cudaGetErrorString(e));
  return TNR_ECUDA;
}

// Per host thread pinned staging for read-backs: copies into pinned memory stay asynchronous, so
// several read-backs and the status word cost one synchronisation instead of one each.
namespace {
struct PinnedStage {
  void *p = nullptr;
  size_t bytes = 0;
  ~PinnedStage() {
    if (p) cudaFreeHost(p);
  }
  void *get(size_t need) {
    if (need > bytes) {
      if (p) cudaFreeHost(p);
      p = nullptr;
      bytes = 0;
      const size_t want = need < 4096 ? 4096 : need;
      if (cudaHostAlloc(&p, want, cudaHostAllocDefault) != cudaSuccess) return nullptr;
      bytes = want;
    }
    return p;
  }
};
thread_local PinnedStage t_stage;
}  // namespace

int read_back_unstaged(cudaStream_t s, const ReadBack *items, int n) {
  int *st = status_ptr();
  if (!st) return TNR_ECUDA;
  for (int i = 0; i < n; ++i)
    TNR_CK(cudaMemcpyAsync(items[i].dst, items[i].src, items[i].bytes, cudaMemcpyDeviceToHost, s));
  int h = 0;
  TNR_CK(cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, s));
  TNR_CK(cudaStreamSynchronize(s));
  if (h != 0) TNR_CK(cudaMemsetAsync(st, 0, sizeof(int), s));
  return h;
}

int read_back(cudaStream_t s, const ReadBack *items, int n) {
  int *st = status_ptr();
  if (!st) return TNR_ECUDA;
  size_t total = sizeof(int);
  for (int i = 0; i < n; ++i) total += (items[i].bytes + 15) & ~size_t(15);
  char *stage = static_cast<char *>(t_stage.get(total));
  if (!stage) return read_back_unstaged(s, items, n);  // no pinned memory: plain copies
  size_t off = sizeof(int);
  for (int i = 0; i < n; ++i) {
    TNR_CK(cudaMemcpyAsync(stage + off, items[i].src, items[i].bytes, cudaMemcpyDeviceToHost, s));
    off += (items[i].bytes + 15) & ~size_t(15);
  }
  TNR_CK(cudaMemcpyAsync(stage, st, sizeof(int), cudaMemcpyDeviceToHost, s));
  TNR_CK(cudaStreamSynchronize(s));
  off = sizeof(int);
  for (int i = 0; i < n; ++i) {
    memcpy(items[i].dst, stage + off, items[i].bytes);
    off += (items[i].bytes + 15) & ~size_t(15);
  }
  int h = 0;
  memcpy(&h, stage, sizeof(int));
  if (h != 0) {  // clear the word for the next call (rare path)
    TNR_CK(cudaMemsetAsync(st, 0, sizeof(int), s));
    TNR_CK(cudaStreamSynchronize(s));
  }
  return h;
}

int read_status(cudaStream_t s) { return read_back(s, nullptr, 0); }

int reset_status(cudaStream_t s) {
  int *p = status_ptr();
  if (!p) return TNR_ECUDA;
  TNR_CK(cudaMemsetAsync(p, 0, sizeof(int), s));
  return TNR_OK;
}

// ---- launch statistics ----
namespace {
struct Stats {
  std::mutex mu;
  int32_t mask = 0;
  int64_t launches[K_NUM_CLASSES] = {0};
  double ms[K_NUM_CLASSES] = {0};
  double work[K_NUM_CLASSES] = {0};
  std::vector<cudaEvent_t> pool;
  struct Pending {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void drain() {
    for (auto &p : pending) {
      float t = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess)
        ms[p.cls] += t;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
};
Stats &S() {
  static Stats s;
  return s;
}
// the event opened by stats_begin, per host thread (each thread launches on its own stream)
thread_local cudaEvent_t t_open_ev[K_NUM_CLASSES] = {nullptr};
const char *kNames[K_NUM_CLASSES] = {"conv_rowptr", "conv_flags", "conv_scan", "conv_fill", "omega", "merge",
                                     "contract",    "contract_tc", "gemm",     "qr",        "qr_small", "qr_piv", "svd", "misc", "round", "diff", "batch"};
}  // namespace

void stats_begin(int cls, cudaStream_t s) {
  Stats &st = S();
  std::lock_guard<std::mutex> g(st.mu);
  st.launches[cls] += 1;
  if (st.mask & (1 << cls)) {
    cudaEvent_t a = st.take();
    cudaEventRecord(a, s);
    t_open_ev[cls] = a;
  }
}

void stats_work(int cls, double w) {
  Stats &st = S();
  std::lock_guard<std::mutex> g(st.mu);
  st.work[cls] += w;
}

void stats_end(int cls, cudaStream_t s) {
  Stats &st = S();
  std::lock_guard<std::mutex> g(st.mu);
  if ((st.mask & (1 << cls)) && t_open_ev[cls]) {
    cudaEvent_t b = st.take();
    cudaEventRecord(b, s);
    st.pending.push_back({cls, t_open_ev[cls], b});
    t_open_ev[cls] = nullptr;
    if (st.pending.size() > 4096) st.drain();
  }
}

}  // namespace tnr

extern "C" {

void tnr_stats_enable(int32_t class_mask) {
  tnr::Stats &st = tnr::S();
  std::lock_guard<std::mutex> g(st.mu);
  st.mask = class_mask;
}

void tnr_stats_reset(void) {
  tnr::Stats &st = tnr::S();
  std::lock_guard<std::mutex> g(st.mu);
  st.drain();
  for (int i = 0; i < tnr::K_NUM_CLASSES; ++i) {
    st.launches[i] = 0;
    st.ms[i] = 0;
    st.work[i] = 0;
  }
}

int tnr_stats(int32_t cls, int64_t *launches, double *ms) {
  tnr::Stats &st = tnr::S();
  std::lock_guard<std::mutex> g(st.mu);
  st.drain();
  if (cls < -1 || cls >= tnr::K_NUM_CLASSES) return TNR_EINVAL;
  int64_t L = 0;
  double T = 0;
  for (int i = 0; i < tnr::K_NUM_CLASSES; ++i) {
    if (cls == -1 || cls == i) {
      L += st.launches[i];
      T += st.ms[i];
    }
  }
  if (launches) *launches = L;
  if (ms) *ms = T;
  return TNR_OK;
}

int tnr_stats_work(int32_t cls, double *work) {
  tnr::Stats &st = tnr::S();
  std::lock_guard<std::mutex> g(st.mu);
  if (cls < -1 || cls >= tnr::K_NUM_CLASSES || !work) return TNR_EINVAL;
  double w = 0;
  for (int i = 0; i < tnr::K_NUM_CLASSES; ++i)
    if (cls == -1 || cls == i) w += st.work[i];
  *work = w;
  return TNR_OK;
}

const char *tnr_stats_class_name(int32_t cls) {
  if (cls < 0 || cls >= tnr::K_NUM_CLASSES) return nullptr;
  return tnr::kNames[cls];
}

const char *tnr_strerror(int status) {
  switch (status) {
    case TNR_OK: return "ok";
    case TNR_EINVAL: return "invalid argument (dims, ranks, sizes or pointers)";
    case TNR_EDUP: return "duplicate (row, col) entry in the COO input";
    case TNR_ENOTSORTED: return "COO input not sorted by (row, col)";
    case TNR_ENONFINITE: return "non-finite value in device data";
    case TNR_ENOMEM: return "workspace or output capacity too small";
    case TNR_ECUDA: return "CUDA runtime error";
    case TNR_ETIMEOUT: return "bounded device wait ran out";
    case TNR_ERANGE: return "index or count outside the supported range";
    default: return "unknown status";
  }
}

int tnr_version(void) { return 1; }

}  // extern "C"
