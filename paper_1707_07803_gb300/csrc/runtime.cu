// Status word, error strings, launch statistics of libtnrsvd.so.
#include <cstdio>
#include <mutex>
#include <vector>

#include "tnr_internal.cuh"

namespace tnr {

static __device__ int g_status_word;

int *status_ptr() {
  static int *cache[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!cache[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
    cache[dev] = static_cast<int *>(p);
  }
  return cache[dev];
}

int check_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TNR_OK;
  fprintf(stderr, "libtnrsvd: CUDA error %d (%s)\n", (int)e, cudaGetErrorString(e));
  return TNR_ECUDA;
}

int read_status(cudaStream_t s) {
  int *p = status_ptr();
  if (!p) return TNR_ECUDA;
  int h = 0;
  TNR_CK(cudaMemcpyAsync(&h, p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TNR_CK(cudaStreamSynchronize(s));
  if (h != 0) {
    int zero = 0;
    TNR_CK(cudaMemcpyAsync(p, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    TNR_CK(cudaStreamSynchronize(s));
  }
  return h;
}

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
  cudaEvent_t open_ev[K_NUM_CLASSES] = {nullptr};
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
const char *kNames[K_NUM_CLASSES] = {"conv_rowptr", "conv_flags", "conv_scan", "conv_fill", "omega", "merge",
                                     "contract",    "contract_tc", "gemm",     "qr",        "qr_small", "qr_piv", "svd", "misc", "round"};
}  // namespace

void stats_begin(int cls, cudaStream_t s) {
  Stats &st = S();
  std::lock_guard<std::mutex> g(st.mu);
  st.launches[cls] += 1;
  if (st.mask & (1 << cls)) {
    cudaEvent_t a = st.take();
    cudaEventRecord(a, s);
    st.open_ev[cls] = a;
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
  if ((st.mask & (1 << cls)) && st.open_ev[cls]) {
    cudaEvent_t b = st.take();
    cudaEventRecord(b, s);
    st.pending.push_back({cls, st.open_ev[cls], b});
    st.open_ev[cls] = nullptr;
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
