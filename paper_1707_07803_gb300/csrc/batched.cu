// Batched TNrSVD: many independent problems solved concurrently on one GPU.
//
// A single solve (Alg. 5.4 with Alg. 5.3) is a chain of short kernels, most of them one CTA,
// with a host round trip per bond for the ranks; on its own it keeps one or a few of the 152 SMs
// busy. Independent problems have no data in common, so the batch runs them side by side: a
// pool of host threads, each owning a CUDA stream, a workspace slice and a device status slot,
// pulls problem indices from an atomic counter and runs the ordinary solve on its stream. The
// GPU interleaves the workers' kernels; each worker's host round trips overlap the others' GPU
// work.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "tnr_internal.cuh"

namespace {

struct StreamSet {
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t start = nullptr;
  ~StreamSet() {
    for (auto s : streams)
      if (s) cudaStreamDestroy(s);
    for (auto e : done)
      if (e) cudaEventDestroy(e);
    if (start) cudaEventDestroy(start);
  }
};

}  // namespace

extern "C" int tnr_solve_batched(int32_t n, tnr_problem *probs, int32_t workers, void *ws, size_t ws_stride,
                                 void *stream) {
  if (n < 0 || (n > 0 && !probs) || workers < 0 || workers >= tnr::kStatusSlots) return TNR_EINVAL;
  if (n == 0) return TNR_OK;
  if (!ws || ws_stride == 0 || ws_stride % 256 != 0) return TNR_EINVAL;
  if (workers == 0) workers = std::min<int32_t>(n, 16);
  workers = std::min<int32_t>(workers, n);
  for (int32_t i = 0; i < n; ++i) probs[i].status = TNR_OK;
  int dev = 0;
  TNR_CK(cudaGetDevice(&dev));
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  StreamSet ss;
  ss.streams.assign(workers, nullptr);
  ss.done.assign(workers, nullptr);
  TNR_CK(cudaEventCreateWithFlags(&ss.start, cudaEventDisableTiming));
  TNR_CK(cudaEventRecord(ss.start, caller));
  for (int w = 0; w < workers; ++w) {
    TNR_CK(cudaStreamCreateWithFlags(&ss.streams[w], cudaStreamNonBlocking));
    TNR_CK(cudaEventCreateWithFlags(&ss.done[w], cudaEventDisableTiming));
    TNR_CK(cudaStreamWaitEvent(ss.streams[w], ss.start, 0));
  }
  std::atomic<int32_t> next{0};
  std::vector<int> worker_rc(workers, TNR_OK);
  auto body = [&](int w) {
    if (cudaSetDevice(dev) != cudaSuccess) {
      worker_rc[w] = TNR_ECUDA;
      return;
    }
    tnr::set_status_slot(1 + w);
    cudaStream_t s = ss.streams[w];
    worker_rc[w] = tnr::reset_status(s);  // a slot may hold an error left by an earlier batch
    char *slice = static_cast<char *>(ws) + static_cast<size_t>(w) * ws_stride;
    while (worker_rc[w] == TNR_OK) {
      const int32_t i = next.fetch_add(1);
      if (i >= n) break;
      tnr_problem &P = probs[i];
      P.status = tnr_solve(P.A, P.k, P.p, P.q, P.seed, &P.opts, P.U, P.S, P.V, slice, ws_stride, s);
      if (P.status != TNR_OK) tnr::reset_status(s);  // keep the slot clean for the next problem
    }
    if (cudaEventRecord(ss.done[w], s) != cudaSuccess) worker_rc[w] = TNR_ECUDA;
    tnr::set_status_slot(0);
  };
  // If a thread cannot be started, the workers already running drain the queue.
  std::vector<std::thread> pool;
  try {
    pool.reserve(workers);
    for (int w = 0; w < workers; ++w) pool.emplace_back(body, w);
  } catch (...) {
  }
  for (auto &t : pool) t.join();
  int batch_rc = pool.empty() ? TNR_ENOMEM : TNR_OK;
  for (size_t w = 0; w < pool.size(); ++w) {
    if (worker_rc[w] == TNR_OK)
      TNR_CK(cudaStreamWaitEvent(caller, ss.done[w], 0));
    else if (batch_rc == TNR_OK)
      batch_rc = worker_rc[w];
  }
  // problems no worker claimed (every worker stopped early) carry the reason
  for (int32_t i = std::min(next.load(), n); i < n; ++i) probs[i].status = batch_rc != TNR_OK ? batch_rc : TNR_ECUDA;
  for (int32_t i = 0; i < n; ++i)
    if (probs[i].status != TNR_OK) return probs[i].status;
  return TNR_OK;
}
