// Merged BF16x4 GEMM launches across contexts that run at the same time (served
// requests, each on its own stream): the H_eff stages of several requests go out as
// one persistent launch over the concatenated tile lists.
//
// Flat combining: a context that wants a GEMM records a "ready" event on its own
// stream and queues its tile list.  If no launch is being assembled, it becomes the
// launcher: it takes up to EXACT_MAX_SLICES queued lists (its own and whatever other
// contexts queued meanwhile, oldest first), makes the merger's stream wait for their
// ready events, launches once and records a "finished" event; every context whose
// list went out makes its own stream wait for that event before its next kernel.
// A context that finds a launch in progress waits until its list has gone out (in
// that launch or the next).  Nothing waits for company: a context alone launches at
// once on its own stream.  A merged launch does wait for the prior work of every
// context in it (their ready events), which couples the requests it carries.  Every tile is
// computed the same way in any launch, so results do not depend on the merging.
#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>

#include "engine.hpp"
#include "kernels.hpp"

namespace tdvp {
namespace {

struct Pending {
  ExactSlice slice;
  int ntiles = 0;
  cudaEvent_t ready = nullptr;
  std::shared_ptr<CUevent_st> finished;  // set when the list has been launched
  bool done = false;
  int rc = 0;
};

struct Merger {
  std::mutex m;
  std::condition_variable cv;
  std::deque<Pending*> queue;
  bool assembling = false;
  cudaStream_t stream = nullptr;
};

Merger g_merger[64];
std::atomic<long long> g_merged_launches{0}, g_merged_slices{0};

thread_local bool t_merge = false;

}  // namespace

bool& merge_launches_here() { return t_merge; }

void merge_counts(long long* launches, long long* slices) {
  if (launches) *launches = g_merged_launches.load();
  if (slices) *slices = g_merged_slices.load();
}

void launch_exact_merged_or_alone(const ExactSlice& slice, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return;
  int dev = 0;
  TDVP_CUDA(cudaGetDevice(&dev));
  if (!t_merge || dev < 0 || dev >= 64) {
    ExactLaunch L{};
    L.nslices = 1;
    L.start[0] = 0;
    L.start[1] = ntiles;
    L.sl[0] = slice;
    launch_gemm_exact_merged(L, s);
    return;
  }
  Merger& M = g_merger[dev];
  Pending me;
  me.slice = slice;
  me.ntiles = ntiles;
  TDVP_CUDA(cudaEventCreateWithFlags(&me.ready, cudaEventDisableTiming));
  TDVP_CUDA(cudaEventRecord(me.ready, s));
  std::unique_lock<std::mutex> lk(M.m);
  if (!M.stream && cudaStreamCreateWithFlags(&M.stream, cudaStreamNonBlocking) != cudaSuccess) {
    lk.unlock();
    cudaEventDestroy(me.ready);
    throw Error(-6, "could not create the merged-launch stream");
  }
  M.queue.push_back(&me);
  while (!me.done) {
    if (M.assembling) {
      M.cv.wait(lk);
      continue;
    }
    // become the launcher for the oldest queued lists
    M.assembling = true;
    std::vector<Pending*> batch;
    while (!M.queue.empty() && (int)batch.size() < EXACT_MAX_SLICES) {
      batch.push_back(M.queue.front());
      M.queue.pop_front();
    }
    lk.unlock();
    int rc = 0;
    if (batch.size() == 1 && batch[0] == &me) {  // alone: launch on the context's own stream
      ExactLaunch L1{};
      L1.nslices = 1;
      L1.start[0] = 0;
      L1.start[1] = ntiles;
      L1.sl[0] = slice;
      launch_gemm_exact_merged(L1, s);
      if (cudaGetLastError() != cudaSuccess) rc = -6;
      lk.lock();
      me.rc = rc;
      me.done = true;
      M.assembling = false;
      M.cv.notify_all();
      continue;
    }
    ExactLaunch L{};
    L.nslices = (int)batch.size();
    L.start[0] = 0;
    for (int i = 0; i < L.nslices; ++i) {
      L.sl[i] = batch[i]->slice;
      L.start[i + 1] = L.start[i] + batch[i]->ntiles;
      if (cudaStreamWaitEvent(M.stream, batch[i]->ready, 0) != cudaSuccess) rc = -6;
    }
    cudaEvent_t fin = nullptr;
    if (rc == 0) {
      launch_gemm_exact_merged(L, M.stream);
      if (cudaGetLastError() != cudaSuccess) rc = -6;
    }
    if (rc == 0 && cudaEventCreateWithFlags(&fin, cudaEventDisableTiming) != cudaSuccess) rc = -6;
    if (rc == 0 && cudaEventRecord(fin, M.stream) != cudaSuccess) rc = -6;
    std::shared_ptr<CUevent_st> shared(fin, [](cudaEvent_t e) {
      if (e) cudaEventDestroy(e);
    });
    if (L.nslices > 1) {
      g_merged_launches.fetch_add(1);
      g_merged_slices.fetch_add(L.nslices);
    }
    lk.lock();
    for (Pending* p : batch) {
      p->finished = shared;
      p->rc = rc;
      p->done = true;
    }
    M.assembling = false;
    M.cv.notify_all();
  }
  lk.unlock();
  cudaEventDestroy(me.ready);  // its wait is enqueued; destruction is deferred until done
  if (me.rc != 0) throw Error(me.rc, "merged BF16x4 launch failed");
  if (me.finished) TDVP_CUDA(cudaStreamWaitEvent(s, me.finished.get(), 0));
}

}  // namespace tdvp
