// Serving loop behind include/tdvp.h (tdvp_server_*): independent quench requests
// of the open Fermi-Hubbard chain (Eq. FHM from the Neel state of Eq. neel, or any
// product state) evolved concurrently on one GPU.
//
// Each request owns a context (its MPS, environments, plans and workspaces stay
// resident on the device for its whole run) and runs on one of max_active worker
// threads, each with its own non-blocking CUDA stream, so the kernels of different
// requests overlap on the device.  Admission is first in, first out: the head of the
// queue is admitted when a worker is free and its footprint estimate fits beside the
// estimates of the running requests within the HBM budget (and within the device's
// free memory).  A request that finishes releases its worker and its share of the
// budget at once, and the next one is admitted while the others keep running
// (continuous batching at request granularity).  Requests share no state, and every
// kernel is deterministic, so a result does not depend on what ran beside it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tdvp.h"

namespace tdvp {
void set_last_error(const char* msg);  // capi.cpp: message for tdvp_last_error()
}

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  tdvp_request r{};
  std::vector<int> occ;  // empty: Neel state
  int state = TDVP_REQ_QUEUED;
  int err = TDVP_OK;
  std::string msg;
  double need = 0;  // footprint estimate, bytes
  double t_submit = 0, t_admit = 0, t_done = 0;
  bool cancel = false;
  // results
  std::vector<double> n, sz, docc, ent;
  double energy = 0, chi_max = 0, steps = 0, heff_flops = 0, dev_peak = 0;
};

double footprint(const tdvp_request& r, int krylov_max) {
  // bytes of a context whose largest bond reaches chi_max (U(1)-equivalent):
  // complex128 blocks of the site tensors and both environments of every bond
  // (taken at the cap), and the two-site working set of one bond (theta, the
  // Krylov basis, the contraction intermediates and the split workspaces).  The
  // coefficients bound the device bytes measured on quenches of the Neel state
  // (U(1)xU(1), the larger of the two symmetries) with a factor of two to spare.
  const double chi = (double)std::max<long long>(r.chi_max, 1);
  const double kmax = (double)std::max(krylov_max, 1);
  return 16.0 * chi * chi * (2.0 * r.L + 2.5 * (kmax + 8.0)) + 64.0e6;
}

int check_request(const tdvp_request* r) {
  if (!r) return TDVP_EINVAL;
  if (r->L < 2 || r->chi_max < 1 || !(r->dt > 0) || !(r->t_final >= 0) || !(r->eps >= 0)) return TDVP_EINVAL;
  if (r->symmetry != TDVP_SYM_U1U1 && r->symmetry != TDVP_SYM_U1SU2) return TDVP_EINVAL;
  if (r->precision < TDVP_PREC_FP64 || r->precision > TDVP_PREC_BF16X4) return TDVP_EINVAL;
  if (r->mode < TDVP_SWEEP_TWO_SITE || r->mode > TDVP_SWEEP_ADAPTIVE) return TDVP_EINVAL;
  if (r->occupations)
    for (int i = 0; i < r->L; ++i)
      if (r->occupations[i] < 0 || r->occupations[i] > 3) return TDVP_EINVAL;
  return TDVP_OK;
}

double percentile(std::vector<double> v, double q) {  // linear between closest ranks
  if (v.empty()) return 0;
  std::sort(v.begin(), v.end());
  const double x = q * (double)(v.size() - 1);
  const size_t i = (size_t)std::floor(x);
  const size_t j = std::min(i + 1, v.size() - 1);
  return v[i] + (x - (double)i) * (v[j] - v[i]);
}

}  // namespace

struct tdvp_server {
  std::mutex m;
  std::condition_variable cv;  // queue, admission, completion and pause changes
  std::deque<long long> queue;
  std::map<long long, std::unique_ptr<Req>> reqs;
  double budget = 0;
  int max_active = 1;
  tdvp_opts base{};
  int device = 0;
  double reserved = 0, peak_reserved = 0;
  int active = 0, peak_active = 0;
  long long next_id = 1;
  bool paused = false, stopping = false;
  Clock::time_point t0 = Clock::now();
  std::vector<std::thread> workers;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  // the head of the queue may start now (called with m held)
  bool admissible() {
    if (paused || queue.empty() || active >= max_active) return false;
    const Req& h = *reqs[queue.front()];
    if (active == 0) return true;  // a request larger than the budget still runs, alone
    if (reserved + h.need > budget) return false;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      return true;  // no reading: the budget alone decides
    }
    return (double)fr >= h.need;
  }

  void run(Req& q, cudaStream_t stream);
  void worker();
};

void tdvp_server::run(Req& q, cudaStream_t stream) {
  const tdvp_request& r = q.r;
  tdvp_opts o = base;
  o.precision = r.precision;
  o.cuda_stream = stream;
  o.device = device;
  tdvp_ctx* ctx = nullptr;
  int rc = q.occ.empty() ? tdvp_create(r.L, r.J, r.U, r.symmetry, &o, &ctx)
                         : tdvp_create_product(r.L, r.J, r.U, r.symmetry, q.occ.data(), &o, &ctx);
  const long long nsteps = std::max<long long>(0, std::llround(r.t_final / r.dt));
  long long k = 0;
  for (; rc == TDVP_OK && k < nsteps; ++k) {
    {
      std::lock_guard<std::mutex> lk(m);
      if (q.cancel || stopping) {
        rc = TDVP_ECANCELED;
        tdvp::set_last_error("request cancelled");
        break;
      }
    }
    int used = 0;
    rc = tdvp_step_mode(ctx, r.dt, r.chi_max, r.eps, r.mode, &used);
  }
  if (rc == TDVP_OK) {
    q.n.assign(r.L, 0);
    q.sz.assign(r.L, 0);
    q.docc.assign(r.L, 0);
    q.ent.assign(std::max(r.L - 1, 1), 0);
    rc = tdvp_measure(ctx, q.n.data(), q.sz.data(), q.docc.data(), q.ent.data(), &q.energy);
  }
  if (rc == TDVP_OK) {
    std::vector<long long> chi(r.L + 1);
    rc = tdvp_bond_dims(ctx, chi.data(), nullptr);
    q.chi_max = (double)*std::max_element(chi.begin(), chi.end());
  }
  if (rc == TDVP_OK) {
    double st[20] = {0};
    rc = tdvp_stats(ctx, st, 20);
    q.heff_flops = st[1];
    q.dev_peak = st[19];
  }
  q.steps = (double)k;
  if (rc != TDVP_OK) q.msg = tdvp_last_error();
  tdvp_destroy(ctx);
  q.err = rc;
}

void tdvp_server::worker() {
  cudaStream_t stream = nullptr;  // created with the first admitted request
  if (cudaSetDevice(device) != cudaSuccess) cudaGetLastError();  // the device admission reads
  std::unique_lock<std::mutex> lk(m);
  for (;;) {
    cv.wait_for(lk, std::chrono::milliseconds(50), [&] { return stopping || admissible(); });
    if (stopping) break;
    if (!admissible()) continue;  // woken by the period: free memory is read again
    const long long id = queue.front();
    queue.pop_front();
    Req& q = *reqs[id];
    q.state = TDVP_REQ_RUNNING;
    q.t_admit = now();
    reserved += q.need;
    ++active;
    peak_active = std::max(peak_active, active);
    peak_reserved = std::max(peak_reserved, reserved);
    lk.unlock();
    int rc = TDVP_OK;
    if (!stream) {
      cudaError_t e = cudaSetDevice(device);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        cudaGetLastError();
        stream = nullptr;
        rc = TDVP_ECUDA;
        q.msg = std::string("worker stream: ") + cudaGetErrorString(e);
      }
    }
    if (rc == TDVP_OK) {
      run(q, stream);
    } else {
      q.err = rc;
    }
    lk.lock();
    q.t_done = now();
    q.state = q.err == TDVP_OK ? TDVP_REQ_DONE : (q.err == TDVP_ECANCELED ? TDVP_REQ_CANCELLED : TDVP_REQ_FAILED);
    reserved -= q.need;
    --active;
    cv.notify_all();
  }
  lk.unlock();
  if (stream) cudaStreamDestroy(stream);
}

extern "C" {

int tdvp_server_footprint(const tdvp_request* req, int krylov_max, double* bytes) {
  if (!bytes || check_request(req) != TDVP_OK) {
    tdvp::set_last_error("tdvp_server_footprint: invalid request or NULL output");
    return TDVP_EINVAL;
  }
  *bytes = footprint(*req, krylov_max > 0 ? krylov_max : 20);
  return TDVP_OK;
}

int tdvp_server_create(double hbm_budget_bytes, int max_active, const tdvp_opts* opts, tdvp_server** out) {
  if (!out || !(hbm_budget_bytes > 0) || max_active < 1 || max_active > 256) {
    tdvp::set_last_error("tdvp_server_create: need out, a positive budget and 1 <= max_active <= 256");
    return TDVP_EINVAL;
  }
  *out = nullptr;
  auto* s = new (std::nothrow) tdvp_server;
  if (!s) {
    tdvp::set_last_error("host allocation failed");
    return TDVP_ENOMEM;
  }
  tdvp_opts_default(&s->base);
  if (opts) s->base = *opts;
  s->base.cuda_stream = nullptr;
  s->device = s->base.device >= 0 ? s->base.device : 0;
  if (s->base.device < 0) {
    int d = 0;
    if (cudaGetDevice(&d) == cudaSuccess) s->device = d;
    cudaGetLastError();
  }
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  try {
    for (int i = 0; i < max_active; ++i) s->workers.emplace_back([s] { s->worker(); });
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->m);
      s->stopping = true;
    }
    s->cv.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
    tdvp::set_last_error("tdvp_server_create: could not start the worker threads");
    return TDVP_EINTERNAL;
  }
  *out = s;
  return TDVP_OK;
}

int tdvp_server_submit(tdvp_server* s, const tdvp_request* req, long long* id) {
  if (!s || !id || check_request(req) != TDVP_OK) {
    tdvp::set_last_error("tdvp_server_submit: invalid request (L >= 2, chi_max >= 1, dt > 0, t_final >= 0, "
                         "eps >= 0, known symmetry/precision/mode, occupations in 0..3) or NULL argument");
    return TDVP_EINVAL;
  }
  auto q = std::make_unique<Req>();
  q->r = *req;
  if (req->occupations) q->occ.assign(req->occupations, req->occupations + req->L);
  q->r.occupations = nullptr;
  q->need = footprint(*req, s->base.krylov_max);
  std::lock_guard<std::mutex> lk(s->m);
  if (s->stopping) {
    tdvp::set_last_error("tdvp_server_submit: server is shutting down");
    return TDVP_ESTATE;
  }
  q->t_submit = s->now();
  *id = s->next_id++;
  s->reqs[*id] = std::move(q);
  s->queue.push_back(*id);
  s->cv.notify_all();
  return TDVP_OK;
}

int tdvp_server_poll(tdvp_server* s, long long id, int* state) {
  if (!s || !state) return TDVP_EINVAL;
  std::lock_guard<std::mutex> lk(s->m);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    tdvp::set_last_error("tdvp_server_poll: unknown request id");
    return TDVP_EINVAL;
  }
  *state = it->second->state;
  return TDVP_OK;
}

int tdvp_server_wait(tdvp_server* s, long long id, int timeout_ms, int* state) {
  if (!s) return TDVP_EINVAL;
  std::unique_lock<std::mutex> lk(s->m);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    tdvp::set_last_error("tdvp_server_wait: unknown request id");
    return TDVP_EINVAL;
  }
  Req& q = *it->second;
  auto ended = [&] { return q.state >= TDVP_REQ_DONE; };
  if (timeout_ms < 0)
    s->cv.wait(lk, ended);
  else if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ended)) {
    if (state) *state = q.state;
    tdvp::set_last_error("tdvp_server_wait: request still queued or running");
    return TDVP_ETIMEOUT;
  }
  if (state) *state = q.state;
  return TDVP_OK;
}

int tdvp_server_result(tdvp_server* s, long long id, double* n, double* sz, double* docc, double* s_ent,
                       double* info, int ninfo) {
  if (!s) return TDVP_EINVAL;
  std::lock_guard<std::mutex> lk(s->m);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    tdvp::set_last_error("tdvp_server_result: unknown request id");
    return TDVP_EINVAL;
  }
  const Req& q = *it->second;
  if (info) {
    const double v[10] = {q.energy, q.chi_max, q.steps, q.heff_flops, q.t_submit, q.t_admit, q.t_done,
                          q.dev_peak, q.need, (double)q.err};
    for (int i = 0; i < ninfo && i < 10; ++i) info[i] = v[i];
  }
  if (q.state < TDVP_REQ_DONE) {
    tdvp::set_last_error("tdvp_server_result: request still queued or running");
    return TDVP_ESTATE;
  }
  if (q.state != TDVP_REQ_DONE) {
    tdvp::set_last_error(q.msg.c_str());
    return q.err;
  }
  const int L = q.r.L;
  if (n) std::copy(q.n.begin(), q.n.end(), n);
  if (sz) std::copy(q.sz.begin(), q.sz.end(), sz);
  if (docc) std::copy(q.docc.begin(), q.docc.end(), docc);
  if (s_ent) std::copy(q.ent.begin(), q.ent.begin() + std::max(L - 1, 0), s_ent);
  return TDVP_OK;
}

int tdvp_server_cancel(tdvp_server* s, long long id) {
  if (!s) return TDVP_EINVAL;
  std::lock_guard<std::mutex> lk(s->m);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    tdvp::set_last_error("tdvp_server_cancel: unknown request id");
    return TDVP_EINVAL;
  }
  Req& q = *it->second;
  if (q.state == TDVP_REQ_QUEUED) {
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), id));
    q.state = TDVP_REQ_CANCELLED;
    q.err = TDVP_ECANCELED;
    q.msg = "request cancelled";
    q.t_admit = q.t_done = s->now();
    s->cv.notify_all();
  } else if (q.state == TDVP_REQ_RUNNING) {
    q.cancel = true;  // honoured at the next step boundary
  }
  return TDVP_OK;
}

int tdvp_server_pause(tdvp_server* s, int paused) {
  if (!s) return TDVP_EINVAL;
  std::lock_guard<std::mutex> lk(s->m);
  s->paused = paused != 0;
  s->cv.notify_all();
  return TDVP_OK;
}

int tdvp_server_stats(tdvp_server* s, double* out, int n) {
  if (!s || !out) return TDVP_EINVAL;
  std::lock_guard<std::mutex> lk(s->m);
  double done = 0, failed = 0, cancelled = 0, queued = 0, running = 0, steps = 0, flops = 0;
  std::vector<double> lat;
  for (auto& kv : s->reqs) {
    const Req& q = *kv.second;
    switch (q.state) {
      case TDVP_REQ_QUEUED: queued += 1; break;
      case TDVP_REQ_RUNNING: running += 1; break;
      case TDVP_REQ_DONE:
        done += 1;
        lat.push_back(q.t_done - q.t_submit);
        steps += q.steps;
        flops += q.heff_flops;
        break;
      case TDVP_REQ_FAILED: failed += 1; break;
      default: cancelled += 1; break;
    }
  }
  const double v[13] = {(double)s->reqs.size(), done, failed, cancelled, queued, running, percentile(lat, 0.5),
                        percentile(lat, 0.99), s->now(), (double)s->peak_active, s->peak_reserved, steps, flops};
  for (int i = 0; i < n && i < 13; ++i) out[i] = v[i];
  return TDVP_OK;
}

int tdvp_server_destroy(tdvp_server* s) {
  if (!s) return TDVP_OK;
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->stopping = true;  // running requests stop at their next step boundary
    for (long long id : s->queue) {
      Req& q = *s->reqs[id];
      q.state = TDVP_REQ_CANCELLED;
      q.err = TDVP_ECANCELED;
    }
    s->queue.clear();
  }
  s->cv.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
  return TDVP_OK;
}

}  // extern "C"
