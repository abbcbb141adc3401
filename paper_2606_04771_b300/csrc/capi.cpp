// extern "C" boundary of the engine (include/tdvp.h): argument checks, host/device
// marshalling and the translation of exceptions into status codes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/tdvp.h"
#include "engine.hpp"

struct tdvp_ctx {
  tdvp::Engine* eng = nullptr;
  tdvp::DevAcct acct;  // device bytes of this context (live and peak)
};

namespace {
thread_local std::string g_last;

int fail(int code, const std::string& msg) {
  g_last = msg;
  return code;
}

template <class F>
int guarded(F f) {
  try {
    f();
    return TDVP_OK;
  } catch (const tdvp::Error& e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(TDVP_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(TDVP_EINTERNAL, e.what());
  }
}

// a call on a context: its device allocations are charged to the context, and its
// BF16x4 GEMMs merge with other contexts' launches when the context asked for that
struct MergeScope {
  bool prev;
  explicit MergeScope(bool on) : prev(tdvp::merge_launches_here()) { tdvp::merge_launches_here() = on; }
  ~MergeScope() { tdvp::merge_launches_here() = prev; }
};
template <class F>
int guarded(tdvp_ctx* ctx, F f) {
  tdvp::DevAcctScope scope(&ctx->acct);
  MergeScope merge(ctx->eng && ctx->eng->opts().merge);
  return guarded(f);
}

// a new context around the engine that make() builds
template <class Make>
int create_ctx(tdvp_ctx** out, Make make) {
  auto* c = new (std::nothrow) tdvp_ctx;
  if (!c) return fail(TDVP_ENOMEM, "host allocation failed");
  const int rc = guarded(c, [&] { c->eng = make(); });
  if (rc != TDVP_OK) {
    delete c;
    return rc;
  }
  *out = c;
  return TDVP_OK;
}

tdvp::Opts to_opts(const tdvp_opts* o) {
  tdvp::Opts r;
  if (o) {
    r.precision = o->precision;
    r.krylov_max = o->krylov_max;
    r.krylov_tol = o->krylov_tol;
    r.timeout_ms = o->timeout_ms;
    r.stream = reinterpret_cast<cudaStream_t>(o->cuda_stream);
    r.device = o->device;
    r.trunc_degen = o->trunc_degeneracy;
    r.merge = o->merge_launches != 0;
  }
  return r;
}

std::vector<tdvp::Sector> sectors(int n, const int* v) {
  std::vector<tdvp::Sector> s;
  for (int i = 0; i < n; ++i) s.push_back({v[3 * i], v[3 * i + 1], v[3 * i + 2]});
  return s;
}

tdvp::BTensor* tensor_of(tdvp_ctx* ctx, int which) {
  tdvp::Engine* e = ctx->eng;
  if (which == 3) {
    e->chain_heff0();
    return &e->theta_layout();
  }
  if (!e->bond_only()) throw tdvp::Error(TDVP_ESTATE, "which 0-2 need a bond-problem context");
  if (which == 0) return &e->theta_layout();
  if (which == 1) return &e->left_env_bp();
  if (which == 2) return &e->right_env_bp();
  throw tdvp::Error(TDVP_EINVAL, "which must be 0..3");
}
}  // namespace

namespace tdvp {
void set_last_error(const char* msg) { g_last = msg; }
}  // namespace tdvp

extern "C" {

void tdvp_opts_default(tdvp_opts* o) {
  if (!o) return;
  o->precision = TDVP_PREC_FP64;
  o->krylov_max = 20;
  o->krylov_tol = 1e-12;
  o->timeout_ms = 0;
  o->cuda_stream = nullptr;
  o->device = -1;
  o->trunc_degeneracy = 1e-8;
  o->merge_launches = 0;
}

int tdvp_create(int L, double J, double U, int symmetry, const tdvp_opts* opts, tdvp_ctx** out) {
  if (!out) return fail(TDVP_EINVAL, "out is NULL");
  *out = nullptr;
  if (symmetry != TDVP_SYM_U1U1 && symmetry != TDVP_SYM_U1SU2) return fail(TDVP_EINVAL, "unknown symmetry");
  return create_ctx(out, [&] {
    tdvp_opts d;
    tdvp_opts_default(&d);
    return new tdvp::Engine(L, J, U, symmetry == TDVP_SYM_U1SU2, to_opts(opts ? opts : &d));
  });
}

int tdvp_create_product(int L, double J, double U, int symmetry, const int* occ, const tdvp_opts* opts,
                        tdvp_ctx** out) {
  if (!out || !occ) return fail(TDVP_EINVAL, "NULL argument");
  *out = nullptr;
  if (symmetry != TDVP_SYM_U1U1 && symmetry != TDVP_SYM_U1SU2) return fail(TDVP_EINVAL, "unknown symmetry");
  if (L < 2) return fail(TDVP_EINVAL, "L must be >= 2");
  return create_ctx(out, [&] {
    tdvp_opts d;
    tdvp_opts_default(&d);
    std::vector<int> o(occ, occ + L);
    return tdvp::Engine::product_state(L, J, U, symmetry == TDVP_SYM_U1SU2, o, to_opts(opts ? opts : &d));
  });
}

int tdvp_create_random(int L, double J, double U, int symmetry, long long chi_target, unsigned long long seed,
                       int center, const tdvp_opts* opts, tdvp_ctx** out) {
  if (!out) return fail(TDVP_EINVAL, "out is NULL");
  *out = nullptr;
  if (symmetry != TDVP_SYM_U1U1 && symmetry != TDVP_SYM_U1SU2) return fail(TDVP_EINVAL, "unknown symmetry");
  return create_ctx(out, [&] {
    tdvp_opts d;
    tdvp_opts_default(&d);
    return tdvp::Engine::random_state(L, J, U, symmetry == TDVP_SYM_U1SU2, chi_target, seed, center,
                                      to_opts(opts ? opts : &d));
  });
}

int tdvp_bond_create(int symmetry, double J, double U, int nl, const int* left, int nr, const int* right,
                     const tdvp_opts* opts, tdvp_ctx** out) {
  if (!out) return fail(TDVP_EINVAL, "out is NULL");
  *out = nullptr;
  if (symmetry != TDVP_SYM_U1U1 && symmetry != TDVP_SYM_U1SU2) return fail(TDVP_EINVAL, "unknown symmetry");
  if (nl < 1 || nr < 1 || !left || !right) return fail(TDVP_EINVAL, "empty sector table");
  return create_ctx(out, [&] {
    tdvp_opts d;
    tdvp_opts_default(&d);
    return tdvp::Engine::bond_problem(symmetry == TDVP_SYM_U1SU2, J, U, sectors(nl, left), sectors(nr, right),
                                      to_opts(opts ? opts : &d));
  });
}

int tdvp_save(tdvp_ctx* ctx, const char* path, double t) {
  if (!ctx || !path) return fail(TDVP_EINVAL, "NULL argument");
  return guarded(ctx, [&] { ctx->eng->save(path, t); });
}

int tdvp_load(const char* path, const tdvp_opts* opts, tdvp_ctx** out, double* t) {
  if (!out || !path) return fail(TDVP_EINVAL, "NULL argument");
  *out = nullptr;
  return create_ctx(out, [&] {
    tdvp_opts d;
    tdvp_opts_default(&d);
    return tdvp::Engine::load(path, to_opts(opts ? opts : &d), t);
  });
}

int tdvp_step(tdvp_ctx* ctx, double dt, long long chi_max, double eps_trunc) {
  if (!ctx) return fail(TDVP_EINVAL, "ctx is NULL");
  return guarded(ctx, [&] { ctx->eng->step(dt, chi_max, eps_trunc); });
}

int tdvp_step_mode(tdvp_ctx* ctx, double dt, long long chi_max, double eps_trunc, int mode, int* used) {
  if (!ctx) return fail(TDVP_EINVAL, "ctx is NULL");
  if (mode < 0 || mode > 2) return fail(TDVP_EINVAL, "mode must be 0, 1 or 2");
  return guarded(ctx, [&] {
    int u = ctx->eng->step_mode(dt, chi_max, eps_trunc, mode);
    if (used) *used = u;
  });
}

int tdvp_bond_update(tdvp_ctx* ctx, int bond, int direction, double dt, long long chi_max, double eps_trunc,
                     double* s_ent) {
  if (!ctx) return fail(TDVP_EINVAL, "ctx is NULL");
  if (direction != 0 && direction != 1) return fail(TDVP_EINVAL, "direction must be 0 or 1");
  return guarded(ctx, [&] { ctx->eng->single_bond(bond, direction, dt, chi_max, eps_trunc, s_ent); });
}

int tdvp_measure_center(tdvp_ctx* ctx, int* site, double* n, double* sz, double* docc) {
  if (!ctx) return fail(TDVP_EINVAL, "ctx is NULL");
  return guarded(ctx, [&] { ctx->eng->measure_center(site, n, sz, docc); });
}

int tdvp_measure(tdvp_ctx* ctx, double* n, double* sz, double* docc, double* s_ent, double* energy) {
  if (!ctx) return fail(TDVP_EINVAL, "ctx is NULL");
  return guarded(ctx, [&] { ctx->eng->measure(n, sz, docc, s_ent, energy); });
}

int tdvp_bond_dims(tdvp_ctx* ctx, long long* chi, long long* chi_red) {
  if (!ctx) return fail(TDVP_EINVAL, "ctx is NULL");
  return guarded(ctx, [&] {
    tdvp::Engine* e = ctx->eng;
    if (e->bond_only()) throw tdvp::Error(TDVP_ESTATE, "bond problem has no chain");
    for (int k = 0; k <= e->L(); ++k) {
      const tdvp::BondSpace& b = e->bond(k);
      long long c = 0, r = 0;
      for (auto& s : b.s) {
        c += (long long)s.d * e->model().mult_dim(s.t);
        r += s.d;
      }
      if (chi) chi[k] = c;
      if (chi_red) chi_red[k] = r;
    }
  });
}

int tdvp_selftest_wait(unsigned int polls, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* d = nullptr;
  int h = 0;
  cudaError_t e = cudaMallocAsync(&d, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    tdvp::launch_wait_selftest(polls, d, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(TDVP_ECUDA, cudaGetErrorString(e));
  if (h) return fail(TDVP_ETIMEOUT, "self-test wait expired as intended");
  return TDVP_OK;
}

int tdvp_merge_count(long long* launches, long long* slices) {
  if (!launches && !slices) return fail(TDVP_EINVAL, "NULL argument");
  tdvp::merge_counts(launches, slices);
  return TDVP_OK;
}

int tdvp_launch_count(long long* out) {
  if (!out) return fail(TDVP_EINVAL, "NULL argument");
  *out = tdvp::launch_count();
  return TDVP_OK;
}

int tdvp_stats(tdvp_ctx* ctx, double* out, int n) {
  if (!ctx || !out) return fail(TDVP_EINVAL, "NULL argument");
  return guarded(ctx, [&] {
    const tdvp::StepStats& s = ctx->eng->stats();
    double v[38] = {s.seconds, (double)s.heff_flops, (double)s.env_flops, (double)s.matvecs, (double)s.max_krylov,
                    s.max_discarded, (double)s.chi_max_seen, s.phase[0], s.phase[1], s.phase[2], s.phase[3],
                    s.phase[4], s.phase[5], (double)s.steps, (double)s.splits, (double)s.sweeps64,
                    (double)s.sweeps32, (double)s.one_site_steps, (double)ctx->acct.live.load(),
                    (double)ctx->acct.peak.load(), s.jacobi32.ms, s.jacobi32.flops, s.jacobi64.ms, s.jacobi64.flops,
                    (double)s.split_pmax, (double)s.split_qmax, s.split_work, s.split_work_small,
                    (double)(s.jacobi32.launches + s.jacobi64.launches),
                    (double)(s.jacobi32.resident + s.jacobi64.resident),
                    (double)(s.jacobi32.cluster + s.jacobi64.cluster), s.env_ms, s.env_bytes,
                    s.gram.ms, s.gram.flops, (double)s.gram_steps, (double)s.gram_fallbacks,
                    (double)(s.jacobi32.ring + s.jacobi64.ring)};
    for (int i = 0; i < n && i < 38; ++i) out[i] = v[i];
  });
}

int tdvp_block_count(tdvp_ctx* ctx, int which, long long* nblocks, long long* nelems) {
  if (!ctx) return fail(TDVP_EINVAL, "ctx is NULL");
  return guarded(ctx, [&] {
    tdvp::BTensor* t = tensor_of(ctx, which);
    if (nblocks) *nblocks = (long long)t->blocks.size();
    if (nelems) *nelems = t->size;
  });
}

int tdvp_block_list(tdvp_ctx* ctx, int which, int* keys, int* dims, long long* offsets) {
  if (!ctx) return fail(TDVP_EINVAL, "ctx is NULL");
  return guarded(ctx, [&] {
    tdvp::BTensor* t = tensor_of(ctx, which);
    for (size_t i = 0; i < t->blocks.size(); ++i) {
      const tdvp::Block& b = t->blocks[i];
      if (keys)
        for (int k = 0; k < 5; ++k) keys[5 * i + k] = b.key[k];
      if (dims) {
        dims[2 * i] = b.rows;
        dims[2 * i + 1] = b.cols;
      }
      if (offsets) offsets[i] = b.off;
    }
  });
}

int tdvp_set_tensor(tdvp_ctx* ctx, int which, const double* data, long long n, int on_device) {
  if (!ctx || !data) return fail(TDVP_EINVAL, "NULL argument");
  if (which != 1 && which != 2) return fail(TDVP_EINVAL, "which must be 1 (L) or 2 (R)");
  return guarded(ctx, [&] {
    tdvp::BTensor* t = tensor_of(ctx, which);
    if (n != t->size) throw tdvp::Error(TDVP_EINVAL, "size mismatch");
    cudaStream_t s = ctx->eng->stream();
    TDVP_CUDA(cudaMemcpyAsync(t->data(), data, n * sizeof(tdvp::cplx),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    TDVP_CUDA(cudaStreamSynchronize(s));
    ctx->eng->environments_changed();
  });
}

int tdvp_heff_apply(tdvp_ctx* ctx, int bond, const double* psi_in, double* psi_out, int on_device) {
  if (!ctx || !psi_in || !psi_out) return fail(TDVP_EINVAL, "NULL argument");
  if (bond != 0) return fail(TDVP_EINVAL, "bond must be 0");
  return guarded(ctx, [&] {
    tdvp::Engine* e = ctx->eng;
    tdvp::HeffPlan& H = e->bond_only() ? e->heff_plan_bond() : e->chain_heff0();
    cudaStream_t s = e->stream();
    const long long n = H.n;
    if (on_device) {
      H.apply(reinterpret_cast<const tdvp::cplx*>(psi_in), reinterpret_cast<tdvp::cplx*>(psi_out), s);
      TDVP_CUDA(cudaStreamSynchronize(s));
      e->check_status();
    } else {
      tdvp::DevBuf din(std::max<long long>(n, 1) * sizeof(tdvp::cplx), s), dout(std::max<long long>(n, 1) * sizeof(tdvp::cplx), s);
      TDVP_CUDA(cudaMemcpyAsync(din.p, psi_in, n * sizeof(tdvp::cplx), cudaMemcpyHostToDevice, s));
      H.apply(din.as<tdvp::cplx>(), dout.as<tdvp::cplx>(), s);
      TDVP_CUDA(cudaMemcpyAsync(psi_out, dout.p, n * sizeof(tdvp::cplx), cudaMemcpyDeviceToHost, s));
      TDVP_CUDA(cudaStreamSynchronize(s));
      e->check_status();
    }
    TDVP_CUDA(cudaGetLastError());
  });
}

int tdvp_heff_groups(tdvp_ctx* ctx, int* ngroups, long long* flops, int* block_group) {
  if (!ctx || !ngroups) return fail(TDVP_EINVAL, "NULL argument");
  return guarded(ctx, [&] {
    tdvp::Engine* e = ctx->eng;
    tdvp::HeffPlan& H = e->bond_only() ? e->heff_plan_bond() : e->chain_heff0();
    const int ng = (int)H.g3.tasks.size();
    *ngroups = ng;
    if (flops)
      for (int g = 0; g < ng; ++g) flops[g] = H.g3.task_flops[g];
    if (block_group) {
      const int nb = (int)e->theta_layout().blocks.size();
      for (int b = 0; b < nb; ++b) block_group[b] = -1;
      for (int g = 0; g < ng; ++g)
        for (int b : H.g3.out_blocks[g]) block_group[b] = g;
    }
  });
}

int tdvp_partition(int n, const double* cost, int nranks, int* owner, double* load) {
  if (n < 0 || nranks < 1 || (n > 0 && (!cost || !owner))) return fail(TDVP_EINVAL, "bad argument");
  for (int i = 0; i < n; ++i)
    if (!(cost[i] >= 0.0)) return fail(TDVP_EINVAL, "tdvp_partition: negative or NaN cost");
  return guarded([&] {
    // longest processing time first: units by cost descending (ties by index), each to
    // the rank with the least load so far (ties to the lowest rank)
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> l(nranks, 0.0);
    for (int i : ord) {
      int best = 0;
      for (int r = 1; r < nranks; ++r)
        if (l[r] < l[best]) best = r;
      owner[i] = best;
      l[best] += cost[i];
    }
    if (load)
      for (int r = 0; r < nranks; ++r) load[r] = l[r];
  });
}

int tdvp_heff_apply_owned(tdvp_ctx* ctx, int bond, const int* group_owner, int rank, const double* psi_in,
                          double* psi_out, int on_device) {
  if (!ctx || !group_owner || !psi_in || !psi_out) return fail(TDVP_EINVAL, "NULL argument");
  if (bond != 0) return fail(TDVP_EINVAL, "bond must be 0");
  if (!on_device) return fail(TDVP_EINVAL, "tdvp_heff_apply_owned takes device pointers");
  return guarded(ctx, [&] {
    tdvp::Engine* e = ctx->eng;
    tdvp::HeffPlan& H = e->bond_only() ? e->heff_plan_bond() : e->chain_heff0();
    std::vector<char> owned(H.g3.tasks.size());
    for (size_t g = 0; g < owned.size(); ++g) owned[g] = group_owner[g] == rank;
    H.apply_owned(reinterpret_cast<const tdvp::cplx*>(psi_in), reinterpret_cast<tdvp::cplx*>(psi_out), owned,
                  e->stream());
    e->check_status();
    TDVP_CUDA(cudaGetLastError());
  });
}

int tdvp_krylov_expm(tdvp_ctx* ctx, int bond, const double* psi_in, double* psi_out, double tau, int on_device,
                     int* krylov_dim, int* launches) {
  if (!ctx || !psi_in || !psi_out) return fail(TDVP_EINVAL, "NULL argument");
  if (bond != 0) return fail(TDVP_EINVAL, "bond must be 0");
  return guarded(ctx, [&] {
    tdvp::Engine* e = ctx->eng;
    tdvp::HeffPlan& H = e->bond_only() ? e->heff_plan_bond() : e->chain_heff0();
    cudaStream_t s = e->stream();
    const long long n = std::max<long long>(H.n, 1);
    tdvp::DevBuf x(n * sizeof(tdvp::cplx), s);
    TDVP_CUDA(cudaMemcpyAsync(x.p, psi_in, H.n * sizeof(tdvp::cplx),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    int k = 0, nl = 0;
    e->krylov(H, x.as<tdvp::cplx>(), tau, &k, &nl);
    TDVP_CUDA(cudaMemcpyAsync(psi_out, x.p, H.n * sizeof(tdvp::cplx),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    TDVP_CUDA(cudaStreamSynchronize(s));
    e->check_status();
    if (krylov_dim) *krylov_dim = k;
    if (launches) *launches = nl;
  });
}

int tdvp_heff_flops(tdvp_ctx* ctx, long long* flops) {
  if (!ctx || !flops) return fail(TDVP_EINVAL, "NULL argument");
  return guarded(ctx, [&] {
    tdvp::Engine* e = ctx->eng;
    *flops = (e->bond_only() ? e->heff_plan_bond() : e->chain_heff0()).flops();
  });
}

int tdvp_heff_profile(tdvp_ctx* ctx, int iters, double* ms, long long* flops, long long* bytes) {
  if (!ctx || iters < 1) return fail(TDVP_EINVAL, "bad argument");
  return guarded(ctx, [&] {
    tdvp::Engine* e = ctx->eng;
    tdvp::HeffPlan& H = e->bond_only() ? e->heff_plan_bond() : e->chain_heff0();
    cudaStream_t s = e->stream();
    const long long n = std::max<long long>(H.n, 1);
    tdvp::DevBuf din(n * sizeof(tdvp::cplx), s), dout(n * sizeof(tdvp::cplx), s);
    tdvp::launch_fill_normal(din.as<tdvp::cplx>(), n, 0x5eedULL, 0, s);  // a non-zero input
    tdvp::Bases4 B{{0, reinterpret_cast<uintptr_t>(din.p), reinterpret_cast<uintptr_t>(dout.p), 0}};
    H.apply(din.as<tdvp::cplx>(), dout.as<tdvp::cplx>(), s);  // warm-up (static operand splits)
    cudaEvent_t ev[4];
    for (auto& x : ev) TDVP_CUDA(cudaEventCreate(&x));
    float acc[3] = {0, 0, 0};
    for (int it = 0; it < iters; ++it) {
      TDVP_CUDA(cudaEventRecord(ev[0], s));
      H.g1.launch(s, B);
      const unsigned e3 = H.g3.dyn_mode == 1 ? H.g3.begin_split(s, B) : 0u;
      TDVP_CUDA(cudaEventRecord(ev[1], s));
      H.lc.launch(s, e3);
      TDVP_CUDA(cudaEventRecord(ev[2], s));
      H.g3.launch(s, B, e3);
      TDVP_CUDA(cudaEventRecord(ev[3], s));
      TDVP_CUDA(cudaEventSynchronize(ev[3]));
      for (int k = 0; k < 3; ++k) {
        float t = 0;
        TDVP_CUDA(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
        acc[k] += t;
      }
    }
    for (auto& x : ev) cudaEventDestroy(x);
    if (ms)
      for (int k = 0; k < 3; ++k) ms[k] = acc[k] / iters;
    if (flops) {
      flops[0] = H.g1.flops;
      flops[1] = 0;
      flops[2] = H.g3.flops;
    }
    if (bytes) {
      bytes[0] = H.g1.bytes;
      bytes[1] = H.lc.bytes;
      bytes[2] = H.g3.bytes;
    }
  });
}

int tdvp_svd(int p, int q, const double* a, double* s, double* u, double* vh, int on_device, void* stream) {
  if (p < 1 || q < 1 || !a || !s || !u || !vh) return fail(TDVP_EINVAL, "bad argument");
  return guarded([&] {
    using tdvp::cplx;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int r = std::min(p, q), P = std::max(p, q), Q = r;
    const size_t na = (size_t)p * q;
    tdvp::DevBuf dA, dU, dVh, dS;
    const cplx* A = reinterpret_cast<const cplx*>(a);
    cplx* Uo = reinterpret_cast<cplx*>(u);
    cplx* Vo = reinterpret_cast<cplx*>(vh);
    double* So = s;
    if (!on_device) {
      dA = tdvp::DevBuf(na * sizeof(cplx), st);
      dU = tdvp::DevBuf((size_t)p * r * sizeof(cplx), st);
      dVh = tdvp::DevBuf((size_t)r * q * sizeof(cplx), st);
      dS = tdvp::DevBuf((size_t)r * sizeof(double), st);
      TDVP_CUDA(cudaMemcpyAsync(dA.p, a, na * sizeof(cplx), cudaMemcpyHostToDevice, st));
      A = dA.as<cplx>();
      Uo = dU.as<cplx>();
      Vo = dVh.as<cplx>();
      So = dS.as<double>();
    }
    tdvp::DevBuf dG((size_t)P * Q * sizeof(cplx), st), dV((size_t)Q * Q * sizeof(cplx), st);
    tdvp::DevBuf dP((size_t)Q * sizeof(int), st), dT(sizeof(tdvp::SvdTask), st), dst(sizeof(int), st);
    TDVP_CUDA(cudaMemsetAsync(dst.p, 0, sizeof(int), st));
    tdvp::CopyPlan gather, scatter;
    {
      tdvp::CopyTask t{};
      t.src = A;
      t.rows = p;
      t.cols = q;
      t.src_rs = q;
      t.src_cs = 1;
      t.dst = dG.as<cplx>();
      if (p >= q) {
        t.dst_rs = 1;
        t.dst_cs = p;
      } else {
        t.dst_rs = q;
        t.dst_cs = 1;
        t.conj = 1;
      }
      gather.tasks.push_back(t);
    }
    gather.finalize(st);
    gather.launch(st);
    tdvp::SvdTask task{dG.as<cplx>(), dV.as<cplx>(), So, dP.as<int>(), P, Q};
    TDVP_CUDA(cudaMemcpyAsync(dT.p, &task, sizeof(task), cudaMemcpyHostToDevice, st));
    tdvp::launch_jacobi_svd(dT.as<tdvp::SvdTask>(), 1, Q, 60, 1e-15, dst.as<int>(), st);
    tdvp::CopyTask tu{}, tv{};
    tu.dst = Uo;
    tu.rows = p;
    tu.cols = r;
    tu.dst_rs = r;
    tu.dst_cs = 1;
    tu.col_map = dP.as<int>();
    tv.dst = Vo;
    tv.rows = r;
    tv.cols = q;
    tv.dst_rs = q;
    tv.dst_cs = 1;
    tv.row_map = dP.as<int>();
    tv.conj = 1;
    if (p >= q) {  // U = G / s, V^H = conj(V)^T
      tu.src = dG.as<cplx>();
      tu.src_rs = 1;
      tu.src_cs = p;
      tu.scale = So;
      tu.scale_mode = 2;
      tv.src = dV.as<cplx>();
      tv.src_rs = q;
      tv.src_cs = 1;
    } else {  // A^H = W S^-1 ... : U = V_jacobi, V^H = conj(G)^T / s
      tu.src = dV.as<cplx>();
      tu.src_rs = 1;
      tu.src_cs = p;
      tv.src = dG.as<cplx>();
      tv.src_rs = q;
      tv.src_cs = 1;
      tv.scale = So;
      tv.scale_mode = 4;
    }
    scatter.tasks = {tu, tv};
    scatter.finalize(st);
    scatter.launch(st);
    int status = 0;
    TDVP_CUDA(cudaMemcpyAsync(&status, dst.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (!on_device) {
      TDVP_CUDA(cudaMemcpyAsync(u, Uo, (size_t)p * r * sizeof(cplx), cudaMemcpyDeviceToHost, st));
      TDVP_CUDA(cudaMemcpyAsync(vh, Vo, (size_t)r * q * sizeof(cplx), cudaMemcpyDeviceToHost, st));
      TDVP_CUDA(cudaMemcpyAsync(s, So, (size_t)r * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    TDVP_CUDA(cudaStreamSynchronize(st));
    TDVP_CUDA(cudaGetLastError());
    if (status) throw tdvp::Error(TDVP_ENUMERIC, "Jacobi SVD did not converge");
  });
}

int tdvp_truncate(int nsec, const int* r, const int* mult, const double* sv, double eps, long long chi_max,
                  double degeneracy, int* kept, double* stats, void* stream) {
  if (nsec < 1 || !r || !mult || !sv || !kept) return fail(TDVP_EINVAL, "tdvp_truncate: NULL argument or nsec < 1");
  if (!(eps >= 0.0) || chi_max < 1 || !(degeneracy >= 0.0))
    return fail(TDVP_EINVAL, "tdvp_truncate: eps < 0, chi_max < 1 or degeneracy < 0");
  long long n = 0;
  for (int k = 0; k < nsec; ++k) {
    if (r[k] < 0 || mult[k] < 1) return fail(TDVP_EINVAL, "tdvp_truncate: r[k] < 0 or mult[k] < 1");
    n += r[k];
  }
  if (n < 1 || n > (1LL << 30)) return fail(TDVP_EINVAL, "tdvp_truncate: total number of values out of range");
  return guarded([&] {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int ni = (int)n;
    tdvp::DevBuf dsv(n * sizeof(double), st), dsec(nsec * sizeof(tdvp::TruncSector), st);
    tdvp::DevBuf doffs(nsec * sizeof(int), st), downer(n * sizeof(int), st), dorder(n * sizeof(int), st);
    tdvp::DevBuf dkept(nsec * sizeof(int), st), dstats(8 * sizeof(double), st), dvals(2 * n * sizeof(double), st);
    std::vector<tdvp::TruncSector> secs(nsec);
    std::vector<int> offs(nsec);
    int o = 0;
    for (int k = 0; k < nsec; ++k) {
      offs[k] = o;
      secs[k] = {dsv.as<double>() + o, r[k], mult[k]};
      o += r[k];
    }
    TDVP_CUDA(cudaMemcpyAsync(dsv.p, sv, n * sizeof(double), cudaMemcpyHostToDevice, st));
    TDVP_CUDA(cudaMemcpyAsync(dsec.p, secs.data(), nsec * sizeof(tdvp::TruncSector), cudaMemcpyHostToDevice, st));
    TDVP_CUDA(cudaMemcpyAsync(doffs.p, offs.data(), nsec * sizeof(int), cudaMemcpyHostToDevice, st));
    tdvp::launch_truncate(dsec.as<tdvp::TruncSector>(), nsec, doffs.as<int>(), ni, eps, chi_max, degeneracy,
                          downer.as<int>(),
                          dorder.as<int>(), dkept.as<int>(), dstats.as<double>(), dvals.as<double>(), st);
    double hs[6];
    TDVP_CUDA(cudaMemcpyAsync(kept, dkept.p, nsec * sizeof(int), cudaMemcpyDeviceToHost, st));
    TDVP_CUDA(cudaMemcpyAsync(hs, dstats.p, 6 * sizeof(double), cudaMemcpyDeviceToHost, st));
    TDVP_CUDA(cudaStreamSynchronize(st));
    TDVP_CUDA(cudaGetLastError());
    if (stats)
      for (int i = 0; i < 6; ++i) stats[i] = hs[i];
  });
}

int tdvp_destroy(tdvp_ctx* ctx) {
  if (!ctx) return TDVP_OK;
  int rc = guarded(ctx, [&] { delete ctx->eng; });
  delete ctx;
  return rc;
}

const char* tdvp_strerror(int code) {
  switch (code) {
    case TDVP_OK: return "ok";
    case TDVP_EINVAL: return "invalid argument";
    case TDVP_ESTATE: return "call not valid for this context";
    case TDVP_ENOMEM: return "out of memory";
    case TDVP_ENUMERIC: return "numerical failure";
    case TDVP_EINTERNAL: return "internal error";
    case TDVP_ECUDA: return "CUDA error";
    case TDVP_ETIMEOUT: return "device wait timed out";
    case TDVP_ECANCELED: return "request cancelled";
    case TDVP_EIO: return "checkpoint file error";
    default: return "unknown error";
  }
}

const char* tdvp_last_error(void) { return g_last.c_str(); }

}  // extern "C"
