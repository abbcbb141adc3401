// tdvp_svd_noalloc: the per-matrix Jacobi SVD of tdvp_svd without any device
// allocation at call time.
//
// Who needs it: a caller that must not allocate device memory while it runs --
// for example a serving process whose own memory pool already holds (nearly) all
// of the GPU's memory, where cudaMalloc would fail or would stall every stream of
// the device while it runs, or code that runs under a frozen memory budget after
// start-up.  Such a caller passes device pointers for the input and the outputs;
// the workspace (the column-major working copy, the right singular vectors, the
// sort permutation and the small task descriptors) lives in one file-scope
// static device array below, which every GPU that loads this library holds
// until the process exits.
//
// Rules of use:
//   - max(p, q) <= TDVP_SVD_NOALLOC_MAX (512); larger sizes are rejected with
//     TDVP_EINVAL and a message.
//   - The first call on a device (with that device current) looks up the
//     array's device address with cudaGetSymbolAddress and caches it.
//   - No call may be made while a stream is capturing: every call copies its work
//     lists from host memory and synchronises its stream before returning.
//   - All calls share the one array and it keeps the last call's contents; every
//     region is rewritten before it is read and the convergence flag is cleared
//     at the start of each call.  Calls whose work overlaps on the GPU (for
//     example on two streams at once) race on the array and must be serialised
//     by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/tdvp.h"
#include "common.hpp"
#include "kernels.hpp"

namespace tdvp {
void set_last_error(const char* msg);  // capi.cpp: message for tdvp_last_error()
namespace {

constexpr int NMAX = TDVP_SVD_NOALLOC_MAX;                    // largest p or q
constexpr int CHUNKS_MAX = 3 * (NMAX * NMAX / LINCOMB_CHUNK);  // gather + two scatters

struct Scratch {
  cplx g[NMAX * NMAX];  // working copy: A (p >= q) or A^H, column-major
  cplx v[NMAX * NMAX];  // right singular vectors of the working copy
  int perm[NMAX];
  int status;
  int pad[3];
  SvdTask task;
  CopyTask copies[3];
  int2 chunks[CHUNKS_MAX];
};

}  // namespace
}  // namespace tdvp

// The workspace of every tdvp_svd_noalloc call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(tdvp::Scratch)];

namespace tdvp {
namespace {

std::mutex g_mu;
void* g_addr[64] = {};  // per device ordinal

int setup(int dev, Scratch** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) {
    set_last_error("tdvp_svd_noalloc: device ordinal out of range");
    return TDVP_EINVAL;
  }
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error("tdvp_svd_noalloc: cudaGetSymbolAddress failed for the workspace");
      return TDVP_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = reinterpret_cast<Scratch*>(g_addr[dev]);
  return TDVP_OK;
}

int add_chunks(int task, int n, int2* chunks, int& nc) {
  for (int e = 0; e < n; e += LINCOMB_CHUNK) {
    if (nc >= CHUNKS_MAX) return -1;
    chunks[nc++] = make_int2(task, e);
  }
  return 0;
}

}  // namespace
}  // namespace tdvp

extern "C" int tdvp_svd_noalloc(int p, int q, const double* a, double* s, double* u, double* vh, void* stream) {
  using namespace tdvp;
  if (p < 1 || q < 1 || !a || !s || !u || !vh) {
    set_last_error("tdvp_svd_noalloc: p, q must be >= 1 and pointers non-NULL");
    return TDVP_EINVAL;
  }
  if (p > NMAX || q > NMAX) {
    set_last_error("tdvp_svd_noalloc: max(p, q) exceeds TDVP_SVD_NOALLOC_MAX (512)");
    return TDVP_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_last_error("tdvp_svd_noalloc: no current CUDA device");
    return TDVP_ECUDA;
  }
  Scratch* S = nullptr;
  int rc = setup(dev, &S);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int r = p < q ? p : q, P = p > q ? p : q, Q = r;
  const cplx* A = reinterpret_cast<const cplx*>(a);
  // descriptors are built on the host stack and copied into the static array
  SvdTask task{S->g, S->v, s, S->perm, P, Q};
  CopyTask c[3] = {};
  int2 chunks[CHUNKS_MAX];
  int nc = 0;
  c[0].src = A;
  c[0].rows = p;
  c[0].cols = q;
  c[0].src_rs = q;
  c[0].src_cs = 1;
  c[0].dst = S->g;
  if (p >= q) {
    c[0].dst_rs = 1;
    c[0].dst_cs = p;
  } else {
    c[0].dst_rs = q;
    c[0].dst_cs = 1;
    c[0].conj = 1;
  }
  c[1].dst = reinterpret_cast<cplx*>(u);
  c[1].rows = p;
  c[1].cols = r;
  c[1].dst_rs = r;
  c[1].dst_cs = 1;
  c[1].col_map = S->perm;
  c[2].dst = reinterpret_cast<cplx*>(vh);
  c[2].rows = r;
  c[2].cols = q;
  c[2].dst_rs = q;
  c[2].dst_cs = 1;
  c[2].row_map = S->perm;
  c[2].conj = 1;
  if (p >= q) {
    c[1].src = S->g;
    c[1].src_rs = 1;
    c[1].src_cs = p;
    c[1].scale = s;
    c[1].scale_mode = 2;
    c[2].src = S->v;
    c[2].src_rs = q;
    c[2].src_cs = 1;
  } else {
    c[1].src = S->v;
    c[1].src_rs = 1;
    c[1].src_cs = p;
    c[2].src = S->g;
    c[2].src_rs = q;
    c[2].src_cs = 1;
    c[2].scale = s;
    c[2].scale_mode = 4;
  }
  if (add_chunks(0, p * q, chunks, nc)) {
    set_last_error("tdvp_svd_noalloc: copy work list exceeds its static capacity");
    return TDVP_EINTERNAL;
  }
  const int ng = nc;
  if (add_chunks(1, p * r, chunks, nc) || add_chunks(2, r * q, chunks, nc)) {
    set_last_error("tdvp_svd_noalloc: copy work list exceeds its static capacity");
    return TDVP_EINTERNAL;
  }
  for (int k = ng; k < nc; ++k) chunks[k].x -= 1;  // scatter chunks index copies[1..2] as tasks 0..1
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&S->task, &task, sizeof(task), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->copies, c, sizeof(c), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->chunks, chunks, nc * sizeof(int2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&S->status, 0, sizeof(int), st);
  if (e != cudaSuccess) {
    set_last_error("tdvp_svd_noalloc: copying descriptors failed");
    return TDVP_ECUDA;
  }
  launch_copy(S->copies, S->chunks, ng, st);
  launch_jacobi_svd(&S->task, 1, Q, 60, 1e-15, &S->status, st);
  launch_copy(S->copies + 1, S->chunks + ng, nc - ng, st);
  int status = 0;
  e = cudaMemcpyAsync(&status, &S->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error("tdvp_svd_noalloc: CUDA error");
    return TDVP_ECUDA;
  }
  if (status) {
    set_last_error("tdvp_svd_noalloc: Jacobi SVD did not converge");
    return TDVP_ENUMERIC;
  }
  return TDVP_OK;
}
