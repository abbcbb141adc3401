// FP64 device kernels of the TDVP engine (CUDA cores, sm_103a).
//
// These are the exact-arithmetic (FP64) building blocks: a grouped complex GEMM
// over planner-built task lists, the MPO linear combination, strided block
// copies, Krylov vector algebra, the small Krylov exponential, one-sided Jacobi
// SVD, truncation selection, block-weighted dots and the entanglement entropy.
// All kernels are symmetry-agnostic; the host planner lowers every contraction
// to task lists (common.hpp).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.hpp"
#include "kernels.hpp"

namespace cg = cooperative_groups;

namespace tdvp {

static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cplx cconj(cplx a) { return {a.x, -a.y}; }
__device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// ---------------------------------------------------------------------------
// K1 (FP64): grouped complex GEMM, 64x64 output tiles, 256 threads, 4x4 per thread
// ---------------------------------------------------------------------------

constexpr int GT = 64;   // tile edge
constexpr int GK = 8;    // k step

__global__ void __launch_bounds__(256) gemm_fp64_kernel(const GemmTask* __restrict__ tasks,
                                                        const GemmSeg* __restrict__ segs,
                                                        const int3* __restrict__ tiles, const Bases4 B,
                                                        const int4* __restrict__ kx, cplx* __restrict__ ws) {
  __shared__ cplx As[GK][GT + 1];
  __shared__ cplx Bs[GK][GT + 1];
  const int3 tr = tiles[blockIdx.x];
  const GemmTask t = tasks[tr.x];
  // the item's K range (a single-segment task split along K) and where it goes
  const int4 ke = kx ? kx[blockIdx.x] : make_int4(0, 0x7fffffff, -1, 0);
  cplx* const cptr = rebase(B, t.c_base, t.c);
  const int m0 = tr.y * GT, n0 = tr.z * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  cplx acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = {0.0, 0.0};

  for (int sgi = 0; sgi < t.seg_count; ++sgi) {
    const GemmSeg sg = segs[t.seg_begin + sgi];
    const cplx* const ap = rebase(B, sg.a_base, sg.a);
    const cplx* const bp = rebase(B, sg.b_base, sg.b);
    const int kend = min(sg.k, ke.y);
    for (int k0 = ke.x; k0 < kend; k0 += GK) {
      // load A tile: GT rows x GK k
      for (int e = threadIdx.x; e < GT * GK; e += 256) {
        int r = e / GK, kk = e % GK;
        int gr = m0 + r, gk = k0 + kk;
        cplx v = {0.0, 0.0};
        if (gr < t.rows && gk < kend) {
          if (sg.op_a == OP_N) v = ap[(long long)gr * sg.lda + gk];
          else v = cconj(ap[(long long)gk * sg.lda + gr]);
        }
        As[kk][r] = v;
      }
      for (int e = threadIdx.x; e < GT * GK; e += 256) {
        int kk = e / GT, c = e % GT;
        int gc = n0 + c, gk = k0 + kk;
        cplx v = {0.0, 0.0};
        if (gc < t.cols && gk < kend) {
          if (sg.op_b == OP_N) v = bp[(long long)gk * sg.ldb + gc];
          else v = cconj(bp[(long long)gc * sg.ldb + gk]);
        }
        Bs[kk][c] = v;
      }
      __syncthreads();
      const double al = sg.alpha;
#pragma unroll
      for (int kk = 0; kk < GK; ++kk) {
        cplx a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          a[i] = As[kk][ty + 16 * i];
          a[i].x *= al;
          a[i].y *= al;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
      }
      __syncthreads();
    }
  }
  if (ke.z >= 0) {  // a K chunk: the whole 64 x 64 partial tile to its slot (zeros outside C)
    cplx* const part = ws + (long long)ke.z * (GT * GT);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[(ty + 16 * i) * GT + tx + 16 * j] = acc[i][j];
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = m0 + ty + 16 * i;
    if (r >= t.rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = n0 + tx + 16 * j;
      if (c < t.cols) cptr[(long long)r * t.ldc + c] = acc[i][j];
    }
  }
}

// C tile = the sum of its K-chunk partials, in chunk order
__global__ void __launch_bounds__(256) gemm_fp64_fix_kernel(const GemmTask* __restrict__ tasks,
                                                            const int4* __restrict__ fix,
                                                            const cplx* __restrict__ ws, const Bases4 B) {
  const int4 f = fix[blockIdx.x];
  const GemmTask t = tasks[f.x];
  cplx* const cptr = rebase(B, t.c_base, t.c);
  const int slot0 = f.w & 0xFFFFF, nch = f.w >> 20;
  const int m0 = f.y * GT, n0 = f.z * GT;
  for (int e = threadIdx.x; e < GT * GT; e += 256) {
    const int r = m0 + e / GT, c = n0 + e % GT;
    if (r >= t.rows || c >= t.cols) continue;
    cplx v = ws[(long long)slot0 * (GT * GT) + e];
    for (int q = 1; q < nch; ++q) {
      const cplx w = ws[(long long)(slot0 + q) * (GT * GT) + e];
      v.x += w.x;
      v.y += w.y;
    }
    cptr[(long long)r * t.ldc + c] = v;
  }
}

void launch_gemm_fp64(const GemmTask* tasks, const GemmSeg* segs, const int3* tiles, int ntiles, const Bases4& B,
                      cudaStream_t s, const int4* kx, cplx* ws) {
  if (ntiles <= 0) return;
  note_launch();
  gemm_fp64_kernel<<<ntiles, 256, 0, s>>>(tasks, segs, tiles, B, kx, ws);
}

void launch_gemm_fp64_fix(const GemmTask* tasks, const int4* fix, int nfix, const cplx* ws, const Bases4& B,
                          cudaStream_t s) {
  if (nfix <= 0) return;
  note_launch();
  gemm_fp64_fix_kernel<<<nfix, 256, 0, s>>>(tasks, fix, ws, B);
}

// ---------------------------------------------------------------------------
// K3: MPO linear combination  out = sum coef * in
// ---------------------------------------------------------------------------

// With tags, every chunk also raises the exponent tags of its rows for the BF16x4
// split of the output (epoch in bits 12-31, the largest biased exponent of max(|Re|,
// |Im|) in bits 0-11; zeros leave a row's tag alone): the rows of a chunk are reduced
// in shared memory first, then merged with one atomicMax per row.
__global__ void __launch_bounds__(256) lincomb_kernel(const LincombTask* __restrict__ tasks,
                                                      const LincombTerm* __restrict__ terms,
                                                      const int2* __restrict__ chunks, unsigned epoch) {
  __shared__ unsigned rmax[LINCOMB_CHUNK];
  const int2 ch = chunks[blockIdx.x];
  const LincombTask t = tasks[ch.x];
  const int n = t.rows * t.cols;
  const int e1 = min(n, ch.y + LINCOMB_CHUNK);
  const int r_first = ch.y / t.cols, r_last = (e1 - 1) / t.cols;
  if (t.tags) {
    for (int i = threadIdx.x; i <= r_last - r_first; i += 256) rmax[i] = 0u;
    __syncthreads();
  }
  for (int e = ch.y + threadIdx.x; e < e1; e += 256) {
    int r = e / t.cols, c = e - r * t.cols;
    cplx acc = {0.0, 0.0};
    for (int k = 0; k < t.term_count; ++k) {
      const LincombTerm tm = terms[t.term_begin + k];
      cplx v = tm.in[(long long)r * tm.ld_in + c];
      acc.x = fma(tm.coef, v.x, acc.x);
      acc.y = fma(tm.coef, v.y, acc.y);
    }
    t.out[(long long)r * t.ld_out + c] = acc;
    if (t.tags) {
      const unsigned ex =
          (unsigned)(((unsigned long long)__double_as_longlong(fmax(fabs(acc.x), fabs(acc.y))) >> 52) & 0x7FF);
      if (ex) atomicMax(&rmax[r - r_first], ex);
    }
  }
  if (t.tags) {
    __syncthreads();
    for (int i = threadIdx.x; i <= r_last - r_first; i += 256)
      if (rmax[i]) atomicMax(&t.tags[r_first + i], (epoch << 12) | rmax[i]);
  }
}

void launch_lincomb(const LincombTask* tasks, const LincombTerm* terms, const int2* chunks, int nchunks,
                    cudaStream_t s, unsigned epoch) {
  if (nchunks <= 0) return;
  note_launch();
  lincomb_kernel<<<nchunks, 256, 0, s>>>(tasks, terms, chunks, epoch);
}

// ---------------------------------------------------------------------------
// strided block copy with optional maps, conjugation and scaling
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) copy_kernel(const CopyTask* __restrict__ tasks, const int2* __restrict__ chunks) {
  const int2 ch = chunks[blockIdx.x];
  const CopyTask t = tasks[ch.x];
  const int n = t.rows * t.cols;
  const double g = t.gscale ? *t.gscale : 1.0;
  for (int e = ch.y + threadIdx.x; e < min(n, ch.y + LINCOMB_CHUNK); e += 256) {
    int r = e / t.cols, c = e - r * t.cols;
    int sr = t.row_map ? t.row_map[r] : r;
    int sc = t.col_map ? t.col_map[c] : c;
    cplx v = t.src[sr * t.src_rs + sc * t.src_cs];
    if (t.conj) v.y = -v.y;
    double f = g;
    switch (t.scale_mode) {
      case 1: f *= t.scale[c]; break;
      case 2: f = t.scale[c] != 0.0 ? f / t.scale[c] : 0.0; break;
      case 3: f *= t.scale[r]; break;
      case 4: f = t.scale[r] != 0.0 ? f / t.scale[r] : 0.0; break;
      default: break;
    }
    v.x *= f;
    v.y *= f;
    t.dst[r * t.dst_rs + c * t.dst_cs] = v;
  }
}

void launch_copy(const CopyTask* tasks, const int2* chunks, int nchunks, cudaStream_t s) {
  if (nchunks <= 0) return;
  note_launch();
  copy_kernel<<<nchunks, 256, 0, s>>>(tasks, chunks);
}

// ---------------------------------------------------------------------------
// K4: Krylov vector algebra (FP64, deterministic two-stage reductions)
// ---------------------------------------------------------------------------

// partial[j * G + g] = sum over block g's range of conj(V_j) * w, j < nv
__global__ void __launch_bounds__(256) dots_partial_kernel(const cplx* __restrict__ V, long long pitch, int nv,
                                                           const cplx* __restrict__ w, long long n,
                                                           cplx* __restrict__ partial, const int* done) {
  if (done && *done) return;
  const int j = blockIdx.y;
  if (j >= nv) return;
  const cplx* v = V + pitch * j;
  cplx acc = {0.0, 0.0};
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    cplx a = v[i], b = w[i];
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
  }
  __shared__ double sx[256], sy[256];
  sx[threadIdx.x] = acc.x;
  sy[threadIdx.x] = acc.y;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sx[threadIdx.x] += sx[threadIdx.x + o];
      sy[threadIdx.x] += sy[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(long long)j * gridDim.x + blockIdx.x] = {sx[0], sy[0]};
}

// out[j] = sum_g partial[j*G+g]; one warp per j, fixed order
__global__ void dots_final_kernel(const cplx* __restrict__ partial, int G, int nv, cplx* __restrict__ out,
                                  const int* done) {
  if (done && *done) return;
  int j = blockIdx.x;
  if (j >= nv) return;
  double x = 0, y = 0;
  for (int g = threadIdx.x; g < G; g += 32) {
    x += partial[(long long)j * G + g].x;
    y += partial[(long long)j * G + g].y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
  }
  if (threadIdx.x == 0) out[j] = {x, y};
}

// w -= sum_j h[j] V_j
__global__ void __launch_bounds__(256) axpy_many_kernel(const cplx* __restrict__ V, long long pitch, int nv,
                                                        const cplx* __restrict__ h, cplx* __restrict__ w,
                                                        long long n, const int* done) {
  if (done && *done) return;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    cplx acc = w[i];
    for (int j = 0; j < nv; ++j) {
      cplx v = V[pitch * j + i], c = h[j];
      acc.x -= c.x * v.x - c.y * v.y;
      acc.y -= c.x * v.y + c.y * v.x;
    }
    w[i] = acc;
  }
}

// out = sum_j coef[j] * V_j * scale   (coef on device, scale = *scal)
__global__ void __launch_bounds__(256) combine_kernel(const cplx* __restrict__ V, long long pitch, const int* nvp,
                                                      const cplx* __restrict__ coef, const double* scal,
                                                      cplx* __restrict__ out, long long n) {
  const int nv = *nvp;
  const double s = scal ? *scal : 1.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    cplx acc = {0.0, 0.0};
    for (int j = 0; j < nv; ++j) {
      cplx v = V[pitch * j + i], c = coef[j];
      acc.x += c.x * v.x - c.y * v.y;
      acc.y += c.x * v.y + c.y * v.x;
    }
    out[i] = {acc.x * s, acc.y * s};
  }
}

// y = x / (*nrm) unless done; if nrm==0 leave y = 0
__global__ void __launch_bounds__(256) scale_kernel(const cplx* __restrict__ x, const double* nrm,
                                                    cplx* __restrict__ y, long long n, const int* done) {
  if (done && *done) return;
  double b = *nrm;
  double f = b > 0 ? 1.0 / b : 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    cplx v = x[i];
    y[i] = {v.x * f, v.y * f};
  }
}

static int blas_grid(long long n) {
  long long g = (n + 255) / 256;
  if (g > 148 * 8) g = 148 * 8;
  if (g < 1) g = 1;
  return (int)g;
}

void launch_dots(const cplx* V, long long pitch, int nv, const cplx* w, long long n, cplx* partial, int G,
                 cplx* out, const int* done, cudaStream_t s) {
  dim3 grid(G, nv);
  note_launch();
  dots_partial_kernel<<<grid, 256, 0, s>>>(V, pitch, nv, w, n, partial, done);
  note_launch();
  dots_final_kernel<<<nv, 32, 0, s>>>(partial, G, nv, out, done);
}

void launch_axpy_many(const cplx* V, long long pitch, int nv, const cplx* h, cplx* w, long long n, const int* done,
                      cudaStream_t s) {
  note_launch();
  axpy_many_kernel<<<blas_grid(n), 256, 0, s>>>(V, pitch, nv, h, w, n, done);
}

void launch_combine(const cplx* V, long long pitch, const int* nv, const cplx* coef, const double* scal, cplx* out,
                    long long n, cudaStream_t s) {
  note_launch();
  combine_kernel<<<blas_grid(n), 256, 0, s>>>(V, pitch, nv, coef, scal, out, n);
}

void launch_scale(const cplx* x, const double* nrm, cplx* y, long long n, const int* done, cudaStream_t s) {
  note_launch();
  scale_kernel<<<blas_grid(n), 256, 0, s>>>(x, nrm, y, n, done);
}

int dots_grid(long long n) { return blas_grid(n) > 296 ? 296 : blas_grid(n); }

// ---------------------------------------------------------------------------
// Krylov bookkeeping kernels (single thread / single warp)
// ---------------------------------------------------------------------------

// st->beta0 = sqrt(Re(nrm2)); st->k = 0; st->done = (beta0 == 0)
__global__ void krylov_init_kernel(KrylovState* st, const cplx* nrm2) {
  double b = sqrt(fmax(nrm2->x, 0.0));
  st->beta0 = b;
  st->k = 0;
  st->done = b > 0.0 ? 0 : 1;
  st->nv = 0;
  st->err = 0.0;
  st->bad = (b == b) ? 0 : 1;
  if (st->bad) st->done = 1;
}

// After the reorthogonalised w and its squared norm: record alpha_k, beta_k, then
// compute c = exp(-i tau T_k) e_1 by a scaled Taylor series of the vector
// (one lane per Krylov index), estimate the error beta_k |c_k| and decide.
__global__ void krylov_step_kernel(KrylovState* st, const cplx* h1, const cplx* nrm2, double tau, double tol,
                                   int kmax) {
  if (st->done) return;
  const int lane = threadIdx.x;
  const int k = st->k;  // index of the vector just applied (0-based)
  if (lane == 0) {
    st->alpha[k] = h1[k].x;
    st->beta[k] = sqrt(fmax(nrm2->x, 0.0));
  }
  __syncwarp();
  const int n = k + 1;
  double al = lane < n ? st->alpha[lane] : 0.0;
  double bl = lane < n - 1 ? st->beta[lane] : 0.0;          // couples lane and lane+1
  double bm = (lane > 0 && lane < n) ? st->beta[lane - 1] : 0.0;  // couples lane-1 and lane
  double rowsum = lane < n ? fabs(al) + bl + bm : 0.0;
  int bad = !(rowsum < 1e12);  // NaN or absurd: stop instead of looping
  for (int o = 16; o > 0; o >>= 1) {
    rowsum = fmax(rowsum, __shfl_xor_sync(0xffffffffu, rowsum, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (bad) {
    if (lane == 0) {
      st->bad = 1;
      st->done = 1;
      st->nv = 0;
    }
    return;
  }
  // steps of |h| ||T||_inf <= 4: the Taylor terms of the unitary exp(-i h T) peak near
  // e^4 / sqrt(8 pi) ~ 11 before they decay (cancellation of ~1e-15 of the result) and fall
  // below 1e-22 within 40 terms; the size of the last terms is checked every fourth term
  int steps = (int)ceil(fabs(tau) * rowsum / 4.0);
  if (steps < 1) steps = 1;
  const double h = tau / steps;
  double xr = lane == 0 ? 1.0 : 0.0, xi = 0.0;
  for (int s = 0; s < steps; ++s) {
    double tr = xr, ti = xi, sr = xr, si = xi;
    for (int m = 1; m <= 64; ++m) {
      // y = T t
      double upr = __shfl_down_sync(0xffffffffu, tr, 1), upi = __shfl_down_sync(0xffffffffu, ti, 1);
      double dnr = __shfl_up_sync(0xffffffffu, tr, 1), dni = __shfl_up_sync(0xffffffffu, ti, 1);
      double yr = al * tr + bl * upr + bm * dnr;
      double yi = al * ti + bl * upi + bm * dni;
      if (lane >= n) yr = yi = 0.0;
      // t = (-i h / m) y
      double f = h / m;
      tr = f * yi;
      ti = -f * yr;
      sr += tr;
      si += ti;
      if ((m & 3) == 0) {
        double mag = fabs(tr) + fabs(ti);
        for (int o = 16; o > 0; o >>= 1) mag = fmax(mag, __shfl_xor_sync(0xffffffffu, mag, o));
        if (mag < 1e-22) break;
      }
    }
    xr = sr;
    xi = si;
  }
  if (lane < n) st->coef[lane] = {xr, xi};
  double last_r = __shfl_sync(0xffffffffu, xr, n - 1), last_i = __shfl_sync(0xffffffffu, xi, n - 1);
  if (lane == 0) {
    double b = st->beta[k];
    double err = b * sqrt(last_r * last_r + last_i * last_i);
    st->err = err;
    st->nv = n;
    if (!(err == err)) {
      st->bad = 1;
      st->nv = 0;
    }
    if (err < tol || b < 1e-14 || n >= kmax) st->done = 1;
    st->k = k + 1;
  }
}

void launch_krylov_init(KrylovState* st, const cplx* nrm2, cudaStream_t s) {
  note_launch();
  krylov_init_kernel<<<1, 1, 0, s>>>(st, nrm2);
}

void launch_krylov_step(KrylovState* st, const cplx* h1, const cplx* nrm2, double tau, double tol, int kmax,
                        cudaStream_t s) {
  note_launch();
  krylov_step_kernel<<<1, 32, 0, s>>>(st, h1, nrm2, tau, tol, kmax);
}

// ---------------------------------------------------------------------------
// K6: one-sided (Hestenes) Jacobi SVD, one CTA per problem
// ---------------------------------------------------------------------------

constexpr int SVD_THREADS = 256;

__device__ void col_pair(cplx* __restrict__ g, int p, int i, int j, double& a, double& b, cplx& c) {
  const int lane = threadIdx.x & 31;
  double sa = 0, sb = 0, cx = 0, cy = 0;
  const cplx* gi = g + (long long)i * p;
  const cplx* gj = g + (long long)j * p;
  for (int r = lane; r < p; r += 32) {
    cplx x = gi[r], y = gj[r];
    sa = fma(x.x, x.x, fma(x.y, x.y, sa));
    sb = fma(y.x, y.x, fma(y.y, y.y, sb));
    cx = fma(x.x, y.x, fma(x.y, y.y, cx));
    cy = fma(x.x, y.y, fma(-x.y, y.x, cy));
  }
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
    cx += __shfl_xor_sync(0xffffffffu, cx, o);
    cy += __shfl_xor_sync(0xffffffffu, cy, o);
  }
  a = sa;
  b = sb;
  c = {cx, cy};
}

__device__ void rotate_cols(cplx* __restrict__ g, int ld, int len, int i, int j, double cs, double sn, cplx e) {
  // g_i' = cs g_i - sn conj(e) g_j ; g_j' = sn e g_i + cs g_j
  const int lane = threadIdx.x & 31;
  cplx* gi = g + (long long)i * ld;
  cplx* gj = g + (long long)j * ld;
  for (int r = lane; r < len; r += 32) {
    cplx x = gi[r], y = gj[r];
    cplx ey = {e.x * y.x + e.y * y.y, e.x * y.y - e.y * y.x};  // conj(e) * y
    cplx ex = {e.x * x.x - e.y * x.y, e.x * x.y + e.y * x.x};  // e * x
    gi[r] = {cs * x.x - sn * ey.x, cs * x.y - sn * ey.y};
    gj[r] = {sn * ex.x + cs * y.x, sn * ex.y + cs * y.y};
  }
}

__global__ void __launch_bounds__(SVD_THREADS) jacobi_svd_kernel(const SvdTask* __restrict__ tasks, int max_sweeps,
                                                                 double tol, int* __restrict__ status) {
  const SvdTask t = tasks[blockIdx.x];
  const int p = t.p, q = t.q;
  const int warp = threadIdx.x >> 5, nwarp = SVD_THREADS / 32;
  for (int e = threadIdx.x; t.v && e < q * q; e += SVD_THREADS) {
    int r = e % q, c = e / q;
    t.v[e] = {r == c ? 1.0 : 0.0, 0.0};
  }
  __shared__ int rotated;
  __syncthreads();
  const int qq = q + (q & 1);
  const int m = qq - 1;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < m; ++r) {
      for (int k = warp; k < qq / 2; k += nwarp) {
        int i, j;
        if (k == 0) {
          i = 0;
          j = 1 + r % m;
        } else {
          i = 1 + (r + k) % m;
          j = 1 + (r - k + m) % m;
        }
        if (i > j) {
          int tmp = i;
          i = j;
          j = tmp;
        }
        if (j >= q) continue;
        double a, b;
        cplx c;
        col_pair(t.g, p, i, j, a, b, c);
        double ac = sqrt(c.x * c.x + c.y * c.y);
        if (ac == 0.0 || ac <= tol * sqrt(a * b)) continue;
        double zeta = (b - a) / (2.0 * ac);
        double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
        cplx e = {c.x / ac, c.y / ac};
        rotate_cols(t.g, p, p, i, j, cs, sn, e);
        if (t.v) rotate_cols(t.v, q, q, i, j, cs, sn, e);
        if ((threadIdx.x & 31) == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (threadIdx.x == 0 && sweep >= max_sweeps) atomicAdd(status, 1);
  // singular values = column norms, then sort descending (rank counting, ties by index)
  for (int j = warp; j < q; j += nwarp) {
    double a, b;
    cplx c;
    col_pair(t.g, p, j, j, a, b, c);
    if ((threadIdx.x & 31) == 0) t.sv[j] = sqrt(a);  // temporarily unsorted
  }
  __syncthreads();
  // rank of each value; write perm, then sorted values into shared staging via sv in place
  extern __shared__ double sbuf[];  // q doubles; NaN ranks last so the ranks stay a permutation
  for (int j = threadIdx.x; j < q; j += SVD_THREADS) {
    double v = t.sv[j];
    sbuf[j] = (v == v) ? v : -1.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < q; j += SVD_THREADS) {
    double vj = sbuf[j];
    int rank = 0;
    for (int i = 0; i < q; ++i) {
      double vi = sbuf[i];
      rank += (vi > vj) || (vi == vj && i < j);
    }
    t.perm[rank] = j;
    t.sv[rank] = vj < 0.0 ? 0.0 : vj;
  }
}

// ---------------------------------------------------------------------------
// K6: one-sided Jacobi SVD of many matrices at once, one cooperative launch
//
// The classical round-robin ordering: the n columns of a problem (n padded to even)
// form n/2 disjoint pairs in each of n - 1 rounds, and a sweep of n - 1 rounds
// meets every pair once.  A single cooperative launch runs every sweep: in each
// round every warp of the grid takes pairs from the work list (all problems, sorted
// by size so that the pairs still active in a round are a prefix), computes the two
// squared norms and the overlap, and applies the complex Jacobi rotation (as in
// jacobi_svd_kernel) to both columns of G and, when present, of V; a grid-wide
// barrier separates rounds.  After each sweep every CTA reads the per-problem
// rotation flags; the loop ends, uniformly over the grid, after a sweep without
// flags.  Columns of up to 32 R rows stay in registers between the reduction and
// the rotation.  The working copies (a bond's worth of sectors) stay in L2.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tourney(int r, int k, int n, int& i, int& j) {
  const int m = n - 1;
  if (k == 0) {
    i = 0;
    j = 1 + r % m;
  } else {
    i = 1 + (r + k) % m;
    j = 1 + (r - k + m) % m;
  }
  if (i > j) {
    int t = i;
    i = j;
    j = t;
  }
}

constexpr int JT = 256;  // threads per CTA of the cooperative Jacobi

// x' = cs x - sn conj(e) y ; y' = sn e x + cs y.  Written with explicit fma so that
// every instantiation (registers or memory, global or shared) rounds the same way.
template <class S, class C2>
__device__ __forceinline__ void rot2(C2& x, C2& y, S cs, S sn, S ex, S ey) {
  const C2 a = x, b = y;
  const S u = fma(ex, b.x, ey * b.y), w = fma(ex, b.y, -(ey * b.x));   // conj(e) y
  const S f = fma(ex, a.x, -(ey * a.y)), h = fma(ex, a.y, ey * a.x);   // e x
  x.x = fma(cs, a.x, -(sn * u));
  x.y = fma(cs, a.y, -(sn * w));
  y.x = fma(sn, f, cs * b.x);
  y.y = fma(sn, h, cs * b.y);
}

// one column pair by one warp, given the two columns of G (p rows) and, when V is
// accumulated, of V (q rows); any address space (global, shared, a cluster peer's
// shared memory).  R > 0: rows lane + 32 k (k < R) in registers.
template <class S, class C2, int R>
__device__ __forceinline__ void warp_pair_cols(C2* __restrict__ gi, C2* __restrict__ gj, C2* __restrict__ vi,
                                               C2* __restrict__ vj, int p, int q, S tol, S tol_flag, S abs_flag,
                                               int* __restrict__ flag) {
  const int lane = threadIdx.x & 31;
  S sa = 0, sb = 0, cx = 0, cy = 0;
  constexpr int RR = R > 0 ? R : 1;
  constexpr bool kPrefetchV = R > 0 && sizeof(S) == 4;
  C2 x[RR], y[RR];
  C2 va[kPrefetchV ? RR : 1], vb[kPrefetchV ? RR : 1];
  if (R > 0) {
#pragma unroll
    for (int k = 0; k < RR; ++k) {
      const int r = lane + 32 * k;
      if (r < p) {
        x[k] = gi[r];
        y[k] = gj[r];
      } else {
        x[k].x = x[k].y = y[k].x = y[k].y = S(0);
      }
    }
    if constexpr (kPrefetchV) {
      // FP32 (the preconditioner, which accumulates V): q <= p <= 32 R.  The two V
      // columns are loaded together with G, so their latency overlaps G's instead of
      // following the rotation decision; unused when the pair does not rotate.
      if (vi) {
#pragma unroll
        for (int k = 0; k < RR; ++k) {
          const int r = lane + 32 * k;
          if (r < q) {
            va[k] = vi[r];
            vb[k] = vj[r];
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < RR; ++k) {
      sa = fma(x[k].x, x[k].x, fma(x[k].y, x[k].y, sa));
      sb = fma(y[k].x, y[k].x, fma(y[k].y, y[k].y, sb));
      cx = fma(x[k].x, y[k].x, fma(x[k].y, y[k].y, cx));
      cy = fma(x[k].x, y[k].y, fma(-x[k].y, y[k].x, cy));
    }
  } else {
#pragma unroll 4
    for (int r = lane; r < p; r += 32) {
      const C2 a = gi[r], b = gj[r];
      sa = fma(a.x, a.x, fma(a.y, a.y, sa));
      sb = fma(b.x, b.x, fma(b.y, b.y, sb));
      cx = fma(a.x, b.x, fma(a.y, b.y, cx));
      cy = fma(a.x, b.y, fma(-a.y, b.x, cy));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
    cx += __shfl_xor_sync(0xffffffffu, cx, o);
    cy += __shfl_xor_sync(0xffffffffu, cy, o);
  }
  const S ac = sqrt(fma(cx, cx, cy * cy));
  if (ac == S(0) || ac <= tol * sqrt(sa * sb)) return;  // warp-uniform
  const S zeta = (sb - sa) / (S(2) * ac);
  const S tt = (zeta >= 0 ? S(1) : S(-1)) / (fabs(zeta) + sqrt(fma(zeta, zeta, S(1))));
  const S cs = S(1) / sqrt(fma(tt, tt, S(1))), sn = cs * tt;
  const S ex = cx / ac, ey = cy / ac;
  if (R > 0) {
#pragma unroll
    for (int k = 0; k < RR; ++k) {
      const int r = lane + 32 * k;
      if (r < p) {
        rot2(x[k], y[k], cs, sn, ex, ey);
        gi[r] = x[k];
        gj[r] = y[k];
      }
    }
  } else {
#pragma unroll 4
    for (int r = lane; r < p; r += 32) {
      C2 a = gi[r], b = gj[r];
      rot2(a, b, cs, sn, ex, ey);
      gi[r] = a;
      gj[r] = b;
    }
  }
  if (vi) {
    if constexpr (kPrefetchV) {  // V rows loaded above (the FP64 instances keep the
                                 // loop below for their register budget)
#pragma unroll
      for (int k = 0; k < RR; ++k) {
        const int r = lane + 32 * k;
        if (r < q) {
          rot2(va[k], vb[k], cs, sn, ex, ey);
          vi[r] = va[k];
          vj[r] = vb[k];
        }
      }
    } else {
#pragma unroll 4
      for (int r = lane; r < q; r += 32) {
        C2 a = vi[r], b = vj[r];
        rot2(a, b, cs, sn, ex, ey);
        vi[r] = a;
        vj[r] = b;
      }
    }
  }
  if (lane == 0 && ac > tol_flag * sqrt(sa * sb) && ac > abs_flag) atomicOr(flag, 1);
}

// column pair (i, j) of a column-major p x q G (and q x q V, or none)
template <class S, class C2, int R>
__device__ __forceinline__ void warp_pair(C2* __restrict__ g, C2* __restrict__ v, int p, int q, int i, int j, S tol,
                                          S tol_flag, S abs_flag, int* __restrict__ flag) {
  warp_pair_cols<S, C2, R>(g + (long long)i * p, g + (long long)j * p, v ? v + (long long)i * q : nullptr,
                           v ? v + (long long)j * q : nullptr, p, q, tol, tol_flag, abs_flag, flag);
}

template <class Task, class S, class C2, int R>
__global__ void __launch_bounds__(JT) jacobi_coop_kernel(const Task* __restrict__ tasks, int nt,
                                                         const int2* __restrict__ work, const int* __restrict__ active,
                                                         int nrounds, int max_sweeps, S tol, S tol_flag, S abs_flag,
                                                         int* __restrict__ flags, int* __restrict__ out,
                                                         int* __restrict__ task_sweeps) {
  cg::grid_group grid = cg::this_grid();
  // pair w goes to CTA w mod G (warp w div G there): consecutive pairs -- the pairs of
  // one large sector -- land on different SMs instead of sharing one SM's pipes
  const int nwarps = (gridDim.x * JT) >> 5;
  const int gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  __shared__ int any_s;
  int* now = flags;
  const int* prev = nullptr;
  int sweep = 0;
  bool conv = false;
  for (; sweep < max_sweeps; ++sweep) {
    if (blockIdx.x == 0)
      for (int e = threadIdx.x; e < nt; e += JT) {
        now[e] = 0;
        if (!prev || prev[e]) ++task_sweeps[e];  // the task takes part in this sweep
      }
    grid.sync();
    for (int r = 0; r < nrounds; ++r) {
      const int na = active[r];
      for (int w = gw; w < na; w += nwarps) {
        const int2 wk = work[w];
        if (prev && prev[wk.x] == 0) continue;  // converged in the previous sweep
        const Task t = tasks[wk.x];
        const int n = t.q + (t.q & 1);
        if (r >= n - 1) continue;
        int i, j;
        tourney(r, wk.y, n, i, j);
        if (j >= t.q) continue;
        warp_pair<S, C2, R>(t.g, t.v, t.p, t.q, i, j, tol, tol_flag, abs_flag, now + wk.x);
      }
      grid.sync();
    }
    if (threadIdx.x == 0) {
      int any = 0;
      for (int e = 0; e < nt; ++e) any |= reinterpret_cast<volatile int*>(now)[e];
      any_s = any;
    }
    __syncthreads();
    const int any = any_s;
    __syncthreads();
    if (!any) {
      conv = true;
      ++sweep;
      break;
    }
    prev = now;
    now = (now == flags) ? flags + nt : flags;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out[0] = sweep;
    out[1] = conv ? 0 : 1;
  }
}

// The same Jacobi for sectors small enough to live in one CTA's shared memory (used
// when every sector of a call is that small): the
// CTA loads its p x q working copy once, runs the sweeps with the same tournament,
// the same pair arithmetic (warp_pair on the shared copy) and the same stopping rule,
// with a CTA barrier per round instead of a grid barrier, and writes the copy back.
// V stays in global memory.  Per sector the result is the one the cooperative
// kernel gives: the rounds see the same pairs in the same order and each pair the
// same operations.
constexpr int RJT = 512;                     // threads per CTA of the resident Jacobi
constexpr int RJ_SMEM = 192 * 1024;          // bytes of the largest resident working copy
constexpr int RJ_QMAX = 2 * (RJT / 32);      // columns: one pair per warp and round

template <class Task, class S, class C2>
__global__ void __launch_bounds__(RJT) jacobi_resident_kernel(const Task* __restrict__ tasks,
                                                              const int* __restrict__ ids, int max_sweeps, S tol,
                                                              S tol_flag, S abs_flag, int* __restrict__ task_sweeps,
                                                              int* __restrict__ nonconv) {
  extern __shared__ __align__(16) unsigned char rj_smem[];
  C2* g = reinterpret_cast<C2*>(rj_smem);
  __shared__ int flag_s;
  const int id = ids[blockIdx.x];
  const Task t = tasks[id];
  const int p = t.p, q = t.q;
  const long long pq = (long long)p * q;
  for (long long e = threadIdx.x; e < pq; e += RJT) g[e] = t.g[e];
  const int warp = threadIdx.x >> 5, nw = RJT >> 5;
  const int n = q + (q & 1);
  int sweep = 0;
  bool conv = false;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) flag_s = 0;
    __syncthreads();
    for (int r = 0; r < n - 1; ++r) {
      for (int k = warp; k < n / 2; k += nw) {
        int i, j;
        tourney(r, k, n, i, j);
        if (j >= q) continue;
        warp_pair<S, C2, 0>(g, t.v, p, q, i, j, tol, tol_flag, abs_flag, &flag_s);
      }
      __syncthreads();
    }
    const int f = flag_s;
    __syncthreads();
    if (!f) {
      conv = true;
      ++sweep;
      break;
    }
  }
  for (long long e = threadIdx.x; e < pq; e += RJT) t.g[e] = g[e];
  if (threadIdx.x == 0) {
    task_sweeps[id] = sweep;
    if (!conv) atomicOr(nonconv, 1);
  }
}

// The same Jacobi with each sector held in the shared memory of one thread-block
// cluster (C CTAs): column c of G (and of V) lives in CTA c mod C, slot c div C.  A
// round's pairs are spread over the cluster's warps, which read and rotate the two
// columns where they live (distributed shared memory); a cluster barrier ends each
// round.  Same tournament, pair arithmetic and stopping rule as the other forms.
constexpr int CJT = 1024;           // threads per CTA of the cluster Jacobi
constexpr int CJ_SMEM = 200 * 1024; // bytes of one CTA's slice

template <class Task, class S, class C2>
__global__ void __launch_bounds__(CJT) jacobi_cluster_kernel(const Task* __restrict__ tasks,
                                                             const int* __restrict__ ids, int max_sweeps, S tol,
                                                             S tol_flag, S abs_flag, int* __restrict__ task_sweeps,
                                                             int* __restrict__ nonconv) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int id = ids[blockIdx.x / C];
  extern __shared__ __align__(16) unsigned char cj_smem[];
  __shared__ int flag_s;
  const Task t = tasks[id];
  const int p = t.p, q = t.q;
  const bool with_v = t.v != nullptr;
  const int slots = (q + C - 1) / C;  // column slots per CTA
  C2* gl = reinterpret_cast<C2*>(cj_smem);
  C2* vl = gl + (long long)slots * p;
  for (int l = 0; rank + C * l < q; ++l) {
    const int c = rank + C * l;
    for (int r = threadIdx.x; r < p; r += CJT) gl[(long long)l * p + r] = t.g[(long long)c * p + r];
    if (with_v)
      for (int r = threadIdx.x; r < q; r += CJT) vl[(long long)l * q + r] = t.v[(long long)c * q + r];
  }
  int* flag0 = cl.map_shared_rank(&flag_s, 0);
  const int warp = threadIdx.x >> 5, nw = CJT >> 5;
  const int gw = rank * nw + warp, W = C * nw;
  const int n = q + (q & 1);
  int sweep = 0;
  bool conv = false;
  for (; sweep < max_sweeps; ++sweep) {
    if (rank == 0 && threadIdx.x == 0) flag_s = 0;
    cl.sync();  // slices loaded (first sweep), flag reset
    for (int r = 0; r < n - 1; ++r) {
      for (int k = gw; k < n / 2; k += W) {
        int i, j;
        tourney(r, k, n, i, j);
        if (j >= q) continue;
        C2* gi = cl.map_shared_rank(gl + (long long)(i / C) * p, i % C);
        C2* gj = cl.map_shared_rank(gl + (long long)(j / C) * p, j % C);
        C2* vi = with_v ? cl.map_shared_rank(vl + (long long)(i / C) * q, i % C) : nullptr;
        C2* vj = with_v ? cl.map_shared_rank(vl + (long long)(j / C) * q, j % C) : nullptr;
        warp_pair_cols<S, C2, 0>(gi, gj, vi, vj, p, q, tol, tol_flag, abs_flag, flag0);
      }
      cl.sync();
    }
    const int f = *reinterpret_cast<volatile int*>(flag0);
    cl.sync();  // every CTA has read the flag before it is reset
    if (!f) {
      conv = true;
      ++sweep;
      break;
    }
  }
  for (int l = 0; rank + C * l < q; ++l) {
    const int c = rank + C * l;
    for (int r = threadIdx.x; r < p; r += CJT) t.g[(long long)c * p + r] = gl[(long long)l * p + r];
    if (with_v)
      for (int r = threadIdx.x; r < q; r += CJT) t.v[(long long)c * q + r] = vl[(long long)l * q + r];
  }
  if (rank == 0 && threadIdx.x == 0) {
    task_sweeps[id] = sweep;
    if (!conv) atomicOr(nonconv, 1);
  }
}

// ---------------------------------------------------------------------------
// The FP32 preconditioner as rings of warps inside thread-block clusters.  A
// sector of n columns (n = q rounded up to even) is served by h = n/2 consecutive
// warps of one cluster, warp k holding the two columns of round-robin pair k (the
// pair tourney(r, k, n) gives) in registers: G rows lane + 32 j and the same rows of
// V.  From one round to the next the circle method moves every column except column
// 0 by one position, so warp k's first column goes to warp k-1 (warp 1's to warp 0's
// second slot) and its second column to warp k+1 (warp 0's to warp 1's second slot,
// the last warp's to its own first slot).  A round is therefore: the pair's
// reduction and rotation in registers, the outgoing columns written into the
// receivers' inboxes (shared memory of the receiving CTA, written through
// distributed shared memory), a cluster barrier, the incoming columns read back.
// The barrier that protects an inbox from being overwritten before its owner has read
// it is split: its arrive follows the reads, its wait precedes the next writes, so
// its latency overlaps the rotation.  Every pair, its order within a sweep and its
// arithmetic (the expressions of warp_pair_cols) are those of the cooperative
// kernel, so the results agree bit for bit; but no grid-wide barrier runs, a round
// costs shared-memory traffic instead of an L2 round trip, and each sector stops after
// its own first sweep without flags (its flags live in shared memory of the CTA that
// holds its warp 0, in three slots used in turn so that a slot is cleared a sweep
// before it is reused).  A per-CTA count of the cluster's unfinished sectors, read
// after a barrier, ends the loop uniformly over the cluster.
// ---------------------------------------------------------------------------
constexpr int RING_NW = 16;    // warps per CTA
constexpr int RING_CMAX = 16;  // CTAs per cluster at most (more than 8 is a non-portable size)
constexpr int RING_RMAX = 10;  // rows per lane at most (p <= 320)

__device__ __forceinline__ unsigned ring_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned ring_cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned ring_cluster_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned ring_mapa(const void* p, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void ring_st(unsigned addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void ring_st_s32(unsigned addr, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ int ring_ld_s32(unsigned addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void ring_or(unsigned addr, int v) {
  asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void ring_add(unsigned addr, int v) {
  asm volatile("red.shared::cluster.add.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// the cluster barrier in two halves (every thread of the cluster takes part in each;
// .aligned: the warp is converged first)
__device__ __forceinline__ void ring_arrive() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void ring_wait() {
  __syncwarp();
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// the pair (x = the lower-indexed column) in registers: warp_pair_cols' expressions
template <int R>
__device__ __forceinline__ void ring_pair(float2 (&x)[R], float2 (&y)[R], float2 (&vx)[R], float2 (&vy)[R], float tol,
                                          float tol_flag, float abs_flag, unsigned flag_addr) {
  float sa = 0, sb = 0, cx = 0, cy = 0;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    sa = fmaf(x[k].x, x[k].x, fmaf(x[k].y, x[k].y, sa));
    sb = fmaf(y[k].x, y[k].x, fmaf(y[k].y, y[k].y, sb));
    cx = fmaf(x[k].x, y[k].x, fmaf(x[k].y, y[k].y, cx));
    cy = fmaf(x[k].x, y[k].y, fmaf(-x[k].y, y[k].x, cy));
  }
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
    cx += __shfl_xor_sync(0xffffffffu, cx, o);
    cy += __shfl_xor_sync(0xffffffffu, cy, o);
  }
  const float ac = sqrt(fmaf(cx, cx, cy * cy));
  if (ac == 0.0f || ac <= tol * sqrt(sa * sb)) return;  // warp-uniform
  const float zeta = (sb - sa) / (2.0f * ac);
  const float tt = (zeta >= 0 ? 1.0f : -1.0f) / (fabs(zeta) + sqrt(fmaf(zeta, zeta, 1.0f)));
  const float cs = 1.0f / sqrt(fmaf(tt, tt, 1.0f)), sn = cs * tt;
  const float ex = cx / ac, ey = cy / ac;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    rot2<float, float2>(x[k], y[k], cs, sn, ex, ey);
    rot2<float, float2>(vx[k], vy[k], cs, sn, ex, ey);
  }
  if ((threadIdx.x & 31) == 0 && ac > tol_flag * sqrt(sa * sb) && ac > abs_flag) ring_or(flag_addr, 1);
}

template <int R>
__device__ __forceinline__ void ring_send(unsigned addr, const float2 (&g)[R], const float2 (&v)[R]) {
  const unsigned lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    ring_st(addr + (lane + 32 * k) * 8u, g[k]);
    ring_st(addr + (32 * R + lane + 32 * k) * 8u, v[k]);
  }
}
template <int R>
__device__ __forceinline__ void ring_recv(const float2* slot, float2 (&g)[R], float2 (&v)[R]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    g[k] = slot[lane + 32 * k];
    v[k] = slot[32 * R + lane + 32 * k];
  }
}
template <int R>
__device__ __forceinline__ void ring_load(const Svd32Task& t, int c, float2 (&g)[R], float2 (&v)[R]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int r = lane + 32 * k;
    g[k] = make_float2(0.0f, 0.0f);
    v[k] = make_float2(0.0f, 0.0f);
    if (c < t.q) {
      if (r < t.p) g[k] = t.g[(long long)c * t.p + r];
      if (r < t.q) v[k] = t.v[(long long)c * t.q + r];
    }
  }
}
template <int R>
__device__ __forceinline__ void ring_store(const Svd32Task& t, int c, const float2 (&g)[R], const float2 (&v)[R]) {
  if (c >= t.q) return;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int r = lane + 32 * k;
    if (r < t.p) t.g[(long long)c * t.p + r] = g[k];
    if (r < t.q) t.v[(long long)c * t.q + r] = v[k];
  }
}

// round-robin players of warp k at round r of a sweep (m = n - 1 rounds)
__device__ __forceinline__ void ring_players(int k, int r, int m, int& a, int& b) {
  if (k == 0) {
    a = 0;
    b = 1 + r % m;
  } else {
    a = 1 + (k + r) % m;
    b = 1 + (m - k + r) % m;
  }
}

// host-built placement: one entry per warp slot of a cluster (C x RING_NW per
// cluster, in cluster rank order); task < 0 marks an idle slot.  w0 is the slot of
// the sector's warp 0 within its cluster.
struct RingWarp {
  int task, k, w0, h;
};

// mbarriers of the ring (local: shared::cta addresses; remote: shared::cluster addresses)
constexpr int RING_WAIT_MAX = 1 << 22;  // polls of a ring wait before it reports a timeout
__device__ __forceinline__ void ring_mb_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void ring_mb_arrive_remote(unsigned addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}
// bounded wait for the completion of the phase with this parity; false on timeout
__device__ __forceinline__ bool ring_mb_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  for (int it = 0; it < RING_WAIT_MAX; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void ring_red_add_release(unsigned addr, int v) {
  asm volatile("red.release.cluster.shared::cluster.add.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ int ring_ld_acquire(unsigned addr) {
  int v;
  asm volatile("ld.acquire.cluster.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

template <int R>
__global__ void __launch_bounds__(RING_NW * 32, 1)
    jacobi_ring_kernel(const Svd32Task* __restrict__ tasks, const RingWarp* __restrict__ slots, int max_sweeps,
                       float tol, float tol_flag, float abs_flag, int* __restrict__ task_sweeps,
                       int* __restrict__ err) {
  extern __shared__ __align__(16) float2 ring_inbox[];  // [RING_NW][2][64 R]
  __shared__ __align__(8) unsigned long long full_bar[RING_NW], free_bar[RING_NW];
  // per sector whose warp 0 sits at this local warp: rotation flags and sweep-end
  // arrival counts, three slots each, used in turn
  __shared__ int sect_s[RING_NW][6];
  const unsigned rank = ring_rank(), csize = ring_cluster_size();
  const int cl = (int)ring_cluster_id();
  const int lw = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const RingWarp wd = slots[((long long)cl * csize + rank) * RING_NW + lw];
  const bool member = wd.task >= 0;
  Svd32Task t{};
  int q = 0, m = 1, K = 0;
  const int k = wd.k, w = wd.w0 + wd.k;
  if (member) {
    t = tasks[wd.task];
    q = t.q;
    m = q + (q & 1) - 1;
    K = wd.h - 1;
  }
  // columns received (full_bar arrivals) and sent (free_bar arrivals) per round: one for
  // the first and the last warp of a ring, two in between
  const int n_io = (member && K >= 1) ? ((k == 0 || k == K) ? 1 : 2) : 1;
  if (threadIdx.x < RING_NW * 6) (&sect_s[0][0])[threadIdx.x] = 0;
  if (lane == 0) {
    ring_mb_init(&full_bar[lw], (unsigned)n_io);
    ring_mb_init(&free_bar[lw], (unsigned)n_io);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  ring_arrive();
  ring_wait();  // every CTA's barriers and counters are set before any remote access
  constexpr int SLOT = 64 * R;  // float2 per inbox slot: G rows, then V rows
  const float2* my_a = ring_inbox + (long long)(lw * 2) * SLOT;
  const float2* my_b = my_a + SLOT;
  auto inbox = [&](int x, int s) {
    return ring_mapa(ring_inbox + (long long)((x % RING_NW) * 2 + s) * SLOT, x / RING_NW);
  };
  auto full_of = [&](int x) { return ring_mapa(&full_bar[x % RING_NW], x / RING_NW); };
  auto free_of = [&](int x) { return ring_mapa(&free_bar[x % RING_NW], x / RING_NW); };
  unsigned sect = 0, dst_a = 0, dst_b = 0, full_a = 0, full_b = 0, free_a = 0, free_b = 0;
  if (member) {
    sect = ring_mapa(&sect_s[wd.w0 % RING_NW][0], wd.w0 / RING_NW);
    if (K >= 1) {
      // sends: first column to warp k-1 (warp 1's to warp 0's second slot), second to warp k+1
      if (k >= 2) {
        dst_a = inbox(w - 1, 0);
        full_a = full_of(w - 1);
      } else if (k == 1) {
        dst_a = inbox(wd.w0, 1);
        full_a = full_of(wd.w0);
      }
      if (k < K) {
        dst_b = inbox(w + 1, 1);
        full_b = full_of(w + 1);
      }
      // receives: second column from warp k-1 (warp 0's from warp 1), first from warp k+1
      free_b = free_of(k == 0 ? w + 1 : w - 1);
      if (k >= 1 && k < K) free_a = free_of(w + 1);
    }
  }
  float2 ga[R], gb[R], va[R], vb[R];
  int pa = 0, pb = 0, lr = 0, sweep = 0;
  unsigned full_par = 0, free_par = 0;
  long long gr = 0;
  bool failed = false;
  if (member) {
    ring_players(k, 0, m, pa, pb);
    ring_load<R>(t, pa, ga, va);
    ring_load<R>(t, pb, gb, vb);
  }
  while (member) {
    if (lr == 0 && k == 0 && lane == 0) {  // clear the next sweep's slots (their last readers are done)
      ring_st_s32(sect + 4u * ((sweep + 1) % 3), 0);
      ring_st_s32(sect + 4u * (3 + (sweep + 1) % 3), 0);
    }
    if (pa < q && pb < q) {
      const unsigned fa = sect + 4u * (sweep % 3);
      if (pa < pb) ring_pair<R>(ga, gb, va, vb, tol, tol_flag, abs_flag, fa);
      else ring_pair<R>(gb, ga, vb, va, tol, tol_flag, abs_flag, fa);
    }
    if (lr == m - 1) {  // the sweep's last round: wait until every warp of the ring has rotated
      __syncwarp();
      int f = 0, ok = 1;
      if (lane == 0) {
        const unsigned cnt = sect + 4u * (3 + sweep % 3);
        ring_red_add_release(cnt, 1);
        int it = 0;
        while (ring_ld_acquire(cnt) < wd.h && ++it < RING_WAIT_MAX) {
        }
        ok = it < RING_WAIT_MAX;
        f = ring_ld_acquire(sect + 4u * (sweep % 3));
      }
      f = __shfl_sync(0xffffffffu, f, 0);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      ++sweep;
      if (!ok) {
        failed = true;
        break;
      }
      if (f == 0 || sweep >= max_sweeps) {  // converged: this warp holds the pair it just rotated
        ring_store<R>(t, pa, ga, va);
        ring_store<R>(t, pb, gb, vb);
        if (k == 0 && lane == 0) task_sweeps[wd.task] = sweep;
        break;
      }
    }
    if (K >= 1) {
      if (gr >= 1) {  // the receivers have read what this warp sent in the previous round
        if (!ring_mb_wait(&free_bar[lw], free_par)) {
          failed = true;
          break;
        }
        free_par ^= 1u;
      }
      if (k >= 1) ring_send<R>(dst_a, ga, va);
      if (k < K) ring_send<R>(dst_b, gb, vb);
      __syncwarp();  // every lane's stores precede lane 0's release
      if (lane == 0) {
        if (k >= 1) ring_mb_arrive_remote(full_a);
        if (k < K) ring_mb_arrive_remote(full_b);
      }
      if (k == K) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          ga[j] = gb[j];
          va[j] = vb[j];
        }
      }
      if (!ring_mb_wait(&full_bar[lw], full_par)) {
        failed = true;
        break;
      }
      full_par ^= 1u;
      if (k >= 1 && k < K) ring_recv<R>(my_a, ga, va);
      ring_recv<R>(my_b, gb, vb);
      __syncwarp();  // every lane's inbox reads precede the credits
      if (lane == 0) {
        ring_mb_arrive_remote(free_b);
        if (k >= 1 && k < K) ring_mb_arrive_remote(free_a);
      }
    }
    ++gr;
    lr = lr + 1 == m ? 0 : lr + 1;
    ring_players(k, lr, m, pa, pb);
  }
  if (failed && lane == 0) atomicOr(err, 1);
  // no CTA leaves while another may still write to its shared memory
  ring_arrive();
  ring_wait();
}

// V = identity for every problem
__global__ void svd_init_v_kernel(const SvdTask* __restrict__ tasks) {
  const SvdTask t = tasks[blockIdx.x];
  if (!t.v) return;
  for (int e = threadIdx.x; e < t.q * t.q; e += blockDim.x) t.v[e] = {(e % t.q) == (e / t.q) ? 1.0 : 0.0, 0.0};
}

// singular values = column norms, sorted descending with perm (NaN last)
__global__ void __launch_bounds__(256) svd_finish_kernel(const SvdTask* __restrict__ tasks) {
  const SvdTask t = tasks[blockIdx.x];
  const int p = t.p, q = t.q;
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int j = warp; j < q; j += nwarp) {
    double a, b;
    cplx c;
    col_pair(t.g, p, j, j, a, b, c);
    if ((threadIdx.x & 31) == 0) t.sv[j] = sqrt(a);
  }
  __syncthreads();
  // rank on integer keys (bit patterns of the non-negative values; NaN last)
  extern __shared__ unsigned long long sb[];
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    double v = t.sv[j];
    sb[j] = (v == v && v >= 0.0) ? (unsigned long long)__double_as_longlong(v) + 1ull : 0ull;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    const unsigned long long kj = sb[j];
    int rank = 0;
    for (int i = 0; i < q; ++i) {
      const unsigned long long ki = sb[i];
      rank += (ki > kj) || (ki == kj && i < j);
    }
    t.perm[rank] = j;
    t.sv[rank] = kj ? __longlong_as_double((long long)(kj - 1ull)) : 0.0;
  }
}

__global__ void svd32_init_v_kernel(const Svd32Task* __restrict__ tasks) {
  const Svd32Task t = tasks[blockIdx.x];
  for (int e = threadIdx.x; e < t.q * t.q; e += blockDim.x)
    t.v[e] = make_float2((e % t.q) == (e / t.q) ? 1.0f : 0.0f, 0.0f);
}

// Pairs (task, k) sorted by task size descending, and per round the number of
// leading pairs whose task still has that round.
template <class Task>
static void pair_schedule(const std::vector<Task>& h_tasks, const std::vector<char>& skip, std::vector<int2>& work,
                          std::vector<int>& active) {
  std::vector<int> ord(h_tasks.size());
  for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) {
    return h_tasks[x].q != h_tasks[y].q ? h_tasks[x].q > h_tasks[y].q : x < y;
  });
  work.clear();
  std::vector<int> nround;  // rounds of the task of each work item
  for (int i : ord) {
    const int q = h_tasks[i].q;
    if (q < 2 || skip[i]) continue;
    const int n = q + (q & 1);
    for (int k = 0; k < n / 2; ++k) {
      work.push_back(make_int2(i, k));
      nround.push_back(n - 1);
    }
  }
  const int max_rounds = nround.empty() ? 0 : nround[0];
  active.assign(max_rounds, 0);
  for (int r = 0; r < max_rounds; ++r) {
    int c = 0;
    while (c < (int)nround.size() && nround[c] > r) ++c;
    active[r] = c;
  }
}

// registers per lane for the longest column: 32 R >= pmax (R = 0: streamed from memory)
static int rows_per_lane(int pmax) {
  for (int R = 1; R <= 16; R *= 2)
    if (32 * R >= pmax) return R;
  return 0;
}

// Cooperative grids launched from different streams never overlap on the device.
// A grid-wide barrier needs every CTA of its grid resident at once; two such grids
// sharing the SMs (two chains evolved on two streams) could each hold SMs that the
// other's missing CTAs wait for.  Every cooperative launch therefore first waits
// for the previous cooperative launch of any other stream on the same device (one
// event per device, re-recorded under a lock).  Kernels that are not cooperative
// keep overlapping freely: they never wait on other CTAs, so a cooperative grid
// that has to wait for SMs they hold gets them when they finish.
struct CoopOrder {
  std::mutex m;
  cudaEvent_t ev = nullptr;
  cudaStream_t last = nullptr;
  bool any = false;
};
static CoopOrder g_coop_order[64];

template <class Launch>
static int coop_ordered(cudaStream_t s, Launch launch) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (dev < 0 || dev >= 64 || cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return launch();  // a captured graph replays in the order it was captured
  CoopOrder& o = g_coop_order[dev];
  std::lock_guard<std::mutex> lk(o.m);
  if (!o.ev && cudaEventCreateWithFlags(&o.ev, cudaEventDisableTiming) != cudaSuccess) return -1;
  if (o.any && o.last != s && cudaStreamWaitEvent(s, o.ev, 0) != cudaSuccess) return -1;
  const int rc = launch();
  if (rc != 0) return rc;
  if (cudaEventRecord(o.ev, s) != cudaSuccess) return -1;
  o.last = s;
  o.any = true;
  return 0;
}

// CTAs per SM of the cooperative Jacobi grid: 4, or TDVP_JACOBI_CTAS_PER_SM (1..8,
// read at every launch; the occupancy limit still applies).  Only the pairs'
// distribution over warps changes; every pair's arithmetic and order do not.
static int coop_ctas_per_sm() {
  const char* e = std::getenv("TDVP_JACOBI_CTAS_PER_SM");
  if (!e || !*e) return 4;
  const int v = std::atoi(e);
  return v < 1 ? 1 : (v > 8 ? 8 : v);
}

template <class Task, class S, class C2, int R>
static int coop_launch(const Task* d_tasks, int nt, const int2* d_work, const int* d_active, int nrounds,
                       int max_sweeps, S tol, S tol_flag, S abs_flag, int* flags, int* out, cudaStream_t s,
                       int* task_sweeps) {
  auto kern = jacobi_coop_kernel<Task, S, C2, R>;
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, JT, 0);
  if (per < 1 || nsm < 1) return -1;
  const int grid = nsm * std::min(per, coop_ctas_per_sm());
  void* args[] = {(void*)&d_tasks,    (void*)&nt,  (void*)&d_work,   (void*)&d_active, (void*)&nrounds,
                  (void*)&max_sweeps, (void*)&tol, (void*)&tol_flag, (void*)&abs_flag, (void*)&flags,
                  (void*)&out,        (void*)&task_sweeps};
  return coop_ordered(s, [&] {
    note_launch();
    return cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(JT), args, 0, s) == cudaSuccess ? 0 : -1;
  });
}

// Largest working copy (bytes) that may run CTA-resident: RJ_SMEM, or the value of
// the environment variable TDVP_JACOBI_RESIDENT_BYTES (read at every call, clamped to
// [0, RJ_SMEM]; 0 sends every sector to the cooperative kernel).  Both paths give
// the same result; the variable only selects where a sector runs.
static long long resident_limit() {
  const char* e = std::getenv("TDVP_JACOBI_RESIDENT_BYTES");
  if (!e || !*e) return RJ_SMEM;
  const long long v = std::atoll(e);
  return v < 0 ? 0 : (v > RJ_SMEM ? RJ_SMEM : v);
}

// Whether the cluster form may run: only when TDVP_JACOBI_CLUSTER=1 (read at every
// call).  It is off by default because it is slower on the workloads measured: a
// sector's pairs then run on the C SMs of its cluster, and clusters of 200 KiB CTAs
// run in waves, while the cooperative form spreads every round's pairs over all SMs
// (the FP64 stage suffers most, the B300's FP64 rate per SM being low).
// TDVP_JACOBI_CLUSTER=32 enables it for the FP32 preconditioner only (the FP64 stage
// keeps the cooperative grid, whose rounds use every SM's FP64 units).
static bool cluster_enabled(bool fp32) {
  const char* e = std::getenv("TDVP_JACOBI_CLUSTER");
  if (!e) return false;
  if (e[0] == '1') return true;
  return fp32 && e[0] == '3' && e[1] == '2';
}

// Smallest cluster size (2, 4 or 8 CTAs) whose slices hold every sector of the call
// (G, and V when accumulated), with the largest slice in *smem; 0 when a sector does
// not fit in 8 CTAs.
template <class Task, class C2>
static int cluster_size_for(const std::vector<Task>& h_tasks, size_t* smem) {
  for (int C = 2; C <= 8; C *= 2) {
    size_t need = 0;
    bool ok = true;
    for (const Task& t : h_tasks) {
      if (t.q < 2) continue;
      const size_t slots = (size_t)(t.q + C - 1) / C;
      const size_t b = slots * ((size_t)t.p + (t.v ? (size_t)t.q : 0)) * sizeof(C2);
      if (b > (size_t)CJ_SMEM) {
        ok = false;
        break;
      }
      need = std::max(need, b);
    }
    if (ok) {
      *smem = need;
      return C;
    }
  }
  return 0;
}

// Whether the ring form may run the FP32 preconditioner: yes unless
// TDVP_JACOBI_RING=0 (read at every call).
static bool ring_enabled() {
  const char* e = std::getenv("TDVP_JACOBI_RING");
  return !(e && e[0] == '0');
}

// Placement of the ring form: sectors (q >= 2) by size, largest first, each on the
// first cluster with room for its h = ceil(q/2) warps (first fit), at consecutive
// warp slots.  Clusters have the fewest CTAs that hold the largest sector (at least
// 2, at most 16; above 8 the size is non-portable): small clusters keep the barrier
// cheap and let more clusters be resident at once.  Returns the rows per lane R
// (p <= 32 R) and sets *csize, or returns 0 when some sector does not fit (more than
// RING_RMAX rows per lane, or more warps than a cluster of 16 holds).
static int ring_plan(const std::vector<Svd32Task>& h, std::vector<RingWarp>& slots, std::vector<int>& nsec,
                     int* csize) {
  std::vector<std::pair<int, int>> order;  // (h, task)
  int pmax = 0, hmax = 0;
  long long hsum = 0;
  for (int e = 0; e < (int)h.size(); ++e) {
    if (h[e].q < 2) continue;
    const int hh = (h[e].q + (h[e].q & 1)) / 2;
    if (h[e].p > 32 * RING_RMAX || hh > RING_CMAX * RING_NW) return 0;
    order.push_back({hh, e});
    pmax = std::max(pmax, h[e].p);
    hmax = std::max(hmax, hh);
    hsum += hh;
  }
  if (order.empty()) return 0;
  const int C = std::max(2, (hmax + RING_NW - 1) / RING_NW);
  const int cap = C * RING_NW;
  std::stable_sort(order.begin(), order.end(), [](const std::pair<int, int>& a, const std::pair<int, int>& b) {
    return a.first > b.first;
  });
  std::vector<int> used;
  slots.clear();
  nsec.clear();
  for (auto& o : order) {
    int c = 0;
    while (c < (int)used.size() && used[c] + o.first > cap) ++c;
    if (c == (int)used.size()) {
      used.push_back(0);
      nsec.push_back(0);
      slots.resize(used.size() * (size_t)cap, RingWarp{-1, 0, 0, 0});
    }
    const int w0 = used[c];
    for (int k = 0; k < o.first; ++k) slots[(size_t)c * cap + w0 + k] = RingWarp{o.second, k, w0, o.first};
    used[c] += o.first;
    nsec[c] += 1;
  }
  *csize = C;
  if (std::getenv("TDVP_RING_DEBUG")) {
    std::fprintf(stderr, "ring: %zu sectors, sum h %lld, h max %d, p max %d, clusters %zu of %d CTAs\n",
                 order.size(), hsum, hmax, pmax, used.size(), C);
    for (auto& o : order) std::fprintf(stderr, "  sector p %d q %d\n", h[o.second].p, h[o.second].q);
  }
  return std::max(2, (pmax + 31) / 32);
}

// check_only: 0 when one cluster of this shape fits on the device, else 1; otherwise
// launch (0 on success, -1 on a launch error)
template <int R>
static int ring_launch_r(bool check_only, int C, const Svd32Task* d_tasks, const RingWarp* d_slots, int ncl,
                         int max_sweeps, float tol, float tol_flag, float abs_flag, int* task_sweeps, int* err,
                         cudaStream_t s) {
  auto kern = jacobi_ring_kernel<R>;
  const size_t smem = (size_t)RING_NW * 2 * 64 * R * sizeof(float2);
  static const bool attr = [smem] {  // once per instantiation, thread-safe (function-local static)
    cudaFuncSetAttribute(jacobi_ring_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(jacobi_ring_kernel<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return true;
  }();
  (void)attr;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  cfg.gridDim = dim3((unsigned)(std::max(ncl, 1) * C));
  cfg.blockDim = dim3(RING_NW * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (check_only) {
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, (void*)kern, &cfg) != cudaSuccess || active < 1) {
      cudaGetLastError();
      return 1;
    }
    if (std::getenv("TDVP_RING_DEBUG")) std::fprintf(stderr, "ring: %d clusters of %d CTAs resident at once\n", active, C);
    return 0;
  }
  note_launch();
  return cudaLaunchKernelEx(&cfg, kern, d_tasks, d_slots, max_sweeps, tol, tol_flag, abs_flag, task_sweeps,
                            err) == cudaSuccess
             ? 0
             : -1;
}

static int ring_launch(int R, bool check_only, int C, const Svd32Task* d_tasks, const RingWarp* d_slots, int ncl,
                       int max_sweeps, float tol, float tol_flag, float abs_flag, int* task_sweeps, int* err,
                       cudaStream_t s) {
#define TDVP_RING_CASE(RR)                                                                                     \
  case RR:                                                                                                     \
    return ring_launch_r<RR>(check_only, C, d_tasks, d_slots, ncl, max_sweeps, tol, tol_flag, abs_flag, \
                             task_sweeps, err, s);
  switch (R) {
    TDVP_RING_CASE(2)
    TDVP_RING_CASE(3)
    TDVP_RING_CASE(4)
    TDVP_RING_CASE(5)
    TDVP_RING_CASE(6)
    TDVP_RING_CASE(7)
    TDVP_RING_CASE(8)
    TDVP_RING_CASE(9)
    TDVP_RING_CASE(10)
    default: return 1;
  }
#undef TDVP_RING_CASE
}

template <class Task, class S, class C2>
static int coop_run(const Task* d_tasks, const std::vector<Task>& h_tasks, int max_sweeps, S tol, S tol_flag,
                    S abs_flag, int* nonconv, bool with_v, JacobiProfile* prof, cudaStream_t s,
                    const ScratchFn& scratch) {
  const int nt = (int)h_tasks.size();
  int pmax = 1;
  // All sectors run CTA-resident when every one of them fits: q <= RJ_QMAX columns
  // (each round is one parallel step of the CTA's warps) and a working copy within the
  // shared-memory limit.  Otherwise all of them share the cooperative grid: a resident
  // launch beside it would add its own rounds to the critical path, and a large sector
  // inside one SM runs its pairs one after another on one SM's FP64 units.
  // Failing that, all sectors run in thread-block clusters when every one fits in the
  // distributed shared memory of 8 CTAs; otherwise on the cooperative grid.
  const long long limit = resident_limit();
  bool all_fit = true;
  for (const Task& t : h_tasks)
    if (t.q >= 2 && (t.q > RJ_QMAX || (long long)t.p * t.q * (long long)sizeof(C2) > limit)) all_fit = false;
  size_t cl_smem = 0;
  int cl_size = 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute cl_attr[1];
  auto cl_kern = jacobi_cluster_kernel<Task, S, C2>;
  if (!all_fit && cluster_enabled(sizeof(S) == 4)) {
    cl_size = cluster_size_for<Task, C2>(h_tasks, &cl_smem);
    if (cl_size > 0) {
      static const bool attr = [] {  // once per process, thread-safe (function-local static)
        cudaFuncSetAttribute(jacobi_cluster_kernel<Task, S, C2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             CJ_SMEM);
        return true;
      }();
      (void)attr;
      int nsec = 0;
      for (const Task& t : h_tasks) nsec += t.q >= 2 ? 1 : 0;
      cfg.gridDim = dim3((unsigned)(nsec * cl_size));
      cfg.blockDim = dim3(CJT);
      cfg.dynamicSmemBytes = cl_smem;
      cfg.stream = s;
      cl_attr[0].id = cudaLaunchAttributeClusterDimension;
      cl_attr[0].val.clusterDim.x = (unsigned)cl_size;
      cl_attr[0].val.clusterDim.y = 1;
      cl_attr[0].val.clusterDim.z = 1;
      cfg.attrs = cl_attr;
      cfg.numAttrs = 1;
      int ncl = 0;  // clusters of this shape that fit on the device at once
      if (cudaOccupancyMaxActiveClusters(&ncl, (void*)cl_kern, &cfg) != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        cl_size = 0;
      }
    }
  }
  // the ring form (FP32 preconditioner): when enabled and every sector fits a ring
  int ring_r = 0, ring_c = 0;
  std::vector<RingWarp> ring_slots;
  std::vector<int> ring_nsec;
  if constexpr (std::is_same<Task, Svd32Task>::value) {
    if (!all_fit && cl_size == 0 && ring_enabled()) ring_r = ring_plan(h_tasks, ring_slots, ring_nsec, &ring_c);
    if (ring_r > 0 && ring_launch(ring_r, true, ring_c, nullptr, nullptr, (int)ring_nsec.size(), 0, 0.f, 0.f, 0.f,
                                  nullptr, nullptr, s) != 0) {
      ring_r = 0;
      ring_slots.clear();
      ring_nsec.clear();
    }
  }
  const bool own_launch = all_fit || cl_size > 0 || ring_r > 0;  // resident, cluster or ring form
  std::vector<char> resident(nt, 0);
  std::vector<int> rid;
  for (int e = 0; e < nt; ++e) {
    const Task& t = h_tasks[e];
    if (t.q < 2) continue;
    if (own_launch) {
      resident[e] = 1;
      rid.push_back(e);
    } else {
      pmax = max(pmax, t.p);
    }
  }
  if (cl_size > 0) {  // largest sectors first, so that their clusters start first
    std::stable_sort(rid.begin(), rid.end(), [&](int a, int b) {
      return (long long)h_tasks[a].p * h_tasks[a].q > (long long)h_tasks[b].p * h_tasks[b].q;
    });
  }
  std::vector<int2> work;
  std::vector<int> active;
  pair_schedule(h_tasks, resident, work, active);
  if (work.empty() && rid.empty()) return 1;
  // one device region for the work lists and the flags: [work | active | rid | flags],
  // each part 16-byte aligned; flags: two sweep buffers [2 nt], out [2] (cooperative
  // sweeps, non-convergence), per-task active sweeps of the cooperative kernel [nt],
  // non-convergence of the resident sectors [1], sweeps of the resident sectors [nt]
  auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const size_t b_work = up16(work.size() * sizeof(int2)), b_act = up16(active.size() * sizeof(int)),
               b_rid = up16(rid.size() * sizeof(int)), b_flags = up16((4 * (size_t)nt + 4) * sizeof(int));
  const size_t b_rslots = up16(ring_slots.size() * sizeof(RingWarp)), b_rnsec = up16(ring_nsec.size() * sizeof(int));
  const size_t b_lists = b_work + b_act + b_rid + b_rslots + b_rnsec;
  char* region = nullptr;
  bool owned = false;
  if (scratch) {
    region = static_cast<char*>(scratch(b_lists + b_flags));
  } else if (cudaMallocAsync((void**)&region, b_lists + b_flags, s) == cudaSuccess) {
    owned = true;
  } else {
    region = nullptr;
  }
  if (!region) {
    cudaGetLastError();
    return JACOBI_ENOMEM;
  }
  std::vector<char> host(b_lists, 0);
  if (!work.empty()) {
    std::memcpy(host.data(), work.data(), work.size() * sizeof(int2));
    std::memcpy(host.data() + b_work, active.data(), active.size() * sizeof(int));
  }
  if (!rid.empty()) std::memcpy(host.data() + b_work + b_act, rid.data(), rid.size() * sizeof(int));
  const size_t o_rslots = b_work + b_act + b_rid, o_rnsec = o_rslots + b_rslots;
  if (!ring_slots.empty()) {
    std::memcpy(host.data() + o_rslots, ring_slots.data(), ring_slots.size() * sizeof(RingWarp));
    std::memcpy(host.data() + o_rnsec, ring_nsec.data(), ring_nsec.size() * sizeof(int));
  }
  if (b_lists) cudaMemcpyAsync(region, host.data(), b_lists, cudaMemcpyHostToDevice, s);
  int2* d_work = work.empty() ? nullptr : reinterpret_cast<int2*>(region);
  int* d_active = work.empty() ? nullptr : reinterpret_cast<int*>(region + b_work);
  int* d_rid = rid.empty() ? nullptr : reinterpret_cast<int*>(region + b_work + b_act);
  int* flags = reinterpret_cast<int*>(region + b_lists);
  int* out = flags + 2 * nt;
  int* tsw = out + 2;
  int* rnc = tsw + nt;
  int* rsw = rnc + 1;
  int* ring_err = rsw + nt;
  cudaMemsetAsync(out, 0, (2 * nt + 4) * sizeof(int), s);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (prof) {
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    cudaEventRecord(ev[0], s);
  }
  int rc = 0;
  if (!rid.empty() && ring_r > 0) {
    if constexpr (std::is_same<Task, Svd32Task>::value) {
      rc = ring_launch(ring_r, false, ring_c, d_tasks, reinterpret_cast<const RingWarp*>(region + o_rslots),
                       (int)ring_nsec.size(), max_sweeps, tol, tol_flag, abs_flag, rsw, ring_err, s) == 0
               ? 0
               : -1;
    }
  } else if (!rid.empty() && cl_size > 0) {
    note_launch();
    if (cudaLaunchKernelEx(&cfg, cl_kern, (const Task*)d_tasks, (const int*)d_rid, max_sweeps, tol, tol_flag, abs_flag,
                           rsw, rnc) != cudaSuccess)
      rc = -1;
  } else if (!rid.empty()) {
    static const bool attr = [] {  // once per process, thread-safe (function-local static)
      cudaFuncSetAttribute(jacobi_resident_kernel<Task, S, C2>, cudaFuncAttributeMaxDynamicSharedMemorySize, RJ_SMEM);
      return true;
    }();
    (void)attr;
    size_t sm = 0;
    for (int e : rid) sm = std::max(sm, (size_t)h_tasks[e].p * h_tasks[e].q * sizeof(C2));
    note_launch();
    jacobi_resident_kernel<Task, S, C2><<<(int)rid.size(), RJT, sm, s>>>(d_tasks, d_rid, max_sweeps, tol, tol_flag,
                                                                         abs_flag, rsw, rnc);
    if (cudaGetLastError() != cudaSuccess) rc = -1;
  }
  if (rc == 0 && !work.empty()) {
    const int nr = (int)active.size();
    auto go = [&](auto r_tag) {
      constexpr int R = decltype(r_tag)::value;
      return coop_launch<Task, S, C2, R>(d_tasks, nt, d_work, d_active, nr, max_sweeps, tol, tol_flag, abs_flag,
                                         flags, out, s, tsw);
    };
    switch (rows_per_lane(pmax)) {
      case 1: rc = go(std::integral_constant<int, 1>()); break;
      case 2: rc = go(std::integral_constant<int, 2>()); break;
      case 4: rc = go(std::integral_constant<int, 4>()); break;
      case 8: rc = go(std::integral_constant<int, 8>()); break;
      case 16: rc = go(std::integral_constant<int, 16>()); break;
      default: rc = go(std::integral_constant<int, 0>()); break;
    }
  }
  if (prof) cudaEventRecord(ev[1], s);
  std::vector<int> h(4 + 2 * nt, 0);
  int sweeps = -1, nc = 1;
  bool timed_out = false;
  if (rc == 0) {
    cudaMemcpyAsync(h.data(), out, (4 + 2 * nt) * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    timed_out = h[3 + 2 * nt] != 0;  // a ring's neighbour exchange gave up waiting
    auto task_sweeps = [&](int e) { return resident[e] ? h[3 + nt + e] : h[2 + e]; };
    sweeps = h[0];  // the cooperative launch's sweeps (0 when it did not run)
    for (int e : rid) sweeps = max(sweeps, task_sweeps(e));
    if (ring_r > 0 && std::getenv("TDVP_RING_DEBUG")) {
      for (int e : rid)
        std::fprintf(stderr, "ring sweeps: p %d q %d sweeps %d\n", h_tasks[e].p, h_tasks[e].q, task_sweeps(e));
    }
    nc = (h[1] | h[2 + nt]) ? 1 : 0;
    if (prof) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) prof->ms += ms;
      for (int e = 0; e < nt; ++e) {
        const double p = h_tasks[e].p, q = h_tasks[e].q;
        prof->flops += (double)task_sweeps(e) * 0.5 * q * (q - 1) * (48.0 * p + (with_v ? 32.0 * q : 0.0));
      }
      prof->launches += 1;
      if (!rid.empty() && cl_size == 0 && ring_r == 0) prof->resident += 1;
      if (!rid.empty() && cl_size > 0) prof->cluster += 1;
      if (!rid.empty() && ring_r > 0) prof->ring += 1;
    }
  }
  if (prof) {
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
  }
  if (owned) cudaFreeAsync(region, s);
  if (nonconv) *nonconv = nc;
  if (timed_out) return JACOBI_ETIMEOUT;
  return rc == 0 ? sweeps : -1;
}

// Jacobi driver: returns the number of sweeps run, or -1 when the cooperative launch
// failed (the CUDA error is left for the caller's check).  V is accumulated (from
// the identity) when the tasks carry v; without v only G is rotated.  Pairs rotate
// when |g_i^H g_j| > tol |g_i||g_j|.  A sweep in which no rotation had |g_i^H g_j|
// above both tol_flag |g_i||g_j| and abs_flag ends the iteration: with tol_flag =
// tol and abs_flag = 0 that is the usual "no rotation at all" test; tol_flag =
// sqrt(tol) relies on the quadratic convergence of cyclic Jacobi (off-diagonal
// delta before a sweep leaves O(delta^2) after it), and abs_flag > 0 ignores pairs
// whose coupling is negligible on the scale of the whole matrix (the split passes
// unit-norm theta, so abs_flag is a weight).  Non-convergence within max_sweeps
// sets *status to 1.
int run_jacobi_rounds(const SvdTask* d_tasks, const std::vector<SvdTask>& h_tasks, int max_sweeps, double tol,
                      int* status, cudaStream_t s, double tol_flag, double abs_flag, JacobiProfile* prof,
                      const ScratchFn& scratch) {
  const int nt = (int)h_tasks.size();
  if (nt == 0) return 0;
  if (!(tol_flag >= tol)) tol_flag = tol;
  int qmax = 1;
  for (auto& t : h_tasks) qmax = max(qmax, t.q);
  note_launch();
  svd_init_v_kernel<<<nt, 256, 0, s>>>(d_tasks);
  int nonconv = 0;
  const bool with_v = h_tasks[0].v != nullptr;
  const int sweeps =
      coop_run<SvdTask, double, cplx>(d_tasks, h_tasks, max_sweeps, tol, tol_flag, abs_flag, &nonconv, with_v, prof, s,
                                      scratch);
  if (sweeps == JACOBI_ENOMEM) return sweeps;
  if (sweeps > 0 && nonconv) {
    int one = 1;
    cudaMemcpyAsync(status, &one, sizeof(int), cudaMemcpyHostToDevice, s);  // reported by the caller's check
    cudaStreamSynchronize(s);
  }
  size_t fs = (size_t)qmax * sizeof(double);
  if (fs > 48 * 1024) cudaFuncSetAttribute(svd_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs);
  note_launch();
  svd_finish_kernel<<<nt, 256, fs, s>>>(d_tasks);
  return sweeps;
}

// ---------------------------------------------------------------------------
// K6 (FP32 preconditioner): the same Jacobi on complex64 copies of G with the right
// rotations accumulated in a complex64 V.  Used by the split-precision modes: V is
// widened to FP64, G = A V is formed again in FP64 and a short FP64 Jacobi finishes
// the SVD, so every singular value the truncation sees is an FP64 one (the FP32
// columns themselves are discarded).  It need not converge: it stops after
// max_sweeps without an error.
// ---------------------------------------------------------------------------

int run_jacobi_rounds32(const Svd32Task* d_tasks, const std::vector<Svd32Task>& h_tasks, int max_sweeps, float tol,
                        float abs_flag, cudaStream_t s, JacobiProfile* prof, const ScratchFn& scratch) {
  const int nt = (int)h_tasks.size();
  if (nt == 0) return 0;
  note_launch();
  svd32_init_v_kernel<<<nt, 256, 0, s>>>(d_tasks);
  return coop_run<Svd32Task, float, float2>(d_tasks, h_tasks, max_sweeps, tol, 0.0f, abs_flag, nullptr, true, prof,
                                            s, scratch);
}


// precision conversions of whole buffers
__global__ void narrow_kernel(const cplx* __restrict__ src, float2* __restrict__ dst, long long n) {
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256)
    dst[e] = make_float2((float)src[e].x, (float)src[e].y);
}
__global__ void widen_kernel(const float2* __restrict__ src, cplx* __restrict__ dst, long long n) {
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256)
    dst[e] = {(double)src[e].x, (double)src[e].y};
}

// X (rows x k, row-major) column kk = column perm[kk] of G (rows x ., column-major)
// divided by sv[kk] (pow2 = 0) or sv[kk]^2 (pow2 = 1)
__global__ void basis64_kernel(const BasisTask* __restrict__ tasks) {
  const BasisTask t = tasks[blockIdx.y];
  const long long n = (long long)t.rows * t.k;
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
    int i = (int)(e / t.k), kk = (int)(e - (long long)i * t.k);
    cplx g = t.g[i + (long long)t.perm[kk] * t.rows];
    double s = t.sv[kk];
    double f = s > 0 ? (t.pow2 ? 1.0 / (s * s) : 1.0 / s) : 0.0;
    t.x[e] = {f * g.x, f * g.y};
  }
}

// F = 1.5 I - 0.5 G for the Newton-Schulz step X <- X F (k x k, row-major)
__global__ void ns_coeff_kernel(const NsTask* __restrict__ tasks) {
  const NsTask t = tasks[blockIdx.y];
  const int n = t.k * t.k;
  for (int e = blockIdx.x * 256 + threadIdx.x; e < n; e += gridDim.x * 256) {
    int i = e / t.k, j = e - i * t.k;
    cplx g = t.g[e];
    t.g[e] = {(i == j ? 1.5 : 0.0) - 0.5 * g.x, -0.5 * g.y};
  }
}

// E = (I - K) / 2 for the Newton-Schulz correction X <- X + X E (k x k, row-major),
// from K's upper triangle only (K Hermitian: K[i][j] = conj(K[j][i]) below it), into e
__global__ void ns_corr_kernel(const NsTask* __restrict__ tasks, const cplx* const* __restrict__ outs) {
  const NsTask t = tasks[blockIdx.y];
  cplx* const e = const_cast<cplx*>(outs[blockIdx.y]);
  const int n = t.k * t.k;
  for (int x = blockIdx.x * 256 + threadIdx.x; x < n; x += gridDim.x * 256) {
    const int i = x / t.k, j = x - i * t.k;
    cplx g = i <= j ? t.g[x] : t.g[(long long)j * t.k + i];
    if (i > j) g.y = -g.y;
    e[x] = {(i == j ? 0.5 : 0.0) - 0.5 * g.x, -0.5 * g.y};
  }
}

static int conv_grid(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1184 ? (b < 1 ? 1 : b) : 1184);
}
void launch_narrow(const cplx* src, float2* dst, long long n, cudaStream_t s) {
  if (n > 0) {
    note_launch();
    narrow_kernel<<<conv_grid(n), 256, 0, s>>>(src, dst, n);
  }
}
void launch_widen(const float2* src, cplx* dst, long long n, cudaStream_t s) {
  if (n > 0) {
    note_launch();
    widen_kernel<<<conv_grid(n), 256, 0, s>>>(src, dst, n);
  }
}
void launch_basis64(const BasisTask* tasks, int n, cudaStream_t s) {
  if (n > 0) {
    note_launch();
    basis64_kernel<<<dim3(32, n), 256, 0, s>>>(tasks);
  }
}
void launch_ns_corr(const NsTask* tasks, const cplx* const* outs, int n, cudaStream_t s) {
  if (n > 0) {
    note_launch();
    ns_corr_kernel<<<dim3(8, n), 256, 0, s>>>(tasks, outs);
  }
}
void launch_ns_coeff(const NsTask* tasks, int n, cudaStream_t s) {
  if (n > 0) {
    note_launch();
    ns_coeff_kernel<<<dim3(8, n), 256, 0, s>>>(tasks);
  }
}

// ---------------------------------------------------------------------------
// Gram finish of the mixed split: one simultaneous-rotation step on a column set G
// whose Gram matrix K = G^H G is nearly diagonal (relative off-diagonals delta of
// the FP32 level after the FP32 Jacobi).  Every pair (a < b) gets the complex Jacobi
// rotation of warp_pair_cols computed from K_aa, K_bb and K_ab, and all of them act at
// once: G <- G Z with Z_ab = sn e, Z_ba = -sn conj(e) (e = K_ab / |K_ab|) and
// Z_ii = sqrt(1 - sum_k |Z_ki|^2).  To first order in delta this zeroes every K_ab
// (the rotation angle tends to K_ab / (K_bb - K_aa)), so one step takes delta to
// O(delta^2), the quadratic convergence of Jacobi methods, as two GEMMs instead of a
// sweep of dependent rounds.  Simultaneous rotations interfere when an angle is large
// (near-degenerate columns): pairs with |tan| > tmax are not rotated, and when such a
// pair carries weight (|K_ab| > abs_flag) flags[1] is set so that the caller finishes
// with the sequential Jacobi instead; a column whose rotations sum to more than a
// quarter of its norm does the same.  flags[0] is set when some pair is above
// tol_flag |g_a||g_b| and abs_flag (the stopping rule of the FP64 Jacobi stage);
// flags[2] receives the largest such relative coupling (float bits, atomicMax).
// Only the upper triangle of C is read (K_ab = conj(C[a][b]) for a < b), so the
// Gram GEMM computes only the tiles on and above the diagonal.  The kernel writes
// X^T = Z^T - I (row-major, xt[i][k] = Z[k][i] - [i == k]); the caller forms
// G + G X.  One warp per row i of X^T (the coefficients of new column i).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) gram_rot_kernel(const GramTask* __restrict__ tasks, double tol, double tol_flag,
                                                       double abs_flag, double tmax, int* __restrict__ flags) {
  const GramTask t = tasks[blockIdx.y];
  const int q = t.q;
  const int i0 = blockIdx.x * 8;  // this CTA's eight rows of X^T (new columns i0 .. i0 + 7)
  if (i0 >= q) return;            // uniform over the CTA
  // staged in shared memory: the diagonal of C, and its columns i0 .. i0 + 7 (row k,
  // column i0 + j at colblk[k * 9 + j]; 9: fewer bank conflicts), which hold K_ki = C[k][i]
  // for k < i; the rest of a row comes from C's row i, read contiguously
  extern __shared__ double gram_smem[];
  double* diag = gram_smem;
  cplx* colblk = reinterpret_cast<cplx*>(gram_smem + ((q + 1) & ~1));
  for (int e = threadIdx.x; e < q; e += blockDim.x) diag[e] = t.c[(long long)e * q + e].x;
  for (int e = threadIdx.x; e < q * 8; e += blockDim.x) {
    const int k = e >> 3, j = e & 7;
    colblk[k * 9 + j] = i0 + j < q ? t.c[(long long)k * q + i0 + j] : cplx{0.0, 0.0};
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = i0 + w;
  bool conv = false, big = false;
  float worst = 0.0f;
  if (i < q) {
    const double si = diag[i];
    double sum = 0.0;
    for (int k = lane; k < q; k += 32) {
      if (k == i) continue;
      const bool lower = k < i;  // pair (a, b) = (k, i), else (i, k)
      const double sa = lower ? diag[k] : si, sb = lower ? si : diag[k];
      const cplx cab = lower ? colblk[k * 9 + w] : t.c[(long long)i * q + k];  // C[a][b]; K_ab = conj(C[a][b])
      // The rotation is computed in FP32 from FP64 inputs (the difference sb - sa is
      // taken in FP64): a relative error of 1e-7 in the angle leaves a coupling of 1e-7
      // of the one it removes, far below what the next step sees.  This part's FP64
      // divisions and square roots would cost ten times more.
      const float cx = (float)cab.x, cy = (float)-cab.y;
      const float ac = sqrtf(fmaf(cx, cx, cy * cy));
      const float nrm = sqrtf((float)sa) * sqrtf((float)sb);
      cplx z = {0.0, 0.0};
      if (ac != 0.0f && nrm > 0.0f && (double)ac > tol * (double)nrm) {  // (weights below FP32's range: not rotated)
        const bool sig = (double)ac > abs_flag;
        if (sig && (double)ac > tol_flag * (double)nrm) {
          conv = true;
          worst = fmaxf(worst, ac / nrm);
        }
        const float zeta = (float)(sb - sa) / (2.0f * ac);
        const float tt = (zeta >= 0 ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
        if (fabsf(tt) <= (float)tmax) {
          const float cs = 1.0f / sqrtf(fmaf(tt, tt, 1.0f)), sn = cs * tt;
          const float ex = cx / ac, ey = cy / ac;
          if (lower) z = {(double)(sn * ex), (double)(sn * ey)};  // Z[a][b] with a = k, b = i
          else z = {(double)(-sn * ex), (double)(sn * ey)};       // Z[b][a] with a = i, b = k
          sum = fma(z.x, z.x, fma(z.y, z.y, sum));
        } else if (sig) {
          big = true;
        }
      }
      t.zt[(long long)i * q + k] = z;
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) {
      if (sum > 0.25 && si > abs_flag) big = true;
      const double d = sum < 1.0 ? sum : 1.0;
      t.zt[(long long)i * q + i] = {-d / (1.0 + sqrt(1.0 - d)), 0.0};  // sqrt(1 - d) - 1 without cancellation
    }
  }
  if (__any_sync(0xffffffffu, conv) && lane == 0) atomicOr(&flags[0], 1);
  if (__any_sync(0xffffffffu, big) && lane == 0) atomicOr(&flags[1], 1);
  for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if (lane == 0 && worst > 0.0f) atomicMax(reinterpret_cast<unsigned*>(&flags[2]), __float_as_uint(worst));
}

// shared memory of gram_rot_kernel for column sets of at most qmax columns
static size_t gram_smem_bytes(int qmax) {
  return (size_t)((qmax + 1) & ~1) * sizeof(double) + (size_t)qmax * 9 * sizeof(cplx);
}

int gram_qmax() { return 1400; }  // 1400 columns: 208 KB of staging

void launch_gram_rot(const GramTask* tasks, int n, int qmax, double tol, double tol_flag, double abs_flag,
                     double tmax, int* flags, cudaStream_t s) {
  if (n <= 0 || qmax <= 0) return;
  static const bool attr = [] {  // once per process, thread-safe (function-local static)
    cudaFuncSetAttribute(gram_rot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)gram_smem_bytes(gram_qmax()));
    return true;
  }();
  (void)attr;
  note_launch();
  gram_rot_kernel<<<dim3((qmax + 7) / 8, n), 256, gram_smem_bytes(qmax), s>>>(tasks, tol, tol_flag, abs_flag, tmax,
                                                                              flags);
}

// g[e] += d[e] for e < n (the Gram step's G <- G + G X, in FP64)
__global__ void add_inplace_kernel(cplx* __restrict__ g, const cplx* __restrict__ d, long long n) {
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
    const cplx a = g[e], b = d[e];
    g[e] = {a.x + b.x, a.y + b.y};
  }
}

void launch_add_inplace(cplx* g, const cplx* d, long long n, cudaStream_t s) {
  if (n <= 0) return;
  note_launch();
  add_inplace_kernel<<<conv_grid(n), 256, 0, s>>>(g, d, n);
}

// singular values (column norms) and their descending order, as at the end of
// run_jacobi_rounds, for column sets orthogonalised by another route
void launch_svd_finish(const SvdTask* tasks, int n, int qmax, cudaStream_t s) {
  if (n <= 0) return;
  size_t fs = (size_t)std::max(qmax, 1) * sizeof(double);
  if (fs > 48 * 1024) cudaFuncSetAttribute(svd_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs);
  note_launch();
  svd_finish_kernel<<<n, 256, fs, s>>>(tasks);
}

void launch_jacobi_svd(const SvdTask* tasks, int ntasks, int max_q, int max_sweeps, double tol, int* status,
                       cudaStream_t s) {
  if (ntasks <= 0) return;
  size_t smem = (size_t)max_q * sizeof(double);
  if (smem > 48 * 1024) cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  note_launch();
  jacobi_svd_kernel<<<ntasks, SVD_THREADS, smem, s>>>(tasks, max_sweeps, tol, status);
}

// ---------------------------------------------------------------------------
// K7: truncation selection over all sectors of a bond (one CTA)
// ---------------------------------------------------------------------------

// Three launches (staging and ranking spread over CTAs, the rules in one CTA of
// TRUNC_THREADS threads).  Flat entry e of sector s is e = offs[s] + i.
// A sector's values r are reduced singular values normalised so that r^2 is the
// weight of the whole multiplet, (2S+1) s^2 with s the singular value of each of its
// 2S+1 states (Sec. S2.1, S2.4); mult = 2S+1 (1 without SU(2)).
// 1. stage value, sector and multiplet size of every entry (NaN ranks last, weight 0),
//    and the per-state weight lambda = r^2 / mult, the ranking key;
// 2. rank every entry (descending lambda, i.e. descending per-state singular value,
//    ties by flat index = sector, then in-sector index) against shared-memory tiles
//    of the keys, order[rank] = e;
// 3. block scans over the sorted list: suffix sums of the weights s^2 (the tail
//    rule) and prefix sums of the multiplet sizes (the chi cap);
// 4. K = min(shortest head whose dropped tail weighs <= eps * total, longest head with
//    at most chi_max states), both taken over the allowed heads (with degen > 0 a head
//    may not end between two entries whose per-state weights agree to within degen,
//    relative); if no allowed head fits under the cap the first allowed head is kept;
//    kept[s] = number of the first K sorted entries that belong to sector s.
constexpr int TRUNC_THREADS = 1024;
constexpr int TRUNC_TILE = 2048;

template <class T>
__device__ T block_exclusive_scan(T v, T* sh, T& total) {
  // sh: TRUNC_THREADS / 32 + 1 entries
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < TRUNC_THREADS / 32 ? sh[lane] : T(0);
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < TRUNC_THREADS / 32) sh[lane] = w;  // inclusive over warps
    if (lane == TRUNC_THREADS / 32 - 1) sh[TRUNC_THREADS / 32] = w;
  }
  __syncthreads();
  T before = (warp > 0 ? sh[warp - 1] : T(0)) + x - v;
  total = sh[TRUNC_THREADS / 32];
  __syncthreads();
  return before;
}

// ranking on integer keys: for non-negative doubles the IEEE bit pattern is monotone,
// the NaN sentinel -1 maps to 0 (the FP64 unit is far too slow on this part for n^2
// floating-point compares)
__device__ __forceinline__ unsigned long long trunc_key(double v) {
  return v >= 0.0 ? (unsigned long long)__double_as_longlong(v) + 1ull : 0ull;
}

// 1. staging: one warp per sector writes the values, per-state weights and owners
__global__ void __launch_bounds__(256) truncate_stage_kernel(const TruncSector* __restrict__ secs, int nsec,
                                                             const int* __restrict__ offs, int n,
                                                             int* __restrict__ owner, int* __restrict__ kept,
                                                             double* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  for (int sct = (blockIdx.x * 256 + threadIdx.x) >> 5; sct < nsec; sct += (gridDim.x * 256) >> 5) {
    const TruncSector t = secs[sct];
    for (int i = lane; i < t.r; i += 32) {
      double v = t.sv[i];
      const bool ok = v == v && v >= 0.0;
      owner[offs[sct] + i] = sct;
      vals[offs[sct] + i] = ok ? v : -1.0;
      vals[n + offs[sct] + i] = ok ? v * v / (double)t.mult : -1.0;
    }
    if (lane == 0) kept[sct] = 0;
  }
}

// 2. ranking: each CTA ranks TRUNC_RANK_PER_CTA entries (descending key, ties by flat
// index) against every key, streamed through shared-memory tiles; order[rank] = e
constexpr int TRUNC_RANK_THREADS = 256;
constexpr int TRUNC_RANK_PER = 4;
constexpr int TRUNC_RANK_PER_CTA = TRUNC_RANK_THREADS * TRUNC_RANK_PER;
__global__ void __launch_bounds__(TRUNC_RANK_THREADS) truncate_rank_kernel(int n, const double* __restrict__ vals,
                                                                           int* __restrict__ order) {
  __shared__ unsigned long long tile[TRUNC_TILE];
  const int tid = threadIdx.x, e0 = blockIdx.x * TRUNC_RANK_PER_CTA;
  unsigned long long mine[TRUNC_RANK_PER];
  int rank[TRUNC_RANK_PER];
#pragma unroll
  for (int j = 0; j < TRUNC_RANK_PER; ++j) {
    const int e = e0 + j * TRUNC_RANK_THREADS + tid;
    mine[j] = e < n ? trunc_key(vals[n + e]) : 0ull;
    rank[j] = 0;
  }
  for (int f0 = 0; f0 < n; f0 += TRUNC_TILE) {
    const int m = min(TRUNC_TILE, n - f0);
    __syncthreads();
    for (int f = tid; f < m; f += TRUNC_RANK_THREADS) tile[f] = trunc_key(vals[n + f0 + f]);
    __syncthreads();
    for (int f = 0; f < m; ++f) {
      const unsigned long long vf = tile[f];
      const int gf = f0 + f;
#pragma unroll
      for (int j = 0; j < TRUNC_RANK_PER; ++j) {
        const int e = e0 + j * TRUNC_RANK_THREADS + tid;
        rank[j] += (vf > mine[j]) || (vf == mine[j] && gf < e);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < TRUNC_RANK_PER; ++j) {
    const int e = e0 + j * TRUNC_RANK_THREADS + tid;
    if (e < n) order[rank[j]] = e;
  }
}

// 3. the rules over the ranked list (one CTA)
__global__ void __launch_bounds__(TRUNC_THREADS) truncate_kernel(const TruncSector* __restrict__ secs, int nsec,
                                                                 const int* __restrict__ offs, int n, double eps,
                                                                 long long chi_max, double degen,
                                                                 int* __restrict__ owner,
                                                                 int* __restrict__ order, int* __restrict__ kept,
                                                                 double* __restrict__ stats,
                                                                 double* __restrict__ vals) {
  const int tid = threadIdx.x;
  (void)nsec;
  (void)offs;
  // sorted entries in contiguous runs per thread: r in [r0, r1)
  const int per = (n + TRUNC_THREADS - 1) / TRUNC_THREADS;
  const int r0 = min(n, tid * per), r1 = min(n, r0 + per);
  double wloc = 0.0;
  long long mloc = 0;
  for (int r = r0; r < r1; ++r) {
    double v = vals[order[r]];
    wloc += v > 0.0 ? v * v : 0.0;
    mloc += secs[owner[order[r]]].mult;
  }
  __shared__ double shd[TRUNC_THREADS / 32 + 1];
  __shared__ long long shl[TRUNC_THREADS / 32 + 1];
  double total;
  long long mtot;
  const double wbefore = block_exclusive_scan(wloc, shd, total);
  const long long mbefore = block_exclusive_scan(mloc, shl, mtot);
  (void)mtot;
  (void)wbefore;
  // weight of all runs after this thread's run, summed as a scan in reverse thread
  // order (a sum of positive terms, not total minus a prefix, so small tails keep
  // their relative accuracy)
  __shared__ double shw[TRUNC_THREADS];
  shw[tid] = wloc;
  __syncthreads();
  double wrev_total;
  const double wafter_mirror = block_exclusive_scan(shw[TRUNC_THREADS - 1 - tid], shd, wrev_total);
  __syncthreads();
  shw[TRUNC_THREADS - 1 - tid] = wafter_mirror;
  __syncthreads();
  const double wafter = shw[tid];
  // a head of K ranked entries may end there unless the entries K-1 and K are
  // degenerate: per-state weights equal to within the relative tolerance degen
  auto cut_ok = [&](int K) -> bool {
    if (K >= n || degen <= 0.0) return true;
    const double a = vals[n + order[K - 1]], b = vals[n + order[K]];
    return !(a - b <= degen * a);
  };
  __shared__ int keep_eps, keep_chi, first_ok;
  if (tid == 0) {
    keep_eps = n;
    keep_chi = 0;
    first_ok = n;
  }
  __syncthreads();
  // tail rule: the smallest allowed head r >= 1 whose dropped tail sum_{r' >= r} w is
  // <= eps * total
  {
    // suffix within the run accumulated from the run's end, plus everything after the run
    double run_tail = 0.0;
    int best = n;
    for (int r = r1 - 1; r >= r0; --r) {
      double v = vals[order[r]];
      run_tail += v > 0.0 ? v * v : 0.0;
      double suf = wafter + run_tail;  // sum over r' >= r
      if (r >= 1 && suf <= eps * total && cut_ok(r)) best = r;
    }
    if (best < n) atomicMin(&keep_eps, best);
  }
  // chi cap: the largest allowed head K with sum_{r < K} mult <= chi_max; failing
  // that, the first allowed head (at least one multiplet is kept)
  {
    long long pre = mbefore;
    int best = 0, first = n;
    for (int r = r0; r < r1; ++r) {
      pre += secs[owner[order[r]]].mult;
      const bool ok = cut_ok(r + 1);
      if (ok && r + 1 < first) first = r + 1;
      if (pre <= chi_max && ok) best = r + 1;
    }
    if (best > 0) atomicMax(&keep_chi, best);
    if (first < n) atomicMin(&first_ok, first);
  }
  __syncthreads();
  if (tid == 0 && keep_chi == 0) keep_chi = first_ok;
  __syncthreads();
  int K = keep_eps < keep_chi ? keep_eps : keep_chi;
  if (K < 1) K = 1;
  double kwl = 0.0;
  long long kcl = 0;
  for (int r = r0; r < r1 && r < K; ++r) {
    const int e = order[r];
    const int sct = owner[e];
    double v = vals[e];
    kwl += v > 0.0 ? v * v : 0.0;
    kcl += secs[sct].mult;
    atomicAdd(&kept[sct], 1);
  }
  double kw;
  long long kchi;
  block_exclusive_scan(kwl, shd, kw);
  block_exclusive_scan(kcl, shl, kchi);
  if (tid == 0) {
    stats[0] = total;
    stats[1] = total - kw;                     // discarded weight
    stats[2] = kw > 0 ? 1.0 / sqrt(kw) : 0.0;  // renormalisation of the kept values
    stats[3] = (double)K;
    stats[4] = (double)kchi;
    stats[5] = keep_chi < keep_eps ? 1.0 : 0.0;  // the chi cap, not the tail rule, set K
  }
}

void launch_truncate(const TruncSector* secs, int nsec, const int* offs, int n, double eps, long long chi_max,
                     double degen, int* owner, int* order, int* kept, double* stats, double* vals, cudaStream_t s) {
  note_launch(3);
  truncate_stage_kernel<<<std::max(1, std::min(148, (nsec + 7) / 8)), 256, 0, s>>>(secs, nsec, offs, n, owner, kept,
                                                                                vals);
  truncate_rank_kernel<<<std::max(1, (n + TRUNC_RANK_PER_CTA - 1) / TRUNC_RANK_PER_CTA), TRUNC_RANK_THREADS, 0, s>>>(
      n, vals, order);
  truncate_kernel<<<1, TRUNC_THREADS, 0, s>>>(secs, nsec, offs, n, eps, chi_max, degen, owner, order, kept, stats,
                                              vals);
}

// ---------------------------------------------------------------------------
// Gauge shift of the one-site sweep: Cholesky QR.  One CTA per matrix, in place,
// right-looking: for each pivot j the row j is scaled by 1/sqrt(K_jj) and the
// trailing upper triangle is updated, K_ik -= conj(R_ji) R_jk; then R^-1 by back
// substitution, one column per thread.  shift_rel > 0 adds shift_rel * tr(K) / q to
// the diagonal first (the shifted first pass of a repeated Cholesky QR, which keeps
// a numerically rank-deficient K factorisable).  A non-positive pivot sets *status.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) chol_inv_kernel(const CholTask* __restrict__ tasks, double shift_rel,
                                                       int* __restrict__ status) {
  const CholTask t = tasks[blockIdx.x];
  const int q = t.q;
  cplx* K = t.k;
  __shared__ double sdiag;
  __shared__ int bad;
  if (threadIdx.x == 0) {
    bad = 0;
    double tr = 0.0;
    for (int j = 0; j < q; ++j) tr += K[(long long)j * q + j].x;
    sdiag = shift_rel > 0.0 ? shift_rel * tr / (q > 0 ? q : 1) : 0.0;
  }
  __syncthreads();
  if (sdiag > 0.0)
    for (int j = threadIdx.x; j < q; j += blockDim.x) K[(long long)j * q + j].x += sdiag;
  __syncthreads();
  for (int j = 0; j < q; ++j) {
    const double d = K[(long long)j * q + j].x;
    if (!(d > 0.0)) {
      if (threadIdx.x == 0) bad = 1;
      break;  // uniform: every thread read the same d
    }
    const double r = sqrt(d), ir = 1.0 / r;
    __syncthreads();
    for (int k = j + threadIdx.x; k < q; k += blockDim.x) {
      cplx v = K[(long long)j * q + k];
      K[(long long)j * q + k] = k == j ? cplx{r, 0.0} : cplx{v.x * ir, v.y * ir};
    }
    __syncthreads();
    const int m = q - j - 1;  // trailing block rows/cols j+1..q-1, upper triangle
    for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
      const int i = j + 1 + (int)(e / m), k = j + 1 + (int)(e % m);
      if (k < i) continue;
      const cplx a = K[(long long)j * q + i], b = K[(long long)j * q + k];  // R_ji, R_jk
      cplx& c = K[(long long)i * q + k];
      c.x -= a.x * b.x + a.y * b.y;  // conj(a) b
      c.y -= a.x * b.y - a.y * b.x;
    }
    __syncthreads();
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) atomicAdd(status, 1);
    return;
  }
  // zero the strict lower triangle, then X = R^-1 column by column (upper triangular)
  for (long long e = threadIdx.x; e < (long long)q * q; e += blockDim.x) {
    const int i = (int)(e / q), k = (int)(e % q);
    if (k < i) K[e] = {0.0, 0.0};
  }
  __syncthreads();
  for (int k = threadIdx.x; k < q; k += blockDim.x) {
    cplx* X = t.rinv;
    for (int i = q - 1; i >= 0; --i) {
      cplx acc = {i == k ? 1.0 : 0.0, 0.0};
      if (i <= k) {
        for (int j = i + 1; j <= k; ++j) {
          const cplx a = K[(long long)i * q + j], x = X[(long long)j * q + k];
          acc.x -= a.x * x.x - a.y * x.y;
          acc.y -= a.x * x.y + a.y * x.x;
        }
        const double ir = 1.0 / K[(long long)i * q + i].x;
        X[(long long)i * q + k] = {acc.x * ir, acc.y * ir};
      } else {
        X[(long long)i * q + k] = {0.0, 0.0};
      }
    }
  }
}

void launch_chol_inv(const CholTask* tasks, int n, double shift_rel, int* status, cudaStream_t s) {
  if (n <= 0) return;
  note_launch();
  chol_inv_kernel<<<n, 256, 0, s>>>(tasks, shift_rel, status);
}

// ---------------------------------------------------------------------------
// K9: block-weighted dots (measurement) and entanglement entropy
// ---------------------------------------------------------------------------

// one CTA per task; out[slot] accumulated with atomics in slot order is not
// deterministic, so each task writes its own partial and a second kernel sums
// the partials of every slot in task order.
__global__ void __launch_bounds__(256) wdot_kernel(const DotTask* __restrict__ tasks, double* __restrict__ partial) {
  const DotTask t = tasks[blockIdx.x];
  double acc = 0.0;
  const int n = t.rows * t.cols;
  for (int e = threadIdx.x; e < n; e += 256) {
    int r = e / t.cols, c = e - r * t.cols;
    cplx x = t.x[(long long)r * t.ldx + c], y = t.y[(long long)r * t.ldy + c];
    acc += x.x * y.x + x.y * y.y;  // Re(conj(x) y)
  }
  __shared__ double sb[256];
  sb[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sb[threadIdx.x] += sb[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = t.weight * sb[0];
}

__global__ void wdot_final_kernel(const DotTask* __restrict__ tasks, const double* __restrict__ partial, int ntasks,
                                  double* __restrict__ out, int nslots) {
  for (int s = threadIdx.x; s < nslots; s += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < ntasks; ++k)
      if (tasks[k].slot == s) acc += partial[k];
    out[s] = acc;
  }
}

void launch_wdot(const DotTask* tasks, int ntasks, double* partial, double* out, int nslots, cudaStream_t s) {
  if (ntasks <= 0) return;
  note_launch();
  wdot_kernel<<<ntasks, 256, 0, s>>>(tasks, partial);
  note_launch();
  wdot_final_kernel<<<1, 256, 0, s>>>(tasks, partial, ntasks, out, nslots);
}

// S = -sum_sectors sum_k lam ln(lam / mult), lam = eigenvalue (weight) of a multiplet
__global__ void entropy_kernel(const TruncSector* __restrict__ secs, int nsec, double* __restrict__ out) {
  double acc = 0.0;
  for (int s = threadIdx.x; s < nsec; s += blockDim.x) {
    for (int i = 0; i < secs[s].r; ++i) {
      double lam = secs[s].sv[i];
      if (lam > 1e-300) acc -= lam * log(lam / secs[s].mult);
    }
  }
  __shared__ double sb[256];
  sb[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sb[threadIdx.x] += sb[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sb[0];
}

// Counter-based complex normal numbers: element i uses SplitMix64(seed, 2i) and
// SplitMix64(seed, 2i+1) as two uniforms for a Box-Muller pair (synthetic states).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void fill_normal_kernel(cplx* __restrict__ p, long long n, unsigned long long seed, long long offset) {
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const unsigned long long c = (unsigned long long)(i + offset);
    const double u1 = ((splitmix64(seed ^ (2 * c)) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (splitmix64(seed ^ (2 * c + 1)) >> 11) * (1.0 / 9007199254740992.0);
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    p[i] = {r * cs, r * sn};
  }
}

void launch_fill_normal(cplx* p, long long n, unsigned long long seed, long long offset, cudaStream_t s) {
  if (n <= 0) return;
  note_launch();
  fill_normal_kernel<<<blas_grid(n), 256, 0, s>>>(p, n, seed, offset);
}

// S = -sum lam ln(lam / mult) with lam = (g s)^2 from kept singular values s
__global__ void entropy_sv_kernel(const TruncSector* __restrict__ secs, int nsec, const double* g, double* out) {
  const double gg = g ? *g : 1.0;
  double acc = 0.0;
  for (int s = threadIdx.x; s < nsec; s += blockDim.x) {
    for (int i = 0; i < secs[s].r; ++i) {
      double x = gg * secs[s].sv[i];
      double lam = x * x;
      if (lam > 1e-300) acc -= lam * log(lam / secs[s].mult);
    }
  }
  __shared__ double sb[256];
  sb[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sb[threadIdx.x] += sb[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sb[0];
}

void launch_entropy_sv(const TruncSector* secs, int nsec, const double* g, double* out, cudaStream_t s) {
  note_launch();
  entropy_sv_kernel<<<1, 256, 0, s>>>(secs, nsec, g, out);
}

void launch_entropy(const TruncSector* secs, int nsec, double* out, cudaStream_t s) {
  note_launch();
  entropy_kernel<<<1, 256, 0, s>>>(secs, nsec, out);
}

}  // namespace tdvp
