// FP64 device kernels of the TDVP engine (CUDA cores, sm_103a).
//
// These are the exact-arithmetic (FP64) building blocks: a grouped complex GEMM
// over planner-built task lists, the MPO linear combination, strided block
// copies, Krylov vector algebra, the small Krylov exponential, one-sided Jacobi
// SVD, truncation selection, block-weighted dots and the entanglement entropy.
// All kernels are symmetry-agnostic; the host planner lowers every contraction
// to task lists (common.hpp).
#include <cuda_runtime.h>

#include <cstdio>
#include <vector>

#include "common.hpp"
#include "kernels.hpp"

namespace tdvp {

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
                                                        const int3* __restrict__ tiles, const Bases4 B) {
  __shared__ cplx As[GK][GT + 1];
  __shared__ cplx Bs[GK][GT + 1];
  const int3 tr = tiles[blockIdx.x];
  const GemmTask t = tasks[tr.x];
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
    for (int k0 = 0; k0 < sg.k; k0 += GK) {
      // load A tile: GT rows x GK k
      for (int e = threadIdx.x; e < GT * GK; e += 256) {
        int r = e / GK, kk = e % GK;
        int gr = m0 + r, gk = k0 + kk;
        cplx v = {0.0, 0.0};
        if (gr < t.rows && gk < sg.k) {
          if (sg.op_a == OP_N) v = ap[(long long)gr * sg.lda + gk];
          else v = cconj(ap[(long long)gk * sg.lda + gr]);
        }
        As[kk][r] = v;
      }
      for (int e = threadIdx.x; e < GT * GK; e += 256) {
        int kk = e / GT, c = e % GT;
        int gc = n0 + c, gk = k0 + kk;
        cplx v = {0.0, 0.0};
        if (gc < t.cols && gk < sg.k) {
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

void launch_gemm_fp64(const GemmTask* tasks, const GemmSeg* segs, const int3* tiles, int ntiles, const Bases4& B,
                      cudaStream_t s) {
  if (ntiles <= 0) return;
  gemm_fp64_kernel<<<ntiles, 256, 0, s>>>(tasks, segs, tiles, B);
}

// ---------------------------------------------------------------------------
// K3: MPO linear combination  out = sum coef * in
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) lincomb_kernel(const LincombTask* __restrict__ tasks,
                                                      const LincombTerm* __restrict__ terms,
                                                      const int2* __restrict__ chunks) {
  const int2 ch = chunks[blockIdx.x];
  const LincombTask t = tasks[ch.x];
  const int n = t.rows * t.cols;
  for (int e = ch.y + threadIdx.x; e < min(n, ch.y + LINCOMB_CHUNK); e += 256) {
    int r = e / t.cols, c = e - r * t.cols;
    cplx acc = {0.0, 0.0};
    for (int k = 0; k < t.term_count; ++k) {
      const LincombTerm tm = terms[t.term_begin + k];
      cplx v = tm.in[(long long)r * tm.ld_in + c];
      acc.x = fma(tm.coef, v.x, acc.x);
      acc.y = fma(tm.coef, v.y, acc.y);
    }
    t.out[(long long)r * t.ld_out + c] = acc;
  }
}

void launch_lincomb(const LincombTask* tasks, const LincombTerm* terms, const int2* chunks, int nchunks,
                    cudaStream_t s) {
  if (nchunks <= 0) return;
  lincomb_kernel<<<nchunks, 256, 0, s>>>(tasks, terms, chunks);
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
  dots_partial_kernel<<<grid, 256, 0, s>>>(V, pitch, nv, w, n, partial, done);
  dots_final_kernel<<<nv, 32, 0, s>>>(partial, G, nv, out, done);
}

void launch_axpy_many(const cplx* V, long long pitch, int nv, const cplx* h, cplx* w, long long n, const int* done,
                      cudaStream_t s) {
  axpy_many_kernel<<<blas_grid(n), 256, 0, s>>>(V, pitch, nv, h, w, n, done);
}

void launch_combine(const cplx* V, long long pitch, const int* nv, const cplx* coef, const double* scal, cplx* out,
                    long long n, cudaStream_t s) {
  combine_kernel<<<blas_grid(n), 256, 0, s>>>(V, pitch, nv, coef, scal, out, n);
}

void launch_scale(const cplx* x, const double* nrm, cplx* y, long long n, const int* done, cudaStream_t s) {
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
  int steps = (int)ceil(fabs(tau) * rowsum / 0.5);
  if (steps < 1) steps = 1;
  const double h = tau / steps;
  double xr = lane == 0 ? 1.0 : 0.0, xi = 0.0;
  for (int s = 0; s < steps; ++s) {
    double tr = xr, ti = xi, sr = xr, si = xi;
    for (int m = 1; m <= 40; ++m) {
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
      double mag = fabs(tr) + fabs(ti);
      for (int o = 16; o > 0; o >>= 1) mag = fmax(mag, __shfl_xor_sync(0xffffffffu, mag, o));
      if (mag < 1e-22) break;
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

void launch_krylov_init(KrylovState* st, const cplx* nrm2, cudaStream_t s) { krylov_init_kernel<<<1, 1, 0, s>>>(st, nrm2); }

void launch_krylov_step(KrylovState* st, const cplx* h1, const cplx* nrm2, double tau, double tol, int kmax,
                        cudaStream_t s) {
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
// K6 (blocked): one-sided Jacobi in rounds over column blocks, many CTAs per matrix
//
// The Q columns of every problem are cut into blocks of bw columns (the block count
// padded to even).  One launch performs one round of the block tournament for every
// problem: each CTA takes one pair of blocks, copies their columns of G and V into
// shared memory, runs one cyclic pass over all column pairs of the 2 bw columns
// (FP64 complex Jacobi rotations, as in jacobi_svd_kernel), and writes them back.  A
// sweep is nb - 1 rounds; a problem whose previous sweep made no rotation is skipped.
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

__global__ void __launch_bounds__(256) bjacobi_round_kernel(const SvdTask* __restrict__ tasks,
                                                            const int2* __restrict__ work, int round, int bw,
                                                            double tol, double tol_flag, int* __restrict__ flag_now,
                                                            const int* __restrict__ flag_prev) {
  const int2 wk = work[blockIdx.x];
  const SvdTask t = tasks[wk.x];
  if (flag_prev && flag_prev[wk.x] == 0) return;  // converged in the previous sweep
  const int nb0 = (t.q + bw - 1) / bw;
  const int nb = nb0 + (nb0 & 1);
  if (nb < 2 || round >= nb - 1) return;
  int I, Jb;
  tourney(round, wk.y, nb, I, Jb);
  const int p = t.p, q = t.q;
  const bool with_v = t.v != nullptr;
  extern __shared__ cplx sm[];
  const int nc = 2 * bw;
  cplx* Gs = sm;                  // nc columns x p rows
  cplx* Vs = sm + (size_t)nc * p;  // nc columns x q rows (when V is accumulated)
  int col[64];
  int ncol = 0;
  for (int c = 0; c < bw; ++c)
    if (I * bw + c < q) col[ncol++] = I * bw + c;
  for (int c = 0; c < bw; ++c)
    if (Jb * bw + c < q) col[ncol++] = Jb * bw + c;
  if (ncol < 2) return;
  for (int cc = 0; cc < ncol; ++cc) {
    const cplx* g = t.g + (long long)col[cc] * p;
    for (int r = threadIdx.x; r < p; r += blockDim.x) Gs[(size_t)cc * p + r] = g[r];
    if (with_v) {
      const cplx* v = t.v + (long long)col[cc] * q;
      for (int r = threadIdx.x; r < q; r += blockDim.x) Vs[(size_t)cc * q + r] = v[r];
    }
  }
  __shared__ int rotated;
  if (threadIdx.x == 0) rotated = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int nn = ncol + (ncol & 1);
  for (int r = 0; r < nn - 1; ++r) {
    for (int k = warp; k < nn / 2; k += nwarp) {
      int i, j;
      tourney(r, k, nn, i, j);
      if (j >= ncol) continue;
      double a, b;
      cplx c;
      col_pair(Gs, p, i, j, a, b, c);
      double ac = sqrt(c.x * c.x + c.y * c.y);
      if (ac == 0.0 || ac <= tol * sqrt(a * b)) continue;
      double zeta = (b - a) / (2.0 * ac);
      double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
      cplx e = {c.x / ac, c.y / ac};
      rotate_cols(Gs, p, p, i, j, cs, sn, e);
      if (with_v) rotate_cols(Vs, q, q, i, j, cs, sn, e);
      if ((threadIdx.x & 31) == 0 && ac > tol_flag * sqrt(a * b)) rotated = 1;
    }
    __syncthreads();
  }
  for (int cc = 0; cc < ncol; ++cc) {
    cplx* g = t.g + (long long)col[cc] * p;
    for (int r = threadIdx.x; r < p; r += blockDim.x) g[r] = Gs[(size_t)cc * p + r];
    if (with_v) {
      cplx* v = t.v + (long long)col[cc] * q;
      for (int r = threadIdx.x; r < q; r += blockDim.x) v[r] = Vs[(size_t)cc * q + r];
    }
  }
  if (threadIdx.x == 0 && rotated) atomicOr(&flag_now[wk.x], 1);
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
  extern __shared__ double sb[];
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    double v = t.sv[j];
    sb[j] = (v == v) ? v : -1.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    double vj = sb[j];
    int rank = 0;
    for (int i = 0; i < q; ++i) {
      double vi = sb[i];
      rank += (vi > vj) || (vi == vj && i < j);
    }
    t.perm[rank] = j;
    t.sv[rank] = vj < 0.0 ? 0.0 : vj;
  }
}

// Blocked Jacobi driver: returns the number of sweeps used (host loop, one sync per sweep).
// V is accumulated (from the identity) when the tasks carry v; without v only G is
// rotated.  A sweep in which no rotation exceeded tol_flag (relative, as tol) ends
// the iteration: with tol_flag = tol that is the usual "no rotation at all" test,
// with tol_flag = sqrt(tol) it relies on the quadratic convergence of cyclic Jacobi
// (off-diagonal delta before a sweep leaves O(delta^2) after it).
int run_blocked_jacobi(const SvdTask* d_tasks, const std::vector<SvdTask>& h_tasks, int max_sweeps, double tol,
                       int* status, cudaStream_t s, double tol_flag) {
  const int nt = (int)h_tasks.size();
  if (nt == 0) return 0;
  if (!(tol_flag >= tol)) tol_flag = tol;
  int pmax = 1, qmax = 1;
  for (auto& t : h_tasks) {
    pmax = max(pmax, t.p);
    qmax = max(qmax, t.q);
  }
  const int vrows = h_tasks[0].v ? qmax : 0;
  // widest block (<= 32 columns) whose pair of column copies fits in shared memory
  int bw = 32;
  while (bw > 1 && (size_t)2 * bw * (pmax + vrows) * sizeof(cplx) > 200 * 1024) bw >>= 1;
  if ((size_t)2 * bw * (pmax + vrows) * sizeof(cplx) > 200 * 1024) return -1;  // caller falls back
  const size_t smem = (size_t)2 * bw * (pmax + vrows) * sizeof(cplx);
  cudaFuncSetAttribute(bjacobi_round_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  std::vector<int2> work;
  int max_rounds = 0;
  for (int i = 0; i < nt; ++i) {
    int nb0 = (h_tasks[i].q + bw - 1) / bw, nb = nb0 + (nb0 & 1);
    for (int k = 0; k < nb / 2; ++k) work.push_back(make_int2(i, k));
    max_rounds = max(max_rounds, nb - 1);
  }
  int2* d_work = nullptr;
  int* flags = nullptr;
  cudaMallocAsync(&d_work, work.size() * sizeof(int2), s);
  cudaMallocAsync(&flags, 2 * nt * sizeof(int), s);
  cudaMemcpyAsync(d_work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
  svd_init_v_kernel<<<nt, 256, 0, s>>>(d_tasks);
  std::vector<int> hf(nt);
  int sweep = 0, *prev = nullptr, *now = flags;
  for (; sweep < max_sweeps; ++sweep) {
    cudaMemsetAsync(now, 0, nt * sizeof(int), s);
    for (int r = 0; r < max_rounds; ++r)
      bjacobi_round_kernel<<<(int)work.size(), 256, smem, s>>>(d_tasks, d_work, r, bw, tol, tol_flag, now, prev);
    cudaMemcpyAsync(hf.data(), now, nt * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    bool any = false;
    for (int v : hf) any |= v != 0;
    if (!any) break;
    prev = now;
    now = (now == flags) ? flags + nt : flags;
  }
  if (sweep >= max_sweeps) {
    int one = 1;
    cudaMemcpyAsync(status, &one, sizeof(int), cudaMemcpyHostToDevice, s);  // reported by the caller's check
    cudaStreamSynchronize(s);
  }
  size_t fs = (size_t)qmax * sizeof(double);
  if (fs > 48 * 1024) cudaFuncSetAttribute(svd_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs);
  svd_finish_kernel<<<nt, 256, fs, s>>>(d_tasks);
  cudaFreeAsync(d_work, s);
  cudaFreeAsync(flags, s);
  return sweep;
}

// ---------------------------------------------------------------------------
// K6 (FP32 preconditioner): blocked one-sided Jacobi on a complex64 copy of G with
// the right rotations accumulated in a complex64 V.  Used by the split-precision
// modes: V is widened to FP64, G = A V is formed again in FP64 and a short FP64
// Jacobi finishes the SVD, so every singular value the truncation sees is an FP64
// one (the FP32 columns themselves are discarded).
// ---------------------------------------------------------------------------

__device__ void col_pair32(const float2* __restrict__ g, int p, int i, int j, float& a, float& b, float2& c) {
  const int lane = threadIdx.x & 31;
  float sa = 0, sb = 0, cx = 0, cy = 0;
  const float2* gi = g + (long long)i * p;
  const float2* gj = g + (long long)j * p;
  for (int r = lane; r < p; r += 32) {
    float2 x = gi[r], y = gj[r];
    sa = fmaf(x.x, x.x, fmaf(x.y, x.y, sa));
    sb = fmaf(y.x, y.x, fmaf(y.y, y.y, sb));
    cx = fmaf(x.x, y.x, fmaf(x.y, y.y, cx));
    cy = fmaf(x.x, y.y, fmaf(-x.y, y.x, cy));
  }
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
    cx += __shfl_xor_sync(0xffffffffu, cx, o);
    cy += __shfl_xor_sync(0xffffffffu, cy, o);
  }
  a = sa;
  b = sb;
  c = make_float2(cx, cy);
}

__device__ void rotate32(float2* __restrict__ g, int ld, int len, int i, int j, float cs, float sn, float2 e) {
  const int lane = threadIdx.x & 31;
  float2* gi = g + (long long)i * ld;
  float2* gj = g + (long long)j * ld;
  for (int r = lane; r < len; r += 32) {
    float2 x = gi[r], y = gj[r];
    float2 ey = make_float2(e.x * y.x + e.y * y.y, e.x * y.y - e.y * y.x);
    float2 ex = make_float2(e.x * x.x - e.y * x.y, e.x * x.y + e.y * x.x);
    gi[r] = make_float2(cs * x.x - sn * ey.x, cs * x.y - sn * ey.y);
    gj[r] = make_float2(sn * ex.x + cs * y.x, sn * ex.y + cs * y.y);
  }
}

__global__ void __launch_bounds__(256) bjacobi32_round_kernel(const Svd32Task* __restrict__ tasks,
                                                              const int2* __restrict__ work, int round, int bw,
                                                              float tol, int* __restrict__ flag_now,
                                                              const int* __restrict__ flag_prev) {
  const int2 wk = work[blockIdx.x];
  const Svd32Task t = tasks[wk.x];
  if (flag_prev && flag_prev[wk.x] == 0) return;
  const int nb0 = (t.q + bw - 1) / bw;
  const int nb = nb0 + (nb0 & 1);
  if (nb < 2 || round >= nb - 1) return;
  int I, Jb;
  tourney(round, wk.y, nb, I, Jb);
  const int p = t.p, q = t.q;
  extern __shared__ float2 sg[];
  float2* sv = sg + (size_t)2 * bw * p;  // V columns after the G columns
  int ncol = 0;
  int col[64];
  for (int c = 0; c < bw; ++c)
    if (I * bw + c < q) col[ncol++] = I * bw + c;
  for (int c = 0; c < bw; ++c)
    if (Jb * bw + c < q) col[ncol++] = Jb * bw + c;
  if (ncol < 2) return;
  for (int cc = 0; cc < ncol; ++cc) {
    const float2* g = t.g + (long long)col[cc] * p;
    const float2* v = t.v + (long long)col[cc] * q;
    for (int r = threadIdx.x; r < p; r += blockDim.x) sg[(size_t)cc * p + r] = g[r];
    for (int r = threadIdx.x; r < q; r += blockDim.x) sv[(size_t)cc * q + r] = v[r];
  }
  __shared__ int rotated;
  if (threadIdx.x == 0) rotated = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int nn = ncol + (ncol & 1);
  for (int r = 0; r < nn - 1; ++r) {
    for (int k = warp; k < nn / 2; k += nwarp) {
      int i, j;
      tourney(r, k, nn, i, j);
      if (j >= ncol) continue;
      float a, b;
      float2 c;
      col_pair32(sg, p, i, j, a, b, c);
      float ac = sqrtf(c.x * c.x + c.y * c.y);
      if (ac == 0.0f || ac <= tol * sqrtf(a * b)) continue;
      float zeta = (b - a) / (2.0f * ac);
      float tt = (zeta >= 0 ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
      float cs = 1.0f / sqrtf(1.0f + tt * tt), sn = cs * tt;
      float2 e = make_float2(c.x / ac, c.y / ac);
      rotate32(sg, p, p, i, j, cs, sn, e);
      rotate32(sv, q, q, i, j, cs, sn, e);
      if ((threadIdx.x & 31) == 0) rotated = 1;
    }
    __syncthreads();
  }
  for (int cc = 0; cc < ncol; ++cc) {
    float2* g = t.g + (long long)col[cc] * p;
    float2* v = t.v + (long long)col[cc] * q;
    for (int r = threadIdx.x; r < p; r += blockDim.x) g[r] = sg[(size_t)cc * p + r];
    for (int r = threadIdx.x; r < q; r += blockDim.x) v[r] = sv[(size_t)cc * q + r];
  }
  if (threadIdx.x == 0 && rotated) atomicOr(&flag_now[wk.x], 1);
}

__global__ void svd32_init_v_kernel(const Svd32Task* __restrict__ tasks) {
  const Svd32Task t = tasks[blockIdx.x];
  for (int e = threadIdx.x; e < t.q * t.q; e += blockDim.x)
    t.v[e] = make_float2((e % t.q) == (e / t.q) ? 1.0f : 0.0f, 0.0f);
}

int run_blocked_jacobi32(const Svd32Task* d_tasks, const std::vector<Svd32Task>& h_tasks, int max_sweeps, float tol,
                         cudaStream_t s) {
  const int nt = (int)h_tasks.size();
  if (nt == 0) return 0;
  int pmax = 1, qmax = 1;
  for (auto& t : h_tasks) {
    pmax = max(pmax, t.p);
    qmax = max(qmax, t.q);
  }
  int bw = 32;
  while (bw > 1 && (size_t)2 * bw * (pmax + qmax) * sizeof(float2) > 200 * 1024) bw >>= 1;
  if ((size_t)2 * bw * (pmax + qmax) * sizeof(float2) > 200 * 1024) return -1;
  const size_t smem = (size_t)2 * bw * (pmax + qmax) * sizeof(float2);
  cudaFuncSetAttribute(bjacobi32_round_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  std::vector<int2> work;
  int max_rounds = 0;
  for (int i = 0; i < nt; ++i) {
    int nb0 = (h_tasks[i].q + bw - 1) / bw, nb = nb0 + (nb0 & 1);
    for (int k = 0; k < nb / 2; ++k) work.push_back(make_int2(i, k));
    max_rounds = max(max_rounds, nb - 1);
  }
  int2* d_work = nullptr;
  int* flags = nullptr;
  cudaMallocAsync(&d_work, (work.empty() ? 1 : work.size()) * sizeof(int2), s);
  cudaMallocAsync(&flags, 2 * nt * sizeof(int), s);
  if (!work.empty()) cudaMemcpyAsync(d_work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
  svd32_init_v_kernel<<<nt, 256, 0, s>>>(d_tasks);
  std::vector<int> hf(nt);
  int sweep = 0, *prev = nullptr, *now = flags;
  for (; sweep < max_sweeps && !work.empty(); ++sweep) {
    cudaMemsetAsync(now, 0, nt * sizeof(int), s);
    for (int r = 0; r < max_rounds; ++r)
      bjacobi32_round_kernel<<<(int)work.size(), 256, smem, s>>>(d_tasks, d_work, r, bw, tol, now, prev);
    cudaMemcpyAsync(hf.data(), now, nt * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    bool any = false;
    for (int v : hf) any |= v != 0;
    if (!any) break;
    prev = now;
    now = (now == flags) ? flags + nt : flags;
  }
  cudaFreeAsync(d_work, s);
  cudaFreeAsync(flags, s);
  return sweep;
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

static int conv_grid(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1184 ? (b < 1 ? 1 : b) : 1184);
}
void launch_narrow(const cplx* src, float2* dst, long long n, cudaStream_t s) {
  if (n > 0) narrow_kernel<<<conv_grid(n), 256, 0, s>>>(src, dst, n);
}
void launch_widen(const float2* src, cplx* dst, long long n, cudaStream_t s) {
  if (n > 0) widen_kernel<<<conv_grid(n), 256, 0, s>>>(src, dst, n);
}
void launch_basis64(const BasisTask* tasks, int n, cudaStream_t s) {
  if (n > 0) basis64_kernel<<<dim3(32, n), 256, 0, s>>>(tasks);
}
void launch_ns_coeff(const NsTask* tasks, int n, cudaStream_t s) {
  if (n > 0) ns_coeff_kernel<<<dim3(8, n), 256, 0, s>>>(tasks);
}

void launch_jacobi_svd(const SvdTask* tasks, int ntasks, int max_q, int max_sweeps, double tol, int* status,
                       cudaStream_t s) {
  if (ntasks <= 0) return;
  size_t smem = (size_t)max_q * sizeof(double);
  if (smem > 48 * 1024) cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  jacobi_svd_kernel<<<ntasks, SVD_THREADS, smem, s>>>(tasks, max_sweeps, tol, status);
}

// ---------------------------------------------------------------------------
// K7: truncation selection over all sectors of a bond (one CTA)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(1024) truncate_kernel(const TruncSector* __restrict__ secs, int nsec,
                                                        const int* __restrict__ offs, int n, double eps,
                                                        long long chi_max, int* __restrict__ owner,
                                                        int* __restrict__ order, int* __restrict__ kept,
                                                        double* __restrict__ stats) {
  // owner[e] = sector of flat entry e ; offs[s] = first flat index of sector s
  for (int s = threadIdx.x; s < nsec; s += blockDim.x) {
    for (int i = 0; i < secs[s].r; ++i) owner[offs[s] + i] = s;
    kept[s] = 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    int se = owner[e];
    double ve = secs[se].sv[e - offs[se]];
    if (!(ve == ve)) ve = -1.0;
    int rank = 0;
    for (int f = 0; f < n; ++f) {
      int sf = owner[f];
      double vf = secs[sf].sv[f - offs[sf]];
      if (!(vf == vf)) vf = -1.0;
      rank += (vf > ve) || (vf == ve && f < e);
    }
    order[rank] = e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double total = 0.0;
    for (int r = 0; r < n; ++r) {
      int e = order[r], se = owner[e];
      double v = secs[se].sv[e - offs[se]];
      total += v * v;
    }
    // longest tail with weight <= eps * total
    int keep_eps = n;
    double tail = 0.0;
    for (int r = n - 1; r >= 1; --r) {
      int e = order[r], se = owner[e];
      double v = secs[se].sv[e - offs[se]];
      if (tail + v * v <= eps * total) {
        tail += v * v;
        keep_eps = r;
      } else {
        break;
      }
    }
    // bond-dimension cap with multiplet sizes, greedy in descending order
    long long chi = 0;
    int keep_chi = 0;
    for (int r = 0; r < n; ++r) {
      int se = owner[order[r]];
      if (r > 0 && chi + secs[se].mult > chi_max) break;
      chi += secs[se].mult;
      keep_chi = r + 1;
    }
    int K = keep_eps < keep_chi ? keep_eps : keep_chi;
    if (K < 1) K = 1;
    double kw = 0.0;
    long long kchi = 0;
    for (int r = 0; r < K; ++r) {
      int e = order[r], se = owner[e];
      double v = secs[se].sv[e - offs[se]];
      kw += v * v;
      kchi += secs[se].mult;
      kept[se] += 1;
    }
    stats[0] = total;
    stats[1] = total - kw;           // discarded weight
    stats[2] = kw > 0 ? 1.0 / sqrt(kw) : 0.0;  // renormalisation of the kept values
    stats[3] = (double)K;
    stats[4] = (double)kchi;
  }
}

void launch_truncate(const TruncSector* secs, int nsec, const int* offs, int n, double eps, long long chi_max,
                     int* owner, int* order, int* kept, double* stats, cudaStream_t s) {
  truncate_kernel<<<1, 1024, 0, s>>>(secs, nsec, offs, n, eps, chi_max, owner, order, kept, stats);
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
  wdot_kernel<<<ntasks, 256, 0, s>>>(tasks, partial);
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
  entropy_sv_kernel<<<1, 256, 0, s>>>(secs, nsec, g, out);
}

void launch_entropy(const TruncSector* secs, int nsec, double* out, cudaStream_t s) {
  entropy_kernel<<<1, 256, 0, s>>>(secs, nsec, out);
}

}  // namespace tdvp
