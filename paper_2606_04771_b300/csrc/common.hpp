// Task descriptors shared by the host planner and the device kernels.
//
// Every contraction of the method (effective Hamiltonian, environment
// updates, two-site tensor formation, measurement) is lowered by the host into
// flat lists of these tasks; the kernels know nothing about symmetry labels.
#pragma once
#include <cstdint>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace tdvp {

struct cplx {
  double x, y;
};

// One output block C (rows x cols, leading dimension ldc, row-major) computed as
// C = sum_seg alpha_seg * op(A_seg) * op(B_seg).  A task with no segment writes zeros.
// Pointers in GemmTask/GemmSeg are relative to one of four launch-time bases
// (base 0 is the null address, i.e. the pointer is absolute); this lets one plan
// serve every Krylov vector without rewriting the task list.
struct Bases4 {
  uintptr_t p[4];
};

struct GemmTask {
  cplx* c;
  int c_base;
  int rows, cols, ldc;
  int seg_begin, seg_count;
  int tiles_m, tiles_n;  // filled by the planner for the tile size in use
  int roff, coff;        // BF16x4: scale-group offsets of this task's rows and columns
  // BF16x4 packed tasks: output row r starts at element c + rowoff[r] (rows of
  // several output blocks stacked in one task) when rowoff is set, else at c + r ldc;
  // tn = complex columns per output tile (a multiple of 16, at most 64; 0 = default)
  const long long* rowoff;
  int tn;
  int b_kmajor;  // BF16x4: the B records are stored column by column (K contiguous)
  int img;       // BF16x4 packed task: a_dig / b_dig hold tile images (DigitOp::img_nkc)
};

// op flags
enum : int { OP_N = 0, OP_C = 1 };  // OP_C: conjugate transpose

struct GemmSeg {
  const cplx* a;
  const cplx* b;
  int a_base, b_base;
  int lda, ldb, k;
  int op_a, op_b;
  double alpha;
  // BF16x4: digit records of the operands in logical orientation (A: rows x k,
  // B: k x cols, row-major, 8 bytes per complex element), filled per launch
  const unsigned long long* a_dig;
  const unsigned long long* b_dig;
  // operand unchanged between launches of its plan (environment blocks): BF16x4
  // splits it at the first launch only
  int a_static, b_static;
};

// BF16x4: one distinct operand block split into digit records.  A operands get a
// power-of-two scale per row, B operands per column; operands that meet in one task
// share their group's scales (grp: offset of the group's first row/column).
struct DigitOp {
  const cplx* src;
  int base;
  int rows, cols;  // logical (after op): A: M x K, B: K x N
  int ld, op;
  double alpha;    // A only
  int side;        // 0: A (row scales), 1: B (column scales)
  int grp;
  unsigned long long* dig;
  // placement in the digit records: element (r, c) goes to dig[(row0 + r) dig_ld +
  // col0 + c] (kmajor: dig[(col0 + c) dig_ld + row0 + r]) and takes the scale of
  // group row grp + row0 + r (A) or column grp + col0 + c (B); an operand of its own
  // has row0 = col0 = 0, dig_ld = cols and kmajor = 0
  int dig_ld, row0, col0, kmajor;
  // tile images (packed plans): img_nkc > 0 writes the digits straight into the BF16
  // planes of the GEMM's shared-memory tiles, tile after tile, at dig (A: 64 complex
  // rows x 16 complex k per 32 KB tile, embedded as [[re, -im], [im, re]]; B: img_tn
  // complex columns x 16 complex k per 16 KB tile), so that the GEMM fetches each
  // stage with bulk copies instead of unpacking records
  int img_nkc, img_tn;
};

template <class T>
__host__ __device__ inline T* rebase(const Bases4& B, int base, T* p) {
  return reinterpret_cast<T*>(B.p[base] + reinterpret_cast<uintptr_t>(p));
}

// out (rows x cols, ld_out) = sum_term coef * in_term (same shape, ld_in)
struct LincombTask {
  cplx* out;
  int rows, cols, ld_out;
  int term_begin, term_count;
  // optional: the BF16x4 exponent tags of the output's rows (one per row, row r at
  // tags[r]), raised to the launch's epoch and the rows' largest binary exponents
  unsigned* tags;
};

struct LincombTerm {
  const cplx* in;
  int ld_in;
  double coef;
};

// Strided copy: dst[r*dst_rs + c*dst_cs] = f(src[r*src_rs + c*src_cs])
// with f = optional conjugation and a per-column (of the destination) scale taken
// from scale[c] (scale_mode 1: multiply, 2: divide, 0: none) and a global factor.
struct CopyTask {
  const cplx* src;
  cplx* dst;
  int rows, cols;
  long long src_rs, src_cs, dst_rs, dst_cs;
  const int* row_map;    // optional: source row of destination row r is row_map[r]
  const int* col_map;    // optional: source column of destination column c is col_map[c]
  const double* scale;   // per destination column (modes 1, 2) or row (modes 3, 4)
  int scale_mode;        // 0 none, 1 *scale[c], 2 /scale[c], 3 *scale[r], 4 /scale[r]
  int conj;
  const double* gscale;  // optional device scalar applied to every element
};

// One Jacobi SVD problem: G is p x q column-major (p >= q) with leading dimension p,
// V is q x q column-major.  On exit G holds U*S in descending order of S, V the right
// singular vectors in the same order, sv[0..q) the singular values.
struct SvdTask {
  cplx* g;
  cplx* v;
  double* sv;   // q values, sorted descending on exit
  int* perm;    // q entries: perm[k] = column of G/V holding the k-th largest value
  int p, q;
};

// Truncation input: one entry per SVD problem (a bond sector)
struct TruncSector {
  const double* sv;  // sorted descending
  int r;             // number of singular values
  int mult;          // 2S+1 (SU(2)) or 1
};

// FP32 Jacobi preconditioner: g is p x q column-major complex64 (p >= q), v the
// q x q column-major accumulated right rotations
struct Svd32Task {
  float2* g;
  float2* v;
  int p, q;
};

// One column set of the mixed split's Gram finish: c is the q x q row-major matrix
// C[a][b] = sum_r G_ra conj(G_rb) (the conjugate of G^H G), zt receives Z^T (row-major
// q x q, zt[i][k] = Z[k][i]) of the simultaneous rotation G <- G Z.
struct GramTask {
  const cplx* c;
  cplx* zt;
  int q;
};

struct BasisTask {  // x[i][kk] = g[i, perm[kk]] / sv[kk] (or / sv[kk]^2); g column-major, rows x .
  const cplx* g;
  const int* perm;
  const double* sv;
  cplx* x;
  int rows, k;
  int pow2;
};

// One Cholesky factorisation K = R^H R of a Hermitian positive definite q x q matrix
// (row-major, overwritten by R, upper triangular) and the inverse rinv = R^-1.
struct CholTask {
  cplx* k;
  cplx* rinv;
  int q;
};

struct NsTask {  // g <- 1.5 I - 0.5 g (k x k)
  cplx* g;
  int k;
};

// Block-weighted inner product contribution: sum_ij weight * conj(x[i,j]) * y[i,j]
struct DotTask {
  const cplx* x;
  const cplx* y;
  int rows, cols, ldx, ldy;
  int slot;      // output slot
  double weight;
};

}  // namespace tdvp
