// Launch wrappers of the device kernels (kernels.cu, split.cu).
#pragma once
#include <cuda_runtime.h>

#include <functional>
#include <vector>

#include "common.hpp"

namespace tdvp {

// Process-wide count of kernel launches made by this library (every launch site
// calls note_launch()); read through tdvp_launch_count.
void note_launch(int n = 1);
long long launch_count();

constexpr int LINCOMB_CHUNK = 1024;  // elements per CTA in lincomb / copy
constexpr int KRYLOV_MAX = 32;       // one warp holds the Krylov coefficients
// Krylov vectors of at most KRYLOV_BATCH_N complex elements: KRYLOV_BATCH iterations are
// queued between two reads of the convergence flags by the host
constexpr long long KRYLOV_BATCH_N = 1 << 16;
constexpr int KRYLOV_BATCH = 4;

// Device-resident Krylov state: the host launches the loop without reading it
// until the end (kernels return immediately once done is set).
struct KrylovState {
  double alpha[KRYLOV_MAX];
  double beta[KRYLOV_MAX];
  cplx coef[KRYLOV_MAX];
  double beta0;
  double err;
  int k;
  int nv;
  int done;
  int bad;  // set when a non-finite value appeared
};

// kx (or nullptr): per tile item its K range and partial slot (-1: write C directly;
// else the 64 x 64 partial goes to ws + slot 4096, single-segment tasks only)
void launch_gemm_fp64(const GemmTask* tasks, const GemmSeg* segs, const int3* tiles, int ntiles, const Bases4& B,
                      cudaStream_t s, const int4* kx = nullptr, cplx* ws = nullptr);
// sums the partial tiles of each split output tile (fix: task, tile row, tile column,
// first slot | count << 20) in slot order and writes C
void launch_gemm_fp64_fix(const GemmTask* tasks, const int4* fix, int nfix, const cplx* ws, const Bases4& B,
                          cudaStream_t s);
// epoch: the BF16x4 split epoch the output row tags are raised to (tasks with tags)
void launch_lincomb(const LincombTask* tasks, const LincombTerm* terms, const int2* chunks, int nchunks,
                    cudaStream_t s, unsigned epoch = 0);
void launch_copy(const CopyTask* tasks, const int2* chunks, int nchunks, cudaStream_t s);

// split-precision tensor-core GEMM (split.cu); kind 0 = 3xTF32 (FP32 accumulation),
// 1 = BF16x4 digits with exact per-order accumulation.  Output tiles are
// split_tile_m() x split_tile_n(kind) complex elements; alpha scales A.
int split_tile_m();
int split_tile_n(int kind);
void launch_gemm_split(int kind, const GemmTask* tasks, const GemmSeg* segs, const int3* tiles, int ntiles,
                       const int* exps, const Bases4& B, int* status, cudaStream_t s);
// One BF16x4 launch over the tile lists of several plans (slices): tile ti of the
// concatenated list is tile ti - start[s] of slice s, start[s] <= ti < start[s + 1].
constexpr int EXACT_MAX_SLICES = 8;
struct ExactSlice {
  const GemmTask* tasks;
  const GemmSeg* segs;
  const int3* tiles;
  const int* exps;
  int* status;
  Bases4 B;
  int img;  // every task holds tile images (GemmTask::img)
};
struct ExactLaunch {
  int nslices;
  int start[EXACT_MAX_SLICES + 1];
  ExactSlice sl[EXACT_MAX_SLICES];
};
void launch_gemm_exact_merged(const ExactLaunch& L, cudaStream_t s);
// merge.cpp: the BF16x4 GEMM of one plan, merged with the plans of other contexts
// that launch at the same moment when merging is on for the calling thread
void launch_exact_merged_or_alone(const ExactSlice& slice, int ntiles, cudaStream_t s);
bool& merge_launches_here();  // thread-local switch, set for the duration of a context's call
void merge_counts(long long* launches, long long* slices);
// BF16x4 operand splitting (once per launch): group exponent tags of this epoch, then
// digit records and exponents.  jobs = (operand, first element) in steps of
// digit_job_size() elements.  tags start at zero; epoch runs 1 .. 2^20 - 1.
int digit_job_size();
int digit_slots();  // longest scale line the fused split handles
constexpr unsigned DIGIT_EPOCH_MAX = (1u << 20) - 1;
// one bounded wait on an mbarrier that never completes; adds 1 to *status on expiry
void launch_wait_selftest(unsigned polls, int* status, cudaStream_t s);
// mode 0: both passes; 1: the tags of this epoch are already set (conversion only);
// 2: every operand holds whole rows (A) / columns (B) of its group, so one kernel per
// operand finds its exponents in shared memory and converts (the tags are not used)
void launch_digits(const DigitOp* ops, int nops, const int2* jobs, int njobs, unsigned* tags, int* exps,
                   unsigned epoch, const Bases4& B, cudaStream_t s, int mode = 0);

int dots_grid(long long n);
void launch_dots(const cplx* V, long long pitch, int nv, const cplx* w, long long n, cplx* partial, int G, cplx* out,
                 const int* done, cudaStream_t s);
void launch_axpy_many(const cplx* V, long long pitch, int nv, const cplx* h, cplx* w, long long n, const int* done,
                      cudaStream_t s);
void launch_combine(const cplx* V, long long pitch, const int* nv, const cplx* coef, const double* scal, cplx* out,
                    long long n, cudaStream_t s);
void launch_scale(const cplx* x, const double* nrm, cplx* y, long long n, const int* done, cudaStream_t s);
void launch_krylov_init(KrylovState* st, const cplx* nrm2, cudaStream_t s);
void launch_krylov_step(KrylovState* st, const cplx* h1, const cplx* nrm2, double tau, double tol, int kmax,
                        cudaStream_t s);

void launch_jacobi_svd(const SvdTask* tasks, int ntasks, int max_q, int max_sweeps, double tol, int* status,
                       cudaStream_t s);
// Time and algorithmic work of the cooperative Jacobi launches a caller asks to be
// profiled: ms summed over the launches (CUDA events around each launch on its
// stream), flops = sum over tasks of (sweeps in which the task was active) x
// q(q-1)/2 pairs x (16p for the two squared norms and the inner product of a column
// pair, 32p for rotating the pair, 32q for rotating the pair's columns of V when V
// is accumulated).  Every visited pair is counted as rotated.
struct JacobiProfile {
  double ms = 0, flops = 0;
  // calls; calls that ran CTA-resident, in clusters, as rings of warps in clusters
  long long launches = 0, resident = 0, cluster = 0, ring = 0;
};
// Device scratch for the small per-call work lists and flags of the Jacobi drivers:
// returns at least `bytes` bytes of device memory, usable in stream order on the
// driver's stream until the next request, or nullptr.  An empty function makes the
// driver allocate (and free) the region itself with cudaMallocAsync.  When no
// region can be had the drivers launch nothing and return JACOBI_ENOMEM.
using ScratchFn = std::function<void*(size_t)>;
constexpr int JACOBI_ENOMEM = -3;
// a bounded wait of the ring form gave up (the kernel stopped; the result is invalid)
constexpr int JACOBI_ETIMEOUT = -4;
// FP32 round-robin Jacobi on complex64 working copies (p >= q), accumulating V
// (from the identity); returns the sweeps run
int run_jacobi_rounds32(const Svd32Task* d_tasks, const std::vector<Svd32Task>& h_tasks, int max_sweeps, float tol,
                        float abs_flag, cudaStream_t s, JacobiProfile* prof = nullptr,
                        const ScratchFn& scratch = ScratchFn());
void launch_narrow(const cplx* src, float2* dst, long long n, cudaStream_t s);
void launch_widen(const float2* src, cplx* dst, long long n, cudaStream_t s);
void launch_basis64(const BasisTask* tasks, int n, cudaStream_t s);
void launch_ns_coeff(const NsTask* tasks, int n, cudaStream_t s);
// E = (I - K) / 2 into outs[i] from the upper triangle of task i's K (Newton-Schulz
// correction form X <- X + X E)
void launch_ns_corr(const NsTask* tasks, const cplx* const* outs, int n, cudaStream_t s);
// in-place Cholesky K = R^H R (upper R) and R^-1 for each task; a non-positive pivot
// adds 1 to *status
void launch_chol_inv(const CholTask* tasks, int n, double shift_rel, int* status, cudaStream_t s);
// round-robin one-sided Jacobi over all tasks at once, one warp per column pair
// (same result layout as launch_jacobi_svd; v may be NULL); returns the sweeps run
int run_jacobi_rounds(const SvdTask* d_tasks, const std::vector<SvdTask>& h_tasks, int max_sweeps, double tol,
                      int* status, cudaStream_t s, double tol_flag = 0.0, double abs_flag = 0.0,
                      JacobiProfile* prof = nullptr, const ScratchFn& scratch = ScratchFn());
// Multiplet selection of the truncation over nsec sectors (n values in all, sector k's
// at offs[k]); degen > 0 keeps degenerate entries (per-state weights equal to that
// relative tolerance) on the same side of the cut; owner, order (n ints), kept (nsec
// ints), stats (6 doubles) and vals (2n doubles, scratch) are device buffers of the
// caller.
void launch_truncate(const TruncSector* secs, int nsec, const int* offs, int n, double eps, long long chi_max,
                     double degen, int* owner, int* order, int* kept, double* stats, double* vals, cudaStream_t s);
// one simultaneous-rotation step of the mixed split's Gram finish over n column sets
// (GramTask; reads the upper triangle of C, writes X^T = Z^T - I; flags: [0] not
// converged, [1] fall back to the sequential Jacobi, [2] largest relative coupling
// above tol_flag as float bits)
void launch_gram_rot(const GramTask* tasks, int n, int qmax, double tol, double tol_flag, double abs_flag,
                     double tmax, int* flags, cudaStream_t s);
// the most columns a column set of the Gram finish may have (its staging in shared memory)
int gram_qmax();
// g += d elementwise over n complex values
void launch_add_inplace(cplx* g, const cplx* d, long long n, cudaStream_t s);
// column norms of G as singular values, sorted descending with perm (SvdTask layout)
void launch_svd_finish(const SvdTask* tasks, int n, int qmax, cudaStream_t s);
void launch_wdot(const DotTask* tasks, int ntasks, double* partial, double* out, int nslots, cudaStream_t s);
void launch_entropy(const TruncSector* secs, int nsec, double* out, cudaStream_t s);
void launch_entropy_sv(const TruncSector* secs, int nsec, const double* g, double* out, cudaStream_t s);
void launch_fill_normal(cplx* p, long long n, unsigned long long seed, long long offset, cudaStream_t s);

}  // namespace tdvp
