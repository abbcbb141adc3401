/*
 * tdvp.h -- C ABI of the B300 two-site TDVP engine for the open Fermi-Hubbard chain.
 *
 * The engine evolves a matrix product state (Eq. MPS, Sec. S2.2) of the open
 * chain H = -J sum_{i,s} (c^dag_{i s} c_{i+1 s} + h.c.) + U sum_i n_{i up} n_{i dn}
 * (Eq. FHM, Sec. 2) from the half-filled Neel state (Eq. neel, Sec. 2.1) with
 * second-order two-site TDVP (Sec. S2.2), Krylov exponentials, per-sector SVD
 * truncation on the truncated weight (Sec. S2.4), and U(1)xU(1) or U(1)xSU(2)
 * block sparsity (Sec. S2.1, Eq. symdecomp).  All device work runs in this
 * library's own kernels on one GPU; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - Return value: 0 on success, a negative TDVP_E* code on failure; no C++
 *     exception crosses this boundary.  tdvp_strerror() names a code and
 *     tdvp_last_error() gives the message of the last failure on this thread.
 *   - Complex numbers are interleaved FP64 pairs (re, im).
 *   - The caller owns every array it passes in; the library owns the context
 *     and every device buffer it allocates.  Calls on one context must be
 *     serialised by the caller; several contexts may share a GPU.
 *   - Sites are 0-indexed; site 0 starts with spin up (sublattice A = even).
 *   - Internally the engine works in the particle-hole frame
 *     c_{i dn} -> (-1)^i c^dag_{i dn}, where the charge SU(2) of Sec. S2.1 is the
 *     ordinary spin SU(2).  Observables returned by tdvp_measure are converted
 *     back to the frame of Eq. (FHM).  Block labels (n, t) exposed by the
 *     block-query functions are in the engine frame: n = particle number to the
 *     left of a bond, t = 2S (U1SU2) or 2S^z (U1U1).
 */
#ifndef TDVP_H_
#define TDVP_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdvp_ctx tdvp_ctx; /* opaque; owns all device state */

enum { TDVP_SYM_U1U1 = 0, TDVP_SYM_U1SU2 = 1 };
/* Precision of the block GEMMs (Lanczos, SVD, truncation and the recoupling
 * coefficients stay FP64 in every mode).
 *   FP64   : CUDA-core FP64.
 *   3XTF32 : tensor cores, x = h + l in TF32, products hh + hl + lh, FP32
 *            accumulation (relative error ~1e-6 on long sums).
 *   BF16X4 : tensor cores, every row of A / column of B scaled by a power of two
 *            and every value cut into four signed 8-bit digits (exact BF16 values);
 *            the digit products of each order are summed exactly in FP32 and
 *            recombined in 64-bit integers (relative error ~1e-9 of the row and
 *            column scales). */
enum { TDVP_PREC_FP64 = 0, TDVP_PREC_3XTF32 = 1, TDVP_PREC_BF16X4 = 2 };

enum {
  TDVP_OK = 0,
  TDVP_EINVAL = -1,   /* invalid argument (L<2, chi_max<1, dt<=0, eps<0, bad sizes) */
  TDVP_ESTATE = -2,   /* call not valid for this context */
  TDVP_ENOMEM = -3,   /* device or host allocation failed */
  TDVP_ENUMERIC = -4, /* an iteration did not converge or produced NaN */
  TDVP_EINTERNAL = -5,/* inconsistent internal bookkeeping */
  TDVP_ECUDA = -6,    /* a CUDA runtime call failed (including "no device") */
  TDVP_ETIMEOUT = -7, /* a bounded device wait gave up (or tdvp_server_wait ran out) */
  TDVP_ECANCELED = -8,/* a served request was cancelled */
  TDVP_EIO = -9       /* a checkpoint file could not be opened, written or renamed */
};

typedef struct {
  int precision;     /* TDVP_PREC_*; default FP64 */
  int krylov_max;    /* maximal Krylov dimension, 1..32; default 20 */
  double krylov_tol; /* stop when beta_k |[exp(-i tau T_k)]_{k,1}| < tol; default 1e-12;
                        0 = always krylov_max matvecs (fixed dimension) */
  int timeout_ms;    /* reserved for bounded device waits; 0 = default */
  void* cuda_stream; /* cudaStream_t to run on, or NULL for an engine-owned stream */
  int device;        /* CUDA device ordinal, or -1 for the current device */
  double trunc_degeneracy; /* truncation (Sec. S2.4): the cut never separates two multiplets
                              whose per-state weights s^2 agree to this relative tolerance
                              (degenerate multiplets are kept or dropped together; see
                              tdvp_truncate); 0 = off; default 1e-8 */
  int merge_launches;      /* != 0: this context's BF16x4 block GEMMs go out in launches
                              shared with the other merging contexts on the device that
                              launch at the same moment (several served requests' H_eff
                              stages in one grouped launch); results are unchanged, bit for
                              bit; default 0 */
} tdvp_opts;

/* Environment: when every sector of a split has at most 32 columns and a working
 * copy within TDVP_JACOBI_RESIDENT_BYTES (read at every split; default and maximum
 * 196608 bytes), each sector's Jacobi runs inside one CTA's shared memory.
 * Otherwise each sector with at most 320 rows runs on a ring of warps in one
 * thread-block cluster (TDVP_JACOBI_RING=0 turns this form off), and the rest share
 * the cooperative grid-wide kernel (TDVP_JACOBI_RESIDENT_BYTES=0 skips the first
 * form).  With TDVP_JACOBI_CLUSTER=1, splits whose sectors each fit in the shared
 * memory of a cluster of at most 8 CTAs run one cluster per sector with the columns
 * stationary in distributed shared memory (off by default: slower on the measured
 * workloads).  All forms give the same result, bit for bit.
 * TDVP_JACOBI_CTAS_PER_SM (1..8, default 4, read at every launch) sets the CTAs
 * per SM of the cooperative Jacobi grid (bounded by its occupancy); results do
 * not depend on it.
 *
 * Device memory: contexts allocate from the current device's default memory pool
 * (cudaMallocAsync on their stream).  The first context created on a device in a
 * process raises that pool's release threshold to TDVP_POOL_KEEP_MB megabytes
 * (default 4096; a higher threshold already set is kept), so that memory freed
 * between two synchronisations is reused instead of being returned and mapped
 * again.  That much freed memory may stay reserved by the process. */

/* Fill *o with the defaults listed above. */
void tdvp_opts_default(tdvp_opts* o);

/* Create a chain of L sites (L >= 2, even for the Neel state at half filling)
 * with hopping J and interaction U, symmetry TDVP_SYM_*, in the Neel state of
 * Eq. (neel) (bond dimension 1).  opts may be NULL for the defaults.
 * Errors: TDVP_EINVAL, TDVP_ENOMEM, TDVP_ECUDA. */
int tdvp_create(int L, double J, double U, int symmetry, const tdvp_opts* opts, tdvp_ctx** out);

/* A chain in a Fock product state instead of the Neel state: occ[i] (i = 0..L-1)
 * is 0 (empty), 1 (up), 2 (down) or 3 (up and down) in the frame of Eq. (FHM).
 * Used for the benchmark's second initial state (Sec. S1: the Neel pattern with a
 * single central vacancy, L odd).  Any L >= 2 and any occupations with
 * TDVP_SYM_U1U1.  TDVP_SYM_U1SU2 accepts only states whose sites are all singly
 * occupied (the engine's particle-hole frame then holds a spin singlet, the sector
 * its U(1)xSU(2) measurement assumes); others give TDVP_EINVAL.  The energy that
 * tdvp_measure reports is that of Eq. (FHM) for any filling.  Errors: TDVP_EINVAL,
 * TDVP_ENOMEM, TDVP_ECUDA. */
int tdvp_create_product(int L, double J, double U, int symmetry, const int* occ, const tdvp_opts* opts,
                        tdvp_ctx** out);

/* Create a chain in a synthetic random state for benchmarking: a right-canonical
 * MPS of L sites (half filling, total spin singlet in the engine frame) whose
 * bond k holds the multiplets (n, t) of k sites that can couple to the total
 * state, with degeneracy min(round(D0 exp(-Q^2/18 - S^2/4.5)), exact multiplet
 * counts of the left and right parts), Q = n - k, S = t/2, D0 chosen so the middle
 * bond reaches chi_target (U(1)-equivalent); block entries are counter-based
 * normal numbers from seed; sites left of `center` are left-orthonormalised,
 * sites right of it right-orthonormalised, the centre is normalised, and the
 * environments on both sides are built.  The state has the
 * benchmark's block structure but no physical meaning.  Errors: TDVP_EINVAL,
 * TDVP_ENOMEM, TDVP_ECUDA. */
int tdvp_create_random(int L, double J, double U, int symmetry, long long chi_target, unsigned long long seed,
                       int center, const tdvp_opts* opts, tdvp_ctx** out);

/* One second-order two-site TDVP time step dt (Sec. S2.2): a left-to-right and a
 * right-to-left half sweep with tau = dt/2.  After each two-site SVD the kept
 * multiplets are the largest singular values (ties broken by sector, then
 * index) such that the discarded weight sum s^2 stays <= eps_trunc * sum s^2
 * and the U(1)-equivalent bond dimension sum d(2S+1) stays <= chi_max
 * (Sec. S2.4); at least one multiplet is kept and the kept values are
 * renormalised to unit norm.  Errors: TDVP_EINVAL (dt<=0, chi_max<1, eps<0),
 * TDVP_ENUMERIC, TDVP_ECUDA, TDVP_ENOMEM. */
int tdvp_step(tdvp_ctx* ctx, double dt, long long chi_max, double eps_trunc);

/* Integrator of tdvp_step_mode. */
enum { TDVP_SWEEP_TWO_SITE = 0, TDVP_SWEEP_ONE_SITE = 1, TDVP_SWEEP_ADAPTIVE = 2 };

/* One time step dt with the chosen integrator (Sec. S2.2).
 *   TDVP_SWEEP_TWO_SITE: exactly tdvp_step.
 *   TDVP_SWEEP_ONE_SITE: the second-order one-site sweep: left to right with
 *     tau = dt/2 every site is evolved forward with the one-site H_eff, split as
 *     M = A C (repeated Cholesky QR in FP64), C is evolved backward with the
 *     zero-site H_eff and absorbed into the next site; right to left mirrors it
 *     with M = C Q.  Bond dimensions never change; chi_max and eps_trunc are not
 *     used; energy and norm are conserved up to the Krylov tolerance.
 *   TDVP_SWEEP_ADAPTIVE: two-site steps until a step in which the chi_max cap
 *     (rather than the discarded-weight rule) set the kept set at some bond; from
 *     then on one-site steps ("switch once the bond dimension has saturated").
 * used (nullable) receives the integrator this step used (0 or 1).  The centre
 * must be on site 0 (it is again afterwards).  Errors: as tdvp_step; a
 * non-positive Cholesky pivot (rank-deficient site tensor) gives TDVP_ENUMERIC. */
int tdvp_step_mode(tdvp_ctx* ctx, double dt, long long chi_max, double eps_trunc, int mode, int* used);

/* One two-site update of the sweep (Sec. S2.2) at bond (bond, bond+1), the unit
 * the full step repeats L-1 times per half sweep: theta formation, the Krylov
 * exponential exp(-i dt/2 H_eff), the per-sector SVD with truncation (same rule
 * as tdvp_step), the environment update, and the backward one-site evolution of
 * the new centre by +dt/2.  direction 0: left to right, the orthogonality
 * centre must be on site `bond` and moves to bond+1; direction 1: right to left,
 * centre on bond+1, moves to `bond`.  *s_ent (nullable) receives the von Neumann
 * entropy of the new bond from the kept singular values.  Errors: TDVP_EINVAL,
 * TDVP_ESTATE (centre elsewhere), TDVP_ENUMERIC, TDVP_ECUDA. */
int tdvp_bond_update(tdvp_ctx* ctx, int bond, int direction, double dt, long long chi_max, double eps_trunc,
                     double* s_ent);

/* <n_i>, <S^z_i>, <n_{i up} n_{i dn}> of the orthogonality-centre site i (*site),
 * in the frame of Eq. (FHM).  Any output may be NULL. */
int tdvp_measure_center(tdvp_ctx* ctx, int* site, double* n, double* sz, double* docc);

/* Observables of the current state (Sec. 3, Figs. 1-2 use n_{i up}); needs the
 * orthogonality centre on site 0 (as after tdvp_create or tdvp_step):
 *   n[L]     <n_i>            sz[L]   <S^z_i> = (<n_{i up}> - <n_{i dn}>)/2
 *   docc[L]  <n_{i up} n_{i dn}>
 *   s_ent[L-1] von Neumann entropy (natural log) of the cut after site k
 *   energy   <H> in the convention of Eq. (FHM)
 * Any pointer may be NULL to skip that output (s_ent is the expensive one).
 * n_{i up} = n_i/2 + S^z_i and n_{i dn} = n_i/2 - S^z_i.  Host pointers. */
int tdvp_measure(tdvp_ctx* ctx, double* n, double* sz, double* docc, double* s_ent, double* energy);

/* Bond dimensions of the L+1 bonds: chi[k] = sum d(2S+1) (U(1)-equivalent) and
 * chi_red[k] = sum d (reduced); either may be NULL. */
int tdvp_bond_dims(tdvp_ctx* ctx, long long* chi, long long* chi_red);

/* Counters since creation: out[0] seconds in tdvp_step, out[1] effective
 * Hamiltonian flops (algorithmic, 8 per complex multiply-add), out[2]
 * environment-update flops, out[3] matvecs, out[4] largest Krylov dimension
 * used, out[5] largest discarded weight, out[6] largest chi seen, out[7..12]
 * wall seconds per phase (theta formation, planning, two-site Krylov, SVD split,
 * environment update, one-site Krylov; filled only when the environment variable
 * TDVP_PROFILE_PHASES=1 was set at creation, which synchronises at phase
 * boundaries), out[13] number of steps, out[14] number of SVD splits, out[15]
 * FP64 Jacobi sweeps summed over the splits (counting the final sweep that found
 * nothing left to rotate), out[16] FP32 preconditioner sweeps (split-precision
 * modes), out[17] one-site steps.  In one-site steps the phase timers hold:
 * out[9] forward one-site Krylov, out[10] gauge shift, out[11] environment update,
 * out[12] zero-site Krylov and absorption.  out[18] device bytes the context
 * holds now and out[19] the most it has held (the buffers of the context's own
 * tensors, plans and workspaces; the few-KB scratch of single launches is not
 * counted).  out[20] milliseconds and out[21] algorithmic flops of the FP32
 * Jacobi launches of the splits, out[22], out[23] the same for the FP64 Jacobi
 * launches (CUDA events around each cooperative launch; flops = over the
 * sectors, sweeps in which the sector was still rotating x q(q-1)/2 column pairs
 * x (48 p + 32 q when the right vectors are accumulated, else 48 p) for a p x q
 * sector, p >= q).  out[24] largest P = max(p, q) and out[25] largest
 * Q = min(p, q) of a sector in the split-precision splits, out[26] the sum of
 * P Q^2 over those sectors and out[27] the same sum over the sectors whose
 * complex64 copy fits in 192 KiB.  out[28] Jacobi calls of the splits and
 * out[29] those that ran CTA-resident, out[30] those that ran in thread-block
 * clusters.  out[31] milliseconds of the environment updates of the two-site
 * bond updates (CUDA events around each update) and out[32] their algorithmic
 * bytes (every operand block read once and every result block written once, over
 * the block-GEMM and MPO linear-combination stages).  out[33] milliseconds and
 * out[34] algorithmic flops (16 p q^2 per sector and step) of the Gram finish of the
 * split-precision splits, out[35] its steps and out[36] the splits it handed to the
 * FP64 Jacobi.  out[37] Jacobi calls of the splits that ran as rings of warps in
 * thread-block clusters.  n = length of out (at most 38). */
int tdvp_stats(tdvp_ctx* ctx, double* out, int n);

/* ---- single-bond problems (the effective-Hamiltonian benchmark) ------------
 * tdvp_bond_create builds the two-site problem between a left bond and a right
 * bond given as sector tables: nl (resp. nr) rows of int triples (n, t, d),
 * n the particle number to the left of the bond, t = 2S (U1SU2) or 2S^z
 * (U1U1), d >= 1 the degeneracy.  The two sites in between are bulk sites of
 * Eq. (FHM) with the MPO channels
 *   [B, c^dag(+1/2), c^dag(-1/2), c(+1/2), c(-1/2), E]
 * (U1SU2: B (0,0), c^dag (+1, 2S=1), c (-1, 2S=1), E (0,0); U1U1: six singlets).
 * The left environment L[a',w,a] and the right environment R[b,w,b'] start at
 * zero; fill them with tdvp_set_tensor.  Errors: TDVP_EINVAL, TDVP_ENOMEM,
 * TDVP_ECUDA. */
int tdvp_bond_create(int symmetry, double J, double U, int nl, const int* left, int nr, const int* right,
                     const tdvp_opts* opts, tdvp_ctx** out);

/* which: 0 = two-site tensor theta, 1 = left environment, 2 = right environment
 * (a bond-problem context), 3 = theta of bond (0,1) of a chain context.
 * Number of blocks and total complex elements. */
int tdvp_block_count(tdvp_ctx* ctx, int which, long long* nblocks, long long* nelems);

/* Block list in storage order.  keys[5*i..]: theta (a, s1, t_c, s2, b) with a, b
 * sector indices, s1, s2 site-multiplet indices and t_c the spin label of the
 * coupled (a s1) channel; environments (a', w, a, 0, 0) / (b, w, b', 0, 0) with w
 * a channel-multiplet index.  dims[2*i..] = (rows, cols); offsets[i] = first
 * complex element; each block is row-major rows x cols.  Any pointer may be NULL. */
int tdvp_block_list(tdvp_ctx* ctx, int which, int* keys, int* dims, long long* offsets);

/* Copy n complex elements (interleaved FP64) into the left (which=1) or right
 * (which=2) environment of a bond problem; on_device != 0 means data is a device
 * pointer.  n must equal the tensor size.  Errors: TDVP_EINVAL, TDVP_ESTATE. */
int tdvp_set_tensor(tdvp_ctx* ctx, int which, const double* data, long long n, int on_device);

/* psi_out = H_eff psi_in for the two-site effective Hamiltonian of Sec. S2.3:
 *   psi'[a',s1',s2',b'] = sum L[a',w,a] W[w,w1,s1',s1] W[w1,w2,s2',s2] R[b,w2,b'] psi[a,s1,s2,b]
 * in the reduced block layout of which = 0 (bond problem) or 3 (chain bond
 * (0,1), valid right after tdvp_create or tdvp_step).  bond must be 0.
 * psi_in and psi_out hold tdvp_block_count elements; on_device != 0 means both
 * are device pointers (no copies), otherwise host pointers (copied in and out).
 * The call is stream-ordered on the context's stream and returns after the
 * result is complete.  Errors: TDVP_EINVAL, TDVP_ESTATE, TDVP_ECUDA. */
int tdvp_heff_apply(tdvp_ctx* ctx, int bond, const double* psi_in, double* psi_out, int on_device);

/* ---- one H_eff.psi over several GPUs (Sec. S2.3, "GPU acceleration": the
 * block products are spread over the GPUs with greedy load balancing) ---------
 * The last GEMM stage of the product writes each output block from one task; the
 * tasks (output groups) are the units that ranks share out.  Each rank computes the
 * first stages in full and the output groups it owns (tdvp_heff_apply_owned); the
 * ranks then exchange their output blocks (an all-gather), and every rank holds
 * the whole psi_out for its replicated Lanczos recurrence.  The partition and the
 * exchange are in the Python binding (paper_2606_04771_b300/shard.py).
 *
 * tdvp_heff_groups: *ngroups receives the number of output groups of the context's
 * H_eff (which = 0 of a bond problem, or chain bond (0,1)); flops[g] (nullable,
 * ngroups entries) their algorithmic flops; block_group[b] (nullable, one entry per
 * block of the tdvp_block_list layout) the group that writes output block b.
 * Errors: TDVP_EINVAL, TDVP_ESTATE. */
int tdvp_heff_groups(tdvp_ctx* ctx, int* ngroups, long long* flops, int* block_group);

/* Greedy longest-processing-time partition of n units with costs cost[0..n) over
 * nranks ranks: units in descending cost (ties by index) each go to the rank with
 * the least load so far (ties to the lowest rank).  owner[i] receives the rank of
 * unit i; load (nullable, nranks entries) the summed cost per rank.  Host only (no
 * device is touched).  Errors: TDVP_EINVAL (n < 0, nranks < 1, NULL, cost < 0). */
int tdvp_partition(int n, const double* cost, int nranks, int* owner, double* load);

/* psi_out = H_eff psi_in restricted to the output groups g with group_owner[g] ==
 * rank: the blocks of the other groups in psi_out are left as they were.  Device
 * pointers only (on_device must be 1); layout and errors as tdvp_heff_apply. */
int tdvp_heff_apply_owned(tdvp_ctx* ctx, int bond, const int* group_owner, int rank, const double* psi_in,
                          double* psi_out, int on_device);

/* psi_out = exp(-i tau H_eff) psi_in with the engine's Krylov exponential
 * (Sec. S2.2): Lanczos with full re-orthogonalisation applied twice, FP64
 * vectors, exp(-i tau T_k) e_1 from a scaled Taylor series on the GPU, stopped
 * adaptively by the estimate beta_k |[exp(-i tau T_k)]_{k,1}| < krylov_tol or at
 * krylov_max.  Same layout, bond and pointer rules as tdvp_heff_apply;
 * *krylov_dim (nullable) receives the number of matvecs used and *launches
 * (nullable) the number of kernel launches.  Errors: TDVP_EINVAL, TDVP_ESTATE,
 * TDVP_ENUMERIC (non-finite recurrence), TDVP_ECUDA. */
int tdvp_krylov_expm(tdvp_ctx* ctx, int bond, const double* psi_in, double* psi_out, double tau, int on_device,
                     int* krylov_dim, int* launches);

/* Algorithmic flops of one tdvp_heff_apply (8 per complex multiply-add of the
 * two block-GEMM stages). */
int tdvp_heff_flops(tdvp_ctx* ctx, long long* flops);

/* Time the three stages of tdvp_heff_apply on the context's stream with CUDA
 * events: stage 0 = environment x theta block GEMMs, 1 = MPO linear
 * combination, 2 = second block GEMM stage.  Runs iters applications on
 * internal buffers; ms[s] = average milliseconds per application of stage s,
 * flops[s] = algorithmic flops per application (8 per complex multiply-add;
 * 0 for stage 1), bytes[s] = algorithmic bytes per application (operands read
 * once, results written once).  Any output pointer may be NULL. */
int tdvp_heff_profile(tdvp_ctx* ctx, int iters, double* ms, long long* flops, long long* bytes);

/* Thin SVD of one complex p x q matrix, A = U diag(s) V^H, with the engine's
 * one-sided Jacobi kernel in FP64 (the per-sector SVD of Sec. S2.2/S2.4).
 * a: p x q row-major; s: min(p,q) values in descending order; u: p x r
 * row-major; vh: r x q row-major, r = min(p,q).  Columns of u (rows of vh)
 * that belong to a zero singular value are returned as zero.  on_device != 0:
 * all four pointers are device pointers, otherwise host pointers.  stream is a
 * cudaStream_t or NULL (the legacy default stream); the call returns after the
 * result is complete.  Workspace is allocated and freed on that stream.
 * Errors: TDVP_EINVAL (p<1, q<1, NULL), TDVP_ENUMERIC (no convergence),
 * TDVP_ENOMEM, TDVP_ECUDA. */
int tdvp_svd(int p, int q, const double* a, double* s, double* u, double* vh, int on_device, void* stream);

/* The truncation's multiplet selection on its own (Sec. S2.4, Sec. S2.1): the
 * step that tdvp_step runs after every two-site SVD, exposed so that callers can
 * check it against a restatement of the rule.  Sector k (k = 0..nsec-1) holds
 * r[k] >= 0 reduced singular values in descending order, stored back to back in
 * sv (sector 0 first, sum r[k] >= 1 values), each the value of one multiplet of
 * mult[k] = 2S+1 states (1 without SU(2)), normalised so that sv^2 is the weight
 * of the whole multiplet (mult[k] s^2 for the singular value s of each of its
 * states).  The rule:
 *   - order all multiplets by the per-state weight sv^2 / mult, descending; ties
 *     go to the lower sector index, then the lower index within the sector;
 *   - K_eps = the smallest K >= 1 such that the weights of the multiplets ranked
 *     K, K+1, ... sum to at most eps times the total weight (whole multiplets
 *     are kept or dropped);
 *   - K_chi = the largest K >= 1 whose first K multiplets hold at most chi_max
 *     states (sum of mult), or 1 if the first alone holds more;
 *   - the first K = min(K_eps, K_chi) ranked multiplets are kept;
 *   - with degeneracy > 0, a head may not end between two ranked multiplets whose
 *     per-state weights a >= b satisfy a - b <= degeneracy * a: K_eps and K_chi
 *     are taken over the allowed heads only (K = all multiplets is always
 *     allowed), and when no allowed head fits under the cap, K_chi is the first
 *     allowed head (tdvp_step uses tdvp_opts.trunc_degeneracy here).
 * kept[k] receives the number of sector k's values kept (always a prefix of the
 * sector).  stats (nullable, 6 doubles): total weight, discarded weight,
 * 1/sqrt(kept weight) (the renormalisation factor of the kept values), K, the
 * states kept (sum of mult), and 1.0 when K_chi < K_eps (the cap set K) else 0.
 * Host pointers; NaN or negative values rank last with weight 0.  stream is a
 * cudaStream_t or NULL; the call returns when the result is on the host.
 * Errors: TDVP_EINVAL (nsec < 1, NULL, r[k] < 0, mult[k] < 1, no values, eps < 0,
 * chi_max < 1, degeneracy < 0), TDVP_ENOMEM, TDVP_ECUDA. */
int tdvp_truncate(int nsec, const int* r, const int* mult, const double* sv, double eps, long long chi_max,
                  double degeneracy, int* kept, double* stats, void* stream);

/* Largest p or q accepted by tdvp_svd_noalloc. */
#define TDVP_SVD_NOALLOC_MAX 512

/* tdvp_svd without any device allocation at call time (the paper has no
 * counterpart; this is a service for callers of this library).  It is meant for
 * callers that must not allocate device memory while they run: a serving
 * process whose own pool already holds nearly all of the GPU's memory (where
 * cudaMalloc would fail, or would stall the device's streams while it runs), or
 * code under a memory budget frozen after start-up.  The caller passes DEVICE
 * pointers for a (p x q row-major), s, u and vh exactly as for tdvp_svd; all
 * workspace lives in one static device array inside this library (about 8 MiB),
 * which every GPU that loads the library holds until the process exits.
 *   - max(p, q) must be <= TDVP_SVD_NOALLOC_MAX, otherwise TDVP_EINVAL.
 *   - The first call on a device (with that device current) performs a one-time
 *     set-up (it looks up the workspace's device address).
 *   - No call may be made while a stream is capturing: every call copies its
 *     work lists from host memory and synchronises its stream before returning.
 *   - Every call uses the same workspace, which keeps the last call's contents
 *     (each call rewrites what it reads and clears its convergence flag).  Calls
 *     that overlap on the GPU race on the workspace: serialise them.
 * stream is a cudaStream_t or NULL; the call returns after the result is
 * complete.  Errors: TDVP_EINVAL, TDVP_ENUMERIC, TDVP_ECUDA. */
int tdvp_svd_noalloc(int p, int q, const double* a, double* s, double* u, double* vh, void* stream);

/* Merged launches so far in the process (tdvp_opts.merge_launches): *launches
 * receives the number of BF16x4 GEMM launches that carried more than one context's
 * work, *slices the number of task lists they carried.  Either may be NULL (not
 * both).  Errors: TDVP_EINVAL. */
int tdvp_merge_count(long long* launches, long long* slices);

/* Number of kernel launches this library has made in the process so far, over
 * every context and entry point (each launch site counts itself on the host
 * when it enqueues the kernel).  out must be non-NULL.  Errors: TDVP_EINVAL. */
int tdvp_launch_count(long long* out);

/* Self-test of failure detection: a kernel waits on an mbarrier that nothing
 * arrives at, gives up after `polls` polls (the same bounded wait the GEMM
 * pipelines use, which there runs 2^24 polls) and reports the expiry.  Returns
 * TDVP_ETIMEOUT when the wait expired -- the expected outcome -- after which the
 * CUDA context stays usable; TDVP_ECUDA on a CUDA error.  stream: cudaStream_t or
 * NULL. */
int tdvp_selftest_wait(unsigned int polls, void* stream);

/* ---- serving: independent quench requests on one GPU ---------------------
 * A server runs up to max_active requests at once, each on its own worker
 * thread and CUDA stream with its own context (MPS, environments, plans and
 * workspaces resident on the device for the whole run), so the kernels of
 * different requests overlap on the device.  Admission is first in, first out:
 * the oldest queued request starts when a worker is free, its footprint estimate
 * (tdvp_server_footprint) fits beside those of the running requests within
 * hbm_budget_bytes, and the device reports at least that much free memory; a
 * request whose estimate alone exceeds the budget runs when nothing else does.
 * A finished request frees its worker and its share of the budget at once and
 * the next one is admitted while the others keep running.  A request is
 * round(t_final / dt) steps of tdvp_step_mode(dt, chi_max, eps, mode) from the
 * Neel state (Eq. neel) or from the product state `occupations` (as in
 * tdvp_create_product), then one tdvp_measure.  Requests share no state and
 * every kernel is deterministic: a result is the same alone and beside others.
 * Calls on one server may come from any threads; tdvp_server_destroy must not
 * overlap other calls on the same server. */
typedef struct tdvp_server tdvp_server;

typedef struct {
  int L;                  /* sites, >= 2 */
  double J, U;            /* hopping and interaction of Eq. (FHM) */
  int symmetry;           /* TDVP_SYM_* */
  int precision;          /* TDVP_PREC_* of this request's contractions */
  int mode;               /* TDVP_SWEEP_* */
  double dt, t_final;     /* dt > 0, t_final >= 0 */
  long long chi_max;      /* U(1)-equivalent bond dimension cap, >= 1 */
  double eps;             /* truncation threshold, >= 0 (Sec. S2.4) */
  const int* occupations; /* [L] in {0,1,2,3} (empty, up, down, both), or NULL for
                             the Neel state; copied at submission */
} tdvp_request;

enum { TDVP_REQ_QUEUED = 0, TDVP_REQ_RUNNING = 1, TDVP_REQ_DONE = 2, TDVP_REQ_FAILED = 3, TDVP_REQ_CANCELLED = 4 };

/* Start a server: hbm_budget_bytes > 0, 1 <= max_active <= 256.  opts gives the
 * Krylov settings and the device (its precision and stream are ignored: each
 * request names its precision and each worker owns a stream); NULL = defaults.
 * No device work happens until the first request is admitted.  Errors:
 * TDVP_EINVAL, TDVP_ENOMEM, TDVP_EINTERNAL. */
int tdvp_server_create(double hbm_budget_bytes, int max_active, const tdvp_opts* opts, tdvp_server** out);

/* The admission estimate of a request, in bytes, for Krylov dimension krylov_max
 * (<= 0: 20): 16 chi_max^2 (2 L + 2.5 (krylov_max + 8)) + 64e6, a bound with a
 * factor of two to spare on the device bytes measured for Neel quenches whose
 * largest bond reached chi_max.  Errors: TDVP_EINVAL. */
int tdvp_server_footprint(const tdvp_request* req, int krylov_max, double* bytes);

/* Queue a request (copied, occupations included); *id receives its id (> 0).
 * Errors: TDVP_EINVAL (see tdvp_request), TDVP_ESTATE (shutting down). */
int tdvp_server_submit(tdvp_server* s, const tdvp_request* req, long long* id);

/* Current state of a request (TDVP_REQ_*).  Errors: TDVP_EINVAL (unknown id). */
int tdvp_server_poll(tdvp_server* s, long long id, int* state);

/* Block until the request has ended (DONE, FAILED or CANCELLED) or timeout_ms
 * has passed (< 0: no limit).  Returns TDVP_OK when it ended (its state in
 * *state, which may be NULL), TDVP_ETIMEOUT otherwise, TDVP_EINVAL for an
 * unknown id. */
int tdvp_server_wait(tdvp_server* s, long long id, int timeout_ms, int* state);

/* Results of an ended request: n, sz, docc [L] and s_ent [L-1] as tdvp_measure
 * (each may be NULL), and info[0..ninfo) with info[0] energy, [1] largest bond
 * dimension reached, [2] steps done, [3] effective-Hamiltonian flops, [4] submit,
 * [5] admission and [6] end time (seconds since the server started), [7] peak
 * device bytes of its context, [8] its footprint estimate, [9] its status code.
 * info is filled in every state.  Returns TDVP_OK for a DONE request, the
 * request's own error code for a FAILED or CANCELLED one (message in
 * tdvp_last_error), TDVP_ESTATE while it is queued or running, TDVP_EINVAL for
 * an unknown id. */
int tdvp_server_result(tdvp_server* s, long long id, double* n, double* sz, double* docc, double* s_ent,
                       double* info, int ninfo);

/* Cancel a request: a queued one ends at once, a running one at its next step
 * boundary (state CANCELLED, code TDVP_ECANCELED); an ended one is left as is.
 * Errors: TDVP_EINVAL (unknown id). */
int tdvp_server_cancel(tdvp_server* s, long long id);

/* Stop (paused != 0) or resume admission; running requests continue. */
int tdvp_server_pause(tdvp_server* s, int paused);

/* Counters: out[0] submitted, [1] done, [2] failed, [3] cancelled, [4] queued,
 * [5] running, [6] p50 and [7] p99 latency in seconds (submission to end, over
 * the DONE requests, linear between closest ranks), [8] seconds since the server
 * started, [9] most requests running at once, [10] most bytes of estimates
 * admitted at once, [11] steps and [12] effective-Hamiltonian flops of the DONE
 * requests.  n = length of out (at most 13). */
int tdvp_server_stats(tdvp_server* s, double* out, int n);

/* Cancel the queued requests, let the running ones stop at their next step
 * boundary, join the workers and free the server.  NULL is accepted. */
int tdvp_server_destroy(tdvp_server* s);

/* ---- checkpoint / resume --------------------------------------------------
 * tdvp_save writes a chain context's state to `path`: the bond sector tables,
 * the site tensors (complex128), the orthogonality centre and the adaptive
 * switch's state, with the caller's time t.  It writes `path`.part and renames
 * it, so an interrupted save leaves any older file intact.  tdvp_load creates a
 * context from such a file (opts as in tdvp_create: the precision and stream of
 * the resumed run) and rebuilds the environments from the sites with the same
 * kernels in the same order, so an FP64 run resumed from a checkpoint repeats
 * the uninterrupted run bit for bit; *t (nullable) receives the stored time.
 * The file is read and checked completely before any device work.  Format
 * (little-endian): "TDVPCKP1"; int32 version (1), L, su2, centre, cap_hit,
 * saturated; float64 J, U, t; per bond k = 0..L an int32 count and count int32
 * triples (n, t, d); per site an int64 element count and the elements;
 * "TDVPEND1".  Errors: TDVP_EINVAL (NULL argument, not a checkpoint, truncated or
 * inconsistent file), TDVP_ESTATE (a bond-problem context), TDVP_EIO (file
 * could not be opened, written or renamed), TDVP_ENOMEM, TDVP_ECUDA. */
int tdvp_save(tdvp_ctx* ctx, const char* path, double t);
int tdvp_load(const char* path, const tdvp_opts* opts, tdvp_ctx** out, double* t);

/* Destroy a context and free its device memory.  NULL is accepted. */
int tdvp_destroy(tdvp_ctx* ctx);

/* Static name of an error code. */
const char* tdvp_strerror(int code);

/* Message of the last failed call on this thread ("" if none). */
const char* tdvp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TDVP_H_ */
