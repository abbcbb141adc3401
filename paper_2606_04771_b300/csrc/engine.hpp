// Two-site TDVP engine on one GPU (host orchestration).
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.hpp"
#include "kernels.hpp"
#include "sym.hpp"

namespace tdvp {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define TDVP_CUDA(x)                                                                                 \
  do {                                                                                               \
    cudaError_t e_ = (x);                                                                            \
    if (e_ != cudaSuccess)                                                                           \
      throw ::tdvp::Error(e_ == cudaErrorMemoryAllocation ? -3 : -6,                                 \
                          std::string(#x) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

// stream-ordered device buffer
// Live and peak device bytes of one context.  Every DevBuf allocated while a
// context's accountant is current on the thread (DevAcctScope, set by the C entry
// points for the duration of a call) is charged to it until it is freed.
struct DevAcct {
  std::atomic<long long> live{0}, peak{0};
  void add(long long b) {
    const long long v = live.fetch_add(b) + b;
    long long p = peak.load();
    while (v > p && !peak.compare_exchange_weak(p, v)) {
    }
  }
};
DevAcct*& current_acct();  // thread-local
struct DevAcctScope {
  DevAcct* prev;
  explicit DevAcctScope(DevAcct* a) : prev(current_acct()) { current_acct() = a; }
  ~DevAcctScope() { current_acct() = prev; }
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  DevAcct* acct = nullptr;
  DevBuf() = default;
  DevBuf(size_t b, cudaStream_t st);
  ~DevBuf();
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
  DevBuf& operator=(DevBuf&& o) noexcept;
  void reset();
  template <class T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

enum Kind { SITE = 0, THETA = 1, LENV = 2, RENV = 3, OMEGA = 4 };

struct Block {
  int key[5];
  int rows, cols;
  long long off;  // complex elements
};

inline uint64_t bkey(int a, int b, int c, int d = 0, int e = 0) {
  return ((uint64_t)(a & 0xfff) << 52) | ((uint64_t)(b & 0xfff) << 40) | ((uint64_t)((c + 2048) & 0xfff) << 28) |
         ((uint64_t)(d & 0xfff) << 16) | ((uint64_t)(e & 0xffff));
}

struct BTensor {
  int kind = SITE;
  std::vector<Block> blocks;
  std::unordered_map<uint64_t, int> map;
  long long size = 0;
  DevBuf buf;
  int find(uint64_t k) const {
    auto it = map.find(k);
    return it == map.end() ? -1 : it->second;
  }
  void add(uint64_t k, int k0, int k1, int k2, int k3, int k4, int r, int c) {
    Block b{{k0, k1, k2, k3, k4}, r, c, size};
    map[k] = (int)blocks.size();
    blocks.push_back(b);
    size += (long long)r * c;
  }
  cplx* ptr(int bi) const { return buf.as<cplx>() + blocks[bi].off; }
  cplx* data() const { return buf.as<cplx>(); }
};

// BF16x4 packed task side: one source block of a task's A operand (rows x K) or B
// operand (K x cols) and where it sits in that operand (first row, first column)
struct PackedSrc {
  const cplx* src;
  int base;
  int rows, cols, ld, op;  // logical shape after op
  double alpha;            // A only
  int row0, col0;
};
// One packed task: its operands are dense record matrices assembled from source
// blocks (positions not covered by a source are zero); side static = every source
// of that side is unchanged between launches of the plan
struct PackedTask {
  std::vector<PackedSrc> a, b;
  bool a_static = false, b_static = false;
};

struct GemmPlan {
  std::vector<GemmTask> tasks;
  std::vector<GemmSeg> segs;
  std::vector<int3> tiles;
  DevBuf dt, ds, dti;
  // only the tiles on and above the diagonal (Hermitian products such as Gram matrices)
  bool upper_only = false;
  // FP64 plans may split large single-segment tiles along K (see finalize)
  bool ksplit = false;
  // BF16x4 packed plans: the operands are tile images (plan_packed)
  bool images_ = false;
  // FP64 plans: the K range of each tile (kbeg, kend, partial slot or -1, 0) when some
  // single-segment tiles are split along K to balance the SMs; the partial tiles
  // (64 x 64 each in dws) of a split output tile are summed in a fixed order by the
  // combine step (fix: task, tile row, tile column, first slot | chunk count << 20)
  std::vector<int4> kext, fix;
  DevBuf dkx, dfix, dws;
  // packed BF16x4 plans (one segment per task, operands assembled from blocks):
  // packed[i] describes task i; rowoffs holds the stacked-output row offsets that a
  // task with row_start[i] >= 0 reads from index row_start[i] on
  std::vector<PackedTask> packed;
  std::vector<long long> rowoffs, row_start;
  DevBuf drow;
  // output blocks (indices into the output tensor's block list) that each task
  // writes, and its algorithmic flops: the units a multi-GPU matvec distributes
  std::vector<std::vector<int>> out_blocks;
  std::vector<long long> task_flops;
  // BF16x4: distinct operands (static: split at the first launch; dynamic: every
  // launch), their split jobs, digit records, group maxima and exponents
  std::vector<DigitOp> dops_s, dops_d;
  std::vector<int2> djobs_s, djobs_d;
  DevBuf ddops_s, djb_s, ddops_d, djb_d, ddig, dtag, dexp;
  int ngrp = 0, ngrp_static = 0;
  mutable bool static_done = false;
  mutable unsigned epoch = 0;  // of the last digit split (exponent tags of older epochs read as empty)
  long long flops = 0;  // algorithmic real flops (8 per complex MAC)
  long long bytes = 0;  // algorithmic bytes: every operand block read once, output written once
  int kind = -1;        // -1 FP64 CUDA cores, 0 3xTF32, 1 BF16x3 tensor cores
  int* status = nullptr;
  // BF16x4 split of the dynamic operands: 0 two passes; 1 their exponent tags are set
  // by the kernel that produces them (the caller passes the epoch of begin_split);
  // 2 every dynamic operand holds whole scale lines (one fused kernel)
  int dyn_mode = 0;
  bool dyn_tags_external = false;  // set by the planner before finalize: mode 1
  void finalize(cudaStream_t s, int kind_ = -1, int* status_ = nullptr);
  void plan_digits(cudaStream_t s);
  void plan_packed(cudaStream_t s);
  // BF16x4: split the static operands if not done yet and return the epoch of the
  // next dynamic split (clearing the tags when the counter would wrap)
  unsigned begin_split(cudaStream_t s, const Bases4& B) const;
  // epoch: 0, or the value begin_split returned (dynamic tags raised by the producer);
  // tiles: a subset of the tile list (device array of n_tiles entries) or nullptr
  void launch(cudaStream_t s, const Bases4& B, unsigned epoch = 0, const int3* tiles_subset = nullptr,
              int n_subset = 0) const;
  unsigned* tags() const { return dtag.as<unsigned>(); }
};

struct LincombPlan {
  std::vector<LincombTask> tasks;
  std::vector<LincombTerm> terms;
  std::vector<int2> chunks;
  DevBuf dt, dm, dc;
  long long bytes = 0;  // algorithmic bytes moved
  void finalize(cudaStream_t s);
  void launch(cudaStream_t s, unsigned epoch = 0) const;
};

struct CopyPlan {
  std::vector<CopyTask> tasks;
  std::vector<int2> chunks;
  DevBuf dt, dc;
  void finalize(cudaStream_t s);
  void launch(cudaStream_t s) const;
};

// effective Hamiltonian (two-site or one-site): GEMM -> lincomb -> GEMM
struct HeffPlan {
  BTensor t1, t2;  // intermediates (own their buffers)
  GemmPlan g1, g3;
  LincombPlan lc;
  long long n = 0;  // vector length (complex); input is base 1, output base 2
  void apply(const cplx* in, cplx* out, cudaStream_t s) const;
  // the whole product except the last stage's tasks outside `owned` (task mask over
  // g3.tasks): the output blocks of those tasks are not written
  void apply_owned(const cplx* in, cplx* out, const std::vector<char>& owned, cudaStream_t s) const;
  long long flops() const { return g1.flops + g3.flops; }
};

struct Opts {
  int precision = 0;
  int krylov_max = 20;
  double krylov_tol = 1e-12;
  int timeout_ms = 0;
  cudaStream_t stream = nullptr;
  int device = -1;
  double trunc_degen = 1e-8;  // degenerate multiplets are cut together (relative, per-state weight)
  bool merge = false;         // BF16x4 GEMMs may merge with other contexts' launches
};

struct StepStats {
  double max_discarded = 0, seconds = 0, heff_seconds = 0;
  long long heff_flops = 0, env_flops = 0, matvecs = 0;
  int max_krylov = 0;
  long long chi_max_seen = 0;
  long long steps = 0;
  // wall seconds per phase when TDVP_PROFILE_PHASES=1: theta formation, planning,
  // two-site Krylov, SVD split, environment update, one-site Krylov
  double phase[6] = {0, 0, 0, 0, 0, 0};
  // Jacobi sweeps summed over the splits: FP64 (the FP64 split, or the FP64 finish
  // of the mixed split) and FP32 (the preconditioner of the mixed split)
  long long sweeps64 = 0, sweeps32 = 0, splits = 0;
  long long one_site_steps = 0;
  // the cooperative Jacobi launches of the splits (CUDA-event time and algorithmic
  // flops, as JacobiProfile): FP32 preconditioner and FP64 stage
  JacobiProfile jacobi32, jacobi64;
  // the Gram finish of the mixed split: device time and algorithmic flops (16 p q^2
  // per set and step: the Gram matrix and the rotation), steps, and the splits it
  // handed to the FP64 Jacobi
  JacobiProfile gram;
  long long gram_steps = 0, gram_fallbacks = 0;
  // sector shapes of the splits: largest P = max(p, q) and Q = min(p, q) seen, and the
  // one-sided Jacobi work sum P Q^2 over all sectors and over those whose complex64
  // copy (P Q x 8 bytes) fits in 192 KiB of shared memory
  long long split_pmax = 0, split_qmax = 0;
  double split_work = 0, split_work_small = 0;
  // environment updates of the two-site bond updates: device milliseconds (CUDA events
  // around each update) and algorithmic bytes (every operand block read once, every
  // result block written once, over the GEMM and linear-combination stages)
  double env_ms = 0, env_bytes = 0;
};

class Engine {
 public:
  Engine(int L, double J, double U, bool su2, const Opts& o);
  ~Engine();

  // chain evolution
  void step(double dt, long long chi_max, double eps);
  // one-site second-order step (bond dimensions fixed), Sec. S2.2
  void step1(double dt);
  // mode 0: two-site, 1: one-site, 2: adaptive (two-site until the chi cap binds in a
  // step's truncation, one-site from then on); returns the mode used (0 or 1)
  int step_mode(double dt, long long chi_max, double eps, int mode);
  // one bond update of the sweep at bond (i, i+1); direction 0: left to right (centre on i),
  // 1: right to left (centre on i+1); s_ent (nullable) receives the new bond's entropy
  void single_bond(int i, int direction, double dt, long long chi_max, double eps, double* s_ent);
  void measure_center(int* site, double* n, double* sz, double* docc);
  int center() const { return center_; }
  void measure(double* n, double* sz, double* docc, double* s_ent, double* energy, double* n_up = nullptr);
  const StepStats& stats() const { return stats_; }
  int L() const { return L_; }
  const BondSpace& bond(int k) const { return bonds_[k]; }
  const Model& model() const { return model_; }
  void check_status();  // throws if a kernel reported non-convergence or a wait timeout
  cudaStream_t stream() const { return stream_; }
  const Opts& opts() const { return opt_; }

  // synthetic single-bond problem (environments and theta given by the caller)
  // synthetic right-canonical random state of L sites with bond dimension about chi_target
  static Engine* random_state(int L, double J, double U, bool su2, long long chi_target, unsigned long long seed,
                              int center, const Opts& o);
  // a Fock product state, occ[i] in {0 empty, 1 up, 2 down, 3 both}
  static Engine* product_state(int L, double J, double U, bool su2, const std::vector<int>& occ, const Opts& o);
  static Engine* bond_problem(bool su2, double J, double U, const std::vector<Sector>& left,
                              const std::vector<Sector>& right, const Opts& o);
  // checkpoint: the chain's bond tables, site tensors, orthogonality centre and the
  // adaptive-switch state, with the caller's time t; load rebuilds the environments
  void save(const std::string& path, double t);
  static Engine* load(const std::string& path, const Opts& o, double* t);
  bool bond_only() const { return bond_only_; }
  BTensor& theta_layout() { return theta_; }
  BTensor& left_env_bp() { return Lenv_[0]; }
  BTensor& right_env_bp() { return Renv_[2]; }
  void heff_apply_bond(const cplx* in, cplx* out);  // device pointers, bond problem only
  HeffPlan& heff_plan_bond() { return *bp_heff_; }
  // the caller rewrote an environment: operands split once per plan are stale
  void environments_changed() {
    if (bp_heff_) bp_heff_->g1.static_done = bp_heff_->g3.static_done = false;
    chain_heff_.reset();
  }
  HeffPlan& chain_heff0();  // two-site H_eff at bond (0,1) of a chain (centre at site 0)
  // x <- exp(-i tau H) x; *k = matvecs used, *launches = kernel launches
  void krylov(HeffPlan& H, cplx* x, double tau, int* k, int* launches);

 private:
  Engine() = default;
  void init_common(bool su2, double J, double U, const Opts& o);
  void init_neel();
  void init_product(const std::vector<int>& occ);
  void build_site_layout(BTensor& t, const BondSpace& l, const BondSpace& r) const;
  void build_theta_layout(BTensor& t, const BondSpace& l, const BondSpace& r) const;
  void build_lenv_layout(BTensor& t, const BondSpace& bra, const BondSpace& ket) const;
  void build_renv_layout(BTensor& t, const BondSpace& ket, const BondSpace& bra) const;
  void alloc(BTensor& t, bool zero);
  void orthonormalize_rows(BTensor& T, const BondSpace& l, const BondSpace& r);
  // boundary environments, then L_1..L_centre and R_{L-1}..R_{centre+1} from the sites
  void build_environments();
  void orthonormalize_cols(BTensor& T, const BondSpace& l, const BondSpace& r);

  void plan_heff2(HeffPlan& p, const BTensor& Lenv, const BTensor& Renv, const BTensor& theta,
                  const BondSpace& bl, const BondSpace& br);
  void plan_heff2_packed(HeffPlan& p, const BTensor& Lenv, const BTensor& Renv, const BTensor& theta,
                         const BondSpace& bl, const BondSpace& br);
  void plan_heff1(HeffPlan& p, const BTensor& Lenv, const BTensor& Renv, const BTensor& M, const BondSpace& bl,
                  const BondSpace& br);
  void update_left_env(const BTensor& Lin, const BTensor& A, BTensor& Lout, const BondSpace& bl,
                       const BondSpace& br);
  void update_right_env(const BTensor& Rin, const BTensor& B, BTensor& Rout, const BondSpace& bl,
                        const BondSpace& br);
  void form_theta(const BTensor& X, const BTensor& Y, BTensor& theta, const BondSpace& bl, const BondSpace& bm,
                  const BondSpace& br);
  // split theta at bond (i,i+1); absorb_right: S goes to Y (left-to-right sweep)
  double split(BTensor& theta, const BondSpace& bl, const BondSpace& br, long long chi_max, double eps,
               bool absorb_right, BondSpace& bm, BTensor& X, BTensor& Y, double* s_ent = nullptr);
  bool gram_finish(cplx* G, cplx* galt, const std::vector<int>& P, const std::vector<int>& Q,
                   const std::vector<long long>& toff);
  double split_mixed(BTensor& theta, const BondSpace& bl, const BondSpace& br, long long chi_max, double eps,
                     bool absorb_right, BondSpace& bm, BTensor& X, BTensor& Y, double* s_ent, bool& ok);
  void bond_update(int i, bool left_to_right, double tau, long long chi_max, double eps, bool backward,
                   double* s_ent);
  // one-site sweep pieces
  void build_bond_layout(BTensor& t, const BondSpace& b) const;
  void plan_heff0(HeffPlan& p, const BTensor& Lenv, const BTensor& Renv, const BTensor& C);
  // Cholesky QR gauge shift: right: M (blocks (a,s,c)) = A C with A left-orthonormal;
  // left: M (blocks (a,s,b)) = C Q with Q right-orthonormal; M is overwritten by A or Q
  void gauge_shift(BTensor& M, const BondSpace& b, BTensor& C, bool right);
  void absorb(const BTensor& C, BTensor& M, bool from_left);  // M <- C M (from_left) or M C
  void site_update1(int i, bool left_to_right, double tau, bool shift);
  int expm(HeffPlan& H, cplx* x, double tau);  // returns the Krylov dimension used

  int L_ = 0;
  Model model_;
  Opts opt_;
  cudaStream_t stream_ = nullptr;
  bool own_stream_ = false;
  std::unique_ptr<Recoupler> rec_;
  std::vector<BondSpace> bonds_;
  std::vector<BTensor> site_;
  std::vector<BTensor> Lenv_, Renv_;
  BTensor theta_;  // bond-problem theta layout
  std::unique_ptr<HeffPlan> bp_heff_, chain_heff_;
  bool bond_only_ = false;
  bool profile_ = false;
  int center_ = 0;  // orthogonality centre
  bool cap_hit_ = false;    // the chi cap set a truncation in the current two-site step
  bool saturated_ = false;  // adaptive mode: one-site steps from now on
  // Krylov workspace
  DevBuf kv_, kw_, kpart_, kh1_, kh2_, knrm_, kstate_;
  long long kcap_ = 0;
  void* pinned_ = nullptr;
  StepStats stats_;
  int* dstatus_ = nullptr;
  // device scratch of the Jacobi drivers' work lists, grown on demand (stream-ordered)
  DevBuf jscratch_;
  ScratchFn jscratch();
  cudaEvent_t env_ev_[2] = {nullptr, nullptr};
  int gemm_kind_ = -1;  // block-GEMM precision of H_eff, environment updates and theta formation

  friend struct BondAccess;
};

}  // namespace tdvp
