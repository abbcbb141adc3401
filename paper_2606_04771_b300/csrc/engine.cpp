// Two-site TDVP engine (host orchestration of the device kernels).
//
// Sec. S2.2: second-order two-site TDVP.  One time step dt is a left-to-right
// half sweep and a right-to-left half sweep with tau = dt/2: at every bond the
// two-site tensor is evolved by exp(-i tau H_eff) (Krylov), split by a
// per-sector SVD with truncation on the truncated weight (Sec. S2.4), the
// environment is updated, and the new centre tensor is evolved backward by
// exp(+i tau H_eff^(1)) except at the last bond of the half sweep.  Sec. S2.3:
// every contraction is a list of dense block products (GEMM tasks), with the
// MPO applied as an FP64-weighted linear combination of blocks in between.
#include "engine.hpp"

#include "../../include/tdvp.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <mutex>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <tuple>

namespace tdvp {

// NVTX range for the duration of a scope (a no-op unless a profiler is attached):
// tdvp_step, tdvp_step_one_site, bond_update, site_update1, krylov, split, env_update
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// device buffers and plan uploads
// ---------------------------------------------------------------------------

DevAcct*& current_acct() {
  thread_local DevAcct* a = nullptr;
  return a;
}

DevBuf::DevBuf(size_t b, cudaStream_t st) : bytes(b), s(st) {
  if (b) {
    TDVP_CUDA(cudaMallocAsync(&p, b, st));
    acct = current_acct();
    if (acct) acct->add((long long)b);
  }
}
DevBuf::~DevBuf() { reset(); }
DevBuf& DevBuf::operator=(DevBuf&& o) noexcept {
  if (this != &o) {
    reset();
    p = o.p;
    bytes = o.bytes;
    s = o.s;
    acct = o.acct;
    o.p = nullptr;
    o.bytes = 0;
    o.acct = nullptr;
  }
  return *this;
}
void DevBuf::reset() {
  if (p) {
    cudaFreeAsync(p, s);
    if (acct) acct->add(-(long long)bytes);
  }
  p = nullptr;
  bytes = 0;
  acct = nullptr;
}

// Host time of a planning section, printed to stderr when TDVP_PLAN_DEBUG is set
// (read once per process).
struct PlanClock {
  const char* name;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  explicit PlanClock(const char* n) : name(n) {}
  ~PlanClock() {
    static const bool on = std::getenv("TDVP_PLAN_DEBUG") != nullptr;
    if (on)
      std::fprintf(stderr, "plan %s %.3f ms\n", name,
                   std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
  }
};

// hash of a small array of ints (FNV-1a over the values), for the planners' maps
struct IntArrayHash {
  template <size_t N>
  size_t operator()(const std::array<int, N>& a) const {
    uint64_t h = 1469598103934665603ull;
    for (int v : a) h = (h ^ (uint64_t)(uint32_t)v) * 1099511628211ull;
    return (size_t)h;
  }
};
template <size_t N, class V>
using IntArrayMap = std::unordered_map<std::array<int, N>, V, IntArrayHash>;

template <class T>
static DevBuf upload(const std::vector<T>& v, cudaStream_t s) {
  DevBuf b(std::max<size_t>(v.size(), 1) * sizeof(T), s);
  if (!v.empty()) TDVP_CUDA(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return b;
}

void GemmPlan::finalize(cudaStream_t s, int kind_, int* status_) {
  PlanClock clk(kind_ == 1 ? (packed.empty() ? "finalize bf16x4" : "finalize bf16x4 packed") : "finalize other");
  kind = kind_;
  status = status_;
  if (!packed.empty() && kind != 1) throw Error(-5, "packed GEMM plans need the BF16x4 kernel");
  static const bool fdbg = std::getenv("TDVP_PLAN_DEBUG") != nullptr;
  auto ft0 = std::chrono::steady_clock::now();
  auto fmark = [&](const char* what) {
    if (!fdbg) return;
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "plan   finalize %s %.3f ms (%zu tasks, %zu segs)\n", what,
                 std::chrono::duration<double, std::milli>(now - ft0).count(), tasks.size(), segs.size());
    ft0 = now;
  };
  // algorithmic bytes: each distinct operand block (base, address) read once, with the
  // size of its last use, and each output written once
  struct Use {
    int base;
    uintptr_t ptr;
    long long n;
  };
  std::vector<Use> seen;
  bytes = 0;
  for (int i = 0; i < (int)tasks.size(); ++i) {
    const GemmTask& t = tasks[i];
    bytes += (long long)t.rows * t.cols * (long long)sizeof(cplx);
    if (!packed.empty()) {
      for (const PackedSrc& q : packed[i].a)
        seen.push_back({q.base, reinterpret_cast<uintptr_t>(q.src), (long long)q.rows * q.cols});
      for (const PackedSrc& q : packed[i].b)
        seen.push_back({q.base, reinterpret_cast<uintptr_t>(q.src), (long long)q.rows * q.cols});
      continue;
    }
    for (int k = 0; k < t.seg_count; ++k) {
      const GemmSeg& g = segs[t.seg_begin + k];
      seen.push_back({g.a_base, reinterpret_cast<uintptr_t>(g.a), (long long)t.rows * g.k});
      seen.push_back({g.b_base, reinterpret_cast<uintptr_t>(g.b), (long long)g.k * t.cols});
    }
  }
  std::stable_sort(seen.begin(), seen.end(), [](const Use& x, const Use& y) {
    return x.base != y.base ? x.base < y.base : x.ptr < y.ptr;
  });
  for (size_t i = 0; i < seen.size(); ++i)
    if (i + 1 == seen.size() || seen[i + 1].base != seen[i].base || seen[i + 1].ptr != seen[i].ptr)
      bytes += seen[i].n * (long long)sizeof(cplx);
  fmark("bytes");
  tiles.clear();
  const int tm = kind < 0 ? 64 : split_tile_m(), tn0 = kind < 0 ? 64 : split_tile_n(kind);
  for (int i = 0; i < (int)tasks.size(); ++i) {
    GemmTask& t = tasks[i];
    const int tn = (kind == 1 && t.tn > 0) ? t.tn : tn0;
    t.tiles_m = (t.rows + tm - 1) / tm;
    t.tiles_n = (t.cols + tn - 1) / tn;
    t.roff = t.coff = 0;
    for (int a = 0; a < t.tiles_m; ++a)
      for (int b = 0; b < t.tiles_n; ++b)
        if (!upper_only || a * tm <= b * tn + tn - 1) tiles.push_back(make_int3(i, a, b));
  }
  kext.clear();
  fix.clear();
  if (kind < 0) {
    // FP64 kernel: one CTA per tile item, scheduled in list order.  This part's FP64
    // pipe is slow enough that a single 64 x 64 tile with K ~ 300 runs for over a
    // millisecond, so a few large tiles would leave most SMs idle: tiles of a
    // single-segment task whose cost exceeds an even share of the work (1/4 of the
    // average over 2 x 148 CTAs) are split along K into chunks written to partial slots
    // and summed afterwards in a fixed order (results do not depend on scheduling).
    // Items go in longest-processing-time order.
    std::vector<long long> ksum(tasks.size(), 0);
    for (int i = 0; i < (int)tasks.size(); ++i)
      for (int k = 0; k < tasks[i].seg_count; ++k) ksum[i] += segs[tasks[i].seg_begin + k].k;
    auto area = [&](const int3& t) {
      const GemmTask& g = tasks[t.x];
      return (long long)std::min(tm, g.rows - t.y * tm) * std::min(tm, g.cols - t.z * tm);
    };
    long long total = 0;
    for (const int3& t : tiles) total += ksum[t.x] * area(t);
    const long long share = std::max<long long>(total / (4 * 2 * 148), 64LL * 64 * 64);
    struct Item {
      int3 t;
      int4 k;
      long long cost;
    };
    std::vector<Item> items;
    int slots = 0;
    for (const int3& t : tiles) {
      const long long c = ksum[t.x] * area(t);
      const int K = (int)ksum[t.x];
      int nch = ksplit && tasks[t.x].seg_count == 1 ? (int)std::min<long long>((c + share - 1) / share, K / 32) : 1;
      if (nch <= 1) {
        items.push_back({t, make_int4(0, K, -1, 0), c});
        continue;
      }
      const int step = ((K + nch - 1) / nch + 7) / 8 * 8;  // multiples of the kernel's k step
      nch = (K + step - 1) / step;
      fix.push_back(make_int4(t.x, t.y, t.z, slots | (nch << 20)));
      for (int q = 0; q < nch; ++q) {
        const int kb = q * step, ke = std::min(K, kb + step);
        items.push_back({t, make_int4(kb, ke, slots + q, 0), (long long)(ke - kb) * area(t)});
      }
      slots += nch;
    }
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.cost > b.cost; });
    tiles.clear();
    if (!fix.empty()) {
      for (const Item& it : items) {
        tiles.push_back(it.t);
        kext.push_back(it.k);
      }
      dkx = upload(kext, s);
      dfix = upload(fix, s);
      dws = DevBuf((size_t)slots * 64 * 64 * sizeof(cplx), s);
    } else {
      for (const Item& it : items) tiles.push_back(it.t);
    }
  }
  if (!rowoffs.empty()) {
    drow = upload(rowoffs, s);
    for (int i = 0; i < (int)tasks.size(); ++i)
      tasks[i].rowoff = (i < (int)row_start.size() && row_start[i] >= 0) ? drow.as<long long>() + row_start[i] : nullptr;
  }
  fmark("tiles");
  if (kind == 1 && !packed.empty()) plan_packed(s);
  else if (kind == 1) plan_digits(s);
  fmark("digits");
  dt = upload(tasks, s);
  ds = upload(segs, s);
  dti = upload(tiles, s);
  fmark("upload");
}

// BF16x4: every distinct operand block (same storage, shape, op and alpha) is split
// once per launch into digit records.  Exactness of a task's accumulation needs one
// scale per output row across all of its A operands and one per output column
// across its B operands, so operands that meet in a task are merged (union-find)
// into scale groups; a group's scales are the maxima over all of its operands.
void GemmPlan::plan_digits(cudaStream_t s) {
  // side, base, ptr, rows, cols, ld, op, alpha, static
  typedef std::tuple<int, int, uintptr_t, int, int, int, int, double, int> Key;
  struct KeyHash {
    size_t operator()(const Key& k) const {
      uint64_t h = 1469598103934665603ull;
      auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
      mix((uint64_t)std::get<0>(k));
      mix((uint64_t)std::get<1>(k));
      mix((uint64_t)std::get<2>(k));
      mix((uint64_t)std::get<3>(k));
      mix((uint64_t)std::get<4>(k));
      mix((uint64_t)std::get<5>(k));
      mix((uint64_t)std::get<6>(k));
      double a = std::get<7>(k);
      uint64_t ab;
      std::memcpy(&ab, &a, sizeof(ab));
      mix(ab);
      mix((uint64_t)std::get<8>(k));
      return (size_t)h;
    }
  };
  std::unordered_map<Key, int, KeyHash> idx;
  idx.reserve(4 * segs.size() + 16);
  std::vector<Key> keys;
  std::vector<int> parent;
  auto get = [&](const Key& k) {
    auto it = idx.find(k);
    if (it != idx.end()) return it->second;
    const int i = (int)keys.size();
    idx[k] = i;
    keys.push_back(k);
    parent.push_back(i);
    return i;
  };
  std::function<int(int)> find = [&](int x) {
    while (parent[x] != x) x = parent[x] = parent[parent[x]];
    return x;
  };
  std::vector<int> first_a(tasks.size(), -1), first_b(tasks.size(), -1);
  std::vector<std::pair<int, int>> segop(segs.size(), {-1, -1});
  for (int i = 0; i < (int)tasks.size(); ++i) {
    const GemmTask& t = tasks[i];
    for (int k = 0; k < t.seg_count; ++k) {
      const int si = t.seg_begin + k;
      const GemmSeg& g = segs[si];
      if (g.k <= 0) continue;
      const int ia = get(Key(0, g.a_base, reinterpret_cast<uintptr_t>(g.a), t.rows, g.k, g.lda, g.op_a, g.alpha,
                             g.a_static != 0));
      const int ib = get(Key(1, g.b_base, reinterpret_cast<uintptr_t>(g.b), g.k, t.cols, g.ldb, g.op_b, 1.0,
                             g.b_static != 0));
      segop[si] = {ia, ib};
      if (first_a[i] < 0) first_a[i] = ia;
      else parent[find(ia)] = find(first_a[i]);
      if (first_b[i] < 0) first_b[i] = ib;
      else parent[find(ib)] = find(first_b[i]);
    }
  }
  // a group is static only if every operand in it is; static groups take the first
  // offsets so that the per-launch maxima reset covers the dynamic range only
  // per union-find root (an operand index): static (1) unless one member is dynamic
  std::vector<int> gstat(keys.size(), -1);
  for (int i = 0; i < (int)keys.size(); ++i) {
    const int r = find(i);
    const int st = std::get<8>(keys[i]);
    gstat[r] = gstat[r] < 0 ? st : (gstat[r] & st);
  }
  std::vector<int> goff(keys.size(), -1);
  long long ng = 0;
  for (int pass = 1; pass >= 0; --pass) {
    if (pass == 0) ngrp_static = (int)ng;
    for (int i = 0; i < (int)keys.size(); ++i) {
      const int r = find(i);
      if (goff[r] >= 0 || gstat[r] != pass) continue;
      goff[r] = (int)ng;
      ng += std::get<0>(keys[r]) == 0 ? std::get<3>(keys[r]) : std::get<4>(keys[r]);
    }
  }
  if (ng > INT32_MAX) throw Error(-5, "GEMM plan too large for 32-bit scale offsets");
  ngrp = (int)ng;
  long long nrec = 0;
  std::vector<long long> roff(keys.size());
  for (int i = 0; i < (int)keys.size(); ++i) {
    roff[i] = nrec;
    nrec += (long long)std::get<3>(keys[i]) * std::get<4>(keys[i]);
  }
  ddig = DevBuf(std::max<long long>(nrec, 1) * sizeof(unsigned long long), s);
  dtag = DevBuf(std::max(ngrp, 1) * sizeof(unsigned), s);
  TDVP_CUDA(cudaMemsetAsync(dtag.p, 0, std::max(ngrp, 1) * sizeof(unsigned), s));
  dexp = DevBuf(std::max(ngrp, 1) * sizeof(int), s);
  epoch = 0;
  unsigned long long* dig = ddig.as<unsigned long long>();
  std::vector<DigitOp> all(keys.size());
  const int job = digit_job_size();
  for (int part = 0; part < 2; ++part) {  // 0: static operands, 1: dynamic
    std::vector<DigitOp>& ops = part == 0 ? dops_s : dops_d;
    std::vector<int2>& jobs = part == 0 ? djobs_s : djobs_d;
    ops.clear();
    jobs.clear();
    for (int i = 0; i < (int)keys.size(); ++i) {
      if ((gstat[find(i)] != 0) != (part == 0)) continue;
      const Key& k = keys[i];
      DigitOp o{};
      o.side = std::get<0>(k);
      o.base = std::get<1>(k);
      o.src = reinterpret_cast<const cplx*>(std::get<2>(k));
      o.rows = std::get<3>(k);
      o.cols = std::get<4>(k);
      o.ld = std::get<5>(k);
      o.op = std::get<6>(k);
      o.alpha = std::get<7>(k);
      o.grp = goff[find(i)];
      o.dig = dig + roff[i];
      o.dig_ld = o.cols;
      o.row0 = o.col0 = 0;
      o.kmajor = 0;
      all[i] = o;
      const long long n = (long long)o.rows * o.cols;
      for (long long e = 0; e < n; e += job) jobs.push_back(make_int2((int)ops.size(), (int)e));
      ops.push_back(o);
    }
  }
  for (int i = 0; i < (int)tasks.size(); ++i) {
    if (first_a[i] >= 0) tasks[i].roff = goff[find(first_a[i])];
    if (first_b[i] >= 0) tasks[i].coff = goff[find(first_b[i])];
  }
  for (int si = 0; si < (int)segs.size(); ++si) {
    segs[si].a_dig = segop[si].first >= 0 ? all[segop[si].first].dig : nullptr;
    segs[si].b_dig = segop[si].second >= 0 ? all[segop[si].second].dig : nullptr;
  }
  ddops_s = upload(dops_s, s);
  djb_s = upload(djobs_s, s);
  ddops_d = upload(dops_d, s);
  djb_d = upload(djobs_d, s);
  static_done = false;
  // the persistent kernel walks the tiles with a stride of the grid: the most
  // expensive (most K chunks) first balances the SMs
  std::vector<int> cost(tasks.size(), 0);
  for (int i = 0; i < (int)tasks.size(); ++i)
    for (int k = 0; k < tasks[i].seg_count; ++k) cost[i] += (segs[tasks[i].seg_begin + k].k + 31) / 32;
  std::stable_sort(tiles.begin(), tiles.end(), [&](const int3& x, const int3& y) { return cost[x.x] > cost[y.x]; });
}

// Packed BF16x4 plan: task i has one segment whose operands are private record
// matrices (A: rows x K, B: K x cols, row-major) assembled from the source blocks of
// packed[i]; every record position no source covers stays zero.  Each task side is
// its own scale group (one scale per A row, one per B column): no operand is shared
// between tasks, so no groups need merging.  Static sides take the first group
// offsets (split once per plan), dynamic sides the rest (split every launch).
void GemmPlan::plan_packed(cudaStream_t s) {
  const int nt = (int)tasks.size();
  std::vector<long long> ga(nt, -1), gb(nt, -1);
  long long ng = 0;
  for (int pass = 1; pass >= 0; --pass) {  // 1: static sides, 0: dynamic
    if (pass == 0) ngrp_static = (int)ng;
    for (int i = 0; i < nt; ++i) {
      if ((int)packed[i].a_static == pass) {
        ga[i] = ng;
        ng += tasks[i].rows;
      }
      if ((int)packed[i].b_static == pass) {
        gb[i] = ng;
        ng += tasks[i].cols;
      }
    }
  }
  if (ng > INT32_MAX) throw Error(-5, "GEMM plan too large for 32-bit scale offsets");
  ngrp = (int)ng;
  // Operands as tile images (the BF16 planes of the GEMM's shared-memory stages, tile
  // after tile, fetched by bulk copies) unless TDVP_HEFF_IMAGES=0, which keeps 8-byte
  // digit records unpacked by the producer warps.  Offsets in 8-byte units.
  const char* ie = std::getenv("TDVP_HEFF_IMAGES");
  const bool images = !(ie && ie[0] == '0');
  images_ = images;
  std::vector<long long> aoff(nt), boff(nt);
  std::vector<int> nkc(nt), tnw(nt);
  long long nrec = 0;
  for (int i = 0; i < nt; ++i) {
    const long long K = segs[tasks[i].seg_begin].k;
    nkc[i] = (int)((K + 15) / 16);
    tnw[i] = tasks[i].tn > 0 ? tasks[i].tn : split_tile_n(1);
    aoff[i] = nrec;
    nrec += images ? (long long)tasks[i].tiles_m * nkc[i] * (32768 / 8) : (long long)tasks[i].rows * K;
    boff[i] = nrec;
    nrec += images ? (long long)tasks[i].tiles_n * nkc[i] * (16384 / 8) : K * tasks[i].cols;
  }
  ddig = DevBuf(std::max<long long>(nrec, 1) * sizeof(unsigned long long), s);
  TDVP_CUDA(cudaMemsetAsync(ddig.p, 0, std::max<long long>(nrec, 1) * sizeof(unsigned long long), s));
  dtag = DevBuf(std::max(ngrp, 1) * sizeof(unsigned), s);
  TDVP_CUDA(cudaMemsetAsync(dtag.p, 0, std::max(ngrp, 1) * sizeof(unsigned), s));
  dexp = DevBuf(std::max(ngrp, 1) * sizeof(int), s);
  epoch = 0;
  unsigned long long* dig = ddig.as<unsigned long long>();
  const int job = digit_job_size();
  dops_s.clear();
  dops_d.clear();
  djobs_s.clear();
  djobs_d.clear();
  auto add = [&](const PackedSrc& q, int side, bool st, long long grp, unsigned long long* base, int ld, int kc,
                 int tn) {
    std::vector<DigitOp>& ops = st ? dops_s : dops_d;
    std::vector<int2>& jobs = st ? djobs_s : djobs_d;
    DigitOp o{};
    o.side = side;
    o.base = q.base;
    o.src = q.src;
    o.rows = q.rows;
    o.cols = q.cols;
    o.ld = q.ld;
    o.op = q.op;
    o.alpha = side == 0 ? q.alpha : 1.0;
    o.grp = (int)grp;
    o.dig = base;
    o.dig_ld = ld;
    o.row0 = q.row0;
    o.col0 = q.col0;
    o.kmajor = side == 1;  // B records column by column (K contiguous)
    o.img_nkc = images ? kc : 0;
    o.img_tn = tn;
    const long long n = (long long)o.rows * o.cols;
    for (long long e = 0; e < n; e += job) jobs.push_back(make_int2((int)ops.size(), (int)e));
    ops.push_back(o);
  };
  for (int i = 0; i < nt; ++i) {
    GemmTask& t = tasks[i];
    GemmSeg& g = segs[t.seg_begin];
    const int K = g.k;
    for (const PackedSrc& q : packed[i].a) add(q, 0, packed[i].a_static, ga[i], dig + aoff[i], K, nkc[i], tnw[i]);
    for (const PackedSrc& q : packed[i].b) add(q, 1, packed[i].b_static, gb[i], dig + boff[i], K, nkc[i], tnw[i]);
    t.b_kmajor = 1;
    t.img = images ? 1 : 0;
    t.roff = (int)ga[i];
    t.coff = (int)gb[i];
    g.a_dig = dig + aoff[i];
    g.b_dig = dig + boff[i];
  }
  ddops_s = upload(dops_s, s);
  djb_s = upload(djobs_s, s);
  ddops_d = upload(dops_d, s);
  djb_d = upload(djobs_d, s);
  static_done = false;
  // dynamic operands that each hold whole scale lines (an A source spanning all K
  // columns, a B source all K rows) are split by one fused kernel
  bool own = true;
  for (const DigitOp& o : dops_d) {
    const int K = o.dig_ld;  // row-major A and K-major B records: lines of length K
    const bool whole = o.side == 0 ? (o.col0 == 0 && o.cols == K) : (o.row0 == 0 && o.rows == K);
    if (!whole || (o.side == 0 ? o.rows : o.cols) > digit_slots()) own = false;
  }
  {
    // the fused kernel gives each operand one CTA; the two passes spread every operand
    // over the conversion's jobs and measure slightly faster on the chi = 4096 bond
    // (0.305 against 0.314 ms per matvec): TDVP_DIGIT_FUSED=1 selects the fused kernel
    const char* e = std::getenv("TDVP_DIGIT_FUSED");
    if (!(e && e[0] == '1')) own = false;
  }
  dyn_mode = dyn_tags_external ? 1 : (own ? 2 : 0);
  std::vector<int> cost(nt, 0);
  for (int i = 0; i < nt; ++i) cost[i] = (segs[tasks[i].seg_begin].k + 31) / 32;
  std::stable_sort(tiles.begin(), tiles.end(), [&](const int3& x, const int3& y) { return cost[x.x] > cost[y.x]; });
}

unsigned GemmPlan::begin_split(cudaStream_t s, const Bases4& B) const {
  if (epoch + 2 > DIGIT_EPOCH_MAX) {  // the tag counter wraps: clear every tag, split all again
    TDVP_CUDA(cudaMemsetAsync(dtag.p, 0, std::max(ngrp, 1) * sizeof(unsigned), s));
    epoch = 0;
    static_done = false;
  }
  if (!static_done) {  // environment operands: split once per plan
    launch_digits(ddops_s.as<DigitOp>(), (int)dops_s.size(), djb_s.as<int2>(), (int)djobs_s.size(),
                  dtag.as<unsigned>(), dexp.as<int>(), ++epoch, B, s);
    static_done = true;
  }
  return ++epoch;
}

void GemmPlan::launch(cudaStream_t s, const Bases4& B, unsigned ep, const int3* tsub, int nsub) const {
  const int3* tl = tsub ? tsub : dti.as<int3>();
  const int nt = tsub ? nsub : (int)tiles.size();
  if (kind < 0) {
    const bool split = !tsub && !kext.empty();
    launch_gemm_fp64(dt.as<GemmTask>(), ds.as<GemmSeg>(), tl, nt, B, s, split ? dkx.as<int4>() : nullptr,
                     dws.as<cplx>());
    if (split) launch_gemm_fp64_fix(dt.as<GemmTask>(), dfix.as<int4>(), (int)fix.size(), dws.as<cplx>(), B, s);
  } else {
    if (kind == 1) {
      const unsigned e = ep ? ep : begin_split(s, B);
      const int mode = dyn_mode == 1 && !ep ? 0 : dyn_mode;  // no producer raised the tags: both passes
      launch_digits(ddops_d.as<DigitOp>(), (int)dops_d.size(), djb_d.as<int2>(), (int)djobs_d.size(),
                    dtag.as<unsigned>(), dexp.as<int>(), e, B, s, mode);
    }
    if (kind == 1)
      launch_exact_merged_or_alone(ExactSlice{dt.as<GemmTask>(), ds.as<GemmSeg>(), tl, dexp.as<int>(), status, B,
                                              images_ ? 1 : 0},
                                   nt,
                                   s);
    else
      launch_gemm_split(kind, dt.as<GemmTask>(), ds.as<GemmSeg>(), tl, nt, dexp.as<int>(), B, status, s);
  }
}

void LincombPlan::finalize(cudaStream_t s) {
  chunks.clear();
  for (int i = 0; i < (int)tasks.size(); ++i) {
    int n = tasks[i].rows * tasks[i].cols;
    for (int e = 0; e < n; e += LINCOMB_CHUNK) chunks.push_back(make_int2(i, e));
  }
  dt = upload(tasks, s);
  dm = upload(terms, s);
  dc = upload(chunks, s);
}

void LincombPlan::launch(cudaStream_t s, unsigned epoch) const {
  launch_lincomb(dt.as<LincombTask>(), dm.as<LincombTerm>(), dc.as<int2>(), (int)chunks.size(), s, epoch);
}

void CopyPlan::finalize(cudaStream_t s) {
  chunks.clear();
  for (int i = 0; i < (int)tasks.size(); ++i) {
    int n = tasks[i].rows * tasks[i].cols;
    for (int e = 0; e < n; e += LINCOMB_CHUNK) chunks.push_back(make_int2(i, e));
  }
  dt = upload(tasks, s);
  dc = upload(chunks, s);
}

void CopyPlan::launch(cudaStream_t s) const { launch_copy(dt.as<CopyTask>(), dc.as<int2>(), (int)chunks.size(), s); }

void HeffPlan::apply_owned(const cplx* in, cplx* out, const std::vector<char>& owned, cudaStream_t s) const {
  if (owned.size() != g3.tasks.size()) throw Error(-1, "one ownership flag per output group");
  std::vector<int3> sub;
  for (const int3& t : g3.tiles)
    if (owned[t.x]) sub.push_back(t);
  DevBuf dsub(std::max<size_t>(sub.size(), 1) * sizeof(int3), s);
  if (!sub.empty())
    TDVP_CUDA(cudaMemcpyAsync(dsub.p, sub.data(), sub.size() * sizeof(int3), cudaMemcpyHostToDevice, s));
  Bases4 B{{0, reinterpret_cast<uintptr_t>(in), reinterpret_cast<uintptr_t>(out), 0}};
  g1.launch(s, B);
  const unsigned e = g3.dyn_mode == 1 ? g3.begin_split(s, B) : 0u;
  lc.launch(s, e);
  g3.launch(s, B, e, dsub.as<int3>(), (int)sub.size());
  TDVP_CUDA(cudaStreamSynchronize(s));  // the tile subset's buffer is freed on return
}

void HeffPlan::apply(const cplx* in, cplx* out, cudaStream_t s) const {
  Bases4 B{{0, reinterpret_cast<uintptr_t>(in), reinterpret_cast<uintptr_t>(out), 0}};
  g1.launch(s, B);
  if (g3.dyn_mode == 1) {  // the linear combination raises the stage-3 operand's exponent tags
    const unsigned e = g3.begin_split(s, B);
    lc.launch(s, e);
    g3.launch(s, B, e);
  } else {
    lc.launch(s);
    g3.launch(s, B);
  }
}

// a Jacobi driver's sweep count, or the CUDA error of a failed cooperative launch
static int jacobi(int sweeps) {
  if (sweeps == JACOBI_ENOMEM) throw Error(-3, "Jacobi work lists: device allocation failed");
  if (sweeps == JACOBI_ETIMEOUT) throw Error(-7, "Jacobi ring: a neighbour exchange timed out");
  if (sweeps < 0) {
    cudaError_t e = cudaGetLastError();
    throw Error(-6, std::string("cooperative Jacobi launch failed: ") + cudaGetErrorString(e));
  }
  return sweeps;
}

// 64-bit key of a recoupled block (a', s1', c', s2', b', w2, b): bond sector indices
// below 4096, the middle label tc' (2S or 2S^z, possibly negative) within +-2047, site
// and channel indices below 8
static inline uint64_t t2key(int ap, int s1p, int tcp, int s2p, int bp, int w2, int b) {
  const int tco = tcp + 2048;
  if ((unsigned)ap >= 4096u || (unsigned)tco >= 4096u || (unsigned)bp >= 4096u || (unsigned)b >= 4096u ||
      (unsigned)s1p >= 8u || (unsigned)s2p >= 8u || (unsigned)w2 >= 8u)
    throw Error(-5, "recoupled block key out of range");
  return ((uint64_t)ap << 45) | ((uint64_t)s1p << 42) | ((uint64_t)tco << 30) | ((uint64_t)s2p << 27) |
         ((uint64_t)bp << 15) | ((uint64_t)w2 << 12) | (uint64_t)b;
}

static inline cplx* as_off(long long off) { return reinterpret_cast<cplx*>(static_cast<uintptr_t>(off) * sizeof(cplx)); }

// ---------------------------------------------------------------------------
// construction
// ---------------------------------------------------------------------------

// The engine's device buffers come from the current device's default memory pool
// (cudaMallocAsync).  With the pool's default release threshold of zero, every stream
// synchronisation hands the unused memory back and the next allocations map it again;
// a bond update allocates and frees its work buffers many times between syncs.  The
// pool is therefore allowed to keep up to TDVP_POOL_KEEP_MB megabytes (default 4096)
// of freed memory, once per device and process; a larger threshold already set is
// left as it is.
static void keep_pool_memory() {
  static std::mutex m;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> g(m);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  done.push_back(dev);
  const char* e = std::getenv("TDVP_POOL_KEEP_MB");
  const unsigned long long want = (unsigned long long)(e && *e ? std::atoll(e) : 4096) << 20;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  unsigned long long cur = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < want)
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, (void*)&want);
  cudaGetLastError();
}

void Engine::init_common(bool su2, double J, double U, const Opts& o) {
  opt_ = o;
  if (o.krylov_max < 1 || o.krylov_max > KRYLOV_MAX) throw Error(-1, "krylov_max must be in [1, 32]");
  if (!(o.krylov_tol >= 0)) throw Error(-1, "krylov_tol must be >= 0 (0: always krylov_max matvecs)");
  if (o.precision < 0 || o.precision > 2) throw Error(-1, "unknown precision");
  if (o.device >= 0) TDVP_CUDA(cudaSetDevice(o.device));
  model_.init(su2, J, U);
  gemm_kind_ = o.precision - 1;
  rec_.reset(new Recoupler(&model_));
  if (o.stream) {
    stream_ = o.stream;
  } else {
    TDVP_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
    own_stream_ = true;
  }
  keep_pool_memory();
  const char* pe = std::getenv("TDVP_PROFILE_PHASES");
  profile_ = pe && pe[0] == '1';
  TDVP_CUDA(cudaMallocHost(&pinned_, 4096));
  TDVP_CUDA(cudaMalloc(&dstatus_, sizeof(int) * 4));
  TDVP_CUDA(cudaMemsetAsync(dstatus_, 0, sizeof(int) * 4, stream_));
}

Engine::Engine(int L, double J, double U, bool su2, const Opts& o) : L_(L) {
  if (L < 2 || (L % 2)) throw Error(-1, "L must be even and >= 2");
  init_common(su2, J, U, o);
  init_neel();
}

Engine* Engine::bond_problem(bool su2, double J, double U, const std::vector<Sector>& left,
                             const std::vector<Sector>& right, const Opts& o) {
  std::unique_ptr<Engine> e(new Engine());
  e->L_ = 2;
  e->bond_only_ = true;
  e->init_common(su2, J, U, o);
  e->bonds_.assign(3, BondSpace());
  e->bonds_[0].s = left;
  e->bonds_[2].s = right;
  for (int k : {0, 2}) {
    e->bonds_[k].build_index();
    if (e->bonds_[k].idx.size() != e->bonds_[k].s.size()) throw Error(-1, "duplicate sector label");
    for (auto& x : e->bonds_[k].s) {
      if (x.d < 1) throw Error(-1, "sector degeneracy must be >= 1");
      if (su2 && x.t < 0) throw Error(-1, "2S must be >= 0");
    }
  }
  e->Lenv_.resize(3);
  e->Renv_.resize(3);
  e->build_lenv_layout(e->Lenv_[0], e->bonds_[0], e->bonds_[0]);
  e->alloc(e->Lenv_[0], true);
  e->build_renv_layout(e->Renv_[2], e->bonds_[2], e->bonds_[2]);
  e->alloc(e->Renv_[2], true);
  e->build_theta_layout(e->theta_, e->bonds_[0], e->bonds_[2]);
  e->bp_heff_.reset(new HeffPlan());
  e->plan_heff2(*e->bp_heff_, e->Lenv_[0], e->Renv_[2], e->theta_, e->bonds_[0], e->bonds_[2]);
  TDVP_CUDA(cudaStreamSynchronize(e->stream_));
  return e.release();
}

// Synthetic state for the sweep benchmark: bond k (k sites to its left) carries the
// multiplets (n, t) of the k-site Hilbert space that can couple with the right part
// to the total singlet at half filling, with degeneracy
//   d = min(round(D0 exp(-Q^2/18 - S^2/4.5)), exact multiplicity left, exact multiplicity right),
// Q = n - k, S = t/2 (U1U1: the SU(2) profile summed over S >= |S^z|), D0 chosen so that
// the middle bond reaches chi_target; then every sector is made reachable and every
// right-canonical row space feasible, blocks are filled with counter-based normal
// numbers and sites 1..L-1 are right-orthonormalised per left sector.
Engine* Engine::product_state(int L, double J, double U, bool su2, const std::vector<int>& occ, const Opts& o) {
  if (L < 2) throw Error(-1, "L must be >= 2");
  std::unique_ptr<Engine> e(new Engine());
  e->L_ = L;
  e->init_common(su2, J, U, o);
  e->init_product(occ);
  return e.release();
}

Engine* Engine::random_state(int L, double J, double U, bool su2, long long chi_target, unsigned long long seed,
                             int center, const Opts& o) {
  if (L < 2 || (L % 2)) throw Error(-1, "L must be even and >= 2");
  if (chi_target < 1) throw Error(-1, "chi_target must be >= 1");
  if (center < 0 || center >= L) throw Error(-1, "center must be a site index");
  std::unique_ptr<Engine> e(new Engine());
  e->L_ = L;
  e->init_common(su2, J, U, o);
  const Model& M = e->model_;
  const int N = L;  // particles in the particle-hole frame at half filling
  typedef std::map<std::pair<int, int>, double> Cnt;
  std::vector<Cnt> cnt(L + 1);
  cnt[0][{0, 0}] = 1.0;
  std::vector<std::pair<int, int>> f;
  for (int k = 0; k < L; ++k)
    for (auto& q : cnt[k])
      for (auto& ms : M.site) {
        M.fuse(q.first.first, q.first.second, ms.n, ms.t, f);
        for (auto& r : f) cnt[k + 1][r] = std::min(cnt[k + 1][r] + q.second, 1e12);
      }
  auto profile = [&](int Q, int t) -> double {
    if (su2) return std::exp(-(double)Q * Q / 18.0 - (t / 2.0) * (t / 2.0) / 4.5);
    double acc = 0.0;  // SU(2) profile summed over S >= |S^z|
    for (int tt = std::abs(t); tt <= 24; tt += 2) acc += std::exp(-(double)Q * Q / 18.0 - (tt / 2.0) * (tt / 2.0) / 4.5);
    return acc;
  };
  auto tables = [&](double D0) {
    std::vector<BondSpace> b(L + 1);
    for (int k = 0; k <= L; ++k) {
      for (auto& q : cnt[k]) {
        int n = q.first.first, t = q.first.second;
        std::pair<int, int> partner = su2 ? std::make_pair(N - n, t) : std::make_pair(N - n, -t);
        auto it = cnt[L - k].find(partner);
        if (it == cnt[L - k].end()) continue;
        double cap = std::min(q.second, it->second);
        double d = std::floor(D0 * profile(n - k, t) + 0.5);
        if (k == 0 || k == L) d = 1.0;
        d = std::min(d, cap);
        if (d >= 1.0) b[k].s.push_back({n, t, (int)d});
      }
    }
    // reachability from the left and feasible right-canonical rows, until stable
    for (int pass = 0; pass < 4; ++pass) {
      for (int k = 0; k < L; ++k) {  // d_{k+1}(b) <= sum over (a, s) fusing into b of d_k(a)
        std::map<std::pair<int, int>, long long> reach;
        for (auto& a : b[k].s)
          for (auto& ms : M.site) {
            M.fuse(a.n, a.t, ms.n, ms.t, f);
            for (auto& r : f) reach[r] += a.d;
          }
        for (auto& x : b[k + 1].s) x.d = (int)std::min<long long>(x.d, reach[{x.n, x.t}]);
      }
      for (int k = L - 1; k >= 0; --k) {  // d_k(a) <= sum over (s, b) of d_{k+1}(b)
        std::map<std::pair<int, int>, int> dn;
        for (auto& x : b[k + 1].s) dn[{x.n, x.t}] = x.d;
        for (auto& a : b[k].s) {
          long long cols = 0;
          for (auto& ms : M.site) {
            M.fuse(a.n, a.t, ms.n, ms.t, f);
            for (auto& r : f) {
              auto it = dn.find(r);
              if (it != dn.end()) cols += it->second;
            }
          }
          a.d = (int)std::min<long long>(a.d, cols);
        }
      }
      for (auto& bb : b) {
        std::vector<Sector> keep;
        for (auto& x : bb.s)
          if (x.d > 0) keep.push_back(x);
        bb.s = keep;
      }
    }
    for (auto& bb : b) {
      std::sort(bb.s.begin(), bb.s.end(), [](const Sector& x, const Sector& y) {
        return x.n != y.n ? x.n < y.n : x.t < y.t;
      });
      bb.build_index();
    }
    return b;
  };
  auto chi_mid = [&](const std::vector<BondSpace>& b) {
    long long c = 0;
    for (auto& x : b[L / 2].s) c += (long long)x.d * M.mult_dim(x.t);
    return c;
  };
  double lo = 0.0, hi = 1.0;
  while (chi_mid(tables(hi)) < chi_target && hi < 1e7) hi *= 2;
  for (int it = 0; it < 50; ++it) {
    double mid = 0.5 * (lo + hi);
    if (chi_mid(tables(mid)) >= chi_target) hi = mid;
    else lo = mid;
  }
  e->bonds_ = tables(hi);
  for (int k = 0; k <= L; ++k)
    if (e->bonds_[k].s.empty()) throw Error(-5, "empty bond in the synthetic state");
  e->site_.resize(L);
  long long off = 0;
  for (int i = 0; i < L; ++i) {
    e->build_site_layout(e->site_[i], e->bonds_[i], e->bonds_[i + 1]);
    e->alloc(e->site_[i], false);
    launch_fill_normal(e->site_[i].data(), e->site_[i].size, seed, off, e->stream_);
    off += e->site_[i].size;
  }
  for (int i = 0; i < center; ++i) e->orthonormalize_cols(e->site_[i], e->bonds_[i], e->bonds_[i + 1]);
  for (int i = center + 1; i < L; ++i) e->orthonormalize_rows(e->site_[i], e->bonds_[i], e->bonds_[i + 1]);
  e->center_ = center;
  {  // normalise the centre tensor
    BTensor& T = e->site_[center];
    DevBuf part((size_t)296 * sizeof(cplx), e->stream_), nrm(sizeof(cplx), e->stream_);
    launch_dots(T.data(), 0, 1, T.data(), T.size, part.as<cplx>(), dots_grid(T.size), nrm.as<cplx>(), nullptr,
                e->stream_);
    cplx h;
    TDVP_CUDA(cudaMemcpyAsync(&h, nrm.p, sizeof(cplx), cudaMemcpyDeviceToHost, e->stream_));
    TDVP_CUDA(cudaStreamSynchronize(e->stream_));
    std::vector<double> inv(1, 1.0 / std::sqrt(h.x));
    DevBuf dinv(sizeof(double), e->stream_);
    TDVP_CUDA(cudaMemcpyAsync(dinv.p, inv.data(), sizeof(double), cudaMemcpyHostToDevice, e->stream_));
    CopyPlan cp;
    CopyTask t{};
    t.src = T.data();
    t.dst = T.data();
    t.rows = 1;
    t.cols = (int)T.size;
    t.src_rs = T.size;
    t.src_cs = 1;
    t.dst_rs = T.size;
    t.dst_cs = 1;
    t.gscale = dinv.as<double>();
    cp.tasks.push_back(t);
    cp.finalize(e->stream_);
    cp.launch(e->stream_);
    TDVP_CUDA(cudaStreamSynchronize(e->stream_));
  }
  e->build_environments();
  return e.release();
}

void Engine::build_environments() {
  const int L = L_;
  const Model& M = model_;
  Lenv_.clear();
  Renv_.clear();
  Lenv_.resize(L + 1);
  Renv_.resize(L + 1);
  std::vector<cplx> one(1, cplx{1.0, 0.0});
  build_lenv_layout(Lenv_[0], bonds_[0], bonds_[0]);
  alloc(Lenv_[0], true);
  int bi = Lenv_[0].find(bkey(0, M.chB, 0));
  TDVP_CUDA(cudaMemcpyAsync(Lenv_[0].ptr(bi), one.data(), sizeof(cplx), cudaMemcpyHostToDevice, stream_));
  build_renv_layout(Renv_[L], bonds_[L], bonds_[L]);
  alloc(Renv_[L], true);
  bi = Renv_[L].find(bkey(0, M.chE, 0));
  TDVP_CUDA(cudaMemcpyAsync(Renv_[L].ptr(bi), one.data(), sizeof(cplx), cudaMemcpyHostToDevice, stream_));
  for (int k = L - 1; k >= center_ + 1; --k)
    update_right_env(Renv_[k + 1], site_[k], Renv_[k], bonds_[k], bonds_[k + 1]);
  for (int k = 0; k < center_; ++k) update_left_env(Lenv_[k], site_[k], Lenv_[k + 1], bonds_[k], bonds_[k + 1]);
  TDVP_CUDA(cudaStreamSynchronize(stream_));
  check_status();
}

// ---------------------------------------------------------------------------
// checkpoint / resume
// ---------------------------------------------------------------------------
// File (little-endian): "TDVPCKP1"; int32 version = 1, L, su2, centre, cap_hit,
// saturated; float64 J, U, t; per bond k = 0..L: int32 count, then count x int32
// (n, t, d); per site i = 0..L-1: int64 element count, then the site tensor's blocks
// as complex128 in the engine's block order (which the bond tables determine);
// "TDVPEND1".  The environments are not stored: they are rebuilt from the sites with
// the same kernels in the same order as when they were made, so a resumed FP64 run
// repeats the uninterrupted one bit for bit.
namespace {
const char kCkptHead[8] = {'T', 'D', 'V', 'P', 'C', 'K', 'P', '1'};
const char kCkptTail[8] = {'T', 'D', 'V', 'P', 'E', 'N', 'D', '1'};

struct CkptHeader {
  int32_t version, L, su2, center, cap_hit, saturated;
  double J, U, t;
};

void put(std::FILE* f, const void* p, size_t n, const std::string& path) {
  if (n && std::fwrite(p, 1, n, f) != n) throw Error(TDVP_EIO, "checkpoint: write failed: " + path);
}
void get(std::FILE* f, void* p, size_t n, const std::string& path) {
  if (n && std::fread(p, 1, n, f) != n) throw Error(TDVP_EINVAL, "checkpoint: truncated file: " + path);
}
struct FileCloser {
  std::FILE* f;
  ~FileCloser() {
    if (f) std::fclose(f);
  }
};
}  // namespace

void Engine::save(const std::string& path, double t) {
  if (bond_only_) throw Error(TDVP_ESTATE, "checkpoint: a bond-problem context has no chain");
  const std::string tmp = path + ".part";
  {
    FileCloser fc{std::fopen(tmp.c_str(), "wb")};
    if (!fc.f) throw Error(TDVP_EIO, "checkpoint: cannot open " + tmp);
    CkptHeader h{1, L_, model_.su2 ? 1 : 0, center_, cap_hit_ ? 1 : 0, saturated_ ? 1 : 0, model_.J, model_.U, t};
    put(fc.f, kCkptHead, 8, tmp);
    put(fc.f, &h, sizeof(h), tmp);
    for (int k = 0; k <= L_; ++k) {
      const int32_t c = (int32_t)bonds_[k].s.size();
      put(fc.f, &c, sizeof(c), tmp);
      for (const Sector& x : bonds_[k].s) {
        const int32_t v[3] = {x.n, x.t, x.d};
        put(fc.f, v, sizeof(v), tmp);
      }
    }
    std::vector<cplx> host;
    for (int i = 0; i < L_; ++i) {
      const int64_t n = site_[i].size;
      host.resize((size_t)n);
      if (n) {
        TDVP_CUDA(cudaMemcpyAsync(host.data(), site_[i].data(), (size_t)n * sizeof(cplx), cudaMemcpyDeviceToHost,
                                  stream_));
        TDVP_CUDA(cudaStreamSynchronize(stream_));
      }
      put(fc.f, &n, sizeof(n), tmp);
      put(fc.f, host.data(), (size_t)n * sizeof(cplx), tmp);
    }
    put(fc.f, kCkptTail, 8, tmp);
    if (std::fflush(fc.f) != 0) throw Error(TDVP_EIO, "checkpoint: write failed: " + tmp);
  }
  if (std::rename(tmp.c_str(), path.c_str()) != 0) throw Error(TDVP_EIO, "checkpoint: cannot rename to " + path);
}

Engine* Engine::load(const std::string& path, const Opts& o, double* t) {
  FileCloser fc{std::fopen(path.c_str(), "rb")};
  if (!fc.f) throw Error(TDVP_EIO, "checkpoint: cannot open " + path);
  char head[8];
  get(fc.f, head, 8, path);
  if (std::memcmp(head, kCkptHead, 8) != 0) throw Error(TDVP_EINVAL, "checkpoint: not a checkpoint file: " + path);
  CkptHeader h;
  get(fc.f, &h, sizeof(h), path);
  if (h.version != 1 || h.L < 2 || h.L > 100000 || h.center < 0 || h.center >= h.L)
    throw Error(TDVP_EINVAL, "checkpoint: bad header: " + path);
  // read and check everything on the host before any device work
  std::vector<BondSpace> bonds(h.L + 1);
  for (int k = 0; k <= h.L; ++k) {
    int32_t c = 0;
    get(fc.f, &c, sizeof(c), path);
    if (c < 1 || c > 1000000) throw Error(TDVP_EINVAL, "checkpoint: bad sector count: " + path);
    for (int j = 0; j < c; ++j) {
      int32_t v[3];
      get(fc.f, v, sizeof(v), path);
      if (v[2] < 1) throw Error(TDVP_EINVAL, "checkpoint: bad sector degeneracy: " + path);
      bonds[k].s.push_back({v[0], v[1], v[2]});
    }
    bonds[k].build_index();
    if (bonds[k].idx.size() != bonds[k].s.size()) throw Error(TDVP_EINVAL, "checkpoint: duplicate sector: " + path);
  }
  std::vector<std::vector<cplx>> sites(h.L);
  for (int i = 0; i < h.L; ++i) {
    int64_t n = 0;
    get(fc.f, &n, sizeof(n), path);
    if (n < 0 || n > (int64_t)1 << 36) throw Error(TDVP_EINVAL, "checkpoint: bad site size: " + path);
    sites[i].resize((size_t)n);
    get(fc.f, sites[i].data(), (size_t)n * sizeof(cplx), path);
  }
  char tail[8];
  get(fc.f, tail, 8, path);
  if (std::memcmp(tail, kCkptTail, 8) != 0) throw Error(TDVP_EINVAL, "checkpoint: bad trailer: " + path);

  std::unique_ptr<Engine> e(new Engine());
  e->L_ = h.L;
  e->init_common(h.su2 != 0, h.J, h.U, o);
  e->bonds_ = std::move(bonds);
  e->site_.resize(h.L);
  for (int i = 0; i < h.L; ++i) {
    e->build_site_layout(e->site_[i], e->bonds_[i], e->bonds_[i + 1]);
    if (e->site_[i].size != (long long)sites[i].size())
      throw Error(TDVP_EINVAL, "checkpoint: site tensor does not match its bond tables: " + path);
    e->alloc(e->site_[i], false);
    if (!sites[i].empty())
      TDVP_CUDA(cudaMemcpyAsync(e->site_[i].data(), sites[i].data(), sites[i].size() * sizeof(cplx),
                                cudaMemcpyHostToDevice, e->stream_));
  }
  e->center_ = h.center;
  e->cap_hit_ = h.cap_hit != 0;
  e->saturated_ = h.saturated != 0;
  e->build_environments();
  if (t) *t = h.t;
  return e.release();
}

// Replace the columns of every right sector b of T (the matrix [sum_(a,s) d_a x d_b]) by
// an orthonormal basis of their column space (left singular vectors): T becomes
// left-canonical, sum_(a,s) T^H T = 1 on every sector.
void Engine::orthonormalize_cols(BTensor& T, const BondSpace& l, const BondSpace& r) {
  std::vector<std::vector<int>> by(r.s.size());
  for (int i = 0; i < (int)T.blocks.size(); ++i) by[T.blocks[i].key[2]].push_back(i);
  std::vector<long long> goff(r.s.size()), voff(r.s.size());
  std::vector<int> soff(r.s.size()), pv(r.s.size());
  long long gt = 0, vt = 0;
  int st = 0;
  for (int b = 0; b < (int)r.s.size(); ++b) {
    int p = 0;
    for (int bi : by[b]) p += T.blocks[bi].rows;
    int q = r.s[b].d;
    if (p < q) throw Error(-5, "infeasible left-canonical sector");
    pv[b] = p;
    goff[b] = gt;
    gt += (long long)p * q;
    voff[b] = vt;
    vt += (long long)q * q;
    soff[b] = st;
    st += q;
  }
  DevBuf dG(std::max<long long>(gt, 1) * sizeof(cplx), stream_), dV(std::max<long long>(vt, 1) * sizeof(cplx), stream_);
  DevBuf dS(std::max(st, 1) * sizeof(double), stream_), dP(std::max(st, 1) * sizeof(int), stream_);
  CopyPlan gather, scatter;
  std::vector<SvdTask> tasks;
  for (int b = 0; b < (int)r.s.size(); ++b) {
    int p = pv[b], q = r.s[b].d, r0 = 0;
    cplx* G = dG.as<cplx>() + goff[b];
    for (int bi : by[b]) {  // G = M, column-major p x q
      const Block& blk = T.blocks[bi];
      CopyTask t{};
      t.src = T.ptr(bi);
      t.rows = blk.rows;
      t.cols = blk.cols;
      t.src_rs = blk.cols;
      t.src_cs = 1;
      t.dst = G + r0;
      t.dst_rs = 1;
      t.dst_cs = p;
      gather.tasks.push_back(t);
      CopyTask u{};  // U = W / s
      u.src = G + r0;
      u.src_rs = 1;
      u.src_cs = p;
      u.col_map = dP.as<int>() + soff[b];
      u.scale = dS.as<double>() + soff[b];
      u.scale_mode = 2;
      u.dst = T.ptr(bi);
      u.rows = blk.rows;
      u.cols = q;
      u.dst_rs = q;
      u.dst_cs = 1;
      scatter.tasks.push_back(u);
      r0 += blk.rows;
    }
    tasks.push_back({G, dV.as<cplx>() + voff[b], dS.as<double>() + soff[b], dP.as<int>() + soff[b], p, q});
  }
  gather.finalize(stream_);
  gather.launch(stream_);
  DevBuf dt = upload(tasks, stream_);
  jacobi(run_jacobi_rounds(dt.as<SvdTask>(), tasks, 40, 1e-14, dstatus_, stream_, 0.0, 0.0, nullptr, jscratch()));
  scatter.finalize(stream_);
  scatter.launch(stream_);
  TDVP_CUDA(cudaStreamSynchronize(stream_));
}

// Replace the rows of every left sector a of T (the matrix [d_a x sum_(s,b) d_b]) by an
// orthonormal basis of their row space (the right singular vectors), which makes T
// right-canonical: sum_(s,b) T T^H = 1 on every sector.
void Engine::orthonormalize_rows(BTensor& T, const BondSpace& l, const BondSpace& r) {
  std::vector<std::vector<int>> by(l.s.size());
  for (int i = 0; i < (int)T.blocks.size(); ++i) by[T.blocks[i].key[0]].push_back(i);
  std::vector<long long> goff(l.s.size()), voff(l.s.size());
  std::vector<int> soff(l.s.size()), qv(l.s.size());
  long long gt = 0, vt = 0;
  int st = 0;
  for (int a = 0; a < (int)l.s.size(); ++a) {
    int q = 0;
    for (int bi : by[a]) q += T.blocks[bi].cols;
    int p = l.s[a].d;
    if (q < p) throw Error(-5, "infeasible right-canonical sector");
    qv[a] = q;
    goff[a] = gt;
    gt += (long long)q * p;
    voff[a] = vt;
    vt += (long long)p * p;
    soff[a] = st;
    st += p;
  }
  DevBuf dG(std::max<long long>(gt, 1) * sizeof(cplx), stream_), dV(std::max<long long>(vt, 1) * sizeof(cplx), stream_);
  DevBuf dS(std::max(st, 1) * sizeof(double), stream_), dP(std::max(st, 1) * sizeof(int), stream_);
  CopyPlan gather, scatter;
  std::vector<SvdTask> tasks;
  for (int a = 0; a < (int)l.s.size(); ++a) {
    int p = l.s[a].d, q = qv[a], c0 = 0;
    cplx* G = dG.as<cplx>() + goff[a];
    for (int bi : by[a]) {  // G = M^H, column-major q x p
      const Block& b = T.blocks[bi];
      CopyTask t{};
      t.src = T.ptr(bi);
      t.rows = b.rows;
      t.cols = b.cols;
      t.src_rs = b.cols;
      t.src_cs = 1;
      t.dst = G + c0;
      t.dst_rs = q;
      t.dst_cs = 1;
      t.conj = 1;
      gather.tasks.push_back(t);
      CopyTask u{};  // row k of V_M^H = conj(W[:, perm k]) / s_k
      u.src = G + c0;
      u.src_rs = q;
      u.src_cs = 1;
      u.row_map = dP.as<int>() + soff[a];
      u.conj = 1;
      u.scale = dS.as<double>() + soff[a];
      u.scale_mode = 4;
      u.dst = T.ptr(bi);
      u.rows = p;
      u.cols = b.cols;
      u.dst_rs = b.cols;
      u.dst_cs = 1;
      scatter.tasks.push_back(u);
      c0 += b.cols;
    }
    tasks.push_back({G, dV.as<cplx>() + voff[a], dS.as<double>() + soff[a], dP.as<int>() + soff[a], q, p});
  }
  gather.finalize(stream_);
  gather.launch(stream_);
  DevBuf dt = upload(tasks, stream_);
  jacobi(run_jacobi_rounds(dt.as<SvdTask>(), tasks, 40, 1e-14, dstatus_, stream_, 0.0, 0.0, nullptr, jscratch()));
  scatter.finalize(stream_);
  scatter.launch(stream_);
  TDVP_CUDA(cudaStreamSynchronize(stream_));
}

void Engine::heff_apply_bond(const cplx* in, cplx* out) {
  if (!bond_only_) throw Error(-2, "not a bond problem");
  bp_heff_->apply(in, out, stream_);
}

HeffPlan& Engine::chain_heff0() {
  if (bond_only_) throw Error(-2, "not a chain");
  if (!chain_heff_) {
    build_theta_layout(theta_, bonds_[0], bonds_[2]);
    chain_heff_.reset(new HeffPlan());
    plan_heff2(*chain_heff_, Lenv_[0], Renv_[2], theta_, bonds_[0], bonds_[2]);
  }
  return *chain_heff_;
}

Engine::~Engine() {
  if (stream_) cudaStreamSynchronize(stream_);
  site_.clear();
  Lenv_.clear();
  Renv_.clear();
  theta_.buf.reset();
  bp_heff_.reset();
  chain_heff_.reset();
  kv_.reset();
  kw_.reset();
  kpart_.reset();
  kh1_.reset();
  kh2_.reset();
  knrm_.reset();
  kstate_.reset();
  jscratch_.reset();
  if (stream_) cudaStreamSynchronize(stream_);
  for (cudaEvent_t& e : env_ev_)
    if (e) cudaEventDestroy(e);
  if (pinned_) cudaFreeHost(pinned_);
  if (dstatus_) cudaFree(dstatus_);
  if (own_stream_) cudaStreamDestroy(stream_);
}

ScratchFn Engine::jscratch() {
  return [this](size_t bytes) -> void* {
    if (jscratch_.bytes < bytes) {
      try {
        jscratch_ = DevBuf(std::max(bytes, (size_t)64 << 10), stream_);
      } catch (const Error&) {
        cudaGetLastError();
        return nullptr;
      }
    }
    return jscratch_.p;
  };
}

void Engine::check_status() {
  int hs[3] = {0, 0, 0};
  TDVP_CUDA(cudaMemcpyAsync(hs, dstatus_, 3 * sizeof(int), cudaMemcpyDeviceToHost, stream_));
  TDVP_CUDA(cudaStreamSynchronize(stream_));
  if (hs[1] != 0) throw Error(-7, "a tensor-core GEMM gave up waiting on a pipeline barrier");
  if (hs[0] != 0) throw Error(-4, "Jacobi iteration did not converge");
  if (hs[2] != 0) throw Error(-4, "Cholesky QR met a non-positive pivot (rank-deficient site tensor)");
}

void Engine::alloc(BTensor& t, bool zero) {
  t.buf = DevBuf(std::max<long long>(t.size, 1) * sizeof(cplx), stream_);
  if (zero) TDVP_CUDA(cudaMemsetAsync(t.buf.p, 0, std::max<long long>(t.size, 1) * sizeof(cplx), stream_));
}

void Engine::build_site_layout(BTensor& t, const BondSpace& l, const BondSpace& r) const {
  t = BTensor();
  t.kind = SITE;
  std::vector<std::pair<int, int>> f;
  for (int a = 0; a < (int)l.s.size(); ++a)
    for (int s = 0; s < (int)model_.site.size(); ++s) {
      model_.fuse(l.s[a].n, l.s[a].t, model_.site[s].n, model_.site[s].t, f);
      for (auto& q : f) {
        int b = r.find(q.first, q.second);
        if (b >= 0) t.add(bkey(a, s, b), a, s, b, 0, 0, l.s[a].d, r.s[b].d);
      }
    }
}

void Engine::build_theta_layout(BTensor& t, const BondSpace& l, const BondSpace& r) const {
  t = BTensor();
  t.kind = THETA;
  std::vector<std::pair<int, int>> fc, fb;
  for (int a = 0; a < (int)l.s.size(); ++a)
    for (int s1 = 0; s1 < (int)model_.site.size(); ++s1) {
      model_.fuse(l.s[a].n, l.s[a].t, model_.site[s1].n, model_.site[s1].t, fc);
      for (auto& c : fc)
        for (int s2 = 0; s2 < (int)model_.site.size(); ++s2) {
          model_.fuse(c.first, c.second, model_.site[s2].n, model_.site[s2].t, fb);
          for (auto& qb : fb) {
            int b = r.find(qb.first, qb.second);
            if (b >= 0) t.add(bkey(a, s1, c.second, s2, b), a, s1, c.second, s2, b, l.s[a].d, r.s[b].d);
          }
        }
    }
}

void Engine::build_lenv_layout(BTensor& t, const BondSpace& bra, const BondSpace& ket) const {
  t = BTensor();
  t.kind = LENV;
  std::vector<std::pair<int, int>> f;
  for (int ap = 0; ap < (int)bra.s.size(); ++ap)
    for (int w = 0; w < (int)model_.chan.size(); ++w)
      for (int a = 0; a < (int)ket.s.size(); ++a) {
        model_.fuse(ket.s[a].n, ket.s[a].t, model_.chan[w].n, model_.chan[w].t, f);
        for (auto& q : f)
          if (q.first == bra.s[ap].n && q.second == bra.s[ap].t)
            t.add(bkey(ap, w, a), ap, w, a, 0, 0, bra.s[ap].d, ket.s[a].d);
      }
}

void Engine::build_renv_layout(BTensor& t, const BondSpace& ket, const BondSpace& bra) const {
  t = BTensor();
  t.kind = RENV;
  std::vector<std::pair<int, int>> f;
  for (int b = 0; b < (int)ket.s.size(); ++b)
    for (int w = 0; w < (int)model_.chan.size(); ++w)
      for (int bp = 0; bp < (int)bra.s.size(); ++bp) {
        model_.fuse(ket.s[b].n, ket.s[b].t, model_.chan[w].n, model_.chan[w].t, f);
        for (auto& q : f)
          if (q.first == bra.s[bp].n && q.second == bra.s[bp].t)
            t.add(bkey(b, w, bp), b, w, bp, 0, 0, ket.s[b].d, bra.s[bp].d);
      }
}

void Engine::init_neel() {
  // Eq. (neel): up on even sites, down on odd sites
  std::vector<int> occ(L_);
  for (int i = 0; i < L_; ++i) occ[i] = (i % 2 == 0) ? 1 : 2;
  init_product(occ);
}

// A Fock product state, occ[i] in {0 empty, 1 up, 2 down, 3 both} (original frame).
// In the particle-hole frame c_dn -> (-1)^i c_dn^dag an up site is doubly occupied,
// a down site empty, an empty site holds a down spin and a doubly occupied site an
// up spin; U(1)xSU(2) takes only states whose frame sites are all singlets (the
// measurement there assumes a total spin 0).  Bond dimension 1 everywhere.
void Engine::init_product(const std::vector<int>& occ) {
  if ((int)occ.size() != L_) throw Error(-1, "one occupation per site");
  const bool su2 = model_.su2;
  bonds_.assign(L_ + 1, BondSpace());
  int n = 0, t = 0;
  std::vector<int> sidx(L_);
  for (int k = 0; k <= L_; ++k) {
    bonds_[k].s = {{n, t, 1}};
    bonds_[k].build_index();
    if (k == L_) break;
    int o = occ[k];
    if (o < 0 || o > 3) throw Error(-1, "occupation codes are 0 (empty), 1 (up), 2 (down), 3 (both)");
    int nn, tt, si;
    switch (o) {
      case 1: nn = 2; tt = 0; si = su2 ? 2 : 3; break;  // up -> doubly occupied
      case 2: nn = 0; tt = 0; si = 0; break;              // down -> empty
      case 0: nn = 1; tt = -1; si = 2; break;             // empty -> down spin
      default: nn = 1; tt = 1; si = 1; break;             // both -> up spin
    }
    if (su2 && nn == 1)
      throw Error(-1, "U(1)xSU(2) needs a spin singlet in the particle-hole frame: every site singly "
                      "occupied (an empty or doubly occupied site breaks it); use U(1)xU(1)");
    sidx[k] = si;
    n += nn;
    t += tt;
  }
  site_.clear();
  site_.resize(L_);
  std::vector<cplx> one(1, cplx{1.0, 0.0});
  for (int i = 0; i < L_; ++i) {
    build_site_layout(site_[i], bonds_[i], bonds_[i + 1]);
    if (site_[i].blocks.size() != 1 || site_[i].blocks[0].key[1] != sidx[i])
      throw Error(-5, "product-state layout must have the one block of the site's state");
    alloc(site_[i], false);
    TDVP_CUDA(cudaMemcpyAsync(site_[i].data(), one.data(), sizeof(cplx), cudaMemcpyHostToDevice, stream_));
  }
  Lenv_.clear();
  Renv_.clear();
  Lenv_.resize(L_ + 1);
  Renv_.resize(L_ + 1);
  build_lenv_layout(Lenv_[0], bonds_[0], bonds_[0]);
  alloc(Lenv_[0], true);
  int bi = Lenv_[0].find(bkey(0, model_.chB, 0));
  TDVP_CUDA(cudaMemcpyAsync(Lenv_[0].ptr(bi), one.data(), sizeof(cplx), cudaMemcpyHostToDevice, stream_));
  build_renv_layout(Renv_[L_], bonds_[L_], bonds_[L_]);
  alloc(Renv_[L_], true);
  bi = Renv_[L_].find(bkey(0, model_.chE, 0));
  TDVP_CUDA(cudaMemcpyAsync(Renv_[L_].ptr(bi), one.data(), sizeof(cplx), cudaMemcpyHostToDevice, stream_));
  for (int k = L_ - 1; k >= 1; --k) update_right_env(Renv_[k + 1], site_[k], Renv_[k], bonds_[k], bonds_[k + 1]);
  TDVP_CUDA(cudaStreamSynchronize(stream_));
}

// ---------------------------------------------------------------------------
// planners
// ---------------------------------------------------------------------------

// Whether BF16x4 two-site H_eff plans use packed tasks: unless TDVP_HEFF_PACKED=0
// (read at every plan), which selects the per-block task lists instead.
static bool heff_packed_enabled() {
  const char* e = std::getenv("TDVP_HEFF_PACKED");
  return !(e && e[0] == '0');
}

// BF16x4 output tile width for a task with n complex columns: n rounded up to 16 when
// n <= 64, else 64
static int packed_tile_n(int n) { return n >= 64 ? 64 : std::max(16, (n + 15) / 16 * 16); }

// Two-site H_eff as packed BF16x4 tasks (same products and recoupling as plan_heff2,
// regrouped into long GEMMs so that the tensor-core tiles are full):
//   stage 1, one task per input sector a: the left-environment blocks L(a',w,a)
//     stacked by rows (M_a = sum d_a') times the theta blocks (a,s1,c,s2,b) side by
//     side (N_a = sum d_b), K = d_a; T1 of sector a is that M_a x N_a matrix and the
//     intermediate T1(a',w,theta block) is its sub-block;
//   stage 2, the recoupling linear combination, writes T2(o,w2,b) into the stage-3
//     operand of its output column sector b' directly;
//   stage 3, one task per output column sector b': the rows of every output block o =
//     (a',s1',c',s2',b') stacked (M = sum d_a'), the (w2, b) channels of the sector
//     side by side (K = sum d_b; blocks that no recoupling term reaches stay zero),
//     times the right-environment blocks R(b,w2,b') stacked by rows (N = d_b'); the
//     output rows go back to their blocks through a row-offset table.
void Engine::plan_heff2_packed(HeffPlan& p, const BTensor& Lenv, const BTensor& Renv, const BTensor& theta,
                               const BondSpace& bl, const BondSpace& br) {
  PlanClock clk("heff2 packed total");
  static const bool pdbg = std::getenv("TDVP_PLAN_DEBUG") != nullptr;
  auto pt0 = std::chrono::steady_clock::now();
  auto pmark = [&](const char* what) {
    if (!pdbg) return;
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "plan heff2 %s %.3f ms\n", what, std::chrono::duration<double, std::milli>(now - pt0).count());
    pt0 = now;
  };
  p = HeffPlan();
  p.n = theta.size;
  const Model& M = model_;
  const int nsl = (int)bl.s.size();
  std::vector<std::vector<int>> lby(nsl), thby(nsl);
  for (int i = 0; i < (int)Lenv.blocks.size(); ++i) lby[Lenv.blocks[i].key[2]].push_back(i);
  for (int tb = 0; tb < (int)theta.blocks.size(); ++tb) thby[theta.blocks[tb].key[0]].push_back(tb);
  // stage 1 layout: T1 block per input sector a
  std::vector<long long> lrow(Lenv.blocks.size(), 0), tcol(theta.blocks.size(), 0);
  std::vector<int> t1blk(nsl, -1), t1cols(nsl, 0);
  p.t1.kind = THETA;
  for (int a = 0; a < nsl; ++a) {
    if (lby[a].empty() || thby[a].empty()) continue;
    int m = 0, n = 0;
    for (int lb : lby[a]) {
      lrow[lb] = m;
      m += Lenv.blocks[lb].rows;
    }
    for (int tb : thby[a]) {
      tcol[tb] = n;
      n += theta.blocks[tb].cols;
    }
    t1blk[a] = (int)p.t1.blocks.size();
    t1cols[a] = n;
    p.t1.add((uint64_t)a, a, 0, 0, 0, 0, m, n);
  }
  alloc(p.t1, false);
  // T1 views, in the order of plan_heff2 (theta block, then L block)
  struct T1View {
    int lb, tb;
    cplx* ptr;
    int ld;
  };
  std::vector<T1View> t1v;
  for (int tb = 0; tb < (int)theta.blocks.size(); ++tb) {
    const int a = theta.blocks[tb].key[0];
    if (t1blk[a] < 0) continue;
    for (int lb : lby[a])
      t1v.push_back({lb, tb, p.t1.ptr(t1blk[a]) + lrow[lb] * t1cols[a] + tcol[tb], t1cols[a]});
  }
  for (int a = 0; a < nsl; ++a) {
    if (t1blk[a] < 0) continue;
    const Block& tb1 = p.t1.blocks[t1blk[a]];
    GemmTask t{};
    t.c = p.t1.ptr(t1blk[a]);
    t.c_base = 0;
    t.rows = tb1.rows;
    t.cols = tb1.cols;
    t.ldc = tb1.cols;
    t.tn = packed_tile_n(tb1.cols);
    t.seg_begin = (int)p.g1.segs.size();
    t.seg_count = 1;
    GemmSeg sg{};
    sg.k = bl.s[a].d;
    sg.alpha = 1.0;
    p.g1.segs.push_back(sg);
    PackedTask pk;
    pk.a_static = true;
    pk.b_static = false;
    for (int lb : lby[a]) {
      const Block& lk = Lenv.blocks[lb];
      pk.a.push_back({Lenv.ptr(lb), 0, lk.rows, lk.cols, lk.cols, OP_N, 1.0, (int)lrow[lb], 0});
    }
    for (int tb : thby[a]) {
      const Block& th = theta.blocks[tb];
      pk.b.push_back({as_off(th.off), 1, th.rows, th.cols, th.cols, OP_N, 1.0, 0, (int)tcol[tb]});
      for (int lb : lby[a]) p.g1.flops += 8LL * Lenv.blocks[lb].rows * th.rows * th.cols;
    }
    p.g1.packed.push_back(std::move(pk));
    p.g1.tasks.push_back(t);
  }
  pmark("stage 1");
  // stage 2: recoupling terms (as plan_heff2).  The output sector b' of a term and the
  // existence of R(b, w2, b') depend on (b, w2, 2S_b') alone: a table filled on first use.
  int tmin = 0, tmax = -1;
  for (int k = 0; k < (int)br.s.size(); ++k) {
    tmin = k ? std::min(tmin, br.s[k].t) : br.s[k].t;
    tmax = k ? std::max(tmax, br.s[k].t) : br.s[k].t;
  }
  const int nch = (int)M.chan.size(), tl = tmax - tmin + 1;
  const bool tabled = tl > 0 && (long long)br.s.size() * nch * tl <= (1LL << 24);
  std::vector<int> bpc(tabled ? (size_t)br.s.size() * nch * tl : 0, -2);
  auto target = [&](int b, int w2, int tbp) {
    int* c = nullptr;
    if (tabled) {
      if (tbp < tmin || tbp > tmax) return -1;  // no sector of br has that spin
      c = &bpc[((size_t)b * nch + w2) * tl + (tbp - tmin)];
      if (*c != -2) return *c;
    }
    int bp = br.find(br.s[b].n + M.chan[w2].n, tbp);
    if (bp >= 0 && Renv.find(bkey(b, w2, bp)) < 0) bp = -1;
    if (c) *c = bp;
    return bp;
  };
  std::unordered_map<uint64_t, int> t2idx;
  std::vector<std::vector<std::pair<int, double>>> t2terms;
  std::vector<std::array<int, 7>> t2keys;
  long long nterm = 0;
  // the views of one theta block come together, and their terms depend on (2S_a', w) alone
  int memo_tb = -1;
  std::vector<std::tuple<int, int, const std::vector<Recouple2>*>> memo;
  for (int i = 0; i < (int)t1v.size(); ++i) {
    const Block& lk = Lenv.blocks[t1v[i].lb];
    const Block& th = theta.blocks[t1v[i].tb];
    int ap = lk.key[0], w = lk.key[1], a = th.key[0], s1 = th.key[1], tc = th.key[2], s2 = th.key[3], b = th.key[4];
    if (t1v[i].tb != memo_tb) {
      memo.clear();
      memo_tb = t1v[i].tb;
    }
    const std::vector<Recouple2>* rcp = nullptr;
    for (const auto& m : memo)
      if (std::get<0>(m) == bl.s[ap].t && std::get<1>(m) == w) {
        rcp = std::get<2>(m);
        break;
      }
    if (!rcp) {
      rcp = &rec_->two_site(bl.s[ap].t, w, bl.s[a].t, s1, tc, s2, br.s[b].t);
      memo.emplace_back(bl.s[ap].t, w, rcp);
    }
    const auto& rc = *rcp;
    nterm += (long long)rc.size();
    for (const auto& e : rc) {
      const int bp = target(b, e.w2, e.tbp);
      if (bp < 0) continue;
      const int nbp = br.s[bp].n;
      if (bl.s[ap].n + M.site[e.s1p].n + M.site[e.s2p].n != nbp) throw Error(-5, "charge mismatch in recoupling");
      const uint64_t key = t2key(ap, e.s1p, e.tcp, e.s2p, bp, e.w2, b);
      auto it = t2idx.find(key);
      int id;
      if (it == t2idx.end()) {
        id = (int)t2keys.size();
        t2idx[key] = id;
        t2keys.push_back({ap, e.s1p, e.tcp, e.s2p, bp, e.w2, b});
        t2terms.emplace_back();
      } else {
        id = it->second;
      }
      t2terms[id].push_back({i, e.f});
    }
  }
  if (pdbg)
    std::fprintf(stderr, "plan heff2 %zu T1 views, %lld recoupling terms, %zu T2 blocks\n", t1v.size(), nterm,
                 t2keys.size());
  pmark("stage 2");
  // stage 3 grouping by output column sector b'
  const int nsr = (int)br.s.size();
  std::vector<std::vector<int>> oby(nsr);  // output (theta) blocks by right sector
  for (int ob = 0; ob < (int)theta.blocks.size(); ++ob) oby[theta.blocks[ob].key[4]].push_back(ob);
  std::vector<long long> orow(theta.blocks.size(), 0);
  // the (w2, b) channels of each output column sector, in increasing (w2, b) order, at
  // column offsets segoff[bp][j]; colof[id] is the column offset of T2 block id
  std::vector<std::vector<std::pair<int, int>>> segcol(nsr);
  std::vector<std::vector<int>> segoff(nsr);
  std::vector<int> gk(nsr, 0), gm(nsr, 0), t2g(nsr, -1), colof(t2keys.size(), 0), obof(t2keys.size(), -1);
  for (int bp = 0; bp < nsr; ++bp) {
    int m = 0;
    for (int ob : oby[bp]) {
      orow[ob] = m;
      m += theta.blocks[ob].rows;
    }
    gm[bp] = m;
  }
  if (nch >= (1 << 8) || nsr >= (1 << 24)) throw Error(-5, "too many sectors or channels for the stage-3 layout");
  auto chkey = [](int bp, int w2, int b) { return ((uint64_t)bp << 32) | ((uint64_t)w2 << 24) | (uint64_t)b; };
  {
    std::unordered_map<uint64_t, int> seen;
    seen.reserve(2 * t2keys.size() + 16);
    for (const auto& k : t2keys)
      if (seen.emplace(chkey(k[4], k[5], k[6]), 0).second) segcol[k[4]].push_back({k[5], k[6]});
    for (int bp = 0; bp < nsr; ++bp) {
      std::sort(segcol[bp].begin(), segcol[bp].end());
      int kk = 0;
      for (const auto& e : segcol[bp]) {
        segoff[bp].push_back(kk);
        seen[chkey(bp, e.first, e.second)] = kk;
        kk += br.s[e.second].d;
      }
      gk[bp] = kk;
    }
    for (int id = 0; id < (int)t2keys.size(); ++id) {
      const auto& k = t2keys[id];
      colof[id] = seen.at(chkey(k[4], k[5], k[6]));
      obof[id] = theta.find(bkey(k[0], k[1], k[2], k[3], k[4]));
    }
  }
  p.t2.kind = THETA;
  for (int bp = 0; bp < nsr; ++bp)
    if (gm[bp] > 0 && gk[bp] > 0) {
      t2g[bp] = (int)p.t2.blocks.size();
      p.t2.add((uint64_t)bp, bp, 0, 0, 0, 0, gm[bp], gk[bp]);
    }
  alloc(p.t2, true);  // (o, w2, b) blocks that no term reaches stay zero
  std::vector<cplx*> t2ptr(t2keys.size());
  for (int id = 0; id < (int)t2keys.size(); ++id) {
    const auto& k = t2keys[id];
    const int bp = k[4];
    const int ob = obof[id];
    if (ob < 0) throw Error(-5, "recoupled block outside the two-site layout");
    t2ptr[id] = p.t2.ptr(t2g[bp]) + orow[ob] * gk[bp] + colof[id];
    LincombTask t{};
    t.out = t2ptr[id];
    t.rows = bl.s[k[0]].d;
    t.cols = br.s[k[6]].d;
    t.ld_out = gk[bp];
    t.term_begin = (int)p.lc.terms.size();
    t.term_count = (int)t2terms[id].size();
    for (auto& tm : t2terms[id]) p.lc.terms.push_back({t1v[tm.first].ptr, t1v[tm.first].ld, tm.second});
    p.lc.tasks.push_back(t);
    p.lc.bytes += (long long)sizeof(cplx) * t.rows * t.cols * (1 + t.term_count);
  }
  // stage 3 tasks
  for (int bp = 0; bp < nsr; ++bp) {
    if (oby[bp].empty()) continue;
    GemmTask t{};
    t.c = nullptr;
    t.c_base = 2;
    t.rows = gm[bp];
    t.cols = br.s[bp].d;
    t.ldc = t.cols;
    t.tn = packed_tile_n(t.cols);
    t.seg_begin = (int)p.g3.segs.size();
    t.seg_count = 1;
    p.g3.row_start.resize(p.g3.tasks.size() + 1, -1);
    p.g3.row_start.back() = (long long)p.g3.rowoffs.size();
    for (int ob : oby[bp]) {
      const Block& o = theta.blocks[ob];
      for (int r = 0; r < o.rows; ++r) p.g3.rowoffs.push_back(o.off + (long long)r * o.cols);
    }
    GemmSeg sg{};
    sg.k = t2g[bp] >= 0 ? gk[bp] : 0;
    sg.alpha = 1.0;
    p.g3.segs.push_back(sg);
    PackedTask pk;
    pk.a_static = false;
    pk.b_static = true;
    if (t2g[bp] >= 0) {
      for (size_t j = 0; j < segcol[bp].size(); ++j) {
        const int w2 = segcol[bp][j].first, b = segcol[bp][j].second;
        const int rb = Renv.find(bkey(b, w2, bp));
        const Block& rk = Renv.blocks[rb];
        pk.b.push_back({Renv.ptr(rb), 0, rk.rows, rk.cols, rk.cols, OP_N, 1.0, segoff[bp][j], 0});
      }
    }
    p.g3.packed.push_back(std::move(pk));
    p.g3.tasks.push_back(t);
    p.g3.out_blocks.push_back(oby[bp]);
    p.g3.task_flops.push_back(0);
  }
  std::vector<int> task_of(nsr, -1);  // output column sector -> stage-3 task
  {
    int ti = 0;
    for (int bp = 0; bp < nsr; ++bp)
      if (!oby[bp].empty()) task_of[bp] = ti++;
    for (int id = 0; id < (int)t2keys.size(); ++id) {
      const auto& k = t2keys[id];
      const int bp = k[4];
      const int ob = obof[id];
      const int rows = bl.s[k[0]].d, cols = br.s[k[6]].d;
      p.g3.packed[task_of[bp]].a.push_back({t2ptr[id], 0, rows, cols, gk[bp], OP_N, 1.0, (int)orow[ob], colof[id]});
      p.g3.flops += 8LL * rows * cols * br.s[bp].d;
      p.g3.task_flops[task_of[bp]] += 8LL * rows * cols * br.s[bp].d;
    }
  }
  pmark("stage 3");
  p.g1.finalize(stream_, gemm_kind_, dstatus_ + 1);
  p.g3.dyn_tags_external = true;
  p.g3.finalize(stream_, gemm_kind_, dstatus_ + 1);
  // the linear combination raises the exponent tags of the stage-3 operand's rows
  for (int id = 0; id < (int)t2keys.size(); ++id)
    p.lc.tasks[id].tags = p.g3.tags() + p.g3.tasks[task_of[t2keys[id][4]]].roff + orow[obof[id]];
  p.lc.finalize(stream_);
}

void Engine::plan_heff2(HeffPlan& p, const BTensor& Lenv, const BTensor& Renv, const BTensor& theta,
                        const BondSpace& bl, const BondSpace& br) {
  if (gemm_kind_ == 1 && heff_packed_enabled()) {
    plan_heff2_packed(p, Lenv, Renv, theta, bl, br);
    return;
  }
  p = HeffPlan();
  p.n = theta.size;
  const Model& M = model_;
  std::vector<std::vector<int>> lby(bl.s.size());
  for (int i = 0; i < (int)Lenv.blocks.size(); ++i) lby[Lenv.blocks[i].key[2]].push_back(i);
  // step 1 layout: T1(a',w,a,s1,c,s2,b) = L(a',w,a) theta(a,s1,c,s2,b)
  struct T1Info {
    int lb, tb;
  };
  std::vector<T1Info> t1info;
  p.t1.kind = THETA;
  for (int tb = 0; tb < (int)theta.blocks.size(); ++tb) {
    const Block& th = theta.blocks[tb];
    for (int lb : lby[th.key[0]]) {
      const Block& lk = Lenv.blocks[lb];
      p.t1.add((uint64_t)t1info.size(), lk.key[0], lk.key[1], tb, 0, 0, lk.rows, th.cols);
      t1info.push_back({lb, tb});
    }
  }
  alloc(p.t1, false);
  for (int i = 0; i < (int)t1info.size(); ++i) {
    const Block& lk = Lenv.blocks[t1info[i].lb];
    const Block& th = theta.blocks[t1info[i].tb];
    GemmTask t{};
    t.c = p.t1.ptr(i);
    t.c_base = 0;
    t.rows = lk.rows;
    t.cols = th.cols;
    t.ldc = th.cols;
    t.seg_begin = (int)p.g1.segs.size();
    t.seg_count = 1;
    GemmSeg sg{};
    sg.a = Lenv.ptr(t1info[i].lb);
    sg.a_static = 1;
    sg.a_base = 0;
    sg.lda = lk.cols;
    sg.b = as_off(th.off);
    sg.b_base = 1;
    sg.ldb = th.cols;
    sg.k = lk.cols;
    sg.op_a = OP_N;
    sg.op_b = OP_N;
    sg.alpha = 1.0;
    p.g1.segs.push_back(sg);
    p.g1.tasks.push_back(t);
    p.g1.flops += 8LL * lk.rows * lk.cols * th.cols;
  }
  // step 2: recoupling into T2(a',s1',c',s2',b',w2,b)
  std::unordered_map<uint64_t, int> t2idx;
  std::vector<std::vector<std::pair<int, double>>> t2terms;
  std::vector<std::array<int, 7>> t2keys;
  for (int i = 0; i < (int)t1info.size(); ++i) {
    const Block& lk = Lenv.blocks[t1info[i].lb];
    const Block& th = theta.blocks[t1info[i].tb];
    int ap = lk.key[0], w = lk.key[1], a = th.key[0], s1 = th.key[1], tc = th.key[2], s2 = th.key[3], b = th.key[4];
    const auto& rc = rec_->two_site(bl.s[ap].t, w, bl.s[a].t, s1, tc, s2, br.s[b].t);
    for (const auto& e : rc) {
      int nbp = br.s[b].n + M.chan[e.w2].n;
      int bp = br.find(nbp, e.tbp);
      if (bp < 0) continue;
      if (Renv.find(bkey(b, e.w2, bp)) < 0) continue;
      if (bl.s[ap].n + M.site[e.s1p].n + M.site[e.s2p].n != nbp) throw Error(-5, "charge mismatch in recoupling");
      const uint64_t key = t2key(ap, e.s1p, e.tcp, e.s2p, bp, e.w2, b);
      auto it = t2idx.find(key);
      int id;
      if (it == t2idx.end()) {
        id = (int)t2keys.size();
        t2idx[key] = id;
        t2keys.push_back({ap, e.s1p, e.tcp, e.s2p, bp, e.w2, b});
        t2terms.emplace_back();
        p.t2.add((uint64_t)id, ap, e.s1p, e.tcp, e.s2p, bp, bl.s[ap].d, br.s[b].d);
      } else {
        id = it->second;
      }
      t2terms[id].push_back({i, e.f});
    }
  }
  alloc(p.t2, false);
  for (int id = 0; id < (int)t2keys.size(); ++id) {
    const Block& bk = p.t2.blocks[id];
    LincombTask t{};
    t.out = p.t2.ptr(id);
    t.rows = bk.rows;
    t.cols = bk.cols;
    t.ld_out = bk.cols;
    t.term_begin = (int)p.lc.terms.size();
    t.term_count = (int)t2terms[id].size();
    for (auto& tm : t2terms[id]) p.lc.terms.push_back({p.t1.ptr(tm.first), p.t1.blocks[tm.first].cols, tm.second});
    p.lc.tasks.push_back(t);
    p.lc.bytes += (long long)sizeof(cplx) * bk.rows * bk.cols * (1 + t.term_count);
  }
  // step 3: theta'(a',s1',c',s2',b') = sum_{w2,b} T2 R(b,w2,b')
  IntArrayMap<5, std::vector<int>> outsegs;
  for (int id = 0; id < (int)t2keys.size(); ++id) {
    auto& k = t2keys[id];
    outsegs[{k[0], k[1], k[2], k[3], k[4]}].push_back(id);
  }
  for (int ob = 0; ob < (int)theta.blocks.size(); ++ob) {
    const Block& o = theta.blocks[ob];
    GemmTask t{};
    t.c = as_off(o.off);
    t.c_base = 2;
    t.rows = o.rows;
    t.cols = o.cols;
    t.ldc = o.cols;
    t.seg_begin = (int)p.g3.segs.size();
    auto it = outsegs.find({o.key[0], o.key[1], o.key[2], o.key[3], o.key[4]});
    int cnt = 0;
    long long tf = 0;
    if (it != outsegs.end()) {
      for (int id : it->second) {
        auto& k = t2keys[id];
        int rb = Renv.find(bkey(k[6], k[5], k[4]));
        const Block& rk = Renv.blocks[rb];
        GemmSeg sg{};
        sg.a = p.t2.ptr(id);
        sg.a_base = 0;
        sg.lda = p.t2.blocks[id].cols;
        sg.b = Renv.ptr(rb);
        sg.b_static = 1;
        sg.b_base = 0;
        sg.ldb = rk.cols;
        sg.k = rk.rows;
        sg.op_a = OP_N;
        sg.op_b = OP_N;
        sg.alpha = 1.0;
        p.g3.segs.push_back(sg);
        p.g3.flops += 8LL * o.rows * rk.rows * rk.cols;
        tf += 8LL * o.rows * rk.rows * rk.cols;
        ++cnt;
      }
    }
    t.seg_count = cnt;
    p.g3.tasks.push_back(t);
    p.g3.out_blocks.push_back({ob});
    p.g3.task_flops.push_back(tf);
  }
  p.g1.finalize(stream_, gemm_kind_, dstatus_ + 1);
  p.lc.finalize(stream_);
  p.g3.finalize(stream_, gemm_kind_, dstatus_ + 1);
}

// shared by the one-site H_eff and the left-environment update: steps 1 and 2
// T1(a',w,a,s,b) = L(a',w,a) X(a,s,b);  T2(a',s',b'',w',b) = sum f T1
// keep(a', s', b'', w', b) decides whether an output is needed.
template <class Keep>
static void plan_l_w(Engine* eng, const Model& M, Recoupler& rec, HeffPlan& p, const BTensor& Lenv, const BTensor& X,
                     const BondSpace& bl, const BondSpace& br, Keep keep,
                     std::vector<std::array<int, 5>>& t2keys, cudaStream_t s,
                     void (Engine::*alloc_fn)(BTensor&, bool)) {
  std::vector<std::vector<int>> lby(bl.s.size());
  for (int i = 0; i < (int)Lenv.blocks.size(); ++i) lby[Lenv.blocks[i].key[2]].push_back(i);
  std::vector<std::pair<int, int>> info;
  for (int xb = 0; xb < (int)X.blocks.size(); ++xb) {
    const Block& x = X.blocks[xb];
    for (int lb : lby[x.key[0]]) {
      const Block& lk = Lenv.blocks[lb];
      p.t1.add((uint64_t)info.size(), lk.key[0], lk.key[1], xb, 0, 0, lk.rows, x.cols);
      info.push_back({lb, xb});
    }
  }
  (eng->*alloc_fn)(p.t1, false);
  for (int i = 0; i < (int)info.size(); ++i) {
    const Block& lk = Lenv.blocks[info[i].first];
    const Block& x = X.blocks[info[i].second];
    GemmTask t{};
    t.c = p.t1.ptr(i);
    t.rows = lk.rows;
    t.cols = x.cols;
    t.ldc = x.cols;
    t.seg_begin = (int)p.g1.segs.size();
    t.seg_count = 1;
    GemmSeg sg{};
    sg.a = Lenv.ptr(info[i].first);
    sg.a_static = 1;
    sg.lda = lk.cols;
    sg.b = as_off(x.off);
    sg.b_base = 1;
    sg.ldb = x.cols;
    sg.k = lk.cols;
    sg.alpha = 1.0;
    p.g1.segs.push_back(sg);
    p.g1.tasks.push_back(t);
    p.g1.flops += 8LL * lk.rows * lk.cols * x.cols;
  }
  IntArrayMap<5, int> idx;
  idx.reserve(4 * info.size() + 16);
  std::vector<std::vector<std::pair<int, double>>> terms;
  for (int i = 0; i < (int)info.size(); ++i) {
    const Block& lk = Lenv.blocks[info[i].first];
    const Block& x = X.blocks[info[i].second];
    int ap = lk.key[0], w = lk.key[1], a = x.key[0], sx = x.key[1], b = x.key[2];
    const auto& rc = rec.one_site(bl.s[ap].t, w, bl.s[a].t, sx, br.s[b].t);
    for (const auto& e : rc) {
      int nbpp = bl.s[ap].n + M.site[e.sp].n;
      int bpp = br.find(nbpp, e.tbpp);
      if (bpp < 0) continue;
      if (br.s[b].n + M.chan[e.wp].n != nbpp) throw Error(-5, "charge mismatch in one-site recoupling");
      std::array<int, 5> key{ap, e.sp, bpp, e.wp, b};
      if (!keep(key)) continue;
      auto it = idx.find(key);
      int id;
      if (it == idx.end()) {
        id = (int)t2keys.size();
        idx[key] = id;
        t2keys.push_back(key);
        terms.emplace_back();
        p.t2.add((uint64_t)id, ap, e.sp, bpp, e.wp, b, bl.s[ap].d, br.s[b].d);
      } else {
        id = it->second;
      }
      terms[id].push_back({i, e.f});
    }
  }
  (eng->*alloc_fn)(p.t2, false);
  for (int id = 0; id < (int)t2keys.size(); ++id) {
    const Block& bk = p.t2.blocks[id];
    LincombTask t{};
    t.out = p.t2.ptr(id);
    t.rows = bk.rows;
    t.cols = bk.cols;
    t.ld_out = bk.cols;
    t.term_begin = (int)p.lc.terms.size();
    t.term_count = (int)terms[id].size();
    for (auto& tm : terms[id]) p.lc.terms.push_back({p.t1.ptr(tm.first), p.t1.blocks[tm.first].cols, tm.second});
    p.lc.tasks.push_back(t);
    p.lc.bytes += (long long)sizeof(cplx) * bk.rows * bk.cols * (1 + t.term_count);
  }
  (void)s;
}

void Engine::plan_heff1(HeffPlan& p, const BTensor& Lenv, const BTensor& Renv, const BTensor& Mt, const BondSpace& bl,
                        const BondSpace& br) {
  PlanClock clk("heff1 total");
  p = HeffPlan();
  p.n = Mt.size;
  std::vector<std::array<int, 5>> t2keys;
  auto keep = [&](const std::array<int, 5>& k) {
    return Renv.find(bkey(k[4], k[3], k[2])) >= 0 && Mt.find(bkey(k[0], k[1], k[2])) >= 0;
  };
  plan_l_w(this, model_, *rec_, p, Lenv, Mt, bl, br, keep, t2keys, stream_, &Engine::alloc);
  IntArrayMap<3, std::vector<int>> outsegs;
  for (int id = 0; id < (int)t2keys.size(); ++id) outsegs[{t2keys[id][0], t2keys[id][1], t2keys[id][2]}].push_back(id);
  for (int ob = 0; ob < (int)Mt.blocks.size(); ++ob) {
    const Block& o = Mt.blocks[ob];
    GemmTask t{};
    t.c = as_off(o.off);
    t.c_base = 2;
    t.rows = o.rows;
    t.cols = o.cols;
    t.ldc = o.cols;
    t.seg_begin = (int)p.g3.segs.size();
    int cnt = 0;
    auto it = outsegs.find({o.key[0], o.key[1], o.key[2]});
    if (it != outsegs.end())
      for (int id : it->second) {
        auto& k = t2keys[id];
        int rb = Renv.find(bkey(k[4], k[3], k[2]));
        const Block& rk = Renv.blocks[rb];
        GemmSeg sg{};
        sg.a = p.t2.ptr(id);
        sg.lda = p.t2.blocks[id].cols;
        sg.b = Renv.ptr(rb);
        sg.b_static = 1;
        sg.ldb = rk.cols;
        sg.k = rk.rows;
        sg.alpha = 1.0;
        p.g3.segs.push_back(sg);
        p.g3.flops += 8LL * o.rows * rk.rows * rk.cols;
        ++cnt;
      }
    t.seg_count = cnt;
    p.g3.tasks.push_back(t);
  }
  p.g1.finalize(stream_, gemm_kind_, dstatus_ + 1);
  p.lc.finalize(stream_);
  p.g3.finalize(stream_, gemm_kind_, dstatus_ + 1);
}

void Engine::update_left_env(const BTensor& Lin, const BTensor& A, BTensor& Lout, const BondSpace& bl,
                             const BondSpace& br) {
  NvtxRange nvtx_range("env_update");
  build_lenv_layout(Lout, br, br);
  alloc(Lout, false);
  HeffPlan p;
  std::vector<std::array<int, 5>> t2keys;
  // T2(a',s',b'',w',b) is needed when L'(b'',w',b) exists and A(a',s',b'') exists
  auto keep = [&](const std::array<int, 5>& k) {
    return Lout.find(bkey(k[2], k[3], k[4])) >= 0 && A.find(bkey(k[0], k[1], k[2])) >= 0;
  };
  plan_l_w(this, model_, *rec_, p, Lin, A, bl, br, keep, t2keys, stream_, &Engine::alloc);
  IntArrayMap<3, std::vector<int>> outsegs;  // (b'', w', b)
  for (int id = 0; id < (int)t2keys.size(); ++id) outsegs[{t2keys[id][2], t2keys[id][3], t2keys[id][4]}].push_back(id);
  for (int ob = 0; ob < (int)Lout.blocks.size(); ++ob) {
    const Block& o = Lout.blocks[ob];
    GemmTask t{};
    t.c = Lout.ptr(ob);
    t.rows = o.rows;
    t.cols = o.cols;
    t.ldc = o.cols;
    t.seg_begin = (int)p.g3.segs.size();
    int cnt = 0;
    auto it = outsegs.find({o.key[0], o.key[1], o.key[2]});
    if (it != outsegs.end())
      for (int id : it->second) {
        auto& k = t2keys[id];
        int ab = A.find(bkey(k[0], k[1], k[2]));
        const Block& ak = A.blocks[ab];
        GemmSeg sg{};
        sg.a = A.ptr(ab);
        sg.lda = ak.cols;
        sg.op_a = OP_C;
        sg.b = p.t2.ptr(id);
        sg.ldb = p.t2.blocks[id].cols;
        sg.k = ak.rows;
        sg.alpha = 1.0;
        p.g3.segs.push_back(sg);
        p.g3.flops += 8LL * o.rows * ak.rows * o.cols;
        ++cnt;
      }
    t.seg_count = cnt;
    p.g3.tasks.push_back(t);
  }
  p.g1.finalize(stream_, gemm_kind_, dstatus_ + 1);
  p.lc.finalize(stream_);
  p.g3.finalize(stream_, gemm_kind_, dstatus_ + 1);
  Bases4 B{{0, reinterpret_cast<uintptr_t>(A.data()), 0, 0}};
  p.g1.launch(stream_, B);
  p.lc.launch(stream_);
  p.g3.launch(stream_, B);
  stats_.env_flops += p.g1.flops + p.g3.flops;
  stats_.env_bytes += (double)(p.g1.bytes + p.lc.bytes + p.g3.bytes);
}

void Engine::update_right_env(const BTensor& Rin, const BTensor& Bt, BTensor& Rout, const BondSpace& bl,
                              const BondSpace& br) {
  NvtxRange nvtx_range("env_update");
  const Model& M = model_;
  build_renv_layout(Rout, bl, bl);
  alloc(Rout, false);
  HeffPlan p;
  std::vector<std::vector<int>> rby(br.s.size());
  for (int i = 0; i < (int)Rin.blocks.size(); ++i) rby[Rin.blocks[i].key[0]].push_back(i);
  // step 1: F1(a,s,b,w',b') = B(a,s,b) R(b,w',b')
  std::vector<std::pair<int, int>> info;
  for (int xb = 0; xb < (int)Bt.blocks.size(); ++xb) {
    const Block& x = Bt.blocks[xb];
    for (int rb : rby[x.key[2]]) {
      const Block& rk = Rin.blocks[rb];
      p.t1.add((uint64_t)info.size(), xb, rk.key[1], rk.key[2], 0, 0, x.rows, rk.cols);
      info.push_back({xb, rb});
    }
  }
  alloc(p.t1, false);
  for (int i = 0; i < (int)info.size(); ++i) {
    const Block& x = Bt.blocks[info[i].first];
    const Block& rk = Rin.blocks[info[i].second];
    GemmTask t{};
    t.c = p.t1.ptr(i);
    t.rows = x.rows;
    t.cols = rk.cols;
    t.ldc = rk.cols;
    t.seg_begin = (int)p.g1.segs.size();
    t.seg_count = 1;
    GemmSeg sg{};
    sg.a = Bt.ptr(info[i].first);
    sg.lda = x.cols;
    sg.b = Rin.ptr(info[i].second);
    sg.ldb = rk.cols;
    sg.k = x.cols;
    sg.alpha = 1.0;
    p.g1.segs.push_back(sg);
    p.g1.tasks.push_back(t);
    p.g1.flops += 8LL * x.rows * x.cols * rk.cols;
  }
  // step 2: F2(a,w,a'',s',b')
  IntArrayMap<5, int> idx;
  idx.reserve(4 * info.size() + 16);
  std::vector<std::array<int, 5>> keys;
  std::vector<std::vector<std::pair<int, double>>> terms;
  for (int i = 0; i < (int)info.size(); ++i) {
    const Block& x = Bt.blocks[info[i].first];
    const Block& rk = Rin.blocks[info[i].second];
    int a = x.key[0], s = x.key[1], b = x.key[2], wp = rk.key[1], bp = rk.key[2];
    const auto& rc = rec_->right_env(bl.s[a].t, s, br.s[b].t, wp, br.s[bp].t);
    for (const auto& e : rc) {
      int napp = bl.s[a].n + M.chan[e.w].n;
      int app = bl.find(napp, e.tapp);
      if (app < 0) continue;
      if (Rout.find(bkey(a, e.w, app)) < 0) continue;
      if (Bt.find(bkey(app, e.sp, bp)) < 0) continue;
      std::array<int, 5> key{a, e.w, app, e.sp, bp};
      auto it = idx.find(key);
      int id;
      if (it == idx.end()) {
        id = (int)keys.size();
        idx[key] = id;
        keys.push_back(key);
        terms.emplace_back();
        p.t2.add((uint64_t)id, a, e.w, app, e.sp, bp, bl.s[a].d, br.s[bp].d);
      } else {
        id = it->second;
      }
      terms[id].push_back({i, e.f});
    }
  }
  alloc(p.t2, false);
  for (int id = 0; id < (int)keys.size(); ++id) {
    const Block& bk = p.t2.blocks[id];
    LincombTask t{};
    t.out = p.t2.ptr(id);
    t.rows = bk.rows;
    t.cols = bk.cols;
    t.ld_out = bk.cols;
    t.term_begin = (int)p.lc.terms.size();
    t.term_count = (int)terms[id].size();
    for (auto& tm : terms[id]) p.lc.terms.push_back({p.t1.ptr(tm.first), p.t1.blocks[tm.first].cols, tm.second});
    p.lc.tasks.push_back(t);
  }
  // step 3: R'(a,w,a'') = sum_{s',b'} F2(a,w,a'',s',b') B(a'',s',b')^H
  IntArrayMap<3, std::vector<int>> outsegs;
  for (int id = 0; id < (int)keys.size(); ++id) outsegs[{keys[id][0], keys[id][1], keys[id][2]}].push_back(id);
  for (int ob = 0; ob < (int)Rout.blocks.size(); ++ob) {
    const Block& o = Rout.blocks[ob];
    GemmTask t{};
    t.c = Rout.ptr(ob);
    t.rows = o.rows;
    t.cols = o.cols;
    t.ldc = o.cols;
    t.seg_begin = (int)p.g3.segs.size();
    int cnt = 0;
    auto it = outsegs.find({o.key[0], o.key[1], o.key[2]});
    if (it != outsegs.end())
      for (int id : it->second) {
        auto& k = keys[id];
        int bb = Bt.find(bkey(k[2], k[3], k[4]));
        const Block& bk = Bt.blocks[bb];
        GemmSeg sg{};
        sg.a = p.t2.ptr(id);
        sg.lda = p.t2.blocks[id].cols;
        sg.b = Bt.ptr(bb);
        sg.ldb = bk.cols;
        sg.op_b = OP_C;
        sg.k = bk.cols;
        sg.alpha = 1.0;
        p.g3.segs.push_back(sg);
        p.g3.flops += 8LL * o.rows * bk.cols * o.cols;
        ++cnt;
      }
    t.seg_count = cnt;
    p.g3.tasks.push_back(t);
  }
  p.g1.finalize(stream_, gemm_kind_, dstatus_ + 1);
  p.lc.finalize(stream_);
  p.g3.finalize(stream_, gemm_kind_, dstatus_ + 1);
  Bases4 B{{0, 0, 0, 0}};
  p.g1.launch(stream_, B);
  p.lc.launch(stream_);
  p.g3.launch(stream_, B);
  stats_.env_flops += p.g1.flops + p.g3.flops;
  stats_.env_bytes += (double)(p.g1.bytes + p.lc.bytes + p.g3.bytes);
}

void Engine::form_theta(const BTensor& X, const BTensor& Y, BTensor& theta, const BondSpace& bl, const BondSpace& bm,
                        const BondSpace& br) {
  build_theta_layout(theta, bl, br);
  alloc(theta, true);
  GemmPlan g;
  std::vector<std::vector<int>> yby(bm.s.size());
  for (int i = 0; i < (int)Y.blocks.size(); ++i) yby[Y.blocks[i].key[0]].push_back(i);
  for (int xi = 0; xi < (int)X.blocks.size(); ++xi) {
    const Block& x = X.blocks[xi];
    for (int yi : yby[x.key[2]]) {
      const Block& y = Y.blocks[yi];
      int tb = theta.find(bkey(x.key[0], x.key[1], bm.s[x.key[2]].t, y.key[1], y.key[2]));
      if (tb < 0) throw Error(-5, "theta block missing");
      GemmTask t{};
      t.c = theta.ptr(tb);
      t.rows = x.rows;
      t.cols = y.cols;
      t.ldc = y.cols;
      t.seg_begin = (int)g.segs.size();
      t.seg_count = 1;
      GemmSeg sg{};
      sg.a = X.ptr(xi);
      sg.lda = x.cols;
      sg.b = Y.ptr(yi);
      sg.ldb = y.cols;
      sg.k = x.cols;
      sg.alpha = 1.0;
      g.segs.push_back(sg);
      g.tasks.push_back(t);
    }
  }
  g.finalize(stream_, gemm_kind_, dstatus_ + 1);
  g.launch(stream_, Bases4{{0, 0, 0, 0}});
}

// ---------------------------------------------------------------------------
// Krylov exponential: x <- exp(-i tau H) x  (Sec. S2.2, Lanczos with full
// re-orthogonalisation applied twice, adaptive dimension)
// ---------------------------------------------------------------------------

void Engine::krylov(HeffPlan& H, cplx* x, double tau, int* k, int* launches) {
  int kd = expm(H, x, tau);
  if (k) *k = kd;
  // 4 set-up launches, 13 per Lanczos iteration (3 H_eff + 6 dots + 2 axpy + step + scale), 1 combine
  if (launches) *launches = 4 + 13 * kd + 1;
}

int Engine::expm(HeffPlan& H, cplx* x, double tau) {
  NvtxRange nvtx_range("krylov");
  const long long n = H.n;
  const int kmax = opt_.krylov_max;
  if (kcap_ < n) {
    kv_ = DevBuf((size_t)(kmax + 1) * n * sizeof(cplx), stream_);
    kw_ = DevBuf((size_t)n * sizeof(cplx), stream_);
    kcap_ = n;
  }
  if (!kpart_.p) {
    kpart_ = DevBuf((size_t)(KRYLOV_MAX + 1) * 296 * sizeof(cplx), stream_);
    kh1_ = DevBuf((KRYLOV_MAX + 1) * sizeof(cplx), stream_);
    kh2_ = DevBuf((KRYLOV_MAX + 1) * sizeof(cplx), stream_);
    knrm_ = DevBuf(2 * sizeof(cplx), stream_);
    kstate_ = DevBuf(sizeof(KrylovState), stream_);
  }
  cplx* V = kv_.as<cplx>();
  cplx* w = kw_.as<cplx>();
  KrylovState* st = kstate_.as<KrylovState>();
  const int G = dots_grid(n);
  cplx* part = kpart_.as<cplx>();
  cplx* h1 = kh1_.as<cplx>();
  cplx* h2 = kh2_.as<cplx>();
  cplx* nrm = knrm_.as<cplx>();
  const int* done = &st->done;
  launch_dots(x, 0, 1, x, n, part, G, nrm, nullptr, stream_);
  launch_krylov_init(st, nrm, stream_);
  launch_scale(x, &st->beta0, V, n, done, stream_);
  KrylovState* hst = reinterpret_cast<KrylovState*>(pinned_);
  // For small problems the host's round trip per iteration costs more than the
  // iteration itself, so up to KRYLOV_BATCH iterations are queued before the host reads
  // the flags: iterations queued after convergence do nothing in the Lanczos kernels
  // (they test the done flag) and their H_eff products only overwrite the scratch
  // vector.  Large problems read the flags after every iteration.
  const int batch = n <= KRYLOV_BATCH_N ? KRYLOV_BATCH : 1;
  for (int k = 0; k < kmax; ++k) {
    cplx* vk = V + (long long)k * n;
    H.apply(vk, w, stream_);
    launch_dots(V, n, k + 1, w, n, part, G, h1, done, stream_);
    launch_axpy_many(V, n, k + 1, h1, w, n, done, stream_);
    launch_dots(V, n, k + 1, w, n, part, G, h2, done, stream_);
    launch_axpy_many(V, n, k + 1, h2, w, n, done, stream_);
    launch_dots(w, 0, 1, w, n, part, G, nrm, done, stream_);
    launch_krylov_step(st, h1, nrm, tau, opt_.krylov_tol, kmax, stream_);
    launch_scale(w, &st->beta[k], V + (long long)(k + 1) * n, n, done, stream_);
    if ((k + 1) % batch != 0 && k + 1 < kmax) continue;
    // k, nv, done, bad
    TDVP_CUDA(cudaMemcpyAsync(&hst->k, &st->k, 4 * sizeof(int), cudaMemcpyDeviceToHost, stream_));
    TDVP_CUDA(cudaStreamSynchronize(stream_));
    if (hst->bad) throw Error(-4, "non-finite value in the Krylov recurrence");
    if (hst->done) break;
  }
  const int used = hst->k;  // matvecs whose results the recurrence took
  stats_.matvecs += used;
  stats_.heff_flops += (long long)used * H.flops();
  stats_.max_krylov = std::max(stats_.max_krylov, used);
  launch_combine(V, n, &st->nv, st->coef, &st->beta0, x, n, stream_);
  return used;
}

// ---------------------------------------------------------------------------
// SVD split with truncation (Sec. S2.4)
// ---------------------------------------------------------------------------

double Engine::split(BTensor& theta, const BondSpace& bl, const BondSpace& br, long long chi_max, double eps,
                     bool absorb_right, BondSpace& bm, BTensor& X, BTensor& Y, double* s_ent) {
  NvtxRange nvtx_range("split");
  if (gemm_kind_ >= 0) {
    bool ok = false;
    double r = split_mixed(theta, bl, br, chi_max, eps, absorb_right, bm, X, Y, s_ent, ok);
    if (ok) return r;
  }
  const Model& M = model_;
  // group blocks by the coupled label c = (n_a + n_s1, t_c)
  struct Grp {
    int n, t;
    std::vector<std::pair<int, int>> rows;  // (a, s1)
    std::vector<std::pair<int, int>> cols;  // (s2, b)
    std::map<std::pair<int, int>, int> roff, coff;
    int p = 0, q = 0;
  };
  std::map<std::pair<int, int>, int> gidx;
  std::vector<Grp> groups;
  for (const Block& b : theta.blocks) {
    int a = b.key[0], s1 = b.key[1], tc = b.key[2], s2 = b.key[3], bb = b.key[4];
    int nc = bl.s[a].n + M.site[s1].n;
    auto key = std::make_pair(nc, tc);
    auto it = gidx.find(key);
    int g;
    if (it == gidx.end()) {
      g = (int)groups.size();
      gidx[key] = g;
      groups.push_back(Grp());
      groups.back().n = nc;
      groups.back().t = tc;
    } else {
      g = it->second;
    }
    Grp& G = groups[g];
    if (!G.roff.count({a, s1})) {
      G.roff[{a, s1}] = G.p;
      G.rows.push_back({a, s1});
      G.p += bl.s[a].d;
    }
    if (!G.coff.count({s2, bb})) {
      G.coff[{s2, bb}] = G.q;
      G.cols.push_back({s2, bb});
      G.q += br.s[bb].d;
    }
  }
  const int ng = (int)groups.size();
  // workspace: per group G (max(p,q) x min(p,q)) and V (min^2), sv, perm
  std::vector<long long> goff(ng), voff(ng);
  std::vector<int> soff(ng);
  long long gtot = 0, vtot = 0;
  int stot = 0;
  for (int g = 0; g < ng; ++g) {
    int P = std::max(groups[g].p, groups[g].q), Q = std::min(groups[g].p, groups[g].q);
    goff[g] = gtot;
    gtot += (long long)P * Q;
    voff[g] = vtot;
    vtot += (long long)Q * Q;
    soff[g] = stot;
    stot += Q;
  }
  DevBuf dG(std::max<long long>(gtot, 1) * sizeof(cplx), stream_);
  DevBuf dV(std::max<long long>(vtot, 1) * sizeof(cplx), stream_);
  DevBuf dS(std::max(stot, 1) * sizeof(double), stream_);
  DevBuf dP(std::max(stot, 1) * sizeof(int), stream_);
  cplx* Gp = dG.as<cplx>();
  cplx* Vp = dV.as<cplx>();
  double* Sp = dS.as<double>();
  int* Pp = dP.as<int>();
  // gather theta blocks into G (M itself if p >= q, else M^H)
  CopyPlan gather;
  for (const Block& b : theta.blocks) {
    int a = b.key[0], s1 = b.key[1], s2 = b.key[3], bb = b.key[4];
    int g = gidx[{bl.s[a].n + M.site[s1].n, b.key[2]}];
    Grp& G = groups[g];
    int r0 = G.roff[{a, s1}], c0 = G.coff[{s2, bb}];
    CopyTask t{};
    t.src = theta.data() + b.off;
    t.rows = b.rows;
    t.cols = b.cols;
    t.src_rs = b.cols;
    t.src_cs = 1;
    if (G.p >= G.q) {  // column-major p x q
      t.dst = Gp + goff[g] + r0 + (long long)c0 * G.p;
      t.dst_rs = 1;
      t.dst_cs = G.p;
    } else {  // M^H: column-major q x p, element (col, row) = conj(M[row][col])
      t.dst = Gp + goff[g] + c0 + (long long)r0 * G.q;
      t.dst_rs = G.q;
      t.dst_cs = 1;
      t.conj = 1;
    }
    gather.tasks.push_back(t);
  }
  gather.finalize(stream_);
  gather.launch(stream_);
  std::vector<SvdTask> st(ng);
  std::vector<TruncSector> ts(ng);
  for (int g = 0; g < ng; ++g) {
    int P = std::max(groups[g].p, groups[g].q), Q = std::min(groups[g].p, groups[g].q);
    st[g] = {Gp + goff[g], Vp + voff[g], Sp + soff[g], Pp + soff[g], P, Q};
    ts[g] = {Sp + soff[g], Q, M.mult_dim(groups[g].t)};
  }
  DevBuf dst = upload(st, stream_);
  stats_.sweeps64 +=
      jacobi(run_jacobi_rounds(dst.as<SvdTask>(), st, 40, 1e-14, dstatus_, stream_, 0.0, 0.0, &stats_.jacobi64,
                               jscratch()));
  stats_.splits += 1;
  // truncation
  DevBuf dts = upload(ts, stream_);
  DevBuf doffs = upload(soff, stream_);
  DevBuf downer(std::max(stot, 1) * sizeof(int), stream_), dorder(std::max(stot, 1) * sizeof(int), stream_);
  DevBuf dkept(std::max(ng, 1) * sizeof(int), stream_), dstats(8 * sizeof(double), stream_);
  DevBuf dvals(2 * std::max(stot, 1) * sizeof(double), stream_);
  launch_truncate(dts.as<TruncSector>(), ng, doffs.as<int>(), stot, eps, chi_max, opt_.trunc_degen, downer.as<int>(),
                  dorder.as<int>(), dkept.as<int>(), dstats.as<double>(), dvals.as<double>(), stream_);
  std::vector<int> kept(ng);
  double hstats[8];
  TDVP_CUDA(cudaMemcpyAsync(kept.data(), dkept.p, ng * sizeof(int), cudaMemcpyDeviceToHost, stream_));
  TDVP_CUDA(cudaMemcpyAsync(hstats, dstats.p, 6 * sizeof(double), cudaMemcpyDeviceToHost, stream_));
  TDVP_CUDA(cudaStreamSynchronize(stream_));
  if (hstats[5] != 0.0) cap_hit_ = true;
  // new bond: kept sectors sorted by (n, t)
  std::vector<std::pair<std::pair<int, int>, int>> ns;
  for (int g = 0; g < ng; ++g)
    if (kept[g] > 0) ns.push_back({{groups[g].n, groups[g].t}, g});
  std::sort(ns.begin(), ns.end());
  bm = BondSpace();
  for (auto& e : ns) bm.s.push_back({e.first.first, e.first.second, kept[e.second]});
  bm.build_index();
  build_site_layout(X, bl, bm);
  build_site_layout(Y, bm, br);
  alloc(X, false);
  alloc(Y, false);
  double* gsc = dstats.as<double>() + 2;
  CopyPlan scatter;
  for (auto& e : ns) {
    int g = e.second;
    const Grp& G = groups[g];
    int k = kept[g];
    int c = bm.find(G.n, G.t);
    const double* sv = Sp + soff[g];
    const int* perm = Pp + soff[g];
    cplx* Gg = Gp + goff[g];
    cplx* Vg = Vp + voff[g];
    bool direct = G.p >= G.q;
    // left factor blocks (a, s1, c): rows r0.. of the left singular vectors
    for (auto& rw : G.rows) {
      int xb = X.find(bkey(rw.first, rw.second, c));
      if (xb < 0) throw Error(-5, "X block missing");
      int r0 = G.roff.at(rw);
      CopyTask t{};
      t.dst = X.ptr(xb);
      t.rows = bl.s[rw.first].d;
      t.cols = k;
      t.dst_rs = k;
      t.dst_cs = 1;
      t.col_map = perm;
      if (direct) {  // U = G / S
        t.src = Gg + r0;
        t.src_rs = 1;
        t.src_cs = G.p;
        t.scale = sv;
        t.scale_mode = absorb_right ? 2 : 0;
      } else {  // U = V
        t.src = Vg + r0;
        t.src_rs = 1;
        t.src_cs = G.p;
        t.scale = sv;
        t.scale_mode = absorb_right ? 0 : 1;
      }
      if (!absorb_right) t.gscale = gsc;
      scatter.tasks.push_back(t);
    }
    for (auto& cl : G.cols) {
      int yb = Y.find(bkey(c, cl.first, cl.second));
      if (yb < 0) throw Error(-5, "Y block missing");
      int c0 = G.coff.at(cl);
      CopyTask t{};
      t.dst = Y.ptr(yb);
      t.rows = k;
      t.cols = br.s[cl.second].d;
      t.dst_rs = t.cols;
      t.dst_cs = 1;
      t.row_map = perm;
      t.conj = 1;
      if (direct) {  // S V^H: dst[kr][col] = S conj(V[col][perm kr])
        t.src = Vg + c0;
        t.src_rs = G.q;
        t.src_cs = 1;
        t.scale = sv;
        t.scale_mode = absorb_right ? 3 : 0;
      } else {  // V_M = W / S: S V_M^H = conj(W)^T
        t.src = Gg + c0;
        t.src_rs = G.q;
        t.src_cs = 1;
        t.scale = sv;
        t.scale_mode = absorb_right ? 0 : 4;
      }
      if (absorb_right) t.gscale = gsc;
      scatter.tasks.push_back(t);
    }
  }
  scatter.finalize(stream_);
  scatter.launch(stream_);
  if (s_ent) {  // entropy of the new bond from the kept, renormalised singular values
    std::vector<TruncSector> ks;
    for (int g = 0; g < ng; ++g)
      if (kept[g] > 0) ks.push_back({Sp + soff[g], kept[g], M.mult_dim(groups[g].t)});
    DevBuf dks = upload(ks, stream_), dS(sizeof(double), stream_);
    launch_entropy_sv(dks.as<TruncSector>(), (int)ks.size(), gsc, dS.as<double>(), stream_);
    TDVP_CUDA(cudaMemcpyAsync(s_ent, dS.p, sizeof(double), cudaMemcpyDeviceToHost, stream_));
    TDVP_CUDA(cudaStreamSynchronize(stream_));
  }
  long long chi = 0;
  for (auto& s : bm.s) chi += (long long)s.d * M.mult_dim(s.t);
  stats_.chi_max_seen = std::max(stats_.chi_max_seen, chi);
  return hstats[1] / (hstats[0] > 0 ? hstats[0] : 1.0);
}

// ---------------------------------------------------------------------------
// Mixed-precision split (tensor-core precision modes).  The per-sector SVD of
// Sec. S2.4 stays an FP64 SVD; FP32 only supplies a preconditioner.  For each
// sector the working copy W (theta, or theta^H when theta is wide) is copied to
// complex64 and an FP32 round-robin Jacobi accumulates its right rotations V32; then,
// in FP64, G = W V32 is formed and a short FP64 Jacobi (no V) makes its columns
// orthogonal -- G = U S with S the FP64 singular values of W up to the O(1e-7)
// departure of V32 from unitarity, far below any truncation threshold.  The FP32
// stage leaves off-diagonals at the FP32 level, so by the quadratic convergence of
// cyclic Jacobi the FP64 stage ends after about two sweeps instead of the ~17 a
// cold start needs (both measured on the chi = 4096 chain).  The basis the sweep keeps (left for left to right, right for right
// to left) is G/S when it is W's column space, otherwise W^H G / S^2
// re-orthonormalised by two Newton-Schulz steps X <- X (3 I - X^H X) / 2 (the
// overlaps it starts from reach ~1e-3 for the vectors of the smallest kept values,
// whose division by S^2 amplifies the O(1e-7) errors of G); the other factor is the exact FP64
// projection of theta onto that basis.  ok is set when the split was done here (the
// caller runs the FP64 split otherwise).
// ---------------------------------------------------------------------------

// Which of the mixed split's own products run as BF16x4 digit products on the tensor
// cores instead of the FP64 pipe: a bit mask from TDVP_SPLIT_GEMM_TC (read at every
// split; default 26): 1 G = W V, 2 the kept basis W^H Z, 4 the Gram matrix of the
// second Newton-Schulz step (the first step's always runs as BF16x4), 8 the projection,
// 16 G = W V of the sectors whose kept basis is G's own column side (G / S). of theta onto the kept basis.  BF16x4 rounds to 2^-30 of each
// operand row's and column's scale (plus ~K 2^-32 for the dropped digit orders).  For
// the kept basis that is a direction error of the smallest kept vectors, which moves
// the truncated state by (a discarded value) x (that error), and for the projection an
// absolute error of ~1e-9 of the state, both below the BF16x4 matvec's own.  G = W V
// and the last Newton-Schulz Gram matrix stay FP64 where the kept basis is W^H G / S^2:
// that product divides G's errors (2^-32 of the largest column) by S^2, and that Gram
// matrix sets the orthonormality of the kept basis.  Where the basis is G / S itself, a
// BF16x4 G is the exact G of W + dW with |dW| ~ 2^-32 |W| (each operand row and column
// keeps its own scale), and the Gram finish, the truncation and the projection then act
// on that matrix: the split is the exact truncated split of a matrix within the BF16x4
// matvec's own error of theta.
static int split_tc_mask() {
  const char* e = std::getenv("TDVP_SPLIT_GEMM_TC");
  return e && *e ? std::atoi(e) : 26;
}

// a float from the environment (read at every call), or the default
static float env_float(const char* name, float dflt) {
  const char* e = std::getenv(name);
  return e && *e ? (float)std::atof(e) : dflt;
}

// Whether the mixed split finishes with the Gram iteration (default) or with the
// FP64 Jacobi (TDVP_SPLIT_FINISH=jacobi; read at every split).
static bool gram_enabled() {
  const char* e = std::getenv("TDVP_SPLIT_FINISH");
  return !(e && std::strcmp(e, "jacobi") == 0);
}

// Largest |tan| of a rotation the Gram step applies simultaneously: 0.1, or
// TDVP_GRAM_TMAX (read at every split; 0 declines every pair of weight, which hands
// the split to the Jacobi with G unchanged).
static double gram_tmax() {
  const char* e = std::getenv("TDVP_GRAM_TMAX");
  if (!e || !*e) return 0.1;
  const double v = std::atof(e);
  return v < 0 ? 0.0 : (v > 1.0 ? 1.0 : v);
}

// FP64 finish of the mixed split by Gram iteration.  G (ng column-major sets of p x q,
// at toff) has nearly orthogonal columns after the FP32 preconditioner.  A step forms
// C = conj(G^H G) (its tiles on and above the diagonal), turns it into the
// simultaneous rotation Z = I + X (gram_rot_kernel) and adds G X to G in FP64.  The
// first two steps form C and G X on the tensor cores (BF16x4 split products: C to
// ~1e-9 of |g_a||g_b|, since each operand row and column carries its own scale, and
// the update to ~1e-9 of the update), which takes the FP32-level off-diagonals to
// the BF16x4 level; the third step forms C with the FP64 GEMM, so its couplings are
// exact to the FP64 level and its update leaves them at about their square.  The
// stopping rule is the FP64 Jacobi's: the split is finished after an FP64 step whose
// couplings were all below 1e-6 relative or 1e-10 absolute (theta has unit norm);
// otherwise two more steps (BF16x4, FP64) run.  Returns true with the result in G, or
// false (G still a valid start, rotated by near-orthogonal steps) when near-degenerate
// columns carry weight or the steps do not settle; the caller then runs the
// sequential Jacobi.  galt receives G X.
bool Engine::gram_finish(cplx* G, cplx* galt, const std::vector<int>& P, const std::vector<int>& Q,
                         const std::vector<long long>& toff) {
  const int ng = (int)P.size();
  std::vector<long long> koff(ng);
  long long kt = 0, ntot = 0;
  int qmax = 0;
  double flops = 0;
  for (int g = 0; g < ng; ++g) {
    koff[g] = kt;
    kt += (long long)Q[g] * Q[g];
    qmax = std::max(qmax, Q[g]);
    ntot = std::max(ntot, toff[g] + (long long)P[g] * Q[g]);
    flops += 12.0 * P[g] * (double)Q[g] * Q[g];  // upper half of C (4 p q^2) and G X (8 p q^2)
  }
  if (qmax < 2 || qmax > gram_qmax()) return false;
  DevBuf dK(kt * sizeof(cplx), stream_), dZ(kt * sizeof(cplx), stream_), dfl(8 * sizeof(int), stream_);
  cplx *Kb = dK.as<cplx>(), *Zb = dZ.as<cplx>();
  int* fl = dfl.as<int>();
  // pointers relative to launch bases: 1 = G, 2 = galt
  GemmPlan pk_tc, pk64, pu;
  std::vector<GramTask> gt;
  for (int g = 0; g < ng; ++g) {
    if (Q[g] < 1) continue;
    GemmTask t{};
    GemmSeg sg{};
    sg.alpha = 1.0;
    t.c = Kb + koff[g];
    t.rows = Q[g];
    t.cols = Q[g];
    t.ldc = Q[g];
    sg.a = as_off(toff[g]);
    sg.a_base = 1;
    sg.lda = P[g];
    sg.b = as_off(toff[g]);
    sg.b_base = 1;
    sg.ldb = P[g];
    sg.op_b = OP_C;
    sg.k = P[g];
    for (GemmPlan* pl : {&pk_tc, &pk64}) {
      t.seg_begin = (int)pl->segs.size();
      t.seg_count = 1;
      pl->segs.push_back(sg);
      pl->tasks.push_back(t);
    }
    GemmTask u{};
    GemmSeg sh{};
    sh.alpha = 1.0;
    u.c = as_off(toff[g]);
    u.c_base = 2;
    u.rows = Q[g];
    u.cols = P[g];
    u.ldc = P[g];
    sh.a = Zb + koff[g];
    sh.lda = Q[g];
    sh.b = as_off(toff[g]);
    sh.b_base = 1;
    sh.ldb = P[g];
    sh.k = Q[g];
    u.seg_begin = (int)pu.segs.size();
    u.seg_count = 1;
    pu.segs.push_back(sh);
    pu.tasks.push_back(u);
    gt.push_back({Kb + koff[g], Zb + koff[g], Q[g]});
  }
  // the Gram matrices are Hermitian: only tiles on and above the diagonal
  pk_tc.upper_only = pk64.upper_only = true;
  pk64.ksplit = true;
  pk_tc.finalize(stream_, 1, dstatus_);
  pk64.finalize(stream_);
  pu.finalize(stream_, 1, dstatus_);
  DevBuf dgt = upload(gt, stream_);
  const double tmax = gram_tmax();
  const Bases4 B{{0, reinterpret_cast<uintptr_t>(G), reinterpret_cast<uintptr_t>(galt), 0}};
  cudaEvent_t ev[2];
  TDVP_CUDA(cudaEventCreate(&ev[0]));
  TDVP_CUDA(cudaEventCreate(&ev[1]));
  TDVP_CUDA(cudaEventRecord(ev[0], stream_));
  auto step = [&](bool fp64, int* f) {
    (fp64 ? pk64 : pk_tc).launch(stream_, B);
    launch_gram_rot(dgt.as<GramTask>(), (int)gt.size(), qmax, 1e-13, 1e-6, 1e-10, tmax, f, stream_);
    pu.launch(stream_, B);
    launch_add_inplace(G, galt, ntot, stream_);
  };
  bool ok = false;
  int steps = 0;
  float worst = 0.0f;
  for (int round = 0; round < 2 && !ok; ++round) {
    TDVP_CUDA(cudaMemsetAsync(fl, 0, 8 * sizeof(int), stream_));
    if (round == 0) {
      step(false, fl);
      steps += 1;
    }
    step(false, fl);
    step(true, fl + 4);
    steps += 2;
    int h[8];
    TDVP_CUDA(cudaMemcpyAsync(h, fl, sizeof(h), cudaMemcpyDeviceToHost, stream_));
    TDVP_CUDA(cudaStreamSynchronize(stream_));
    worst = std::max(worst, *reinterpret_cast<float*>(&h[6]));
    if (h[1] || h[5]) break;  // near-degenerate columns of weight: the Jacobi finishes
    ok = h[4] == 0;           // the FP64 step saw no coupling above the stopping rule
  }
  TDVP_CUDA(cudaEventRecord(ev[1], stream_));
  TDVP_CUDA(cudaEventSynchronize(ev[1]));
  float ms = 0;
  if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) stats_.gram.ms += ms;
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  stats_.gram.flops += steps * flops;
  stats_.gram.launches += 1;
  stats_.gram_steps += steps;
  if (!ok) stats_.gram_fallbacks += 1;
  if (std::getenv("TDVP_GRAM_DEBUG"))
    std::fprintf(stderr, "gram: %d steps, ok=%d, last FP64 step's largest relative coupling %.3g\n", steps, (int)ok,
                 (double)worst);
  return ok;
}

double Engine::split_mixed(BTensor& theta, const BondSpace& bl, const BondSpace& br, long long chi_max, double eps,
                           bool absorb_right, BondSpace& bm, BTensor& X, BTensor& Y, double* s_ent, bool& ok) {
  // TDVP_SPLIT_DEBUG: wall time of each section (synchronising after each one)
  static const bool sdbg = std::getenv("TDVP_SPLIT_DEBUG") != nullptr;
  auto st0 = std::chrono::steady_clock::now();
  auto smark = [&](const char* what) {
    if (!sdbg) return;
    cudaStreamSynchronize(stream_);
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "split %s %.3f ms\n", what, std::chrono::duration<double, std::milli>(now - st0).count());
    st0 = now;
  };
  NvtxRange nvtx_range("split");
  const Model& M = model_;
  ok = false;
  struct Grp {
    int n, t;
    std::vector<std::pair<int, int>> rows, cols;
    std::map<std::pair<int, int>, int> roff, coff;
    int p = 0, q = 0;
  };
  std::map<std::pair<int, int>, int> gidx;
  std::vector<Grp> groups;
  for (const Block& b : theta.blocks) {
    int a = b.key[0], s1 = b.key[1], tc = b.key[2], s2 = b.key[3], bb = b.key[4];
    auto key = std::make_pair(bl.s[a].n + M.site[s1].n, tc);
    auto it = gidx.find(key);
    int g;
    if (it == gidx.end()) {
      g = (int)groups.size();
      gidx[key] = g;
      groups.push_back(Grp());
      groups.back().n = key.first;
      groups.back().t = tc;
    } else {
      g = it->second;
    }
    Grp& G = groups[g];
    if (!G.roff.count({a, s1})) {
      G.roff[{a, s1}] = G.p;
      G.rows.push_back({a, s1});
      G.p += bl.s[a].d;
    }
    if (!G.coff.count({s2, bb})) {
      G.coff[{s2, bb}] = G.q;
      G.cols.push_back({s2, bb});
      G.q += br.s[bb].d;
    }
  }
  const int ng = (int)groups.size();
  auto bigP = [](const Grp& G) { return std::max(G.p, G.q); };
  auto smallQ = [](const Grp& G) { return std::min(G.p, G.q); };
  // the kept basis is W's column space (U of W) when the sweep needs the side W's rows index
  auto from_g = [&](const Grp& G) { return absorb_right == (G.p >= G.q); };
  auto xrows = [&](const Grp& G) { return absorb_right ? G.p : G.q; };
  std::vector<long long> toff(ng), voff(ng);
  std::vector<int> soff(ng);
  long long ttot = 0, vtot = 0;
  int stot = 0;
  for (int g = 0; g < ng; ++g) {
    toff[g] = ttot;
    ttot += (long long)groups[g].p * groups[g].q;
    voff[g] = vtot;
    vtot += (long long)smallQ(groups[g]) * smallQ(groups[g]);
    soff[g] = stot;
    stot += smallQ(groups[g]);
  }
  const long long tt1 = std::max<long long>(ttot, 1), vt1 = std::max<long long>(vtot, 1);
  DevBuf dT(tt1 * sizeof(cplx), stream_), dW(tt1 * sizeof(cplx), stream_), dG(tt1 * sizeof(cplx), stream_);
  DevBuf dW32(tt1 * sizeof(float2), stream_), dV32(vt1 * sizeof(float2), stream_), dV(vt1 * sizeof(cplx), stream_);
  DevBuf dS(std::max(stot, 1) * sizeof(double), stream_), dP(std::max(stot, 1) * sizeof(int), stream_);
  cplx *T64 = dT.as<cplx>(), *W64 = dW.as<cplx>(), *G64 = dG.as<cplx>(), *V64 = dV.as<cplx>();
  float2 *W32 = dW32.as<float2>(), *V32 = dV32.as<float2>();
  double* Sp = dS.as<double>();
  int* Pp = dP.as<int>();
  // theta row-major p x q (for the projections) and W column-major P x Q
  CopyPlan gather;
  for (const Block& b : theta.blocks) {
    int a = b.key[0], s1 = b.key[1], s2 = b.key[3], bb = b.key[4];
    int g = gidx[{bl.s[a].n + M.site[s1].n, b.key[2]}];
    Grp& G = groups[g];
    const int r0 = G.roff[{a, s1}], c0 = G.coff[{s2, bb}];
    CopyTask t{};
    t.src = theta.data() + b.off;
    t.rows = b.rows;
    t.cols = b.cols;
    t.src_rs = b.cols;
    t.src_cs = 1;
    t.dst = T64 + toff[g] + (long long)r0 * G.q + c0;
    t.dst_rs = G.q;
    t.dst_cs = 1;
    gather.tasks.push_back(t);
    CopyTask w = t;
    if (G.p >= G.q) {  // W = theta, column-major p x q
      w.dst = W64 + toff[g] + r0 + (long long)c0 * G.p;
      w.dst_rs = 1;
      w.dst_cs = G.p;
    } else {  // W = theta^H, column-major q x p
      w.dst = W64 + toff[g] + c0 + (long long)r0 * G.q;
      w.dst_rs = G.q;
      w.dst_cs = 1;
      w.conj = 1;
    }
    gather.tasks.push_back(w);
  }
  gather.finalize(stream_);
  gather.launch(stream_);
  smark("setup+gather");
  const int tcm = split_tc_mask();
  auto kind_of = [&](int bit) { return (tcm & bit) ? 1 : -1; };
  // FP32 preconditioner
  launch_narrow(W64, W32, ttot, stream_);
  std::vector<Svd32Task> st32(ng);
  for (int g = 0; g < ng; ++g) st32[g] = {W32 + toff[g], V32 + voff[g], bigP(groups[g]), smallQ(groups[g])};
  for (int g = 0; g < ng; ++g) {
    const double P = bigP(groups[g]), Q = smallQ(groups[g]);
    stats_.split_pmax = std::max<long long>(stats_.split_pmax, (long long)P);
    stats_.split_qmax = std::max<long long>(stats_.split_qmax, (long long)Q);
    stats_.split_work += P * Q * Q;
    if (P * Q * 8.0 <= 192.0 * 1024.0) stats_.split_work_small += P * Q * Q;
  }
  DevBuf dst32 = upload(st32, stream_);
  // FP32 stage: rotate while |g_i^H g_j| > 2e-5 |g_i||g_j|, at most 24 sweeps (it
  // need not converge: the FP64 stage finishes whatever is left).  A sweep ends the
  // stage when its rotations were all below that or below min(1e-10, eps / 10) in
  // absolute terms (theta has unit norm): couplings between columns of negligible
  // weight, which FP32 cannot resolve anyway, do not keep it going (the FP64 finish
  // uses the same kind of absolute floor).  TDVP_FP32_TOL / TDVP_FP32_ABS override.
  const float abs32 = (float)std::min(1e-10, 0.1 * eps);
  const int sw32 =
      jacobi(run_jacobi_rounds32(dst32.as<Svd32Task>(), st32, 24, env_float("TDVP_FP32_TOL", 2e-5f),
                                 env_float("TDVP_FP32_ABS", abs32), stream_, &stats_.jacobi32, jscratch()));
  ok = true;
  stats_.sweeps32 += sw32;
  smark("fp32 jacobi");
  stats_.splits += 1;
  launch_widen(V32, V64, vtot, stream_);
  // G = W V in FP64: row-major G^T (Q x P) = V^T (Q x Q) W^T (Q x P)
  {
    // gp[1]: the groups whose kept basis is G's own column side, gp[0]: the others
    GemmPlan gp[2];
    for (int g = 0; g < ng; ++g) {
      const int P = bigP(groups[g]), Q = smallQ(groups[g]);
      GemmPlan& pl = gp[from_g(groups[g]) ? 1 : 0];
      GemmTask t{};
      GemmSeg sg{};
      sg.alpha = 1.0;
      t.c = G64 + toff[g];
      t.rows = Q;
      t.cols = P;
      t.ldc = P;
      sg.a = V64 + voff[g];
      sg.lda = Q;
      sg.b = W64 + toff[g];
      sg.ldb = P;
      sg.k = Q;
      t.seg_begin = (int)pl.segs.size();
      t.seg_count = 1;
      pl.segs.push_back(sg);
      pl.tasks.push_back(t);
    }
    for (int k = 0; k < 2; ++k) {
      if (gp[k].tasks.empty()) continue;
      gp[k].ksplit = true;
      gp[k].finalize(stream_, (tcm & 1) || (k == 1 && (tcm & 16)) ? 1 : -1, dstatus_);
      gp[k].launch(stream_, Bases4{{0, 0, 0, 0}});
    }
  }
  smark("G = W V");
  std::vector<SvdTask> st(ng);
  std::vector<TruncSector> ts(ng);
  for (int g = 0; g < ng; ++g) {
    st[g] = {G64 + toff[g], nullptr, Sp + soff[g], Pp + soff[g], bigP(groups[g]), smallQ(groups[g])};
    ts[g] = {Sp + soff[g], smallQ(groups[g]), M.mult_dim(groups[g].t)};
  }
  DevBuf dst = upload(st, stream_);
  // FP64 stage: rotate above 1e-13 (relative); stop after a sweep whose rotations were
  // all below 1e-6 relative (quadratic convergence leaves ~1e-12) or below 1e-10 in
  // absolute terms (theta has unit norm, so that is a weight a decade below the
  // smallest truncation threshold in use; on the L=60 quench the observables do not
  // move against tighter settings while the stage needs fewer sweeps)
  // The Gram finish (gram_finish) reaches the same stopping point with GEMMs; the
  // Jacobi runs when it declines (near-degenerate columns of weight) or when
  // TDVP_SPLIT_FINISH=jacobi.
  std::vector<int> gp(ng), gq(ng);
  for (int g = 0; g < ng; ++g) {
    gp[g] = bigP(groups[g]);
    gq[g] = smallQ(groups[g]);
  }
  if (gram_enabled() && gram_finish(G64, W64, gp, gq, toff)) {
    int qm = 1;
    for (int g = 0; g < ng; ++g) qm = std::max(qm, gq[g]);
    launch_svd_finish(dst.as<SvdTask>(), ng, qm, stream_);
  } else {
    stats_.sweeps64 += jacobi(run_jacobi_rounds(dst.as<SvdTask>(), st, 30, 1e-13, dstatus_, stream_, 1e-6, 1e-10,
                                                &stats_.jacobi64, jscratch()));
  }
  smark("fp64 finish");
  DevBuf dts = upload(ts, stream_), doffs = upload(soff, stream_);
  DevBuf downer(std::max(stot, 1) * sizeof(int), stream_), dorder(std::max(stot, 1) * sizeof(int), stream_);
  DevBuf dkept(std::max(ng, 1) * sizeof(int), stream_), dstats(8 * sizeof(double), stream_);
  DevBuf dvals(2 * std::max(stot, 1) * sizeof(double), stream_);
  launch_truncate(dts.as<TruncSector>(), ng, doffs.as<int>(), stot, eps, chi_max, opt_.trunc_degen, downer.as<int>(),
                  dorder.as<int>(), dkept.as<int>(), dstats.as<double>(), dvals.as<double>(), stream_);
  std::vector<int> kept(ng);
  double hstats[8];
  TDVP_CUDA(cudaMemcpyAsync(kept.data(), dkept.p, ng * sizeof(int), cudaMemcpyDeviceToHost, stream_));
  TDVP_CUDA(cudaMemcpyAsync(hstats, dstats.p, 6 * sizeof(double), cudaMemcpyDeviceToHost, stream_));
  TDVP_CUDA(cudaStreamSynchronize(stream_));
  if (hstats[5] != 0.0) cap_hit_ = true;
  smark("truncation (sync)");
  std::vector<std::pair<std::pair<int, int>, int>> ns;
  for (int g = 0; g < ng; ++g)
    if (kept[g] > 0) ns.push_back({{groups[g].n, groups[g].t}, g});
  std::sort(ns.begin(), ns.end());
  bm = BondSpace();
  for (auto& e : ns) bm.s.push_back({e.first.first, e.first.second, kept[e.second]});
  bm.build_index();
  // kept basis X (xrows x k, row-major) on the side the sweep needs
  std::vector<long long> xoff(ng, 0), zoff(ng, 0), koff(ng, 0), poff(ng, 0);
  long long xt = 0, zt = 0, kt = 0, pt = 0;
  for (int g = 0; g < ng; ++g) {
    const Grp& G = groups[g];
    const int k = kept[g];
    if (!k) continue;
    xoff[g] = xt;
    xt += (long long)xrows(G) * k;
    if (!from_g(G)) {
      zoff[g] = zt;
      zt += (long long)bigP(G) * k;
      koff[g] = kt;
      kt += (long long)k * k;
    }
    poff[g] = pt;
    pt += (long long)(absorb_right ? G.q : G.p) * k;
  }
  DevBuf dX(std::max<long long>(xt, 1) * sizeof(cplx), stream_), dZ(std::max<long long>(zt, 1) * sizeof(cplx), stream_);
  DevBuf dK(std::max<long long>(kt, 1) * sizeof(cplx), stream_), dPr(std::max<long long>(pt, 1) * sizeof(cplx), stream_);
  cplx *Xb = dX.as<cplx>(), *Zb = dZ.as<cplx>(), *Kb = dK.as<cplx>(), *Pr = dPr.as<cplx>();
  std::vector<BasisTask> bt;
  bool any_ns = false;
  for (int g = 0; g < ng; ++g) {
    const Grp& G = groups[g];
    if (!kept[g]) continue;
    if (from_g(G)) {
      bt.push_back({G64 + toff[g], Pp + soff[g], Sp + soff[g], Xb + xoff[g], bigP(G), kept[g], 0});
    } else {
      bt.push_back({G64 + toff[g], Pp + soff[g], Sp + soff[g], Zb + zoff[g], bigP(G), kept[g], 1});
      any_ns = true;
    }
  }
  DevBuf dbt = upload(bt, stream_);
  launch_basis64(dbt.as<BasisTask>(), (int)bt.size(), stream_);
  if (any_ns) {
    // X = W^H Z: theta Z (left to right, W = theta^H) or theta^H Z (right to left, W = theta)
    GemmPlan xp;
    std::vector<NsTask> nt;
    for (int g = 0; g < ng; ++g) {
      const Grp& G = groups[g];
      const int k = kept[g];
      if (!k || from_g(G)) continue;
      GemmTask t{};
      GemmSeg sg{};
      sg.alpha = 1.0;
      t.c = Xb + xoff[g];
      t.rows = xrows(G);
      t.cols = k;
      t.ldc = k;
      sg.a = T64 + toff[g];
      sg.lda = G.q;
      sg.b = Zb + zoff[g];
      sg.ldb = k;
      if (absorb_right) {
        sg.k = G.q;
      } else {
        sg.op_a = OP_C;
        sg.k = G.p;
      }
      t.seg_begin = (int)xp.segs.size();
      t.seg_count = 1;
      xp.segs.push_back(sg);
      xp.tasks.push_back(t);
      nt.push_back({Kb + koff[g], k});
    }
    xp.ksplit = true;
    xp.finalize(stream_, kind_of(2), dstatus_);
    xp.launch(stream_, Bases4{{0, 0, 0, 0}});
    // Newton-Schulz, X <- X (3 I - X^H X) / 2 = X + X E with E = (I - X^H X) / 2, two
    // steps (with one, the entropies of a chi = 4096 sweep moved by 2.6e-7 against 2.7e-8).
    // Only its tiles on and above the diagonal of K = X^H X are formed.  X's columns of
    // small singular values start about u32 sigma_max / sigma (up to ~1e-3) away from
    // orthonormal, and the first step brings that to its square: its K may carry the
    // 2^-30 relative error of BF16x4 digit products.  The second step's K, which sets the
    // orthonormality reached, is formed on the FP64 pipe.  E is of the size of X's
    // departure from orthonormality, so the correction X E runs as BF16x4 digit products
    // (error ~2^-30 |E| of X) and is added to X in FP64.
    std::vector<const cplx*> eptr;
    long long et = 0;
    for (const NsTask& x : nt) et += (long long)x.k * x.k;
    DevBuf dE(std::max<long long>(et, 1) * sizeof(cplx), stream_);
    {
      long long o = 0;
      for (const NsTask& x : nt) {
        eptr.push_back(dE.as<cplx>() + o);
        o += (long long)x.k * x.k;
      }
    }
    DevBuf dnt = upload(nt, stream_), dep = upload(eptr, stream_);
    for (int it = 0; it < 2; ++it) {
      GemmPlan g1, g2;
      LincombPlan add;
      int ti = 0;
      for (int g = 0; g < ng; ++g) {
        const Grp& G = groups[g];
        const int k = kept[g];
        if (!k || from_g(G)) continue;
        const int dim = xrows(G);
        GemmTask t{};
        GemmSeg sg{};
        sg.alpha = 1.0;
        t.c = Kb + koff[g];
        t.rows = k;
        t.cols = k;
        t.ldc = k;
        sg.a = Xb + xoff[g];
        sg.lda = k;
        sg.op_a = OP_C;
        sg.b = Xb + xoff[g];
        sg.ldb = k;
        sg.k = dim;
        t.seg_begin = (int)g1.segs.size();
        t.seg_count = 1;
        g1.segs.push_back(sg);
        g1.tasks.push_back(t);
        GemmTask u{};
        GemmSeg sh{};
        sh.alpha = 1.0;
        u.c = Zb + zoff[g];
        u.rows = dim;
        u.cols = k;
        u.ldc = k;
        sh.a = Xb + xoff[g];
        sh.lda = k;
        sh.b = eptr[ti];
        sh.ldb = k;
        sh.k = k;
        u.seg_begin = (int)g2.segs.size();
        u.seg_count = 1;
        g2.segs.push_back(sh);
        g2.tasks.push_back(u);
        // X += Z (Z rows >= X rows, packed at the same pitch k)
        LincombTask lt{};
        lt.out = Xb + xoff[g];
        lt.rows = dim;
        lt.cols = k;
        lt.ld_out = k;
        lt.term_begin = (int)add.terms.size();
        lt.term_count = 2;
        add.terms.push_back({Xb + xoff[g], k, 1.0});
        add.terms.push_back({Zb + zoff[g], k, 1.0});
        add.tasks.push_back(lt);
        ++ti;
      }
      g1.upper_only = true;
      g1.ksplit = true;
      g1.finalize(stream_, (tcm & 4) || it == 0 ? 1 : -1, dstatus_);
      g1.launch(stream_, Bases4{{0, 0, 0, 0}});
      launch_ns_corr(dnt.as<NsTask>(), dep.as<const cplx*>(), (int)nt.size(), stream_);
      g2.finalize(stream_, 1, dstatus_);
      g2.launch(stream_, Bases4{{0, 0, 0, 0}});
      add.finalize(stream_);
      add.launch(stream_);
    }
  }
  smark("kept basis + Newton-Schulz");
  // exact projection for the other factor: C = X^H T (left to right) or M = T X (right to left)
  GemmPlan pg;
  for (int g = 0; g < ng; ++g) {
    const Grp& G = groups[g];
    const int k = kept[g];
    if (!k) continue;
    GemmTask t{};
    GemmSeg sg{};
    sg.alpha = 1.0;
    if (absorb_right) {
      t.c = Pr + poff[g];
      t.rows = k;
      t.cols = G.q;
      t.ldc = G.q;
      sg.a = Xb + xoff[g];
      sg.lda = k;
      sg.op_a = OP_C;
      sg.b = T64 + toff[g];
      sg.ldb = G.q;
      sg.k = G.p;
    } else {
      t.c = Pr + poff[g];
      t.rows = G.p;
      t.cols = k;
      t.ldc = k;
      sg.a = T64 + toff[g];
      sg.lda = G.q;
      sg.b = Xb + xoff[g];
      sg.ldb = k;
      sg.k = G.q;
    }
    t.seg_begin = (int)pg.segs.size();
    t.seg_count = 1;
    pg.segs.push_back(sg);
    pg.tasks.push_back(t);
  }
  pg.ksplit = true;
  pg.finalize(stream_, kind_of(8), dstatus_);
  pg.launch(stream_, Bases4{{0, 0, 0, 0}});
  smark("projection");
  // renormalise the kept state to unit norm
  DevBuf part((size_t)296 * sizeof(cplx), stream_), nrm(sizeof(cplx), stream_), dgs(sizeof(double), stream_);
  launch_dots(Pr, 0, 1, Pr, pt, part.as<cplx>(), dots_grid(pt), nrm.as<cplx>(), nullptr, stream_);
  cplx hn;
  TDVP_CUDA(cudaMemcpyAsync(&hn, nrm.p, sizeof(cplx), cudaMemcpyDeviceToHost, stream_));
  TDVP_CUDA(cudaStreamSynchronize(stream_));
  double gsc = hn.x > 0 ? 1.0 / std::sqrt(hn.x) : 1.0;
  TDVP_CUDA(cudaMemcpyAsync(dgs.p, &gsc, sizeof(double), cudaMemcpyHostToDevice, stream_));
  build_site_layout(X, bl, bm);
  smark("norm (sync)");
  build_site_layout(Y, bm, br);
  alloc(X, false);
  alloc(Y, false);
  CopyPlan scatter;
  for (auto& e : ns) {
    int g = e.second;
    const Grp& G = groups[g];
    const int k = kept[g];
    const int c = bm.find(G.n, G.t);
    for (auto& rw : G.rows) {
      int xb = X.find(bkey(rw.first, rw.second, c));
      if (xb < 0) throw Error(-5, "X block missing");
      int r0 = G.roff.at(rw);
      CopyTask t{};
      t.dst = X.ptr(xb);
      t.rows = bl.s[rw.first].d;
      t.cols = k;
      t.dst_rs = k;
      t.dst_cs = 1;
      if (absorb_right) {  // A = X rows
        t.src = Xb + xoff[g] + (long long)r0 * k;
      } else {  // centre M = T X rows
        t.src = Pr + poff[g] + (long long)r0 * k;
        t.gscale = dgs.as<double>();
      }
      t.src_rs = k;
      t.src_cs = 1;
      scatter.tasks.push_back(t);
    }
    for (auto& cl : G.cols) {
      int yb = Y.find(bkey(c, cl.first, cl.second));
      if (yb < 0) throw Error(-5, "Y block missing");
      int c0 = G.coff.at(cl);
      CopyTask t{};
      t.dst = Y.ptr(yb);
      t.rows = k;
      t.cols = br.s[cl.second].d;
      t.dst_rs = t.cols;
      t.dst_cs = 1;
      if (absorb_right) {  // centre C = X^H T columns
        t.src = Pr + poff[g] + c0;
        t.src_rs = G.q;
        t.src_cs = 1;
        t.gscale = dgs.as<double>();
      } else {  // B = X^H: B[kk][col] = conj(X[c0 + col][kk])
        t.src = Xb + xoff[g] + (long long)c0 * k;
        t.src_rs = 1;
        t.src_cs = k;
        t.conj = 1;
      }
      scatter.tasks.push_back(t);
    }
  }
  scatter.finalize(stream_);
  scatter.launch(stream_);
  if (s_ent) {
    std::vector<TruncSector> ks;
    for (int g = 0; g < ng; ++g)
      if (kept[g] > 0) ks.push_back({Sp + soff[g], kept[g], M.mult_dim(groups[g].t)});
    DevBuf dks = upload(ks, stream_), dE(sizeof(double), stream_);
    launch_entropy_sv(dks.as<TruncSector>(), (int)ks.size(), dstats.as<double>() + 2, dE.as<double>(), stream_);
    TDVP_CUDA(cudaMemcpyAsync(s_ent, dE.p, sizeof(double), cudaMemcpyDeviceToHost, stream_));
  }
  smark("scatter + entropy");
  TDVP_CUDA(cudaStreamSynchronize(stream_));
  long long chi = 0;
  for (auto& x : bm.s) chi += (long long)x.d * M.mult_dim(x.t);
  stats_.chi_max_seen = std::max(stats_.chi_max_seen, chi);
  return hstats[1] / (hstats[0] > 0 ? hstats[0] : 1.0);
}

// ---------------------------------------------------------------------------
// the time step (Sec. S2.2)
// ---------------------------------------------------------------------------

// One two-site update at bond (i, i+1) of the second-order sweep (Sec. S2.2):
// theta = X_i Y_{i+1}, theta <- exp(-i tau H_eff) theta, SVD split with truncation,
// environment update, and (when backward) the one-site backward evolution of the new
// centre by +tau.  left_to_right: centre i -> i+1, otherwise i+1 -> i.
void Engine::bond_update(int i, bool left_to_right, double tau, long long chi_max, double eps, bool backward,
                         double* s_ent) {
  NvtxRange nvtx_range("bond_update");
  auto tp = std::chrono::steady_clock::now();
  auto mark = [&](int ph) {
    if (!profile_) return;
    cudaStreamSynchronize(stream_);
    auto now = std::chrono::steady_clock::now();
    stats_.phase[ph] += std::chrono::duration<double>(now - tp).count();
    tp = now;
  };
  BTensor theta;
  form_theta(site_[i], site_[i + 1], theta, bonds_[i], bonds_[i + 1], bonds_[i + 2]);
  mark(0);
  {
    HeffPlan H;
    plan_heff2(H, Lenv_[i], Renv_[i + 2], theta, bonds_[i], bonds_[i + 2]);
    mark(1);
    expm(H, theta.data(), tau);
    mark(2);
  }
  BondSpace bm;
  BTensor X, Y;
  double disc = split(theta, bonds_[i], bonds_[i + 2], chi_max, eps, left_to_right, bm, X, Y, s_ent);
  stats_.max_discarded = std::max(stats_.max_discarded, disc);
  bonds_[i + 1] = bm;
  site_[i] = std::move(X);
  site_[i + 1] = std::move(Y);
  mark(3);
  if (!env_ev_[0]) {
    TDVP_CUDA(cudaEventCreate(&env_ev_[0]));
    TDVP_CUDA(cudaEventCreate(&env_ev_[1]));
  }
  TDVP_CUDA(cudaEventRecord(env_ev_[0], stream_));
  if (left_to_right) {
    update_left_env(Lenv_[i], site_[i], Lenv_[i + 1], bonds_[i], bonds_[i + 1]);
    TDVP_CUDA(cudaEventRecord(env_ev_[1], stream_));
    mark(4);
    center_ = i + 1;
    if (backward) {
      HeffPlan H1;
      plan_heff1(H1, Lenv_[i + 1], Renv_[i + 2], site_[i + 1], bonds_[i + 1], bonds_[i + 2]);
      mark(1);
      expm(H1, site_[i + 1].data(), -tau);
      mark(5);
    }
  } else {
    update_right_env(Renv_[i + 2], site_[i + 1], Renv_[i + 1], bonds_[i + 1], bonds_[i + 2]);
    TDVP_CUDA(cudaEventRecord(env_ev_[1], stream_));
    mark(4);
    center_ = i;
    if (backward) {
      HeffPlan H1;
      plan_heff1(H1, Lenv_[i], Renv_[i + 1], site_[i], bonds_[i], bonds_[i + 1]);
      mark(1);
      expm(H1, site_[i].data(), -tau);
      mark(5);
    }
  }
  // device time of the environment update (the backward Krylov step has usually
  // synchronised the stream already)
  float ms = 0.f;
  TDVP_CUDA(cudaEventSynchronize(env_ev_[1]));
  if (cudaEventElapsedTime(&ms, env_ev_[0], env_ev_[1]) == cudaSuccess) stats_.env_ms += ms;
}

void Engine::step(double dt, long long chi_max, double eps) {
  NvtxRange nvtx_range("tdvp_step");
  if (bond_only_) throw Error(-2, "a bond problem has no chain to evolve");
  if (!(dt > 0) || chi_max < 1 || !(eps >= 0)) throw Error(-1, "invalid step arguments");
  if (center_ != 0) throw Error(-2, "a full time step starts with the orthogonality centre on site 0");
  chain_heff_.reset();
  auto t0 = std::chrono::steady_clock::now();
  const double tau = dt / 2;
  const int L = L_;
  for (int i = 0; i + 1 < L; ++i) bond_update(i, true, tau, chi_max, eps, i + 2 < L, nullptr);
  for (int i = L - 2; i >= 0; --i) bond_update(i, false, tau, chi_max, eps, i > 0, nullptr);
  TDVP_CUDA(cudaStreamSynchronize(stream_));
  check_status();
  stats_.seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  stats_.steps += 1;
}

// ---------------------------------------------------------------------------
// one-site TDVP (Sec. S2.2: after the bond dimension has saturated the sweep
// updates one site at a time and needs no truncated SVD)
// ---------------------------------------------------------------------------

// bond matrix on a bond: one d x d block per sector (it is an SU(2) scalar)
void Engine::build_bond_layout(BTensor& t, const BondSpace& b) const {
  t = BTensor();
  t.kind = OMEGA;
  for (int c = 0; c < (int)b.s.size(); ++c) t.add(bkey(c, 0, c), c, 0, c, 0, 0, b.s[c].d, b.s[c].d);
}

// Zero-site H_eff on the bond matrix: C'(a') = sum_{w,a} L(a',w,a) C(a) R(a,w,a').
// In the reduced form every recoupling factor is 1: C is a scalar, so the Clebsch-
// Gordan structure of L, C(a w|a'), meets the identical structure of R and
// contracts to the identity by orthonormality.
void Engine::plan_heff0(HeffPlan& p, const BTensor& Lenv, const BTensor& Renv, const BTensor& C) {
  p = HeffPlan();
  p.n = C.size;
  p.t1.kind = THETA;
  std::vector<int> t1l;                      // L block of each T1 block
  std::map<int, std::vector<int>> by_out;    // a' -> T1 blocks
  for (int lb = 0; lb < (int)Lenv.blocks.size(); ++lb) {
    const Block& lk = Lenv.blocks[lb];
    const int ap = lk.key[0], w = lk.key[1], a = lk.key[2];
    if (C.find(bkey(a, 0, a)) < 0 || C.find(bkey(ap, 0, ap)) < 0) continue;
    if (Renv.find(bkey(a, w, ap)) < 0) continue;
    const int id = (int)t1l.size();
    p.t1.add((uint64_t)id, ap, w, a, 0, 0, lk.rows, lk.cols);
    t1l.push_back(lb);
    by_out[ap].push_back(id);
  }
  alloc(p.t1, false);
  for (int i = 0; i < (int)t1l.size(); ++i) {
    const Block& lk = Lenv.blocks[t1l[i]];
    const Block& cb = C.blocks[C.find(bkey(lk.key[2], 0, lk.key[2]))];
    GemmTask t{};
    t.c = p.t1.ptr(i);
    t.rows = lk.rows;
    t.cols = cb.cols;
    t.ldc = cb.cols;
    t.seg_begin = (int)p.g1.segs.size();
    t.seg_count = 1;
    GemmSeg sg{};
    sg.a = Lenv.ptr(t1l[i]);
    sg.a_static = 1;
    sg.lda = lk.cols;
    sg.b = as_off(cb.off);
    sg.b_base = 1;
    sg.ldb = cb.cols;
    sg.k = lk.cols;
    sg.alpha = 1.0;
    p.g1.segs.push_back(sg);
    p.g1.tasks.push_back(t);
    p.g1.flops += 8LL * lk.rows * lk.cols * cb.cols;
  }
  for (int ob = 0; ob < (int)C.blocks.size(); ++ob) {
    const Block& o = C.blocks[ob];
    GemmTask t{};
    t.c = as_off(o.off);
    t.c_base = 2;
    t.rows = o.rows;
    t.cols = o.cols;
    t.ldc = o.cols;
    t.seg_begin = (int)p.g3.segs.size();
    int cnt = 0;
    auto it = by_out.find(o.key[0]);
    if (it != by_out.end())
      for (int id : it->second) {
        const Block& tb = p.t1.blocks[id];
        const int rb = Renv.find(bkey(tb.key[2], tb.key[1], o.key[0]));
        const Block& rk = Renv.blocks[rb];
        GemmSeg sg{};
        sg.a = p.t1.ptr(id);
        sg.lda = tb.cols;
        sg.b = Renv.ptr(rb);
        sg.b_static = 1;
        sg.ldb = rk.cols;
        sg.k = rk.rows;
        sg.alpha = 1.0;
        p.g3.segs.push_back(sg);
        p.g3.flops += 8LL * o.rows * rk.rows * rk.cols;
        ++cnt;
      }
    t.seg_count = cnt;
    p.g3.tasks.push_back(t);
  }
  p.g1.finalize(stream_, gemm_kind_, dstatus_ + 1);
  p.lc.finalize(stream_);
  p.g3.finalize(stream_, gemm_kind_, dstatus_ + 1);
}

// Gauge shift by repeated Cholesky QR in FP64: two passes; if the first factorisation
// meets a non-positive pivot (numerically rank-deficient sector) three passes, the
// first with a diagonal shift of 1e-14 tr(K)/q (the later passes restore
// orthonormality).  right: per right-bond
// sector c the matrix M_c (rows (a,s), q = d_c columns) becomes A_c with M_c = A_c C_c,
// C_c = R3 R2 R1.  left: per left-bond sector a, M_a (p = d_a rows, columns (s,b)) =
// R^H Q via the Gram matrix M_a M_a^H; C_a = (R3 R2 R1)^H so that M_a = C_a Q_a.
void Engine::gauge_shift(BTensor& M, const BondSpace& b, BTensor& C, bool right) {
  std::map<int, std::vector<int>> by;  // bond sector -> blocks of M
  for (int bi = 0; bi < (int)M.blocks.size(); ++bi) by[M.blocks[bi].key[right ? 2 : 0]].push_back(bi);
  build_bond_layout(C, b);
  alloc(C, true);
  std::vector<long long> off(b.s.size(), 0);
  long long tot = 0;
  for (int c = 0; c < (int)b.s.size(); ++c) {
    off[c] = tot;
    tot += (long long)b.s[c].d * b.s[c].d;
  }
  DevBuf dK(std::max<long long>(tot, 1) * sizeof(cplx), stream_), dRi(std::max<long long>(tot, 1) * sizeof(cplx), stream_);
  DevBuf dT(std::max<long long>(tot, 1) * sizeof(cplx), stream_);
  cplx *Kb = dK.as<cplx>(), *Ri = dRi.as<cplx>(), *Tb = dT.as<cplx>();
  BTensor other;
  other.kind = M.kind;
  other.blocks = M.blocks;
  other.map = M.map;
  other.size = M.size;
  alloc(other, false);
  BTensor* cur = &M;
  BTensor* nxt = &other;
  std::vector<CholTask> ct;
  for (auto& e : by) ct.push_back({Kb + off[e.first], Ri + off[e.first], b.s[e.first].d});
  DevBuf dct = upload(ct, stream_);
  // CholQR2 (two unshifted passes, orthonormal to rounding whenever the first
  // factorisation succeeds); a non-positive pivot in the first pass restarts with
  // the shifted three-pass form
  int npass = 2;
  double shift0 = 0.0;
  for (int pass = 0; pass < npass; ++pass) {
    GemmPlan gk, ga, gr;
    for (auto& e : by) {
      const int c = e.first, q = b.s[c].d;
      GemmTask t{};
      t.c = Kb + off[c];
      t.rows = q;
      t.cols = q;
      t.ldc = q;
      t.seg_begin = (int)gk.segs.size();
      for (int bi : e.second) {
        const Block& bk = M.blocks[bi];
        GemmSeg sg{};
        sg.alpha = 1.0;
        sg.a = cur->ptr(bi);
        sg.b = cur->ptr(bi);
        sg.lda = bk.cols;
        sg.ldb = bk.cols;
        if (right) {  // K = sum blk^H blk
          sg.op_a = OP_C;
          sg.k = bk.rows;
        } else {  // K = sum blk blk^H
          sg.op_b = OP_C;
          sg.k = bk.cols;
        }
        gk.segs.push_back(sg);
      }
      t.seg_count = (int)e.second.size();
      gk.tasks.push_back(t);
    }
    gk.finalize(stream_);
    gk.launch(stream_, Bases4{{0, 0, 0, 0}});
    launch_chol_inv(dct.as<CholTask>(), (int)ct.size(), pass == 0 ? shift0 : 0.0, dstatus_ + 2, stream_);
    if (pass == 0 && shift0 == 0.0) {
      int bad = 0;
      TDVP_CUDA(cudaMemcpyAsync(&bad, dstatus_ + 2, sizeof(int), cudaMemcpyDeviceToHost, stream_));
      TDVP_CUDA(cudaStreamSynchronize(stream_));
      if (bad) {
        TDVP_CUDA(cudaMemsetAsync(dstatus_ + 2, 0, sizeof(int), stream_));
        shift0 = 1e-14;
        npass = 3;
        pass = -1;  // M (= cur) is untouched until the first swap
        continue;
      }
    }
    // A = M R^-1 (right) or Q = R^-H M (left), block by block
    for (auto& e : by) {
      const int c = e.first, q = b.s[c].d;
      for (int bi : e.second) {
        const Block& bk = M.blocks[bi];
        GemmTask t{};
        t.c = nxt->ptr(bi);
        t.rows = bk.rows;
        t.cols = bk.cols;
        t.ldc = bk.cols;
        t.seg_begin = (int)ga.segs.size();
        t.seg_count = 1;
        GemmSeg sg{};
        sg.alpha = 1.0;
        if (right) {
          sg.a = cur->ptr(bi);
          sg.lda = bk.cols;
          sg.b = Ri + off[c];
          sg.ldb = q;
          sg.k = q;
        } else {
          sg.a = Ri + off[c];
          sg.lda = q;
          sg.op_a = OP_C;
          sg.b = cur->ptr(bi);
          sg.ldb = bk.cols;
          sg.k = q;
        }
        ga.segs.push_back(sg);
        ga.tasks.push_back(t);
      }
    }
    ga.finalize(stream_);
    ga.launch(stream_, Bases4{{0, 0, 0, 0}});
    // accumulated factor: C = R (first pass) or C <- R C
    if (pass > 0)
      for (auto& e : by) {
        const int c = e.first, q = b.s[c].d;
        GemmTask t{};
        t.c = Tb + off[c];
        t.rows = q;
        t.cols = q;
        t.ldc = q;
        t.seg_begin = (int)gr.segs.size();
        t.seg_count = 1;
        GemmSeg sg{};
        sg.alpha = 1.0;
        sg.a = Kb + off[c];  // R: the upper triangle of K after the factorisation
        sg.lda = q;
        sg.b = C.ptr(C.find(bkey(c, 0, c)));
        sg.ldb = q;
        sg.k = q;
        gr.segs.push_back(sg);
        gr.tasks.push_back(t);
      }
    if (pass == 0) {
      CopyPlan cp;  // C = R
      for (auto& e : by) {
        const int c = e.first, q = b.s[c].d;
        CopyTask t{};
        t.src = Kb + off[c];
        t.dst = C.ptr(C.find(bkey(c, 0, c)));
        t.rows = q;
        t.cols = q;
        t.src_rs = q;
        t.src_cs = 1;
        t.dst_rs = q;
        t.dst_cs = 1;
        cp.tasks.push_back(t);
      }
      cp.finalize(stream_);
      cp.launch(stream_);
    } else {
      gr.finalize(stream_);
      gr.launch(stream_, Bases4{{0, 0, 0, 0}});
      CopyPlan cp;  // C = T
      for (auto& e : by) {
        const int c = e.first, q = b.s[c].d;
        CopyTask t{};
        t.src = Tb + off[c];
        t.dst = C.ptr(C.find(bkey(c, 0, c)));
        t.rows = q;
        t.cols = q;
        t.src_rs = q;
        t.src_cs = 1;
        t.dst_rs = q;
        t.dst_cs = 1;
        cp.tasks.push_back(t);
      }
      cp.finalize(stream_);
      cp.launch(stream_);
    }
    std::swap(cur, nxt);
  }
  if (cur != &M) std::swap(M.buf, other.buf);
  if (!right) {  // C_a = (R3 R2 R1)^H
    CopyPlan cp;
    for (auto& e : by) {
      const int c = e.first, q = b.s[c].d;
      CopyTask t{};
      t.src = C.ptr(C.find(bkey(c, 0, c)));
      t.dst = Tb + off[c];
      t.rows = q;
      t.cols = q;
      t.src_rs = 1;
      t.src_cs = q;
      t.dst_rs = q;
      t.dst_cs = 1;
      t.conj = 1;
      cp.tasks.push_back(t);
    }
    cp.finalize(stream_);
    cp.launch(stream_);
    TDVP_CUDA(cudaMemcpyAsync(C.data(), Tb, std::max<long long>(tot, 1) * sizeof(cplx), cudaMemcpyDeviceToDevice,
                              stream_));
  }
}

// M <- C M (blocks (c, s, b) of the site to the right of the bond) or M <- M C
// (blocks (a, s, c) of the site to the left)
void Engine::absorb(const BTensor& C, BTensor& M, bool from_left) {
  BTensor out;
  out.kind = M.kind;
  out.blocks = M.blocks;
  out.map = M.map;
  out.size = M.size;
  alloc(out, false);
  GemmPlan g;
  for (int bi = 0; bi < (int)M.blocks.size(); ++bi) {
    const Block& bk = M.blocks[bi];
    const int c = from_left ? bk.key[0] : bk.key[2];
    const int cb = C.find(bkey(c, 0, c));
    if (cb < 0) throw Error(-5, "bond matrix block missing");
    const Block& ck = C.blocks[cb];
    GemmTask t{};
    t.c = out.ptr(bi);
    t.rows = bk.rows;
    t.cols = bk.cols;
    t.ldc = bk.cols;
    t.seg_begin = (int)g.segs.size();
    t.seg_count = 1;
    GemmSeg sg{};
    sg.alpha = 1.0;
    if (from_left) {
      sg.a = C.ptr(cb);
      sg.lda = ck.cols;
      sg.b = M.ptr(bi);
      sg.ldb = bk.cols;
      sg.k = ck.cols;
    } else {
      sg.a = M.ptr(bi);
      sg.lda = bk.cols;
      sg.b = C.ptr(cb);
      sg.ldb = ck.cols;
      sg.k = bk.cols;
    }
    g.segs.push_back(sg);
    g.tasks.push_back(t);
    g.flops += 8LL * bk.rows * bk.cols * sg.k;
  }
  g.finalize(stream_, gemm_kind_, dstatus_ + 1);
  g.launch(stream_, Bases4{{0, 0, 0, 0}});
  stats_.env_flops += g.flops;
  std::swap(M.buf, out.buf);
}

// one site of the one-site sweep: forward evolution of the centre by tau, then (if
// shift) the gauge shift towards the sweep direction, the environment update, the
// backward evolution of the bond matrix by tau and its absorption into the next site
void Engine::site_update1(int i, bool left_to_right, double tau, bool shift) {
  NvtxRange nvtx_range("site_update1");
  auto tp = std::chrono::steady_clock::now();
  auto mark = [&](int ph) {
    if (!profile_) return;
    cudaStreamSynchronize(stream_);
    auto now = std::chrono::steady_clock::now();
    stats_.phase[ph] += std::chrono::duration<double>(now - tp).count();
    tp = now;
  };
  {
    HeffPlan H1;
    plan_heff1(H1, Lenv_[i], Renv_[i + 1], site_[i], bonds_[i], bonds_[i + 1]);
    mark(1);
    expm(H1, site_[i].data(), tau);
    mark(2);
  }
  if (!shift) return;
  BTensor C;
  if (left_to_right) {
    gauge_shift(site_[i], bonds_[i + 1], C, true);
    mark(3);
    update_left_env(Lenv_[i], site_[i], Lenv_[i + 1], bonds_[i], bonds_[i + 1]);
    mark(4);
    HeffPlan H0;
    plan_heff0(H0, Lenv_[i + 1], Renv_[i + 1], C);
    mark(1);
    expm(H0, C.data(), -tau);
    absorb(C, site_[i + 1], true);
    mark(5);
    center_ = i + 1;
  } else {
    gauge_shift(site_[i], bonds_[i], C, false);
    mark(3);
    update_right_env(Renv_[i + 1], site_[i], Renv_[i], bonds_[i], bonds_[i + 1]);
    mark(4);
    HeffPlan H0;
    plan_heff0(H0, Lenv_[i], Renv_[i], C);
    mark(1);
    expm(H0, C.data(), -tau);
    absorb(C, site_[i - 1], false);
    mark(5);
    center_ = i - 1;
  }
}

void Engine::step1(double dt) {
  NvtxRange nvtx_range("tdvp_step_one_site");
  if (bond_only_) throw Error(-2, "a bond problem has no chain to evolve");
  if (!(dt > 0)) throw Error(-1, "invalid step arguments");
  if (center_ != 0) throw Error(-2, "a full time step starts with the orthogonality centre on site 0");
  chain_heff_.reset();
  auto t0 = std::chrono::steady_clock::now();
  const double tau = dt / 2;
  const int L = L_;
  for (int i = 0; i < L; ++i) site_update1(i, true, tau, i + 1 < L);
  for (int i = L - 1; i >= 0; --i) site_update1(i, false, tau, i > 0);
  TDVP_CUDA(cudaStreamSynchronize(stream_));
  check_status();
  stats_.seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  stats_.steps += 1;
  stats_.one_site_steps += 1;
}

int Engine::step_mode(double dt, long long chi_max, double eps, int mode) {
  if (mode < 0 || mode > 2) throw Error(-1, "mode must be 0 (two-site), 1 (one-site) or 2 (adaptive)");
  if (mode == 1 || (mode == 2 && saturated_)) {
    step1(dt);
    return 1;
  }
  cap_hit_ = false;
  step(dt, chi_max, eps);
  if (mode == 2 && cap_hit_) saturated_ = true;
  return 0;
}

void Engine::single_bond(int i, int direction, double dt, long long chi_max, double eps, double* s_ent) {
  if (bond_only_) throw Error(-2, "a bond problem has no chain");
  if (i < 0 || i + 1 >= L_ || !(dt > 0) || chi_max < 1 || !(eps >= 0)) throw Error(-1, "invalid bond update");
  const bool lr = direction == 0;
  if ((lr && center_ != i) || (!lr && center_ != i + 1))
    throw Error(-2, "the orthogonality centre is not on the bond's source site");
  chain_heff_.reset();
  auto t0 = std::chrono::steady_clock::now();
  bond_update(i, lr, dt / 2, chi_max, eps, true, s_ent);
  TDVP_CUDA(cudaStreamSynchronize(stream_));
  check_status();
  stats_.seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// <n>, <S^z>, <docc> of the orthogonality-centre site (left part left-canonical,
// right part right-canonical): sum over centre blocks of O_s Tr(M^H M).
void Engine::measure_center(int* site, double* n, double* sz, double* docc) {
  if (bond_only_) throw Error(-2, "a bond problem has no chain");
  const Model& M = model_;
  const BTensor& T = site_[center_];
  const int NS = 5;
  std::vector<DotTask> dts;
  for (int bi = 0; bi < (int)T.blocks.size(); ++bi) {
    const Block& b = T.blocks[bi];
    int s = b.key[1];
    double w[NS] = {M.occ_n[s], M.occ_up[s], M.occ_dn[s], M.occ_d[s], 1.0};
    for (int k = 0; k < NS; ++k)
      if (w[k] != 0.0) dts.push_back({T.ptr(bi), T.ptr(bi), b.rows, b.cols, b.cols, b.cols, k, w[k]});
  }
  DevBuf ddt = upload(dts, stream_);
  DevBuf dpart(std::max<size_t>(dts.size(), 1) * sizeof(double), stream_), dout(NS * sizeof(double), stream_);
  launch_wdot(ddt.as<DotTask>(), (int)dts.size(), dpart.as<double>(), dout.as<double>(), NS, stream_);
  double r[NS];
  TDVP_CUDA(cudaMemcpyAsync(r, dout.p, NS * sizeof(double), cudaMemcpyDeviceToHost, stream_));
  TDVP_CUDA(cudaStreamSynchronize(stream_));
  const double nrm = r[4] > 0 ? r[4] : 1.0;
  const double nup = r[1] / nrm, ndn = r[2] / nrm, dd = r[3] / nrm;
  const double n_up = nup, n_dn = 1.0 - ndn;
  if (site) *site = center_;
  if (n) *n = n_up + n_dn;
  if (sz) *sz = 0.5 * (n_up - n_dn);
  if (docc) *docc = nup - dd;
}

// ---------------------------------------------------------------------------
// measurement (a9): overlap environments from the centre at site 0
// ---------------------------------------------------------------------------

void Engine::measure(double* n_out, double* sz_out, double* docc_out, double* s_ent, double* energy,
                     double* n_up_out) {
  if (bond_only_) throw Error(-2, "a bond problem has no chain to measure");
  if (center_ != 0) throw Error(-2, "tdvp_measure needs the orthogonality centre on site 0 (after tdvp_step)");
  const Model& M = model_;
  const int L = L_;
  // Omega_0 = 1 on the single sector of the left edge
  BTensor Om;
  Om.kind = OMEGA;
  for (int a = 0; a < (int)bonds_[0].s.size(); ++a) Om.add(bkey(a, 0, a), a, 0, a, 0, 0, bonds_[0].s[a].d, bonds_[0].s[a].d);
  alloc(Om, true);
  std::vector<cplx> one(1, cplx{1.0, 0.0});
  TDVP_CUDA(cudaMemcpyAsync(Om.data(), one.data(), sizeof(cplx), cudaMemcpyHostToDevice, stream_));
  const int NS = 5;  // slots per site: n, n_up, n_dn, n_up n_dn, norm
  DevBuf dres((size_t)L * NS * sizeof(double), stream_);
  DevBuf dent((size_t)std::max(L - 1, 1) * sizeof(double), stream_);
  for (int i = 0; i < L; ++i) {
    const BTensor& T = site_[i];
    // X(a,s,b) = Omega_a T(a,s,b)
    BTensor X;
    for (int bi = 0; bi < (int)T.blocks.size(); ++bi) {
      const Block& b = T.blocks[bi];
      X.add((uint64_t)bi, b.key[0], b.key[1], b.key[2], 0, 0, b.rows, b.cols);
    }
    alloc(X, false);
    GemmPlan g1, g2;
    for (int bi = 0; bi < (int)T.blocks.size(); ++bi) {
      const Block& b = T.blocks[bi];
      int ob = Om.find(bkey(b.key[0], 0, b.key[0]));
      GemmTask t{};
      t.c = X.ptr(bi);
      t.rows = b.rows;
      t.cols = b.cols;
      t.ldc = b.cols;
      t.seg_begin = (int)g1.segs.size();
      t.seg_count = 1;
      GemmSeg sg{};
      sg.a = Om.ptr(ob);
      sg.lda = b.rows;
      sg.b = T.ptr(bi);
      sg.ldb = b.cols;
      sg.k = b.rows;
      sg.alpha = 1.0;
      g1.segs.push_back(sg);
      g1.tasks.push_back(t);
    }
    g1.finalize(stream_);
    g1.launch(stream_, Bases4{{0, 0, 0, 0}});
    // local expectation values
    std::vector<DotTask> dts;
    for (int bi = 0; bi < (int)T.blocks.size(); ++bi) {
      const Block& b = T.blocks[bi];
      int s = b.key[1];
      double w[NS] = {M.occ_n[s], M.occ_up[s], M.occ_dn[s], M.occ_d[s], 1.0};
      for (int k = 0; k < NS; ++k)
        if (w[k] != 0.0) dts.push_back({T.ptr(bi), X.ptr(bi), b.rows, b.cols, b.cols, b.cols, i * NS + k, w[k]});
    }
    DevBuf ddt = upload(dts, stream_);
    DevBuf dpart(std::max<size_t>(dts.size(), 1) * sizeof(double), stream_);
    // write into a per-site staging then copy: wdot writes all slots [0, nslots)
    DevBuf dsite((size_t)(L * NS) * sizeof(double), stream_);
    launch_wdot(ddt.as<DotTask>(), (int)dts.size(), dpart.as<double>(), dsite.as<double>(), L * NS, stream_);
    TDVP_CUDA(cudaMemcpyAsync(dres.as<double>() + i * NS, dsite.as<double>() + i * NS, NS * sizeof(double),
                              cudaMemcpyDeviceToDevice, stream_));
    if (i == L - 1) break;
    // Omega_{i+1}(b) = sum_{a,s} T(a,s,b)^H X(a,s,b)
    BTensor On;
    On.kind = OMEGA;
    const BondSpace& br = bonds_[i + 1];
    for (int b = 0; b < (int)br.s.size(); ++b) On.add(bkey(b, 0, b), b, 0, b, 0, 0, br.s[b].d, br.s[b].d);
    alloc(On, true);
    std::vector<std::vector<int>> byb(br.s.size());
    for (int bi = 0; bi < (int)T.blocks.size(); ++bi) byb[T.blocks[bi].key[2]].push_back(bi);
    for (int b = 0; b < (int)br.s.size(); ++b) {
      GemmTask t{};
      t.c = On.ptr(b);
      t.rows = br.s[b].d;
      t.cols = br.s[b].d;
      t.ldc = br.s[b].d;
      t.seg_begin = (int)g2.segs.size();
      t.seg_count = (int)byb[b].size();
      for (int bi : byb[b]) {
        const Block& tb = T.blocks[bi];
        GemmSeg sg{};
        sg.a = T.ptr(bi);
        sg.lda = tb.cols;
        sg.op_a = OP_C;
        sg.b = X.ptr(bi);
        sg.ldb = tb.cols;
        sg.k = tb.rows;
        sg.alpha = 1.0;
        g2.segs.push_back(sg);
      }
      g2.tasks.push_back(t);
    }
    g2.finalize(stream_);
    g2.launch(stream_, Bases4{{0, 0, 0, 0}});
    if (s_ent) {
      // eigenvalues of each Omega block (Hermitian PSD: singular values) -> entropy
      int ns = (int)br.s.size();
      std::vector<long long> go(ns);
      std::vector<int> so(ns);
      long long gt = 0, vt = 0;
      int stt = 0;
      for (int b = 0; b < ns; ++b) {
        go[b] = gt;
        gt += (long long)br.s[b].d * br.s[b].d;
        so[b] = stt;
        stt += br.s[b].d;
      }
      vt = gt;
      DevBuf dG(gt * sizeof(cplx), stream_), dV(vt * sizeof(cplx), stream_);
      DevBuf dS(stt * sizeof(double), stream_), dP(stt * sizeof(int), stream_);
      TDVP_CUDA(cudaMemcpyAsync(dG.p, On.data(), gt * sizeof(cplx), cudaMemcpyDeviceToDevice, stream_));
      std::vector<SvdTask> st(ns);
      std::vector<TruncSector> ts(ns);
      for (int b = 0; b < ns; ++b) {
        st[b] = {dG.as<cplx>() + go[b], dV.as<cplx>() + go[b], dS.as<double>() + so[b], dP.as<int>() + so[b],
                 br.s[b].d, br.s[b].d};
        ts[b] = {dS.as<double>() + so[b], br.s[b].d, M.mult_dim(br.s[b].t)};
      }
      DevBuf dst = upload(st, stream_), dts2 = upload(ts, stream_);
      jacobi(run_jacobi_rounds(dst.as<SvdTask>(), st, 40, 1e-14, dstatus_, stream_, 0.0, 0.0, nullptr, jscratch()));
      launch_entropy(dts2.as<TruncSector>(), ns, dent.as<double>() + i, stream_);
      TDVP_CUDA(cudaStreamSynchronize(stream_));
    }
    Om = std::move(On);
    TDVP_CUDA(cudaStreamSynchronize(stream_));
  }
  std::vector<double> res((size_t)L * NS);
  TDVP_CUDA(cudaMemcpyAsync(res.data(), dres.p, res.size() * sizeof(double), cudaMemcpyDeviceToHost, stream_));
  std::vector<double> ent(std::max(L - 1, 1));
  if (s_ent)
    TDVP_CUDA(cudaMemcpyAsync(ent.data(), dent.p, (L - 1) * sizeof(double), cudaMemcpyDeviceToHost, stream_));
  if (energy) {
    HeffPlan H1;
    plan_heff1(H1, Lenv_[0], Renv_[1], site_[0], bonds_[0], bonds_[1]);
    DevBuf out(std::max<long long>(H1.n, 1) * sizeof(cplx), stream_);
    H1.apply(site_[0].data(), out.as<cplx>(), stream_);
    DevBuf part((size_t)296 * sizeof(cplx), stream_), e(sizeof(cplx), stream_);
    launch_dots(site_[0].data(), 0, 1, out.as<cplx>(), H1.n, part.as<cplx>(), dots_grid(H1.n), e.as<cplx>(), nullptr,
                stream_);
    cplx he;
    TDVP_CUDA(cudaMemcpyAsync(&he, e.p, sizeof(cplx), cudaMemcpyDeviceToHost, stream_));
    TDVP_CUDA(cudaStreamSynchronize(stream_));
    // the MPO's on-site term -U n'_up n'_dn + (U/2) n' differs from U n_up n_dn of Eq.
    // (FHM) by U S'^z per site, i.e. by U (N - L)/2 in total = U t_L / 2 with t_L the
    // 2S'^z of the last bond (zero at half filling and for every U(1)xSU(2) state)
    *energy = he.x + (model_.su2 ? 0.0 : 0.5 * model_.U * bonds_[L_].s[0].t);
  }
  TDVP_CUDA(cudaStreamSynchronize(stream_));
  check_status();
  // back to the frame of Eq. (FHM): n_up = n'_up, n_dn = 1 - n'_dn
  for (int i = 0; i < L; ++i) {
    const double* r = &res[(size_t)i * NS];
    double nup = r[1], ndn = r[2], dd = r[3];
    double n_up = nup, n_dn = 1.0 - ndn;
    if (n_out) n_out[i] = n_up + n_dn;
    if (sz_out) sz_out[i] = 0.5 * (n_up - n_dn);
    if (docc_out) docc_out[i] = nup - dd;
    if (n_up_out) n_up_out[i] = n_up;
  }
  if (s_ent)
    for (int k = 0; k < L - 1; ++k) s_ent[k] = ent[k];
}

}  // namespace tdvp
