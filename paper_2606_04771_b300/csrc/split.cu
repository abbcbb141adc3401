// K1 (split precision): grouped complex GEMM on the 5th-generation tensor cores.
//
// The same task lists as the FP64 kernel (C = sum_seg alpha op(A) op(B), FP64
// complex blocks) are computed with tcgen05.mma:
//   * the complex product is embedded as one real product,
//       [C_r; C_i] rows (2m, 2m+1) = [[A_r, -A_i]; [A_i, A_r]] [B_r; B_i],
//     so a 64 x 128 complex output tile is one 128 x 128 FP32 accumulator in TMEM;
//   * every FP64 operand is split on the fly into precision pieces: 3xTF32
//     (x = h + l, products h*h + h*l + l*h, FP32 accumulation in TMEM) or BF16x4
//     (scaled signed digits, exact per-order accumulation; gemm_exact_kernel);
//   * producer warps load FP64 tiles from global memory, split them and store
//     them in the 128-byte-swizzled K-major layout the MMA descriptors expect;
//     one thread issues the MMAs; the accumulator is read back from TMEM
//     (tcgen05.ld) and written as FP64 complex results (the BF16x4 kernel is
//     persistent with separate epilogue warps and two accumulator sets).
// Every mbarrier wait is bounded: on expiry the kernel records an error in
// *status, stops issuing work, releases its TMEM and returns.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "common.hpp"
#include "kernels.hpp"

namespace tdvp {

namespace {

constexpr int TM = 64;         // complex rows per tile (UMMA M = 128 real-embedded rows)
constexpr int TN = 128;        // complex columns per tile (UMMA N)
constexpr int NPROD = 128;     // producer / epilogue threads (warps 0-3)
constexpr int NTHREADS = 160;  // + one MMA warp
constexpr int STAGES = 2;
constexpr uint32_t SPIN_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok;
}

// bounded wait: returns false (and flags *err) when the limit is hit
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* err) {
  for (uint32_t it = 0; it < SPIN_LIMIT; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 1023) == 1023 && *err) return false;
  }
  *err = 1;
  return false;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// arrive on a stage's full barrier announcing the bytes its bulk copies will bring
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
// global -> shared bulk copy (16-byte aligned, size a multiple of 16) completing on b
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                      // leading-dimension offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride between 8-row groups
  d |= (uint64_t)1 << 46;                      // descriptor version for this architecture
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// instruction descriptor: D f32, A/B format fmt (kind::tf32: 2, kind::f16 bf16: 1), K-major, M=128, N
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t M, uint32_t N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (KIND == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// byte offset of element (row, kk) with 4-byte elements in a K-major SW128 tile (32 per row)
__device__ __forceinline__ uint32_t sw_off4(int row, int kk) {
  return row * 128 + ((((kk >> 2) ^ (row & 7)) & 7) << 4) + ((kk & 3) << 2);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Split configuration of the 3xTF32 kernel: 2 planes (h, l), K-chunk = 16 complex k
// = 32 tf32 = one 128-byte swizzle atom row per plane per stage.
template <int KIND>
struct Cfg;
template <>
struct Cfg<0> {
  static constexpr int PLANES = 2, KC = 16, ESZ = 4, KSTEP = 8;
};

constexpr int PLANE_BYTES = 128 * 128;  // 128 rows x 128 bytes

// split x into the pieces of the chosen format
template <int KIND>
__device__ __forceinline__ void split_val(double x, float* out) {
  float h = tf32_round((float)x);
  float l = tf32_round((float)(x - (double)h));
  out[0] = h;
  out[1] = l;
}

template <int KIND>
__device__ __forceinline__ void store_pair(uint8_t* plane, int row, int kk, float v0, float v1) {
  *reinterpret_cast<float2*>(plane + sw_off4(row, kk)) = make_float2(v0, v1);
}

template <int KIND>
__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_split_kernel(const GemmTask* __restrict__ tasks, const GemmSeg* __restrict__ segs,
                      const int3* __restrict__ tiles, const Bases4 B, int* __restrict__ status) {
  using C = Cfg<KIND>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-align the stage buffers
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage_base = smem;  // STAGES x (PLANES A + PLANES B) planes
  __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int err;

  const int3 tr = tiles[blockIdx.x];
  const GemmTask t = tasks[tr.x];
  cplx* const cptr = rebase(B, t.c_base, t.c);
  const int m0 = tr.y * TM, n0 = tr.z * TN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // total K chunks of this task
  int nchunks = 0;
  for (int s = 0; s < t.seg_count; ++s) nchunks += (segs[t.seg_begin + s].k + C::KC - 1) / C::KC;

  if (nchunks == 0) {  // no contribution: the output tile is zero
    for (int e = tid; e < TM * TN; e += NTHREADS) {
      int r = m0 + e / TN, c = n0 + e % TN;
      if (r < t.rows && c < t.cols) cptr[(long long)r * t.ldc + c] = {0.0, 0.0};
    }
    return;
  }

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], NPROD / 32);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* verr = &err;

  if (warp < 4) {
    // ---------------- producers ----------------
    int it = 0;
    for (int sgi = 0; sgi < t.seg_count && !*verr; ++sgi) {
      const GemmSeg sg = segs[t.seg_begin + sgi];
      const cplx* ap = rebase(B, sg.a_base, sg.a);
      const cplx* bp = rebase(B, sg.b_base, sg.b);
      const double al = sg.alpha;
      for (int k0 = 0; k0 < sg.k; k0 += C::KC, ++it) {
        const int s = it % STAGES;
        if (!mbar_wait(&empty_bar[s], ((it / STAGES) & 1) ^ 1, verr)) break;
        uint8_t* st = stage_base + (size_t)s * (2 * C::PLANES) * PLANE_BYTES;
        // A: TM complex rows x KC complex k -> rows (2m, 2m+1), columns (2k, 2k+1)
        for (int e = tid; e < TM * C::KC; e += NPROD) {
          const int m = e / C::KC, k = e % C::KC;
          const int gr = m0 + m, gk = k0 + k;
          cplx v = {0.0, 0.0};
          if (gr < t.rows && gk < sg.k) {
            if (sg.op_a == OP_N) v = ap[(long long)gr * sg.lda + gk];
            else {
              v = ap[(long long)gk * sg.lda + gr];
              v.y = -v.y;
            }
          }
          float re[2], im[2];
          split_val<KIND>(v.x * al, re);
          split_val<KIND>(v.y * al, im);
#pragma unroll
          for (int p = 0; p < C::PLANES; ++p) {
            uint8_t* pl = st + p * PLANE_BYTES;
            store_pair<KIND>(pl, 2 * m, 2 * k, re[p], -im[p]);
            store_pair<KIND>(pl, 2 * m + 1, 2 * k, im[p], re[p]);
          }
        }
        // B: KC complex k x TN complex n -> K-major rows n, columns (2k, 2k+1)
        for (int e = tid; e < TN * C::KC; e += NPROD) {
          const int n = e % TN, k = e / TN;
          const int gc = n0 + n, gk = k0 + k;
          cplx v = {0.0, 0.0};
          if (gc < t.cols && gk < sg.k) {
            if (sg.op_b == OP_N) v = bp[(long long)gk * sg.ldb + gc];
            else {
              v = bp[(long long)gc * sg.ldb + gk];
              v.y = -v.y;
            }
          }
          float re[2], im[2];
          split_val<KIND>(v.x, re);
          split_val<KIND>(v.y, im);
#pragma unroll
          for (int p = 0; p < C::PLANES; ++p) {
            uint8_t* pl = st + (C::PLANES + p) * PLANE_BYTES;
            store_pair<KIND>(pl, n, 2 * k, re[p], im[p]);
          }
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full_bar[s]);
      }
    }
    // ---------------- epilogue ----------------
    if (mbar_wait(&done_bar, 0, verr)) {
      tc_fence_after();
      const int row = warp * 32 + lane;  // real-embedded row = TMEM lane
      const int m = row >> 1, part = row & 1;
      const int gr = m0 + m;
      for (int c0 = 0; c0 < TN; c0 += 32) {
        uint32_t v[32];
        const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(addr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (gr < t.rows) {
          double* out = reinterpret_cast<double*>(cptr + (t.rowoff ? t.rowoff[gr] : (long long)gr * t.ldc));
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int gc = n0 + c0 + j;
            if (gc < t.cols) out[2 * gc + part] = (double)__uint_as_float(v[j]);
          }
        }
      }
    }
  } else if (warp == 4 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t idesc = make_idesc(KIND == 0 ? 2u : 1u, 128, TN);
    uint32_t acc = 0;
    int it = 0;
    bool ok = true;
    for (int sgi = 0; sgi < t.seg_count && ok; ++sgi) {
      const int kk = segs[t.seg_begin + sgi].k;
      for (int k0 = 0; k0 < kk; k0 += C::KC, ++it) {
        const int s = it % STAGES;
        if (!mbar_wait(&full_bar[s], (it / STAGES) & 1, verr)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t st = smem_u32(stage_base + (size_t)s * (2 * C::PLANES) * PLANE_BYTES);
#pragma unroll
        for (int q = 0; q < 128 / (C::KSTEP * C::ESZ); ++q) {
          const uint32_t koff = q * C::KSTEP * C::ESZ;
          const uint64_t ah = sw128_desc(st + koff), alo = sw128_desc(st + PLANE_BYTES + koff);
          const uint64_t bh = sw128_desc(st + 2 * PLANE_BYTES + koff), blo = sw128_desc(st + 3 * PLANE_BYTES + koff);
          mma<KIND>(tmem, ah, bh, idesc, acc);
          acc = 1;
          mma<KIND>(tmem, ah, blo, idesc, 1);
          mma<KIND>(tmem, alo, bh, idesc, 1);
        }
        mma_commit(&empty_bar[s]);
      }
    }
    if (ok) mma_commit(&done_bar);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
  }
  if (tid == 0 && err) atomicAdd(status, 1);
}

// ---------------------------------------------------------------------------
// BF16x4 with exact accumulation (Ozaki-style splitting)
//
// Every complex output row m of a tile gets a power-of-two scale 2^e_m >= max|A[m,:]|
// and every output column n a scale 2^f_n >= max|B[:,n]| (over all segments of the
// task).  Each FP64 value x is turned into the integer X = round(x 2^(30-e)) with
// |X| <= 2^30, written as X = s0 2^24 + s1 2^16 + s2 2^8 + s3 with signed digits
// |s_i| <= 128 (exact BF16 values).  Products s_i(a) s_j(b) are integers below 2^14,
// so the FP32 sums of all products of one order o = i + j (o = 0..3) held in four
// TMEM accumulators are exact integers (for any realistic K); the epilogue forms
// V = ((acc0 2^8 + acc1) 2^8 + acc2) 2^8 + acc3 in 64-bit integers and converts once.  Dropped products (order >= 4) and the rounding of X
// bound the error by ~2^-30 of the row/column scales.  With x = 2^(e-30) X and
// X_a X_b = sum_o 2^(8(6-o)) (order-o digit products), the kept orders give
// 2^24 V, hence C = 2^(e_m + f_n - 36) V.
// ---------------------------------------------------------------------------

constexpr int XN = 64;                  // complex columns per tile
constexpr int XKC = 16;                 // complex k per chunk (32 bf16 = one 64-byte row)
constexpr int XA_PLANE = 128 * 64;      // one A digit plane: 128 embedded rows x 64 bytes
constexpr int XB_PLANE = 64 * 64;       // one B digit plane: 64 rows x 64 bytes
constexpr int XSTAGE = 4 * XA_PLANE + 4 * XB_PLANE;  // 48 KB: 4 A planes + 4 B planes
constexpr int XSTAGES = 4;              // 192 KB of stages: one persistent CTA per SM
constexpr int XPROD = 256;              // producer threads (warps 0-7)
constexpr int XMMA_WARP = XPROD / 32;   // MMA issuer warp (8)
constexpr int XEPI = 256;               // epilogue threads (warps 9-16, two per TMEM lane quarter)
constexpr int XTHREADS = XPROD + 32 + XEPI;
constexpr int XACC = 4 * XN;            // TMEM columns of one accumulator set (four orders)


// X = round(x 2^(30 - e)) as int (|X| <= 2^30); x must satisfy |x| <= 2^e
__device__ __forceinline__ int fixed30(double x, int e) {
  if (e <= -2000) return 0;
  const unsigned long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero or subnormal: below 2^-1022, far under the scale
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  // x = mant 2^(ex - 1075); X = mant 2^(ex - 1075 + 30 - e) = mant >> r
  const int r = 1045 + e - ex;
  long long X;
  if (r >= 64) X = 0;
  else if (r <= 0) X = (long long)(mant << (-r));  // cannot happen for |x| <= 2^e (r >= 22)
  else X = (long long)((mant + (1ull << (r - 1))) >> r);
  return (b >> 63) ? -(int)X : (int)X;
}

// Bit pattern of the double V * 2^ee, built with integer operations only (64-bit
// int-to-float conversions run on the FP64-rate pipe of this part): exact for
// |V| < 2^53, rounded to nearest (ties away) above; 0 when V = 0 or the result falls
// below the normal range.
__device__ __forceinline__ long long scaled_double_bits(long long V, int ee) {
  if (V == 0) return 0;
  const unsigned long long sgn = V < 0 ? (1ull << 63) : 0ull;
  unsigned long long u = V < 0 ? 0ull - (unsigned long long)V : (unsigned long long)V;
  int msb = 63 - __clzll((long long)u);
  if (msb > 52) {  // keep 53 significant bits
    int sh = msb - 52;
    u = (u + (1ull << (sh - 1))) >> sh;
    if (u >> 53) {  // the rounding carried into a new bit
      u >>= 1;
      ++sh;
    }
    ee += sh;
    msb = 52;
  }
  const int ex = msb + 1023 + ee;
  if (ex <= 0) return (long long)sgn;
  const unsigned long long mant = (u << (52 - msb)) & ((1ull << 52) - 1);
  return (long long)(sgn | ((unsigned long long)ex << 52) | mant);
}

__device__ __forceinline__ void digits4(int X, float* d) {
  // X = d0 2^24 + d1 2^16 + d2 2^8 + d3, |d_i| <= 128
  int r = X;
  int d3 = ((r + 128) & 255) - 128;
  r = (r - d3) >> 8;
  int d2 = ((r + 128) & 255) - 128;
  r = (r - d2) >> 8;
  int d1 = ((r + 128) & 255) - 128;
  r = (r - d1) >> 8;
  d[0] = (float)r;
  d[1] = (float)d1;
  d[2] = (float)d2;
  d[3] = (float)d3;
}

// K-major tiles with 64-byte rows (32 bf16) in the 64-byte swizzle: the 16-byte chunk
// index of a row is XORed with (row / 2) mod 4 (the address bits 7-8 folded onto bits
// 4-5); 8-row groups are 512 bytes apart
__device__ __forceinline__ uint32_t sw64_off2(int row, int kk) {
  return row * 64 + ((((kk >> 3) ^ (row >> 1)) & 3) << 4) + ((kk & 7) << 1);
}

__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;              // leading-dimension offset (unused for this layout)
  d |= (uint64_t)(512 >> 4) << 32;     // stride between 8-row groups
  d |= (uint64_t)1 << 46;              // descriptor version for this architecture
  d |= (uint64_t)4 << 61;              // 64-byte swizzle
  return d;
}

__device__ __forceinline__ void st_bf2_64(uint8_t* plane, int row, int kk, float v0, float v1) {
  *reinterpret_cast<__nv_bfloat162*>(plane + sw64_off2(row, kk)) = __floats2bfloat162_rn(v0, v1);
}

template <int NCOL>
__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(addr)
      : "memory");
}

// ---- operand splitting, once per launch --------------------------------------
// pass 1: per-row (A) / per-column (B) maxima of |Re|, |Im| into the operand's scale
// group.  Only the binary exponent of a maximum matters (the scale is the power of two
// just above it), so each group row / column holds a 32-bit tag: the launch's epoch in
// bits 12-31 and the largest biased exponent seen in bits 0-11; an unsigned atomicMax
// keeps the newest epoch's largest exponent, and a tag of an older epoch means "no
// non-zero element in this launch" -- no reset pass is needed between launches.  One
// CTA per operand walks its elements in storage order (coalesced) and reduces into
// shared-memory slots, then merges the slots into the group.
constexpr int DIGIT_SLOTS = 6144;  // 24 KB of slots; longer rows/columns go to global atomics

__device__ __forceinline__ unsigned biased_exp(double x) {
  return (unsigned)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
}

__global__ void __launch_bounds__(256) digit_max_kernel(const DigitOp* __restrict__ ops,
                                                        const int2* __restrict__ jobs, const Bases4 B,
                                                        unsigned* __restrict__ tags, unsigned epoch, int job) {
  // one CTA per job: elements [e0, e0 + job) of one operand (the jobs of
  // digit_convert_kernel), so a large operand is reduced by many CTAs at once
  const int2 jb = jobs[blockIdx.x];
  const DigitOp o = ops[jb.x];
  const cplx* src = rebase(B, o.base, o.src);
  extern __shared__ unsigned slot[];
  const int nslot = o.side == 0 ? o.rows : o.cols;
  const int goff = o.side == 0 ? o.row0 : o.col0;  // the operand's first row / column in its group
  const bool local = nslot <= DIGIT_SLOTS;
  const double sa = (o.side == 0 && o.alpha != 1.0) ? fabs(o.alpha) : 1.0;
  if (local)
    for (int i = threadIdx.x; i < nslot; i += 256) slot[i] = 0u;
  __syncthreads();
  const long long n = min((long long)o.rows * o.cols, (long long)jb.y + job);
  // storage order: OP_N stores rows of length cols, OP_C stores columns of length rows
  const int inner = o.op == OP_N ? o.cols : o.rows;
#pragma unroll 4
  for (long long e = jb.y + threadIdx.x; e < n; e += 256) {
    const int outer = (int)(e / inner), in = (int)(e - (long long)outer * inner);
    const cplx v = src[(long long)outer * o.ld + in];
    const int r = o.op == OP_N ? outer : in, c = o.op == OP_N ? in : outer;
    const unsigned ex = biased_exp(sa * fmax(fabs(v.x), fabs(v.y)));
    if (!ex) continue;  // zero (or subnormal, which the split rounds to zero)
    const int sidx = o.side == 0 ? r : c;
    if (local) atomicMax(&slot[sidx], ex);
    else atomicMax(&tags[o.grp + goff + sidx], (epoch << 12) | ex);
  }
  __syncthreads();
  if (local)
    for (int i = threadIdx.x; i < nslot; i += 256) {
      const unsigned ex = slot[i];
      if (ex) atomicMax(&tags[o.grp + goff + i], (epoch << 12) | ex);
    }
}

// the scale exponent of a group row / column in this launch: the smallest e with
// max|x| <= 2^e, or -2000 when the row / column holds no non-zero element
__device__ __forceinline__ int tag_exp(unsigned tag, unsigned epoch) {
  return (tag >> 12) == epoch ? (int)(tag & 0xFFF) - 1022 : -2000;
}

__device__ __forceinline__ unsigned long long pack_digits(double re, double im, int e) {
  float d[4], f[4];
  digits4(fixed30(re, e), d);
  digits4(fixed30(im, e), f);
  unsigned long long w = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    w |= (unsigned long long)((unsigned)((int)d[i]) & 0xFFu) << (8 * i);
    w |= (unsigned long long)((unsigned)((int)f[i]) & 0xFFu) << (8 * (4 + i));
  }
  return w;
}

// one element's digits into the operand's records, or into its tile image (the
// planes of the GEMM stage it will be copied to, in the stage's swizzled layout)
__device__ __forceinline__ void store_digits(const DigitOp& o, int r, int c, double re, double im, int e) {
  if (o.img_nkc <= 0) {
    const long long at = o.kmajor ? (long long)(o.col0 + c) * o.dig_ld + o.row0 + r
                                  : (long long)(o.row0 + r) * o.dig_ld + o.col0 + c;
    o.dig[at] = pack_digits(re, im, e);
    return;
  }
  float dr[4], di[4];
  digits4(fixed30(re, e), dr);
  digits4(fixed30(im, e), di);
  uint8_t* base = reinterpret_cast<uint8_t*>(o.dig);
  if (o.side == 0) {  // A: row R, k; embedded rows 2m (re, -im) and 2m + 1 (im, re)
    const int R = o.row0 + r, k = o.col0 + c, m = R & 63, kk = k & 15;
    uint8_t* t = base + ((long long)(R >> 6) * o.img_nkc + (k >> 4)) * (4 * XA_PLANE);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      st_bf2_64(t + p * XA_PLANE, 2 * m, 2 * kk, dr[p], -di[p]);
      st_bf2_64(t + p * XA_PLANE, 2 * m + 1, 2 * kk, di[p], dr[p]);
    }
  } else {  // B: k, column n; row n of the tile holds (re, im)
    const int k = o.row0 + r, n = o.col0 + c, kk = k & 15;
    uint8_t* t = base + ((long long)(n / o.img_tn) * o.img_nkc + (k >> 4)) * (4 * XB_PLANE);
#pragma unroll
    for (int p = 0; p < 4; ++p) st_bf2_64(t + p * XB_PLANE, n % o.img_tn, 2 * kk, dr[p], di[p]);
  }
}


// pass 2: every element of every operand as one 8-byte record (Re digits 0-3, Im
// digits 0-3, signed bytes) at its place in the digit records (row-major, or column-
// major for a K-major B operand); jobs = (operand, first element).  The thread of
// column 0 (A) or row 0 (B) also stores the exponent for the GEMM's epilogue.
constexpr int DIGIT_JOB = 4096;
__global__ void __launch_bounds__(256) digit_convert_kernel(const DigitOp* __restrict__ ops,
                                                            const int2* __restrict__ jobs, const Bases4 B,
                                                            const unsigned* __restrict__ tags, unsigned epoch,
                                                            int* __restrict__ exps) {
  const int2 jb = jobs[blockIdx.x];
  const DigitOp o = ops[jb.x];
  const cplx* src = rebase(B, o.base, o.src);
  const long long n = (long long)o.rows * o.cols;
  const long long e1 = min(n, (long long)jb.y + DIGIT_JOB);
#pragma unroll 4
  for (long long e = jb.y + threadIdx.x; e < e1; e += 256) {
    // K-major B operands are walked column by column (their records are contiguous
    // along a column), everything else row by row
    int r, c;
    if (o.kmajor) {
      c = (int)(e / o.rows);
      r = (int)(e - (long long)c * o.rows);
    } else {
      r = (int)(e / o.cols);
      c = (int)(e - (long long)r * o.cols);
    }
    cplx v = o.op == OP_N ? src[(long long)r * o.ld + c] : src[(long long)c * o.ld + r];
    if (o.op != OP_N) v.y = -v.y;
    if (o.alpha != 1.0) {
      v.x *= o.alpha;
      v.y *= o.alpha;
    }
    const int gi = o.grp + (o.side == 0 ? o.row0 + r : o.col0 + c);
    const int ex = tag_exp(tags[gi], epoch);
    if (o.side == 0 ? c == 0 : r == 0) exps[gi] = ex;
    store_digits(o, r, c, v.x, v.y, ex);
  }
}

// Both passes in one kernel for an operand that holds whole rows (A) / columns (B) of
// its scale group (every element of such a line is in this operand): one CTA per
// operand reduces the line exponents in shared memory, then converts every element
// and stores the line exponents.  The lines have at most DIGIT_SLOTS entries.
__global__ void __launch_bounds__(256) digit_split_own_kernel(const DigitOp* __restrict__ ops, const Bases4 B,
                                                              int* __restrict__ exps) {
  const DigitOp o = ops[blockIdx.x];
  const cplx* src = rebase(B, o.base, o.src);
  extern __shared__ unsigned slot[];
  const int nslot = o.side == 0 ? o.rows : o.cols;
  const double sa = (o.side == 0 && o.alpha != 1.0) ? fabs(o.alpha) : 1.0;
  for (int i = threadIdx.x; i < nslot; i += 256) slot[i] = 0u;
  __syncthreads();
  const long long n = (long long)o.rows * o.cols;
  const int inner = o.op == OP_N ? o.cols : o.rows;
  for (long long e = threadIdx.x; e < n; e += 256) {
    const int outer = (int)(e / inner), in = (int)(e - (long long)outer * inner);
    const cplx v = src[(long long)outer * o.ld + in];
    const int r = o.op == OP_N ? outer : in, c = o.op == OP_N ? in : outer;
    const unsigned ex = biased_exp(sa * fmax(fabs(v.x), fabs(v.y)));
    if (ex) atomicMax(&slot[o.side == 0 ? r : c], ex);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nslot; i += 256)
    exps[o.grp + (o.side == 0 ? o.row0 : o.col0) + i] = slot[i] ? (int)slot[i] - 1022 : -2000;
  for (long long e = threadIdx.x; e < n; e += 256) {
    int r, c;
    if (o.kmajor) {
      c = (int)(e / o.rows);
      r = (int)(e - (long long)c * o.rows);
    } else {
      r = (int)(e / o.cols);
      c = (int)(e - (long long)r * o.cols);
    }
    cplx v = o.op == OP_N ? src[(long long)r * o.ld + c] : src[(long long)c * o.ld + r];
    if (o.op != OP_N) v.y = -v.y;
    if (o.alpha != 1.0) {
      v.x *= o.alpha;
      v.y *= o.alpha;
    }
    const unsigned ex = slot[o.side == 0 ? r : c];
    store_digits(o, r, c, v.x, v.y, ex ? (int)ex - 1022 : -2000);
  }
}

__device__ __forceinline__ float sbyte(unsigned long long w, int i) { return (float)(int)(signed char)(w >> (8 * i)); }

// the B record a producer thread handles: element e of a chunk (XKC k x XN columns);
// consecutive threads take consecutive columns of one k (row-major records, loads
// coalesced along the row) or consecutive k of one column (K-major records, loads
// coalesced along the column, and the bf16 stores of a warp fill one 128-byte row of
// the swizzled plane, free of bank conflicts)
__device__ __forceinline__ void b_coords(int e, int kmajor, int& n, int& k) {
  if (kmajor) {
    n = e / XKC;
    k = e % XKC;
  } else {
    n = e % XN;
    k = e / XN;
  }
}

__device__ __forceinline__ int task_chunks(const GemmTask& t, const GemmSeg* __restrict__ segs) {
  int n = 0;
  for (int s = 0; s < t.seg_count; ++s) n += (segs[t.seg_begin + s].k + XKC - 1) / XKC;
  return n;
}

// Persistent, warp-specialised BF16x4 kernel: one CTA per SM walks the tile list
// (sorted by cost) with stride gridDim.x.  Warps 0-7 unpack digit records into BF16
// planes of a two-stage ring, warp 8 issues the MMAs into one of two TMEM
// accumulator sets, warps 9-16 drain the other set (exact combination, scaling,
// FP64 stores) while the next tile accumulates.
// The tiles of up to EXACT_MAX_SLICES task lists (one GEMM plan each, with its own
// bases, exponents and status word) run in one launch: tile ti of the concatenated
// list belongs to slice s with L.start[s] <= ti < L.start[s + 1].  Every tile is
// computed the same way whichever launch and CTA take it.
__device__ __forceinline__ int slice_of(const ExactLaunch& L, int ti) {
  int s = L.nslices - 1;
  while (s > 0 && ti < L.start[s]) --s;
  return s;
}

// IMG: every task of the launch holds tile images; one producer thread then walks its
// tiles with their descriptors loaded once per tile and fetches every stage by bulk
// copies (the full barriers count that one arrival), and warps 1-7 have no work.
template <bool IMG>
__global__ void __launch_bounds__(XTHREADS, 1) gemm_exact_kernel(const __grid_constant__ ExactLaunch L) {
  const int ntiles = L.start[L.nslices];
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* stage_base =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full_bar[XSTAGES], empty_bar[XSTAGES], tfull[2], tempty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int err;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < XSTAGES; ++s) {
      mbar_init(&full_bar[s], IMG ? 1 : XPROD / 32);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], XEPI / 32);
    }
    err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(2 * XACC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* verr = &err;

  if (IMG && warp < XPROD / 32) {
    // ---------------- producer: bulk copies of tile images ----------------
    if (warp == 0 && lane == 0) {
      int it = 0;
      for (int ti = blockIdx.x; ti < ntiles && !*verr; ti += gridDim.x) {
        const int sl = slice_of(L, ti);
        const ExactSlice& S = L.sl[sl];
        const int3 tr = S.tiles[ti - L.start[sl]];
        const GemmTask t = S.tasks[tr.x];
        if (task_chunks(t, S.segs) == 0) continue;  // the MMA issuer skips it too
        const GemmSeg sg = S.segs[t.seg_begin];     // packed tasks: one segment
        const int nkc = (sg.k + XKC - 1) / XKC;
        const uint8_t* ga =
            reinterpret_cast<const uint8_t*>(sg.a_dig) + (long long)tr.y * nkc * (long long)(4 * XA_PLANE);
        const uint8_t* gb =
            reinterpret_cast<const uint8_t*>(sg.b_dig) + (long long)tr.z * nkc * (long long)(4 * XB_PLANE);
        bool ok = true;
        for (int kc = 0; kc < nkc; ++kc, ++it) {
          const int s = it % XSTAGES;
          if (!mbar_wait(&empty_bar[s], ((it / XSTAGES) & 1) ^ 1, verr)) {
            ok = false;
            break;
          }
          uint8_t* st = stage_base + (size_t)s * XSTAGE;
          mbar_arrive_expect(&full_bar[s], 4 * XA_PLANE + 4 * XB_PLANE);
          bulk_g2s(st, ga + (long long)kc * (4 * XA_PLANE), 4 * XA_PLANE, &full_bar[s]);
          bulk_g2s(st + 4 * XA_PLANE, gb + (long long)kc * (4 * XB_PLANE), 4 * XB_PLANE, &full_bar[s]);
        }
        if (!ok) break;
      }
    }
  } else if (warp < XPROD / 32) {
    // ---------------- producers ----------------
    // The CTA's chunks (tile, segment, k0) in order; the records of the next chunk are
    // loaded into registers before the current chunk is unpacked, so the loads of one
    // chunk overlap the shared-memory stores of the previous one.
    const int gtid = tid;
    constexpr int GT = XPROD;
    constexpr int NA = TM * XKC / GT, NB = XN * XKC / GT;
    auto advance = [&](int& ti, int& sgi, int& k0) -> bool {
      k0 += XKC;
      while (ti < ntiles) {
        const int sl = slice_of(L, ti);
        const ExactSlice& S = L.sl[sl];
        const GemmTask& t = S.tasks[S.tiles[ti - L.start[sl]].x];
        while (sgi < t.seg_count) {
          if (k0 < S.segs[t.seg_begin + sgi].k) return true;
          ++sgi;
          k0 = 0;
        }
        ti += gridDim.x;
        sgi = 0;
        k0 = 0;
      }
      return false;
    };
    auto fetch = [&](int ti, int sgi, int k0, unsigned long long* wa, unsigned long long* wb) {
      const int sl = slice_of(L, ti);
      const ExactSlice& S = L.sl[sl];
      const int3 tr = S.tiles[ti - L.start[sl]];
      const GemmTask& t = S.tasks[tr.x];
      const GemmSeg& sg = S.segs[t.seg_begin + sgi];
      const int tn = t.tn > 0 ? t.tn : XN;
      const int m0 = tr.y * TM, n0 = tr.z * tn, kk = sg.k, rows = t.rows, cols = t.cols;
      const unsigned long long* ad = sg.a_dig;
      const unsigned long long* bd = sg.b_dig;
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int e = gtid + j * GT, m = e / XKC, k = e % XKC;
        const int gr = m0 + m, gk = k0 + k;
        wa[j] = (gr < rows && gk < kk) ? __ldg(ad + (long long)gr * kk + gk) : 0ull;
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        int n, k;
        b_coords(gtid + j * GT, t.b_kmajor, n, k);
        const int gc = n0 + n, gk = k0 + k;
        wb[j] = (n < tn && gc < cols && gk < kk)
                    ? __ldg(bd + (t.b_kmajor ? (long long)gc * kk + gk : (long long)gk * cols + gc))
                    : 0ull;
      }
    };
    auto is_img = [&](int tix) {
      const int sl = slice_of(L, tix);
      return L.sl[sl].tasks[L.sl[sl].tiles[tix - L.start[sl]].x].img != 0;
    };
    int ti = blockIdx.x, sgi = 0, k0 = -XKC;
    bool have = advance(ti, sgi, k0);
    unsigned long long wa[NA], wb[NB], na_[NA], nb_[NB];
    if (have && !is_img(ti)) fetch(ti, sgi, k0, wa, wb);
    for (int it = 0; have && !*verr; ++it) {
      const int bsl = slice_of(L, ti);
      const int bkm = L.sl[bsl].tasks[L.sl[bsl].tiles[ti - L.start[bsl]].x].b_kmajor;
      int ti2 = ti, sgi2 = sgi, k02 = k0;
      const bool have2 = advance(ti2, sgi2, k02);
      if (have2 && !is_img(ti2)) fetch(ti2, sgi2, k02, na_, nb_);
      const int s = it % XSTAGES;
      if (!mbar_wait(&empty_bar[s], ((it / XSTAGES) & 1) ^ 1, verr)) break;
      uint8_t* st = stage_base + (size_t)s * XSTAGE;
      if (is_img(ti)) {
        // tile images: one thread fetches the stage's A and B planes with two bulk
        // copies; the other producer warps only arrive, as the barrier counts eight
        if (warp == 0 && lane == 0) {
          const ExactSlice& S = L.sl[bsl];
          const int3 tr = S.tiles[ti - L.start[bsl]];
          const GemmTask& t = S.tasks[tr.x];
          const GemmSeg& sg = S.segs[t.seg_begin + sgi];
          const int nkc = (sg.k + XKC - 1) / XKC, kc = k0 / XKC;
          const uint8_t* ga = reinterpret_cast<const uint8_t*>(sg.a_dig) +
                              ((long long)tr.y * nkc + kc) * (long long)(4 * XA_PLANE);
          const uint8_t* gb = reinterpret_cast<const uint8_t*>(sg.b_dig) +
                              ((long long)tr.z * nkc + kc) * (long long)(4 * XB_PLANE);
          mbar_arrive_expect(&full_bar[s], 4 * XA_PLANE + 4 * XB_PLANE);
          bulk_g2s(st, ga, 4 * XA_PLANE, &full_bar[s]);
          bulk_g2s(st + 4 * XA_PLANE, gb, 4 * XB_PLANE, &full_bar[s]);
        } else if (lane == 0) {
          mbar_arrive(&full_bar[s]);
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < NA; ++j) wa[j] = na_[j];
#pragma unroll
        for (int j = 0; j < NB; ++j) wb[j] = nb_[j];
        ti = ti2;
        sgi = sgi2;
        k0 = k02;
        have = have2;
        continue;
      }
      // A: 64 complex rows x 16 complex k -> 4 digit planes of 128 rows x 32 bf16,
      // B: 16 complex k x 64 complex n -> 4 digit planes of 64 rows x 32 bf16.  A half
      // warp fills one 64-byte row; the upper half warp writes its two embedded rows in
      // the other order, so that each store instruction touches two rows 3 apart (the
      // two halves of the 128 banks' worth) rather than 2 apart (the same banks).
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int e = gtid + j * GT, m = e / XKC, k = e % XKC;
        const bool up = (lane >> 4) & 1;
        const int r0 = 2 * m + (up ? 1 : 0), r1 = 4 * m + 1 - r0;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const float re = sbyte(wa[j], p), im = sbyte(wa[j], 4 + p);
          uint8_t* pl = st + p * XA_PLANE;
          // row 2m holds (re, -im), row 2m+1 holds (im, re)
          st_bf2_64(pl, r0, 2 * k, up ? im : re, up ? re : -im);
          st_bf2_64(pl, r1, 2 * k, up ? re : im, up ? -im : re);
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        int n, k;
        b_coords(gtid + j * GT, bkm, n, k);
#pragma unroll
        for (int p = 0; p < 4; ++p)
          st_bf2_64(st + 4 * XA_PLANE + p * XB_PLANE, n, 2 * k, sbyte(wb[j], p), sbyte(wb[j], 4 + p));
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_bar[s]);
#pragma unroll
      for (int j = 0; j < NA; ++j) wa[j] = na_[j];
#pragma unroll
      for (int j = 0; j < NB; ++j) wb[j] = nb_[j];
      ti = ti2;
      sgi = sgi2;
      k0 = k02;
      have = have2;
    }
  } else if (warp == XMMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int it = 0, j = 0;
      bool ok = true;
      for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
        const int sl = slice_of(L, ti);
        const GemmSeg* segs = L.sl[sl].segs;
        const GemmTask t = L.sl[sl].tasks[L.sl[sl].tiles[ti - L.start[sl]].x];
        if (task_chunks(t, segs) == 0) continue;
        const uint32_t idesc = make_idesc(1u, 128, (uint32_t)(t.tn > 0 ? t.tn : XN));
        const int buf = j & 1;
        if (!mbar_wait(&tempty[buf], ((j >> 1) & 1) ^ 1, verr)) break;
        tc_fence_after();
        const uint32_t acc = tmem + buf * XACC;
        uint32_t started = 0;  // bit o set once accumulator o has been written
        for (int sgi = 0; sgi < t.seg_count && ok; ++sgi) {
          const int kk = segs[t.seg_begin + sgi].k;
          for (int k0 = 0; k0 < kk; k0 += XKC, ++it) {
            const int s = it % XSTAGES;
            if (!mbar_wait(&full_bar[s], (it / XSTAGES) & 1, verr)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t st = smem_u32(stage_base + (size_t)s * XSTAGE);
            // 2 k-steps of 16 bf16 (8 complex k, 32 bytes); the last chunk of a
            // segment issues only the steps that hold data
            const int nks = min(2, (kk - k0 + 7) >> 3);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              if (q >= nks) break;
              const uint32_t koff = q * 32;
              uint64_t a[4], b[4];
#pragma unroll
              for (int p = 0; p < 4; ++p) {
                a[p] = sw64_desc(st + p * XA_PLANE + koff);
                b[p] = sw64_desc(st + 4 * XA_PLANE + p * XB_PLANE + koff);
              }
#pragma unroll
              for (int o = 0; o < 4; ++o) {
#pragma unroll
                for (int i = 0; i <= o; ++i) {
                  mma<1>(acc + o * XN, a[i], b[o - i], idesc, (started >> o) & 1);
                  started |= 1u << o;
                }
              }
            }
            mma_commit(&empty_bar[s]);
          }
        }
        if (ok) mma_commit(&tfull[buf]);
        ++j;
      }
    }
  } else {
    // ---------------- epilogue (warps 9-16: warp w reads TMEM lane quarter w mod 4;
    // the two warps of a quarter take one half of the 64 columns each) ----------------
    const int quarter = warp & 3;
    const int half = (warp - XMMA_WARP - 1) >> 2;
    const int etid = tid - (XPROD + 32);  // 0..255
    int j = 0;
    for (int ti = blockIdx.x; ti < ntiles && !*verr; ti += gridDim.x) {
      const int sl = slice_of(L, ti);
      const ExactSlice& S = L.sl[sl];
      const GemmSeg* segs = S.segs;
      const int* exps = S.exps;
      const int3 tr = S.tiles[ti - L.start[sl]];
      const GemmTask t = S.tasks[tr.x];
      cplx* const cptr = rebase(S.B, t.c_base, t.c);
      const int tn = t.tn > 0 ? t.tn : XN;
      const int m0 = tr.y * TM, n0 = tr.z * tn;
      if (task_chunks(t, segs) == 0) {  // no contribution: the output tile is zero
        for (int e = etid; e < TM * XN; e += XEPI) {
          const int r = m0 + e / XN, c = n0 + e % XN;
          if (r < t.rows && e % XN < tn && c < t.cols)
            cptr[t.rowoff ? t.rowoff[r] + c : (long long)r * t.ldc + c] = {0.0, 0.0};
        }
        continue;
      }
      const int buf = j & 1;
      if (!mbar_wait(&tfull[buf], (j >> 1) & 1, verr)) break;
      tc_fence_after();
      const int row = quarter * 32 + lane;
      const int m = row >> 1, part = row & 1;
      const int gr = m0 + m;
      const int re_m = gr < t.rows ? exps[t.roff + gr] : 0;
      const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + buf * XACC;
      // the two warps of a lane quarter take alternate 16-column groups of the tile
      for (int c0 = half * 16; c0 < tn; c0 += 32) {
        uint32_t a0[16], a1[16], a2[16], a3[16];
        tmem_ld16<16>(lane_addr + 0 * XN + c0, a0);
        tmem_ld16<16>(lane_addr + 1 * XN + c0, a1);
        tmem_ld16<16>(lane_addr + 2 * XN + c0, a2);
        tmem_ld16<16>(lane_addr + 3 * XN + c0, a3);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (gr < t.rows) {
          double* out = reinterpret_cast<double*>(cptr + (t.rowoff ? t.rowoff[gr] : (long long)gr * t.ldc));
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int gc = n0 + c0 + jj;
            if (gc >= t.cols) continue;
            // the accumulators hold exact integers below 2^24: 32-bit conversions
            long long V = __float2int_rn(__uint_as_float(a0[jj]));
            V = (V << 8) + __float2int_rn(__uint_as_float(a1[jj]));
            V = (V << 8) + __float2int_rn(__uint_as_float(a2[jj]));
            V = (V << 8) + __float2int_rn(__uint_as_float(a3[jj]));
            const int ee = re_m + exps[t.coff + gc] - 36;
            out[2 * gc + part] = __longlong_as_double(scaled_double_bits(V, ee));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      ++j;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * XACC) : "memory");
  }
  if (tid == 0 && err)
    for (int q = 0; q < L.nslices; ++q) atomicAdd(L.sl[q].status, 1);
}

template <int KIND>
size_t smem_bytes() {
  return (size_t)STAGES * 2 * Cfg<KIND>::PLANES * PLANE_BYTES + 1024;
}

// Self-test of the bounded-wait path: one thread waits on an mbarrier that nothing
// arrives at, polls it `polls` times, gives up and records the expiry -- the same
// give-up-and-report sequence every pipeline wait of the GEMM kernels follows.
__global__ void wait_selftest_kernel(uint32_t polls, int* __restrict__ status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool done = false;
    for (uint32_t it = 0; it < polls && !done; ++it) done = mbar_try(&bar, 0);
    if (!done) atomicAdd(status, 1);
  }
}

}  // namespace

int split_tile_m() { return TM; }
int split_tile_n(int kind) { return kind == 0 ? TN : XN; }

void launch_gemm_split(int kind, const GemmTask* tasks, const GemmSeg* segs, const int3* tiles, int ntiles,
                       const int* exps, const Bases4& B, int* status, cudaStream_t s) {
  if (ntiles <= 0) return;
  if (kind == 0) {
    const size_t sm = smem_bytes<0>();
    static const bool init = [sm] {  // once per process, thread-safe (function-local static)
      cudaFuncSetAttribute(gemm_split_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      return true;
    }();
    (void)init;
    note_launch();
    gemm_split_kernel<0><<<ntiles, NTHREADS, sm, s>>>(tasks, segs, tiles, B, status);
  } else {
    ExactLaunch L{};
    L.nslices = 1;
    L.start[0] = 0;
    L.start[1] = ntiles;
    L.sl[0] = {tasks, segs, tiles, exps, status, B};
    launch_gemm_exact_merged(L, s);
  }
}

void launch_gemm_exact_merged(const ExactLaunch& L, cudaStream_t s) {
  const int ntiles = L.start[L.nslices];
  if (ntiles <= 0) return;
  const size_t sm = (size_t)XSTAGES * XSTAGE + 1024;
  static const int nsm = [sm] {  // once per process, thread-safe (function-local static)
    cudaFuncSetAttribute(gemm_exact_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(gemm_exact_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n < 1 ? 1 : n;
  }();
  bool img = true;
  for (int i = 0; i < L.nslices; ++i) img = img && L.sl[i].img != 0;
  note_launch();
  if (img) gemm_exact_kernel<true><<<ntiles < nsm ? ntiles : nsm, XTHREADS, sm, s>>>(L);
  else gemm_exact_kernel<false><<<ntiles < nsm ? ntiles : nsm, XTHREADS, sm, s>>>(L);
}

int digit_job_size() { return DIGIT_JOB; }
int digit_slots() { return DIGIT_SLOTS; }

void launch_wait_selftest(unsigned polls, int* status, cudaStream_t s) {
  note_launch();
  wait_selftest_kernel<<<1, 32, 0, s>>>(polls, status);
}

void launch_digits(const DigitOp* ops, int nops, const int2* jobs, int njobs, unsigned* tags, int* exps,
                   unsigned epoch, const Bases4& B, cudaStream_t s, int mode) {
  if (nops <= 0) return;
  const size_t sm = DIGIT_SLOTS * sizeof(unsigned);
  if (mode == 2) {
    note_launch();
    digit_split_own_kernel<<<nops, 256, sm, s>>>(ops, B, exps);
    return;
  }
  if (mode == 0) {
    note_launch();
    digit_max_kernel<<<njobs, 256, sm, s>>>(ops, jobs, B, tags, epoch, digit_job_size());
  }
  note_launch();
  digit_convert_kernel<<<njobs, 256, 0, s>>>(ops, jobs, B, tags, epoch, exps);
}

}  // namespace tdvp
