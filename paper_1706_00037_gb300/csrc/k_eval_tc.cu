// k_eval_tc.cu -- Evaluate(x) of Fig. 2 as a tensor-core contraction.
//
// Problem (P) with Q symmetric gives f(x) = x^t Q x = sum_j x_j sum_{k<=j} Q'_jk x_k
// with Q' = 2 tril(Q,-1) + diag(Q), so a batch needs only the lower block
// triangle of D = X Q'^t (X: S x n starts, 0/1).  D is formed on the 5th-gen
// tensor cores (tcgen05.mma kind::f16, bf16 operands, fp32 accumulation in
// tensor memory) and never written out: an epilogue folds f_s += sum_j x_sj D_sj
// in int64 and adds it to f with one atomic per row and work unit.
//
// Exactness: x is 0/1 and |Q'| <= 256, both exact in bf16; every product is an
// exact integer and one work unit sums at most KCH*BK = 1024 of them, so every
// fp32 partial is an integer below 2^18 < 2^24 and is exact.  Integer atomics
// make the result independent of the order in which units finish.
//
// Kernel structure (one persistent CTA per SM, 6 warps):
//   warp 0  one thread issues TMA loads of A = unpacked X (128 x 64 bf16) and
//           B = Q' rows (256 x 64 bf16) into a 4-stage shared-memory ring;
//   warp 1  allocates 512 TMEM columns (two 128 x 256 fp32 accumulators) and
//           one thread issues the MMAs (M=128, N=256, K=16);
//   warps 2-5  the epilogue: tcgen05.ld of the accumulator rows, int64 dot
//           with the solution bits, atomicAdd into f.
// A work unit is (m-tile of 128 starts, N-block J of 256 columns, a K chunk of
// at most 16 steps of 64 inside [0, 256 (J+1))); units run largest first,
// round-robin over the CTAs, with the two accumulators letting the epilogue of
// one unit overlap the MMAs of the next.  Every wait is bounded: on timeout the
// kernel records UBQP_DEVERR_TIMEOUT, drains its in-flight copies and MMAs,
// frees its tensor memory and returns.
//
// Variants in this file: the fused A operand (four more warps write the 0/1
// rows into the shared-memory stage from the bits), the A operand in tensor
// memory, the Y mode (y = Q x of the passing starts, the ascent's start-up:
// since Q' + Q'^t = 2Q, each N-block sums its lower-triangle K steps from Q'
// and its upper-triangle steps from Q'^t, and the epilogue halves the
// result), and for batches of instances the merged kernels: one
// fused evaluation and one Y-mode product over work lists that mix the units
// of every instance, each unit naming its instance and that instance's tensor
// maps (arrays in global memory).
#include <cuda.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "ubqp_internal.cuh"

namespace ubqp {
namespace {

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int KCH = 16;  // max K steps (of BK) per work unit
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = 512;
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + 256;
// fused variant: two more warps build the A operand from the solution bits,
// with a 256-entry byte -> 8 bf16 table in shared memory
constexpr int A_WRITERS = 128;  // one row of the A tile per thread
constexpr int THREADS_FUSED = THREADS + A_WRITERS;
constexpr int SMEM_BYTES_FUSED = SMEM_BYTES;
constexpr uint64_t kWaitNs = 2000ull * 1000 * 1000;
// Tensor-memory A operand (eval_ts_kernel): the 0/1 rows are written into
// tensor memory by tcgen05.st, so shared memory carries only B.  N = 192 so
// that two accumulators (384 columns) and four A stages (4 x 32 columns of
// 64 bf16 per row) fill the 512 columns.
// The A ring (written locally, no memory latency to hide) and the B ring (TMA
// loads from L2, whose latency the stages hide) advance independently: eight
// B stages fill the shared memory.
constexpr int BN_TS = 192;
constexpr int B_BYTES_TS = BN_TS * BK * 2;
constexpr int STAGES_A_TS = 4;
constexpr int STAGES_B_TS = 4;
constexpr uint32_t ACOL_TS = 2 * BN_TS;  // first A-stage column
constexpr int A_WRITERS_TS = 256;  // two warps per lane quarter, 16 columns each
constexpr int THREADS_TS = THREADS + A_WRITERS_TS;
constexpr int SMEM_BYTES_TS = 1024 + STAGES_B_TS * B_BYTES_TS + 256;

// Instruction descriptor, kind::f16: D fp32 (bits 4-5 = 1), A bf16 (7-9 = 1),
// B bf16 (10-12 = 1), both K-major (15, 16 = 0), N/8 at 17-22, M/16 at 24-28.
constexpr uint32_t IDESC_TS = (1u << 4) | (1u << 7) | (1u << 10) |
                              ((uint32_t)(BN_TS >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false when this CTA is aborting (timeout here or elsewhere).
__device__ __noinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag,
                                       unsigned* err) {
  uint64_t t0 = 0;
  for (uint32_t i = 0;; ++i) {
    if (mbar_try(b, parity)) return true;
    if ((i & 63) == 63) {
      if (*abort_flag) return false;
      const uint64_t t = gtimer();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > kWaitNs) {
        *abort_flag = 1;
        atomicOr(err, UBQP_DEVERR_TIMEOUT);
        return false;
      }
    }
  }
}
// Bounded wait used while draining: ignores the abort flag.
__device__ __noinline__ void mbar_drain(uint64_t* b, uint32_t parity) {
  const uint64_t t0 = gtimer();
  while (!mbar_try(b, parity)) {
    if (gtimer() - t0 > kWaitNs) return;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), LBO unused for this layout (encoded as 16 bytes),
// descriptor version 1 (bit 46), swizzle mode 2 = 128B (bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}

// D (+)= A B with A (128 x 16 bf16) in tensor memory at tmem_a (row i in lane
// i, two elements per 32-bit column) and B from shared memory.
__device__ __forceinline__ void mma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t b,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %4, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(accumulate), "r"(IDESC_TS)
      : "memory");
}

#define UBQP_S8(i) "r"(v[i]), "r"(v[i + 1]), "r"(v[i + 2]), "r"(v[i + 3]), \
                   "r"(v[i + 4]), "r"(v[i + 5]), "r"(v[i + 6]), "r"(v[i + 7])
// 16 consecutive 32-bit columns of this thread's lane; the warp may only
// address its own quarter of the lanes (32 * (warp % 4) ...).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10,"
      " %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      UBQP_S8(0), UBQP_S8(8)
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
#undef UBQP_S8

#define UBQP_R8(i) "=r"(r[i]), "=r"(r[i + 1]), "=r"(r[i + 2]), "=r"(r[i + 3]), \
                   "=r"(r[i + 4]), "=r"(r[i + 5]), "=r"(r[i + 6]), "=r"(r[i + 7])
// 32 consecutive 32-bit columns of this thread's lane, loaded and waited for
// in one statement (so no use of r can be scheduled before the wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10,"
      " %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27,"
      " %28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : UBQP_R8(0), UBQP_R8(8), UBQP_R8(16), UBQP_R8(24)
      : "r"(taddr)
      : "memory");
}
#undef UBQP_R8

#define UBQP_R8(i) "=r"(r[i]), "=r"(r[i + 1]), "=r"(r[i + 2]), "=r"(r[i + 3]), \
                   "=r"(r[i + 4]), "=r"(r[i + 5]), "=r"(r[i + 6]), "=r"(r[i + 7])
// 64 consecutive 32-bit columns of this thread's lane, loaded and waited for
// in one statement (so no use of r can be scheduled before the wait).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10,"
      " %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27,"
      " %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44,"
      " %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61,"
      " %62, %63}, [%64];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : UBQP_R8(0), UBQP_R8(8), UBQP_R8(16), UBQP_R8(24), UBQP_R8(32), UBQP_R8(40),
        UBQP_R8(48), UBQP_R8(56)
      : "r"(taddr)
      : "memory");
}
#undef UBQP_R8

// The evaluation epilogue's share of 64 accumulator columns: the sum of the
// columns whose solution bit is set.  Every column value is an integer of
// magnitude at most 2^18 (a unit sums at most 1024 products of magnitude
// <= 256), so each fp32 partial over 16 columns (<= 2^22) is exact.
__device__ __forceinline__ int row_dot64(uint32_t taddr, uint64_t bits) {
  uint32_t r[64];
  tmem_ld64(taddr, r);
  float p[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < 16; ++i) {
#pragma unroll
    for (int g = 0; g < 4; ++g)
      if ((bits >> (16 * g + i)) & 1ull) p[g] += __uint_as_float(r[16 * g + i]);
  }
  return __float2int_rn(p[0]) + __float2int_rn(p[1]) + __float2int_rn(p[2]) +
         __float2int_rn(p[3]);
}

struct Unit {
  int nb, k0, nk, mt;
};
__device__ __forceinline__ Unit unit_of(const int4* __restrict__ chunks, int m_tiles, int u) {
  const int4 c = chunks[u / m_tiles];
  return Unit{c.x, c.y, c.z, u % m_tiles};
}
// Row `row` of the A tile of unit u: one solution word per K step (zero past
// the unit's K steps, W, S, or when u is past the last unit).  The A writers
// load the next unit's words while they write the current unit's, so the
// load latency is paid once per CTA, not once per unit.
__device__ __forceinline__ void unit_words(const uint64_t* __restrict__ X, int n, int W, int64_t S,
                                           const int4* __restrict__ chunks, int m_tiles,
                                           int n_units, int u, int row, uint64_t (&wa)[KCH]) {
  const uint64_t* x0p = nullptr;
  int k0 = 0, nk = 0;
  if (u < n_units) {
    const Unit un = unit_of(chunks, m_tiles, u);
    const int64_t s0 = (int64_t)un.mt * BM + row;
    if (s0 < S) x0p = X + s0 * W;
    k0 = un.k0;
    nk = un.nk;
  }
#pragma unroll
  for (int i = 0; i < KCH; ++i) {
    const int kw = k0 + i;
    const bool in = i < nk && kw < W;
    wa[i] = (x0p && in) ? (__ldg(x0p + kw) & valid_mask(n, kw)) : 0ull;
  }
}

// Sixteen bits -> sixteen bf16 values 0.0 / 1.0 (bit i = element i), as eight
// words of two: with m = x | (x << 15), bit 2j of x sits at bit 2j of m and
// bit 2j+1 at bit 2j+16, so ((m >> 2j) & 0x10001) * 0x3F80 (bf16 1.0) is word j.
// Three operations per word.
__device__ __forceinline__ void expand16(uint32_t x16, uint32_t (&v)[8]) {
  const uint32_t m = x16 | (x16 << 15);
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = ((m >> (2 * j)) & 0x10001u) * 0x3F80u;
}

// YMODE = false: f_s += sum_j x_sj D_sj over the lower block triangle (Evaluate).
// YMODE = true:  Y = (Xe Q'^t + Xe Q') / 2 = Xe Q (Q symmetric), N-block J
// taking K steps [0, 4(J+1)) of Q' (tmB) and then [4J, n_tc/64) of Q'^t
// (tmU), accumulated in fp32 with vector atomics -- y = Q x for the starts an
// ascent climbs.  Exact: a unit's partial is an integer of magnitude <= 2^18,
// its half a multiple of 1/2, and every sum of halves stays below 2^22.
// FUSED (evaluation only): the A operand is written to shared memory directly
// from the bit-packed solutions by warps 6-9 (no unpacked copy in global
// memory); otherwise both operands arrive by TMA.
template <bool YMODE, bool FUSED>
__global__ void __launch_bounds__(FUSED ? THREADS_FUSED : THREADS, 1)
eval_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmU, const uint64_t* __restrict__ X, int n,
               int W, int64_t S, int m_tiles,
               const int4* __restrict__ chunks, int n_chunks, int64_t* __restrict__ f,
               const int64_t* __restrict__ count, float* __restrict__ Y, int64_t ldy,
               unsigned* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      // the TMA arrival (+ one arrival per A-writer warp)
      mbar_init(&full[s], FUSED ? 1 + A_WRITERS / 32 : 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // Launched as a programmatic dependent of the unpacking (or of whatever
  // kernel precedes it on the stream): everything above overlaps that grid's
  // tail; nothing below reads memory before it has finished.  The kernel
  // after the evaluation (the screen) may then be scheduled; the ascent after
  // the start-up product waits for its completion.
  pdl_wait();
  if (!YMODE) pdl_release();
  int64_t rows = S;
  if (YMODE) {
    const int64_t c = *count;
    rows = c < S ? (c > 0 ? c : 0) : S;
    m_tiles = (int)((rows + BM - 1) / BM);
  }
  const int n_units = n_chunks * m_tiles;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      if (!FUSED)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA))
                     : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      if (YMODE)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmU))
                     : "memory");
      int pending[STAGES];
      for (int s = 0; s < STAGES; ++s) pending[s] = -1;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const Unit un = unit_of(chunks, m_tiles, u);
        for (int ks = 0; ks < un.nk; ++ks) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, err)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + stage * STAGE_BYTES;
          mbar_expect_tx(&full[stage], FUSED ? B_BYTES : STAGE_BYTES);
          int kx = (un.k0 + ks) * BK;
          const CUtensorMap* mb = &tmB;
          if (YMODE) {  // past the block's lower-triangle steps: Q'^t from the block's diagonal
            const int c = un.k0 + ks, ql = (un.nb + 1) * (BN / BK);
            if (c >= ql) {
              mb = &tmU;
              kx = (un.nb * (BN / BK) + c - ql) * BK;
            }
          }
          if (!FUSED) tma_load_2d(sa, &tmA, kx, un.mt * BM, &full[stage]);
          tma_load_2d(sa + A_BYTES, mb, kx, un.nb * BN, &full[stage]);
          pending[stage] = (int)phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {  // let every issued copy land before the CTA exits
        for (int s = 0; s < STAGES; ++s)
          if (pending[s] >= 0) mbar_drain(&full[s], (uint32_t)pending[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int t = 0;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++t) {
        const Unit un = unit_of(chunks, m_tiles, u);
        const int a = t & 1;
        const uint32_t aphase = (uint32_t)((t >> 1) & 1);
        if (!mbar_wait(&tempty[a], aphase ^ 1u, abort_flag, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(a * BN);
        for (int ks = 0; ks < un.nk; ++ks) {
          if (!mbar_wait(&full[stage], phase, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = su32(smem + stage * STAGE_BYTES);
          const uint64_t adesc = sdesc(sa), bdesc = sdesc(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            mma_bf16(d, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk),
                     (ks | kk) != 0 ? 1u : 0u);
          mma_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) mma_commit(&tfull[a]);
      }
      if (!ok) {  // wait for the MMAs already issued before TMEM is freed
        mma_commit(drain);
        mbar_drain(drain, 0);
      }
    }
  } else if (FUSED && warp >= THREADS / 32) {
    // ---------------- A writers (warps 6-9): row t of the A tile, one 64-bit
    // word of solution bits per K step, expanded arithmetically into the
    // 128-byte-swizzled K-major layout the MMA descriptor reads
    const int t = threadIdx.x - THREADS;
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    uint64_t wa[KCH], wn[KCH];
    unit_words(X, n, W, S, chunks, m_tiles, n_units, blockIdx.x, t, wa);
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const Unit un = unit_of(chunks, m_tiles, u);
      unit_words(X, n, W, S, chunks, m_tiles, n_units, u + gridDim.x, t, wn);
#pragma unroll
      for (int ks = 0; ks < KCH; ++ks) {
        if (ks >= un.nk) break;
        const uint64_t w0 = wa[ks];
        // the warp arrives as one below: leave together
        const bool got = mbar_wait(&empty[stage], phase ^ 1u, abort_flag, err);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        uint8_t* r0 = smem + stage * STAGE_BYTES + t * 128;
#pragma unroll
        for (int p = 0; p < 4; ++p) {  // 16-byte chunks 2p, 2p + 1
          uint32_t v[8];
          expand16((uint32_t)(w0 >> (16 * p)) & 0xFFFFu, v);
          *reinterpret_cast<uint4*>(r0 + (((2 * p) ^ (t & 7)) << 4)) =
              make_uint4(v[0], v[1], v[2], v[3]);
          *reinterpret_cast<uint4*>(r0 + (((2 * p + 1) ^ (t & 7)) << 4)) =
              make_uint4(v[4], v[5], v[6], v[7]);
        }
        // make the generic-proxy writes visible to the tensor cores' reads,
        // then one arrival for the warp's 32 rows
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[stage]);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
#pragma unroll
      for (int i = 0; i < KCH; ++i) wa[i] = wn[i];
    }
  } else {
    // ---------------- epilogue: warps 2..5 cover TMEM lanes 64-95, 96-127, 0-31, 32-63
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int t = 0;
    // the solution words of a unit's 256 columns in this row, loaded one unit
    // ahead (their latency off the accumulator hand-off)
    auto unit_xw = [&](int u, uint64_t (&w4)[4]) {
      const uint64_t* xp = nullptr;
      int w0 = 0;
      if (!YMODE && u < n_units) {
        const Unit v = unit_of(chunks, m_tiles, u);
        const int64_t sv = (int64_t)v.mt * BM + row;
        if (sv < S) xp = X + sv * W;
        w0 = v.nb * 4;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) w4[i] = (xp && w0 + i < W) ? xp[w0 + i] : 0ull;
    };
    uint64_t xw[4];
    unit_xw(blockIdx.x, xw);
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++t) {
      const Unit un = unit_of(chunks, m_tiles, u);
      const int a = t & 1;
      const uint32_t aphase = (uint32_t)((t >> 1) & 1);
      uint64_t xn[4];
      unit_xw(u + gridDim.x, xn);
      // the warp arrives as one on tempty below: leave together
      const bool got = mbar_wait(&tfull[a], aphase, abort_flag, err);
      if (!__all_sync(0xffffffffu, got)) break;
      tc_fence_after();
      const int64_t s = (int64_t)un.mt * BM + row;
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN);
      if (YMODE) {
        float* yrow = Y + s * ldy + (int64_t)un.nb * BN;
#pragma unroll 1
        for (int cc = 0; cc < BN / 32; ++cc) {
          uint32_t r[32];
          tmem_ld32(base + (uint32_t)(cc * 32), r);
          if (s < rows) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
              atomicAdd(reinterpret_cast<float4*>(yrow + cc * 32 + 4 * i),
                        make_float4(0.5f * __uint_as_float(r[4 * i]),
                                    0.5f * __uint_as_float(r[4 * i + 1]),
                                    0.5f * __uint_as_float(r[4 * i + 2]),
                                    0.5f * __uint_as_float(r[4 * i + 3])));
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[a]);
      } else {
        int acc = 0;
#pragma unroll 1
        for (int cc = 0; cc < BN / 64; ++cc) acc += row_dot64(base + (uint32_t)(cc * 64), xw[cc]);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[a]);
        if (s < S && acc != 0)
          atomicAdd(reinterpret_cast<unsigned long long*>(&f[s]),
                    (unsigned long long)(long long)acc);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) xw[i] = xn[i];
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// Row `row` of the A tile of merged unit u (as unit_words, for the instance
// the unit belongs to).
__device__ __forceinline__ void munit_words(const EvalInst* __restrict__ insts,
                                            const MUnit* __restrict__ units, int n_units, int u,
                                            int row, uint64_t (&wa)[KCH]) {
  const uint64_t* x0p = nullptr;
  int k0 = 0, nk = 0, n = 0, W = 0;
  if (u < n_units) {
    const MUnit un = units[u];
    const EvalInst e = insts[un.inst];
    const int64_t s0 = (int64_t)un.mt * BM + row;
    if (s0 < e.S) x0p = e.X + s0 * e.W;
    k0 = un.k0;
    nk = un.nk;
    n = e.n;
    W = e.W;
  }
#pragma unroll
  for (int i = 0; i < KCH; ++i) {
    const int kw = k0 + i;
    const bool in = i < nk && kw < W;
    wa[i] = (x0p && in) ? (__ldg(x0p + kw) & valid_mask(n, kw)) : 0ull;
  }
}

// The evaluation of every instance of a batch in one persistent launch: the
// fused kernel above (A operand written from the solution bits, B = Q' by TMA,
// int64 row-dot epilogue) over a merged list of work units (instance, chunk,
// m-tile) of all instances, largest chunks first.  Each unit names its
// instance, whose starts, values and Q' tensor map (an array in global
// memory) it uses.  A timeout is recorded in `err`.
__global__ void __launch_bounds__(THREADS_FUSED, 1)
eval_tc_multi_kernel(const EvalInst* __restrict__ insts, const CUtensorMap* __restrict__ maps,
                     const MUnit* __restrict__ units, int n_units, unsigned* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1 + A_WRITERS / 32);  // the TMA arrival + one per A-writer warp
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (B only)
      int pending[STAGES];
      for (int s = 0; s < STAGES; ++s) pending[s] = -1;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const MUnit un = units[u];
        const CUtensorMap* map = maps + un.inst;
        for (int ks = 0; ks < un.nk; ++ks) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, err)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + stage * STAGE_BYTES;
          mbar_expect_tx(&full[stage], B_BYTES);
          tma_load_2d(sa + A_BYTES, map, (un.k0 + ks) * BK, un.nb * BN, &full[stage]);
          pending[stage] = (int)phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {  // let every issued copy land before the CTA exits
        for (int s = 0; s < STAGES; ++s)
          if (pending[s] >= 0) mbar_drain(&full[s], (uint32_t)pending[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int t = 0;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++t) {
        const int nk = units[u].nk;
        const int a = t & 1;
        const uint32_t aphase = (uint32_t)((t >> 1) & 1);
        if (!mbar_wait(&tempty[a], aphase ^ 1u, abort_flag, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(a * BN);
        for (int ks = 0; ks < nk; ++ks) {
          if (!mbar_wait(&full[stage], phase, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = su32(smem + stage * STAGE_BYTES);
          const uint64_t adesc = sdesc(sa), bdesc = sdesc(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            mma_bf16(d, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk),
                     (ks | kk) != 0 ? 1u : 0u);
          mma_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) mma_commit(&tfull[a]);
      }
      if (!ok) {  // wait for the MMAs already issued before TMEM is freed
        mma_commit(drain);
        mbar_drain(drain, 0);
      }
    }
  } else if (warp >= THREADS / 32) {
    // ---------------- A writers (warps 6-9): row t of the A tile
    const int t = threadIdx.x - THREADS;
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    uint64_t wa[KCH], wn[KCH];
    munit_words(insts, units, n_units, blockIdx.x, t, wa);
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const int nk = units[u].nk;
      munit_words(insts, units, n_units, u + gridDim.x, t, wn);
#pragma unroll
      for (int ks = 0; ks < KCH; ++ks) {
        if (ks >= nk) break;
        const uint64_t w0 = wa[ks];
        // the warp arrives as one below: leave together
        const bool got = mbar_wait(&empty[stage], phase ^ 1u, abort_flag, err);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        uint8_t* r0 = smem + stage * STAGE_BYTES + t * 128;
#pragma unroll
        for (int p = 0; p < 4; ++p) {  // 16-byte chunks 2p, 2p + 1
          uint32_t v[8];
          expand16((uint32_t)(w0 >> (16 * p)) & 0xFFFFu, v);
          *reinterpret_cast<uint4*>(r0 + (((2 * p) ^ (t & 7)) << 4)) =
              make_uint4(v[0], v[1], v[2], v[3]);
          *reinterpret_cast<uint4*>(r0 + (((2 * p + 1) ^ (t & 7)) << 4)) =
              make_uint4(v[4], v[5], v[6], v[7]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[stage]);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
#pragma unroll
      for (int i = 0; i < KCH; ++i) wa[i] = wn[i];
    }
  } else {
    // ---------------- epilogue: warps 2..5 cover TMEM lanes 64-95, 96-127, 0-31, 32-63
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int t = 0;
    // the unit's solution words in this row, loaded one unit ahead
    auto unit_xw = [&](int u, uint64_t (&w4)[4]) {
      const uint64_t* xp = nullptr;
      int w0 = 0, Wv = 0;
      if (u < n_units) {
        const MUnit v = units[u];
        const EvalInst& ev = insts[v.inst];
        const int64_t sv = (int64_t)v.mt * BM + row;
        if (sv < ev.S) xp = ev.X + sv * ev.W;
        w0 = v.nb * 4;
        Wv = ev.W;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) w4[i] = (xp && w0 + i < Wv) ? xp[w0 + i] : 0ull;
    };
    uint64_t xw[4];
    unit_xw(blockIdx.x, xw);
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++t) {
      const MUnit un = units[u];
      const EvalInst e = insts[un.inst];
      const int a = t & 1;
      const uint32_t aphase = (uint32_t)((t >> 1) & 1);
      uint64_t xn[4];
      unit_xw(u + gridDim.x, xn);
      const bool got = mbar_wait(&tfull[a], aphase, abort_flag, err);
      if (!__all_sync(0xffffffffu, got)) break;
      tc_fence_after();
      const int64_t s = (int64_t)un.mt * BM + row;
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN);
      int acc = 0;
#pragma unroll 1
      for (int cc = 0; cc < BN / 64; ++cc) acc += row_dot64(base + (uint32_t)(cc * 64), xw[cc]);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[a]);
      if (s < e.S && acc != 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(&e.f[s]),
                  (unsigned long long)(long long)acc);
#pragma unroll
      for (int i = 0; i < 4; ++i) xw[i] = xn[i];
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// The start-up products y = Q x of the passing starts of every instance of a
// batch in one persistent launch: the staged kernel's Y mode (A = the unpacked
// passing starts by TMA, B = Q by TMA, fp32 vector atomics into Y) over a
// merged list of units (instance, full-square chunk, m-tile).  Whether a unit
// has work depends on the instance's passing count, read on the device: every
// role skips the units whose m-tile starts at or past it, in the same order,
// so the stage and accumulator hand-offs stay paired.
__global__ void __launch_bounds__(THREADS, 1)
eval_tc_multi_y_kernel(const YInst* __restrict__ yi, const CUtensorMap* __restrict__ mapsA,
                       const CUtensorMap* __restrict__ mapsB, const CUtensorMap* __restrict__ mapsU,
                       const MUnit* __restrict__ units, int n_units, unsigned* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // does unit u have work: its m-tile starts below the instance's count
  auto active = [&](const MUnit& un) {
    const YInst& e = yi[un.inst];
    const int64_t c = *e.count;
    const int64_t rows = c < e.S ? (c > 0 ? c : 0) : e.S;
    return (int64_t)un.mt * BM < rows;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int pending[STAGES];
      for (int s = 0; s < STAGES; ++s) pending[s] = -1;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const MUnit un = units[u];
        if (!active(un)) continue;
        const CUtensorMap* mA = mapsA + un.inst;
        for (int ks = 0; ks < un.nk; ++ks) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, err)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + stage * STAGE_BYTES;
          mbar_expect_tx(&full[stage], STAGE_BYTES);
          // as the single-instance Y mode: Q' below the block's diagonal, Q'^t from it
          const int c = un.k0 + ks, ql = (un.nb + 1) * (BN / BK);
          const CUtensorMap* mb = c < ql ? mapsB + un.inst : mapsU + un.inst;
          const int kx = (c < ql ? c : un.nb * (BN / BK) + c - ql) * BK;
          tma_load_2d(sa, mA, kx, un.mt * BM, &full[stage]);
          tma_load_2d(sa + A_BYTES, mb, kx, un.nb * BN, &full[stage]);
          pending[stage] = (int)phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {  // let every issued copy land before the CTA exits
        for (int s = 0; s < STAGES; ++s)
          if (pending[s] >= 0) mbar_drain(&full[s], (uint32_t)pending[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int t = 0;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const MUnit un = units[u];
        if (!active(un)) continue;
        const int a = t & 1;
        const uint32_t aphase = (uint32_t)((t >> 1) & 1);
        ++t;
        if (!mbar_wait(&tempty[a], aphase ^ 1u, abort_flag, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(a * BN);
        for (int ks = 0; ks < un.nk; ++ks) {
          if (!mbar_wait(&full[stage], phase, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = su32(smem + stage * STAGE_BYTES);
          const uint64_t adesc = sdesc(sa), bdesc = sdesc(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            mma_bf16(d, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk),
                     (ks | kk) != 0 ? 1u : 0u);
          mma_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) mma_commit(&tfull[a]);
      }
      if (!ok) {  // wait for the MMAs already issued before TMEM is freed
        mma_commit(drain);
        mbar_drain(drain, 0);
      }
    }
  } else {
    // ---------------- epilogue: warps 2..5 cover TMEM lanes 64-95, 96-127, 0-31, 32-63
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int t = 0;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
      const MUnit un = units[u];
      if (!active(un)) continue;
      const YInst& e = yi[un.inst];
      const int64_t c = *e.count;
      const int64_t rows = c < e.S ? (c > 0 ? c : 0) : e.S;
      const int a = t & 1;
      const uint32_t aphase = (uint32_t)((t >> 1) & 1);
      ++t;
      const bool got = mbar_wait(&tfull[a], aphase, abort_flag, err);
      if (!__all_sync(0xffffffffu, got)) break;
      tc_fence_after();
      const int64_t s = (int64_t)un.mt * BM + row;
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN);
      float* yrow = e.Y + s * (int64_t)e.n_tc + (int64_t)un.nb * BN;
#pragma unroll 1
      for (int cc = 0; cc < BN / 32; ++cc) {
        uint32_t r[32];
        tmem_ld32(base + (uint32_t)(cc * 32), r);
        if (s < rows) {
#pragma unroll
          for (int i = 0; i < 8; ++i)
            atomicAdd(reinterpret_cast<float4*>(yrow + cc * 32 + 4 * i),
                      make_float4(0.5f * __uint_as_float(r[4 * i]),
                                  0.5f * __uint_as_float(r[4 * i + 1]),
                                  0.5f * __uint_as_float(r[4 * i + 2]),
                                  0.5f * __uint_as_float(r[4 * i + 3])));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[a]);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// Evaluate with the A operand in tensor memory (UBQP_EVAL_TC_TMEM).  Same
// work units and epilogue as eval_tc_kernel with N-blocks of 192 columns;
// warp 0 loads only B (Q' rows) by TMA, warps 6-13 expand each start's 64
// solution bits per K step into 32 columns of bf16 pairs (two warps per lane
// quarter, 16 columns each) and store them into the stage's tensor-memory
// columns (tcgen05.st), warp 1 issues the MMAs with A from tensor memory.
// Shared memory carries 48 KB per K step (B written by TMA and read by the
// MMA) instead of 96 KB.  Measured slower than the staged kernel at every
// Table 1 size (n = 7000: 91 vs 60 us per 1000 starts; tensor pipe 31% active)
// whatever the B-ring depth (4 or 8), the writer count (4 or 8 warps) or the
// word prefetch; kept as a selectable, bit-exact path.
__global__ void __launch_bounds__(THREADS_TS, 1)
eval_ts_kernel(const __grid_constant__ CUtensorMap tmB, const uint64_t* __restrict__ X, int n,
               int W, int64_t S, int m_tiles, const int4* __restrict__ chunks, int n_chunks,
               int64_t* __restrict__ f, unsigned* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  uint64_t* fullB = reinterpret_cast<uint64_t*>(smem + STAGES_B_TS * B_BYTES_TS);
  uint64_t* emptyB = fullB + STAGES_B_TS;
  uint64_t* fullA = emptyB + STAGES_B_TS;
  uint64_t* emptyA = fullA + STAGES_A_TS;
  uint64_t* tfull = emptyA + STAGES_A_TS;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_units = n_chunks * m_tiles;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES_B_TS; ++s) {
      mbar_init(&fullB[s], 1);  // the TMA arrival
      mbar_init(&emptyB[s], 1);
    }
    for (int s = 0; s < STAGES_A_TS; ++s) {
      mbar_init(&fullA[s], A_WRITERS_TS / 32);  // one arrival per writer warp
      mbar_init(&emptyA[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: B only
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      int pending[STAGES_B_TS];
      for (int s = 0; s < STAGES_B_TS; ++s) pending[s] = -1;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const Unit un = unit_of(chunks, m_tiles, u);
        for (int ks = 0; ks < un.nk; ++ks) {
          if (!mbar_wait(&emptyB[stage], phase ^ 1u, abort_flag, err)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&fullB[stage], B_BYTES_TS);
          tma_load_2d(smem + stage * B_BYTES_TS, &tmB, (un.k0 + ks) * BK, un.nb * BN_TS,
                      &fullB[stage]);
          pending[stage] = (int)phase;
          if (++stage == STAGES_B_TS) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {  // let every issued copy land before the CTA exits
        for (int s = 0; s < STAGES_B_TS; ++s)
          if (pending[s] >= 0) mbar_drain(&fullB[s], (uint32_t)pending[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int stage = 0, sa = 0;
      uint32_t phase = 0, pa = 0;
      bool ok = true;
      int t = 0;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++t) {
        const Unit un = unit_of(chunks, m_tiles, u);
        const int a = t & 1;
        const uint32_t aphase = (uint32_t)((t >> 1) & 1);
        if (!mbar_wait(&tempty[a], aphase ^ 1u, abort_flag, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(a * BN_TS);
        for (int ks = 0; ks < un.nk; ++ks) {
          if (!mbar_wait(&fullB[stage], phase, abort_flag, err) ||
              !mbar_wait(&fullA[sa], pa, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t bdesc = sdesc(su32(smem + stage * B_BYTES_TS));
          const uint32_t ta = tmem + ACOL_TS + (uint32_t)(sa * (BK / 2));
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            mma_bf16_ts(d, ta + (uint32_t)(8 * kk), bdesc + (uint64_t)(2 * kk),
                        (ks | kk) != 0 ? 1u : 0u);
          mma_commit(&emptyB[stage]);
          mma_commit(&emptyA[sa]);
          if (++stage == STAGES_B_TS) {
            stage = 0;
            phase ^= 1u;
          }
          if (++sa == STAGES_A_TS) {
            sa = 0;
            pa ^= 1u;
          }
        }
        if (ok) mma_commit(&tfull[a]);
      }
      if (!ok) {  // wait for the MMAs already issued before TMEM is freed
        mma_commit(drain);
        mbar_drain(drain, 0);
      }
    }
  } else if (warp >= THREADS / 32) {
    // ---------------- A writers (warps 6-13): this warp's quarter of the 128
    // rows (lanes) and half of the 64 solution bits per K step -> 16 columns
    // of bf16 pairs
    const int wq = warp & 3;
    const int half = (warp - THREADS / 32) >> 2;
    const int row = wq * 32 + lane;
    const uint32_t tA = tmem + ((uint32_t)(wq * 32) << 16) + ACOL_TS + (uint32_t)(16 * half);
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    uint64_t wa[KCH], wn[KCH];
    unit_words(X, n, W, S, chunks, m_tiles, n_units, blockIdx.x, row, wa);
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const Unit un = unit_of(chunks, m_tiles, u);
      unit_words(X, n, W, S, chunks, m_tiles, n_units, u + gridDim.x, row, wn);
#pragma unroll
      for (int ks = 0; ks < KCH; ++ks) {
        if (ks >= un.nk) break;
        // the tcgen05.st below is warp-collective: leave together
        const bool got = mbar_wait(&emptyA[stage], phase ^ 1u, abort_flag, err);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t v[16];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          uint32_t v8[8];
          expand16((uint32_t)(wa[ks] >> (32 * half + 16 * p)) & 0xFFFFu, v8);
#pragma unroll
          for (int j = 0; j < 8; ++j) v[8 * p + j] = v8[j];
        }
        tmem_st16(tA + (uint32_t)(stage * (BK / 2)), v);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&fullA[stage]);
        if (++stage == STAGES_A_TS) {
          stage = 0;
          phase ^= 1u;
        }
      }
#pragma unroll
      for (int i = 0; i < KCH; ++i) wa[i] = wn[i];
    }
  } else {
    // ---------------- epilogue: warps 2..5 cover TMEM lanes 64-95, 96-127, 0-31, 32-63
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int t = 0;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++t) {
      const Unit un = unit_of(chunks, m_tiles, u);
      const int a = t & 1;
      const uint32_t aphase = (uint32_t)((t >> 1) & 1);
      const bool got = mbar_wait(&tfull[a], aphase, abort_flag, err);
      if (!__all_sync(0xffffffffu, got)) break;  // tcgen05.ld is warp-collective
      tc_fence_after();
      const int64_t s = (int64_t)un.mt * BM + row;
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN_TS);
      uint64_t xw[BN_TS / 64];
#pragma unroll
      for (int i = 0; i < BN_TS / 64; ++i) {
        const int w = un.nb * (BN_TS / 64) + i;
        xw[i] = (s < S && w < W) ? X[s * W + w] : 0ull;
      }
      int acc = 0;
#pragma unroll 1
      for (int cc = 0; cc < BN_TS / 64; ++cc)
        acc += row_dot64(base + (uint32_t)(cc * 64), xw[cc]);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[a]);
      if (s < S && acc != 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(&f[s]), (unsigned long long)(long long)acc);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// Self-test of the bounded wait: an mbarrier that expects one arrival and gets
// none; the same try-wait / global-timer loop as mbar_wait, with a caller limit.
__global__ void selftest_wait_kernel(uint64_t limit_ns, int32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint64_t t0 = gtimer();
    int32_t st = 0;
    for (uint32_t i = 0;; ++i) {
      if (mbar_try(&bar, 0)) break;  // never: nothing arrives
      if ((i & 63) == 63 && gtimer() - t0 > limit_ns) {
        st = UBQP_ERR_TIMEOUT;
        break;
      }
    }
    *status = st;
  }
}

// Rows of 0.0/1.0 bf16 (the A operand of the staged kernel) from the bit-packed
// starts: S_p x n_tc, row t is start t (t < S), or with idx start idx[t] for
// t < *count and zero up to the next multiple of 128 (the last m-tile the
// product reads; rows beyond are not written); columns >= n are zero.  With Y
// the product's rows t < *count are zeroed for its accumulation.  Blocks (of
// kUnpackThreads) take rows: the row's words are read once into shared
// memory, then each thread expands 8-column pieces of it (no 64-bit division).
constexpr int kUnpackThreads = 256;
static_assert(kUnpackThreads * 64 >= UBQP_MAX_N, "one word per thread covers a row");
__device__ __forceinline__ void unpack_rows(const uint64_t* __restrict__ X, int n, int W,
                                            int64_t S, const int32_t* __restrict__ idx,
                                            const int64_t* __restrict__ count, int64_t S_p,
                                            int n_tc, uint4* __restrict__ Xe,
                                            float* __restrict__ Y, int64_t block,
                                            int64_t blocks) {
  __shared__ uint64_t words[kUnpackThreads];
  const int per_row = n_tc / 16;
  int64_t rows = S, rows_p = S_p;
  if (idx) {
    const int64_t c = *count;
    rows = c < S ? (c > 0 ? c : 0) : S;
    rows_p = (rows + BM - 1) / BM * BM;
  }
  for (int64_t r = block; r < rows_p; r += blocks) {
    const uint64_t* xr = nullptr;
    if (r < rows) {
      const int64_t src = idx ? (int64_t)idx[r] : r;
      if (src >= 0 && src < S) xr = X + src * W;
    }
    const int w = threadIdx.x;
    words[w] = (xr && w < W) ? (xr[w] & valid_mask(n, w)) : 0ull;
    __syncthreads();
    // consecutive threads write consecutive 16-byte pieces (8 columns each)
    uint4* er = Xe + 2 * r * per_row;
    for (int h = threadIdx.x; h < 2 * per_row; h += blockDim.x) {
      const uint32_t x8 = (uint32_t)(words[h >> 3] >> ((h & 7) * 8)) & 0xFFu;
      uint32_t v[8];
      expand16(x8, v);
      er[h] = make_uint4(v[0], v[1], v[2], v[3]);
      if (Y && r < rows) {
        float4* yr = reinterpret_cast<float4*>(Y + r * (int64_t)n_tc + 8 * h);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        yr[0] = z;
        yr[1] = z;
      }
    }
    __syncthreads();  // words[] is rewritten for the next row
  }
}

// The evaluation's and the start-up's unpacking, a programmatic dependent of
// the kernel before it (pdl_enter).  It lets the product that follows on the
// stream start its set-up at once; that kernel waits for this grid to finish
// before it reads what this one writes.  With fz, fz[0 .. nfz) is zeroed: the
// evaluation's values f for its accumulation, or the ascent's start counter,
// in place of a separate memset.
__global__ void unpack_bits_bf16(const uint64_t* __restrict__ X, int n, int W, int64_t S,
                                 const int32_t* __restrict__ idx,
                                 const int64_t* __restrict__ count, int64_t S_p, int n_tc,
                                 uint4* __restrict__ Xe, float* __restrict__ Y,
                                 int64_t* __restrict__ fz, int64_t nfz) {
  pdl_enter();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; fz && t < nfz;
       t += (int64_t)gridDim.x * blockDim.x)
    fz[t] = 0;
  unpack_rows(X, n, W, S, idx, count, S_p, n_tc, Xe, Y, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

// Every instance of a batch (instance blockIdx.y): the passing starts of the
// start-up product unpacked, and their Y rows zeroed.
__global__ void unpack_batch_bf16(const YInst* __restrict__ yi) {
  const YInst& e = yi[blockIdx.y];
  unpack_rows(e.X, e.n, e.W, e.S, e.idx, e.count, e.S_p, e.n_tc, e.Xe, e.Y, (int64_t)blockIdx.x,
              (int64_t)gridDim.x);
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Opt each tensor-core kernel into its dynamic shared memory once per process
// (the attribute is per function; the first call from any thread sets it).
template <bool YMODE, bool FUSED>
cudaError_t set_smem_attr_once() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    err = cudaFuncSetAttribute(eval_tc_kernel<YMODE, FUSED>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               FUSED ? SMEM_BYTES_FUSED : SMEM_BYTES);
  });
  return err;
}

cudaError_t set_smem_attr_ts_once() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    err = cudaFuncSetAttribute(eval_ts_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               SMEM_BYTES_TS);
  });
  return err;
}

// 2-D bf16 row-major tensor [rows][cols], box = box_rows x 64 columns, 128B swizzle.
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int box_rows) {
  EncodeFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int64_t padded_starts(int64_t S) { return (S + BM - 1) / BM * BM; }

// Scratch of the allocation-free evaluation (ubqp_eval_noalloc): the unpacked
// solutions live in this file-scope device array instead of caller workspace.
// CUDA places it on a device when it loads this file's module there (lazily by
// default: the first launch of a kernel of this file or the first address
// lookup below) and keeps it until the process exits.
static __device__ __align__(256) uint8_t g_eval_scratch[UBQP_EVAL_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
// device address of g_eval_scratch per device, with the id of the CUDA context
// it was looked up in (a cudaDeviceReset ends that context and the address
// with it)
void* g_scratch_addr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id (for the life of the process) of the context current on this
// thread; false when there is none or the driver cannot say.
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
    cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

}  // namespace

size_t eval_tc_static_capacity() { return (size_t)UBQP_EVAL_NOALLOC_MAX_BYTES; }

// Device address of the static scratch on the current device.  The host-side
// name g_eval_scratch is only a stand-in; the real address comes from
// cudaGetSymbolAddress with the device current, looked up on the first call in
// each context of the device and kept for the later calls in that context.
// (The lookup loads this file's module if CUDA has not yet, which places the
// array on the device.)  Without a context id from the driver every call
// looks the address up.
cudaError_t eval_tc_static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  unsigned long long id = 0;
  bool have_id = current_context_id(&id);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev] || !have_id || id != g_scratch_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_eval_scratch);
    if (e) return e;
    // the lookup has made the device's context current: key the address by it
    have_id = current_context_id(&id);
    g_scratch_addr[dev] = have_id ? p : nullptr;
    g_scratch_ctx[dev] = have_id ? id : 0;
    *out = p;
    return cudaSuccess;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t eval_tc_workspace(const ubqp_q* h, int64_t S) {
  return (size_t)padded_starts(S) * (size_t)h->n_tc * 2;
}

// Work chunks {N-block, first K step, K steps, 0}, sorted largest first.
// Evaluation: for N-block J the K range is [0, 256 (J+1)) (lower block
// triangle); ascent start-up (y = Q x): the full K range for every J.  Both are
// split into near-equal chunks of at most KCH steps.
// N-blocks of bn columns over n_tc; the K range of block J is capped at n_tc.
static std::vector<int4> make_chunks(int n_tc, int bn, bool full, int kch = KCH) {
  std::vector<int4> ch;
  const int NB = (n_tc + bn - 1) / bn;
  const int nk_full = n_tc / BK;
  for (int J = 0; J < NB; ++J) {
    const int nk = full ? nk_full : std::min((J + 1) * (bn / BK), nk_full);
    const int parts = (nk + kch - 1) / kch;
    for (int p = 0, k0 = 0; p < parts; ++p) {
      const int len = nk / parts + (p < nk % parts ? 1 : 0);
      ch.push_back(make_int4(J, k0, len, 0));
      k0 += len;
    }
  }
  std::stable_sort(ch.begin(), ch.end(), [](const int4& a, const int4& b) { return a.z > b.z; });
  return ch;
}

// The start-up's chunks: y = (Q' x + Q'^t x) / 2, so N-block J runs its K steps
// [0, 4(J+1)) of Q' and then [4J, n_tc/64) of Q'^t: one combined sequence of
// n_tc/64 + 4 steps per block (the diagonal block's halves from both), split
// into near-equal chunks of at most kch steps, largest first.  Combined step c
// of block J is Q' step c below 4(J+1), else Q'^t step 4J + c - 4(J+1).
static std::vector<int4> make_chunks_y(int n_tc, int kch = KCH) {
  std::vector<int4> ch;
  const int NB = n_tc / BN, nk = n_tc / BK + BN / BK;
  for (int J = 0; J < NB; ++J) {
    const int parts = (nk + kch - 1) / kch;
    for (int p = 0, k0 = 0; p < parts; ++p) {
      const int len = nk / parts + (p < nk % parts ? 1 : 0);
      ch.push_back(make_int4(J, k0, len, 0));
      k0 += len;
    }
  }
  std::stable_sort(ch.begin(), ch.end(), [](const int4& a, const int4& b) { return a.z > b.z; });
  return ch;
}

// The evaluation's work chunks with at most kch (1..16) K steps of 64 each
// (the handle's own table uses 16): a schedule a batch plan may tune.
std::vector<int4> eval_tc_chunks(int n_tc, int kch) {
  return make_chunks(n_tc, BN, false, std::max(1, std::min(kch, KCH)));
}

std::vector<MUnit> eval_tc_multi_units(const ubqp_q* const* qs, int count, int64_t S, int kch) {
  std::vector<MUnit> us;
  const int m_tiles = (int)(padded_starts(S) / BM);
  for (int i = 0; i < count; ++i) {
    for (const int4& c : make_chunks(qs[i]->n_tc, BN, false, std::max(1, std::min(kch, KCH))))
      for (int mt = 0; mt < m_tiles; ++mt) us.push_back(MUnit{c.x, c.y, c.z, mt, i, 0, 0, 0});
  }
  std::stable_sort(us.begin(), us.end(),
                   [](const MUnit& a, const MUnit& b) { return a.nk > b.nk; });
  return us;
}

cudaError_t launch_eval_tc_multi(const EvalInst* insts, const void* maps, const MUnit* units,
                                 int n_units, unsigned* err, int sm_count, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(eval_tc_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_BYTES_FUSED);
  });
  if (attr != cudaSuccess) return attr;
  if (n_units < 1) return cudaSuccess;
  const int grid = n_units < sm_count ? n_units : sm_count;
  eval_tc_multi_kernel<<<grid, THREADS_FUSED, SMEM_BYTES_FUSED, st>>>(
      insts, reinterpret_cast<const CUtensorMap*>(maps), units, n_units, err);
  return cudaGetLastError();
}

std::vector<MUnit> eval_tc_multi_y_units(const ubqp_q* const* qs, int count, int64_t S) {
  std::vector<MUnit> us;
  const int m_tiles = (int)(padded_starts(S) / BM);
  for (int i = 0; i < count; ++i) {
    for (const int4& c : make_chunks_y(qs[i]->n_tc))
      for (int mt = 0; mt < m_tiles; ++mt) us.push_back(MUnit{c.x, c.y, c.z, mt, i, 0, 0, 0});
  }
  std::stable_sort(us.begin(), us.end(),
                   [](const MUnit& a, const MUnit& b) { return a.nk > b.nk; });
  return us;
}

cudaError_t launch_startup_multi(const YInst* yi, int count, int64_t max_items, const void* mapsA,
                                 const void* mapsB, const void* mapsU, const MUnit* units,
                                 int n_units, unsigned* err, int sm_count, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(eval_tc_multi_y_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  });
  if (attr != cudaSuccess) return attr;
  if (count < 1 || n_units < 1) return cudaSuccess;
  // blocks take rows of every instance (blockIdx.y)
  int64_t blocks = (max_items + 255) / 256;
  if (blocks > 256) blocks = 256;
  if (blocks < 1) blocks = 1;
  unpack_batch_bf16<<<dim3((unsigned)blocks, (unsigned)count), kUnpackThreads, 0, st>>>(yi);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int grid = n_units < sm_count ? n_units : sm_count;
  eval_tc_multi_y_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(
      yi, reinterpret_cast<const CUtensorMap*>(mapsA), reinterpret_cast<const CUtensorMap*>(mapsB),
      reinterpret_cast<const CUtensorMap*>(mapsU), units, n_units, err);
  return cudaGetLastError();
}

size_t eval_tc_chunk_bytes(int n_tc) {
  return sizeof(int4) * (make_chunks(n_tc, BN, false).size() + make_chunks_y(n_tc).size() +
                         make_chunks(n_tc, BN_TS, false).size());
}

// The three chunk tables of one padded size, built once per process and size.
struct ChunkTables {
  std::vector<int4> all;  // evaluation, full square, 192-column evaluation
  int n_eval = 0, n_full = 0, n_ts = 0;
};
static const ChunkTables& chunk_tables(int n_tc) {
  static std::mutex mu;
  static std::map<int, ChunkTables> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(n_tc);
  if (it != cache.end()) return it->second;
  ChunkTables t;
  std::vector<int4> full = make_chunks_y(n_tc), ts = make_chunks(n_tc, BN_TS, false);
  t.all = make_chunks(n_tc, BN, false);
  t.n_eval = (int)t.all.size();
  t.n_full = (int)full.size();
  t.n_ts = (int)ts.size();
  t.all.insert(t.all.end(), full.begin(), full.end());
  t.all.insert(t.all.end(), ts.begin(), ts.end());
  return cache.emplace(n_tc, std::move(t)).first->second;
}

// Copy the chunk tables to the device (async on `st`; the host tables live in
// a process-wide cache).  h->tc_chunks may already point at caller-provided
// memory of eval_tc_chunk_bytes(n_tc) bytes.
cudaError_t eval_tc_upload_tables(ubqp_q* h, cudaStream_t st) {
  const ChunkTables& t = chunk_tables(h->n_tc);
  h->tc_nchunks = t.n_eval;
  h->tc_nchunks_y = t.n_full;
  h->tc_nchunks_ts = t.n_ts;
  cudaError_t e;
  if (!h->tc_chunks && (e = cudaMalloc(&h->tc_chunks, sizeof(int4) * t.all.size()))) return e;
  return cudaMemcpyAsync(h->tc_chunks, t.all.data(), sizeof(int4) * t.all.size(),
                         cudaMemcpyHostToDevice, st);
}

// The TMA descriptors of the prepared operands (host only).
cudaError_t eval_tc_prepare(ubqp_q* h, cudaStream_t) {
  h->tc_ok = make_map(reinterpret_cast<CUtensorMap*>(h->tc_mapB), h->Qt, h->n_tc, h->n_tc, BN) &&
             make_map(reinterpret_cast<CUtensorMap*>(h->tc_mapU), h->Qu, h->n_tc, h->n_tc, BN) &&
             make_map(reinterpret_cast<CUtensorMap*>(h->tc_mapB_ts), h->Qt, h->n_tc, h->n_tc,
                      BN_TS);
  return cudaSuccess;
}

// Launch a product kernel as a programmatic dependent of the unpacking kernel
// launched just before it on the same stream (the kernel waits for that grid
// with griddepcontrol.wait before its first dependent read).
template <bool YMODE, bool FUSED>
cudaError_t launch_product(int grid, int threads, int smem, cudaStream_t st,
                           const CUtensorMap& mapA, const CUtensorMap& mapB,
                           const CUtensorMap& mapU, const uint64_t* X, int n, int W, int64_t S,
                           int m_tiles, const int4* chunks, int n_chunks, int64_t* f,
                           const int64_t* count, float* Y, int64_t ldy, unsigned* err) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  void* args[] = {const_cast<CUtensorMap*>(&mapA), const_cast<CUtensorMap*>(&mapB),
                  const_cast<CUtensorMap*>(&mapU), &X, &n, &W, &S, &m_tiles, &chunks, &n_chunks,
                  &f, &count, &Y, &ldy, &err};
  return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(&eval_tc_kernel<YMODE, FUSED>),
                             args);
}

size_t ascent_tc_workspace(const ubqp_q* h, int64_t S) {
  return (size_t)padded_starts(S) * (size_t)h->n_tc * (2 + 4);
}

// y = Q x for the starts idx[0 .. *count) into Y (fp32, row t = idx[t], stride
// n_tc), on the tensor cores.  ws holds the unpacked starts then Y.
bool eval_tc_map_A(void* out128, const void* Xe, int64_t S, int n_tc) {
  return make_map(reinterpret_cast<CUtensorMap*>(out128), Xe, padded_starts(S), n_tc, BM);
}

cudaError_t launch_ascent_init_tc(const ubqp_q* h, const uint64_t* X, const int32_t* idx,
                                  const int64_t* count, int64_t S, void* ws, size_t ws_bytes,
                                  float** Y_out, cudaStream_t st, const void* mapA_in,
                                  unsigned long long* zero_next) {
  if (!h->tc_ok) return cudaErrorNotSupported;
  const int64_t S_p = padded_starts(S);
  if (ws_bytes < ascent_tc_workspace(h, S)) return cudaErrorInvalidValue;
  uint8_t* Xe = reinterpret_cast<uint8_t*>(ws);
  float* Y = reinterpret_cast<float*>(Xe + (size_t)S_p * h->n_tc * 2);
  cudaError_t e;
  {
    const int64_t blocks = std::min<int64_t>(S_p, (int64_t)h->sm_count * 8);
    if ((e = launch_pdl(unpack_bits_bf16, dim3((unsigned)blocks), dim3(kUnpackThreads), 0, st, X,
                        h->n, h->W, S, idx, count, S_p, h->n_tc, reinterpret_cast<uint4*>(Xe), Y,
                        reinterpret_cast<int64_t*>(zero_next), (int64_t)(zero_next ? 1 : 0))))
      return e;
  }
  alignas(64) CUtensorMap mapA;
  if (mapA_in) mapA = *reinterpret_cast<const CUtensorMap*>(mapA_in);
  else if (!make_map(&mapA, Xe, S_p, h->n_tc, BM)) return cudaErrorInvalidValue;
  if ((e = set_smem_attr_once<true, false>())) return e;
  const int m_tiles = (int)(S_p / BM);
  const int n_units = h->tc_nchunks_y * m_tiles;
  const int grid = n_units < h->sm_count ? n_units : h->sm_count;
  if ((e = launch_product<true, false>(
           grid, THREADS, SMEM_BYTES, st, mapA, *reinterpret_cast<const CUtensorMap*>(h->tc_mapB),
           *reinterpret_cast<const CUtensorMap*>(h->tc_mapU), X, h->n, h->W, S, m_tiles,
           reinterpret_cast<const int4*>(h->tc_chunks) + h->tc_nchunks, h->tc_nchunks_y, nullptr,
           count, Y, (int64_t)h->n_tc, h->err)))
    return e;
  *Y_out = Y;
  return cudaSuccess;
}

cudaError_t launch_selftest_wait(uint64_t limit_ns, int32_t* status, cudaStream_t st) {
  selftest_wait_kernel<<<1, 32, 0, st>>>(limit_ns, status);
  return cudaGetLastError();
}

cudaError_t launch_eval_ts(const ubqp_q* h, const uint64_t* X, int64_t S, int64_t* f,
                           cudaStream_t st) {
  if (!h->tc_ok) return cudaErrorNotSupported;
  cudaError_t e;
  if ((e = cudaMemsetAsync(f, 0, sizeof(int64_t) * S, st))) return e;
  const int m_tiles = (int)(padded_starts(S) / BM);
  const int n_units = h->tc_nchunks_ts * m_tiles;
  const int grid = n_units < h->sm_count ? n_units : h->sm_count;
  if ((e = set_smem_attr_ts_once())) return e;
  const int4* ch = reinterpret_cast<const int4*>(h->tc_chunks) + h->tc_nchunks + h->tc_nchunks_y;
  eval_ts_kernel<<<grid, THREADS_TS, SMEM_BYTES_TS, st>>>(
      *reinterpret_cast<const CUtensorMap*>(h->tc_mapB_ts), X, h->n, h->W, S, m_tiles, ch,
      h->tc_nchunks_ts, f, h->err);
  return cudaGetLastError();
}

cudaError_t launch_eval_tc(const ubqp_q* h, const uint64_t* X, int64_t S, int64_t* f, void* ws,
                           size_t ws_bytes, cudaStream_t st, const void* mapA_in, bool fused,
                           const int4* chunks_in, int nchunks_in) {
  if (!h->tc_ok) return cudaErrorNotSupported;
  const int64_t S_p = padded_starts(S);
  cudaError_t e;
  alignas(64) CUtensorMap mapA;
  if (fused) {
    mapA = *reinterpret_cast<const CUtensorMap*>(h->tc_mapB);  // unused by the fused kernel
    if ((e = cudaMemsetAsync(f, 0, sizeof(int64_t) * S, st))) return e;
  } else {
    if (ws_bytes < eval_tc_workspace(h, S)) return cudaErrorInvalidValue;
    if (mapA_in) mapA = *reinterpret_cast<const CUtensorMap*>(mapA_in);
    else if (!make_map(&mapA, ws, S_p, h->n_tc, BM)) return cudaErrorInvalidValue;
    // the unpacking also zeroes f
    const int64_t blocks = std::min<int64_t>(S_p, (int64_t)h->sm_count * 8);
    if ((e = launch_pdl(unpack_bits_bf16, dim3((unsigned)blocks), dim3(kUnpackThreads), 0, st, X,
                        h->n, h->W, S, nullptr, nullptr, S_p, h->n_tc,
                        reinterpret_cast<uint4*>(ws), nullptr, f, S)))
      return e;
  }
  const int m_tiles = (int)(S_p / BM);
  const int4* ch = chunks_in ? chunks_in : reinterpret_cast<const int4*>(h->tc_chunks);
  const int nch = chunks_in ? nchunks_in : h->tc_nchunks;
  const int n_units = nch * m_tiles;
  const int grid = n_units < h->sm_count ? n_units : h->sm_count;
  const CUtensorMap& mapB = *reinterpret_cast<const CUtensorMap*>(h->tc_mapB);
  if (fused) {
    if ((e = set_smem_attr_once<false, true>())) return e;
    eval_tc_kernel<false, true><<<grid, THREADS_FUSED, SMEM_BYTES_FUSED, st>>>(
        mapA, mapB, mapB, X, h->n, h->W, S, m_tiles, ch, nch, f, nullptr, nullptr, 0, h->err);
  } else {
    if ((e = set_smem_attr_once<false, false>())) return e;
    return launch_product<false, false>(grid, THREADS, SMEM_BYTES, st, mapA, mapB, mapB, X, h->n,
                                        h->W, S, m_tiles, ch, nch, f, nullptr, nullptr, 0,
                                        h->err);
  }
  return cudaGetLastError();
}

}  // namespace ubqp
