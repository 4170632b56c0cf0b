// ascent_core.cuh -- the move machinery of the batched steepest ascent and of
// path relinking (kernels and launch helpers), shared by k_ascent.cu and
// k_ascent_trace.cu.  Internal to libubqp.  The design is described at the
// top of k_ascent.cu.
#pragma once
#include <climits>

#include "ubqp_internal.cuh"

namespace ubqp {
namespace {

constexpr int64_t kTimeoutNs = 20ll * 1000 * 1000 * 1000;  // per start
// Runner-up rows copied one move ahead.  Measured at n = 7000 / 2500 / 1500
// (passing starts of 1000 random ones): one row is 3-13% faster than none;
// two or more cost more in reductions and copies than their hits save.
constexpr int kSpecRows = 1;
// shared-memory slots (16 bytes each) of a group of T threads: two buffers of
// R rows x C chunks per thread, laid out thread-minor
template <int T, int C, int R>
constexpr int spec_slot_count() {
  return R > 0 ? T * 2 * R * C : 1;
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// acc + d * (signed byte i of w), for d in {-1, +1}, in one dp4a: the second
// operand holds d in byte i and zeros elsewhere.
__device__ __forceinline__ int byte_sel(int i, int d) {
  return (int)((unsigned)(d & 0xFF) << (8 * i));
}

// The R best entries (gain r.x, tag r.y) held one per lane across a warp,
// excluding the entry tagged `first`: their tags in decreasing order of gain
// (ties to the lower lane), INT_MAX where fewer entries remain.  One max
// reduction per rank on gain * 32 + (31 - lane) (|gain| < 2^26), then one
// shuffle per rank for the tags.
template <int R>
__device__ __forceinline__ void runners_up(int2 r, int first, int* cand) {
  const int lane = threadIdx.x & 31;
  int key = (r.y == first || r.y == INT_MAX) ? INT_MIN : r.x * 32 + (31 - lane);
  int wl[R];
  bool ok[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int m = __reduce_max_sync(0xffffffffu, key);
    ok[i] = m != INT_MIN;
    wl[i] = 31 - (m & 31);
    if (lane == wl[i]) key = INT_MIN;
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int t = __shfl_sync(0xffffffffu, r.y, wl[i]);
    cand[i] = ok[i] ? t : INT_MAX;
  }
}

// Negate S and toggle the x bit of element ek (relinking: freeze it) with a
// binary decision on ek: about log2(E) branches instead of E predicated ops.
template <int LO, int HI, int E, bool RL>
__device__ __forceinline__ void flip_tree(int (&S)[E], int (&Ck)[E], int ek) {
  if constexpr (HI - LO == 1) {
    S[LO] = RL ? 0 : -S[LO];
    Ck[LO] = RL ? INT_MIN : (Ck[LO] ^ 1);
  } else {
    constexpr int MID = (LO + HI) / 2;
    if (ek < MID) flip_tree<LO, MID, E, RL>(S, Ck, ek);
    else flip_tree<MID, HI, E, RL>(S, Ck, ek);
  }
}

template <int T>
struct Group;

// One warp per start.
template <>
struct Group<32> {
  __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
  int2 mine;  // this lane's entry of the last reduction
  // returns {max gain, 2k + x_k} over the group
  __device__ __forceinline__ int2 reduce(int gain, int jx) {
    const int m = __reduce_max_sync(0xffffffffu, gain);
    const int c = __reduce_min_sync(0xffffffffu, gain == m ? jx : INT_MAX);
    mine = make_int2(gain, jx);
    return make_int2(m, c);
  }
  // runners-up of the last reduction among the lanes' own maxima
  template <int R>
  __device__ __forceinline__ void runners(int first, int* cand) const {
    runners_up<R>(mine, first, cand);
  }
  __device__ __forceinline__ bool any(bool p) { return __any_sync(0xffffffffu, p); }
  __device__ __forceinline__ void sync() { __syncwarp(); }
  __device__ __forceinline__ int sum(int v) { return __reduce_add_sync(0xffffffffu, v); }
};

// One block per start.
template <int T>
struct Group {
  static constexpr int NW = T / 32;
  int2 (*rec)[NW];  // [2][NW] shared
  int parity;
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  int2 mine;  // warp `lane`'s winner in the last reduction
  // returns {max gain, 2k + x_k} over the group
  __device__ __forceinline__ int2 reduce(int gain, int jx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = __reduce_max_sync(0xffffffffu, gain);
    const int c = __reduce_min_sync(0xffffffffu, gain == m ? jx : INT_MAX);
    if (lane == 0) rec[parity][warp] = make_int2(m, c);
    __syncthreads();
    const int2 r = lane < NW ? rec[parity][lane] : make_int2(INT_MIN, INT_MAX);
    const int m2 = __reduce_max_sync(0xffffffffu, r.x);
    const int c2 = __reduce_min_sync(0xffffffffu, r.x == m2 ? r.y : INT_MAX);
    parity ^= 1;
    mine = r;
    return make_int2(m2, c2);
  }
  // runners-up of the last reduction among the warps' winners
  template <int R>
  __device__ __forceinline__ void runners(int first, int* cand) const {
    runners_up<R>(mine, first, cand);
  }
  __device__ __forceinline__ bool any(bool p) { return __syncthreads_or(p) != 0; }
  __device__ __forceinline__ void sync() { __syncthreads(); }
  __device__ __forceinline__ int sum(int v) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = __reduce_add_sync(0xffffffffu, v);
    if (lane == 0) rec[parity][warp] = make_int2(s, 0);
    __syncthreads();
    const int r = lane < NW ? rec[parity][lane].x : 0;
    parity ^= 1;
    return __reduce_add_sync(0xffffffffu, r);
  }
};

// TS consecutive threads of a larger block owning one start (TS >= 64, a
// multiple of 32): the block-group operations of Group<TS> on the named
// barrier `bar` (1..15) instead of the block-wide one, so that several
// sub-groups of one block climb different starts independently.
__device__ __forceinline__ void named_sync(int bar, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool named_or(int bar, int count, bool p) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n"
      " bar.red.or.pred po, %2, %3, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)p), "r"(bar), "r"(count)
      : "memory");
  return out != 0;
}

template <int TS>
struct SubGroup {
  static constexpr int NW = TS / 32;
  int2 (*rec)[NW];  // [2][NW] shared, this sub-group's
  int parity;
  int base;  // first thread of the sub-group
  int bar;   // its named barrier
  __device__ __forceinline__ int rank() const { return (int)threadIdx.x - base; }
  int2 mine;
  __device__ __forceinline__ int2 reduce(int gain, int jx) {
    const int lane = threadIdx.x & 31, warp = rank() >> 5;
    const int m = __reduce_max_sync(0xffffffffu, gain);
    const int c = __reduce_min_sync(0xffffffffu, gain == m ? jx : INT_MAX);
    if (lane == 0) rec[parity][warp] = make_int2(m, c);
    named_sync(bar, TS);
    const int2 r = lane < NW ? rec[parity][lane] : make_int2(INT_MIN, INT_MAX);
    const int m2 = __reduce_max_sync(0xffffffffu, r.x);
    const int c2 = __reduce_min_sync(0xffffffffu, r.x == m2 ? r.y : INT_MAX);
    parity ^= 1;
    mine = r;
    return make_int2(m2, c2);
  }
  template <int R>
  __device__ __forceinline__ void runners(int first, int* cand) const {
    runners_up<R>(mine, first, cand);
  }
  __device__ __forceinline__ bool any(bool p) { return named_or(bar, TS, p); }
  __device__ __forceinline__ void sync() { named_sync(bar, TS); }
  __device__ __forceinline__ int sum(int v) {
    const int lane = threadIdx.x & 31, warp = rank() >> 5;
    const int sv = __reduce_add_sync(0xffffffffu, v);
    if (lane == 0) rec[parity][warp] = make_int2(sv, 0);
    named_sync(bar, TS);
    const int r = lane < NW ? rec[parity][lane].x : 0;
    parity ^= 1;
    return __reduce_add_sync(0xffffffffu, r);
  }
};

// Path relinking of one pair (see relink_block_kernel): the guiding solution,
// the outputs and a trace of the flipped indices (n entries of scratch).
struct RelinkArgs {
  const uint64_t* g;
  uint64_t* x_best;
  int64_t* f_best;
  int32_t* dist;
  uint16_t* trace;
};

// RL = false: steepest ascent of x_g in place (f_s updated, flips to flips_s).
// RL = true: path relinking from x_g (read only, value *f_s) toward rl->g --
// the same move machinery, but only variables where x and g differ are
// candidates, every step is taken whatever its gain, a flipped variable leaves
// the candidate set, and the best solution strictly between the endpoints is
// the result.
template <int T, int C, int R, bool RL = false, bool TR = false, class G = Group<T>>
__device__ __forceinline__ void ascend_one(const int8_t* __restrict__ Q8, int64_t ldq,
                                           int64_t ldy, int n,
                                           int W, uint64_t* __restrict__ x_g,
                                           int64_t* __restrict__ f_s, int32_t max_flips,
                                           int32_t* __restrict__ flips_s,
                                           unsigned* __restrict__ err, uint64_t* xs,
                                           uint4* spec_slots,
                                           const float* __restrict__ y_g, G& grp,
                                           const RelinkArgs* rl = nullptr,
                                           uint16_t* __restrict__ trace_row = nullptr,
                                           int64_t trace_cap = 0) {
  constexpr int E = 16 * C;
  constexpr int CW = 16 * T;  // indices per chunk
  static_assert(E <= 32, "local index must fit 5 bits");
  const int g = grp.rank();

  int y[E], S[E], Ck[E];
  int ndiff = 0;  // relinking: owned variables where x and g differ
  // ---- owned bits of x; C and S per element
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int j0 = c * CW + 16 * g;
    uint32_t nib = 0, diff = 0xFFFFu;
    if (j0 < n) {
      nib = (uint32_t)((x_g[j0 >> 6] >> (j0 & 63)) & 0xFFFFull);
      if (n - j0 < 16) nib &= (1u << (n - j0)) - 1u;
      if (RL) {
        uint32_t gn = (uint32_t)((rl->g[j0 >> 6] >> (j0 & 63)) & 0xFFFFull);
        if (n - j0 < 16) gn &= (1u << (n - j0)) - 1u;
        diff = nib ^ gn;
        ndiff += __popc(diff);
      }
    }
#pragma unroll
    for (int o = 0; o < 16; ++o) {
      const int e = c * 16 + o, j = j0 + o;
      const int xb = (int)((nib >> o) & 1u);
      y[e] = 0;
      if (j < n && ((diff >> o) & 1u)) {
        const int qjj = Q8[(int64_t)j * ldq + j];
        S[e] = xb ? -128 : 128;
        Ck[e] = 64 * qjj + 2 * (31 - e) + xb;
      } else {
        S[e] = 0;
        Ck[e] = INT_MIN;
      }
    }
  }
  // ---- y = Q x on the owned columns: from the tensor-core start-up when
  // given (y_g, exact integers in fp32), else by adding the rows k with x_k = 1
  if (y_g) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int j0 = c * CW + 16 * g;
      if (j0 < ldy) {
        const float4* src = reinterpret_cast<const float4*>(y_g + j0);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float4 t4 = src[v];
          y[c * 16 + 4 * v + 0] = __float2int_rn(t4.x);
          y[c * 16 + 4 * v + 1] = __float2int_rn(t4.y);
          y[c * 16 + 4 * v + 2] = __float2int_rn(t4.z);
          y[c * 16 + 4 * v + 3] = __float2int_rn(t4.w);
        }
      }
    }
  }
  for (int w = 0; w < W && !y_g; ++w) {
    uint64_t word = x_g[w] & valid_mask(n, w);
    while (word) {
      constexpr int RF = C == 1 ? 4 : 2;  // rows in flight
      int ks[RF];
      int nk = 0;
#pragma unroll
      for (int r = 0; r < RF; ++r) {
        ks[r] = 0;
        if (word) {
          ks[r] = w * 64 + __ffsll((long long)word) - 1;
          word &= word - 1;
          nk = r + 1;
        }
      }
      uint4 q[RF][C];
#pragma unroll
      for (int r = 0; r < RF; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int j0 = c * CW + 16 * g;
          q[r][c] = (r < nk && j0 < ldq)
                        ? __ldg(reinterpret_cast<const uint4*>(Q8 + (int64_t)ks[r] * ldq + j0))
                        : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
      for (int r = 0; r < RF; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int wv[4] = {(int)q[r][c].x, (int)q[r][c].y, (int)q[r][c].z, (int)q[r][c].w};
#pragma unroll
          for (int o = 0; o < 16; ++o)
            y[c * 16 + o] = __dp4a(wv[o >> 2], byte_sel(o & 3, 1), y[c * 16 + o]);
        }
    }
  }
  // ---- first argmax
  int kmax = INT_MIN;
#pragma unroll
  for (int e = 0; e < E; ++e) kmax = max(kmax, Ck[e] + S[e] * y[e]);
  // Speculation: the next move is often the runner-up of the previous
  // reduction (about 40% of moves at n = 7000), so each move copies this
  // thread's chunks of the runner-up rows (prow) into its own shared-memory
  // slots with cp.async; a hit reads them there instead of waiting for a
  // dependent L2 round trip.  Two buffers alternate: the copies of move t go
  // to buffer t % 2 and are read at move t + 1.  Each thread reads only the
  // bytes it copied, so its own cp.async.wait_group orders them.
  constexpr int RR = R > 0 ? R : 1;
  int cand[RR], prow[RR];
#pragma unroll
  for (int i = 0; i < RR; ++i) prow[i] = -1;
  // slot (buffer b, row i, chunk c) of thread g at plane ((b RR + i) C + c):
  // planes of T x 16 bytes, threads side by side, so a warp's copies and
  // reads cover all banks without conflicts
  const uint32_t slot0 = (uint32_t)__cvta_generic_to_shared(spec_slots) + (uint32_t)g * 16;
  int buf = 0;
  auto reduce_key = [&](int kt) {
    const int gain = kt >> 6;
    const int e = 31 - ((kt >> 1) & 31);
    const int j = (e >> 4) * CW + 16 * g + (e & 15);
    return grp.reduce(gain, (j << 1) | (kt & 1));
  };
  int2 best = reduce_key(kmax);

  int64_t fval = *f_s;
  int flips = 0;
  // relinking: path length, best intermediate value and its step
  const int dist = RL ? grp.sum(ndiff) : 0;
  int64_t fbest = fval;
  int tbest = 0;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (RL) {
      if (flips >= dist - 1) break;  // the last step only reaches g
    } else {
      if (max_flips > 0 && flips >= max_flips) break;
      if (best.x <= 0) break;
    }
    if ((flips & 1023) == 1023) {
      const bool late = (int64_t)(globaltimer() - t0) > kTimeoutNs;
      if (grp.any(late)) {
        if (g == 0) atomicOr(err, UBQP_DEVERR_TIMEOUT);
        break;
      }
    }
    const int k = best.y >> 1;
    const int d = (best.y & 1) ? -1 : 1;  // 1 - 2 x_k before the flip
    const int dsel[4] = {byte_sel(0, d), byte_sel(1, d), byte_sel(2, d), byte_sel(3, d)};
    fval += best.x;
    ++flips;
    if (RL) {
      if (flips < dist && (tbest == 0 || fval > fbest)) {
        fbest = fval;
        tbest = flips;
      }
      if (g == 0) rl->trace[flips - 1] = (uint16_t)k;
    }
    if constexpr (TR) {  // the move record: flipped indices in order
      if (g == 0 && flips <= trace_cap) trace_row[flips - 1] = (uint16_t)k;
    }
    uint4 q[C];
    bool hit = false;
    if constexpr (R > 0) {
      int hi = -1;
#pragma unroll
      for (int i = 0; i < R; ++i)
        if (prow[i] == k) hi = i;
      if (hi >= 0) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        const uint32_t a = slot0 + (uint32_t)(((buf ^ 1) * RR + hi) * C) * (T * 16);
#pragma unroll
        for (int c = 0; c < C; ++c)
          asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(q[c].x), "=r"(q[c].y), "=r"(q[c].z), "=r"(q[c].w)
                       : "r"(a + (uint32_t)(c * T * 16)));
        hit = true;
      }
    }
    if (!hit) {
      const int8_t* row = Q8 + (int64_t)k * ldq;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int j0 = c * CW + 16 * g;
        q[c] = j0 < ldq ? __ldg(reinterpret_cast<const uint4*>(row + j0))
                        : make_uint4(0, 0, 0, 0);
      }
    }
    if constexpr (R > 0) {  // fetch the runners-up's rows for the next move
      grp.template runners<R>(best.y, cand);
      // the copies into this buffer two moves ago have landed
      asm volatile("cp.async.wait_group 1;" ::: "memory");
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int r = cand[i] >> 1;
        prow[i] = r < n ? r : -1;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int j0 = c * CW + 16 * g;
          // chunks at or beyond ldq are not copied: their elements have
          // S = 0, so whatever the slot holds never changes a key
          if (prow[i] >= 0 && j0 < ldq) {
            const int8_t* src = Q8 + (int64_t)prow[i] * ldq + j0;
            const uint32_t a = slot0 + (uint32_t)((buf * RR + i) * C + c) * (T * 16);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(src)
                         : "memory");
          }
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      buf ^= 1;
    }
    // the owner of k flips x_k: negate S_k, toggle the x bit in C_k (when
    // relinking, k leaves the candidates instead: S_k = 0, C_k = INT_MIN)
    const int kc = k / CW, kr = k - kc * CW;
    if ((kr >> 4) == g) {
      const int ek = kc * 16 + (kr & 15);
      flip_tree<0, E, E, RL>(S, Ck, ek);
    }
    int km[4] = {INT_MIN, INT_MIN, INT_MIN, INT_MIN};
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int wv[4] = {(int)q[c].x, (int)q[c].y, (int)q[c].z, (int)q[c].w};
#pragma unroll
      for (int o = 0; o < 16; o += 2) {
        const int e = c * 16 + o;
        y[e] = __dp4a(wv[o >> 2], dsel[o & 3], y[e]);
        y[e + 1] = __dp4a(wv[o >> 2], dsel[(o + 1) & 3], y[e + 1]);
        km[(o >> 1) & 3] = __vimax3_s32(km[(o >> 1) & 3], Ck[e] + S[e] * y[e],
                                        Ck[e + 1] + S[e + 1] * y[e + 1]);
      }
    }
    kmax = max(max(km[0], km[1]), max(km[2], km[3]));
    best = reduce_key(kmax);
  }
  // copies still in flight must land before the slots serve another start
  if (R > 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
  if constexpr (RL) {
    // ---- the best intermediate: x with the first tbest traced flips applied
    if (g == 0) {
      *rl->f_best = fbest;
      if (rl->dist) *rl->dist = dist;
    }
    for (int w = g; w < W; w += T) xs[w] = x_g[w];
    grp.sync();
    for (int t = g; t < tbest; t += T) {
      const int k = rl->trace[t];
      atomicXor(reinterpret_cast<unsigned long long*>(&xs[k >> 6]), 1ull << (k & 63));
    }
    grp.sync();
    for (int w = g; w < W; w += T) rl->x_best[w] = xs[w];
    grp.sync();
    return;
  }
  // ---- write back f, flips and x
  if (g == 0) {
    *f_s = fval;
    if (flips_s) *flips_s = flips;
  }
  for (int w = g; w < W; w += T) xs[w] = 0;
  grp.sync();
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int j0 = c * CW + 16 * g;
    uint64_t bits = 0;
#pragma unroll
    for (int o = 0; o < 16; ++o) bits |= (uint64_t)(Ck[c * 16 + o] & 1 & (S[c * 16 + o] != 0)) << o;
    if (bits) atomicOr(reinterpret_cast<unsigned long long*>(&xs[j0 >> 6]),
                       (unsigned long long)(bits << (j0 & 63)));
  }
  grp.sync();
  for (int w = g; w < W; w += T) x_g[w] = xs[w];
  grp.sync();
}

// The first wave of listed starts goes one per group in launch order (the
// block scheduler spreads them over the SMs); the rest are taken from the
// counter *next (zero at launch) one at a time as groups finish, so the long
// and short climbs even out over the SMs.  next == NULL: round robin.
// TR: also record each start's flipped indices in order, row s of trace (ldt
// entries; moves beyond ldt are made but not recorded).  OCC: blocks per SM
// the registers are sized for.  The kernel climbs only when the number of
// listed starts lies in [cnt_lo, cnt_hi] and returns at once otherwise, so
// that two launches of different OCC can share one list, each taking the
// counts it is faster for, with no host round trip for the count.  A
// programmatic dependent of the kernel before it on the stream (pdl_wait).
template <int T, int C, int R, bool TR, int OCC>
__global__ void __launch_bounds__(T, OCC)
ascent_block_kernel(const int8_t* __restrict__ Q8, int64_t ldq, int n, int W,
                    uint64_t* __restrict__ X, int64_t* __restrict__ f,
                    const int32_t* __restrict__ idx, const int64_t* __restrict__ count,
                    int64_t S, int32_t max_flips, int32_t* __restrict__ flips,
                    const float* __restrict__ Y, int64_t ldy, unsigned* __restrict__ err,
                    unsigned long long* __restrict__ next, uint16_t* __restrict__ trace,
                    int64_t ldt, int64_t cnt_lo, int64_t cnt_hi) {
  __shared__ int2 rec[2][T / 32];
  __shared__ uint64_t xs[UBQP_MAX_N / 64];
  __shared__ uint4 spec_slots[spec_slot_count<T, C, R>()];
  __shared__ unsigned long long ticket;
  Group<T> grp{rec, 0};
  pdl_wait();  // no early release: see pdl_release
  if (err[1] != 0) return;  // Q failed its symmetry check: no climb
  const int64_t cnt = *count;
  if (cnt < cnt_lo || cnt > cnt_hi) return;  // the other launch's counts
  auto take = [&](int64_t t) -> int64_t {  // the block's next start
    if (t < 0) return blockIdx.x;
    if (!next) return t + gridDim.x;
    if (threadIdx.x == 0) ticket = atomicAdd(next, 1ull);
    __syncthreads();
    const int64_t v = (int64_t)gridDim.x + (int64_t)ticket;
    __syncthreads();
    return v;
  };
  for (int64_t t = take(-1); t < cnt; t = take(t)) {
    const int s = idx[t];
    if (s < 0 || s >= S) {
      if (threadIdx.x == 0) atomicOr(err, UBQP_DEVERR_BADIDX);
      continue;
    }
    ascend_one<T, C, R, false, TR>(Q8, ldq, ldy, n, W, X + (int64_t)s * W, f + s, max_flips,
                                   flips ? flips + s : nullptr, err, xs, spec_slots,
                                   Y ? Y + t * ldy : nullptr, grp, nullptr,
                                   TR ? trace + (int64_t)s * ldt : nullptr, ldt);
  }
}

// All passing starts of a batch of instances in one persistent launch: item
// t = (instance, position in its passing list); every instance has n <= 16 T C.
template <int T, int C, int R>
__global__ void __launch_bounds__(T, 1)
ascent_batch_kernel(const BatchDesc* __restrict__ d, const int2* __restrict__ items,
                    const int64_t* __restrict__ n_items, int32_t max_flips,
                    unsigned long long* __restrict__ next) {
  __shared__ int2 rec[2][T / 32];
  __shared__ uint64_t xs[UBQP_MAX_N / 64];
  __shared__ uint4 spec_slots[spec_slot_count<T, C, R>()];
  __shared__ unsigned long long ticket;
  Group<T> grp{rec, 0};
  const int64_t cnt = *n_items;
  // the first wave one item per block, the rest from the counter (as in
  // ascent_block_kernel)
  auto take = [&](int64_t t) -> int64_t {
    if (t < 0) return blockIdx.x;
    if (!next) return t + gridDim.x;
    if (threadIdx.x == 0) ticket = atomicAdd(next, 1ull);
    __syncthreads();
    const int64_t v = (int64_t)gridDim.x + (int64_t)ticket;
    __syncthreads();
    return v;
  };
  for (int64_t t = take(-1); t < cnt; t = take(t)) {
    const int2 it = items[t];
    const BatchDesc& b = d[it.x];
    if (b.err[1] != 0) continue;  // Q failed its symmetry check: no climb
    const int s = b.idx[it.y];
    if (s < 0 || s >= b.S) {
      if (threadIdx.x == 0) atomicOr(b.err, UBQP_DEVERR_BADIDX);
      continue;
    }
    ascend_one<T, C, R>(b.Q8, b.ldq, b.ldy, b.n, b.W, b.X + (int64_t)s * b.W, b.f + s, max_flips,
                     b.flips ? b.flips + s : nullptr, b.err, xs, spec_slots,
                     b.Y ? b.Y + (int64_t)it.y * b.ldy : nullptr, grp);
  }
}

// All passing starts of a batch of instances in one persistent launch, packed
// by size.  Class c (0 .. 3) holds the instances whose n fits a sub-group of
// T >> c threads (16 (T >> c) C elements; T >> 3 = 32 is one warp), and its
// items form the range ranges[c] = {first item, items, 0, 0} (instances come
// largest first, so each class is contiguous).  Each block runs the classes
// in turn, split into 2^c sub-groups for class c, and every sub-group takes
// the class's next start from its counter next[c] as soon as it has finished
// the previous one: a block climbs up to eight small starts at once, and no
// sub-group waits for another's longer climb except at the three class
// boundaries.
template <int T, int C, int R, int TS>
__device__ __forceinline__ void climb_item(const BatchDesc* __restrict__ d, int2 it,
                                           int32_t max_flips, int2* rec_flat, uint64_t* xs,
                                           uint4* spec_slots, int sg) {
  const BatchDesc& b = d[it.x];
  if (b.err[1] != 0) return;  // Q failed its symmetry check: no climb
  const int s = b.idx[it.y];
  if (s < 0 || s >= b.S) {
    if ((int)threadIdx.x == sg * TS) atomicOr(b.err, UBQP_DEVERR_BADIDX);
    return;
  }
  if constexpr (TS == T) {
    Group<T> grp{reinterpret_cast<int2 (*)[T / 32]>(rec_flat), 0};
    ascend_one<T, C, R>(b.Q8, b.ldq, b.ldy, b.n, b.W, b.X + (int64_t)s * b.W, b.f + s, max_flips,
                        b.flips ? b.flips + s : nullptr, b.err, xs, spec_slots,
                        b.Y ? b.Y + (int64_t)it.y * b.ldy : nullptr, grp);
  } else if constexpr (TS == 32) {  // one warp per start: warp-level reductions only
    Group<32> grp;
    ascend_one<32, C, R>(b.Q8, b.ldq, b.ldy, b.n, b.W, b.X + (int64_t)s * b.W, b.f + s,
                         max_flips, b.flips ? b.flips + s : nullptr, b.err, xs + sg * (32 * C / 4),
                         spec_slots + sg * spec_slot_count<32, C, R>(),
                         b.Y ? b.Y + (int64_t)it.y * b.ldy : nullptr, grp);
  } else {
    SubGroup<TS> grp{reinterpret_cast<int2 (*)[TS / 32]>(rec_flat + sg * 2 * (TS / 32)), 0,
                     sg * TS, 1 + sg};
    ascend_one<TS, C, R>(b.Q8, b.ldq, b.ldy, b.n, b.W, b.X + (int64_t)s * b.W, b.f + s,
                         max_flips, b.flips ? b.flips + s : nullptr, b.err,
                         xs + sg * (TS * C / 4), spec_slots + sg * spec_slot_count<TS, C, R>(),
                         b.Y ? b.Y + (int64_t)it.y * b.ldy : nullptr, grp);
  }
}

// The sub-groups of one class take its starts: the first wave spread over the
// blocks (start sg * blocks + block, so that a short list lands one start per
// block, not several on the blocks of one SM), then from the class's counter
// (or, without counters, round robin over all sub-groups of the grid).
template <int T, int C, int R, int TS>
__device__ __forceinline__ void climb_class(const BatchDesc* __restrict__ d,
                                            const int2* __restrict__ items, int4 range,
                                            int32_t max_flips, unsigned long long* next,
                                            int2* rec_flat, uint64_t* xs, uint4* spec_slots,
                                            long long* slot) {
  constexpr int K = T / TS;
  const int sg = (int)threadIdx.x / TS, r = (int)threadIdx.x % TS;
  auto sg_sync = [&]() {
    if constexpr (TS == T) __syncthreads();
    else if constexpr (TS == 32) __syncwarp();
    else named_sync(1 + sg, TS);
  };
  const long long wave = (long long)gridDim.x * K;
  for (long long k = 0;; ++k) {
    long long t = (long long)sg * gridDim.x + blockIdx.x;
    if (k > 0) {
      if (r == 0) slot[sg] = next ? wave + (long long)atomicAdd(next, 1ull) : t + k * wave;
      sg_sync();
      t = slot[sg];
      sg_sync();  // every thread has read slot[sg] before its leader writes it again
    }
    if (t >= range.y) break;
    climb_item<T, C, R, TS>(d, items[range.x + t], max_flips, rec_flat, xs, spec_slots, sg);
  }
}

template <int T, int C, int R>
__global__ void __launch_bounds__(T, 2)
ascent_batch_packed_kernel(const BatchDesc* __restrict__ d, const int2* __restrict__ items,
                           const int4* __restrict__ ranges, int32_t max_flips,
                           unsigned long long* __restrict__ next) {
  static_assert(T / 8 == 32, "sub-groups down to one warp");
  __shared__ int2 rec_flat[2 * (T / 32)];
  __shared__ uint64_t xs[T * C / 4];
  __shared__ uint4 spec_slots[spec_slot_count<T, C, R>()];
  __shared__ long long slot[8];
  climb_class<T, C, R, T>(d, items, ranges[0], max_flips, next ? next : nullptr, rec_flat, xs,
                          spec_slots, slot);
  __syncthreads();
  climb_class<T, C, R, T / 2>(d, items, ranges[1], max_flips, next ? next + 1 : nullptr,
                              rec_flat, xs, spec_slots, slot);
  __syncthreads();
  climb_class<T, C, R, T / 4>(d, items, ranges[2], max_flips, next ? next + 2 : nullptr,
                              rec_flat, xs, spec_slots, slot);
  __syncthreads();
  climb_class<T, C, R, T / 8>(d, items, ranges[3], max_flips, next ? next + 3 : nullptr,
                              rec_flat, xs, spec_slots, slot);
}

// Four independent warps per block, one start each (n <= 512); a
// programmatic dependent like the block kernel.
template <int C, int R, bool TR>
__global__ void __launch_bounds__(128)
ascent_warp_kernel(const int8_t* __restrict__ Q8, int64_t ldq, int n, int W,
                   uint64_t* __restrict__ X, int64_t* __restrict__ f,
                   const int32_t* __restrict__ idx, const int64_t* __restrict__ count,
                   int64_t S, int32_t max_flips, int32_t* __restrict__ flips,
                   const float* __restrict__ Y, int64_t ldy, unsigned* __restrict__ err,
                   unsigned long long* __restrict__ next, uint16_t* __restrict__ trace,
                   int64_t ldt) {
  __shared__ uint64_t xs_all[4][16];
  __shared__ uint4 spec_slots[4 * spec_slot_count<32, C, R>()];
  Group<32> grp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  pdl_wait();  // no early release: see pdl_release
  if (err[1] != 0) return;  // Q failed its symmetry check: no climb
  const int64_t cnt = *count;
  auto take = [&](int64_t t) -> int64_t {  // the warp's next start (see the block kernel)
    if (t < 0) return (int64_t)blockIdx.x * 4 + warp;
    if (!next) return t + (int64_t)gridDim.x * 4;
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(next, 1ull);
    return (int64_t)gridDim.x * 4 + (int64_t)__shfl_sync(0xffffffffu, v, 0);
  };
  for (int64_t t = take(-1); t < cnt; t = take(t)) {
    const int s = idx[t];
    if (s < 0 || s >= S) {
      if (lane == 0) atomicOr(err, UBQP_DEVERR_BADIDX);
      continue;
    }
    ascend_one<32, C, R, false, TR>(Q8, ldq, ldy, n, W, X + (int64_t)s * W, f + s, max_flips,
                                    flips ? flips + s : nullptr, err, xs_all[warp],
                                    spec_slots + warp * spec_slot_count<32, C, R>(),
                                    Y ? Y + t * ldy : nullptr, grp, nullptr,
                                    TR ? trace + (int64_t)s * ldt : nullptr, ldt);
  }
}

// Path relinking of pairs p < P: from X[p] (value f[p]) toward G[p]; the best
// intermediate solution to Xb[p], its value to fb[p], the distance to dist[p]
// (may be NULL).  trace: P rows of ldt uint16 scratch.  Y: y = Q X[p] rows from
// the tensor-core start-up, or NULL.
template <int T, int C, int R>
__global__ void __launch_bounds__(T, 1)
relink_block_kernel(const int8_t* __restrict__ Q8, int64_t ldq, int n, int W,
                    const uint64_t* __restrict__ X, const int64_t* __restrict__ f,
                    const uint64_t* __restrict__ G, int64_t P, uint64_t* __restrict__ Xb,
                    int64_t* __restrict__ fb, int32_t* __restrict__ dist,
                    uint16_t* __restrict__ trace, int64_t ldt, const float* __restrict__ Y,
                    int64_t ldy, unsigned* __restrict__ err,
                    unsigned long long* __restrict__ next) {
  __shared__ int2 rec[2][T / 32];
  __shared__ uint64_t xs[UBQP_MAX_N / 64];
  __shared__ uint4 spec_slots[spec_slot_count<T, C, R>()];
  __shared__ unsigned long long ticket;
  Group<T> grp{rec, 0};
  if (err[1] != 0) return;  // Q failed its symmetry check: no walk
  // the first wave one pair per block, the rest from the counter (as in
  // ascent_block_kernel)
  auto take = [&](int64_t t) -> int64_t {
    if (t < 0) return blockIdx.x;
    if (!next) return t + gridDim.x;
    if (threadIdx.x == 0) ticket = atomicAdd(next, 1ull);
    __syncthreads();
    const int64_t v = (int64_t)gridDim.x + (int64_t)ticket;
    __syncthreads();
    return v;
  };
  for (int64_t p = take(-1); p < P; p = take(p)) {
    const RelinkArgs a{G + p * W, Xb + p * W, fb + p, dist ? dist + p : nullptr,
                       trace + p * ldt};
    int64_t f0 = f[p];
    ascend_one<T, C, R, true>(Q8, ldq, ldy, n, W, const_cast<uint64_t*>(X + p * W), &f0, 0,
                              nullptr, err, xs, spec_slots, Y ? Y + p * ldy : nullptr, grp, &a);
  }
}

template <int C, int R>
__global__ void __launch_bounds__(128)
relink_warp_kernel(const int8_t* __restrict__ Q8, int64_t ldq, int n, int W,
                   const uint64_t* __restrict__ X, const int64_t* __restrict__ f,
                   const uint64_t* __restrict__ G, int64_t P, uint64_t* __restrict__ Xb,
                   int64_t* __restrict__ fb, int32_t* __restrict__ dist,
                   uint16_t* __restrict__ trace, int64_t ldt, const float* __restrict__ Y,
                   int64_t ldy, unsigned* __restrict__ err,
                   unsigned long long* __restrict__ next) {
  __shared__ uint64_t xs_all[4][16];
  __shared__ uint4 spec_slots[4 * spec_slot_count<32, C, R>()];
  Group<32> grp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (err[1] != 0) return;  // Q failed its symmetry check: no walk
  auto take = [&](int64_t t) -> int64_t {  // the warp's next pair (see the block kernel)
    if (t < 0) return (int64_t)blockIdx.x * 4 + warp;
    if (!next) return t + (int64_t)gridDim.x * 4;
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(next, 1ull);
    return (int64_t)gridDim.x * 4 + (int64_t)__shfl_sync(0xffffffffu, v, 0);
  };
  for (int64_t p = take(-1); p < P; p = take(p)) {
    const RelinkArgs a{G + p * W, Xb + p * W, fb + p, dist ? dist + p : nullptr,
                       trace + p * ldt};
    int64_t f0 = f[p];
    ascend_one<32, C, R, true>(Q8, ldq, ldy, n, W, const_cast<uint64_t*>(X + p * W), &f0, 0,
                               nullptr, err, xs_all[warp],
                               spec_slots + warp * spec_slot_count<32, C, R>(),
                               Y ? Y + p * ldy : nullptr, grp, &a);
  }
}

template <class K>
int resident_grid(K kernel, int threads, int sm_count) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm * sm_count;
}

template <int T, int C, bool TR, int OCC>
cudaError_t launch_block_occ(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                             const int64_t* count, int64_t S, int32_t max_flips, int32_t* flips,
                             const float* Y, unsigned long long* next, uint16_t* trace,
                             int64_t ldt, int64_t cnt_lo, int64_t cnt_hi, cudaStream_t st) {
  int grid = resident_grid(ascent_block_kernel<T, C, kSpecRows, TR, OCC>, T, h->sm_count);
  if ((int64_t)grid > S) grid = (int)S;
  return launch_pdl(ascent_block_kernel<T, C, kSpecRows, TR, OCC>, dim3(grid), dim3(T), 0, st,
                    h->Q8, h->ldq, h->n, h->W, X, f, idx, count, S, max_flips, flips, Y,
                    (int64_t)h->n_tc, h->err, next, trace, ldt, cnt_lo, cnt_hi);
}

// Block groups, registers sized for one block per SM: with at most one listed
// start per SM every start climbs alone on its SM, and this gives the shortest
// chain (measured at n = 7000: 1.91 ms for the ~52 passers of 1000 random
// starts, against 2.14 ms with registers sized for two).  The smaller groups
// (64 and 128 threads) still fit several blocks per SM.  Climbs only for
// counts up to cnt_hi; returns its resident capacity (blocks per SM x SMs).
template <int T, int C, bool TR>
cudaError_t launch_block(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                         const int64_t* count, int64_t S, int32_t max_flips, int32_t* flips,
                         const float* Y, unsigned long long* next, uint16_t* trace, int64_t ldt,
                         int64_t cnt_hi, cudaStream_t st) {
  return launch_block_occ<T, C, TR, 1>(h, X, f, idx, count, S, max_flips, flips, Y, next, trace,
                                       ldt, 0, cnt_hi, st);
}
template <int T, int C, bool TR>
int64_t block_capacity(const ubqp_q* h) {
  return resident_grid(ascent_block_kernel<T, C, kSpecRows, TR, 1>, T, h->sm_count);
}

// With more listed starts than the one-block-per-SM launch holds at once,
// several blocks per SM overlap one chain's waits with the others' work:
// groups of two 16-index chunks per thread, the fewest threads that hold n,
// and as many blocks per SM as their registers allow (measured, 1000 starts
// all climbed: n = 2000 0.94 vs 1.25 ms, 3000 2.02 vs 2.97, 4000 3.17 vs 4.02,
// 6000 7.29 vs 8.63; n = 5000 with 8192 diversified starts, ~4500 passing:
// 9.6 vs 13.5 ms).  Up to n = 1024 the one-block-per-SM groups, six per SM,
// are faster at every count, and so are 256-thread groups above n = 6144.
// The count is known only on the device, so for a list that may exceed the
// capacity both launches are made; each climbs only for its own range of
// counts and the other returns at once.
template <bool TR>
cudaError_t launch_block_many(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                              const int64_t* count, int64_t S, int32_t max_flips,
                              int32_t* flips, const float* Y, unsigned long long* next,
                              uint16_t* trace, int64_t ldt, int64_t cnt_lo, cudaStream_t st) {
  const int n = h->n;
#define UBQP_MANY(TT, OCC)                                                                   \
  return launch_block_occ<TT, 2, TR, OCC>(h, X, f, idx, count, S, max_flips, flips, Y, next, \
                                          trace, ldt, cnt_lo, INT64_MAX, st)
  if (n <= 2048) UBQP_MANY(64, 8);
  if (n <= 3072) UBQP_MANY(96, 5);
  if (n <= 4096) UBQP_MANY(128, 4);
  if (n <= 5120) UBQP_MANY(160, 3);
  if (n <= 6144) UBQP_MANY(192, 2);
  if (n <= 8192) UBQP_MANY(256, 2);
#undef UBQP_MANY
  return cudaErrorInvalidValue;
}

template <int C, bool TR>
cudaError_t launch_warp(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                        const int64_t* count, int64_t S, int32_t max_flips, int32_t* flips,
                        const float* Y, unsigned long long* next, uint16_t* trace, int64_t ldt,
                        cudaStream_t st) {
  int grid = resident_grid(ascent_warp_kernel<C, kSpecRows, TR>, 128, h->sm_count);
  const int64_t need = (S + 3) / 4;
  if ((int64_t)grid > need) grid = (int)need;
  return launch_pdl(ascent_warp_kernel<C, kSpecRows, TR>, dim3(grid), dim3(128), 0, st, h->Q8,
                    h->ldq, h->n, h->W, X, f, idx, count, S, max_flips, flips, Y,
                    (int64_t)h->n_tc, h->err, next, trace, ldt);
}

// One ascent launch over the listed starts, with the group shape that holds
// n; for 1024 < n <= 8192 and a list that may be longer than that launch's
// resident capacity, also the several-blocks-per-SM launch, the two splitting
// the counts at the capacity.
template <bool TR>
cudaError_t launch_ascent_shaped(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                                 const int64_t* count, int64_t S, int32_t max_flips,
                                 int32_t* flips, const float* Y, unsigned long long* next,
                                 uint16_t* trace, int64_t ldt, cudaStream_t st,
                                 bool next_zeroed) {
  const int n = h->n;
  if (next && !next_zeroed) {
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
#define UBQP_ASC_ARGS h, X, f, idx, count, S, max_flips, flips, Y, next, trace, ldt
  if (n <= 256) return launch_warp<1, TR>(UBQP_ASC_ARGS, st);
  if (n <= 512) return launch_warp<2, TR>(UBQP_ASC_ARGS, st);
  if (n <= 1024) return launch_block<64, 1, TR>(UBQP_ASC_ARGS, INT64_MAX, st);
  if (n > 8192) return launch_block<512, 2, TR>(UBQP_ASC_ARGS, INT64_MAX, st);
  const int64_t cap = n <= 2048 ? block_capacity<128, 1, TR>(h)
                      : n <= 4096 ? block_capacity<256, 1, TR>(h)
                                  : block_capacity<256, 2, TR>(h);
  const bool many = S > cap;
  const int64_t hi = many ? cap : INT64_MAX;
  cudaError_t e = n <= 2048   ? launch_block<128, 1, TR>(UBQP_ASC_ARGS, hi, st)
                  : n <= 4096 ? launch_block<256, 1, TR>(UBQP_ASC_ARGS, hi, st)
                              : launch_block<256, 2, TR>(UBQP_ASC_ARGS, hi, st);
  if (e != cudaSuccess || !many) return e;
  return launch_block_many<TR>(UBQP_ASC_ARGS, cap + 1, st);
#undef UBQP_ASC_ARGS
}

template <int T, int C>
cudaError_t launch_ascent_batch_tc(const BatchDesc* d, const int2* items, const int64_t* n_items,
                                   int32_t max_flips, int grid, unsigned long long* next,
                                   cudaStream_t st) {
  if (next) {
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  ascent_batch_kernel<T, C, kSpecRows><<<grid, T, 0, st>>>(d, items, n_items, max_flips, next);
  return cudaGetLastError();
}

template <int T, int C>
cudaError_t launch_relink_block(const ubqp_q* h, const uint64_t* X, const int64_t* f,
                                const uint64_t* G, int64_t P, uint64_t* Xb, int64_t* fb,
                                int32_t* dist, uint16_t* trace, int64_t ldt, const float* Y,
                                unsigned long long* next, cudaStream_t st) {
  int grid = resident_grid(relink_block_kernel<T, C, kSpecRows>, T, h->sm_count);
  if ((int64_t)grid > P) grid = (int)P;
  relink_block_kernel<T, C, kSpecRows><<<grid, T, 0, st>>>(
      h->Q8, h->ldq, h->n, h->W, X, f, G, P, Xb, fb, dist, trace, ldt, Y, h->n_tc, h->err,
      next);
  return cudaGetLastError();
}

template <int C>
cudaError_t launch_relink_warp(const ubqp_q* h, const uint64_t* X, const int64_t* f,
                               const uint64_t* G, int64_t P, uint64_t* Xb, int64_t* fb,
                               int32_t* dist, uint16_t* trace, int64_t ldt, const float* Y,
                               unsigned long long* next, cudaStream_t st) {
  int grid = resident_grid(relink_warp_kernel<C, kSpecRows>, 128, h->sm_count);
  const int64_t need = (P + 3) / 4;
  if ((int64_t)grid > need) grid = (int)need;
  relink_warp_kernel<C, kSpecRows><<<grid, 128, 0, st>>>(
      h->Q8, h->ldq, h->n, h->W, X, f, G, P, Xb, fb, dist, trace, ldt, Y, h->n_tc, h->err,
      next);
  return cudaGetLastError();
}

}  // namespace
}  // namespace ubqp
