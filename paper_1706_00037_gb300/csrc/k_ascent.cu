// k_ascent.cu -- PerformSteepestAscent of Fig. 2, batched: every listed start
// is climbed by 1-bit flips, always taking the flip of largest gain (lowest
// index on ties) while the gain is positive.  Gains are the 1-flip move values
// of Glover et al. (2002) that the Pseudocode section cites,
//     Delta_j = Q_jj + 2 (1 - 2 x_j) y_j,   y = Q x,
// and flipping bit k (d = 1 - 2 x_k before the flip) changes them by
//     Delta_j += 2 (1 - 2 x_j) d Q_jk  (j != k),   Delta_k -> -Delta_k.
//
// Design.  A group of T threads owns one start at a time (one warp for
// n <= 512, else one block).  Thread g owns E = 16*C elements, in chunks of 16
// consecutive indices: element e lives at j = (e/16)*16T + 16g + e%16, so one
// move loads row k of the int8 Q (= column k, Q being symmetric) with C fully
// coalesced 16-byte loads per thread.  Per element the thread keeps in
// registers only the argmax key and two dp4a selectors:
//     key_j = 32 Delta_j + (31 - e)      (gain first, then lower index)
//     SP_j  = 64 (1 - 2 x_j) in the byte lane of j's coefficient, SN_j = -SP_j,
// so a move is, per element, key_j = dp4a(row word, SP_j or SN_j, key_j) and a
// running max: two instructions (the sign of d picks the selector set for the
// whole move).  The owner of k negates key_k (with the diagonal correction),
// swaps its selectors and flips its x bit.  Four independent running maxima
// keep the dependency chains short.  The group reduces (gain, 2j + x_j): a warp
// uses one redux.sync on a packed 32-bit (gain, warp-local index) key when the
// gain bound allows it (|Delta| < 2^21), else two; a block then combines its
// warps' records from shared memory with a small register tree.
//
// Start-up: y = Q x of every listed start comes from the tensor-core product of
// the ascent workspace when given (exact integers in fp32), else each group
// sums the rows k with x_k = 1 on the CUDA cores.  Rows are read from L2 (the
// int8 Q of one instance, e.g. 49 MB at n = 7000, stays resident there);
// nothing per move goes to HBM.
#include <climits>

#include "ubqp_internal.cuh"

namespace ubqp {
namespace {

constexpr int64_t kTimeoutNs = 20ll * 1000 * 1000 * 1000;  // per start

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Selector placing the signed byte v in lane i (for dp4a).
__device__ __forceinline__ int lane_sel(int i, int v) {
  return (int)((unsigned)(v & 0xFF) << (8 * i));
}

__device__ __forceinline__ int word_of(const uint4& q, int i) {
  return (int)(i == 0 ? q.x : i == 1 ? q.y : i == 2 ? q.z : q.w);
}

// Winner of a group reduction: the move's gain and 2k + x_k.
struct Win {
  int gain, jx;
};

__device__ __forceinline__ bool better(int2 a, int2 b) {
  return a.x > b.x || (a.x == b.x && a.y < b.y);
}

// Warp-level best from each thread's best key.  kt = 32 gain + (31 - e),
// e = the thread's local element, x = its x bit.  PACKED: one redux on
// gain * 1024 + (1023 - warp-local index); needs |gain| < 2^21.
template <int T, bool PACKED>
__device__ __forceinline__ int2 warp_best(int kt, int xbit, int g, int lane) {
  constexpr int CW = 16 * T;
  const int gain = kt >> 5;
  const int e = 31 - (kt & 31);
  const int wl = (e >> 4) * 512 + lane * 16 + (e & 15);  // order of j within the warp
  if (PACKED) {
    // a thread whose elements all lie beyond n carries the INT_MIN sentinel;
    // clamp it below every real gain so the packed product cannot overflow
    const int kw = max(gain, -(1 << 21)) * 1024 + (1023 - wl);
    const int m = __reduce_max_sync(0xffffffffu, kw);
    const int lw = 1023 - (m & 1023);
    const int lane_w = (lw >> 4) & 31;
    const int jw = (lw >> 9) * CW + 16 * (g - lane + lane_w) + (lw & 15);
    const int xw = __shfl_sync(0xffffffffu, xbit, lane_w);
    return make_int2(m >> 10, 2 * jw + xw);
  } else {
    const int j = (e >> 4) * CW + 16 * g + (e & 15);
    const int m = __reduce_max_sync(0xffffffffu, gain);
    const int c = __reduce_min_sync(0xffffffffu, gain == m ? 2 * j + xbit : INT_MAX);
    return make_int2(m, c);
  }
}

// One warp per start.
template <bool PACKED>
struct WarpGroup {
  static constexpr int T = 32;
  __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
  __device__ __forceinline__ Win reduce(int kt, int xbit) {
    const int g = rank();
    const int2 w = warp_best<32, PACKED>(kt, xbit, g, g);
    return Win{w.x, w.y};
  }
  __device__ __forceinline__ bool any(bool p) { return __any_sync(0xffffffffu, p); }
  __device__ __forceinline__ void sync() { __syncwarp(); }
};

// One block per start.
template <int TT, bool PACKED>
struct BlockGroup {
  static constexpr int T = TT;
  static constexpr int NW = TT / 32;
  int2 (*rec)[NW];  // [2][NW] shared: {gain, 2j + x}
  int parity;
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  __device__ __forceinline__ Win reduce(int kt, int xbit) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int2 w = warp_best<TT, PACKED>(kt, xbit, threadIdx.x, lane);
    if (lane == 0) rec[parity][warp] = w;
    __syncthreads();
    // every thread combines the NW records: a tree of pairwise bests
    int2 r[NW];
#pragma unroll
    for (int i = 0; i < NW; i += 2) {
      const int4 v = *reinterpret_cast<const int4*>(&rec[parity][i]);
      r[i] = make_int2(v.x, v.y);
      r[i + 1] = make_int2(v.z, v.w);
    }
#pragma unroll
    for (int step = 1; step < NW; step *= 2)
#pragma unroll
      for (int i = 0; i + step < NW; i += 2 * step)
        if (better(r[i + step], r[i])) r[i] = r[i + step];
    parity ^= 1;
    return Win{r[0].x, r[0].y};
  }
  __device__ __forceinline__ bool any(bool p) { return __syncthreads_or(p) != 0; }
  __device__ __forceinline__ void sync() { __syncthreads(); }
};

template <int C, class G>
__device__ __forceinline__ void ascend_one(const int8_t* __restrict__ Q8, int64_t ldq,
                                           int64_t ldy, int n, int W,
                                           uint64_t* __restrict__ x_g,
                                           int64_t* __restrict__ f_s, int32_t max_flips,
                                           int32_t* __restrict__ flips_s,
                                           unsigned* __restrict__ err, uint64_t* xs,
                                           const float* __restrict__ y_g, G& grp) {
  constexpr int T = G::T;
  constexpr int E = 16 * C;
  constexpr int CW = 16 * T;  // indices per chunk
  static_assert(E <= 32, "local index must fit 5 bits");
  const int g = grp.rank();

  // ---- owned bits of x
  uint32_t xm = 0;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int j0 = c * CW + 16 * g;
    if (j0 < n) {
      uint32_t nib = (uint32_t)((x_g[j0 >> 6] >> (j0 & 63)) & 0xFFFFull);
      if (n - j0 < 16) nib &= (1u << (n - j0)) - 1u;
      xm |= nib << (16 * c);
    }
  }
  // ---- y = Q x on the owned columns
  int key[E];
#pragma unroll
  for (int e = 0; e < E; ++e) key[e] = 0;  // holds y until the keys are formed
  if (y_g) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int j0 = c * CW + 16 * g;
      if (j0 < ldy) {
        const float4* src = reinterpret_cast<const float4*>(y_g + j0);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float4 t4 = src[v];
          key[c * 16 + 4 * v + 0] = __float2int_rn(t4.x);
          key[c * 16 + 4 * v + 1] = __float2int_rn(t4.y);
          key[c * 16 + 4 * v + 2] = __float2int_rn(t4.z);
          key[c * 16 + 4 * v + 3] = __float2int_rn(t4.w);
        }
      }
    }
  } else {
    for (int w = 0; w < W; ++w) {
      uint64_t word = x_g[w] & valid_mask(n, w);
      while (word) {
        constexpr int R = C == 1 ? 4 : 2;  // rows in flight
        int ks[R];
        int nk = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          ks[r] = 0;
          if (word) {
            ks[r] = w * 64 + __ffsll((long long)word) - 1;
            word &= word - 1;
            nk = r + 1;
          }
        }
        uint4 q[R][C];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const int j0 = c * CW + 16 * g;
            q[r][c] = (r < nk && j0 < ldq) ? __ldg(reinterpret_cast<const uint4*>(
                                                 Q8 + (int64_t)ks[r] * ldq + j0))
                                           : make_uint4(0, 0, 0, 0);
          }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < C; ++c)
#pragma unroll
            for (int o = 0; o < 16; ++o)
              key[c * 16 + o] =
                  __dp4a(word_of(q[r][c], o >> 2), lane_sel(o & 3, 1), key[c * 16 + o]);
      }
    }
  }
  // ---- keys and selectors; elements beyond n never win and never change
  int SP[E], SN[E];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int o = 0; o < 16; ++o) {
      const int e = c * 16 + o, j = c * CW + 16 * g + o;
      if (j < n) {
        const int s = ((xm >> e) & 1u) ? -1 : 1;
        const int qjj = Q8[(int64_t)j * ldq + j];
        key[e] = 32 * (qjj + 2 * s * key[e]) + (31 - e);
        SP[e] = lane_sel(o & 3, 64 * s);
        SN[e] = lane_sel(o & 3, -64 * s);
      } else {
        key[e] = INT_MIN;
        SP[e] = 0;
        SN[e] = 0;
      }
    }
  auto thread_best = [&]() {
    int km0 = INT_MIN, km1 = INT_MIN, km2 = INT_MIN, km3 = INT_MIN;
#pragma unroll
    for (int e = 0; e < E; e += 4) {
      km0 = max(km0, key[e]);
      km1 = max(km1, key[e + 1]);
      km2 = max(km2, key[e + 2]);
      km3 = max(km3, key[e + 3]);
    }
    return max(max(km0, km1), max(km2, km3));
  };
  auto reduce_keys = [&](int kt) {
    const int e = 31 - (kt & 31);
    return grp.reduce(kt, (int)((xm >> e) & 1u));
  };
  Win best = reduce_keys(thread_best());

  int64_t fval = *f_s;
  int flips = 0;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (max_flips > 0 && flips >= max_flips) break;
    if (best.gain <= 0) break;
    if ((flips & 1023) == 1023) {
      const bool late = (int64_t)(globaltimer() - t0) > kTimeoutNs;
      if (grp.any(late)) {
        if (g == 0) atomicOr(err, UBQP_DEVERR_TIMEOUT);
        break;
      }
    }
    const int k = best.jx >> 1;
    const bool dpos = (best.jx & 1) == 0;  // d = 1 - 2 x_k before the flip
    fval += best.gain;
    ++flips;
    const int8_t* row = Q8 + (int64_t)k * ldq;
    uint4 q[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int j0 = c * CW + 16 * g;
      q[c] = j0 < ldq ? __ldg(reinterpret_cast<const uint4*>(row + j0)) : make_uint4(0, 0, 0, 0);
    }
    // the owner of k flips x_k: key_k -> key of -Delta_k (pre-corrected for the
    // -64 Q_kk the generic update below adds with the new selectors), swap the
    // selectors, toggle the bit
    const int kc = k / CW, kr = k - kc * CW;
    if ((kr >> 4) == g) {
      const int ko = kr & 15, ek = kc * 16 + ko;
      int qw = 0;
#pragma unroll
      for (int c = 0; c < C; ++c)
        if (c == kc) qw = word_of(q[c], ko >> 2);
      const int qkk = (int)(int8_t)(qw >> (8 * (ko & 3)));
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e == ek) {
          key[e] = -key[e] + 2 * (31 - e) + 64 * qkk;
          const int t = SP[e];
          SP[e] = SN[e];
          SN[e] = t;
        }
      xm ^= 1u << ek;
    }
    if (dpos) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int o = 0; o < 16; ++o)
          key[c * 16 + o] = __dp4a(word_of(q[c], o >> 2), SP[c * 16 + o], key[c * 16 + o]);
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int o = 0; o < 16; ++o)
          key[c * 16 + o] = __dp4a(word_of(q[c], o >> 2), SN[c * 16 + o], key[c * 16 + o]);
    }
    best = reduce_keys(thread_best());
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
    const uint64_t bits = (xm >> (16 * c)) & 0xFFFFu;
    if (bits) atomicOr(reinterpret_cast<unsigned long long*>(&xs[j0 >> 6]),
                       (unsigned long long)(bits << (j0 & 63)));
  }
  grp.sync();
  for (int w = g; w < W; w += T) x_g[w] = xs[w];
  grp.sync();
}

template <int T, int C, bool PACKED>
__global__ void __launch_bounds__(T, 1)
ascent_block_kernel(const int8_t* __restrict__ Q8, int64_t ldq, int n, int W,
                    uint64_t* __restrict__ X, int64_t* __restrict__ f,
                    const int32_t* __restrict__ idx, const int64_t* __restrict__ count,
                    int64_t S, int32_t max_flips, int32_t* __restrict__ flips,
                    const float* __restrict__ Y, int64_t ldy, unsigned* __restrict__ err) {
  __shared__ __align__(16) int2 rec[2][T / 32];
  __shared__ uint64_t xs[UBQP_MAX_N / 64];
  BlockGroup<T, PACKED> grp{rec, 0};
  const int64_t cnt = *count;
  for (int64_t t = blockIdx.x; t < cnt; t += gridDim.x) {
    const int s = idx[t];
    if (s < 0 || s >= S) {
      if (threadIdx.x == 0) atomicOr(err, UBQP_DEVERR_BADIDX);
      continue;
    }
    ascend_one<C>(Q8, ldq, ldy, n, W, X + (int64_t)s * W, f + s, max_flips,
                  flips ? flips + s : nullptr, err, xs, Y ? Y + t * ldy : nullptr, grp);
  }
}

// Four independent warps per block, one start each (n <= 512).
template <int C, bool PACKED>
__global__ void __launch_bounds__(128)
ascent_warp_kernel(const int8_t* __restrict__ Q8, int64_t ldq, int n, int W,
                   uint64_t* __restrict__ X, int64_t* __restrict__ f,
                   const int32_t* __restrict__ idx, const int64_t* __restrict__ count,
                   int64_t S, int32_t max_flips, int32_t* __restrict__ flips,
                   const float* __restrict__ Y, int64_t ldy, unsigned* __restrict__ err) {
  __shared__ uint64_t xs_all[4][16];
  WarpGroup<PACKED> grp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t cnt = *count;
  for (int64_t t = (int64_t)blockIdx.x * 4 + warp; t < cnt; t += (int64_t)gridDim.x * 4) {
    const int s = idx[t];
    if (s < 0 || s >= S) {
      if (lane == 0) atomicOr(err, UBQP_DEVERR_BADIDX);
      continue;
    }
    ascend_one<C>(Q8, ldq, ldy, n, W, X + (int64_t)s * W, f + s, max_flips,
                  flips ? flips + s : nullptr, err, xs_all[warp], Y ? Y + t * ldy : nullptr,
                  grp);
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

struct Args {
  const ubqp_q* h;
  uint64_t* X;
  int64_t* f;
  const int32_t* idx;
  const int64_t* count;
  int64_t S;
  int32_t max_flips;
  int32_t* flips;
  const float* Y;
  cudaStream_t st;
};

template <int T, int C, bool PACKED>
cudaError_t launch_block(const Args& a) {
  auto kern = ascent_block_kernel<T, C, PACKED>;
  int grid = resident_grid(kern, T, a.h->sm_count);
  if ((int64_t)grid > a.S) grid = (int)a.S;
  kern<<<grid, T, 0, a.st>>>(a.h->Q8, a.h->ldq, a.h->n, a.h->W, a.X, a.f, a.idx, a.count, a.S,
                             a.max_flips, a.flips, a.Y, a.h->n_tc, a.h->err);
  return cudaGetLastError();
}

template <int C, bool PACKED>
cudaError_t launch_warp(const Args& a) {
  auto kern = ascent_warp_kernel<C, PACKED>;
  int grid = resident_grid(kern, 128, a.h->sm_count);
  const int64_t need = (a.S + 3) / 4;
  if ((int64_t)grid > need) grid = (int)need;
  kern<<<grid, 128, 0, a.st>>>(a.h->Q8, a.h->ldq, a.h->n, a.h->W, a.X, a.f, a.idx, a.count,
                               a.S, a.max_flips, a.flips, a.Y, a.h->n_tc, a.h->err);
  return cudaGetLastError();
}

template <bool PACKED>
cudaError_t launch_sized(const Args& a) {
  const int n = a.h->n;
  if (n <= 256) return launch_warp<1, PACKED>(a);
  if (n <= 512) return launch_warp<2, PACKED>(a);
  if (n <= 1024) return launch_block<64, 1, PACKED>(a);
  if (n <= 2048) return launch_block<128, 1, PACKED>(a);
  if (n <= 4096) return launch_block<256, 1, PACKED>(a);
  if (n <= 8192) return launch_block<256, 2, PACKED>(a);
  if (n <= 16384) return launch_block<512, 2, PACKED>(a);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_ascent(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                          const int64_t* count, int64_t S, int32_t max_flips, int32_t* flips,
                          const float* Y, cudaStream_t st) {
  const Args a{h, X, f, idx, count, S, max_flips, flips, Y, st};
  // |Delta_j| <= |Q_jj| + 2 sum_k |Q_jk| <= max|Q| (2n + 1): the packed key
  // holds gains below 2^21 in magnitude
  const int64_t bound = (int64_t)h->max_abs * (2 * (int64_t)h->n + 1);
  return bound < (1 << 21) ? launch_sized<true>(a) : launch_sized<false>(a);
}

}  // namespace ubqp
