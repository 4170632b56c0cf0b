// k_ascent.cu -- PerformSteepestAscent of Fig. 2, batched: every listed start
// is climbed by 1-bit flips, always taking the flip of largest gain (lowest
// index on ties) while the gain is positive.  Gains follow the 1-flip move
// values of Glover et al. (2002) that the Pseudocode section cites:
//     Delta_i = Q_ii + 2 (1 - 2 x_i) y_i,  y = Q x,
//     after flipping k (d = 1 - 2 x_k):  Delta_j += 2 (1 - 2 x_j) d Q_jk (j != k),
//                                        Delta_k  = -Delta_k.
//
// Design: a group of G threads owns one start at a time (G = 32: one warp, for
// n <= 512; G = 256: one block).  Thread g of the group owns the 4*C elements
// j = c*4G + 4g + e (c < C, e < 4) and keeps their gains in registers, so a
// move streams one int8 row of Q (row k = column k, Q being symmetric) with
// fully coalesced 4-byte loads, updates the gains and finds the next argmax in
// the same pass.  The argmax key packs (gain, lowest index, x bit) into one
// int64 so that a single max-reduction decides the move and tells every thread
// the bit it flips.  Rows are read from L2 (the int8 Q of one instance, e.g.
// 49 MB at n = 7000, stays resident there); nothing per move goes to HBM.
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

__device__ __forceinline__ int sbyte(int w, int e) { return (int)(int8_t)(w >> (8 * e)); }

__device__ __forceinline__ long long make_key(int gain, int j, int xbit) {
  const unsigned low = ((unsigned)(0x7FFFFFFF - j) << 1) | (unsigned)xbit;
  return (long long)gain * 4294967296LL + (long long)low;
}

// Max-reduction of a key over the group.
template <int G>
struct GroupReduce;

template <>
struct GroupReduce<32> {
  __device__ __forceinline__ long long max(long long k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      long long v = __shfl_xor_sync(0xffffffffu, k, o);
      k = v > k ? v : k;
    }
    return k;
  }
  __device__ __forceinline__ bool any(bool p) { return __any_sync(0xffffffffu, p); }
  __device__ __forceinline__ void sync() { __syncwarp(); }
};

template <>
struct GroupReduce<256> {
  static constexpr int NW = 8;
  long long (*buf)[NW];  // [2][NW] in shared memory
  int parity;
  __device__ __forceinline__ long long max(long long k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      long long v = __shfl_xor_sync(0xffffffffu, k, o);
      k = v > k ? v : k;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) buf[parity][warp] = k;
    __syncthreads();
    k = lane < NW ? buf[parity][lane] : LLONG_MIN;
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) {
      long long v = __shfl_xor_sync(0xffffffffu, k, o);
      k = v > k ? v : k;
    }
    k = __shfl_sync(0xffffffffu, k, 0);
    parity ^= 1;
    return k;
  }
  __device__ __forceinline__ bool any(bool p) { return __syncthreads_or(p) != 0; }
  __device__ __forceinline__ void sync() { __syncthreads(); }
};

// Ascent of one start by a group of G threads; g = rank in the group.
template <int G, int C>
__device__ __forceinline__ void ascend_one(const int8_t* __restrict__ Q8, int64_t ldq, int n,
                                           int W, uint64_t* __restrict__ x_g,
                                           int64_t* __restrict__ f_s, int32_t max_flips,
                                           int32_t* __restrict__ flips_s,
                                           unsigned* __restrict__ err, uint64_t* xs,
                                           GroupReduce<G>& red, int g) {
  static_assert(4 * C <= 64, "bit mask holds 64 elements per thread");
  // ---- owned bits of x
  uint64_t bits = 0;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int j0 = c * 4 * G + 4 * g;
    if (j0 < n) {
      uint64_t nib = (x_g[j0 >> 6] >> (j0 & 63)) & 0xFull;
      const int valid = n - j0;
      if (valid < 4) nib &= (1ull << valid) - 1ull;
      bits |= nib << (4 * c);
    }
  }
  // ---- y = Q x over the owned columns: sum the rows k with x_k = 1
  int D[C][4];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) D[c][e] = 0;
  for (int w = 0; w < W; ++w) {
    uint64_t word = x_g[w] & valid_mask(n, w);
    while (word) {
      // up to R rows in flight
      constexpr int R = C <= 4 ? 4 : (C <= 8 ? 2 : 1);
      int ks[R];
      int nk = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (word) {
          ks[r] = w * 64 + __ffsll((long long)word) - 1;
          word &= word - 1;
          nk = r + 1;
        } else {
          ks[r] = -1;
        }
      }
      int q[R][C];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int j0 = c * 4 * G + 4 * g;
          q[r][c] = (r < nk && j0 < ldq)
                        ? __ldg(reinterpret_cast<const int*>(Q8 + (int64_t)ks[r] * ldq + j0))
                        : 0;
        }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
          for (int e = 0; e < 4; ++e) D[c][e] += sbyte(q[r][c], e);
    }
  }
  // ---- gains; elements beyond n get a sentinel that never wins
  int bv = INT_MIN, bi = 0;
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = c * 4 * G + 4 * g + e;
      if (j < n) {
        const int qjj = Q8[(int64_t)j * ldq + j];
        const int s = ((bits >> (4 * c + e)) & 1ull) ? -1 : 1;
        D[c][e] = qjj + 2 * s * D[c][e];
      } else {
        D[c][e] = INT_MIN;
      }
      if (D[c][e] > bv) { bv = D[c][e]; bi = 4 * c + e; }
    }
  long long key = red.max(make_key(bv, (bi >> 2) * 4 * G + 4 * g + (bi & 3),
                                   (int)((bits >> bi) & 1ull)));
  int64_t fval = *f_s;
  int flips = 0;
  const uint64_t t0 = globaltimer();
  for (;;) {
    const long long dk = key >> 32;
    if (max_flips > 0 && flips >= max_flips) break;
    if (dk <= 0) break;
    if ((flips & 1023) == 1023) {
      const bool late = (int64_t)(globaltimer() - t0) > kTimeoutNs;
      if (red.any(late)) {
        if (g == 0) atomicOr(err, UBQP_DEVERR_TIMEOUT);
        break;
      }
    }
    const unsigned low = (unsigned)(key & 0xFFFFFFFFll);
    const int k = 0x7FFFFFFF - (int)(low >> 1);
    const int d2 = (low & 1u) ? -2 : 2;  // 2 d, d = 1 - 2 x_k (before the flip)
    fval += dk;
    ++flips;
    const int8_t* row = Q8 + (int64_t)k * ldq;
    int q[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int j0 = c * 4 * G + 4 * g;
      q[c] = j0 < ldq ? __ldg(reinterpret_cast<const int*>(row + j0)) : 0;
    }
    const int kc = k / (4 * G);
    const int kr = k - kc * 4 * G;
    const int kc_mine = ((kr >> 2) == g) ? kc : -1;
    const int ke = kr & 3;
    bv = INT_MIN;
    bi = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      if (c == kc_mine) {
        // the owner of k: Delta_k -> -Delta_k, taking into account the generic
        // update below, which sees the new bit and adds -2 Q_kk
        const int qkk = sbyte(q[c], ke);
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (e == ke) D[c][e] = -D[c][e] + 2 * qkk;
        bits ^= 1ull << (4 * c + ke);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = ((bits >> (4 * c + e)) & 1ull) ? -d2 : d2;
        D[c][e] += m * sbyte(q[c], e);
        if (D[c][e] > bv) { bv = D[c][e]; bi = 4 * c + e; }
      }
    }
    key = red.max(make_key(bv, (bi >> 2) * 4 * G + 4 * g + (bi & 3),
                           (int)((bits >> bi) & 1ull)));
  }
  // ---- write back f, flips and x
  if (g == 0) {
    *f_s = fval;
    if (flips_s) *flips_s = flips;
  }
  for (int w = g; w < W; w += G) xs[w] = 0;
  red.sync();
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int j0 = c * 4 * G + 4 * g;
    const uint64_t nib = (bits >> (4 * c)) & 0xFull;
    if (nib) atomicOr(reinterpret_cast<unsigned long long*>(&xs[j0 >> 6]),
                      (unsigned long long)(nib << (j0 & 63)));
  }
  red.sync();
  for (int w = g; w < W; w += G) x_g[w] = xs[w];
  red.sync();
}

template <int C>
__global__ void __launch_bounds__(256)
ascent_block_kernel(const int8_t* __restrict__ Q8, int64_t ldq, int n, int W,
                    uint64_t* __restrict__ X, int64_t* __restrict__ f,
                    const int32_t* __restrict__ idx, const int64_t* __restrict__ count,
                    int64_t S, int32_t max_flips, int32_t* __restrict__ flips,
                    unsigned* __restrict__ err) {
  __shared__ long long red_buf[2][8];
  __shared__ uint64_t xs[UBQP_MAX_N / 64];
  GroupReduce<256> red{red_buf, 0};
  const int64_t cnt = *count;
  for (int64_t t = blockIdx.x; t < cnt; t += gridDim.x) {
    const int s = idx[t];
    if (s < 0 || s >= S) {
      if (threadIdx.x == 0) atomicOr(err, UBQP_DEVERR_BADIDX);
      continue;
    }
    ascend_one<256, C>(Q8, ldq, n, W, X + (int64_t)s * W, f + s, max_flips,
                       flips ? flips + s : nullptr, err, xs, red, threadIdx.x);
  }
}

template <int C>
__global__ void __launch_bounds__(128)
ascent_warp_kernel(const int8_t* __restrict__ Q8, int64_t ldq, int n, int W,
                   uint64_t* __restrict__ X, int64_t* __restrict__ f,
                   const int32_t* __restrict__ idx, const int64_t* __restrict__ count,
                   int64_t S, int32_t max_flips, int32_t* __restrict__ flips,
                   unsigned* __restrict__ err) {
  __shared__ uint64_t xs_all[4][8];
  GroupReduce<32> red;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t cnt = *count;
  for (int64_t t = (int64_t)blockIdx.x * 4 + warp; t < cnt; t += (int64_t)gridDim.x * 4) {
    const int s = idx[t];
    if (s < 0 || s >= S) {
      if (lane == 0) atomicOr(err, UBQP_DEVERR_BADIDX);
      continue;
    }
    ascend_one<32, C>(Q8, ldq, n, W, X + (int64_t)s * W, f + s, max_flips,
                      flips ? flips + s : nullptr, err, xs_all[warp], red, lane);
  }
}

template <class K>
int resident_grid(K kernel, int threads, int sm_count) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * sm_count;
}

template <int C>
cudaError_t launch_block(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                         const int64_t* count, int64_t S, int32_t max_flips, int32_t* flips,
                         cudaStream_t st) {
  int grid = resident_grid(ascent_block_kernel<C>, 256, h->sm_count);
  if ((int64_t)grid > S) grid = (int)S;
  ascent_block_kernel<C><<<grid, 256, 0, st>>>(h->Q8, h->ldq, h->n, h->W, X, f, idx, count,
                                               S, max_flips, flips, h->err);
  return cudaGetLastError();
}

template <int C>
cudaError_t launch_warp(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                        const int64_t* count, int64_t S, int32_t max_flips, int32_t* flips,
                        cudaStream_t st) {
  int grid = resident_grid(ascent_warp_kernel<C>, 128, h->sm_count);
  int64_t need = (S + 3) / 4;
  if ((int64_t)grid > need) grid = (int)need;
  ascent_warp_kernel<C><<<grid, 128, 0, st>>>(h->Q8, h->ldq, h->n, h->W, X, f, idx, count, S,
                                              max_flips, flips, h->err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ascent(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                          const int64_t* count, int64_t S, int32_t max_flips, int32_t* flips,
                          cudaStream_t st) {
  const int n = h->n;
  if (n <= 512) {
    switch ((n + 127) / 128) {
      case 1: return launch_warp<1>(h, X, f, idx, count, S, max_flips, flips, st);
      case 2: return launch_warp<2>(h, X, f, idx, count, S, max_flips, flips, st);
      case 3: return launch_warp<3>(h, X, f, idx, count, S, max_flips, flips, st);
      default: return launch_warp<4>(h, X, f, idx, count, S, max_flips, flips, st);
    }
  }
#define UBQP_BLOCK_CASE(CC) \
  case CC: return launch_block<CC>(h, X, f, idx, count, S, max_flips, flips, st);
  switch ((n + 1023) / 1024) {
    UBQP_BLOCK_CASE(1)
    UBQP_BLOCK_CASE(2)
    UBQP_BLOCK_CASE(3)
    UBQP_BLOCK_CASE(4)
    UBQP_BLOCK_CASE(5)
    UBQP_BLOCK_CASE(6)
    UBQP_BLOCK_CASE(7)
    UBQP_BLOCK_CASE(8)
    UBQP_BLOCK_CASE(9)
    UBQP_BLOCK_CASE(10)
    UBQP_BLOCK_CASE(11)
    UBQP_BLOCK_CASE(12)
    UBQP_BLOCK_CASE(13)
    UBQP_BLOCK_CASE(14)
    UBQP_BLOCK_CASE(15)
    UBQP_BLOCK_CASE(16)
    default: return cudaErrorInvalidValue;
  }
#undef UBQP_BLOCK_CASE
}

}  // namespace ubqp
