// k_best.cu -- UpdateBestAndT's bookkeeping (Fig. 2): the best of a batch of
// objective values, lowest start index on ties, and a copy of its solution;
// plus the per-round statistics that ubqp_solve reports.
#include <climits>

#include "ubqp_internal.cuh"

namespace ubqp {
namespace {

constexpr int THREADS = 1024;
constexpr int WARPS = THREADS / 32;

__device__ void block_best(const int64_t* __restrict__ f, const uint64_t* __restrict__ X,
                           int64_t S, int W, uint64_t* __restrict__ best_x,
                           int64_t* __restrict__ best_f) {
  __shared__ long long s_max[WARPS], s_arg[WARPS];
  __shared__ long long s_best;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long mx = LLONG_MIN, am = LLONG_MAX;
  for (int64_t b = threadIdx.x; b < S; b += THREADS) {
    long long v = f[b];
    if (v > mx) { mx = v; am = b; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long om = __shfl_xor_sync(0xffffffffu, mx, o);
    long long oa = __shfl_xor_sync(0xffffffffu, am, o);
    if (om > mx || (om == mx && oa < am)) { mx = om; am = oa; }
  }
  if (lane == 0) { s_max[warp] = mx; s_arg[warp] = am; }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = LLONG_MIN, a = LLONG_MAX;
    for (int i = 0; i < WARPS; ++i)
      if (s_max[i] > m || (s_max[i] == m && s_arg[i] < a)) { m = s_max[i]; a = s_arg[i]; }
    best_f[0] = m;
    best_f[1] = a;
    s_best = a;
  }
  __syncthreads();
  const long long a = s_best;
  for (int w = threadIdx.x; w < W; w += THREADS) best_x[w] = X[a * W + w];
}

// A programmatic dependent of the kernel before it (pdl_enter).
__global__ void __launch_bounds__(THREADS)
best_kernel(const int64_t* __restrict__ f, const uint64_t* __restrict__ X, int64_t S, int W,
            uint64_t* __restrict__ best_x, int64_t* __restrict__ best_f) {
  pdl_enter();
  block_best(f, X, S, W, best_x, best_f);
}

// One block per instance of a batch.
__global__ void __launch_bounds__(THREADS) best_batch_kernel(const BatchDesc* __restrict__ d) {
  const BatchDesc& b = d[blockIdx.x];
  block_best(b.f, b.X, b.S, b.W, b.best_x, b.best_f);
}

// The batch's ascent work list: (instance, position in its passing list) for
// every passing start, instances in the given order (largest first).
// The instances order[k0 .. k0 + m) (m <= THREADS) of a batch's lists: each
// thread reads one instance's passing count (and, for the packed list, its
// unit class), then one thread turns them into exclusive offsets in shared
// memory, so that no global load waits inside the loop over instances.  With
// skip0 the instances of class 0 (climbed by launches of their own) add no
// items.
struct ListChunk {
  int inst[THREADS];
  int cls[THREADS];
  long long cnt[THREADS], base[THREADS], ubase[THREADS];
  long long base_end, ubase_end;
};
__device__ void list_chunk(const BatchDesc* __restrict__ d, const int32_t* __restrict__ order,
                           int k0, int m, int T, int C, bool packed, bool skip0, ListChunk& L) {
  if ((int)threadIdx.x < m) {
    const int i = order[k0 + (int)threadIdx.x];
    const int n = d[i].n;
    L.inst[threadIdx.x] = i;
    L.cnt[threadIdx.x] = *d[i].count;
    L.cls[threadIdx.x] = !packed                 ? 0
                         : n <= 16 * (T >> 3) * C ? 3
                         : n <= 16 * (T >> 2) * C ? 2
                         : n <= 16 * (T >> 1) * C ? 1
                                                  : 0;
    if (skip0 && L.cls[threadIdx.x] == 0) L.cnt[threadIdx.x] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long b = L.base_end, ub = L.ubase_end;
    for (int j = 0; j < m; ++j) {
      L.base[j] = b;
      L.ubase[j] = ub;
      const long long per = 1ll << L.cls[j];
      b += L.cnt[j];
      ub += (L.cnt[j] + per - 1) / per;
    }
    L.base_end = b;
    L.ubase_end = ub;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(THREADS)
batch_items_kernel(const BatchDesc* __restrict__ d, const int32_t* __restrict__ order, int count,
                   int2* __restrict__ items, int64_t* __restrict__ n_items) {
  __shared__ ListChunk L;
  if (threadIdx.x == 0) L.base_end = L.ubase_end = 0;
  for (int k0 = 0; k0 < count; k0 += THREADS) {
    const int m = count - k0 < THREADS ? count - k0 : THREADS;
    list_chunk(d, order, k0, m, 0, 0, false, false, L);
    for (int j = 0; j < m; ++j)
      for (long long t = threadIdx.x; t < L.cnt[j]; t += THREADS)
        items[L.base[j] + t] = make_int2(L.inst[j], (int)t);
    __syncthreads();  // L is rewritten by the next chunk
  }
  if (threadIdx.x == 0) *n_items = L.base_end;
}

// The work list of the packed batch ascent: the items as batch_items_kernel
// writes them, and the range {first item, items, 0, 0} of each class c = 0 ..
// 3, an instance being of the largest class whose sub-group of T >> c threads
// (16 (T >> c) C elements) holds its n.  Instances come largest first, so
// each class's items are contiguous.  With skip0 class 0 is left out (its
// instances climb in launches of their own).
__global__ void __launch_bounds__(THREADS)
batch_units_kernel(const BatchDesc* __restrict__ d, const int32_t* __restrict__ order, int count,
                   int T, int C, int skip0, int2* __restrict__ items, int4* __restrict__ ranges,
                   int64_t* __restrict__ n_items) {
  __shared__ ListChunk L;
  __shared__ long long cbeg[4], ccnt[4];
  if (threadIdx.x == 0) {
    L.base_end = L.ubase_end = 0;
    for (int c = 0; c < 4; ++c) cbeg[c] = -1, ccnt[c] = 0;
  }
  for (int k0 = 0; k0 < count; k0 += THREADS) {
    const int m = count - k0 < THREADS ? count - k0 : THREADS;
    list_chunk(d, order, k0, m, T, C, true, skip0 != 0, L);
    if (threadIdx.x == 0)
      for (int j = 0; j < m; ++j) {
        const int c = L.cls[j];
        if (cbeg[c] < 0) cbeg[c] = L.base[j];
        ccnt[c] += L.cnt[j];
      }
    for (int j = 0; j < m; ++j)
      for (long long t = threadIdx.x; t < L.cnt[j]; t += THREADS)
        items[L.base[j] + t] = make_int2(L.inst[j], (int)t);
    __syncthreads();  // L is rewritten by the next chunk
  }
  if (threadIdx.x == 0) {
    for (int c = 0; c < 4; ++c)
      ranges[c] = make_int4(cbeg[c] < 0 ? 0 : (int)cbeg[c], (int)ccnt[c], 0, 0);
    *n_items = L.base_end;
  }
}

// The passing starts of R rounds held back to back (round r's S values at
// r*S, its passing list at idx[r*S], its count at counts[r]) as one list of
// global start indices r*S + idx, and its length.  R <= 1024.
__global__ void __launch_bounds__(THREADS)
concat_rounds_kernel(const int32_t* __restrict__ idx, const int64_t* __restrict__ counts, int R,
                     int64_t S, int32_t* __restrict__ idx_all, int64_t* __restrict__ count_all) {
  __shared__ int64_t off[1025];
  if (threadIdx.x == 0) {
    int64_t o = 0;
    for (int r = 0; r < R; ++r) {
      off[r] = o;
      const int64_t c = counts[r];
      o += c < 0 ? 0 : (c > S ? S : c);
    }
    off[R] = o;
    *count_all = o;
  }
  __syncthreads();
  for (int r = 0; r < R; ++r) {
    const int64_t c = off[r + 1] - off[r];
    for (int64_t t = threadIdx.x; t < c; t += THREADS)
      idx_all[off[r] + t] = (int32_t)(r * S + idx[r * S + t]);
  }
}

// The round's statistics {passed, total flips, max flips of one start, batch
// max, best index, sum} from the passing list, the flip counts, the screen's
// statistics and the best-of; one block.
__device__ void block_solve_stats(const int64_t* __restrict__ count,
                                  const int32_t* __restrict__ idx,
                                  const int32_t* __restrict__ flips,
                                  const int64_t* __restrict__ sstats,
                                  const int64_t* __restrict__ best, int64_t* __restrict__ out) {
  __shared__ long long s_tot[WARPS], s_mx[WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c = *count;
  long long tot = 0, mx = 0;
  for (int64_t t = threadIdx.x; t < c; t += THREADS) {
    long long v = flips[idx[t]];
    tot += v;
    mx = v > mx ? v : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    long long v = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  if (lane == 0) { s_tot[warp] = tot; s_mx[warp] = mx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0, m = 0;
    for (int i = 0; i < WARPS; ++i) {
      t += s_tot[i];
      m = s_mx[i] > m ? s_mx[i] : m;
    }
    out[0] = c;
    out[1] = t;
    out[2] = m;
    out[3] = sstats[1];
    out[4] = best[1];
    out[5] = sstats[0];
  }
}

__global__ void __launch_bounds__(THREADS)
solve_stats_kernel(const int64_t* __restrict__ count, const int32_t* __restrict__ idx,
                   const int32_t* __restrict__ flips, const int64_t* __restrict__ sstats,
                   const int64_t* __restrict__ best, int64_t* __restrict__ out) {
  block_solve_stats(count, idx, flips, sstats, best, out);
}

// The best-of, then the statistics (the best-of's value and index written by
// this block before its barrier are what they read); a programmatic
// dependent of the ascent.
__global__ void __launch_bounds__(THREADS)
best_stats_kernel(const int64_t* __restrict__ f, const uint64_t* __restrict__ X, int64_t S, int W,
                  uint64_t* __restrict__ best_x, int64_t* __restrict__ best_f,
                  const int64_t* __restrict__ count, const int32_t* __restrict__ idx,
                  const int32_t* __restrict__ flips, const int64_t* __restrict__ sstats,
                  int64_t* __restrict__ out) {
  pdl_enter();
  block_best(f, X, S, W, best_x, best_f);
  __syncthreads();
  block_solve_stats(count, idx, flips, sstats, best_f, out);
}

// UpdateBestAndT of Fig. 2 after a round: the round's best {value, index}
// (block_best into cand_x / cand) replaces the incumbent when strictly better;
// history[round] = incumbent value; stats {passed, flips} accumulate the
// round's counts.  One launch, a programmatic dependent of the ascent.
__global__ void __launch_bounds__(THREADS)
search_update_kernel(const int64_t* __restrict__ f, const uint64_t* __restrict__ X, int64_t S,
                     int W, uint64_t* __restrict__ cand_x, int64_t* __restrict__ cand,
                     const int64_t* __restrict__ count, const int32_t* __restrict__ idx,
                     const int32_t* __restrict__ flips, int64_t* __restrict__ inc_f,
                     uint64_t* __restrict__ inc_x, int64_t* __restrict__ history,
                     int64_t* __restrict__ stats) {
  __shared__ long long s_tot[WARPS];
  __shared__ int s_take;
  pdl_enter();
  block_best(f, X, S, W, cand_x, cand);
  __syncthreads();  // cand, written by thread 0, is read below
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c = *count;
  long long tot = 0;
  for (int64_t t = threadIdx.x; t < c; t += THREADS) tot += flips[idx[t]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  if (lane == 0) s_tot[warp] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < WARPS; ++i) t += s_tot[i];
    stats[0] += c;
    stats[1] += t;
    s_take = cand[0] > inc_f[0];
    if (s_take) inc_f[0] = cand[0];
    *history = inc_f[0];
  }
  __syncthreads();
  if (s_take)
    for (int w = threadIdx.x; w < W; w += THREADS) inc_x[w] = X[cand[1] * W + w];
}

__global__ void set_u64_kernel(uint64_t* dst, uint64_t v) { *dst = v; }

}  // namespace

cudaError_t launch_search_update(const int64_t* f, const uint64_t* X, int64_t S, int W,
                                 uint64_t* cand_x, int64_t* cand, const int64_t* count,
                                 const int32_t* idx, const int32_t* flips, int64_t* inc_f,
                                 uint64_t* inc_x, int64_t* history, int64_t* stats,
                                 cudaStream_t st) {
  return launch_pdl(search_update_kernel, dim3(1), dim3(THREADS), 0, st, f, X, S, W, cand_x, cand,
                    count, idx, flips, inc_f, inc_x, history, stats);
}

cudaError_t launch_set_u64(uint64_t* dst, uint64_t v, cudaStream_t st) {
  set_u64_kernel<<<1, 1, 0, st>>>(dst, v);
  return cudaGetLastError();
}

cudaError_t launch_best_batch(const BatchDesc* d, int count, cudaStream_t st) {
  best_batch_kernel<<<count, THREADS, 0, st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_batch_items(const BatchDesc* d, const int32_t* order, int count, int2* items,
                               int64_t* n_items, cudaStream_t st) {
  batch_items_kernel<<<1, THREADS, 0, st>>>(d, order, count, items, n_items);
  return cudaGetLastError();
}

cudaError_t launch_batch_units(const BatchDesc* d, const int32_t* order, int count, int T, int C,
                               bool skip0, int2* items, int4* ranges, int64_t* n_items,
                               cudaStream_t st) {
  batch_units_kernel<<<1, THREADS, 0, st>>>(d, order, count, T, C, skip0 ? 1 : 0, items, ranges,
                                            n_items);
  return cudaGetLastError();
}

cudaError_t launch_concat_rounds(const int32_t* idx, const int64_t* counts, int R, int64_t S,
                                 int32_t* idx_all, int64_t* count_all, cudaStream_t st) {
  concat_rounds_kernel<<<1, THREADS, 0, st>>>(idx, counts, R, S, idx_all, count_all);
  return cudaGetLastError();
}

cudaError_t launch_best(const int64_t* f, const uint64_t* X, int64_t S, int W,
                        uint64_t* best_x, int64_t* best_f, cudaStream_t st) {
  return launch_pdl(best_kernel, dim3(1), dim3(THREADS), 0, st, f, X, S, W, best_x, best_f);
}

cudaError_t launch_best_stats(const int64_t* f, const uint64_t* X, int64_t S, int W,
                              uint64_t* best_x, int64_t* best_f, const int64_t* count,
                              const int32_t* idx, const int32_t* flips, const int64_t* sstats,
                              int64_t* out, cudaStream_t st) {
  return launch_pdl(best_stats_kernel, dim3(1), dim3(THREADS), 0, st, f, X, S, W, best_x, best_f,
                    count, idx, flips, sstats, out);
}

cudaError_t launch_solve_stats(const int64_t* count, const int32_t* idx, const int32_t* flips,
                               const double* /*Tm*/, const int64_t* sstats,
                               const int64_t* best, int64_t* out, cudaStream_t st) {
  solve_stats_kernel<<<1, THREADS, 0, st>>>(count, idx, flips, sstats, best, out);
  return cudaGetLastError();
}

}  // namespace ubqp
