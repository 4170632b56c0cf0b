// k_screen.cu -- the screen of the Pseudocode section: T(lambda) = Mean +
// lambda (Max - Mean) over the batch, then the stable list of indices with
// f_b > T (Fig. 2).  Two single-block kernels: the statistics (an exact int64
// sum and a max with its lowest index, by warp shuffles), and the threshold in
// double with explicitly rounded operations (no FMA) followed by a block-wide
// ballot/prefix-sum compaction.  One launch runs both for a whole batch; the
// split launches let a batch sharded over ranks combine the statistics before
// the threshold.
#include <climits>

#include "ubqp_internal.cuh"

namespace ubqp {
namespace {

constexpr int THREADS = 1024;
constexpr int WARPS = THREADS / 32;

// stats = {sum of f, max f, lowest index attaining it + offset}; one block.
__device__ void block_screen_stats(const int64_t* __restrict__ f, int64_t S, int64_t offset,
                                   int64_t* __restrict__ stats) {
  __shared__ long long s_sum[WARPS];
  __shared__ long long s_max[WARPS];
  __shared__ long long s_arg[WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long sum = 0, mx = LLONG_MIN, am = LLONG_MAX;
  for (int64_t b = threadIdx.x; b < S; b += THREADS) {
    long long v = f[b];
    sum += v;
    if (v > mx) { mx = v; am = b; }  // increasing b per thread: keeps lowest
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    long long om = __shfl_xor_sync(0xffffffffu, mx, o);
    long long oa = __shfl_xor_sync(0xffffffffu, am, o);
    if (om > mx || (om == mx && oa < am)) { mx = om; am = oa; }
  }
  if (lane == 0) { s_sum[warp] = sum; s_max[warp] = mx; s_arg[warp] = am; }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0, m = LLONG_MIN, a = LLONG_MAX;
    for (int i = 0; i < WARPS; ++i) {
      t += s_sum[i];
      if (s_max[i] > m || (s_max[i] == m && s_arg[i] < a)) { m = s_max[i]; a = s_arg[i]; }
    }
    stats[0] = t;
    stats[1] = m;
    stats[2] = (S > 0) ? a + offset : LLONG_MAX;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(THREADS)
screen_stats_kernel(const int64_t* __restrict__ f, int64_t S, int64_t offset,
                    int64_t* __restrict__ stats) {
  block_screen_stats(f, S, offset, stats);
}

// T from the (possibly multi-rank) stats, then the stable list of local
// indices with f_b > T.
__device__ void block_screen_apply(const int64_t* __restrict__ f, int64_t S,
                                   const int64_t* gstats, int64_t S_total, double lambda,
                                   int32_t* __restrict__ idx, int64_t* __restrict__ count,
                                   double* __restrict__ Tm, const int64_t* gmax = nullptr) {
  __shared__ int s_cnt[WARPS];
  __shared__ double s_T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    const double mean = __ddiv_rn(__ll2double_rn(gstats[0]), __ll2double_rn(S_total));
    const double diff = __dsub_rn(__ll2double_rn(gmax ? gmax[0] : gstats[1]), mean);
    const double scaled = __dmul_rn(lambda, diff);
    const double T = __dadd_rn(mean, scaled);
    s_T = T;
    Tm[0] = T;
    Tm[1] = mean;
  }
  __syncthreads();
  const double T = s_T;
  int64_t base = 0;
  for (int64_t b0 = 0; b0 < S; b0 += THREADS) {
    const int64_t b = b0 + threadIdx.x;
    const bool pass = b < S && __ll2double_rn(f[b]) > T;
    const unsigned bal = __ballot_sync(0xffffffffu, pass);
    if (lane == 0) s_cnt[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int i = 0; i < WARPS; ++i) {
      int c = s_cnt[i];
      before += (i < warp) ? c : 0;
      total += c;
    }
    if (pass) idx[base + before + __popc(bal & ((1u << lane) - 1u))] = (int32_t)b;
    base += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

// A programmatic dependent of the kernel before it (pdl_enter).
__global__ void __launch_bounds__(THREADS)
screen_apply_kernel(const int64_t* __restrict__ f, int64_t S, const int64_t* __restrict__ gstats,
                    int64_t S_total, double lambda, int32_t* __restrict__ idx,
                    int64_t* __restrict__ count, double* __restrict__ Tm,
                    const int64_t* __restrict__ gmax) {
  pdl_enter();
  block_screen_apply(f, S, gstats, S_total, lambda, idx, count, Tm, gmax);
}

// The whole screen of one batch in one block (statistics, then threshold and
// compaction): the unsharded ubqp_screen, a programmatic dependent of the
// evaluation.
__global__ void __launch_bounds__(THREADS)
screen_kernel(const int64_t* __restrict__ f, int64_t S, double lambda, int32_t* __restrict__ idx,
              int64_t* __restrict__ count, double* __restrict__ Tm, int64_t* __restrict__ stats) {
  pdl_enter();
  block_screen_stats(f, S, 0, stats);
  block_screen_apply(f, S, stats, S, lambda, idx, count, Tm);
}

// One block per instance of a batch: the screen of ubqp_screen on its values.
__global__ void __launch_bounds__(THREADS)
screen_batch_kernel(const BatchDesc* __restrict__ d, double lambda) {
  const BatchDesc& b = d[blockIdx.x];
  block_screen_stats(b.f, b.S, 0, b.stats);
  block_screen_apply(b.f, b.S, b.stats, b.S, lambda, b.idx, b.count, b.Tm);
}

}  // namespace

cudaError_t launch_screen_stats(const int64_t* f, int64_t S, int64_t offset, int64_t* stats,
                                cudaStream_t st) {
  screen_stats_kernel<<<1, THREADS, 0, st>>>(f, S, offset, stats);
  return cudaGetLastError();
}

cudaError_t launch_screen(const int64_t* f, int64_t S, double lambda, int32_t* idx,
                          int64_t* count, double* Tm, int64_t* stats, cudaStream_t st) {
  return launch_pdl(screen_kernel, dim3(1), dim3(THREADS), 0, st, f, S, lambda, idx, count, Tm,
                    stats);
}

cudaError_t launch_screen_batch(const BatchDesc* d, int count, double lambda, cudaStream_t st) {
  screen_batch_kernel<<<count, THREADS, 0, st>>>(d, lambda);
  return cudaGetLastError();
}

cudaError_t launch_screen_apply(const int64_t* f, int64_t S, const int64_t* gstats,
                                int64_t S_total, double lambda, int32_t* idx, int64_t* count,
                                double* Tm, cudaStream_t st, const int64_t* gmax) {
  return launch_pdl(screen_apply_kernel, dim3(1), dim3(THREADS), 0, st, f, S, gstats, S_total,
                    lambda, idx, count, Tm, gmax);
}

}  // namespace ubqp
