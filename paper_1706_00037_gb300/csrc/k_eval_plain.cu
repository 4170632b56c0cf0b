// k_eval_plain.cu -- Evaluate(x) of Fig. 2 on the CUDA cores, one block per
// solution: f = sum_{j : x_j = 1} sum_k Q_jk x_k.  Each warp takes rows j with
// x_j = 1 and dots them with the solution unpacked to bytes in shared memory,
// 16 coefficients per lane per step with dp4a.  This is the per-solution
// comparison path of the tensor-core evaluation; it needs no workspace.
#include "ubqp_internal.cuh"

namespace ubqp {
namespace {

constexpr int THREADS = 256;

__global__ void __launch_bounds__(THREADS)
eval_plain_kernel(const int8_t* __restrict__ Q8, int64_t ldq, int n, int W,
                  const uint64_t* __restrict__ X, int64_t S, int64_t* __restrict__ f) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t* xs = reinterpret_cast<uint64_t*>(smem);        // W words
  uint8_t* xb = smem + ((W * 8 + 15) / 16) * 16;            // ldq bytes of 0/1
  __shared__ long long part[THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t s = blockIdx.x; s < S; s += gridDim.x) {
    for (int w = threadIdx.x; w < W; w += THREADS) xs[w] = X[s * W + w] & valid_mask(n, w);
    __syncthreads();
    for (int j = threadIdx.x; j < ldq; j += THREADS)
      xb[j] = (j < W * 64) ? (uint8_t)((xs[j >> 6] >> (j & 63)) & 1ULL) : (uint8_t)0;
    __syncthreads();
    long long acc = 0;
    for (int j = warp; j < n; j += THREADS / 32) {
      if (!((xs[j >> 6] >> (j & 63)) & 1ULL)) continue;
      const int4* row = reinterpret_cast<const int4*>(Q8 + (int64_t)j * ldq);
      const int4* xv = reinterpret_cast<const int4*>(xb);
      int r = 0;
      for (int c = lane; c * 16 < n; c += 32) {
        int4 q = __ldg(row + c);
        int4 b = xv[c];
        r = __dp4a(q.x, b.x, r);
        r = __dp4a(q.y, b.y, r);
        r = __dp4a(q.z, b.z, r);
        r = __dp4a(q.w, b.w, r);
      }
      acc += r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long t = 0;
      for (int i = 0; i < THREADS / 32; ++i) t += part[i];
      f[s] = t;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_eval_plain(const ubqp_q* h, const uint64_t* X, int64_t S, int64_t* f,
                              cudaStream_t st) {
  size_t smem = ((h->W * 8 + 15) / 16) * 16 + (size_t)h->ldq;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(eval_plain_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
  }
  int64_t blocks = S < (int64_t)h->sm_count * 8 ? S : (int64_t)h->sm_count * 8;
  eval_plain_kernel<<<(unsigned)blocks, THREADS, smem, st>>>(h->Q8, h->ldq, h->n, h->W, X,
                                                             S, f);
  return cudaGetLastError();
}

}  // namespace ubqp
