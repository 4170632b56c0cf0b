// k_prepare.cu -- one pass over Q: symmetry check (problem (P) requires a
// symmetric Q), max|Q|, the padded int8 copy read by the ascent, the bf16
// tensor-core operands Q' = 2*tril(Q,-1) + diag(Q) (evaluation) and Q (the
// ascent's y = Q x), and the row sums behind the
// first-derivative start of Fig. 2 (CalculateFirstDerivativeSolution).
#include <cuda_bf16.h>

#include "ubqp_internal.cuh"

namespace ubqp {
namespace {

constexpr int TILE = 32;
constexpr int ROWS = 8;  // block is TILE x ROWS threads, 4 rows per thread

__global__ void __launch_bounds__(TILE* ROWS)
prepare_tiles(const int8_t* __restrict__ Q, int n, int64_t ldq_in, int8_t* __restrict__ Q8,
              int64_t ldq, uint16_t* __restrict__ Qt, uint16_t* __restrict__ Qf, int n_tc,
              int32_t* __restrict__ rowsum,
              unsigned* __restrict__ flags) {
  __shared__ int8_t tr[TILE][TILE + 4];
  const int bj = blockIdx.y * TILE, bk = blockIdx.x * TILE;
  const int tx = threadIdx.x, ty = threadIdx.y;
  // transposed tile: rows bk.., cols bj..
  for (int r = ty; r < TILE; r += ROWS) {
    int row = bk + r, col = bj + tx;
    tr[r][tx] = (row < n && col < n) ? Q[(int64_t)row * ldq_in + col] : (int8_t)0;
  }
  __syncthreads();
  unsigned asym = 0;
  int amax = 0;
  for (int r = ty; r < TILE; r += ROWS) {
    const int j = bj + r, k = bk + tx;
    int v = 0;
    if (j < n && k < n) {
      v = Q[(int64_t)j * ldq_in + k];
      if ((int8_t)v != tr[tx][r]) asym = 1;
      Q8[(int64_t)j * ldq + k] = (int8_t)v;
      int w = k < j ? 2 * v : (k == j ? v : 0);
      Qt[(int64_t)j * n_tc + k] = __bfloat16_as_ushort(__float2bfloat16_rn((float)w));
      Qf[(int64_t)j * n_tc + k] = __bfloat16_as_ushort(__float2bfloat16_rn((float)v));
    }
    amax = max(amax, abs(v));
    // row partial sum over this tile's 32 columns
    int s = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tx == 0 && j < n && s != 0) atomicAdd(&rowsum[j], s);
  }
  unsigned any = __ballot_sync(0xffffffffu, asym);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if (tx == 0) {
    if (any) atomicAdd(&flags[0], 1u);
    atomicMax(&flags[1], (unsigned)amax);
  }
}

__global__ void first_derivative_bits(const int32_t* __restrict__ rowsum, int n, int W,
                                      uint64_t* __restrict__ x0) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  uint64_t bits = 0;
  for (int b = 0; b < 64; ++b) {
    int j = w * 64 + b;
    if (j < n && rowsum[j] > 0) bits |= 1ULL << b;
  }
  x0[w] = bits;
}

}  // namespace

cudaError_t launch_prepare(const int8_t* Q, int n, int64_t ldq_in, ubqp_q* h,
                           cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->Q8, 0, (size_t)h->n * h->ldq, st))) return e;
  if ((e = cudaMemsetAsync(h->Qt, 0, (size_t)h->n_tc * h->n_tc * 2, st))) return e;
  if ((e = cudaMemsetAsync(h->Qf, 0, (size_t)h->n_tc * h->n_tc * 2, st))) return e;
  if ((e = cudaMemsetAsync(h->rowsum, 0, sizeof(int32_t) * n, st))) return e;
  if ((e = cudaMemsetAsync(h->scratch_flags, 0, 2 * sizeof(unsigned), st))) return e;
  if ((e = cudaMemsetAsync(h->err, 0, sizeof(unsigned), st))) return e;
  dim3 grid((n + TILE - 1) / TILE, (n + TILE - 1) / TILE), block(TILE, ROWS);
  prepare_tiles<<<grid, block, 0, st>>>(Q, n, ldq_in, h->Q8, h->ldq, h->Qt, h->Qf, h->n_tc,
                                         h->rowsum, h->scratch_flags);
  if ((e = cudaGetLastError())) return e;
  first_derivative_bits<<<(h->W + 127) / 128, 128, 0, st>>>(h->rowsum, n, h->W, h->x0);
  return cudaGetLastError();
}

}  // namespace ubqp
