// k_prepare.cu -- one pass over Q: symmetry check (problem (P) requires a
// symmetric Q), max|Q|, the padded int8 copy read by the ascent, the bf16
// tensor-core operands Q' = 2*tril(Q,-1) + diag(Q) (evaluation) and its
// transpose 2*triu(Q,1) + diag(Q) (with Q', the ascent's y = Q x), and the row
// sums behind the first-derivative start of Fig. 2
// (CalculateFirstDerivativeSolution).
#include <cuda_bf16.h>

#include "ubqp_internal.cuh"

namespace ubqp {
namespace {

constexpr int PT = 64;        // tile edge
constexpr int PTHREADS = 256;  // 4 threads per tile row, 16 columns each

// Four bytes of row j from column k (zero at or beyond n): one 32-bit load
// when the four are inside the row and W4 (4-byte aligned rows), else bytes.
template <bool W4>
__device__ __forceinline__ uint32_t row_word(const int8_t* __restrict__ Q, int64_t ldq_in, int n,
                                             int j, int k) {
  if (j >= n) return 0;
  const int8_t* p = Q + (int64_t)j * ldq_in + k;
  if (W4 && k + 3 < n) return *reinterpret_cast<const uint32_t*>(p);
  uint32_t w = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (k + b < n) w |= (uint32_t)(uint8_t)p[b] << (8 * b);
  return w;
}

// Largest column of Q' that the tensor-core evaluation reads in rows
// j0 .. j0 + PT - 1: an N-block of 256 rows (192 in the tensor-memory
// variant) reads K up to the end of its own block.  Tiles of Q' beyond it are
// never read and are not written.
__device__ __forceinline__ int qt_kmax(int j0) {
  const int jl = j0 + PT - 1;
  return max((jl / 256 + 1) * 256, (jl / 192 + 1) * 192) - 1;
}

// One symmetric pair of 64 x 64 tiles per block: T = Q[bi rows][bj cols] and
// U = Q[bj rows][bi cols] (bi <= bj; the diagonal tile pairs with itself), so
// every byte of Q is read once.  Both are staged in shared memory four bytes
// at a time (32-bit loads when the caller's rows are 4-byte aligned); T is
// compared with U transposed (the symmetry check of problem (P)); then for
// each of the two tiles every thread takes 16 consecutive columns of one row
// and writes them as 16-byte vectors: the int8 copy (rows < n), Q' = 2
// tril(Q,-1) + diag(Q) (tiles the evaluation reads) and Q'^t = 2 triu(Q,1) +
// diag(Q) (the upper block triangle, which the start-up reads), both in bf16
// and zero outside n (so the padded squares need no separate clearing), and
// adds its row's partial sum.  It also tracks max|Q|.
template <bool W4>
__global__ void __launch_bounds__(PTHREADS)
prepare_pairs(const int8_t* __restrict__ Q, int n, int64_t ldq_in, int8_t* __restrict__ Q8,
              int64_t ldq, uint16_t* __restrict__ Qt, uint16_t* __restrict__ Qu, int n_tc,
              int32_t* __restrict__ rowsum, unsigned* __restrict__ flags) {
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (bi > bj) return;  // the pair (bj, bi) covers this tile
  __shared__ __align__(16) int8_t tile[2][PT][PT + 4];  // T, then U
  const int t = threadIdx.x;
  const int r0[2] = {bi * PT, bj * PT}, c0s[2] = {bj * PT, bi * PT};
  const int nt = bi == bj ? 1 : 2;
  for (int u = 0; u < nt; ++u)
    for (int i = t; i < PT * PT / 4; i += PTHREADS) {
      const int r = i / (PT / 4), c = (i % (PT / 4)) * 4;
      *reinterpret_cast<uint32_t*>(&tile[u][r][c]) =
          row_word<W4>(Q, ldq_in, n, r0[u] + r, c0s[u] + c);
    }
  __syncthreads();
  const int r = t >> 2, c0 = (t & 3) * 16;
  unsigned asym = 0;
  int amax = 0;
  for (int u = 0; u < nt; ++u) {
    const int j = r0[u] + r, kb = c0s[u];
    const int8_t(*other)[PT + 4] = tile[nt - 1 - u];  // the transposed partner
    int sum = 0;
    uint32_t b8[4] = {0, 0, 0, 0};
    uint32_t ht[8], hu[8];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int k = kb + c0 + i;
      const int v = tile[u][r][c0 + i];
      if (u == 0) asym |= (unsigned)(v != other[c0 + i][r]);
      amax = max(amax, abs(v));
      sum += v;
      b8[i >> 2] |= (uint32_t)(uint8_t)v << (8 * (i & 3));
      const int w = k < j ? 2 * v : (k == j ? v : 0);
      const int wu = k > j ? 2 * v : (k == j ? v : 0);
      const uint32_t bt = __bfloat16_as_ushort(__float2bfloat16_rn((float)w));
      const uint32_t bu = __bfloat16_as_ushort(__float2bfloat16_rn((float)wu));
      if (i & 1) {
        ht[i >> 1] |= bt << 16;
        hu[i >> 1] |= bu << 16;
      } else {
        ht[i >> 1] = bt;
        hu[i >> 1] = bu;
      }
    }
    const int k = kb + c0;
    if (j < n && k < ldq)
      *reinterpret_cast<uint4*>(Q8 + (int64_t)j * ldq + k) =
          make_uint4(b8[0], b8[1], b8[2], b8[3]);
    if (j < n_tc && k < n_tc) {
      if (kb <= qt_kmax(r0[u])) {
        uint4* dt = reinterpret_cast<uint4*>(Qt + (int64_t)j * n_tc + k);
        dt[0] = make_uint4(ht[0], ht[1], ht[2], ht[3]);
        dt[1] = make_uint4(ht[4], ht[5], ht[6], ht[7]);
      }
      if (kb >= r0[u] / 256 * 256) {  // the upper block triangle of 256-row blocks
        uint4* du = reinterpret_cast<uint4*>(Qu + (int64_t)j * n_tc + k);
        du[0] = make_uint4(hu[0], hu[1], hu[2], hu[3]);
        du[1] = make_uint4(hu[4], hu[5], hu[6], hu[7]);
      }
    }
    // the row's partial sum over this tile: the 4 threads of row r are lanes
    // 4m .. 4m+3 of one warp
    sum += __shfl_xor_sync(0xffffffffu, sum, 1);
    sum += __shfl_xor_sync(0xffffffffu, sum, 2);
    if ((t & 3) == 0 && j < n && sum != 0) atomicAdd(&rowsum[j], sum);
  }
  const unsigned any = __ballot_sync(0xffffffffu, asym);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((t & 31) == 0) {
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
  // Q8 columns from n_tc to ldq are outside the tiles: clear the copy first
  if (h->ldq > h->n_tc && (e = cudaMemsetAsync(h->Q8, 0, (size_t)h->n * h->ldq, st))) return e;
  if ((e = cudaMemsetAsync(h->rowsum, 0, sizeof(int32_t) * n, st))) return e;
  if ((e = cudaMemsetAsync(h->scratch_flags, 0, 2 * sizeof(unsigned), st))) return e;
  if ((e = cudaMemsetAsync(h->err, 0, sizeof(unsigned), st))) return e;
  const int tiles = h->n_tc / PT;
  dim3 grid(tiles, tiles);
  if (((uintptr_t)Q & 3) == 0 && (ldq_in & 3) == 0)
    prepare_pairs<true><<<grid, PTHREADS, 0, st>>>(Q, n, ldq_in, h->Q8, h->ldq, h->Qt, h->Qu,
                                                   h->n_tc, h->rowsum, h->scratch_flags);
  else
    prepare_pairs<false><<<grid, PTHREADS, 0, st>>>(Q, n, ldq_in, h->Q8, h->ldq, h->Qt, h->Qu,
                                                    h->n_tc, h->rowsum, h->scratch_flags);
  if ((e = cudaGetLastError())) return e;
  first_derivative_bits<<<(h->W + 127) / 128, 128, 0, st>>>(h->rowsum, n, h->W, h->x0);
  return cudaGetLastError();
}

}  // namespace ubqp
