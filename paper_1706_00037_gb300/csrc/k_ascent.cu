// k_ascent.cu -- PerformSteepestAscent of Fig. 2, batched: every listed start
// is climbed by 1-bit flips, always taking the flip of largest gain (lowest
// index on ties) while the gain is positive.  Gains are the 1-flip move values
// of Glover et al. (2002) that the Pseudocode section cites,
//     Delta_j = Q_jj + 2 (1 - 2 x_j) y_j,   y = Q x,
// and a flip of bit k (d = 1 - 2 x_k before the flip) changes y by d times
// column k of Q (= row k, Q being symmetric) and negates the sign of x_k.
//
// Design.  A group of T threads owns one start at a time (one warp for
// n <= 512, else one block).  Thread g owns E = 16*C elements, in chunks of 16
// consecutive indices: element e lives at j = (e/16)*16T + 16g + e%16, so one
// move loads row k of the int8 Q (= column k, Q being symmetric) with C fully
// coalesced 16-byte loads per thread.  Per element the thread keeps, in
// registers,
//     y_j,   S_j = 128 (1 - 2 x_j),   C_j = 64 Q_jj + 2 (31 - e) + x_j,
// so that the argmax key  key_j = C_j + S_j y_j = 64 Delta_j + 2 (31 - e) + x_j
// costs one multiply-add.  A move is therefore, per element: y += d q as one
// dp4a (d placed in the coefficient's byte lane), key = C + S y, and a running
// max kept in four independent chains.  The key orders by gain, then by lower
// index inside the thread, and carries x_j in its low bit; across threads the
// group reduces (gain, 2j + x) with warp max/min reductions (redux.sync), so
// every thread learns k, x_k and Delta_k.  The thread owning k negates S_k and
// toggles the x bit of C_k.  Rows are read from L2 (the int8 Q of one
// instance, e.g. 49 MB at n = 7000, stays resident there); nothing per move
// goes to HBM.  The chain of moves is latency-bound: per move a dependent L2
// row fetch, the update and a block-wide reduction.  The fetch is taken off
// the chain when the move was predicted: every move also copies the row of
// the reduction's runner-up into shared memory, and the next move is that
// row often enough (about 40% at n = 7000) to pay for the copies.
//
// Start-up: y = Q x of every listed start comes from the tensor-core product of
// the ascent workspace when given (exact integers in fp32), else each group
// sums the rows k with x_k = 1 on the CUDA cores.
#include "ascent_core.cuh"

namespace ubqp {

cudaError_t launch_relink(const ubqp_q* h, const uint64_t* X, const int64_t* f, const uint64_t* G,
                          int64_t P, uint64_t* Xb, int64_t* fb, int32_t* dist, uint16_t* trace,
                          int64_t ldt, const float* Y, unsigned long long* next,
                          cudaStream_t st) {
  const int n = h->n;
  if (next) {
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
#define UBQP_RL_ARGS h, X, f, G, P, Xb, fb, dist, trace, ldt, Y, next, st
  if (n <= 256) return launch_relink_warp<1>(UBQP_RL_ARGS);
  if (n <= 512) return launch_relink_warp<2>(UBQP_RL_ARGS);
  if (n <= 1024) return launch_relink_block<64, 1>(UBQP_RL_ARGS);
  if (n <= 2048) return launch_relink_block<128, 1>(UBQP_RL_ARGS);
  if (n <= 4096) return launch_relink_block<256, 1>(UBQP_RL_ARGS);
  if (n <= 8192) return launch_relink_block<256, 2>(UBQP_RL_ARGS);
  if (n <= 16384) return launch_relink_block<512, 2>(UBQP_RL_ARGS);
#undef UBQP_RL_ARGS
  return cudaErrorInvalidValue;
}

bool ascent_batch_supported(int T, int C) {
  return (T == 64 || T == 128 || T == 256 || T == 512) && (C == 1 || C == 2);
}

int ascent_batch_grid(int T, int C, int sm_count) {
  int per_sm = 0;
  cudaError_t e = cudaErrorInvalidValue;
#define UBQP_OCC(TT, CC)                                                                     \
  if (T == TT && C == CC)                                                                    \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                       \
        &per_sm, ascent_batch_kernel<TT, CC, kSpecRows>, TT, 0);
  UBQP_OCC(64, 1) UBQP_OCC(64, 2) UBQP_OCC(128, 1) UBQP_OCC(128, 2)
  UBQP_OCC(256, 1) UBQP_OCC(256, 2) UBQP_OCC(512, 1) UBQP_OCC(512, 2)
#undef UBQP_OCC
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm * sm_count;
}

cudaError_t launch_ascent_batch(const BatchDesc* d, const int2* items, const int64_t* n_items,
                                int T, int C, int32_t max_flips, int grid,
                                unsigned long long* next, cudaStream_t st) {
#define UBQP_ASC(TT, CC)                                                                      \
  if (T == TT && C == CC)                                                                     \
    return launch_ascent_batch_tc<TT, CC>(d, items, n_items, max_flips, grid, next, st);
  UBQP_ASC(64, 1) UBQP_ASC(64, 2) UBQP_ASC(128, 1) UBQP_ASC(128, 2)
  UBQP_ASC(256, 1) UBQP_ASC(256, 2) UBQP_ASC(512, 1) UBQP_ASC(512, 2)
#undef UBQP_ASC
  return cudaErrorInvalidValue;
}

bool ascent_packed_supported(int T, int C) { return T == 256 && (C == 1 || C == 2); }

int ascent_packed_grid(int T, int C, int sm_count) {
  int per_sm = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (T == 256 && C == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, ascent_batch_packed_kernel<256, 1, kSpecRows>, 256, 0);
  if (T == 256 && C == 2)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, ascent_batch_packed_kernel<256, 2, kSpecRows>, 256, 0);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm * sm_count;
}

cudaError_t launch_ascent_batch_packed(const BatchDesc* d, const int2* items, const int4* ranges,
                                       int T, int C, int32_t max_flips, int grid,
                                       unsigned long long* next, cudaStream_t st) {
  if (next) {  // one start counter per class
    cudaError_t e = cudaMemsetAsync(next, 0, 4 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  if (T == 256 && C == 1)
    ascent_batch_packed_kernel<256, 1, kSpecRows><<<grid, 256, 0, st>>>(d, items, ranges,
                                                                         max_flips, next);
  else if (T == 256 && C == 2)
    ascent_batch_packed_kernel<256, 2, kSpecRows><<<grid, 256, 0, st>>>(d, items, ranges,
                                                                         max_flips, next);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_ascent(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                          const int64_t* count, int64_t S, int32_t max_flips, int32_t* flips,
                          const float* Y, unsigned long long* next, cudaStream_t st,
                          bool next_zeroed) {
  return launch_ascent_shaped<false>(h, X, f, idx, count, S, max_flips, flips, Y, next, nullptr,
                                     0, st, next_zeroed);
}

}  // namespace ubqp
