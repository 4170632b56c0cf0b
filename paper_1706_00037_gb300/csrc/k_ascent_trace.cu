// k_ascent_trace.cu -- the steepest ascent of k_ascent.cu with a record of its
// moves: the same kernels instantiated to also write each climbed start's
// flipped indices, in order, to a caller array.  The sequence of moves is what
// PerformSteepestAscent of Fig. 2 defines (largest 1-flip gain, lowest index
// on ties, while the gain is positive), so the record lets a caller compare
// whole trajectories, not only their end points.  Kept in its own translation
// unit so that the plain ascent's kernels are compiled, and run, untouched.
#include "ascent_core.cuh"

namespace ubqp {

cudaError_t launch_ascent_traced(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                                 const int64_t* count, int64_t S, int32_t max_flips,
                                 int32_t* flips, const float* Y, unsigned long long* next,
                                 uint16_t* trace, int64_t ldt, cudaStream_t st,
                                 bool next_zeroed) {
  return launch_ascent_shaped<true>(h, X, f, idx, count, S, max_flips, flips, Y, next, trace,
                                    ldt, st, next_zeroed);
}

}  // namespace ubqp
