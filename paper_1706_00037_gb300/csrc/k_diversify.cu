// k_diversify.cu -- start generation: uniform random solutions (the sample of
// EvaluateRandomStarts, Fig. 2) or Diversify(x, best, i, Q_cols) of Fig. 2
// around an incumbent: Glover's h-pattern on even loop counters and breeding
// with a random partner on odd ones.  One thread per output word; pure writes.
#include "ubqp_internal.cuh"

namespace ubqp {
namespace {

// Starts s_begin .. s_begin + S_local - 1 of a batch of S_total (loop counter
// i = round * S_total + s), written to X[(s - s_begin) * W + w].
__global__ void diversify_words(const uint64_t* __restrict__ x0, int n, int W, int mode,
                                uint64_t seed, uint64_t round, int64_t S_total, int64_t s_begin,
                                int64_t S_local, int div_H, uint64_t* __restrict__ X,
                                const uint64_t* __restrict__ seed_dev) {
  if (seed_dev) seed = *seed_dev;
  const int64_t total = S_local * W;
  const int64_t S = S_total;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = t / W;
    const int w = (int)(t - sl * W);
    const int64_t s = s_begin + sl;
    uint64_t v;
    if (mode == UBQP_MODE_RANDOM) {
      v = stream_word(seed, (uint64_t)s, (uint64_t)w);
    } else {
      const uint64_t i = round * (uint64_t)S + (uint64_t)s;
      const uint64_t inc = x0[w];
      if (i == 0) {
        v = inc;
      } else if ((i & 1ULL) == 0) {
        // h-pattern: flip p with p mod h == o, p in this word
        const uint64_t jp = i >> 1;
        const uint64_t H = (uint64_t)(div_H < n ? div_H : n);
        const uint64_t h = 1 + (jp - 1) % H;
        const uint64_t o = ((jp - 1) / H) % h;
        const uint64_t base = (uint64_t)w * 64;
        uint64_t p = base + (o + h - base % h) % h;
        uint64_t flip = 0;
        for (; p < base + 64; p += h) flip |= 1ULL << (p - base);
        v = inc ^ flip;
      } else {
        const uint64_t m = 1 + ((i - 1) >> 1) % 6;
        const uint64_t partner = stream_word(seed, (1ULL << 63) | i, (uint64_t)w);
        uint64_t mask = ~0ULL;
        for (uint64_t k = 0; k < m; ++k)
          mask &= stream_word(seed, (1ULL << 62) | (8 * i + k), (uint64_t)w);
        v = (inc & ~mask) | (partner & mask);
      }
    }
    X[t] = v & valid_mask(n, w);
  }
}

}  // namespace

cudaError_t launch_diversify(const uint64_t* x0, int n, int mode, uint64_t seed,
                             uint64_t round, int64_t S_total, int64_t s_begin,
                             int64_t S_local, int div_H, uint64_t* X, cudaStream_t st,
                             const uint64_t* seed_dev) {
  const int W = (int)words_of(n);
  int64_t total = S_local * W;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  diversify_words<<<(unsigned)blocks, 256, 0, st>>>(x0, n, W, mode, seed, round, S_total,
                                                   s_begin, S_local, div_H, X, seed_dev);
  return cudaGetLastError();
}

}  // namespace ubqp
