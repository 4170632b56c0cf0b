// k_diversify.cu -- start generation: uniform random solutions (the sample of
// EvaluateRandomStarts, Fig. 2) or Diversify(x, best, i, Q_cols) of Fig. 2
// around an incumbent: Glover's h-pattern on even loop counters and breeding
// with a random partner on odd ones.  One thread per output word; pure writes.
#include "ubqp_internal.cuh"

namespace ubqp {
namespace {

// Word w of start s of a batch of S (loop counter i = round * S + s).
__device__ __forceinline__ uint64_t start_word(const uint64_t* __restrict__ x0, int n, int mode,
                                               uint64_t seed, uint64_t round, int64_t S,
                                               int64_t s, int w, int div_H) {
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
  return v & valid_mask(n, w);
}

// Starts s_begin .. s_begin + S_local - 1 of a batch of S_total (loop counter
// i = round * S_total + s), written to X[(s - s_begin) * W + w]; a
// programmatic dependent of whatever precedes it on the stream.
__global__ void diversify_words(const uint64_t* __restrict__ x0, int n, int W, int mode,
                                uint64_t seed, uint64_t round, int64_t S_total, int64_t s_begin,
                                int64_t S_local, int div_H, uint64_t* __restrict__ X,
                                const uint64_t* __restrict__ seed_dev,
                                int32_t* __restrict__ flips0) {
  pdl_enter();
  if (seed_dev) seed = *seed_dev;
  const int64_t total = S_local * W;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = t / W;
    const int w = (int)(t - sl * W);
    X[t] = start_word(x0, n, mode, seed, round, S_total, s_begin + sl, w, div_H);
    if (flips0 && w == 0) flips0[sl] = 0;
  }
}

// Every instance of a batch in one launch (instance blockIdx.y): its S starts
// around its own first-derivative start, and its values and flip counts
// zeroed for the evaluation's and the ascent's accumulation.
__global__ void diversify_batch_words(const BatchDesc* __restrict__ d, int mode,
                                      const uint64_t* __restrict__ seed_dev, uint64_t round,
                                      int div_H) {
  const BatchDesc& b = d[blockIdx.y];
  const uint64_t seed = *seed_dev;
  const int64_t total = b.S * b.W;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / b.W;
    const int w = (int)(t - s * b.W);
    b.X[t] = start_word(b.x0, b.n, mode, seed, round, b.S, s, w, div_H);
    if (w == 0) {
      b.f[s] = 0;
      b.flips[s] = 0;
    }
  }
}

}  // namespace

cudaError_t launch_diversify(const uint64_t* x0, int n, int mode, uint64_t seed,
                             uint64_t round, int64_t S_total, int64_t s_begin,
                             int64_t S_local, int div_H, uint64_t* X, cudaStream_t st,
                             const uint64_t* seed_dev, int32_t* flips0) {
  const int W = (int)words_of(n);
  int64_t total = S_local * W;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  return launch_pdl(diversify_words, dim3((unsigned)blocks), dim3(256), 0, st, x0, n, W, mode,
                    seed, round, S_total, s_begin, S_local, div_H, X, seed_dev, flips0);
}

cudaError_t launch_diversify_batch(const BatchDesc* d, int count, int64_t max_words, int mode,
                                   const uint64_t* seed_dev, uint64_t round, int div_H,
                                   cudaStream_t st) {
  int64_t blocks = (max_words + 255) / 256;
  if (blocks > 64) blocks = 64;
  if (blocks < 1) blocks = 1;
  diversify_batch_words<<<dim3((unsigned)blocks, (unsigned)count), 256, 0, st>>>(
      d, mode, seed_dev, round, div_H);
  return cudaGetLastError();
}

}  // namespace ubqp
