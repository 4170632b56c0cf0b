/*
 * ubqp_oracle.c -- TEST INFRASTRUCTURE: the CPU oracle for the UBQP hot path.
 *
 * This file is the checker, not the product.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg load it.  It is written for a reader
 * holding the paper (Lewis, arXiv 1706.00037): every function names the
 * passage it restates, uses the paper's notation where the paper has one, and
 * does nothing clever -- no blocking, no fusion, no reordering.  All integer
 * work is int64; the one floating-point quantity (the screening threshold) is
 * computed in IEEE double with separate round-to-nearest operations (the file
 * is compiled with -ffp-contract=off so that no FMA is formed).
 *
 * Where the paper is silent (the exact diversification rule, tie-breaks, the
 * row-sum-zero case of the first-derivative start) the reading used here is
 * stated beside the code.
 */
#include "ubqp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_GOLDEN 0x9E3779B97F4A7C15ULL

/* SplitMix64 as published by Steele, Lea & Flood (OOPSLA 2014): advance the
 * state by the golden gamma, then apply the variant-13 finaliser. */
uint64_t orc_splitmix64(uint64_t state) {
  uint64_t z = state + ORC_GOLDEN;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t orc_rng(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return orc_splitmix64(seed ^ (stream * ORC_GOLDEN) ^ ctr);
}

static int orc_bit(const uint64_t* x, int64_t j) {
  return (int)((x[j >> 6] >> (j & 63)) & 1ULL);
}

static void orc_set_bit(uint64_t* x, int64_t j, int v) {
  uint64_t m = 1ULL << (j & 63);
  if (v) x[j >> 6] |= m; else x[j >> 6] &= ~m;
}

static int64_t orc_words(int32_t n) { return ((int64_t)n + 63) / 64; }

/* Problem (P) states Q is an n-by-n symmetric matrix. */
int orc_validate(const int8_t* Q, int32_t n, int64_t ldq, int32_t* maxabs) {
  int32_t m = 0;
  int sym = 1;
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t j = 0; j < n; ++j) {
      int32_t v = Q[(int64_t)i * ldq + j];
      if (v < 0) v = -v;
      if (v > m) m = v;
      if (Q[(int64_t)i * ldq + j] != Q[(int64_t)j * ldq + i]) sym = 0;
    }
  }
  if (maxabs) *maxabs = m;
  return sym ? 0 : -2;
}

/* Problem (P), Introduction: x_o = f(x) = x^t Q x with x_i in {0,1}. */
int64_t orc_f(const int8_t* Q, int32_t n, int64_t ldq, const uint64_t* x) {
  int64_t f = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (!orc_bit(x, i)) continue;
    for (int32_t j = 0; j < n; ++j) {
      if (orc_bit(x, j)) f += Q[(int64_t)i * ldq + j];
    }
  }
  return f;
}

/* Evaluate / EvaluateRandomStarts of Fig. 2: xQx for every solution. */
void orc_eval(const int8_t* Q, int32_t n, int64_t ldq, const uint64_t* X,
              int64_t S, int64_t* f) {
  int64_t W = orc_words(n);
  for (int64_t s = 0; s < S; ++s) f[s] = orc_f(Q, n, ldq, X + s * W);
}

/* CalculateFirstDerivativeSolution of Fig. 2, as the Pseudocode section
 * explains it: sum row i of Q and set x_i = 1 if that sum is positive.
 * Reading: a row sum of exactly zero is not positive, so x_i = 0. */
void orc_first_derivative(const int8_t* Q, int32_t n, int64_t ldq, uint64_t* x0) {
  int64_t W = orc_words(n);
  memset(x0, 0, (size_t)W * sizeof(uint64_t));
  for (int32_t i = 0; i < n; ++i) {
    int64_t r = 0;
    for (int32_t j = 0; j < n; ++j) r += Q[(int64_t)i * ldq + j];
    orc_set_bit(x0, i, r > 0);
  }
}

/*
 * Start generation.  The paper evaluates a sample of uniformly random
 * solutions (EvaluateRandomStarts, Fig. 2) -- mode 0 -- and, in the main loop,
 * derives new starts from the incumbent with Diversify(x, best, i, Q_cols),
 * where the number of variables changed depends on the loop counter i and new
 * solutions are made by blending two solutions, after Glover's (1998)
 * diversification generators -- mode 1.  The paper does not print the rule;
 * the reading fixed here is:
 *   i = round*S + s is the loop counter of start s.
 *   i = 0: the incumbent itself (Fig. 2 diversifies only when i > 0).
 *   i even > 0: Glover's h-pattern.  j' = i/2, H = min(n, div_H),
 *     h = 1 + (j'-1) mod H, o = ((j'-1) div H) mod h; flip every bit p with
 *     p mod h == o (h = 1 complements the incumbent).
 *   i odd: breeding with a uniform random partner; each bit is taken from the
 *     partner where a mask is set, the mask being the AND of
 *     m = 1 + ((i-1)/2 mod 6) random words.
 * Random words come from orc_rng: RANDOM word w of start s uses stream s;
 * the partner of counter i uses stream 2^63 | i; mask word t of counter i uses
 * stream 2^62 | (8i + t).  Bits >= n are cleared.
 * DIVERSIFY: parity unpinned against the paper (which prints no rule); the
 * tests pin this reading's own structure -- hand-worked h-patterns, the
 * blend's independence from the incumbent and its bit frequency 2^-m.
 */
void orc_diversify(const uint64_t* x0, int32_t n, int32_t mode, uint64_t seed,
                   uint64_t round, int64_t S, int32_t div_H, uint64_t* X) {
  int64_t W = orc_words(n);
  for (int64_t s = 0; s < S; ++s) {
    uint64_t* x = X + s * W;
    if (mode == 0) {
      for (int64_t w = 0; w < W; ++w) x[w] = orc_rng(seed, (uint64_t)s, (uint64_t)w);
    } else {
      uint64_t i = round * (uint64_t)S + (uint64_t)s;
      for (int64_t w = 0; w < W; ++w) x[w] = x0[w];
      if (i > 0 && i % 2 == 0) {
        uint64_t jp = i / 2;
        uint64_t H = (uint64_t)(div_H < n ? div_H : n);
        uint64_t h = 1 + (jp - 1) % H;
        uint64_t o = ((jp - 1) / H) % h;
        for (int32_t p = 0; p < n; ++p) {
          if ((uint64_t)p % h == o) orc_set_bit(x, p, !orc_bit(x, p));
        }
      } else if (i % 2 == 1) {
        uint64_t m = 1 + ((i - 1) / 2) % 6;
        for (int64_t w = 0; w < W; ++w) {
          uint64_t partner = orc_rng(seed, (1ULL << 63) | i, (uint64_t)w);
          uint64_t mask = ~0ULL;
          for (uint64_t t = 0; t < m; ++t)
            mask &= orc_rng(seed, (1ULL << 62) | (8 * i + t), (uint64_t)w);
          x[w] = (x0[w] & ~mask) | (partner & mask);
        }
      }
    }
    /* solution bits beyond n are zero by convention */
    for (int64_t j = n; j < W * 64; ++j) orc_set_bit(x, j, 0);
  }
}

/*
 * Screening, Pseudocode section: T(lambda) = Mean + lambda (Max - Mean), and
 * a start proceeds to steepest ascent when its xQx exceeds T (Fig. 2, strict
 * ">").  Reading: Mean and Max are taken over the batch being screened; the
 * sum is exact in int64; mean = sum / S, then T by one subtraction, one
 * multiplication and one addition, each rounded to nearest.
 */
void orc_screen(const int64_t* f, int64_t S, double lambda, int32_t* idx,
                int64_t* count, double* T, double* mean, int64_t* maxv,
                int64_t* argmax, int64_t* sum) {
  int64_t total = 0, mx = f[0], am = 0;
  for (int64_t b = 0; b < S; ++b) {
    total += f[b];
    if (f[b] > mx) { mx = f[b]; am = b; }
  }
  double mu = (double)total / (double)S;
  double diff = (double)mx - mu;
  double scaled = lambda * diff;
  double t = mu + scaled;
  int64_t c = 0;
  for (int64_t b = 0; b < S; ++b) {
    if ((double)f[b] > t) idx[c++] = (int32_t)b;
  }
  *count = c;
  *T = t;
  *mean = mu;
  *maxv = mx;
  *argmax = am;
  if (sum) *sum = total;
}

/* The pass test f_b > sum/S + lambda (max - sum/S) in exact rational form.
 * lambda = m * 2^-e with integer m (every finite double is dyadic), so the test
 * is  S f_b 2^e > sum 2^e + m (S max - sum), evaluated in 128-bit integers. */
int orc_screen_exact(const int64_t* f, int64_t S, double lambda, uint8_t* pass) {
  if (!(lambda >= 0.0 && lambda <= 1.0)) return -1;
  int64_t total = 0, mx = f[0];
  for (int64_t b = 0; b < S; ++b) {
    total += f[b];
    if (f[b] > mx) mx = f[b];
  }
  int e = 0;
  double m = lambda;
  while (m != floor(m)) { m *= 2.0; ++e; }  /* exact: scaling by 2 */
  if (e > 60) return -1;
  __int128 scale = (__int128)1 << e;
  __int128 rhs = (__int128)total * scale +
                 (__int128)(int64_t)m * ((__int128)S * mx - total);
  for (int64_t b = 0; b < S; ++b) {
    __int128 lhs = (__int128)S * f[b] * scale;
    pass[b] = lhs > rhs;
  }
  return 0;
}

/*
 * PerformSteepestAscent(x, xQx, max_its) of Fig. 2: repeatedly make the
 * single-bit flip that improves the objective most, until no flip improves it
 * or max_its flips have been made; no tabu list and no cycling check.  The gain
 * of flipping bit i is the 1-flip move value of Glover et al. (2002), cited in
 * the Pseudocode section:
 *     Delta_i = Q_ii + 2 (1 - 2 x_i) y_i,   y = Q x,
 * and after flipping bit k (d = 1 - 2 x_k before the flip)
 *     Delta_j += 2 (1 - 2 x_j) d Q_jk  (j != k),   Delta_k = -Delta_k.
 * Readings: ties go to the lowest index; a flip improves only if Delta > 0;
 * max_flips 0 means no cap.
 */
int32_t orc_ascent1(const int8_t* Q, int32_t n, int64_t ldq, uint64_t* x,
                    int64_t* f, int32_t max_flips, int32_t* trace,
                    int32_t trace_cap) {
  int64_t* y = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* D = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) {
    int64_t acc = 0;
    for (int32_t j = 0; j < n; ++j)
      if (orc_bit(x, j)) acc += Q[(int64_t)i * ldq + j];
    y[i] = acc;
  }
  for (int32_t i = 0; i < n; ++i)
    D[i] = Q[(int64_t)i * ldq + i] + 2 * (1 - 2 * orc_bit(x, i)) * y[i];
  int32_t flips = 0;
  while (n > 0) {
    if (max_flips > 0 && flips == max_flips) break;
    int32_t k = 0;
    for (int32_t i = 1; i < n; ++i)
      if (D[i] > D[k]) k = i;
    if (D[k] <= 0) break;
    *f += D[k];
    int64_t d = 1 - 2 * orc_bit(x, k);
    orc_set_bit(x, k, !orc_bit(x, k));
    for (int32_t j = 0; j < n; ++j) {
      if (j == k) continue;
      D[j] += 2 * (1 - 2 * orc_bit(x, j)) * d * Q[(int64_t)j * ldq + k];
    }
    D[k] = -D[k];
    if (trace && flips < trace_cap) trace[flips] = k;
    ++flips;
  }
  free(y);
  free(D);
  return flips;
}

void orc_ascent(const int8_t* Q, int32_t n, int64_t ldq, uint64_t* X,
                int64_t* f, const int32_t* idx, int64_t count,
                int32_t max_flips, int32_t* flips) {
  int64_t W = orc_words(n);
  for (int64_t t = 0; t < count; ++t) {
    int64_t s = idx[t];
    int32_t c = orc_ascent1(Q, n, ldq, X + s * W, f + s, max_flips, NULL, 0);
    if (flips) flips[s] = c;
  }
}

/* UpdateBestAndT of Fig. 2 keeps the best solution; reading: lowest index on
 * ties. */
int64_t orc_best(const int64_t* f, int64_t S, int64_t* best_index) {
  int64_t b = 0;
  for (int64_t s = 1; s < S; ++s)
    if (f[s] > f[b]) b = s;
  if (best_index) *best_index = b;
  return f[b];
}

/* One pass of Fig. 2's loop body over a batch of S starts. */
void orc_solve(const int8_t* Q, int32_t n, int64_t ldq, int64_t S,
               double lambda, int32_t max_flips, uint64_t seed, int32_t mode,
               int32_t div_H, uint64_t* best_x, int64_t* best_f,
               int64_t* stats, double* stats_fp) {
  int64_t W = orc_words(n);
  uint64_t* x0 = (uint64_t*)calloc((size_t)W, sizeof(uint64_t));
  uint64_t* X = (uint64_t*)calloc((size_t)(S * W), sizeof(uint64_t));
  int64_t* f = (int64_t*)calloc((size_t)S, sizeof(int64_t));
  int32_t* idx = (int32_t*)calloc((size_t)S, sizeof(int32_t));
  int32_t* flips = (int32_t*)calloc((size_t)S, sizeof(int32_t));
  orc_first_derivative(Q, n, ldq, x0);
  orc_diversify(x0, n, mode, seed, 0, S, div_H, X);
  orc_eval(Q, n, ldq, X, S, f);
  int64_t count = 0, maxv = 0, argmax = 0, sum = 0;
  double T = 0, mean = 0;
  orc_screen(f, S, lambda, idx, &count, &T, &mean, &maxv, &argmax, &sum);
  orc_ascent(Q, n, ldq, X, f, idx, count, max_flips, flips);
  int64_t bi = 0;
  *best_f = orc_best(f, S, &bi);
  memcpy(best_x, X + bi * W, (size_t)W * sizeof(uint64_t));
  if (stats) {
    int64_t tot = 0, mxf = 0;
    for (int64_t s = 0; s < S; ++s) {
      tot += flips[s];
      if (flips[s] > mxf) mxf = flips[s];
    }
    stats[0] = count;
    stats[1] = tot;
    stats[2] = mxf;
    stats[3] = maxv;
    stats[4] = bi;
    stats[5] = sum;
  }
  if (stats_fp) {
    stats_fp[0] = T;
    stats_fp[1] = mean;
  }
  free(x0);
  free(X);
  free(f);
  free(idx);
  free(flips);
}

/* Exhaustive enumeration of problem (P) for small n. */
int64_t orc_brute_force(const int8_t* Q, int32_t n, int64_t ldq,
                        uint64_t* argmax_bits) {
  uint64_t best_p = 0;
  int64_t best = 0;
  uint64_t x[1];
  for (uint64_t p = 0; p < (1ULL << n); ++p) {
    x[0] = p;
    int64_t v = orc_f(Q, n, ldq, x);
    if (p == 0 || v > best) { best = v; best_p = p; }
  }
  if (argmax_bits) *argmax_bits = best_p;
  return best;
}

/*
 * The search of Fig. 2 run in rounds of S starts (the loop body applied to a
 * batch at a time).  Before the loop: EvaluateRandomStarts -- the mean of
 * num_samples uniform random solutions (RANDOM mode, seed) -- and
 * CalculateFirstDerivativeSolution, whose value is the initial Max.  Round r:
 * S starts diversified around the incumbent with loop counters r*S + s (so the
 * very first start, i = 0, is the first-derivative solution itself), their
 * values, the screen T = Mean + lambda (Max - Mean) with the sample Mean and
 * the incumbent's value as Max (the text after Fig. 2: Mean from sampling, Max
 * the best so far), ascent of every start with xQx > T, then UpdateBestAndT:
 * the round's best replaces the incumbent when strictly better (so Max and T
 * rise).  Reading: within a round the incumbent and T stay fixed (batched).
 * history[r] = incumbent value after round r; stats = {passed, flips} totals.
 */
void orc_search(const int8_t* Q, int32_t n, int64_t ldq, int64_t num_samples,
                int64_t S, int32_t rounds, double lambda, int32_t max_flips,
                uint64_t seed, int32_t div_H, uint64_t* best_x, int64_t* best_f,
                int64_t* history, int64_t* stats) {
  int64_t W = orc_words(n);
  /* sample mean */
  uint64_t* Xs = (uint64_t*)calloc((size_t)(num_samples * W), sizeof(uint64_t));
  int64_t* fs = (int64_t*)calloc((size_t)num_samples, sizeof(int64_t));
  orc_diversify(NULL, n, 0, seed, 0, num_samples, div_H, Xs);
  orc_eval(Q, n, ldq, Xs, num_samples, fs);
  int64_t sample_sum = 0;
  for (int64_t b = 0; b < num_samples; ++b) sample_sum += fs[b];
  double mean = (double)sample_sum / (double)num_samples;
  free(Xs);
  free(fs);
  /* incumbent = first-derivative start */
  uint64_t* inc = (uint64_t*)calloc((size_t)W, sizeof(uint64_t));
  orc_first_derivative(Q, n, ldq, inc);
  int64_t inc_f = orc_f(Q, n, ldq, inc);
  uint64_t* X = (uint64_t*)calloc((size_t)(S * W), sizeof(uint64_t));
  int64_t* f = (int64_t*)calloc((size_t)S, sizeof(int64_t));
  int32_t* flips = (int32_t*)calloc((size_t)S, sizeof(int32_t));
  int64_t passed = 0, total_flips = 0;
  for (int32_t r = 0; r < rounds; ++r) {
    orc_diversify(inc, n, 1, seed, (uint64_t)r, S, div_H, X);
    orc_eval(Q, n, ldq, X, S, f);
    double diff = (double)inc_f - mean;
    double scaled = lambda * diff;
    double T = mean + scaled;
    for (int64_t s = 0; s < S; ++s) {
      flips[s] = 0;
      if ((double)f[s] > T) {
        flips[s] = orc_ascent1(Q, n, ldq, X + s * W, f + s, max_flips, NULL, 0);
        ++passed;
        total_flips += flips[s];
      }
    }
    int64_t bi = 0;
    int64_t bf = orc_best(f, S, &bi);
    if (bf > inc_f) {
      inc_f = bf;
      memcpy(inc, X + bi * W, (size_t)W * sizeof(uint64_t));
    }
    history[r] = inc_f;
  }
  memcpy(best_x, inc, (size_t)W * sizeof(uint64_t));
  *best_f = inc_f;
  stats[0] = passed;
  stats[1] = total_flips;
  stats[2] = sample_sum;
  free(inc);
  free(X);
  free(f);
  free(flips);
}

/* Path relinking: the solution-polishing phase the Experiments section names
 * for after the multi-start phase, and the Path Relinking phase of Glover's
 * template (Glover 1998) that Fig. 1's concepts come from.  From the
 * initiating solution x toward the guiding solution g: while x and g differ,
 * flip the differing variable whose flip gains most (the 1-flip move value
 * Q_kk + 2 (1 - 2 x_k) y_k; lowest index on ties), whether the gain is
 * positive or not, until x = g.  Reading: the result is the best solution
 * strictly between the endpoints (after 1 .. |D|-1 flips, the earliest on
 * ties), since both endpoints are already known; with |D| < 2 there is none
 * and the result is x itself.  Returns |D|, the Hamming distance. */
int32_t orc_relink1(const int8_t* Q, int32_t n, int64_t ldq, const uint64_t* x_init,
                    const uint64_t* g, uint64_t* x_best, int64_t* f_best) {
  int64_t W = orc_words(n);
  uint64_t* x = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)W);
  int64_t* y = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  memcpy(x, x_init, sizeof(uint64_t) * (size_t)W);
  for (int32_t i = 0; i < n; ++i) {
    int64_t acc = 0;
    for (int32_t j = 0; j < n; ++j)
      if (orc_bit(x, j)) acc += Q[(int64_t)i * ldq + j];
    y[i] = acc;
  }
  int64_t fx = orc_f(Q, n, ldq, x);
  int32_t dist = 0;
  for (int32_t j = 0; j < n; ++j) dist += orc_bit(x, j) != orc_bit(g, j);
  memcpy(x_best, x, sizeof(uint64_t) * (size_t)W);
  *f_best = fx;
  int have = 0;
  for (int32_t t = 1; t <= dist; ++t) {
    int32_t k = -1;
    int64_t dk = 0;
    for (int32_t j = 0; j < n; ++j) {
      if (orc_bit(x, j) == orc_bit(g, j)) continue;
      int64_t dj = Q[(int64_t)j * ldq + j] + 2 * (1 - 2 * orc_bit(x, j)) * y[j];
      if (k < 0 || dj > dk) {
        k = j;
        dk = dj;
      }
    }
    /* flip k: y changes by (1 - 2 x_k) times column k */
    int64_t d = 1 - 2 * orc_bit(x, k);
    orc_set_bit(x, k, !orc_bit(x, k));
    for (int32_t j = 0; j < n; ++j) y[j] += d * Q[(int64_t)j * ldq + k];
    fx += dk;
    if (t < dist && (!have || fx > *f_best)) {
      have = 1;
      *f_best = fx;
      memcpy(x_best, x, sizeof(uint64_t) * (size_t)W);
    }
  }
  free(x);
  free(y);
  return dist;
}

void orc_relink(const int8_t* Q, int32_t n, int64_t ldq, const uint64_t* X,
                const uint64_t* G, int64_t P, uint64_t* X_best, int64_t* f_best,
                int32_t* dist) {
  int64_t W = orc_words(n);
  for (int64_t p = 0; p < P; ++p) {
    int32_t d = orc_relink1(Q, n, ldq, X + p * W, G + p * W, X_best + p * W, f_best + p);
    if (dist) dist[p] = d;
  }
}
