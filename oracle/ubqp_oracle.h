/*
 * ubqp_oracle.h -- TEST INFRASTRUCTURE: the CPU oracle for the UBQP hot path.
 *
 * Plain, slow, single-threaded C with int64 arithmetic throughout (and the
 * one FP64 threshold of the screen).  It restates the method of Lewis,
 * "A Diversified Multi-Start Algorithm for Unconstrained Binary Quadratic
 * Problems Leveraging the Graphics Processor Unit" (arXiv 1706.00037):
 * problem (P) of the Introduction, and the Pseudocode section (Fig. 2 and the
 * text around it).  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library; the CUDA library never does, and
 * the two share no source.
 *
 * Layouts (host memory):
 *   Q   int8, row-major, n rows of stride ldq >= n bytes; Q[i*ldq + j].
 *   x   bit-packed solution: W = ceil(n/64) uint64 words, bit j of x is
 *       (x[j/64] >> (j%64)) & 1; bits >= n are zero.
 *   X   S solutions back to back, X[s*W + w].
 */
#ifndef UBQP_ORACLE_H
#define UBQP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* SplitMix64 (Steele, Lea & Flood 2014): the first output of the sequential
 * generator whose state starts at `state`. */
uint64_t orc_splitmix64(uint64_t state);
/* Counter-based stream: splitmix64(seed ^ stream*0x9E3779B97F4A7C15 ^ ctr). */
uint64_t orc_rng(uint64_t seed, uint64_t stream, uint64_t ctr);

/* 0 if Q is symmetric, -2 otherwise; *maxabs = max |Q_ij|. */
int orc_validate(const int8_t* Q, int32_t n, int64_t ldq, int32_t* maxabs);

/* f(x) = x^t Q x, problem (P). */
int64_t orc_f(const int8_t* Q, int32_t n, int64_t ldq, const uint64_t* x);
/* f for S packed solutions. */
void orc_eval(const int8_t* Q, int32_t n, int64_t ldq, const uint64_t* X,
              int64_t S, int64_t* f);

/* First-derivative start: x0_i = 1 iff sum_j Q_ij > 0. */
void orc_first_derivative(const int8_t* Q, int32_t n, int64_t ldq, uint64_t* x0);

/* Start generation.  mode 0 = RANDOM (uniform bits), 1 = DIVERSIFY
 * (loop-counter-driven flips and breeding around x0).  DIVERSIFY is a reading
 * of a rule the paper does not print: parity unpinned against the paper (its
 * own structure is pinned). */
void orc_diversify(const uint64_t* x0, int32_t n, int32_t mode, uint64_t seed,
                   uint64_t round, int64_t S, int32_t div_H, uint64_t* X);

/* Screen T(lambda) = Mean + lambda (Max - Mean); pass iff f_b > T.
 * Writes the passing indices ascending to idx and their number to *count. */
void orc_screen(const int64_t* f, int64_t S, double lambda, int32_t* idx,
                int64_t* count, double* T, double* mean, int64_t* maxv,
                int64_t* argmax, int64_t* sum);
/* The same pass test done in exact rational arithmetic (for 0 <= lambda <= 1);
 * pass[b] = 1/0.  Returns -1 if lambda is outside the supported range. */
int orc_screen_exact(const int64_t* f, int64_t S, double lambda, uint8_t* pass);

/* 1-flip steepest ascent of one solution, in place.  Returns the number of
 * flips.  max_flips 0 = unlimited.  trace (may be NULL) receives the flipped
 * indices, at most trace_cap of them. */
int32_t orc_ascent1(const int8_t* Q, int32_t n, int64_t ldq, uint64_t* x,
                    int64_t* f, int32_t max_flips, int32_t* trace,
                    int32_t trace_cap);
/* Ascent of X[idx[t]], t < count; flips[idx[t]] receives the flip count
 * (flips may be NULL). */
void orc_ascent(const int8_t* Q, int32_t n, int64_t ldq, uint64_t* X,
                int64_t* f, const int32_t* idx, int64_t count,
                int32_t max_flips, int32_t* flips);

/* Best of S values, lowest index on ties. */
int64_t orc_best(const int64_t* f, int64_t S, int64_t* best_index);

/* One round of the method: first-derivative start, S starts, evaluation,
 * screen, ascent of the passing starts, best-of.  stats (may be NULL) gets
 * {passed, total_flips, max_flips_seen, batch_max, best_index, sum}, and
 * stats_fp {T, mean}. */
void orc_solve(const int8_t* Q, int32_t n, int64_t ldq, int64_t S,
               double lambda, int32_t max_flips, uint64_t seed, int32_t mode,
               int32_t div_H, uint64_t* best_x, int64_t* best_f,
               int64_t* stats, double* stats_fp);

/* The search of Fig. 2 in rounds of S starts around the incumbent, with the
 * random-sample Mean and the incumbent value as Max in T(lambda).  history
 * (rounds entries) receives the incumbent value after each round; stats =
 * {passed, total flips, sample sum}. */
void orc_search(const int8_t* Q, int32_t n, int64_t ldq, int64_t num_samples,
                int64_t S, int32_t rounds, double lambda, int32_t max_flips,
                uint64_t seed, int32_t div_H, uint64_t* best_x, int64_t* best_f,
                int64_t* history, int64_t* stats);

/* Path relinking from x toward g: flip, among the variables where they still
 * differ, the one of largest 1-flip gain (lowest index on ties; negative gains
 * included) until x = g.  x_best / *f_best receive the best solution strictly
 * between the endpoints (the earliest on ties), or x itself when the distance
 * is below 2.  Returns the Hamming distance. */
int32_t orc_relink1(const int8_t* Q, int32_t n, int64_t ldq, const uint64_t* x,
                    const uint64_t* g, uint64_t* x_best, int64_t* f_best);
/* orc_relink1 for P pairs (X[p], G[p]); dist (may be NULL) gets the distances. */
void orc_relink(const int8_t* Q, int32_t n, int64_t ldq, const uint64_t* X,
                const uint64_t* G, int64_t P, uint64_t* X_best, int64_t* f_best,
                int32_t* dist);

/* Exhaustive search over all 2^n solutions (n <= 24): global maximum and the
 * lowest-numbered maximiser (solution number = its bit pattern). */
int64_t orc_brute_force(const int8_t* Q, int32_t n, int64_t ldq,
                        uint64_t* argmax_bits);

#ifdef __cplusplus
}
#endif
#endif
