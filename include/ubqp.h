/*
 * ubqp.h -- C ABI of libubqp: the GB300 (sm_103a) hot path of the
 * GPU-screened diversified multi-start method for the Unconstrained Binary
 * Quadratic Problem (M. Lewis, arXiv 1706.00037).
 *
 *   maximise f(x) = x^t Q x,  x in {0,1}^n,  Q symmetric integer   -- problem (P),
 *   Introduction.
 *
 * The routines mirror the steps of Fig. 2 (Pseudocode section): the
 * first-derivative start, start generation (EvaluateRandomStarts / Diversify),
 * evaluation of xQx, the screen T(lambda) = Mean + lambda (Max - Mean), steepest
 * ascent by 1-bit flips (PerformSteepestAscent) and keeping the best solution
 * (UpdateBestAndT).  Every result is exact integer arithmetic; the only
 * floating-point value is the screening threshold.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Pointers named *_dev (and every array argument unless stated otherwise)
 *    are DEVICE pointers owned by the caller.  The library never frees caller
 *    memory, allocates device memory only inside a ubqp_q handle, and never
 *    synchronises a stream unless the call's comment says so.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work of a call is enqueued on it, in order.  Most
 *    kernels are launched with programmatic stream serialisation and let the
 *    next kernel be scheduled before they finish; an ordinary launch after a
 *    call is ordered as usual, but a kernel of the caller's that is itself
 *    launched with programmatic serialisation must wait for its grid
 *    dependency (griddepcontrol.wait) before it reads what the call wrote.
 *  - A solution x is bit-packed: W = ceil(n/64) uint64 words, bit j of x is
 *    (x[j/64] >> (j%64)) & 1.  A batch of S solutions is S*W words, solution s
 *    at X[s*W].  Bits >= n ("pad bits") must be 0; every routine that reads
 *    solutions ignores them and every routine that writes solutions clears them.
 *  - Return value: UBQP_OK or a negative ubqp_status.  Argument errors are
 *    reported synchronously, before any work is enqueued.  A failed launch
 *    returns UBQP_ERR_CUDA.  Errors found by a kernel while it runs (a wait
 *    that timed out) are recorded in the handle and returned by the next
 *    ubqp_sync() on that handle.  ubqp_last_error() gives a one-line detail of
 *    the last failure on the calling thread.
 *  - Exactness: the evaluation runs on the tensor cores in bf16 x bf16 -> fp32,
 *    exact because every operand is an integer of magnitude <= 256 and every
 *    partial sum an integer below 2^24.  ubqp_eval checks this bound at run time
 *    (2 * max|Q| * n_pad < 2^24) and returns UBQP_ERR_RANGE when it fails.
 */
#ifndef UBQP_H
#define UBQP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define UBQP_ABI_VERSION 5

typedef enum ubqp_status {
  UBQP_OK = 0,
  UBQP_ERR_ARG = -1,           /* bad pointer, size, alignment or flag            */
  UBQP_ERR_NOT_SYMMETRIC = -2, /* Q is not symmetric (problem (P))               */
  UBQP_ERR_RANGE = -3,         /* the exactness bound of the evaluation fails     */
  UBQP_ERR_NOMEM = -4,         /* device allocation failed / workspace too small  */
  UBQP_ERR_CUDA = -5,          /* a CUDA runtime call or launch failed            */
  UBQP_ERR_TIMEOUT = -6,       /* a kernel's bounded wait expired                 */
  UBQP_ERR_UNSUPPORTED = -7    /* size or mode this build does not handle         */
} ubqp_status;

/* Start generation modes (see ubqp_diversify). */
enum { UBQP_MODE_RANDOM = 0, UBQP_MODE_DIVERSIFY = 1 };
/* Evaluation paths (see ubqp_eval). */
enum {
  UBQP_EVAL_AUTO = 0,
  UBQP_EVAL_TC = 1,
  UBQP_EVAL_PLAIN = 2,
  UBQP_EVAL_TC_STAGED = 3,
  UBQP_EVAL_TC_TMEM = 4
};

/* Opaque prepared instance: device-resident Q in the layouts the kernels use,
 * its row sums, max|Q|, the first-derivative start and an error word. */
typedef struct ubqp_q ubqp_q;

/* Static description of an error code; never NULL. */
const char* ubqp_strerror(int status);
/* Detail of the last failing call on this thread ("" if none). */
const char* ubqp_last_error(void);
/* UBQP_ABI_VERSION of the loaded library. */
int ubqp_abi_version(void);

/*
 * ubqp_q_prepare -- copy Q to the device once (the one large host/device
 * transfer of Fig. 2's MoveQtoGPU, Pseudocode section) and prepare it.
 *   Q_dev   n rows of int8 coefficients, row stride ldq >= n bytes, in device
 *           memory or in page-locked host memory (cudaHostAlloc or
 *           cudaHostRegister), which the preparing kernel then reads in place
 *           over the host link instead of a separate copy; pageable host
 *           memory is rejected (UBQP_ERR_ARG).  Bytes beyond column n of a row
 *           are ignored.  Not retained.
 *   n       1 <= n <= 16384.
 *   out     receives the handle (NULL on failure).
 * Checks that Q is symmetric (UBQP_ERR_NOT_SYMMETRIC otherwise), records max|Q|,
 * builds the padded int8 copy used by the ascent, the tensor-core operands
 * (bf16: Q' for ubqp_eval, Q for the ascent's start-up), the row sums and the
 * first-derivative start.  Allocates about n_pad^2 * 5 bytes of device memory
 * (n_pad = n rounded up to 1024) owned by the handle.  Synchronises `stream`
 * once to read the validation result.
 */
int ubqp_q_prepare(const int8_t* Q_dev, int32_t n, int64_t ldq, void* stream,
                   ubqp_q** out);
/* Free a handle (NULL is a no-op).  Work using it must have completed. */
void ubqp_q_destroy(ubqp_q* q);
/* ubqp_q_prepare into caller device memory: `arena` (256-byte aligned, at
 * least ubqp_q_arena_size(n) bytes) receives every device buffer of the handle,
 * so the call makes no device allocation; the arena must outlive the handle,
 * whose ubqp_q_destroy then frees host memory only.  Same checks, same
 * synchronisation as ubqp_q_prepare. */
size_t ubqp_q_arena_size(int32_t n);
int ubqp_q_prepare_into(const int8_t* Q_dev, int32_t n, int64_t ldq, void* arena,
                        size_t arena_bytes, void* stream, ubqp_q** out);
/* ubqp_q_prepare_into without the synchronisation: the preparation is only
 * enqueued on `stream` and the handle returned at once, so the host can go on
 * (e.g. prepare the next instance while the current one is solved).  Argument
 * errors return synchronously as before; the symmetry check and max|Q| are
 * read by the first ubqp_sync on the handle: it returns UBQP_ERR_NOT_SYMMETRIC
 * for an asymmetric Q, and so does every later ubqp_sync (whatever ran on the
 * handle in between computed on the asymmetric Q and is meaningless).  Until
 * then ubqp_q_info reports max_abs = -1 and the exactness checks assume the
 * int8 bound 128.  Work on another stream must be ordered after `stream`, and
 * the stream given to that first ubqp_sync must be `stream` or one ordered
 * after it.  Q_dev must not change until the preparation has run. */
int ubqp_q_prepare_into_async(const int8_t* Q_dev, int32_t n, int64_t ldq, void* arena,
                              size_t arena_bytes, void* stream, ubqp_q** out);
/* Size and layout of a prepared instance; any output pointer may be NULL.
 * n_pad is the padded row stride of the device copies. */
int ubqp_q_info(const ubqp_q* q, int32_t* n, int32_t* words, int32_t* n_pad,
                int32_t* max_abs, int64_t* device_bytes);
/* Synchronise `stream` and report (then clear) any error a kernel recorded in
 * the handle's error word since the last ubqp_sync; the reads and the reset
 * run on `stream`, so work queued on other streams (the next solve, say) is
 * not waited for.  For a handle from
 * ubqp_q_prepare_into_async the first call also reads the symmetry check and
 * max|Q|; an asymmetric Q gives UBQP_ERR_NOT_SYMMETRIC from then on. */
int ubqp_sync(const ubqp_q* q, void* stream);

/*
 * ubqp_first_derivative -- CalculateFirstDerivativeSolution (Fig. 2): the
 * start with x_i = 1 iff sum_j Q_ij > 0 (a zero sum gives x_i = 0).  Copies the
 * handle's precomputed start (W words) to x0_dev.  Async on `stream`.
 */
int ubqp_first_derivative(const ubqp_q* q, uint64_t* x0_dev, void* stream);

/*
 * ubqp_diversify -- S starts, written to X_dev (S*W words).  Async.
 *   mode UBQP_MODE_RANDOM: uniform random solutions (the sample of
 *        EvaluateRandomStarts, Fig. 2): word w of start s is
 *        splitmix64(seed ^ s*0x9E3779B97F4A7C15 ^ w), pad bits cleared.
 *   mode UBQP_MODE_DIVERSIFY: Diversify(x, best, i, Q_cols) of Fig. 2 around
 *        the incumbent x0_dev (NULL = the first-derivative start).  Start s has
 *        loop counter i = round*S + s: i = 0 is the incumbent, even i flips every
 *        bit p with p mod h == o (Glover's h-pattern; j' = i/2, H = min(n,
 *        div_H), h = 1 + (j'-1) mod H, o = ((j'-1)/H) mod h), odd i blends the
 *        incumbent with a random partner through the AND of 1 + ((i-1)/2 mod 6)
 *        random mask words.  div_H >= 1.
 * SplitMix64 is the generator of Steele, Lea & Flood (2014).
 */
int ubqp_diversify(const ubqp_q* q, const uint64_t* x0_dev, int32_t mode,
                   uint64_t seed, uint64_t round, int64_t S, int32_t div_H,
                   uint64_t* X_dev, void* stream);
/* Starts s_begin .. s_begin+S_local-1 of a batch of S_total (loop counters
 * round*S_total + s, RANDOM streams s), written to X_dev[0 .. S_local*W): the
 * slice of ubqp_diversify's output that one rank of a sharded batch needs. */
int ubqp_diversify_range(const ubqp_q* q, const uint64_t* x0_dev, int32_t mode,
                         uint64_t seed, uint64_t round, int64_t S_total,
                         int64_t s_begin, int64_t S_local, int32_t div_H,
                         uint64_t* X_dev, void* stream);

/*
 * ubqp_eval -- Evaluate(x) of Fig. 2 for a batch: f_dev[s] = x_s^t Q x_s (int64),
 * s < S.  Async.
 *   path UBQP_EVAL_TC: tensor-core contraction.  With Q' = 2*tril(Q,-1) +
 *        diag(Q), f = sum_j x_j sum_{k<=j} Q'_jk x_k, so only the lower block
 *        triangle of X * Q'^t is formed (tcgen05 kind::f16, bf16 operands,
 *        fp32 accumulation in tensor memory, exact), and an int64 epilogue
 *        folds the row-dot with x without writing the product.  The 0/1
 *        operand is built in shared memory straight from the bit-packed
 *        solutions; needs no workspace.
 *   path UBQP_EVAL_TC_STAGED: the same contraction with the solutions first
 *        unpacked to bf16 in device scratch and both operands fed by TMA;
 *        needs ws_bytes >= ubqp_eval_workspace_size(q, S, path) (16-byte
 *        aligned).
 *   path UBQP_EVAL_TC_TMEM: the same contraction with the 0/1 operand
 *        written into tensor memory (tcgen05.st) straight from the bits and
 *        read from there by the MMA (192-column blocks), so shared memory
 *        carries only Q'; needs no workspace.
 *   path UBQP_EVAL_PLAIN: one block per solution on the CUDA cores (dp4a);
 *        needs no workspace.
 *   path UBQP_EVAL_AUTO: UBQP_EVAL_TC_STAGED, except UBQP_EVAL_TC for
 *        n_pad <= 1024 (n rounded up to 256) with S >= 4096 (the faster of
 *        the two, measured).
 * Returns UBQP_ERR_RANGE if the exactness bound fails (see top of file).
 */
size_t ubqp_eval_workspace_size(const ubqp_q* q, int64_t S, int32_t path);
int ubqp_eval(const ubqp_q* q, const uint64_t* X_dev, int64_t S, int64_t* f_dev,
              int32_t path, void* ws, size_t ws_bytes, void* stream);

/*
 * ubqp_eval_noalloc -- the staged tensor-core evaluation of ubqp_eval
 * (UBQP_EVAL_TC_STAGED; same results, bit for bit) for callers that cannot
 * allocate device memory or hand the library a workspace: for example a host whose device memory is entirely
 * reserved by another allocator (a framework's caching pool, an application
 * with a fixed memory budget), or a latency-critical loop that must not run
 * cudaMalloc/cudaFree, which can synchronise the whole device.  The paper has
 * no counterpart; this is an interface convenience only.
 *   The scratch for the unpacked solutions is a static device array of
 *   UBQP_EVAL_NOALLOC_MAX_BYTES built into the library.  CUDA places it on a
 *   device when it loads the library's evaluation module there, which with
 *   CUDA's default lazy module loading is the first evaluation (any path) or
 *   the first call of this entry point on that device -- not the loading of
 *   the library -- and it stays there until the process exits.  A caller that
 *   is about to hand the rest of a device's memory to another allocator should
 *   therefore make one call (or one ubqp_q_prepare and ubqp_eval) first.
 *   A call needs ceil(S/128)*128 * n_tc * 2 bytes of it (n_tc = n rounded up
 *   to 256); larger requests return UBQP_ERR_UNSUPPORTED (e.g. 1000 starts fit
 *   up to n = 8192, which uses all of it).  The call allocates nothing and
 *   calls no cudaMalloc/cudaFree.  The array's device address is looked up
 *   (cudaGetSymbolAddress) with the device current on the first call in each
 *   CUDA context of a device (again after a cudaDeviceReset); make that first
 *   call before any stream capture.  All calls share the one array and it
 *   keeps the last call's contents (each call overwrites the part it uses):
 *   calls whose work overlaps on the GPU -- concurrent streams, or several
 *   host threads -- race on it and must be serialised by the caller.  Async
 *   on `stream`.
 */
#define UBQP_EVAL_NOALLOC_MAX_BYTES (16u << 20)
int ubqp_eval_noalloc(const ubqp_q* q, const uint64_t* X_dev, int64_t S,
                      int64_t* f_dev, void* stream);

/*
 * ubqp_screen -- the screening function of the Pseudocode section,
 * T(lambda) = Mean + lambda (Max - Mean), Mean and Max over the S values f_dev,
 * and the pass test f_b > T of Fig. 2 (strict).  Async.
 *   idx_dev     S int32: the passing indices, ascending, in idx_dev[0..count).
 *   count_dev   1 int64: their number.
 *   Tm_dev      2 doubles: {T, Mean}.
 *   stats_dev   3 int64: {sum of f, Max, lowest index attaining Max}.
 * The sum is exact in int64; Mean = sum / S, then T = Mean + lambda*(Max - Mean)
 * as one subtraction, one multiplication and one addition in double, each
 * rounded to nearest (no fused multiply-add).  Requires 1 <= S < 2^31.
 */
int ubqp_screen(const int64_t* f_dev, int64_t S, double lambda, int32_t* idx_dev,
                int64_t* count_dev, double* Tm_dev, int64_t* stats_dev,
                void* stream);

/*
 * The screen in two steps, for a batch sharded over several ranks (each rank
 * holding a contiguous range of the starts):
 * ubqp_screen_stats -- stats_dev (3 int64) = {sum of f, Max, lowest index
 *   attaining Max + offset} over this rank's S values (offset = the global
 *   index of its first start).  The ranks combine these exactly (sum: add;
 *   Max: max; index: the lowest among the ranks attaining the global Max).
 * ubqp_screen_apply -- with the combined gstats_dev {sum, Max, ...} of all
 *   S_total starts: Tm_dev = {T, Mean} computed as in ubqp_screen with
 *   Mean = sum / S_total (every rank obtains the identical T), then the passing
 *   local indices of this rank's f_dev, ascending, in idx_dev[0 .. *count_dev).
 *   (ubqp_search uses it with the random sample's sum and size and the
 *   incumbent's value as Max.)
 * ubqp_screen is ubqp_screen_stats (offset 0) followed by ubqp_screen_apply
 * with S_total = S.  Both async.
 */
int ubqp_screen_stats(const int64_t* f_dev, int64_t S, int64_t offset,
                      int64_t* stats_dev, void* stream);
int ubqp_screen_apply(const int64_t* f_dev, int64_t S, const int64_t* gstats_dev,
                      int64_t S_total, double lambda, int32_t* idx_dev,
                      int64_t* count_dev, double* Tm_dev, void* stream);

/*
 * ubqp_ascent -- PerformSteepestAscent(x, xQx, max_its) of Fig. 2 for the
 * solutions X_dev[idx_dev[t]], t < *count_dev, in place: repeatedly flip the
 * bit with the largest 1-flip gain Delta_i = Q_ii + 2(1-2x_i)(Qx)_i (Glover et
 * al. 2002), lowest index on ties, while that gain is > 0 and fewer than
 * max_flips flips were made (max_flips 0 = no cap).  f_dev[s] must hold
 * f(x_s) on entry and holds the ascended value on exit.  flips_dev (S int32,
 * may be NULL) receives each ascended start's flip count; entries of starts
 * not listed are left untouched.  The indices must be distinct and in [0, S)
 * (an index outside is skipped and reported by ubqp_sync).  count is read on
 * the device (no sync).  S is the length of X_dev/f_dev.  Async.
 *   ws / ws_bytes: device scratch (16-byte aligned) of at least
 *   ubqp_ascent_workspace_size(q, S) bytes lets the start-up y = Q x of all
 *   listed starts run as one tensor-core product (bf16 Q, fp32 accumulation,
 *   exact), and the groups take the listed starts one at a time from a
 *   counter there as they finish (so long and short climbs even out over the
 *   SMs); with ws NULL or smaller the start-up sums the rows of Q on the CUDA
 *   cores and the starts are dealt round robin.  Results are identical either
 *   way.
 */
size_t ubqp_ascent_workspace_size(const ubqp_q* q, int64_t S);
int ubqp_ascent(const ubqp_q* q, uint64_t* X_dev, int64_t* f_dev,
                const int32_t* idx_dev, const int64_t* count_dev, int64_t S,
                int32_t max_flips, int32_t* flips_dev, void* ws, size_t ws_bytes,
                void* stream);
/*
 * ubqp_ascent_trace -- ubqp_ascent with a record of its moves: the same climb
 * (identical X, f and flips), and the flipped indices of each listed start s,
 * in the order PerformSteepestAscent of Fig. 2 takes them (largest 1-flip gain,
 * lowest index on ties), written to trace_dev[s*ldt + t] for t < min(flips,
 * ldt).  Moves beyond ldt are made but not recorded; entries at or beyond a
 * start's flip count and the rows of starts not listed are left untouched.
 *   trace_dev  S rows of ldt uint16 (n <= 16384 < 2^16), device memory.
 *   ldt        >= 1; a row of n entries records every move of a start that
 *              flips each variable at most once, 4n is ample in practice.
 * Same arguments, workspace and errors otherwise (UBQP_ERR_ARG: trace_dev NULL
 * or ldt < 1).  A testing and analysis aid: the record costs one store per move.
 */
int ubqp_ascent_trace(const ubqp_q* q, uint64_t* X_dev, int64_t* f_dev,
                      const int32_t* idx_dev, const int64_t* count_dev, int64_t S,
                      int32_t max_flips, int32_t* flips_dev, uint16_t* trace_dev,
                      int64_t ldt, void* ws, size_t ws_bytes, void* stream);

/*
 * ubqp_best -- UpdateBestAndT's bookkeeping (Fig. 2): the largest of the S
 * values f_dev, the lowest index on ties.  Writes best_f_dev[0] = value,
 * best_f_dev[1] = index and copies that solution's W words to best_x_dev.  Async.
 */
int ubqp_best(const int64_t* f_dev, const uint64_t* X_dev, int64_t S,
              int32_t words, uint64_t* best_x_dev, int64_t* best_f_dev,
              void* stream);

/* One round of the loop body of Fig. 2 over a batch of starts. */
typedef struct ubqp_params {
  int64_t num_starts; /* S >= 1                                            */
  double lambda;      /* screening parameter                                */
  int32_t max_flips;  /* ascent cap per start, 0 = none                     */
  int32_t mode;       /* UBQP_MODE_RANDOM or UBQP_MODE_DIVERSIFY            */
  uint64_t seed;      /* start-generation seed                              */
  uint64_t round;     /* loop-counter offset: start s has i = round*S + s   */
  int32_t div_H;      /* h-pattern period bound (>= 1; 64 is customary)     */
  int32_t eval_path;  /* UBQP_EVAL_*                                         */
} ubqp_params;

typedef struct ubqp_stats {
  int64_t passed;         /* starts that passed the screen                 */
  int64_t total_flips;    /* flips over all ascended starts                */
  int64_t max_flips_seen; /* largest flip count of one start               */
  int64_t batch_max;      /* Max of the screen (before ascent)             */
  int64_t best_index;     /* start that gave the best solution             */
  int64_t sum;            /* sum of evaluated f (before ascent)            */
  double T;               /* screening threshold                           */
  double mean;            /* Mean of the screen                            */
} ubqp_stats;

/*
 * ubqp_solve -- one round on one stream with no host round trip: starts from
 * the first-derivative solution (ubqp_diversify with x0 = NULL), ubqp_eval,
 * ubqp_screen, ubqp_ascent of the passing starts, ubqp_best.  Writes best_x_dev
 * (W words) and best_f_dev[0..1] = {best f, start index}.  ws must hold
 * ubqp_solve_workspace_size(q, p) bytes (16-byte aligned).  If stats_host is
 * not NULL the call synchronises `stream`, fills it and also reports any
 * kernel-recorded error (as ubqp_sync does); otherwise it is fully async.
 */
size_t ubqp_solve_workspace_size(const ubqp_q* q, const ubqp_params* p);
int ubqp_solve(const ubqp_q* q, const ubqp_params* p, uint64_t* best_x_dev,
               int64_t* best_f_dev, ubqp_stats* stats_host, void* ws,
               size_t ws_bytes, void* stream);

/*
 * ubqp_solve_rounds -- R independent rounds of ubqp_solve on one instance, run
 * together.  Round k is ubqp_solve with seed p->seed + k and loop-counter
 * offset p->round + k: its own S starts, its own screen T(lambda) over its own
 * S values, its own climbs and best, and its result is bit-identical to that
 * call.  Together means one evaluation launch over the R*S starts and one
 * climb launch over the passing starts of every round, so the SMs that one
 * round's few passing starts leave idle climb the other rounds' (at n = 7000
 * about 54 of 1000 random starts pass, one chain per SM on a 152-SM GPU).
 *   R           1 .. 1024, with R * num_starts < 2^31.
 *   best_x_dev  R*W words: round k's best solution at k*W.
 *   best_f_dev  2R int64: round k's {best value, start index within the
 *               round} at 2k.
 *   ws          ubqp_solve_rounds_workspace_size(q, p, R) bytes (16-byte
 *               aligned; 0 for invalid arguments).
 * Fully async on `stream`.  The paper runs its rounds one after another, each
 * from the incumbent of the last (ubqp_search); independent rounds, the
 * multi-start of the paper restarted with fresh seeds, have no such order.
 */
size_t ubqp_solve_rounds_workspace_size(const ubqp_q* q, const ubqp_params* p, int32_t R);
int ubqp_solve_rounds(const ubqp_q* q, const ubqp_params* p, int32_t R, uint64_t* best_x_dev,
                      int64_t* best_f_dev, void* ws, size_t ws_bytes, void* stream);

/*
 * Batches of instances: one round (as ubqp_solve, with the same parameters) for
 * every instance of a batch of uneven n, run together.  Start generation and
 * the tensor-core evaluation are one launch each for all instances (the
 * evaluation one persistent launch over the work units of every instance) or,
 * as the tuner decides, per-instance launches on internal streams; the
 * screen, the ascent of every passing start of every instance (one persistent
 * launch, largest instances first) and the best-of are one launch each; the
 * start-up products y = Q x of the passing starts run per instance on the
 * internal streams.  Each instance's result is bit-identical to ubqp_solve on
 * that instance alone.
 *
 * ubqp_batch_create -- plan a batch over `count` prepared instances (all on the
 *   current device; the handles must outlive the plan).  Allocates the plan's
 *   device memory (workspace, results, descriptors) and internal streams.
 * ubqp_batch_run -- one round for all instances with start-generation seed
 *   `seed` (replaces p->seed), async on `stream`; launches the captured graph
 *   when there is one.
 * ubqp_batch_tune -- the autotuner: times the run for the candidate ascent
 *   group shapes (threads x chunks that hold the largest n, one start per
 *   group, or packed: 256-thread blocks climbing up to eight starts at once
 *   in sub-groups of 32, 64, 128 or 256 threads, the smallest that holds the
 *   instance's n, each taking its next start as soon as its climb ends; the
 *   instances too large for half a block climb in launches of their own
 *   beside it), the
 *   evaluation paths, one merged launch for the start generation and the
 *   tensor-core evaluation of all instances (one persistent launch over the
 *   work units of every instance, largest first) or one launch per instance,
 *   the evaluation's schedule (at most 16, 12 or 8 K steps of 64 per work
 *   chunk) and the fork/join stream counts on this batch and keeps the
 *   fastest; drops a captured graph.  Synchronises `stream`.
 * ubqp_batch_capture -- records one run into a CUDA graph (after one plain
 *   run); later ubqp_batch_run calls replay it.  Synchronises `stream`.
 * ubqp_batch_result -- device pointers to instance i's best solution (W words)
 *   and {value, start index} (2 int64), valid after the run completes.
 * ubqp_batch_config -- the configuration in use (any pointer may be NULL).
 * ubqp_batch_schedule -- the rest of it: *packed = 1 when the climb is packed,
 *   *eval_kch = the K steps per evaluation work chunk, *eval_merged = 1 when
 *   start generation and the evaluation of all instances are one launch each
 *   (any pointer may be NULL).
 * ubqp_batch_set -- pin the configuration instead of tuning it: ascent group
 *   shape (threads x chunks; packed: 256 x 1 or 256 x 2, else 64..512 x 1..2,
 *   holding the largest n), packed 0/1, eval_kch 8, 12 or 16, eval_merged 0/1
 *   (1 needs the tensor-core evaluation); drops a captured graph.
 *   UBQP_ERR_UNSUPPORTED for a shape that is not built or cannot hold the
 *   largest n, or a merged evaluation without the tensor-core path.
 * The paper runs one instance at a time; batching is this library's addition.
 */
typedef struct ubqp_batch ubqp_batch;
int ubqp_batch_create(const ubqp_q* const* qs, int32_t count, const ubqp_params* p,
                      ubqp_batch** out);
void ubqp_batch_destroy(ubqp_batch* b);
int ubqp_batch_run(ubqp_batch* b, uint64_t seed, void* stream);
int ubqp_batch_tune(ubqp_batch* b, void* stream);
int ubqp_batch_capture(ubqp_batch* b, void* stream);
int ubqp_batch_result(const ubqp_batch* b, int32_t i, const uint64_t** best_x_dev,
                      const int64_t** best_f_dev);
int ubqp_batch_config(const ubqp_batch* b, int32_t* asc_threads, int32_t* asc_chunks,
                      int32_t* eval_path, int32_t* streams, int32_t* graph);
int ubqp_batch_schedule(const ubqp_batch* b, int32_t* packed, int32_t* eval_kch,
                        int32_t* eval_merged);
int ubqp_batch_set(ubqp_batch* b, int32_t asc_threads, int32_t asc_chunks, int32_t packed,
                   int32_t eval_kch, int32_t eval_merged);
/* Copies instance i's result to caller memory (W words, 2 int64), async. */
int ubqp_batch_get(const ubqp_batch* b, int32_t i, uint64_t* best_x_dev, int64_t* best_f_dev,
                   void* stream);

/*
 * Serving: a request loop that solves instances as they arrive, with
 * continuous batching.  A request is one instance (host coefficients) solved
 * by one round with the server's parameters and its own seed; the result is
 * bit-identical to ubqp_solve on that instance alone.  The server runs
 * `workers` lanes (threads with their own CUDA streams).  A free lane admits,
 * in arrival order, every waiting request that fits -- up to max_batch
 * requests whose device memory fits the budget -- and runs them as one batch:
 * per-request upload, preparation, start generation and evaluation on the
 * lane's streams, then one shared launch each for the screen, the climb of
 * every passing start of every request (one persistent launch, several small
 * starts per block; requests too large for half a block climb in launches of
 * their own beside it) and the best-of.  Requests that arrive while batches run
 * are taken together by the next free lane, so batches grow with the load,
 * and the lanes' batches overlap on the GPU.  Request memory comes from the
 * device's stream-ordered pool.  The paper solves one instance per run;
 * serving is this library's addition.
 *   memory_budget  device bytes the server's requests may hold together
 *                  (0 = workers x the bytes of a max_n request); a request
 *                  larger than the budget still runs, alone.
 *   max_batch      requests one lane runs together (0 = 16; at most 1024).
 * ubqp_server_submit -- enqueue (returns at once with a ticket).  Q_host: n rows
 *   of ldq int8 coefficients in host memory that must stay valid until the
 *   request completes (pinned memory makes the upload asynchronous).  n above
 *   max_n returns UBQP_ERR_UNSUPPORTED.
 * ubqp_server_wait -- block until the ticket completes, then return
 *   best_f[0..1] = {value, start index}, best_x_host (W words, may be NULL) and
 *   the submit-to-completion latency in seconds; releases the ticket.
 * ubqp_server_poll -- *done = 1 when the ticket has completed.
 * ubqp_server_destroy -- finish every queued request, stop the workers.
 */
typedef struct ubqp_server ubqp_server;
typedef struct ubqp_server_config {
  int32_t workers;        /* lanes: concurrent batches (threads, streams), 1..64 */
  int32_t max_n;          /* largest n accepted                                  */
  int64_t memory_budget;  /* device bytes, 0 = derived                           */
  ubqp_params params;     /* round parameters (seed comes from each request)     */
  int32_t max_batch;      /* requests per batch, 0 = 16                          */
} ubqp_server_config;
int ubqp_server_create(const ubqp_server_config* cfg, ubqp_server** out);
int ubqp_server_submit(ubqp_server* s, const int8_t* Q_host, int32_t n, int64_t ldq,
                       uint64_t seed, int64_t* ticket);
int ubqp_server_wait(ubqp_server* s, int64_t ticket, int64_t* best_f, uint64_t* best_x_host,
                     double* latency_s);
int ubqp_server_poll(ubqp_server* s, int64_t ticket, int32_t* done);
size_t ubqp_server_request_bytes(const ubqp_server* s, int32_t n);
void ubqp_server_destroy(ubqp_server* s);
/* Batches run so far, the requests they held and the largest batch (any
 * pointer may NULL). */
int ubqp_server_stats(ubqp_server* s, int64_t* batches, int64_t* requests, int64_t* largest);
/* Fault injection (tests): the next `count` admitted requests fail as if their
 * device allocation had failed -- they complete with UBQP_ERR_NOMEM from
 * ubqp_server_wait, nothing is launched for them, and the server keeps
 * serving the requests after them. */
int ubqp_server_inject_alloc_failures(ubqp_server* s, int32_t count);

/*
 * ubqp_selftest_timeout -- checks the bounded-wait mechanism every kernel wait
 * of this library uses: one block waits on a shared-memory mbarrier phase that
 * nothing completes, gives up after `limit_us` microseconds (1 .. 1e6),
 * records UBQP_ERR_TIMEOUT in *status_dev (int32, device) and returns.
 * Synchronises `stream` and returns the status it read, so the expected result
 * is UBQP_ERR_TIMEOUT with the context still usable afterwards.
 */
int ubqp_selftest_timeout(uint32_t limit_us, int32_t* status_dev, void* stream);

/*
 * Path relinking (intensification).  The Experiments section names path
 * relinking as the polishing phase to follow the multi-start phase, and the
 * Conclusions find the method short of intensification; Fig. 1's concepts
 * come from Glover's (1998) template, whose second phase it is.  For each pair
 * p < P: from the initiating solution X_dev[p] (value f_dev[p], as from
 * ubqp_eval) toward the guiding solution G_dev[p], flip at each step, among the
 * variables where the two still differ, the one of largest 1-flip gain
 * Q_kk + 2 (1 - 2 x_k) y_k (lowest index on ties; negative gains are taken
 * too), until the two agree.  Xbest_dev[p] (W words) receives the best solution
 * strictly between the endpoints (the earliest on ties) and fbest_dev[p] its
 * value; when the pair differs in fewer than 2 variables there is none and the
 * result is X_dev[p] itself.  dist_dev[p] (may be NULL) receives the Hamming
 * distance.  The results are typically polished with ubqp_ascent.
 *   ws: at least ubqp_relink_workspace_size(q, P, 0) bytes (16-byte aligned;
 *   a trace of the flipped indices); with ubqp_relink_workspace_size(q, P, 1)
 *   bytes y = Qx of the initiating solutions is formed on the tensor cores.
 *   Async on `stream`; errors as ubqp_ascent (UBQP_ERR_NOMEM: ws too small).
 */
size_t ubqp_relink_workspace_size(const ubqp_q* q, int64_t P, int32_t tensor_startup);
int ubqp_relink(const ubqp_q* q, const uint64_t* X_dev, const int64_t* f_dev,
                const uint64_t* G_dev, int64_t P, uint64_t* Xbest_dev, int64_t* fbest_dev,
                int32_t* dist_dev, void* ws, size_t ws_bytes, void* stream);

/* The search of Fig. 2, run in rounds of starts_per_round starts. */
typedef struct ubqp_search_params {
  int64_t num_samples;      /* random solutions behind Mean (EvaluateRandomStarts) */
  int64_t starts_per_round; /* S: starts per round (the loop body on a batch)      */
  int32_t rounds;           /* rounds; loop counters run 0 .. rounds*S - 1         */
  int32_t max_flips;        /* ascent cap per start, 0 = none                      */
  double lambda;            /* screening parameter                                 */
  uint64_t seed;            /* seed of the sample and of the diversification       */
  int32_t div_H;            /* h-pattern period bound (>= 1)                       */
  int32_t eval_path;        /* UBQP_EVAL_*                                          */
} ubqp_search_params;

/*
 * ubqp_search -- the whole loop of Fig. 2 on the device, batched by rounds:
 * Mean = mean of num_samples uniform random solutions (EvaluateRandomStarts);
 * the incumbent starts as the first-derivative solution, whose value is the
 * first Max (CalculateFirstDerivativeSolution, CalculateT).  Round r
 * diversifies starts_per_round starts around the current incumbent (loop
 * counters r*S + s, as ubqp_diversify), evaluates them, screens them with
 * T = Mean + lambda (Max - Mean) where Max is the incumbent's value, climbs
 * every start above T, and replaces the incumbent by the round's best when
 * that is strictly better (UpdateBestAndT).  Within a round the incumbent and
 * T are fixed.  Outputs (device): best_x_dev (W words), best_f_dev[0] (its
 * value; 1 int64), history_dev[r] = incumbent value after round r (rounds
 * int64), stats_dev = {starts that passed, flips, sum over the sample}
 * (3 int64).  No host round trip: fully async on `stream`.  ws must hold
 * ubqp_search_workspace_size(q, p) bytes (16-byte aligned).  Errors:
 * UBQP_ERR_ARG for a NULL pointer, counts out of range or a lambda that is not
 * finite; UBQP_ERR_NOMEM for a short workspace.
 */
size_t ubqp_search_workspace_size(const ubqp_q* q, const ubqp_search_params* p);
int ubqp_search(const ubqp_q* q, const ubqp_search_params* p, uint64_t* best_x_dev,
                int64_t* best_f_dev, int64_t* history_dev, int64_t* stats_dev,
                void* ws, size_t ws_bytes, void* stream);
/*
 * ubqp_search_resume -- checkpoint/resume of the search: continues a search
 * whose state is (best_x_dev, best_f_dev[0], stats_dev[0..2]) as ubqp_search or
 * an earlier resumption left it, running rounds first_round .. first_round +
 * p->rounds - 1 (loop counters as ubqp_search's) with the same parameters; the
 * state is updated in place (stats accumulate; stats_dev[2], the sample sum
 * behind Mean, is read, not recomputed) and history_dev[i] gets the incumbent
 * value after round first_round + i.  ubqp_search with R1 + R2 rounds equals
 * ubqp_search with R1 rounds followed by this call with first_round R1 and
 * R2 rounds, bit for bit.  Same workspace and errors as ubqp_search.
 */
int ubqp_search_resume(const ubqp_q* q, const ubqp_search_params* p, int32_t first_round,
                       uint64_t* best_x_dev, int64_t* best_f_dev, int64_t* history_dev,
                       int64_t* stats_dev, void* ws, size_t ws_bytes, void* stream);

/*
 * Measurement helpers: the two rates the ascent's roofline is made of, measured
 * on the device the library runs on (not part of the method; the paper has no
 * counterpart).  The steepest ascent reads one int8 row of Q (n bytes) per move
 * from L2 and does about 3n integer operations per move (the gain update, the
 * key and the comparison of each element), so its moves/s are bounded by
 * min(L2 read rate / n, integer rate / 3n).  Each call only enqueues one
 * kernel on `stream`; the caller times it (CUDA events) and divides.
 * ubqp_peak_l2_read -- `reps` passes of 16-byte reads (cached in L2, not L1)
 *   over the caller's device buffer (16-byte aligned, `bytes` >= 16; a buffer
 *   well below the L2 size stays resident there after the first pass), every
 *   SM taking part.  Bytes read = reps * (bytes rounded down to 16).
 *   sink_dev: one uint32 of device memory, written only for a buffer whose
 *   words xor to a particular value (use a zero-filled buffer).
 * ubqp_peak_int32 -- kind 0: independent int32 multiply-add chains (the int32
 *   instruction rate); kind 1: the ascent's per-element update (dp4a gain
 *   update, multiply-add key, three-way max), counted as 3 operations per
 *   element.  ubqp_peak_int32_ops gives the operations one call performs on
 *   the current device (0 for bad arguments).
 */
int ubqp_peak_l2_read(const void* buf_dev, size_t bytes, int32_t reps, uint32_t* sink_dev,
                      void* stream);
int64_t ubqp_peak_int32_ops(int32_t kind, int64_t iters);
int ubqp_peak_int32(int32_t kind, int64_t iters, uint32_t* sink_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* UBQP_H */
