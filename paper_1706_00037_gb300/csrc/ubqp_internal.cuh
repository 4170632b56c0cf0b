// ubqp_internal.cuh -- types and launchers shared by the translation units of
// libubqp.  Not part of the public ABI (include/ubqp.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ubqp.h"

#define UBQP_ROW_ALIGN 1024  // row stride of the int8 copy (ascent rows)
#define UBQP_TC_ALIGN 256    // padding of the tensor-core operand
#define UBQP_MAX_N 16384

// Error word bits recorded by kernels (cleared by ubqp_sync).
#define UBQP_DEVERR_TIMEOUT 1u
#define UBQP_DEVERR_BADIDX 2u

struct ubqp_q {
  int32_t n;        // variables
  int32_t W;        // words per solution
  int64_t ldq;      // row stride of Q8 (multiple of UBQP_ROW_ALIGN)
  int32_t n_tc;     // n rounded up to UBQP_TC_ALIGN (rows/cols of Qt)
  int32_t max_abs;  // max |Q_ij|; -1 while a deferred validation is unread
  int8_t* Q8;       // n x ldq int8, zero beyond column n
  uint16_t* Qt;     // n_tc x n_tc bf16 bits of Q' = 2 tril(Q,-1) + diag(Q); only the
                    // tiles the evaluation reads (row j: columns below the end of
                    // its 256- and 192-row blocks) are written
  uint16_t* Qu;     // n_tc x n_tc bf16 bits of Q'^t = 2 triu(Q,1) + diag(Q); only the
                    // upper block triangle (row j: columns from the start of its
                    // 256-row block) is written.  With Qt it gives the ascent's
                    // start-up y = Q x = (Q' x + Q'^t x) / 2
  int32_t* rowsum;  // n
  uint64_t* x0;     // W words: first-derivative start
  unsigned* err;    // device error word
  unsigned* scratch_flags;  // device: [0] asymmetric count, [1] max |Q|
  int64_t device_bytes;
  int sm_count;
  int device;
  // tensor-core evaluation: work chunks of the lower block triangle (int4
  // {N-block, first K step, K steps, 0}) and the TMA descriptor of Qt
  void* tc_chunks;   // evaluation chunks, the full-square chunks, the 192-column chunks
  int tc_nchunks;
  int tc_nchunks_y;
  int tc_nchunks_ts;  // chunks of the tensor-memory-A evaluation (192-column blocks)
  bool tc_ok;
  bool owns_memory;  // false when the buffers were carved from caller memory
  // deferred validation (ubqp_q_prepare_into_async): the symmetry check and
  // max |Q| stay in scratch_flags until the first ubqp_sync reads them
  mutable bool deferred;
  mutable bool asymmetric;
  alignas(64) unsigned char tc_mapB[128];  // TMA descriptor of Qt
  alignas(64) unsigned char tc_mapU[128];  // TMA descriptor of Qu
  alignas(64) unsigned char tc_mapB_ts[128];  // TMA descriptor of Qt, 192-row boxes
};

#include <nvtx3/nvToolsExt.h>

namespace ubqp {

// The tensor-core evaluation UBQP_EVAL_AUTO takes for S starts of an instance
// padded to n_tc: the fused operand build only for small instances with many
// starts, the staged one otherwise (measured on GB300, L2 flushed: 1000
// starts at n = 2500 staged 19.6 us vs fused 22.2, at n = 7000 51.9 vs 64.2;
// 8192 starts at n = 200 staged 19.1 vs fused 16.0, at n = 1500 36.5 vs 38.0).
// Results are identical either way.
inline bool eval_auto_fused(int n_tc, int64_t S) { return n_tc <= 1024 && S >= 4096; }

// An NVTX range named after the API call, for timeline tools (a no-op
// without one attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define UBQP_RANGE(name) ::ubqp::NvtxRange ubqp_nvtx_range_(name)

// Programmatic dependent launch.  The kernels of one round (start generation,
// unpacking, evaluation, screen, start-up, ascent, best-of) are launched with
// programmatic stream serialisation, so that a kernel's blocks can be
// scheduled while the kernel before it on the stream is still running.  Each
// such kernel calls pdl_wait() before its first access to global memory:
// griddepcontrol.wait returns once the preceding grid has completed and its
// writes are visible (at once for a kernel launched without the attribute).
// pdl_release() (griddepcontrol.launch_dependents) then lets the next kernel
// be scheduled; a kernel that does not call it releases the next one when it
// completes.  Since every kernel of the chain waits before it can finish, each
// one also finishes after everything queued before it, and at most one kernel
// waits while another runs.  The start-up product and the ascent do not
// release early: the ascent hands its first starts to its blocks in launch
// order and relies on the block scheduler spreading them over idle SMs, which
// blocks placed beside a running kernel would not be.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_release();
}

template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

// One instance of a batch (device-resident descriptor of the batched stages).
struct BatchDesc {
  const uint64_t* x0;  // first-derivative start (W words)
  const int8_t* Q8;
  int64_t ldq;
  int n, W;
  int64_t S;
  uint64_t* X;        // S x W starts
  int64_t* f;         // S values
  int32_t* idx;       // S passing indices
  int64_t* count;     // 1
  double* Tm;         // 2: T, Mean
  int64_t* stats;     // 3: sum, max, argmax
  int32_t* flips;     // S
  const float* Y;     // start-up y = Q x (rows = passing starts), or null
  int64_t ldy;
  unsigned* err;
  uint64_t* best_x;   // W
  int64_t* best_f;    // 2: value, index
};

// One instance of a merged evaluation, and a work unit of it: chunk {N-block
// nb, first K step k0, K steps nk} of instance `inst`, m-tile mt.
struct EvalInst {
  const uint64_t* X;
  int64_t* f;
  int64_t S;
  int n, W;
};
struct MUnit {
  int nb, k0, nk, mt, inst, pad0, pad1, pad2;
};
// One instance of a merged start-up product y = Q x of the passing starts:
// its starts, passing list and count, the unpacked rows Xe (A operand,
// S_p x n_tc bf16) and the product Y (S_p x n_tc fp32) in its scratch.
struct YInst {
  const uint64_t* X;
  const int32_t* idx;
  const int64_t* count;
  uint4* Xe;
  float* Y;
  int64_t S, S_p;
  int n, W, n_tc, pad;
};

__host__ __device__ inline int64_t words_of(int64_t n) { return (n + 63) / 64; }

// SplitMix64 (Steele, Lea & Flood 2014): the first output of the sequential
// generator started at `state`.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t state) {
  uint64_t z = state + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t stream_word(uint64_t seed, uint64_t stream,
                                                         uint64_t ctr) {
  return splitmix64(seed ^ (stream * 0x9E3779B97F4A7C15ULL) ^ ctr);
}

// Mask of the valid bits of word w of an n-bit solution.
__host__ __device__ __forceinline__ uint64_t valid_mask(int64_t n, int64_t w) {
  int64_t lo = w * 64;
  if (n >= lo + 64) return ~0ULL;
  if (n <= lo) return 0ULL;
  return (1ULL << (n - lo)) - 1ULL;
}

// Records a one-line detail for ubqp_last_error() and returns status.
int record_error(int status, const char* fmt, ...) __attribute__((format(printf, 2, 3)));

// ---- launchers (each returns cudaError_t of its launch) --------------------
cudaError_t launch_prepare(const int8_t* Q, int n, int64_t ldq_in, ubqp_q* h,
                           cudaStream_t st);
// seed_dev: when not null the seed is read from device memory at run time
// (lets a captured graph be replayed with a new seed).  flips0: when not null,
// flips0[0 .. S_local) is zeroed as well (a round's flip counts).
cudaError_t launch_diversify(const uint64_t* x0, int n, int mode, uint64_t seed,
                             uint64_t round, int64_t S_total, int64_t s_begin,
                             int64_t S_local, int div_H, uint64_t* X, cudaStream_t st,
                             const uint64_t* seed_dev = nullptr, int32_t* flips0 = nullptr);
// Every instance of a batch in one launch: starts (seed read from seed_dev)
// into each d[i].X, d[i].f and d[i].flips zeroed; max_words = the largest S W.
cudaError_t launch_diversify_batch(const BatchDesc* d, int count, int64_t max_words, int mode,
                                   const uint64_t* seed_dev, uint64_t round, int div_H,
                                   cudaStream_t st);
cudaError_t launch_eval_plain(const ubqp_q* h, const uint64_t* X, int64_t S,
                              int64_t* f, cudaStream_t st);
size_t eval_tc_workspace(const ubqp_q* h, int64_t S);
cudaError_t eval_tc_upload_tables(ubqp_q* h, cudaStream_t st);
cudaError_t eval_tc_prepare(ubqp_q* h, cudaStream_t st);
size_t eval_tc_chunk_bytes(int n_tc);
std::vector<int4> eval_tc_chunks(int n_tc, int kch);
// The merged work list of a batch's evaluation (all instances, S starts each,
// chunks of at most kch K steps), largest chunks first; and its launch.
// maps: `count` CUtensorMap of the instances' Q' (the handles' own), 64-byte
// aligned in device memory; f of every instance zeroed before.
std::vector<MUnit> eval_tc_multi_units(const ubqp_q* const* qs, int count, int64_t S, int kch);
cudaError_t launch_eval_tc_multi(const EvalInst* insts, const void* maps, const MUnit* units,
                                 int n_units, unsigned* err, int sm_count, cudaStream_t st);
// The start-up products of every instance of a batch in two launches: the
// unpacking of all passing starts (and the zeroing of their Y rows), then one
// persistent tensor-core launch over the merged work list of the full-square
// chunks of every instance (units past an instance's passing count are
// skipped).  mapsA / mapsB / mapsU: `count` CUtensorMap each (the unpacked
// rows of each instance, its Q' and its Q'^t), 64-byte aligned in device memory.
std::vector<MUnit> eval_tc_multi_y_units(const ubqp_q* const* qs, int count, int64_t S);
cudaError_t launch_startup_multi(const YInst* yi, int count, int64_t max_items, const void* mapsA,
                                 const void* mapsB, const void* mapsU, const MUnit* units,
                                 int n_units, unsigned* err, int sm_count, cudaStream_t st);
size_t eval_tc_static_capacity();
size_t ascent_tc_workspace(const ubqp_q* h, int64_t S);
// The ascent's start-up y = Q x of the listed starts on the tensor cores, into
// ws (Y_out: the product).  zero_next: a counter that the unpacking zeroes
// for the ascent launched after it (or NULL).
cudaError_t launch_ascent_init_tc(const ubqp_q* h, const uint64_t* X, const int32_t* idx,
                                  const int64_t* count, int64_t S, void* ws, size_t ws_bytes,
                                  float** Y_out, cudaStream_t st,
                                  const void* mapA_in = nullptr,
                                  unsigned long long* zero_next = nullptr);
cudaError_t eval_tc_static_scratch(void** out);
// mapA_in: a TMA descriptor (128 bytes) of the unpacked starts in ws made by
// eval_tc_map_A, or nullptr to build one per call.
// fused: build the A operand in shared memory from the bits (no workspace);
// otherwise unpack into ws first and feed both operands by TMA.
// chunks_in / nchunks_in: a work-chunk table in device memory (as
// eval_tc_chunks makes) in place of the handle's own.
cudaError_t launch_eval_tc(const ubqp_q* h, const uint64_t* X, int64_t S, int64_t* f,
                           void* ws, size_t ws_bytes, cudaStream_t st,
                           const void* mapA_in = nullptr, bool fused = false,
                           const int4* chunks_in = nullptr, int nchunks_in = 0);
bool eval_tc_map_A(void* out128, const void* Xe, int64_t S, int n_tc);
cudaError_t launch_screen_stats(const int64_t* f, int64_t S, int64_t offset, int64_t* stats,
                                cudaStream_t st);
// gmax: where the maximum is read (NULL: gstats[1]).
cudaError_t launch_screen_apply(const int64_t* f, int64_t S, const int64_t* gstats,
                                int64_t S_total, double lambda, int32_t* idx, int64_t* count,
                                double* Tm, cudaStream_t st, const int64_t* gmax = nullptr);
cudaError_t launch_selftest_wait(uint64_t limit_ns, int32_t* status, cudaStream_t st);
// Evaluation with the A operand in tensor memory (no workspace).
cudaError_t launch_eval_ts(const ubqp_q* h, const uint64_t* X, int64_t S, int64_t* f,
                           cudaStream_t st);
// next: as in launch_ascent (zeroed here; NULL: round robin)
cudaError_t launch_relink(const ubqp_q* h, const uint64_t* X, const int64_t* f, const uint64_t* G,
                          int64_t P, uint64_t* Xb, int64_t* fb, int32_t* dist, uint16_t* trace,
                          int64_t ldt, const float* Y, unsigned long long* next,
                          cudaStream_t st);
// next: a device counter the launch zeroes (unless next_zeroed: an earlier
// kernel on the stream did) and the groups take starts from (NULL: round
// robin).
cudaError_t launch_ascent(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                          const int64_t* count, int64_t S, int32_t max_flips,
                          int32_t* flips, const float* Y, unsigned long long* next,
                          cudaStream_t st, bool next_zeroed = false);
// launch_ascent that also writes start s's flipped indices, in order, to
// trace[s * ldt ...] (the first ldt of them).
cudaError_t launch_ascent_traced(const ubqp_q* h, uint64_t* X, int64_t* f, const int32_t* idx,
                                 const int64_t* count, int64_t S, int32_t max_flips,
                                 int32_t* flips, const float* Y, unsigned long long* next,
                                 uint16_t* trace, int64_t ldt, cudaStream_t st,
                                 bool next_zeroed = false);
// R rounds' passing lists (back to back, round r at idx + r S, count counts[r])
// concatenated as global start indices r S + idx into idx_all, total count_all.
cudaError_t launch_concat_rounds(const int32_t* idx, const int64_t* counts, int R, int64_t S,
                                 int32_t* idx_all, int64_t* count_all, cudaStream_t st);
cudaError_t launch_best(const int64_t* f, const uint64_t* X, int64_t S, int W,
                        uint64_t* best_x, int64_t* best_f, cudaStream_t st);
// The round's best of f / X into cand_x / cand, then UpdateBestAndT: the
// incumbent inc_f / inc_x, history and stats (one launch).
cudaError_t launch_search_update(const int64_t* f, const uint64_t* X, int64_t S, int W,
                                 uint64_t* cand_x, int64_t* cand, const int64_t* count,
                                 const int32_t* idx, const int32_t* flips, int64_t* inc_f,
                                 uint64_t* inc_x, int64_t* history, int64_t* stats,
                                 cudaStream_t st);
// batched stages: one launch over all instances of a batch
cudaError_t launch_screen(const int64_t* f, int64_t S, double lambda, int32_t* idx,
                          int64_t* count, double* Tm, int64_t* stats, cudaStream_t st);
cudaError_t launch_screen_batch(const BatchDesc* d, int count, double lambda, cudaStream_t st);
cudaError_t launch_batch_items(const BatchDesc* d, const int32_t* order, int count, int2* items,
                               int64_t* n_items, cudaStream_t st);
// next: as in launch_ascent (zeroed here; NULL: round robin)
cudaError_t launch_ascent_batch(const BatchDesc* d, const int2* items, const int64_t* n_items,
                                int T, int C, int32_t max_flips, int grid,
                                unsigned long long* next, cudaStream_t st);
// packed batch ascent: blocks of T threads split into sub-groups of T, T/2,
// T/4 or T/8 threads by n; the items of each of the four classes form one
// range (ranges: 4 int4 {first item, items, 0, 0}; n_items: the item count),
// and next holds one start counter per class (4 x 8 bytes, zeroed by the
// launch; NULL: round robin).  skip0: class 0 left out of the list (its
// instances climbed by launch_ascent of their own; see packed_own_climb)
cudaError_t launch_batch_units(const BatchDesc* d, const int32_t* order, int count, int T, int C,
                               bool skip0, int2* items, int4* ranges, int64_t* n_items,
                               cudaStream_t st);
// Packed batch climbs leave the instances too large for half a block (class
// 0) to the single-instance launcher, whose group shapes for large n climb
// faster (n = 5000, ~450 passers: 1.40 ms with 160-thread groups three per SM
// against 2.01 ms packed).
inline bool packed_own_climb(int n, int T, int C) { return n > 16 * (T / 2) * C; }
cudaError_t launch_ascent_batch_packed(const BatchDesc* d, const int2* items, const int4* ranges,
                                       int T, int C, int32_t max_flips, int grid,
                                       unsigned long long* next, cudaStream_t st);
bool ascent_packed_supported(int T, int C);
int ascent_packed_grid(int T, int C, int sm_count);
int ascent_batch_grid(int T, int C, int sm_count);
bool ascent_batch_supported(int T, int C);
cudaError_t launch_best_batch(const BatchDesc* d, int count, cudaStream_t st);
cudaError_t launch_set_u64(uint64_t* dst, uint64_t v, cudaStream_t st);
cudaError_t launch_solve_stats(const int64_t* count, const int32_t* idx,
                               const int32_t* flips, const double* Tm,
                               const int64_t* sstats, const int64_t* best,
                               int64_t* out, cudaStream_t st);
// launch_best followed by launch_solve_stats (its best = best_f), in one launch
cudaError_t launch_best_stats(const int64_t* f, const uint64_t* X, int64_t S, int W,
                              uint64_t* best_x, int64_t* best_f, const int64_t* count,
                              const int32_t* idx, const int32_t* flips, const int64_t* sstats,
                              int64_t* out, cudaStream_t st);

}  // namespace ubqp
