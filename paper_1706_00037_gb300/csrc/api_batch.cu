// api_batch.cu -- many instances of uneven n solved together: one round of
// Fig. 2's loop body (start generation, evaluation, screen, ascent of the
// passing starts, best-of) for every instance of a batch.
//
// Execution plan of one run:
//   fork   per instance, on a pool of internal streams: start generation and
//          the tensor-core (or CUDA-core) evaluation;
//   join   one launch screens every instance (a block per instance);
//   fork   per instance: the tensor-core start-up y = Q x of its passing starts;
//   join   one launch builds the work list (largest instances first), one
//          persistent launch climbs every passing start of every instance,
//          one launch takes each instance's best.
// With the tensor-core evaluation the forks can instead be single launches for
// all instances: start generation, one persistent evaluation over the merged
// work list (instance, chunk, m-tile) of every instance, largest chunks
// first, and for the start-up one unpacking launch and one persistent product
// over the merged full-square work list, units past an instance's passing
// count skipped on the device.
// The climb is either one start per group of the plan's shape, or packed: a
// 256-thread block climbs up to four starts of one instance at once in
// sub-groups of 64 or 128 threads when the instance's n fits them.
// The whole run can be captured into a CUDA graph and replayed (the seed lives
// in device memory so a replay can use a new one).  An autotuner times, on the
// batch itself, the candidate ascent group shapes (plain and packed), the
// evaluation path, one merged evaluation launch or one per instance, the
// evaluation's schedule (K steps per work chunk: 16, 12 or 8) and the stream
// count, and keeps the fastest; every choice gives identical results.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ubqp_internal.cuh"

namespace {

#define bfail ubqp::record_error

#define UBQP_BCUDA(call)                                                             \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) return bfail(UBQP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct alignas(64) TmaDesc {
  unsigned char bytes[128];
};

}  // namespace

struct ubqp_batch {
  int count = 0;
  ubqp_params p{};
  int sm_count = 0;
  std::vector<const ubqp_q*> qs;
  std::vector<int32_t> order;            // instances by decreasing n
  // device memory (one allocation)
  char* dmem = nullptr;
  size_t dbytes = 0;
  ubqp::BatchDesc* d_desc = nullptr;
  int32_t* d_order = nullptr;
  int2* d_items = nullptr;
  int64_t* d_nitems = nullptr;
  uint64_t* d_seed = nullptr;
  std::vector<ubqp::BatchDesc> h_desc;
  std::vector<void*> scratch;            // per instance: unpacked starts, then y
  std::vector<size_t> scratch_bytes;
  std::vector<TmaDesc> mapA;             // TMA descriptor of each scratch
  int4* d_units = nullptr;               // packed ascent: the item range of each class
  int64_t* d_nunits = nullptr;           // the item count, then the four class counters
  unsigned long long* d_next = nullptr;  // per instance: the start counter of its own climb
  // evaluation schedules: per instance, chunk tables of at most 8 and 12 K steps
  // (the handle's own table has 16)
  static constexpr int kAltKch[2] = {8, 12};
  std::vector<int4*> alt_chunks[2];
  std::vector<int> alt_nchunks[2];
  // configuration (autotuned)
  int asc_T = 256, asc_C = 1, eval_path = UBQP_EVAL_TC, nstreams = 8;
  int asc_grid = 0;
  bool packed = false;                   // packed ascent (sub-groups by n)
  int eval_kch = 16;                     // K steps per evaluation work chunk
  // the merged evaluation: start generation and the tensor-core evaluation of
  // every instance in one launch each (work lists for 16, 12 and 8 K steps)
  bool eval_merged = false;
  bool merged_ok = false;
  ubqp::EvalInst* d_einst = nullptr;
  void* d_maps = nullptr;
  ubqp::MUnit* d_munits[3] = {nullptr, nullptr, nullptr};
  int n_munits[3] = {0, 0, 0};
  int64_t max_words = 0;
  // ... and the start-up products of the passing starts (unpack + one launch)
  ubqp::YInst* d_yinst = nullptr;
  void* d_mapsA = nullptr;
  void* d_mapsU = nullptr;
  ubqp::MUnit* d_yunits = nullptr;
  int n_yunits = 0;
  int64_t max_items = 0;
  int max_n = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
  cudaStream_t cap_stream = nullptr;     // capture stream (the legacy stream cannot capture)
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
};

namespace {

void pick_default_shape(ubqp_batch* b) {
  const int n = b->max_n;
  if (n <= 1024) { b->asc_T = 64; b->asc_C = 1; }
  else if (n <= 2048) { b->asc_T = 128; b->asc_C = 1; }
  else if (n <= 4096) { b->asc_T = 256; b->asc_C = 1; }
  else if (n <= 8192) { b->asc_T = 512; b->asc_C = 1; }
  else { b->asc_T = 512; b->asc_C = 2; }
}

// One run of the batch on `stream` (capturable: no host synchronisation).
int kch_slot(int kch) { return kch == 16 ? 0 : kch == 12 ? 1 : 2; }

int run_body(ubqp_batch* b, cudaStream_t st) {
  const int K = std::min<int>(b->nstreams, (int)b->streams.size());
  const ubqp_params& p = b->p;
  if (b->eval_merged && b->eval_path == UBQP_EVAL_TC) {
    // ---- one launch each: every instance's starts (values and flip counts
    // zeroed), every instance's evaluation
    UBQP_BCUDA(ubqp::launch_diversify_batch(b->d_desc, b->count, b->max_words, p.mode,
                                            b->d_seed, p.round, p.div_H, st));
    const int k = kch_slot(b->eval_kch);
    UBQP_BCUDA(ubqp::launch_eval_tc_multi(b->d_einst, b->d_maps, b->d_munits[k], b->n_munits[k],
                                          b->qs[0]->err, b->sm_count, st));
  } else {
  // ---- fork: start generation and evaluation per instance
  UBQP_BCUDA(cudaEventRecord(b->ev_fork, st));
  for (int k = 0; k < K; ++k) UBQP_BCUDA(cudaStreamWaitEvent(b->streams[k], b->ev_fork, 0));
  for (int i = 0; i < b->count; ++i) {
    cudaStream_t s = b->streams[i % K];
    const ubqp_q* q = b->qs[i];
    const ubqp::BatchDesc& d = b->h_desc[i];
    UBQP_BCUDA(ubqp::launch_diversify(q->x0, q->n, p.mode, p.seed, p.round, p.num_starts, 0,
                                      p.num_starts, p.div_H, d.X, s, b->d_seed));
    if (b->eval_path == UBQP_EVAL_TC) {
      // fused or staged operand build, as UBQP_EVAL_AUTO picks for this size
      const int alt = b->eval_kch == ubqp_batch::kAltKch[0] ? 0
                      : b->eval_kch == ubqp_batch::kAltKch[1] ? 1 : -1;
      UBQP_BCUDA(ubqp::launch_eval_tc(q, d.X, p.num_starts, d.f, b->scratch[i],
                                      b->scratch_bytes[i], s, b->mapA[i].bytes,
                                      ubqp::eval_auto_fused(q->n_tc, p.num_starts),
                                      alt >= 0 ? b->alt_chunks[alt][i] : nullptr,
                                      alt >= 0 ? b->alt_nchunks[alt][i] : 0));
    } else {
      UBQP_BCUDA(ubqp::launch_eval_plain(q, d.X, p.num_starts, d.f, s));
    }
    UBQP_BCUDA(cudaMemsetAsync(d.flips, 0, sizeof(int32_t) * p.num_starts, s));
  }
  for (int k = 0; k < K; ++k) {
    UBQP_BCUDA(cudaEventRecord(b->ev_join[k], b->streams[k]));
    UBQP_BCUDA(cudaStreamWaitEvent(st, b->ev_join[k], 0));
  }
  }
  // ---- one launch: every instance's screen
  UBQP_BCUDA(ubqp::launch_screen_batch(b->d_desc, b->count, p.lambda, st));
  if (b->eval_merged && b->eval_path == UBQP_EVAL_TC) {
    // ---- one launch each: unpack every instance's passing starts, then the
    // start-up products y = Q x of all of them
    UBQP_BCUDA(ubqp::launch_startup_multi(b->d_yinst, b->count, b->max_items, b->d_mapsA,
                                          b->d_maps, b->d_mapsU, b->d_yunits, b->n_yunits,
                                          b->qs[0]->err, b->sm_count, st));
  } else {
  // ---- fork: tensor-core start-up of each instance's passing starts
  UBQP_BCUDA(cudaEventRecord(b->ev_fork, st));
  for (int k = 0; k < K; ++k) UBQP_BCUDA(cudaStreamWaitEvent(b->streams[k], b->ev_fork, 0));
  for (int i = 0; i < b->count; ++i) {
    const ubqp::BatchDesc& d = b->h_desc[i];
    if (!d.Y) continue;
    float* Y = nullptr;
    UBQP_BCUDA(ubqp::launch_ascent_init_tc(b->qs[i], d.X, d.idx, d.count, p.num_starts,
                                           b->scratch[i], b->scratch_bytes[i], &Y,
                                           b->streams[i % K], b->mapA[i].bytes));
  }
  for (int k = 0; k < K; ++k) {
    UBQP_BCUDA(cudaEventRecord(b->ev_join[k], b->streams[k]));
    UBQP_BCUDA(cudaStreamWaitEvent(st, b->ev_join[k], 0));
  }
  }
  // ---- one launch each: work list, every climb, every best
  if (b->packed) {
    // instances too large for half a block climb in launches of their own on
    // the fork streams, beside the packed launch of the others
    const bool own = ubqp::packed_own_climb(b->max_n, b->asc_T, b->asc_C);
    UBQP_BCUDA(ubqp::launch_batch_units(b->d_desc, b->d_order, b->count, b->asc_T, b->asc_C,
                                        own, b->d_items, b->d_units, b->d_nunits, st));
    if (own) {
      UBQP_BCUDA(cudaEventRecord(b->ev_fork, st));
      for (int k = 0; k < K; ++k) UBQP_BCUDA(cudaStreamWaitEvent(b->streams[k], b->ev_fork, 0));
      for (int k = 0, j = 0; k < b->count; ++k) {
        const int i = b->order[k];
        const ubqp_q* q = b->qs[i];
        if (!ubqp::packed_own_climb(q->n, b->asc_T, b->asc_C)) continue;
        const ubqp::BatchDesc& d = b->h_desc[i];
        UBQP_BCUDA(ubqp::launch_ascent(q, d.X, d.f, d.idx, d.count, p.num_starts, p.max_flips,
                                       d.flips, d.Y, b->d_next + i, b->streams[j++ % K]));
      }
    }
    // the class counters: the words after the item count
    UBQP_BCUDA(ubqp::launch_ascent_batch_packed(
        b->d_desc, b->d_items, b->d_units, b->asc_T, b->asc_C, p.max_flips, b->asc_grid,
        reinterpret_cast<unsigned long long*>(b->d_nunits + 1), st));
    if (own)
      for (int k = 0; k < K; ++k) {
        UBQP_BCUDA(cudaEventRecord(b->ev_join[k], b->streams[k]));
        UBQP_BCUDA(cudaStreamWaitEvent(st, b->ev_join[k], 0));
      }
  } else {
    UBQP_BCUDA(ubqp::launch_batch_items(b->d_desc, b->d_order, b->count, b->d_items,
                                        b->d_nitems, st));
    // the item counter: the second word of the 16-byte item-count slot
    UBQP_BCUDA(ubqp::launch_ascent_batch(b->d_desc, b->d_items, b->d_nitems, b->asc_T, b->asc_C,
                                         p.max_flips, b->asc_grid,
                                         reinterpret_cast<unsigned long long*>(b->d_nitems + 1),
                                         st));
  }
  UBQP_BCUDA(ubqp::launch_best_batch(b->d_desc, b->count, st));
  return UBQP_OK;
}

void drop_graph(ubqp_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

int set_shape(ubqp_batch* b, int T, int C, bool packed = false) {
  if (packed ? !ubqp::ascent_packed_supported(T, C) : !ubqp::ascent_batch_supported(T, C))
    return bfail(UBQP_ERR_UNSUPPORTED, "ascent shape %dx%d not built", T, C);
  if (16 * T * C < b->max_n)
    return bfail(UBQP_ERR_UNSUPPORTED, "ascent shape %dx%d cannot hold n=%d", T, C, b->max_n);
  b->asc_T = T;
  b->asc_C = C;
  b->packed = packed;
  b->asc_grid = packed ? ubqp::ascent_packed_grid(T, C, b->sm_count)
                       : ubqp::ascent_batch_grid(T, C, b->sm_count);
  return UBQP_OK;
}

}  // namespace

extern "C" {

void ubqp_batch_destroy(ubqp_batch* b) {
  if (!b) return;
  drop_graph(b);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  cudaFree(b->dmem);
  delete b;
}

int ubqp_batch_create(const ubqp_q* const* qs, int32_t count, const ubqp_params* p,
                      ubqp_batch** out) {
  if (!out) return bfail(UBQP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!qs || !p || count < 1) return bfail(UBQP_ERR_ARG, "NULL argument or count < 1");
  if (p->num_starts < 1 || p->num_starts >= ((int64_t)1 << 31) || p->max_flips < 0 ||
      (p->mode != UBQP_MODE_RANDOM && p->mode != UBQP_MODE_DIVERSIFY) ||
      (p->mode == UBQP_MODE_DIVERSIFY && p->div_H < 1))
    return bfail(UBQP_ERR_ARG, "invalid parameters");
  ubqp_batch* b = new (std::nothrow) ubqp_batch();
  if (!b) return bfail(UBQP_ERR_NOMEM, "host allocation failed");
  b->count = count;
  b->p = *p;
  b->qs.assign(qs, qs + count);
  int dev = 0;
  for (int i = 0; i < count; ++i) {
    if (!qs[i]) {
      delete b;
      return bfail(UBQP_ERR_ARG, "instance %d is NULL", i);
    }
    if (i == 0) dev = qs[0]->device;
    if (qs[i]->device != dev) {
      delete b;
      return bfail(UBQP_ERR_ARG, "instances live on different devices");
    }
    b->max_n = std::max(b->max_n, qs[i]->n);
  }
  b->sm_count = qs[0]->sm_count;
  b->order.resize(count);
  for (int i = 0; i < count; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int a, int c) { return qs[a]->n > qs[c]->n; });
  // ---- carve one device allocation
  const int64_t S = p->num_starts;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += up256(bytes);
    return at;
  };
  const size_t o_desc = take(sizeof(ubqp::BatchDesc) * count);
  const size_t o_order = take(sizeof(int32_t) * count);
  const size_t o_items = take(sizeof(int2) * (size_t)S * count);
  const size_t o_nitems = take(16);
  const size_t o_units = take(std::max<size_t>(sizeof(int4) * (size_t)S * count, 4 * sizeof(int4)));
  const size_t o_nunits = take(5 * sizeof(int64_t));  // item count, one start counter per class
  const size_t o_next = take(sizeof(unsigned long long) * (size_t)count);
  const size_t o_seed = take(16);
  // the merged evaluation: instances, tensor maps, work lists
  const size_t o_einst = take(sizeof(ubqp::EvalInst) * count);
  const size_t o_maps = take(128 * (size_t)count);
  bool all_tc = true;
  for (int i = 0; i < count; ++i) all_tc = all_tc && qs[i]->tc_ok;
  std::vector<ubqp::MUnit> mu[3];
  size_t o_mu[3] = {0, 0, 0};
  for (int k = 0; k < 3; ++k) {
    if (all_tc) mu[k] = ubqp::eval_tc_multi_units(qs, count, S, k == 0 ? 16 : k == 1 ? 12 : 8);
    o_mu[k] = take(sizeof(ubqp::MUnit) * std::max<size_t>(mu[k].size(), 1));
  }
  const size_t o_yinst = take(sizeof(ubqp::YInst) * count);
  const size_t o_mapsA = take(128 * (size_t)count);
  const size_t o_mapsU = take(128 * (size_t)count);
  std::vector<ubqp::MUnit> yu;
  if (all_tc) yu = ubqp::eval_tc_multi_y_units(qs, count, S);
  const size_t o_yu = take(sizeof(ubqp::MUnit) * std::max<size_t>(yu.size(), 1));
  // the alternative evaluation schedules of each instance
  std::vector<std::vector<int4>> alt_tab[2];
  std::vector<size_t> o_alt[2];
  for (int a = 0; a < 2; ++a) {
    for (int i = 0; i < count; ++i) {
      alt_tab[a].push_back(qs[i]->tc_ok ? ubqp::eval_tc_chunks(qs[i]->n_tc,
                                                               ubqp_batch::kAltKch[a])
                                        : std::vector<int4>());
      o_alt[a].push_back(take(sizeof(int4) * std::max<size_t>(alt_tab[a][i].size(), 1)));
    }
  }
  struct Off {
    size_t X, f, idx, count, Tm, stats, flips, bx, bf, scratch, scratch_bytes;
  };
  std::vector<Off> offs(count);
  for (int i = 0; i < count; ++i) {
    const ubqp_q* q = qs[i];
    Off& o = offs[i];
    o.X = take((size_t)S * q->W * 8);
    o.f = take((size_t)S * 8);
    o.idx = take((size_t)S * 4);
    o.count = take(8);
    o.Tm = take(16);
    o.stats = take(24);
    o.flips = take((size_t)S * 4);
    o.bx = take((size_t)q->W * 8);
    o.bf = take(16);
    const size_t ev = ubqp::eval_tc_workspace(q, S), as = ubqp::ascent_tc_workspace(q, S);
    o.scratch_bytes = std::max(ev, as);
    o.scratch = take(o.scratch_bytes);
  }
  b->dbytes = off;
  if (cudaMalloc(&b->dmem, b->dbytes) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return bfail(UBQP_ERR_NOMEM, "device allocation of %zu bytes failed", off);
  }
  b->d_desc = (ubqp::BatchDesc*)(b->dmem + o_desc);
  b->d_order = (int32_t*)(b->dmem + o_order);
  b->d_items = (int2*)(b->dmem + o_items);
  b->d_nitems = (int64_t*)(b->dmem + o_nitems);
  b->d_units = (int4*)(b->dmem + o_units);
  b->d_einst = (ubqp::EvalInst*)(b->dmem + o_einst);
  b->d_yinst = (ubqp::YInst*)(b->dmem + o_yinst);
  b->d_mapsA = b->dmem + o_mapsA;
  b->d_mapsU = b->dmem + o_mapsU;
  b->d_yunits = (ubqp::MUnit*)(b->dmem + o_yu);
  b->n_yunits = (int)yu.size();
  if (!yu.empty() && cudaMemcpy(b->d_yunits, yu.data(), sizeof(ubqp::MUnit) * yu.size(),
                                cudaMemcpyHostToDevice) != cudaSuccess) {
    ubqp_batch_destroy(b);
    return bfail(UBQP_ERR_CUDA, "work list upload failed");
  }
  b->d_maps = b->dmem + o_maps;
  b->merged_ok = all_tc;
  for (int k = 0; k < 3; ++k) {
    b->d_munits[k] = (ubqp::MUnit*)(b->dmem + o_mu[k]);
    b->n_munits[k] = (int)mu[k].size();
    if (!mu[k].empty() && cudaMemcpy(b->d_munits[k], mu[k].data(),
                                     sizeof(ubqp::MUnit) * mu[k].size(),
                                     cudaMemcpyHostToDevice) != cudaSuccess) {
      ubqp_batch_destroy(b);
      return bfail(UBQP_ERR_CUDA, "work list upload failed");
    }
  }
  b->d_nunits = (int64_t*)(b->dmem + o_nunits);
  b->d_next = (unsigned long long*)(b->dmem + o_next);
  for (int a = 0; a < 2; ++a) {
    for (int i = 0; i < count; ++i) {
      b->alt_chunks[a].push_back((int4*)(b->dmem + o_alt[a][i]));
      b->alt_nchunks[a].push_back((int)alt_tab[a][i].size());
      if (!alt_tab[a][i].empty() &&
          cudaMemcpy(b->alt_chunks[a][i], alt_tab[a][i].data(),
                     sizeof(int4) * alt_tab[a][i].size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        ubqp_batch_destroy(b);
        return bfail(UBQP_ERR_CUDA, "schedule upload failed");
      }
    }
  }
  b->d_seed = (uint64_t*)(b->dmem + o_seed);
  b->h_desc.resize(count);
  b->scratch.resize(count);
  b->scratch_bytes.resize(count);
  b->mapA.assign(count, TmaDesc{});
  for (int i = 0; i < count; ++i) {
    const ubqp_q* q = qs[i];
    const Off& o = offs[i];
    ubqp::BatchDesc& d = b->h_desc[i];
    d.x0 = q->x0;
    d.Q8 = q->Q8;
    d.ldq = q->ldq;
    d.n = q->n;
    d.W = q->W;
    d.S = S;
    d.X = (uint64_t*)(b->dmem + o.X);
    d.f = (int64_t*)(b->dmem + o.f);
    d.idx = (int32_t*)(b->dmem + o.idx);
    d.count = (int64_t*)(b->dmem + o.count);
    d.Tm = (double*)(b->dmem + o.Tm);
    d.stats = (int64_t*)(b->dmem + o.stats);
    d.flips = (int32_t*)(b->dmem + o.flips);
    d.best_x = (uint64_t*)(b->dmem + o.bx);
    d.best_f = (int64_t*)(b->dmem + o.bf);
    d.err = q->err;
    b->scratch[i] = b->dmem + o.scratch;
    b->scratch_bytes[i] = o.scratch_bytes;
    // the start-up product writes y after the unpacked starts in the scratch
    const int64_t S_p = (S + 127) / 128 * 128;
    d.Y = q->tc_ok ? (const float*)((char*)b->scratch[i] + (size_t)S_p * q->n_tc * 2) : nullptr;
    d.ldy = q->n_tc;
    // TMA descriptor of the unpacked starts in this instance's scratch
    if (q->tc_ok && !ubqp::eval_tc_map_A(b->mapA[i].bytes, b->scratch[i], S, q->n_tc))
      d.Y = nullptr;
  }
  {
    std::vector<ubqp::EvalInst> ei(count);
    std::vector<ubqp::YInst> yi(count);
    std::vector<unsigned char> maps(128 * (size_t)count), mA(128 * (size_t)count),
        mU(128 * (size_t)count);
    const int64_t S_p = (S + 127) / 128 * 128;
    for (int i = 0; i < count; ++i) {
      const ubqp::BatchDesc& d = b->h_desc[i];
      ei[i] = ubqp::EvalInst{d.X, d.f, d.S, d.n, d.W};
      b->max_words = std::max<int64_t>(b->max_words, d.S * d.W);
      memcpy(maps.data() + 128 * (size_t)i, qs[i]->tc_mapB, 128);
      // the start-up: the unpacked rows at the scratch's start, Y after them
      yi[i] = ubqp::YInst{d.X, d.idx, d.count, (uint4*)b->scratch[i], const_cast<float*>(d.Y),
                          S, S_p, d.n, d.W, qs[i]->n_tc, 0};
      b->max_items = std::max<int64_t>(b->max_items, S_p * (qs[i]->n_tc / 16));
      memcpy(mA.data() + 128 * (size_t)i, b->mapA[i].bytes, 128);
      memcpy(mU.data() + 128 * (size_t)i, qs[i]->tc_mapU, 128);
      if (!d.Y) b->merged_ok = false;
    }
    if (cudaMemcpy(b->d_einst, ei.data(), sizeof(ubqp::EvalInst) * count,
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_maps, maps.data(), maps.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_yinst, yi.data(), sizeof(ubqp::YInst) * count,
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_mapsA, mA.data(), mA.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_mapsU, mU.data(), mU.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      ubqp_batch_destroy(b);
      return bfail(UBQP_ERR_CUDA, "descriptor upload failed");
    }
  }
  if (cudaMemcpy(b->d_desc, b->h_desc.data(), sizeof(ubqp::BatchDesc) * count,
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_order, b->order.data(), sizeof(int32_t) * count,
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_seed, &p->seed, 8, cudaMemcpyHostToDevice) != cudaSuccess) {
    ubqp_batch_destroy(b);
    return bfail(UBQP_ERR_CUDA, "descriptor upload failed");
  }
  // ---- streams and events of the fork/join plan
  b->streams.resize(16);
  b->ev_join.resize(16);
  for (int k = 0; k < 16; ++k) {
    if (cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) != cudaSuccess) {
      ubqp_batch_destroy(b);
      return bfail(UBQP_ERR_CUDA, "stream creation failed");
    }
  }
  if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    ubqp_batch_destroy(b);
    return bfail(UBQP_ERR_CUDA, "event creation failed");
  }
  pick_default_shape(b);
  b->nstreams = std::min(8, count);
  b->eval_path = p->eval_path == UBQP_EVAL_PLAIN ? UBQP_EVAL_PLAIN : UBQP_EVAL_TC;  // TC = fused
  for (int i = 0; i < count && b->eval_path == UBQP_EVAL_TC; ++i)
    if (!qs[i]->tc_ok) b->eval_path = UBQP_EVAL_PLAIN;
  b->eval_merged = b->merged_ok && b->eval_path == UBQP_EVAL_TC;
  int r = set_shape(b, b->asc_T, b->asc_C);
  if (r) {
    ubqp_batch_destroy(b);
    return r;
  }
  *out = b;
  return UBQP_OK;
}

int ubqp_batch_run(ubqp_batch* b, uint64_t seed, void* stream) {
  if (!b) return bfail(UBQP_ERR_ARG, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  UBQP_BCUDA(ubqp::launch_set_u64(b->d_seed, seed, st));  // read by the diversify kernels
  if (b->exec) {
    UBQP_BCUDA(cudaGraphLaunch(b->exec, st));
    return UBQP_OK;
  }
  return run_body(b, st);
}

int ubqp_batch_capture(ubqp_batch* b, void* stream) {
  if (!b) return bfail(UBQP_ERR_ARG, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  drop_graph(b);
  // one plain run first: lazy module loading and first-call attributes happen
  // outside the capture
  int r = run_body(b, st);
  if (r) return r;
  UBQP_BCUDA(cudaStreamSynchronize(st));
  cudaStream_t cs = b->cap_stream;
  UBQP_BCUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  r = run_body(b, cs);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (r) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return bfail(UBQP_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) {
    drop_graph(b);
    return bfail(UBQP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  return UBQP_OK;
}

// Times the run for candidate configurations on this batch and keeps the
// fastest: the ascent group shape (threads x chunks able to hold the largest
// n), the evaluation path, and the number of fork/join streams.  Synchronises.
int ubqp_batch_tune(ubqp_batch* b, void* stream) {
  if (!b) return bfail(UBQP_ERR_ARG, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  drop_graph(b);
  cudaEvent_t e0, e1;
  UBQP_BCUDA(cudaEventCreate(&e0));
  UBQP_BCUDA(cudaEventCreate(&e1));
  auto time_run = [&](float* ms) -> int {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      UBQP_BCUDA(cudaEventRecord(e0, st));
      int r = run_body(b, st);
      if (r) return r;
      UBQP_BCUDA(cudaEventRecord(e1, st));
      UBQP_BCUDA(cudaEventSynchronize(e1));
      float t = 0;
      UBQP_BCUDA(cudaEventElapsedTime(&t, e0, e1));
      if (rep > 0) best = std::min(best, t);  // first repetition warms up
    }
    *ms = best;
    return UBQP_OK;
  };
  int r = UBQP_OK;
  float cur = 0;
  if ((r = time_run(&cur))) goto done;
  {  // ascent group shape
    const int shapes[8][2] = {{64, 1}, {64, 2}, {128, 1}, {128, 2},
                              {256, 1}, {256, 2}, {512, 1}, {512, 2}};
    int bt = b->asc_T, bc = b->asc_C;
    bool bp = b->packed;
    for (auto& sh : shapes) {
      if (16 * sh[0] * sh[1] < b->max_n || (!bp && sh[0] == bt && sh[1] == bc)) continue;
      if (16 * sh[0] * sh[1] > 4 * std::max(b->max_n, 1024)) continue;  // far too wide
      if ((r = set_shape(b, sh[0], sh[1]))) goto done;
      float t = 0;
      if ((r = time_run(&t))) goto done;
      if (t < cur) { cur = t; bt = sh[0]; bc = sh[1]; bp = false; }
    }
    if ((r = set_shape(b, bt, bc))) goto done;
    // the packed ascent (sub-groups of 256, 128 or 64 threads by n)
    for (int c : {1, 2}) {
      if (16 * 256 * c < b->max_n || 16 * 256 * c > 4 * std::max(b->max_n, 1024)) continue;
      if ((r = set_shape(b, 256, c, true))) goto done;
      float t = 0;
      if ((r = time_run(&t))) goto done;
      if (t < cur) { cur = t; bt = 256; bc = c; bp = true; }
    }
    if ((r = set_shape(b, bt, bc, bp))) goto done;
  }
  {  // evaluation path
    bool all_tc = true;
    for (const ubqp_q* q : b->qs) all_tc = all_tc && q->tc_ok;
    if (all_tc) {
      const int keep = b->eval_path;
      b->eval_path = keep == UBQP_EVAL_TC ? UBQP_EVAL_PLAIN : UBQP_EVAL_TC;
      float t = 0;
      if ((r = time_run(&t))) goto done;
      if (t < cur) cur = t; else b->eval_path = keep;
    }
  }
  if (b->eval_path == UBQP_EVAL_TC && b->merged_ok) {  // one merged launch or per instance
    const bool keep = b->eval_merged;
    b->eval_merged = !keep;
    float t = 0;
    if ((r = time_run(&t))) goto done;
    if (t < cur) cur = t; else b->eval_merged = keep;
  }
  if (b->eval_path == UBQP_EVAL_TC) {  // evaluation schedule: K steps per work chunk
    const int keep = b->eval_kch;
    int bestk = keep;
    for (int k : {16, ubqp_batch::kAltKch[1], ubqp_batch::kAltKch[0]}) {
      if (k == keep) continue;
      b->eval_kch = k;
      float t = 0;
      if ((r = time_run(&t))) goto done;
      if (t < cur) { cur = t; bestk = k; }
    }
    b->eval_kch = bestk;
  }
  {  // fork/join streams
    const int keep = b->nstreams;
    int bestk = keep;
    for (int k : {1, 4, 8, 16}) {
      if (k == keep || k > b->count) continue;
      b->nstreams = k;
      float t = 0;
      if ((r = time_run(&t))) goto done;
      if (t < cur) { cur = t; bestk = k; }
    }
    b->nstreams = bestk;
  }
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}

int ubqp_batch_config(const ubqp_batch* b, int32_t* asc_threads, int32_t* asc_chunks,
                      int32_t* eval_path, int32_t* streams, int32_t* graph) {
  if (!b) return bfail(UBQP_ERR_ARG, "batch is NULL");
  if (asc_threads) *asc_threads = b->asc_T;
  if (asc_chunks) *asc_chunks = b->asc_C;
  if (eval_path) *eval_path = b->eval_path;
  if (streams) *streams = b->nstreams;
  if (graph) *graph = b->exec != nullptr;
  return UBQP_OK;
}

int ubqp_batch_set(ubqp_batch* b, int32_t asc_threads, int32_t asc_chunks, int32_t packed,
                   int32_t eval_kch, int32_t eval_merged) {
  if (!b) return bfail(UBQP_ERR_ARG, "batch is NULL");
  if (eval_kch != 16 && eval_kch != ubqp_batch::kAltKch[0] && eval_kch != ubqp_batch::kAltKch[1])
    return bfail(UBQP_ERR_ARG, "eval_kch must be 8, 12 or 16");
  if (eval_merged && !(b->merged_ok && b->eval_path == UBQP_EVAL_TC))
    return bfail(UBQP_ERR_UNSUPPORTED, "merged evaluation needs the tensor-core path");
  const int r = set_shape(b, asc_threads, asc_chunks, packed != 0);
  if (r) return r;
  drop_graph(b);
  b->eval_kch = eval_kch;
  b->eval_merged = eval_merged != 0;
  return UBQP_OK;
}

int ubqp_batch_schedule(const ubqp_batch* b, int32_t* packed, int32_t* eval_kch,
                        int32_t* eval_merged) {
  if (!b) return bfail(UBQP_ERR_ARG, "batch is NULL");
  if (packed) *packed = b->packed ? 1 : 0;
  if (eval_kch) *eval_kch = b->eval_kch;
  if (eval_merged) *eval_merged = b->eval_merged ? 1 : 0;
  return UBQP_OK;
}

int ubqp_batch_result(const ubqp_batch* b, int32_t i, const uint64_t** best_x_dev,
                      const int64_t** best_f_dev) {
  if (!b || i < 0 || i >= b->count) return bfail(UBQP_ERR_ARG, "bad batch or index");
  if (best_x_dev) *best_x_dev = b->h_desc[i].best_x;
  if (best_f_dev) *best_f_dev = b->h_desc[i].best_f;
  return UBQP_OK;
}

int ubqp_batch_get(const ubqp_batch* b, int32_t i, uint64_t* best_x_dev, int64_t* best_f_dev,
                   void* stream) {
  if (!b || i < 0 || i >= b->count || !best_x_dev || !best_f_dev)
    return bfail(UBQP_ERR_ARG, "bad batch, index or pointer");
  cudaStream_t st = (cudaStream_t)stream;
  UBQP_BCUDA(cudaMemcpyAsync(best_x_dev, b->h_desc[i].best_x, 8 * (size_t)b->h_desc[i].W,
                             cudaMemcpyDeviceToDevice, st));
  UBQP_BCUDA(cudaMemcpyAsync(best_f_dev, b->h_desc[i].best_f, 16, cudaMemcpyDeviceToDevice, st));
  return UBQP_OK;
}

}  // extern "C"
