// api_server.cu -- a request loop that solves UBQP instances as they arrive,
// with continuous batching.
//
// Each request is one instance (host coefficients, n, seed) to be solved by
// one round of Fig. 2's loop body with the server's parameters (the result of
// ubqp_solve on that instance alone, bit for bit).  The server runs `workers`
// lanes, each a thread with its own CUDA streams.  A free lane admits, in
// arrival order, every waiting request that fits -- up to max_batch requests
// whose device memory fits the server's budget (admission by memory) -- and
// runs them as one batch on the device:
//   per request, on the lane's fork streams: the coefficient upload, the
//     preparation, start generation and evaluation;
//   one launch screens every request of the batch;
//   per request: the tensor-core start-up y = Q x of its passing starts;
//   one persistent launch climbs every passing start of every request of the
//     batch (the packed climb of the batch plans: several small starts per
//     block), one launch takes every request's best;
//   the results come back and the batch's requests complete together.
// Requests that arrive while batches run wait for the next free lane, which
// takes all of them at once, so the batches grow with the load; the lanes'
// batches overlap on the device.  A request's device memory (the uploaded
// coefficients, the prepared instance, its workspace and result) comes from
// the device's stream-ordered memory pool, so admission and release make no
// synchronising allocator calls.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ubqp_internal.cuh"

namespace {

#define sfail ubqp::record_error

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

int64_t rup(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

struct Request {
  int64_t ticket = 0;
  const int8_t* Q = nullptr;
  int32_t n = 0;
  int64_t ldq = 0;
  uint64_t seed = 0;
  size_t bytes = 0;
  double t_submit = 0, t_done = 0;
  bool done = false;
  int status = UBQP_OK;
  int64_t best_f[2] = {0, 0};
  std::vector<uint64_t> best_x;
};

struct alignas(64) TmaDesc {
  unsigned char bytes[128];
};

constexpr int kForkStreams = 4;
constexpr int kDefaultMaxBatch = 16;

}  // namespace

// One lane: a thread, its streams and the device memory of one batch's work
// list (descriptors, order, items, units, counters).
struct ServerLane {
  cudaStream_t st = nullptr;
  cudaStream_t fork[kForkStreams] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kForkStreams] = {};
  ubqp::BatchDesc* h_desc = nullptr;  // pinned host: descriptors of the batch
  int32_t* h_order = nullptr;         // pinned host: requests by decreasing n
  uint64_t* h_x = nullptr;            // pinned host: results
  int64_t* h_f = nullptr;
  char* dmem = nullptr;
  ubqp::BatchDesc* d_desc = nullptr;
  int32_t* d_order = nullptr;
  int2* d_items = nullptr;
  int4* d_units = nullptr;
  int64_t* d_nitems = nullptr;  // the item count, then the start counter(s): one per class packed
  std::thread th;
};

struct ubqp_server {
  ubqp_server_config cfg{};
  int device = 0;
  int max_batch = kDefaultMaxBatch;
  int sm_count = 0;
  int asc_T = 256, asc_C = 1;
  bool packed = true;
  int asc_grid = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  int64_t next_ticket = 1;
  int64_t mem_used = 0;
  int in_flight = 0;
  bool stop = false;
  int inject_alloc_failures = 0;  // the next admissions fail as if out of memory
  int64_t n_batches = 0, n_batched = 0, largest = 0;  // batches run and their sizes
  std::vector<std::unique_ptr<ServerLane>> lanes;
};

namespace {

int resolve_path(const ubqp_server_config& c, int n_tc) {
  const int p = c.params.eval_path;
  if (p != UBQP_EVAL_AUTO) return p;
  return ubqp::eval_auto_fused(n_tc, c.params.num_starts) ? UBQP_EVAL_TC : UBQP_EVAL_TC_STAGED;
}

// Device bytes of one request of size n, carved in this order (each piece
// 256-byte aligned): coefficients, prepared instance, starts, values, passing
// indices, flip counts, small results (count, T and Mean, screen stats, and at
// kClimbCounter the start counter of a climb of its own), best solution and
// value, and the scratch the evaluation and the start-up share.
constexpr size_t kClimbCounter = 64;
struct ReqLayout {
  size_t Q, arena, X, f, idx, flips, small, bx, bf, scratch, scratch_bytes, total;
};
ReqLayout req_layout(const ubqp_server_config& c, int32_t n) {
  const int64_t S = c.params.num_starts, W = (n + 63) / 64;
  const int64_t n_tc = rup(n, UBQP_TC_ALIGN), S_p = rup(S, 128);
  ReqLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (size_t)rup((int64_t)bytes, 256);
    return at;
  };
  L.Q = take((size_t)n * (size_t)rup(n, 16));
  L.arena = take(ubqp_q_arena_size(n));
  L.X = take((size_t)(S * W * 8));
  L.f = take((size_t)S * 8);
  L.idx = take((size_t)S * 4);
  L.flips = take((size_t)S * 4);
  L.small = take(256);
  L.bx = take((size_t)W * 8);
  L.bf = take(16);
  const bool staged = resolve_path(c, (int)n_tc) == UBQP_EVAL_TC_STAGED;
  const int64_t ev = staged ? S_p * n_tc * 2 : 0;
  L.scratch_bytes = (size_t)std::max<int64_t>(ev, S_p * n_tc * 6);  // start-up: Xe then Y
  L.scratch = take(L.scratch_bytes);
  L.total = off;
  return L;
}

size_t request_bytes(const ubqp_server_config& c, int32_t n) { return req_layout(c, n).total; }

// One admitted request on its way through a batch.
struct Slot {
  Request* r = nullptr;
  char* buf = nullptr;
  ubqp_q* h = nullptr;
  int status = UBQP_OK;
  TmaDesc mapA{};
  bool have_mapA = false;
};

#define LCUDA(call)                                                         \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      cudaGetLastError();                                                   \
      return sfail(UBQP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    }                                                                       \
  } while (0)

// Uploads, prepares and solves the batch's live slots together on the lane's
// streams (no host synchronisation inside); a failure fails the whole batch.
int run_batch(ubqp_server* s, ServerLane& L, std::vector<Slot*>& live) {
  const ubqp_server_config& c = s->cfg;
  const ubqp_params& p = c.params;
  const int64_t S = p.num_starts;
  const int m = (int)live.size();
  auto fork = [&]() -> int {
    LCUDA(cudaEventRecord(L.ev_fork, L.st));
    for (int f = 0; f < kForkStreams; ++f) LCUDA(cudaStreamWaitEvent(L.fork[f], L.ev_fork, 0));
    return UBQP_OK;
  };
  auto join = [&]() -> int {
    for (int f = 0; f < kForkStreams; ++f) {
      LCUDA(cudaEventRecord(L.ev_join[f], L.fork[f]));
      LCUDA(cudaStreamWaitEvent(L.st, L.ev_join[f], 0));
    }
    return UBQP_OK;
  };
  // ---- fork: per request, largest first over the fork streams: the upload
  // of its coefficients, its preparation, start generation and evaluation
  for (int k = 0; k < m; ++k) L.h_order[k] = k;
  std::stable_sort(L.h_order, L.h_order + m,
                   [&](int a, int b) { return live[a]->r->n > live[b]->r->n; });
  int st = fork();
  if (st) return st;
  for (int k = 0; k < m; ++k) {
    const int i = L.h_order[k];
    Slot& sl = *live[i];
    Request* r = sl.r;
    cudaStream_t fs = L.fork[k % kForkStreams];
    const ReqLayout RL = req_layout(c, r->n);
    const int64_t ldq_dev = rup(r->n, 16);
    int8_t* Qd = (int8_t*)(sl.buf + RL.Q);
    LCUDA(cudaMemcpy2DAsync(Qd, ldq_dev, r->Q, r->ldq, r->n, r->n, cudaMemcpyHostToDevice, fs));
    if ((st = ubqp_q_prepare_into_async(Qd, r->n, ldq_dev, sl.buf + RL.arena,
                                        ubqp_q_arena_size(r->n), fs, &sl.h)))
      return st;
    ubqp::BatchDesc& d = L.h_desc[i];
    const ubqp_q* q = sl.h;
    d.x0 = q->x0;
    d.Q8 = q->Q8;
    d.ldq = q->ldq;
    d.n = q->n;
    d.W = q->W;
    d.S = S;
    d.X = (uint64_t*)(sl.buf + RL.X);
    d.f = (int64_t*)(sl.buf + RL.f);
    d.idx = (int32_t*)(sl.buf + RL.idx);
    d.count = (int64_t*)(sl.buf + RL.small);
    d.Tm = (double*)(sl.buf + RL.small + 8);
    d.stats = (int64_t*)(sl.buf + RL.small + 24);
    d.flips = (int32_t*)(sl.buf + RL.flips);
    d.best_x = (uint64_t*)(sl.buf + RL.bx);
    d.best_f = (int64_t*)(sl.buf + RL.bf);
    d.err = q->err;
    void* scratch = sl.buf + RL.scratch;
    sl.have_mapA = q->tc_ok && ubqp::eval_tc_map_A(sl.mapA.bytes, scratch, S, q->n_tc);
    d.Y = sl.have_mapA ? (const float*)((char*)scratch + (size_t)rup(S, 128) * q->n_tc * 2)
                       : nullptr;
    d.ldy = q->n_tc;
    LCUDA(ubqp::launch_diversify(q->x0, q->n, p.mode, r->seed, p.round, S, 0, S, p.div_H, d.X,
                                 fs));
    const int path = resolve_path(c, q->n_tc);
    if (path == UBQP_EVAL_PLAIN || !q->tc_ok) {
      LCUDA(ubqp::launch_eval_plain(q, d.X, S, d.f, fs));
    } else if (path == UBQP_EVAL_TC_TMEM) {
      LCUDA(ubqp::launch_eval_ts(q, d.X, S, d.f, fs));
    } else {
      LCUDA(ubqp::launch_eval_tc(q, d.X, S, d.f, scratch, RL.scratch_bytes, fs,
                                 sl.have_mapA ? sl.mapA.bytes : nullptr,
                                 path == UBQP_EVAL_TC));
    }
    LCUDA(cudaMemsetAsync(d.flips, 0, sizeof(int32_t) * S, fs));
  }
  if ((st = join())) return st;
  // the descriptors are complete on the host only now: copy them for the
  // batched launches
  LCUDA(cudaMemcpyAsync(L.d_desc, L.h_desc, sizeof(ubqp::BatchDesc) * m, cudaMemcpyHostToDevice,
                        L.st));
  LCUDA(cudaMemcpyAsync(L.d_order, L.h_order, sizeof(int32_t) * m, cudaMemcpyHostToDevice, L.st));
  // ---- one launch: every request's screen
  LCUDA(ubqp::launch_screen_batch(L.d_desc, m, p.lambda, L.st));
  // ---- fork: the start-up y = Q x of every request's passing starts
  if ((st = fork())) return st;
  for (int k = 0; k < m; ++k) {
    const int i = L.h_order[k];
    Slot& sl = *live[i];
    const ubqp::BatchDesc& d = L.h_desc[i];
    if (!d.Y) continue;
    const ReqLayout RL = req_layout(c, sl.h->n);
    float* Y = nullptr;
    LCUDA(ubqp::launch_ascent_init_tc(sl.h, d.X, d.idx, d.count, S, sl.buf + RL.scratch,
                                      RL.scratch_bytes, &Y, L.fork[k % kForkStreams],
                                      sl.mapA.bytes));
  }
  if ((st = join())) return st;
  // ---- one persistent launch climbs every passing start of the batch
  unsigned long long* next = reinterpret_cast<unsigned long long*>(L.d_nitems + 1);
  if (s->packed) {
    // requests too large for half a block climb in launches of their own on
    // the fork streams, beside the packed launch of the others
    const bool own = ubqp::packed_own_climb(live[L.h_order[0]]->r->n, s->asc_T, s->asc_C);
    LCUDA(ubqp::launch_batch_units(L.d_desc, L.d_order, m, s->asc_T, s->asc_C, own, L.d_items,
                                   L.d_units, L.d_nitems, L.st));
    if (own) {
      if ((st = fork())) return st;
      for (int k = 0, j = 0; k < m; ++k) {
        const int i = L.h_order[k];
        Slot& sl = *live[i];
        if (!ubqp::packed_own_climb(sl.h->n, s->asc_T, s->asc_C)) continue;
        const ubqp::BatchDesc& d = L.h_desc[i];
        const ReqLayout RL = req_layout(c, sl.h->n);
        // the climb's start counter: past the small results
        auto* cnt = reinterpret_cast<unsigned long long*>(sl.buf + RL.small + kClimbCounter);
        LCUDA(ubqp::launch_ascent(sl.h, d.X, d.f, d.idx, d.count, S, p.max_flips, d.flips, d.Y,
                                  cnt, L.fork[j++ % kForkStreams]));
      }
    }
    LCUDA(ubqp::launch_ascent_batch_packed(L.d_desc, L.d_items, L.d_units, s->asc_T, s->asc_C,
                                           p.max_flips, s->asc_grid, next, L.st));
    if (own && (st = join())) return st;
  } else {
    LCUDA(ubqp::launch_batch_items(L.d_desc, L.d_order, m, L.d_items, L.d_nitems, L.st));
    LCUDA(ubqp::launch_ascent_batch(L.d_desc, L.d_items, L.d_nitems, s->asc_T, s->asc_C,
                                    p.max_flips, s->asc_grid, next, L.st));
  }
  LCUDA(ubqp::launch_best_batch(L.d_desc, m, L.st));
  // ---- results back
  const int32_t Wmax = (c.max_n + 63) / 64;
  for (int k = 0; k < m; ++k) {
    const ubqp::BatchDesc& d = L.h_desc[k];
    LCUDA(cudaMemcpyAsync(L.h_x + (size_t)k * Wmax, d.best_x, 8 * (size_t)d.W,
                          cudaMemcpyDeviceToHost, L.st));
    LCUDA(cudaMemcpyAsync(L.h_f + 2 * k, d.best_f, 16, cudaMemcpyDeviceToHost, L.st));
  }
  return UBQP_OK;
}

void lane_main(ubqp_server* s, ServerLane* L) {
  cudaSetDevice(s->device);
  const int32_t Wmax = (s->cfg.max_n + 63) / 64;
  for (;;) {
    std::vector<Request*> group;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // the head of the queue goes first; it is admitted when its memory fits
      // the budget (or nothing else is in flight, so it cannot starve), and
      // the requests behind it join the batch while they fit too
      s->cv_work.wait(lk, [&] {
        if (s->stop && s->queue.empty()) return true;
        if (s->queue.empty()) return false;
        const Request* h = s->queue.front();
        return s->mem_used + (int64_t)h->bytes <= s->cfg.memory_budget || s->in_flight == 0;
      });
      if (s->queue.empty()) break;
      while (!s->queue.empty() && (int)group.size() < s->max_batch) {
        Request* h = s->queue.front();
        const bool fits = s->mem_used + (int64_t)h->bytes <= s->cfg.memory_budget;
        if (!fits && !(group.empty() && s->in_flight == 0)) break;
        s->queue.pop_front();
        s->mem_used += (int64_t)h->bytes;
        ++s->in_flight;
        if (s->inject_alloc_failures > 0) {
          --s->inject_alloc_failures;
          h->status = UBQP_ERR_NOMEM;  // marks this admission's allocation as failed
        }
        group.push_back(h);
      }
    }
    if (!group.empty()) s->cv_work.notify_all();  // another lane may take the rest
    std::vector<Slot> slots(group.size());
    std::vector<Slot*> live;
    for (size_t k = 0; k < group.size(); ++k) {
      Slot& sl = slots[k];
      sl.r = group[k];
      if (sl.r->status == UBQP_ERR_NOMEM) {
        sl.status = UBQP_ERR_NOMEM;  // injected failure: nothing allocated
      } else if (cudaMallocAsync((void**)&sl.buf, sl.r->bytes, L->st) != cudaSuccess) {
        cudaGetLastError();
        sl.status = UBQP_ERR_NOMEM;
        sl.buf = nullptr;
      } else {
        live.push_back(&sl);
      }
    }
    int bst = live.empty() ? UBQP_OK : run_batch(s, *L, live);
    if (!live.empty()) {
      // a batch that failed part-way may have left work on the fork streams
      // that the lane's stream never joined: let it finish before the
      // buffers are freed
      if (bst)
        for (int f = 0; f < kForkStreams; ++f) cudaStreamSynchronize(L->fork[f]);
      if (cudaStreamSynchronize(L->st) != cudaSuccess) {
        cudaGetLastError();
        if (!bst) bst = sfail(UBQP_ERR_CUDA, "server batch failed");
      }
    }
    for (size_t k = 0; k < live.size(); ++k) {
      Slot& sl = *live[k];
      int st = bst;
      if (sl.h) {
        const int hs = ubqp_sync(sl.h, L->st);  // deferred validation, recorded errors
        if (!st) st = hs;
      } else if (!st) {
        st = UBQP_ERR_CUDA;
      }
      if (!st) {
        const int W = (sl.r->n + 63) / 64;
        sl.r->best_x.assign(L->h_x + k * (size_t)Wmax, L->h_x + k * (size_t)Wmax + W);
        sl.r->best_f[0] = L->h_f[2 * k];
        sl.r->best_f[1] = L->h_f[2 * k + 1];
      }
      sl.status = st;
      ubqp_q_destroy(sl.h);
      cudaFreeAsync(sl.buf, L->st);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const double t = now_s();
      if (!live.empty()) {
        ++s->n_batches;
        s->n_batched += (int64_t)live.size();
        s->largest = std::max<int64_t>(s->largest, (int64_t)live.size());
      }
      for (Slot& sl : slots) {
        s->mem_used -= (int64_t)sl.r->bytes;
        --s->in_flight;
        sl.r->status = sl.status;
        sl.r->t_done = t;
        sl.r->done = true;
      }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  cudaStreamSynchronize(L->st);
}

void destroy_lane(ServerLane* L) {
  for (int f = 0; f < kForkStreams; ++f) {
    if (L->fork[f]) cudaStreamDestroy(L->fork[f]);
    if (L->ev_join[f]) cudaEventDestroy(L->ev_join[f]);
  }
  if (L->ev_fork) cudaEventDestroy(L->ev_fork);
  if (L->st) cudaStreamDestroy(L->st);
  cudaFreeHost(L->h_desc);
  cudaFreeHost(L->h_order);
  cudaFreeHost(L->h_x);
  cudaFreeHost(L->h_f);
  cudaFree(L->dmem);
}

int make_lane(ubqp_server* s, ServerLane* L) {
  const int B = s->max_batch;
  const int64_t S = s->cfg.params.num_starts;
  const int32_t Wmax = (s->cfg.max_n + 63) / 64;
  if (cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&L->ev_fork, cudaEventDisableTiming) != cudaSuccess)
    return UBQP_ERR_CUDA;
  for (int f = 0; f < kForkStreams; ++f)
    if (cudaStreamCreateWithFlags(&L->fork[f], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&L->ev_join[f], cudaEventDisableTiming) != cudaSuccess)
      return UBQP_ERR_CUDA;
  if (cudaMallocHost(&L->h_desc, sizeof(ubqp::BatchDesc) * B) != cudaSuccess ||
      cudaMallocHost(&L->h_order, sizeof(int32_t) * B) != cudaSuccess ||
      cudaMallocHost(&L->h_x, sizeof(uint64_t) * (size_t)Wmax * B) != cudaSuccess ||
      cudaMallocHost(&L->h_f, sizeof(int64_t) * 2 * B) != cudaSuccess)
    return UBQP_ERR_NOMEM;
  const size_t o_desc = 0;
  const size_t o_order = rup(sizeof(ubqp::BatchDesc) * B, 256);
  const size_t o_items = o_order + rup(sizeof(int32_t) * B, 256);
  const size_t o_units = o_items + rup(sizeof(int2) * (size_t)S * B, 256);
  const size_t o_cnt =
      o_units + rup(std::max<int64_t>(sizeof(int4) * (size_t)S * B, 4 * sizeof(int4)), 256);
  if (cudaMalloc(&L->dmem, o_cnt + 256) != cudaSuccess) return UBQP_ERR_NOMEM;
  L->d_desc = (ubqp::BatchDesc*)(L->dmem + o_desc);
  L->d_order = (int32_t*)(L->dmem + o_order);
  L->d_items = (int2*)(L->dmem + o_items);
  L->d_units = (int4*)(L->dmem + o_units);
  L->d_nitems = (int64_t*)(L->dmem + o_cnt);
  return UBQP_OK;
}

}  // namespace

extern "C" {

size_t ubqp_server_request_bytes(const ubqp_server* s, int32_t n) {
  if (!s || n < 1 || n > s->cfg.max_n) return 0;
  return request_bytes(s->cfg, n);
}

int ubqp_server_create(const ubqp_server_config* cfg, ubqp_server** out) {
  if (!out) return sfail(UBQP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg || cfg->workers < 1 || cfg->workers > 64 || cfg->max_n < 1 ||
      cfg->max_n > UBQP_MAX_N || cfg->memory_budget < 0 || cfg->max_batch < 0 ||
      cfg->max_batch > 1024 || cfg->params.num_starts < 1 ||
      cfg->params.num_starts >= ((int64_t)1 << 31) || cfg->params.max_flips < 0 ||
      (cfg->params.mode != UBQP_MODE_RANDOM && cfg->params.mode != UBQP_MODE_DIVERSIFY) ||
      (cfg->params.mode == UBQP_MODE_DIVERSIFY && cfg->params.div_H < 1))
    return sfail(UBQP_ERR_ARG, "invalid server configuration");
  std::unique_ptr<ubqp_server> s(new (std::nothrow) ubqp_server());
  if (!s) return sfail(UBQP_ERR_NOMEM, "host allocation failed");
  s->cfg = *cfg;
  s->max_batch = cfg->max_batch > 0 ? cfg->max_batch : kDefaultMaxBatch;
  if (cudaGetDevice(&s->device) != cudaSuccess) return sfail(UBQP_ERR_CUDA, "no device");
  if (cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device) !=
      cudaSuccess)
    return sfail(UBQP_ERR_CUDA, "device query failed");
  if (s->cfg.memory_budget == 0)
    s->cfg.memory_budget = (int64_t)request_bytes(s->cfg, s->cfg.max_n) * s->cfg.workers;
  // the batch climb: packed 256-thread blocks up to n = 8192, one start per
  // 512-thread block beyond
  if (cfg->max_n <= 4096) {
    s->asc_T = 256;
    s->asc_C = 1;
  } else if (cfg->max_n <= 8192) {
    s->asc_T = 256;
    s->asc_C = 2;
  } else {
    s->asc_T = 512;
    s->asc_C = 2;
    s->packed = false;
  }
  s->asc_grid = s->packed ? ubqp::ascent_packed_grid(s->asc_T, s->asc_C, s->sm_count)
                          : ubqp::ascent_batch_grid(s->asc_T, s->asc_C, s->sm_count);
  // keep freed pool memory cached so admissions never return to the OS allocator
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  for (int k = 0; k < cfg->workers; ++k) {
    std::unique_ptr<ServerLane> L(new (std::nothrow) ServerLane());
    if (!L) return sfail(UBQP_ERR_NOMEM, "host allocation failed");
    const int st = make_lane(s.get(), L.get());
    if (st) {
      destroy_lane(L.get());
      for (auto& l : s->lanes) destroy_lane(l.get());
      return sfail(st, "server lane set-up failed");
    }
    s->lanes.push_back(std::move(L));
  }
  for (auto& l : s->lanes) l->th = std::thread(lane_main, s.get(), l.get());
  *out = s.release();
  return UBQP_OK;
}

int ubqp_server_submit(ubqp_server* s, const int8_t* Q_host, int32_t n, int64_t ldq,
                       uint64_t seed, int64_t* ticket) {
  if (!s || !Q_host || !ticket) return sfail(UBQP_ERR_ARG, "NULL argument");
  if (n < 1 || n > s->cfg.max_n)
    return sfail(UBQP_ERR_UNSUPPORTED, "n=%d outside [1, %d] of this server", n, s->cfg.max_n);
  if (ldq < n) return sfail(UBQP_ERR_ARG, "ldq < n");
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return sfail(UBQP_ERR_NOMEM, "host allocation failed");
  r->Q = Q_host;
  r->n = n;
  r->ldq = ldq;
  r->seed = seed;
  r->bytes = request_bytes(s->cfg, n);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return sfail(UBQP_ERR_ARG, "server is stopping");
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->reqs.emplace(r->ticket, std::move(r));
  }
  s->cv_work.notify_all();
  return UBQP_OK;
}

int ubqp_server_poll(ubqp_server* s, int64_t ticket, int32_t* done) {
  if (!s || !done) return sfail(UBQP_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(UBQP_ERR_ARG, "unknown ticket %lld", (long long)ticket);
  *done = it->second->done ? 1 : 0;
  return UBQP_OK;
}

int ubqp_server_wait(ubqp_server* s, int64_t ticket, int64_t* best_f, uint64_t* best_x_host,
                     double* latency_s) {
  if (!s) return sfail(UBQP_ERR_ARG, "NULL server");
  std::unique_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(UBQP_ERR_ARG, "unknown ticket %lld", (long long)ticket);
    Request* rp = it->second.get();
    s->cv_done.wait(lk, [&] { return rp->done; });
    r = std::move(it->second);
    s->reqs.erase(it);
  }
  if (r->status != UBQP_OK)
    return sfail(r->status, "request %lld failed with status %d", (long long)ticket, r->status);
  if (best_f) {
    best_f[0] = r->best_f[0];
    best_f[1] = r->best_f[1];
  }
  if (best_x_host)
    for (size_t w = 0; w < r->best_x.size(); ++w) best_x_host[w] = r->best_x[w];
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  return UBQP_OK;
}

int ubqp_server_stats(ubqp_server* s, int64_t* batches, int64_t* requests, int64_t* largest) {
  if (!s) return sfail(UBQP_ERR_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->n_batches;
  if (requests) *requests = s->n_batched;
  if (largest) *largest = s->largest;
  return UBQP_OK;
}

int ubqp_server_inject_alloc_failures(ubqp_server* s, int32_t count) {
  if (!s || count < 0) return sfail(UBQP_ERR_ARG, "NULL server or count < 0");
  std::lock_guard<std::mutex> lk(s->mu);
  s->inject_alloc_failures = count;
  return UBQP_OK;
}

void ubqp_server_destroy(ubqp_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& l : s->lanes)
    if (l->th.joinable()) l->th.join();
  for (auto& l : s->lanes) destroy_lane(l.get());
  delete s;
}

}  // extern "C"
