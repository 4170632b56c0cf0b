// api_server.cu -- a request loop that solves UBQP instances as they arrive.
//
// Each request is one instance (host coefficients, n, seed) to be solved by
// one round of Fig. 2's loop body (ubqp_solve with the server's parameters).
// Worker threads, one CUDA stream each, take requests in arrival order as soon
// as a worker is free AND the request's device memory fits in the server's
// budget (admission by memory); several requests are therefore in flight on
// the GPU at once and their kernels overlap.  A request's device memory (the
// uploaded coefficients, the prepared instance, the solve workspace and the
// result) comes from the device's stream-ordered memory pool, so admission and
// release make no synchronising allocator calls.  Results are bit-identical to
// solving the same request alone.
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

}  // namespace

struct ubqp_server {
  ubqp_server_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  int64_t next_ticket = 1;
  int64_t mem_used = 0;
  int in_flight = 0;
  bool stop = false;
  int inject_alloc_failures = 0;  // the next admissions fail as if out of memory
  std::vector<std::thread> workers;
};

namespace {

// Device bytes of one request of size n: coefficients, prepared instance,
// solve workspace and result.
size_t request_bytes(const ubqp_server_config& c, int32_t n) {
  const int64_t S = c.params.num_starts, W = (n + 63) / 64;
  const int64_t n_tc = rup(n, UBQP_TC_ALIGN), S_p = rup(S, 128);
  int64_t ws = rup(S * W * 8, 256) + rup(S * 8, 256) + 2 * rup(S * 4, 256) + 256;
  const bool staged = c.params.eval_path == UBQP_EVAL_TC_STAGED ||
                      (c.params.eval_path == UBQP_EVAL_AUTO && n_tc > 4096);
  const int64_t ev = staged ? S_p * n_tc * 2 : 0;
  ws += rup(std::max<int64_t>(ev, S_p * n_tc * 6 + 256), 256);  // + the ascent's start counter
  return (size_t)(rup((int64_t)n * rup(n, 16), 256) + (int64_t)ubqp_q_arena_size(n) + ws +
                  rup(W * 8, 256) + 256);
}

void worker_main(ubqp_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  const int32_t Wmax = (s->cfg.max_n + 63) / 64;
  uint64_t* hx = nullptr;
  int64_t* hf = nullptr;
  cudaMallocHost(&hx, 8 * (size_t)Wmax);
  cudaMallocHost(&hf, 16);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // the head of the queue goes first; it is admitted when its memory fits
      // the budget (or nothing else is in flight, so it cannot starve)
      s->cv_work.wait(lk, [&] {
        if (s->stop && s->queue.empty()) return true;
        if (s->queue.empty()) return false;
        const Request* h = s->queue.front();
        return s->mem_used + (int64_t)h->bytes <= s->cfg.memory_budget || s->in_flight == 0;
      });
      if (s->queue.empty()) break;
      r = s->queue.front();
      s->queue.pop_front();
      s->mem_used += (int64_t)r->bytes;
      ++s->in_flight;
      if (s->inject_alloc_failures > 0) {
        --s->inject_alloc_failures;
        r->status = UBQP_ERR_NOMEM;  // marks this admission's allocation as failed
      }
    }
    int status = UBQP_OK;
    char* buf = nullptr;
    ubqp_q* h = nullptr;
    const int32_t n = r->n, W = (n + 63) / 64;
    const int64_t ldq_dev = rup(n, 16);
    if (r->status == UBQP_ERR_NOMEM) {
      status = UBQP_ERR_NOMEM;  // injected failure: nothing allocated
    } else if (cudaMallocAsync((void**)&buf, r->bytes, st) != cudaSuccess) {
      cudaGetLastError();
      status = UBQP_ERR_NOMEM;
    }
    if (status == UBQP_OK) {
      char* p = buf;
      int8_t* Qd = (int8_t*)p;
      p += rup((int64_t)n * ldq_dev, 256);
      void* arena = p;
      const size_t arena_bytes = ubqp_q_arena_size(n);
      p += arena_bytes;
      uint64_t* bx = (uint64_t*)p;
      p += rup(W * 8, 256);
      int64_t* bf = (int64_t*)p;
      p += 256;
      void* ws = p;
      const size_t ws_bytes = r->bytes - (size_t)(p - buf);
      // coefficients: rows of n bytes from the caller's host rows of ldq bytes
      if (cudaMemcpy2DAsync(Qd, ldq_dev, r->Q, r->ldq, n, n, cudaMemcpyHostToDevice, st) !=
          cudaSuccess) {
        cudaGetLastError();
        status = UBQP_ERR_CUDA;
      }
      if (status == UBQP_OK)
        status = ubqp_q_prepare_into_async(Qd, n, ldq_dev, arena, arena_bytes, st, &h);
      ubqp_params prm = s->cfg.params;
      prm.seed = r->seed;
      if (status == UBQP_OK) status = ubqp_solve(h, &prm, bx, bf, nullptr, ws, ws_bytes, st);
      if (status == UBQP_OK &&
          (cudaMemcpyAsync(hx, bx, 8 * (size_t)W, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
           cudaMemcpyAsync(hf, bf, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess))
        status = UBQP_ERR_CUDA;
      if (status == UBQP_OK) status = ubqp_sync(h, st);
      else cudaStreamSynchronize(st);
      if (status == UBQP_OK) {
        r->best_x.assign(hx, hx + W);
        r->best_f[0] = hf[0];
        r->best_f[1] = hf[1];
      }
      ubqp_q_destroy(h);
      cudaFreeAsync(buf, st);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->mem_used -= (int64_t)r->bytes;
      --s->in_flight;
      r->status = status;
      r->t_done = now_s();
      r->done = true;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  cudaStreamSynchronize(st);
  cudaFreeHost(hx);
  cudaFreeHost(hf);
  cudaStreamDestroy(st);
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
      cfg->max_n > UBQP_MAX_N || cfg->memory_budget < 0 || cfg->params.num_starts < 1 ||
      cfg->params.num_starts >= ((int64_t)1 << 31) || cfg->params.max_flips < 0 ||
      (cfg->params.mode != UBQP_MODE_RANDOM && cfg->params.mode != UBQP_MODE_DIVERSIFY) ||
      (cfg->params.mode == UBQP_MODE_DIVERSIFY && cfg->params.div_H < 1))
    return sfail(UBQP_ERR_ARG, "invalid server configuration");
  std::unique_ptr<ubqp_server> s(new (std::nothrow) ubqp_server());
  if (!s) return sfail(UBQP_ERR_NOMEM, "host allocation failed");
  s->cfg = *cfg;
  if (cudaGetDevice(&s->device) != cudaSuccess) return sfail(UBQP_ERR_CUDA, "no device");
  if (s->cfg.memory_budget == 0)
    s->cfg.memory_budget = (int64_t)request_bytes(s->cfg, s->cfg.max_n) * s->cfg.workers;
  // keep freed pool memory cached so admissions never return to the OS allocator
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  for (int k = 0; k < cfg->workers; ++k) s->workers.emplace_back(worker_main, s.get());
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
  for (auto& t : s->workers) t.join();
  delete s;
}

}  // extern "C"
