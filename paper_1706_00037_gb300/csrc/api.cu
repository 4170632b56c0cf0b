// api.cu -- the extern "C" boundary of libubqp (declared in include/ubqp.h):
// argument checks, the prepared-instance handle, workspace carving and the
// one-round solve that chains the kernels on one stream.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "ubqp_internal.cuh"

namespace {
thread_local char g_last_error[512] = "";
}  // namespace

namespace ubqp {
int record_error(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return status;
}
}  // namespace ubqp

namespace {

#define fail ubqp::record_error

int cuda_fail(cudaError_t e, const char* what) {
  return fail(UBQP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define UBQP_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// max |Q| for the exactness checks: the int8 bound while a deferred
// validation is unread
int64_t coeff_bound(const ubqp_q* q) { return q->max_abs >= 0 ? q->max_abs : 128; }

// Workspace of ubqp_ascent: the tensor-core start-up's scratch, then 256
// bytes holding the counter the climbs take starts from.
size_t ascent_ws_bytes(const ubqp_q* q, int64_t S) {
  return ubqp::ascent_tc_workspace(q, S) + 256;
}

// The address a kernel reads Q through: device or managed memory as given,
// page-locked host memory through its device mapping; NULL otherwise.
const int8_t* kernel_readable(const int8_t* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (a.type == cudaMemoryTypeHost && a.devicePointer)
    return static_cast<const int8_t*>(a.devicePointer);
  return nullptr;
}

// AUTO: the staged or the fused tensor-core evaluation, whichever is faster
// for this size (ubqp::eval_auto_fused).
int resolve_path(const ubqp_q* q, int64_t S, int path) {
  if (path != UBQP_EVAL_AUTO) return path;
  return (q && ubqp::eval_auto_fused(q->n_tc, S)) ? UBQP_EVAL_TC : UBQP_EVAL_TC_STAGED;
}

// Workspace of ubqp_solve, carved in this order (each piece 256-byte aligned).
struct SolveLayout {
  size_t X, f, idx, flips, small, eval, total;
};
// The evaluation and the ascent's start-up run one after the other, so they
// share one scratch region sized for the larger of the two.
constexpr size_t kSmallBytes = 256;  // count, Tm, screen stats, stats out

SolveLayout solve_layout(const ubqp_q* q, const ubqp_params* p) {
  SolveLayout L{};
  const int64_t S = p->num_starts;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += (size_t)round_up((int64_t)bytes, 256);
    return at;
  };
  L.X = take((size_t)S * q->W * 8);
  L.f = take((size_t)S * 8);
  L.idx = take((size_t)S * 4);
  L.flips = take((size_t)S * 4);
  L.small = take(kSmallBytes);
  const int path = resolve_path(q, S, p->eval_path);
  const size_t ev = path == UBQP_EVAL_TC_STAGED ? ubqp::eval_tc_workspace(q, S) : 0;
  const size_t as = ascent_ws_bytes(q, S);
  L.eval = take(ev > as ? ev : as);
  L.total = off;
  return L;
}

}  // namespace

extern "C" {

const char* ubqp_strerror(int status) {
  switch (status) {
    case UBQP_OK: return "ok";
    case UBQP_ERR_ARG: return "invalid argument";
    case UBQP_ERR_NOT_SYMMETRIC: return "Q is not symmetric";
    case UBQP_ERR_RANGE: return "coefficients exceed the exactness bound of the evaluation";
    case UBQP_ERR_NOMEM: return "out of device memory or workspace too small";
    case UBQP_ERR_CUDA: return "CUDA error";
    case UBQP_ERR_TIMEOUT: return "a kernel wait timed out";
    case UBQP_ERR_UNSUPPORTED: return "unsupported size or mode";
    default: return "unknown status";
  }
}

const char* ubqp_last_error(void) { return g_last_error; }

int ubqp_abi_version(void) { return UBQP_ABI_VERSION; }

void ubqp_q_destroy(ubqp_q* q) {
  if (!q) return;
  if (q->owns_memory) {
    cudaFree(q->Q8);
    cudaFree(q->Qt);
    cudaFree(q->Qu);
    cudaFree(q->rowsum);
    cudaFree(q->x0);
    cudaFree(q->err);
    cudaFree(q->tc_chunks);
  }
  delete q;
}

namespace {

struct HandleLayout {
  size_t q8, qt, rowsum, x0, err, chunks, total;
};

HandleLayout handle_layout(int32_t n) {
  HandleLayout L{};
  const int64_t ldq = round_up(n, UBQP_ROW_ALIGN), n_tc = round_up(n, UBQP_TC_ALIGN);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += (size_t)round_up((int64_t)bytes, 256);
    return at;
  };
  L.q8 = take((size_t)n * ldq);
  L.qt = take((size_t)n_tc * n_tc * 2 * 2);  // Qt then Qf
  L.rowsum = take(sizeof(int32_t) * n);
  L.x0 = take(8 * (size_t)ubqp::words_of(n));
  L.err = take(16);
  L.chunks = take(ubqp::eval_tc_chunk_bytes((int)n_tc));
  L.total = off;
  return L;
}

int prepare_impl(const int8_t* Q_dev, int32_t n, int64_t ldq, void* stream, void* arena,
                 size_t arena_bytes, ubqp_q** out, bool deferred = false) {
  if (!out) return fail(UBQP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!Q_dev) return fail(UBQP_ERR_ARG, "Q_dev is NULL");
  if (n < 1 || n > UBQP_MAX_N) return fail(UBQP_ERR_UNSUPPORTED, "n=%d outside [1, %d]", n, UBQP_MAX_N);
  if (ldq < n) return fail(UBQP_ERR_ARG, "ldq=%lld < n=%d", (long long)ldq, n);
  const int8_t* Q_k = kernel_readable(Q_dev);
  if (!Q_k) return fail(UBQP_ERR_ARG, "Q_dev is neither device nor page-locked host memory");
  const HandleLayout L = handle_layout(n);
  if (arena) {
    if (((uintptr_t)arena & 255) != 0) return fail(UBQP_ERR_ARG, "arena not 256-byte aligned");
    if (arena_bytes < L.total)
      return fail(UBQP_ERR_NOMEM, "arena %zu < %zu bytes", arena_bytes, L.total);
  }
  cudaStream_t st = (cudaStream_t)stream;
  ubqp_q* h = new (std::nothrow) ubqp_q();
  if (!h) return fail(UBQP_ERR_NOMEM, "host allocation failed");
  h->n = n;
  h->W = (int32_t)ubqp::words_of(n);
  h->ldq = round_up(n, UBQP_ROW_ALIGN);
  h->n_tc = (int32_t)round_up(n, UBQP_TC_ALIGN);
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) !=
          cudaSuccess) {
    delete h;
    return fail(UBQP_ERR_CUDA, "cannot query the current device");
  }
  size_t q8 = (size_t)n * h->ldq, qt = (size_t)h->n_tc * h->n_tc * 2;
  if (arena) {
    char* a = (char*)arena;
    h->owns_memory = false;
    h->Q8 = (int8_t*)(a + L.q8);
    h->Qt = (uint16_t*)(a + L.qt);
    h->Qu = (uint16_t*)(a + L.qt + qt);
    h->rowsum = (int32_t*)(a + L.rowsum);
    h->x0 = (uint64_t*)(a + L.x0);
    h->err = (unsigned*)(a + L.err);
    h->tc_chunks = a + L.chunks;
  } else {
    h->owns_memory = true;
    if (cudaMalloc(&h->Q8, q8) != cudaSuccess || cudaMalloc(&h->Qt, qt) != cudaSuccess ||
        cudaMalloc(&h->Qu, qt) != cudaSuccess ||
        cudaMalloc(&h->rowsum, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc(&h->x0, sizeof(uint64_t) * h->W) != cudaSuccess ||
        cudaMalloc(&h->err, 4 * sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      ubqp_q_destroy(h);
      return fail(UBQP_ERR_NOMEM, "device allocation of %zu bytes failed", q8 + 2 * qt);
    }
  }
  h->scratch_flags = h->err + 1;
  h->device_bytes = (int64_t)L.total;
  cudaError_t e = ubqp::launch_prepare(Q_k, n, ldq, h, st);
  if (e == cudaSuccess) e = ubqp::eval_tc_upload_tables(h, st);
  if (deferred) {  // no synchronisation: ubqp_sync reads the check
    if (e == cudaSuccess) e = ubqp::eval_tc_prepare(h, st);
    if (e != cudaSuccess) {
      ubqp_q_destroy(h);
      return cuda_fail(e, "prepare");
    }
    h->max_abs = -1;
    h->deferred = true;
    *out = h;
    return UBQP_OK;
  }
  unsigned flags[2] = {0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(flags, h->scratch_flags, sizeof(flags), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the one synchronisation
  if (e != cudaSuccess) {
    ubqp_q_destroy(h);
    return cuda_fail(e, "prepare");
  }
  if (flags[0] != 0) {
    ubqp_q_destroy(h);
    return fail(UBQP_ERR_NOT_SYMMETRIC, "Q is not symmetric (%u tiles differ)", flags[0]);
  }
  h->max_abs = (int32_t)flags[1];
  if ((e = ubqp::eval_tc_prepare(h, st)) != cudaSuccess) {
    ubqp_q_destroy(h);
    return cuda_fail(e, "eval_tc_prepare");
  }
  *out = h;
  return UBQP_OK;
}

}  // namespace

int ubqp_q_prepare(const int8_t* Q_dev, int32_t n, int64_t ldq, void* stream, ubqp_q** out) {
  UBQP_RANGE("ubqp:q_prepare");
  g_last_error[0] = 0;
  return prepare_impl(Q_dev, n, ldq, stream, nullptr, 0, out);
}

size_t ubqp_q_arena_size(int32_t n) {
  if (n < 1 || n > UBQP_MAX_N) return 0;
  return handle_layout(n).total;
}

int ubqp_q_prepare_into(const int8_t* Q_dev, int32_t n, int64_t ldq, void* arena,
                        size_t arena_bytes, void* stream, ubqp_q** out) {
  UBQP_RANGE("ubqp:q_prepare_into");
  g_last_error[0] = 0;
  if (!arena) return fail(UBQP_ERR_ARG, "arena is NULL");
  return prepare_impl(Q_dev, n, ldq, stream, arena, arena_bytes, out);
}

int ubqp_q_prepare_into_async(const int8_t* Q_dev, int32_t n, int64_t ldq, void* arena,
                              size_t arena_bytes, void* stream, ubqp_q** out) {
  UBQP_RANGE("ubqp:q_prepare_into_async");
  g_last_error[0] = 0;
  if (!arena) return fail(UBQP_ERR_ARG, "arena is NULL");
  return prepare_impl(Q_dev, n, ldq, stream, arena, arena_bytes, out, true);
}

int ubqp_q_info(const ubqp_q* q, int32_t* n, int32_t* words, int32_t* n_pad, int32_t* max_abs,
                int64_t* device_bytes) {
  if (!q) return fail(UBQP_ERR_ARG, "q is NULL");
  if (n) *n = q->n;
  if (words) *words = q->W;
  if (n_pad) *n_pad = (int32_t)q->ldq;
  if (max_abs) *max_abs = q->max_abs;
  if (device_bytes) *device_bytes = q->device_bytes;
  return UBQP_OK;
}

int ubqp_sync(const ubqp_q* q, void* stream) {
  if (!q) return fail(UBQP_ERR_ARG, "q is NULL");
  // every read and the reset stay on `stream` (a plain cudaMemcpy would also
  // wait for work queued on other streams, e.g. the next solve)
  cudaStream_t st = (cudaStream_t)stream;
  UBQP_CUDA(cudaStreamSynchronize(st));
  if (q->deferred) {  // the validation of ubqp_q_prepare_into_async
    unsigned flags[2] = {0, 0};
    UBQP_CUDA(cudaMemcpyAsync(flags, q->scratch_flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
    UBQP_CUDA(cudaStreamSynchronize(st));
    q->deferred = false;
    q->asymmetric = flags[0] != 0;
    const_cast<ubqp_q*>(q)->max_abs = (int32_t)flags[1];
  }
  if (q->asymmetric) return fail(UBQP_ERR_NOT_SYMMETRIC, "Q is not symmetric");
  unsigned e = 0;
  UBQP_CUDA(cudaMemcpyAsync(&e, q->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  UBQP_CUDA(cudaStreamSynchronize(st));
  if (e) {
    UBQP_CUDA(cudaMemsetAsync(q->err, 0, sizeof(unsigned), st));
    UBQP_CUDA(cudaStreamSynchronize(st));
    if (e & UBQP_DEVERR_TIMEOUT) return fail(UBQP_ERR_TIMEOUT, "a kernel wait timed out");
    return fail(UBQP_ERR_ARG, "a kernel saw an index outside [0, S)");
  }
  return UBQP_OK;
}

int ubqp_first_derivative(const ubqp_q* q, uint64_t* x0_dev, void* stream) {
  if (!q || !x0_dev) return fail(UBQP_ERR_ARG, "NULL argument");
  UBQP_CUDA(cudaMemcpyAsync(x0_dev, q->x0, 8 * (size_t)q->W, cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
  return UBQP_OK;
}

}  // extern "C"

// ubqp_diversify_range, and with flips0 the round's flip counts zeroed in the
// same launch (ubqp_solve).
static int diversify_impl(const ubqp_q* q, const uint64_t* x0_dev, int32_t mode, uint64_t seed,
                          uint64_t round, int64_t S_total, int64_t s_begin, int64_t S_local,
                          int32_t div_H, uint64_t* X_dev, void* stream, int32_t* flips0) {
  if (!q || !X_dev) return fail(UBQP_ERR_ARG, "NULL argument");
  if (S_total < 0 || s_begin < 0 || S_local < 0 || s_begin + S_local > S_total)
    return fail(UBQP_ERR_ARG, "range [%lld, %lld) outside a batch of %lld", (long long)s_begin,
                (long long)(s_begin + S_local), (long long)S_total);
  if (mode != UBQP_MODE_RANDOM && mode != UBQP_MODE_DIVERSIFY)
    return fail(UBQP_ERR_ARG, "unknown mode %d", mode);
  if (mode == UBQP_MODE_DIVERSIFY && div_H < 1) return fail(UBQP_ERR_ARG, "div_H < 1");
  if (S_local == 0) return UBQP_OK;
  const uint64_t* x0 = x0_dev ? x0_dev : q->x0;
  UBQP_CUDA(ubqp::launch_diversify(x0, q->n, mode, seed, round, S_total, s_begin, S_local, div_H,
                                   X_dev, (cudaStream_t)stream, nullptr, flips0));
  return UBQP_OK;
}

extern "C" {

int ubqp_diversify_range(const ubqp_q* q, const uint64_t* x0_dev, int32_t mode, uint64_t seed,
                         uint64_t round, int64_t S_total, int64_t s_begin, int64_t S_local,
                         int32_t div_H, uint64_t* X_dev, void* stream) {
  UBQP_RANGE("ubqp:diversify");
  return diversify_impl(q, x0_dev, mode, seed, round, S_total, s_begin, S_local, div_H, X_dev,
                        stream, nullptr);
}

int ubqp_diversify(const ubqp_q* q, const uint64_t* x0_dev, int32_t mode, uint64_t seed,
                   uint64_t round, int64_t S, int32_t div_H, uint64_t* X_dev, void* stream) {
  if (S < 0) return fail(UBQP_ERR_ARG, "S < 0");
  return ubqp_diversify_range(q, x0_dev, mode, seed, round, S, 0, S, div_H, X_dev, stream);
}

size_t ubqp_eval_workspace_size(const ubqp_q* q, int64_t S, int32_t path) {
  if (!q || S < 0) return 0;
  return resolve_path(q, S, path) == UBQP_EVAL_TC_STAGED ? ubqp::eval_tc_workspace(q, S) : 0;
}

int ubqp_eval(const ubqp_q* q, const uint64_t* X_dev, int64_t S, int64_t* f_dev, int32_t path,
              void* ws, size_t ws_bytes, void* stream) {
  UBQP_RANGE("ubqp:eval");
  if (!q || !X_dev || !f_dev) return fail(UBQP_ERR_ARG, "NULL argument");
  if (S < 0) return fail(UBQP_ERR_ARG, "S < 0");
  path = resolve_path(q, S, path);
  if (path != UBQP_EVAL_TC && path != UBQP_EVAL_PLAIN && path != UBQP_EVAL_TC_STAGED &&
      path != UBQP_EVAL_TC_TMEM)
    return fail(UBQP_ERR_ARG, "unknown eval path %d", path);
  if (S == 0) return UBQP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (path == UBQP_EVAL_PLAIN) {
    UBQP_CUDA(ubqp::launch_eval_plain(q, X_dev, S, f_dev, st));
    return UBQP_OK;
  }
  // bf16 operands: |2 Q_jk| <= 256 is exact; fp32 partial sums stay below 2^24
  if ((int64_t)2 * coeff_bound(q) * q->n_tc >= (1 << 24))
    return fail(UBQP_ERR_RANGE, "2*max|Q|*n_pad = %lld >= 2^24",
                (long long)2 * coeff_bound(q) * q->n_tc);
  if (path == UBQP_EVAL_TC_TMEM) {
    cudaError_t e = ubqp::launch_eval_ts(q, X_dev, S, f_dev, st);
    if (e == cudaErrorNotSupported)
      return fail(UBQP_ERR_UNSUPPORTED, "tensor-core evaluation not available for this size");
    if (e != cudaSuccess) return cuda_fail(e, "eval_ts");
    return UBQP_OK;
  }
  const bool fused = path == UBQP_EVAL_TC;
  const size_t need = fused ? 0 : ubqp::eval_tc_workspace(q, S);
  if (ws_bytes < need || (need && !ws))
    return fail(UBQP_ERR_NOMEM, "eval workspace %zu < %zu bytes", ws_bytes, need);
  if (((uintptr_t)ws & 15) != 0) return fail(UBQP_ERR_ARG, "workspace not 16-byte aligned");
  cudaError_t e = ubqp::launch_eval_tc(q, X_dev, S, f_dev, ws, ws_bytes, st, nullptr, fused);
  if (e == cudaErrorNotSupported)
    return fail(UBQP_ERR_UNSUPPORTED, "tensor-core evaluation not available for this size");
  if (e != cudaSuccess) return cuda_fail(e, "eval_tc");
  return UBQP_OK;
}

int ubqp_eval_noalloc(const ubqp_q* q, const uint64_t* X_dev, int64_t S, int64_t* f_dev,
                      void* stream) {
  UBQP_RANGE("ubqp:eval_noalloc");
  if (!q || !X_dev || !f_dev) return fail(UBQP_ERR_ARG, "NULL argument");
  if (S < 0) return fail(UBQP_ERR_ARG, "S < 0");
  if (S == 0) return UBQP_OK;
  if ((int64_t)2 * coeff_bound(q) * q->n_tc >= (1 << 24))
    return fail(UBQP_ERR_RANGE, "2*max|Q|*n_pad = %lld >= 2^24",
                (long long)2 * coeff_bound(q) * q->n_tc);
  const size_t need = ubqp::eval_tc_workspace(q, S);
  if (need > ubqp::eval_tc_static_capacity())
    return fail(UBQP_ERR_UNSUPPORTED,
                "ubqp_eval_noalloc: %lld starts at n=%d need %zu bytes of scratch, more than "
                "the built-in %zu; use ubqp_eval with a workspace",
                (long long)S, q->n, need, ubqp::eval_tc_static_capacity());
  void* scratch = nullptr;
  cudaError_t e = ubqp::eval_tc_static_scratch(&scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(eval scratch)");
  e = ubqp::launch_eval_tc(q, X_dev, S, f_dev, scratch, ubqp::eval_tc_static_capacity(),
                           (cudaStream_t)stream, nullptr, /*fused=*/false);
  if (e == cudaErrorNotSupported)
    return fail(UBQP_ERR_UNSUPPORTED, "tensor-core evaluation not available for this size");
  if (e != cudaSuccess) return cuda_fail(e, "eval_tc (static scratch)");
  return UBQP_OK;
}

int ubqp_screen_stats(const int64_t* f_dev, int64_t S, int64_t offset, int64_t* stats_dev,
                      void* stream) {
  if (!f_dev || !stats_dev) return fail(UBQP_ERR_ARG, "NULL argument");
  if (S < 0 || S >= ((int64_t)1 << 31) || offset < 0)
    return fail(UBQP_ERR_ARG, "S=%lld or offset=%lld out of range", (long long)S,
                (long long)offset);
  UBQP_CUDA(ubqp::launch_screen_stats(f_dev, S, offset, stats_dev, (cudaStream_t)stream));
  return UBQP_OK;
}

int ubqp_screen_apply(const int64_t* f_dev, int64_t S, const int64_t* gstats_dev,
                      int64_t S_total, double lambda, int32_t* idx_dev, int64_t* count_dev,
                      double* Tm_dev, void* stream) {
  if (!f_dev || !gstats_dev || !idx_dev || !count_dev || !Tm_dev)
    return fail(UBQP_ERR_ARG, "NULL argument");
  if (S < 0 || S >= ((int64_t)1 << 31) || S_total < 1)
    return fail(UBQP_ERR_ARG, "S=%lld / S_total=%lld out of range", (long long)S,
                (long long)S_total);
  if (!(lambda == lambda) || lambda > 1e300 || lambda < -1e300)
    return fail(UBQP_ERR_ARG, "lambda is not finite");
  UBQP_CUDA(ubqp::launch_screen_apply(f_dev, S, gstats_dev, S_total, lambda, idx_dev, count_dev,
                                      Tm_dev, (cudaStream_t)stream));
  return UBQP_OK;
}

int ubqp_screen(const int64_t* f_dev, int64_t S, double lambda, int32_t* idx_dev,
                int64_t* count_dev, double* Tm_dev, int64_t* stats_dev, void* stream) {
  UBQP_RANGE("ubqp:screen");
  if (!f_dev || !idx_dev || !count_dev || !Tm_dev || !stats_dev)
    return fail(UBQP_ERR_ARG, "NULL argument");
  if (S < 1 || S >= ((int64_t)1 << 31)) return fail(UBQP_ERR_ARG, "S=%lld outside [1, 2^31)", (long long)S);
  if (!(lambda == lambda) || lambda > 1e300 || lambda < -1e300)
    return fail(UBQP_ERR_ARG, "lambda is not finite");
  UBQP_CUDA(ubqp::launch_screen(f_dev, S, lambda, idx_dev, count_dev, Tm_dev, stats_dev,
                                (cudaStream_t)stream));
  return UBQP_OK;
}

size_t ubqp_ascent_workspace_size(const ubqp_q* q, int64_t S) {
  if (!q || S < 0) return 0;
  return ascent_ws_bytes(q, S);
}

// ubqp_ascent and ubqp_ascent_trace: the tensor-core start-up when the
// workspace allows, then one ascent launch (traced when trace_dev is given).
static int ascent_impl(const ubqp_q* q, uint64_t* X_dev, int64_t* f_dev, const int32_t* idx_dev,
                       const int64_t* count_dev, int64_t S, int32_t max_flips,
                       int32_t* flips_dev, uint16_t* trace_dev, int64_t ldt, void* ws,
                       size_t ws_bytes, void* stream) {
  if (!q || !X_dev || !f_dev || !idx_dev || !count_dev) return fail(UBQP_ERR_ARG, "NULL argument");
  if (S < 0 || S >= ((int64_t)1 << 31)) return fail(UBQP_ERR_ARG, "S outside [0, 2^31)");
  if (max_flips < 0) return fail(UBQP_ERR_ARG, "max_flips < 0");
  if (ws && ((uintptr_t)ws & 15) != 0) return fail(UBQP_ERR_ARG, "workspace not 16-byte aligned");
  if (S == 0) return UBQP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // the start counter in the workspace's last 256 bytes (round robin without)
  const size_t as = ascent_ws_bytes(q, S);
  unsigned long long* next =
      ws && ws_bytes >= as
          ? reinterpret_cast<unsigned long long*>(static_cast<char*>(ws) + as - 256)
          : nullptr;
  float* Y = nullptr;
  if (ws && ws_bytes >= ubqp::ascent_tc_workspace(q, S) &&
      (int64_t)coeff_bound(q) * q->n_tc < (1 << 24)) {
    // the start-up's unpacking also zeroes the counter
    cudaError_t e = ubqp::launch_ascent_init_tc(q, X_dev, idx_dev, count_dev, S, ws, ws_bytes,
                                                &Y, st, nullptr, next);
    if (e == cudaErrorNotSupported) Y = nullptr;
    else if (e != cudaSuccess) return cuda_fail(e, "ascent start-up (tensor cores)");
  }
  const bool zeroed = Y != nullptr;
  if (trace_dev)
    UBQP_CUDA(ubqp::launch_ascent_traced(q, X_dev, f_dev, idx_dev, count_dev, S, max_flips,
                                         flips_dev, Y, next, trace_dev, ldt, st, zeroed));
  else
    UBQP_CUDA(ubqp::launch_ascent(q, X_dev, f_dev, idx_dev, count_dev, S, max_flips, flips_dev,
                                  Y, next, st, zeroed));
  return UBQP_OK;
}

int ubqp_ascent(const ubqp_q* q, uint64_t* X_dev, int64_t* f_dev, const int32_t* idx_dev,
                const int64_t* count_dev, int64_t S, int32_t max_flips, int32_t* flips_dev,
                void* ws, size_t ws_bytes, void* stream) {
  UBQP_RANGE("ubqp:ascent");
  return ascent_impl(q, X_dev, f_dev, idx_dev, count_dev, S, max_flips, flips_dev, nullptr, 0,
                     ws, ws_bytes, stream);
}

int ubqp_ascent_trace(const ubqp_q* q, uint64_t* X_dev, int64_t* f_dev, const int32_t* idx_dev,
                      const int64_t* count_dev, int64_t S, int32_t max_flips, int32_t* flips_dev,
                      uint16_t* trace_dev, int64_t ldt, void* ws, size_t ws_bytes,
                      void* stream) {
  UBQP_RANGE("ubqp:ascent_trace");
  if (!trace_dev || ldt < 1) return fail(UBQP_ERR_ARG, "trace_dev is NULL or ldt < 1");
  return ascent_impl(q, X_dev, f_dev, idx_dev, count_dev, S, max_flips, flips_dev, trace_dev,
                     ldt, ws, ws_bytes, stream);
}

// Relinking workspace: [trace: P rows of n rounded up to 8 uint16][pair count]
// [tensor-core start-up of P starts, optional]
static int64_t relink_trace_ld(const ubqp_q* q) { return ((int64_t)q->n + 7) / 8 * 8; }
static size_t relink_base_bytes(const ubqp_q* q, int64_t P) {
  return (size_t)((P * relink_trace_ld(q) * 2 + 255) / 256 * 256) + 256;
}

int ubqp_selftest_timeout(uint32_t limit_us, int32_t* status_dev, void* stream) {
  if (!status_dev || limit_us < 1 || limit_us > 1000000)
    return fail(UBQP_ERR_ARG, "status_dev NULL or limit_us outside [1, 1e6]");
  cudaStream_t st = (cudaStream_t)stream;
  UBQP_CUDA(ubqp::launch_selftest_wait((uint64_t)limit_us * 1000, status_dev, st));
  int32_t status = 0;
  UBQP_CUDA(cudaMemcpyAsync(&status, status_dev, sizeof(status), cudaMemcpyDeviceToHost, st));
  UBQP_CUDA(cudaStreamSynchronize(st));
  if (status != UBQP_OK) return fail(status, "self-test wait gave up after %u us", limit_us);
  return UBQP_OK;
}

size_t ubqp_relink_workspace_size(const ubqp_q* q, int64_t P, int32_t tensor_startup) {
  if (!q || P < 0) return 0;
  return relink_base_bytes(q, P) + (tensor_startup ? ubqp::ascent_tc_workspace(q, P) : 0);
}

int ubqp_relink(const ubqp_q* q, const uint64_t* X_dev, const int64_t* f_dev,
                const uint64_t* G_dev, int64_t P, uint64_t* Xbest_dev, int64_t* fbest_dev,
                int32_t* dist_dev, void* ws, size_t ws_bytes, void* stream) {
  UBQP_RANGE("ubqp:relink");
  if (!q || !X_dev || !f_dev || !G_dev || !Xbest_dev || !fbest_dev)
    return fail(UBQP_ERR_ARG, "NULL argument");
  if (P < 0 || P >= ((int64_t)1 << 31)) return fail(UBQP_ERR_ARG, "P outside [0, 2^31)");
  if (P == 0) return UBQP_OK;
  if (!ws || ((uintptr_t)ws & 15) != 0)
    return fail(UBQP_ERR_ARG, "workspace NULL or not 16-byte aligned");
  const size_t base = relink_base_bytes(q, P);
  if (ws_bytes < base)
    return fail(UBQP_ERR_NOMEM, "relink workspace of %zu bytes, need at least %zu", ws_bytes,
                base);
  cudaStream_t st = (cudaStream_t)stream;
  uint16_t* trace = reinterpret_cast<uint16_t*>(ws);
  // the base's last 256 bytes: the pair count of the start-up, then the
  // counter the walks take pairs from
  int64_t* count = reinterpret_cast<int64_t*>(static_cast<char*>(ws) + base - 256);
  unsigned long long* next = reinterpret_cast<unsigned long long*>(count + 1);
  float* Y = nullptr;
  if (ws_bytes >= base + ubqp::ascent_tc_workspace(q, P) &&
      (int64_t)coeff_bound(q) * q->n_tc < (1 << 24)) {
    UBQP_CUDA(ubqp::launch_set_u64(reinterpret_cast<uint64_t*>(count), (uint64_t)P, st));
    cudaError_t e = ubqp::launch_ascent_init_tc(q, X_dev, nullptr, count, P,
                                                static_cast<char*>(ws) + base, ws_bytes - base,
                                                &Y, st);
    if (e == cudaErrorNotSupported) Y = nullptr;
    else if (e != cudaSuccess) return cuda_fail(e, "relink start-up (tensor cores)");
  }
  UBQP_CUDA(ubqp::launch_relink(q, X_dev, f_dev, G_dev, P, Xbest_dev, fbest_dev, dist_dev, trace,
                                relink_trace_ld(q), Y, next, st));
  return UBQP_OK;
}

int ubqp_best(const int64_t* f_dev, const uint64_t* X_dev, int64_t S, int32_t words,
              uint64_t* best_x_dev, int64_t* best_f_dev, void* stream) {
  UBQP_RANGE("ubqp:best");
  if (!f_dev || !X_dev || !best_x_dev || !best_f_dev) return fail(UBQP_ERR_ARG, "NULL argument");
  if (S < 1 || words < 1) return fail(UBQP_ERR_ARG, "S < 1 or words < 1");
  UBQP_CUDA(ubqp::launch_best(f_dev, X_dev, S, words, best_x_dev, best_f_dev,
                              (cudaStream_t)stream));
  return UBQP_OK;
}

// Workspace of ubqp_solve_rounds: R rounds' starts, values, passing lists,
// the combined list, flip counts and small results back to back, then the
// scratch the evaluation and the climb of all R*S starts share.
struct RoundsLayout {
  size_t X, f, idx, idx_all, flips, counts, Tm, sstats, count_all, eval, total;
};
RoundsLayout rounds_layout(const ubqp_q* q, const ubqp_params* p, int32_t R) {
  RoundsLayout L{};
  const int64_t S = p->num_starts, RS = S * R;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += (size_t)round_up((int64_t)bytes, 256);
    return at;
  };
  L.X = take((size_t)RS * q->W * 8);
  L.f = take((size_t)RS * 8);
  L.idx = take((size_t)RS * 4);
  L.idx_all = take((size_t)RS * 4);
  L.flips = take((size_t)RS * 4);
  L.counts = take((size_t)R * 8);
  L.Tm = take((size_t)R * 16);
  L.sstats = take((size_t)R * 24);
  L.count_all = take(8);
  const int path = resolve_path(q, RS, p->eval_path);
  const size_t ev = path == UBQP_EVAL_TC_STAGED ? ubqp::eval_tc_workspace(q, RS) : 0;
  const size_t as = ascent_ws_bytes(q, RS);
  L.eval = take(ev > as ? ev : as);
  L.total = off;
  return L;
}

size_t ubqp_solve_workspace_size(const ubqp_q* q, const ubqp_params* p) {
  if (!q || !p || p->num_starts < 1) return 0;
  return solve_layout(q, p).total;
}

int ubqp_solve(const ubqp_q* q, const ubqp_params* p, uint64_t* best_x_dev, int64_t* best_f_dev,
               ubqp_stats* stats_host, void* ws, size_t ws_bytes, void* stream) {
  UBQP_RANGE("ubqp:solve");
  if (!q || !p || !best_x_dev || !best_f_dev || !ws) return fail(UBQP_ERR_ARG, "NULL argument");
  if (p->num_starts < 1 || p->num_starts >= ((int64_t)1 << 31))
    return fail(UBQP_ERR_ARG, "num_starts outside [1, 2^31)");
  if (((uintptr_t)ws & 15) != 0) return fail(UBQP_ERR_ARG, "workspace not 16-byte aligned");
  const SolveLayout L = solve_layout(q, p);
  if (ws_bytes < L.total) return fail(UBQP_ERR_NOMEM, "workspace %zu < %zu bytes", ws_bytes, L.total);
  const int64_t S = p->num_starts;
  char* base = (char*)ws;
  uint64_t* X = (uint64_t*)(base + L.X);
  int64_t* f = (int64_t*)(base + L.f);
  int32_t* idx = (int32_t*)(base + L.idx);
  int32_t* flips = (int32_t*)(base + L.flips);
  int64_t* count = (int64_t*)(base + L.small);
  double* Tm = (double*)(base + L.small + 8);
  int64_t* sstats = (int64_t*)(base + L.small + 24);
  int64_t* sout = (int64_t*)(base + L.small + 48);
  cudaStream_t st = (cudaStream_t)stream;
  int r;
  // the starts, with the round's flip counts zeroed in the same launch
  if ((r = diversify_impl(q, nullptr, p->mode, p->seed, p->round, S, 0, S, p->div_H, X, stream,
                          flips)))
    return r;
  if ((r = ubqp_eval(q, X, S, f, p->eval_path, base + L.eval, L.total - L.eval, stream)))
    return r;
  if ((r = ubqp_screen(f, S, p->lambda, idx, count, Tm, sstats, stream))) return r;
  if ((r = ubqp_ascent(q, X, f, idx, count, S, p->max_flips, flips, base + L.eval,
                       L.total - L.eval, stream)))
    return r;
  // the best-of and the round's statistics in one launch
  UBQP_CUDA(ubqp::launch_best_stats(f, X, S, q->W, best_x_dev, best_f_dev, count, idx, flips,
                                    sstats, sout, st));
  if (stats_host) {
    int64_t hs[6];
    double hd[2];
    UBQP_CUDA(cudaMemcpyAsync(hs, sout, sizeof(hs), cudaMemcpyDeviceToHost, st));
    UBQP_CUDA(cudaMemcpyAsync(hd, Tm, sizeof(hd), cudaMemcpyDeviceToHost, st));
    if ((r = ubqp_sync(q, stream))) return r;
    stats_host->passed = hs[0];
    stats_host->total_flips = hs[1];
    stats_host->max_flips_seen = hs[2];
    stats_host->batch_max = hs[3];
    stats_host->best_index = hs[4];
    stats_host->sum = hs[5];
    stats_host->T = hd[0];
    stats_host->mean = hd[1];
  }
  return UBQP_OK;
}

size_t ubqp_solve_rounds_workspace_size(const ubqp_q* q, const ubqp_params* p, int32_t R) {
  if (!q || !p || p->num_starts < 1 || R < 1 || R > 1024 ||
      p->num_starts * (int64_t)R >= ((int64_t)1 << 31))
    return 0;
  return rounds_layout(q, p, R).total;
}

int ubqp_solve_rounds(const ubqp_q* q, const ubqp_params* p, int32_t R, uint64_t* best_x_dev,
                      int64_t* best_f_dev, void* ws, size_t ws_bytes, void* stream) {
  UBQP_RANGE("ubqp:solve_rounds");
  if (!q || !p || !best_x_dev || !best_f_dev || !ws) return fail(UBQP_ERR_ARG, "NULL argument");
  if (R < 1 || R > 1024) return fail(UBQP_ERR_ARG, "R outside [1, 1024]");
  if (p->num_starts < 1 || p->num_starts * (int64_t)R >= ((int64_t)1 << 31))
    return fail(UBQP_ERR_ARG, "num_starts * R outside [1, 2^31)");
  if (((uintptr_t)ws & 15) != 0) return fail(UBQP_ERR_ARG, "workspace not 16-byte aligned");
  const RoundsLayout L = rounds_layout(q, p, R);
  if (ws_bytes < L.total) return fail(UBQP_ERR_NOMEM, "workspace %zu < %zu bytes", ws_bytes, L.total);
  const int64_t S = p->num_starts, RS = S * R;
  const int W = q->W;
  char* base = (char*)ws;
  uint64_t* X = (uint64_t*)(base + L.X);
  int64_t* f = (int64_t*)(base + L.f);
  int32_t* idx = (int32_t*)(base + L.idx);
  int32_t* idx_all = (int32_t*)(base + L.idx_all);
  int32_t* flips = (int32_t*)(base + L.flips);
  int64_t* counts = (int64_t*)(base + L.counts);
  double* Tm = (double*)(base + L.Tm);
  int64_t* sstats = (int64_t*)(base + L.sstats);
  int64_t* count_all = (int64_t*)(base + L.count_all);
  cudaStream_t st = (cudaStream_t)stream;
  int r;
  // round k: the starts of ubqp_solve with seed + k and loop-counter offset round + k
  for (int k = 0; k < R; ++k)
    if ((r = ubqp_diversify(q, nullptr, p->mode, p->seed + (uint64_t)k, p->round + (uint64_t)k,
                            S, p->div_H, X + (int64_t)k * S * W, stream)))
      return r;
  // one evaluation of all R*S starts
  if ((r = ubqp_eval(q, X, RS, f, p->eval_path, base + L.eval, L.total - L.eval, stream)))
    return r;
  // each round's own screen over its own S values
  for (int k = 0; k < R; ++k)
    if ((r = ubqp_screen(f + (int64_t)k * S, S, p->lambda, idx + (int64_t)k * S, counts + k,
                         Tm + 2 * k, sstats + 3 * k, stream)))
      return r;
  // one climb of every round's passing starts
  UBQP_CUDA(ubqp::launch_concat_rounds(idx, counts, R, S, idx_all, count_all, st));
  UBQP_CUDA(cudaMemsetAsync(flips, 0, sizeof(int32_t) * RS, st));
  if ((r = ubqp_ascent(q, X, f, idx_all, count_all, RS, p->max_flips, flips, base + L.eval,
                       L.total - L.eval, stream)))
    return r;
  // each round's best, the lowest start index within the round on ties
  for (int k = 0; k < R; ++k)
    if ((r = ubqp_best(f + (int64_t)k * S, X + (int64_t)k * S * W, S, W, best_x_dev + (int64_t)k * W,
                       best_f_dev + 2 * k, stream)))
      return r;
  return UBQP_OK;
}

// Workspace of ubqp_search.
struct SearchLayout {
  size_t Xs, fs, X, f, idx, flips, small, inc_x, cand_x, scratch, total;
};

SearchLayout search_layout(const ubqp_q* q, const ubqp_search_params* p) {
  SearchLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += (size_t)round_up((int64_t)bytes, 256);
    return at;
  };
  const int64_t S = p->starts_per_round, NS = p->num_samples;
  L.Xs = take((size_t)NS * q->W * 8);
  L.fs = take((size_t)NS * 8);
  L.X = take((size_t)S * q->W * 8);
  L.f = take((size_t)S * 8);
  L.idx = take((size_t)S * 4);
  L.flips = take((size_t)S * 4);
  L.small = take(256);
  L.inc_x = take((size_t)q->W * 8);
  L.cand_x = take((size_t)q->W * 8);
  // the samples and the rounds' starts are evaluated apart (each count may
  // resolve AUTO its own way)
  const bool staged = resolve_path(q, S, p->eval_path) == UBQP_EVAL_TC_STAGED ||
                      resolve_path(q, NS, p->eval_path) == UBQP_EVAL_TC_STAGED;
  const int64_t big = S > NS ? S : NS;
  const size_t ev = staged ? ubqp::eval_tc_workspace(q, big) : 0;
  const size_t as = ascent_ws_bytes(q, S);
  L.scratch = take(ev > as ? ev : as);
  L.total = off;
  return L;
}

size_t ubqp_search_workspace_size(const ubqp_q* q, const ubqp_search_params* p) {
  if (!q || !p || p->starts_per_round < 1 || p->num_samples < 1) return 0;
  return search_layout(q, p).total;
}

namespace {

// Validation and workspace carving shared by ubqp_search and its resumption.
struct SearchBufs {
  uint64_t *Xs, *X, *inc_x, *cand_x;
  int64_t *fs, *f, *count, *gstats, *sstats, *cand;
  int32_t *idx, *flips;
  double* Tm;
  void* scratch;
  size_t scratch_bytes;
};

int search_check(const ubqp_q* q, const ubqp_search_params* p, uint64_t* best_x_dev,
                 int64_t* best_f_dev, int64_t* history_dev, int64_t* stats_dev, void* ws,
                 size_t ws_bytes, SearchBufs* b) {
  if (!q || !p || !best_x_dev || !best_f_dev || !stats_dev || !ws)
    return fail(UBQP_ERR_ARG, "NULL argument");
  if (p->starts_per_round < 1 || p->starts_per_round >= ((int64_t)1 << 31) ||
      p->num_samples < 1 || p->num_samples >= ((int64_t)1 << 31) || p->rounds < 0 ||
      p->max_flips < 0)
    return fail(UBQP_ERR_ARG, "starts, samples, rounds or max_flips out of range");
  if (!(p->lambda == p->lambda) || p->lambda > 1e300 || p->lambda < -1e300)
    return fail(UBQP_ERR_ARG, "lambda is not finite");
  if (p->rounds > 0 && !history_dev) return fail(UBQP_ERR_ARG, "history_dev is NULL");
  if (((uintptr_t)ws & 15) != 0) return fail(UBQP_ERR_ARG, "workspace not 16-byte aligned");
  const SearchLayout L = search_layout(q, p);
  if (ws_bytes < L.total) return fail(UBQP_ERR_NOMEM, "workspace %zu < %zu bytes", ws_bytes, L.total);
  char* base = (char*)ws;
  b->Xs = (uint64_t*)(base + L.Xs);
  b->fs = (int64_t*)(base + L.fs);
  b->X = (uint64_t*)(base + L.X);
  b->f = (int64_t*)(base + L.f);
  b->idx = (int32_t*)(base + L.idx);
  b->flips = (int32_t*)(base + L.flips);
  b->count = (int64_t*)(base + L.small);
  b->Tm = (double*)(base + L.small + 8);
  b->gstats = (int64_t*)(base + L.small + 24);
  b->sstats = (int64_t*)(base + L.small + 48);
  b->cand = (int64_t*)(base + L.small + 72);
  b->inc_x = (uint64_t*)(base + L.inc_x);
  b->cand_x = (uint64_t*)(base + L.cand_x);
  b->scratch = base + L.scratch;
  b->scratch_bytes = L.total - L.scratch;
  return UBQP_OK;
}

// Rounds first_round .. first_round + p->rounds - 1 of the loop of Fig. 2 around
// the incumbent b.inc_x / best_f_dev, with gstats[0] holding the sample sum.
int search_rounds(const ubqp_q* q, const ubqp_search_params* p, int32_t first_round,
                  const SearchBufs& b, int64_t* best_f_dev, int64_t* history_dev,
                  int64_t* stats_dev, void* stream) {
  const int64_t S = p->starts_per_round, NS = p->num_samples;
  cudaStream_t st = (cudaStream_t)stream;
  int r;
  for (int32_t i = 0; i < p->rounds; ++i) {
    const uint64_t rd = (uint64_t)first_round + (uint64_t)i;
    // the round's starts around the incumbent, its flip counts zeroed in the
    // same launch
    if ((r = diversify_impl(q, b.inc_x, UBQP_MODE_DIVERSIFY, p->seed, rd, S, 0, S, p->div_H,
                            b.X, stream, b.flips)))
      return r;
    if ((r = ubqp_eval(q, b.X, S, b.f, p->eval_path, b.scratch, b.scratch_bytes, stream)))
      return r;
    // T from the sample's Mean and the incumbent's value, read in place
    UBQP_CUDA(ubqp::launch_screen_apply(b.f, S, b.gstats, NS, p->lambda, b.idx, b.count, b.Tm,
                                        st, best_f_dev));
    if ((r = ubqp_ascent(q, b.X, b.f, b.idx, b.count, S, p->max_flips, b.flips, b.scratch,
                         b.scratch_bytes, stream)))
      return r;
    // the round's best and UpdateBestAndT in one launch
    UBQP_CUDA(ubqp::launch_search_update(b.f, b.X, S, q->W, b.cand_x, b.cand, b.count, b.idx,
                                         b.flips, best_f_dev, b.inc_x, history_dev + i,
                                         stats_dev, st));
  }
  return UBQP_OK;
}

}  // namespace

int ubqp_search(const ubqp_q* q, const ubqp_search_params* p, uint64_t* best_x_dev,
                int64_t* best_f_dev, int64_t* history_dev, int64_t* stats_dev, void* ws,
                size_t ws_bytes, void* stream) {
  UBQP_RANGE("ubqp:search");
  SearchBufs b;
  int r;
  if ((r = search_check(q, p, best_x_dev, best_f_dev, history_dev, stats_dev, ws, ws_bytes, &b)))
    return r;
  const int64_t NS = p->num_samples;
  cudaStream_t st = (cudaStream_t)stream;
  // EvaluateRandomStarts: the sample's sum gives Mean
  if ((r = ubqp_diversify(q, nullptr, UBQP_MODE_RANDOM, p->seed, 0, NS, p->div_H, b.Xs, stream)))
    return r;
  if ((r = ubqp_eval(q, b.Xs, NS, b.fs, p->eval_path, b.scratch, b.scratch_bytes, stream)))
    return r;
  if ((r = ubqp_screen_stats(b.fs, NS, 0, b.sstats, stream))) return r;
  UBQP_CUDA(cudaMemcpyAsync(b.gstats, b.sstats, 8, cudaMemcpyDeviceToDevice, st));
  // CalculateFirstDerivativeSolution: the incumbent and the initial Max
  UBQP_CUDA(cudaMemcpyAsync(b.inc_x, q->x0, 8 * (size_t)q->W, cudaMemcpyDeviceToDevice, st));
  if ((r = ubqp_eval(q, b.inc_x, 1, best_f_dev, p->eval_path, b.scratch, b.scratch_bytes,
                     stream)))
    return r;
  UBQP_CUDA(cudaMemsetAsync(stats_dev, 0, 3 * sizeof(int64_t), st));
  if ((r = search_rounds(q, p, 0, b, best_f_dev, history_dev, stats_dev, stream))) return r;
  UBQP_CUDA(cudaMemcpyAsync(stats_dev + 2, b.sstats, 8, cudaMemcpyDeviceToDevice, st));
  UBQP_CUDA(cudaMemcpyAsync(best_x_dev, b.inc_x, 8 * (size_t)q->W, cudaMemcpyDeviceToDevice, st));
  return UBQP_OK;
}

int ubqp_search_resume(const ubqp_q* q, const ubqp_search_params* p, int32_t first_round,
                       uint64_t* best_x_dev, int64_t* best_f_dev, int64_t* history_dev,
                       int64_t* stats_dev, void* ws, size_t ws_bytes, void* stream) {
  UBQP_RANGE("ubqp:search_resume");
  SearchBufs b;
  int r;
  if ((r = search_check(q, p, best_x_dev, best_f_dev, history_dev, stats_dev, ws, ws_bytes, &b)))
    return r;
  if (first_round < 0) return fail(UBQP_ERR_ARG, "first_round < 0");
  cudaStream_t st = (cudaStream_t)stream;
  // the saved state: incumbent, its value, and the sample sum behind Mean
  UBQP_CUDA(cudaMemcpyAsync(b.inc_x, best_x_dev, 8 * (size_t)q->W, cudaMemcpyDeviceToDevice, st));
  UBQP_CUDA(cudaMemcpyAsync(b.gstats, stats_dev + 2, 8, cudaMemcpyDeviceToDevice, st));
  if ((r = search_rounds(q, p, first_round, b, best_f_dev, history_dev, stats_dev, stream)))
    return r;
  UBQP_CUDA(cudaMemcpyAsync(best_x_dev, b.inc_x, 8 * (size_t)q->W, cudaMemcpyDeviceToDevice, st));
  return UBQP_OK;
}

}  // extern "C"
