// k_peaks.cu -- measurement kernels for the rooflines of the ascent: the rate
// at which the SMs read an L2-resident buffer, and the rate of the integer
// instructions the ascent's per-element work is made of.  The steepest ascent
// of the Pseudocode section reads one row of Q per move from L2 and does a few
// integer operations per element; its roofline is the smaller of the L2 read
// rate divided by the row bytes and the integer rate divided by the work per
// move.  These kernels measure both rates on the device the library runs on;
// the caller times them with events (the method itself never calls them).
#include <climits>

#include "ubqp_internal.cuh"

namespace ubqp {
namespace {

constexpr int kPeakThreads = 256;

// Every thread streams 16-byte words of the buffer (L2 only, not L1), four
// loads in flight, `reps` passes; the xor of all words decides a store that
// never happens for a zero-filled buffer, which keeps the loads alive.
__global__ void __launch_bounds__(kPeakThreads)
l2_read_kernel(const uint4* __restrict__ buf, int64_t words, int reps, uint32_t* sink) {
  uint32_t acc = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int r = 0; r < reps; ++r) {
    int64_t i = t0;
    for (; i + 3 * stride < words; i += 4 * stride) {
      const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride),
                  c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
      acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^
             d.z ^ d.w;
    }
    for (; i < words; i += stride) {
      const uint4 a = __ldcg(buf + i);
      acc ^= a.x ^ a.y ^ a.z ^ a.w;
    }
  }
  if (acc == 0x9E3779B9u) sink[0] = acc;
}

// kind 0: eight independent int32 multiply-add chains per thread (the plain
// int32 instruction rate).  kind 1: the ascent's element update on sixteen
// elements per thread -- per element y += d q (dp4a with d in the byte lane),
// key = C + S y (multiply-add), and a running maximum folding two keys per
// three-way max.
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads, 4)
int_rate_kernel(int64_t iters, uint32_t seed, uint32_t* sink) {
  uint32_t out = 0;
  if (KIND == 0) {
    int a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (int)(seed + threadIdx.x * 8 + i);
    const int m = (int)(seed | 1u), c = (int)(seed >> 3);
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = a[i] * m + c;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) out ^= (uint32_t)a[i];
  } else {
    constexpr int E = 16;
    int y[E], S[E], Ck[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      y[e] = (int)(seed + threadIdx.x + e);
      S[e] = (e & 1) ? -128 : 128;
      Ck[e] = 64 * (e - 8) + e;
    }
    int w = (int)(seed * 2654435761u + threadIdx.x);
    int km = 0;
    for (int64_t t = 0; t < iters; ++t) {
      const int sel[4] = {(int)(t & 1) ? 0xFF : 0x01, (int)(t & 1) ? 0xFF00 : 0x0100,
                          (int)(t & 1) ? 0xFF0000 : 0x010000,
                          (int)(t & 1) ? (int)0xFF000000 : 0x01000000};
      int k[4] = {INT_MIN, INT_MIN, INT_MIN, INT_MIN};
#pragma unroll
      for (int e = 0; e < E; e += 2) {
        y[e] = __dp4a(w, sel[e & 3], y[e]);
        y[e + 1] = __dp4a(w, sel[(e + 1) & 3], y[e + 1]);
        k[(e >> 1) & 3] = __vimax3_s32(k[(e >> 1) & 3], Ck[e] + S[e] * y[e],
                                       Ck[e + 1] + S[e + 1] * y[e + 1]);
      }
      km ^= max(max(k[0], k[1]), max(k[2], k[3]));
      w = w * 1664525 + 1013904223;
    }
    out = (uint32_t)km;
#pragma unroll
    for (int e = 0; e < E; ++e) out ^= (uint32_t)y[e];
  }
  if (out == 0x9E3779B9u) sink[0] = out;
}

int peak_grid() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}

}  // namespace
}  // namespace ubqp

extern "C" {

int ubqp_peak_l2_read(const void* buf_dev, size_t bytes, int32_t reps, uint32_t* sink_dev,
                      void* stream) {
  if (!buf_dev || !sink_dev || bytes < 16 || reps < 1 || ((uintptr_t)buf_dev & 15) != 0)
    return ubqp::record_error(UBQP_ERR_ARG, "ubqp_peak_l2_read: bad buffer, size or reps");
  const int sms = ubqp::peak_grid();
  if (sms < 1) return ubqp::record_error(UBQP_ERR_CUDA, "no device");
  ubqp::l2_read_kernel<<<sms * 8, ubqp::kPeakThreads, 0, (cudaStream_t)stream>>>(
      static_cast<const uint4*>(buf_dev), (int64_t)(bytes / 16), reps, sink_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? UBQP_OK
                          : ubqp::record_error(UBQP_ERR_CUDA, "l2_read: %s", cudaGetErrorString(e));
}

int64_t ubqp_peak_int32_ops(int32_t kind, int64_t iters) {
  const int sms = ubqp::peak_grid();
  if (sms < 1 || (kind != 0 && kind != 1) || iters < 1) return 0;
  const int64_t threads = (int64_t)sms * 4 * ubqp::kPeakThreads;
  return threads * iters * (kind == 0 ? 8 : 16 * 3);
}

int ubqp_peak_int32(int32_t kind, int64_t iters, uint32_t* sink_dev, void* stream) {
  if (!sink_dev || (kind != 0 && kind != 1) || iters < 1)
    return ubqp::record_error(UBQP_ERR_ARG, "ubqp_peak_int32: bad kind, iters or sink");
  const int sms = ubqp::peak_grid();
  if (sms < 1) return ubqp::record_error(UBQP_ERR_CUDA, "no device");
  cudaStream_t st = (cudaStream_t)stream;
  if (kind == 0)
    ubqp::int_rate_kernel<0><<<sms * 4, ubqp::kPeakThreads, 0, st>>>(iters, 12345u, sink_dev);
  else
    ubqp::int_rate_kernel<1><<<sms * 4, ubqp::kPeakThreads, 0, st>>>(iters, 12345u, sink_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? UBQP_OK
                          : ubqp::record_error(UBQP_ERR_CUDA, "int_rate: %s", cudaGetErrorString(e));
}

}  // extern "C"
