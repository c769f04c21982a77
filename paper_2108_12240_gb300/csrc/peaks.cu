// Arithmetic-unit throughput probe (measurement utility; see bhac_measure_peaks
// in the public header).  Each kernel keeps every thread of a full device busy
// with independent chains of one operation, so the achieved rate is the
// unit's throughput, not its latency; the rates are timed with CUDA events on
// a stream of the caller.  The stage kernels are bound by the FP64 unit, and
// these figures are what the roofline's ALU peak is checked against.
#include <cuda_runtime.h>

#include "../../include/bhac_gb300.h"

namespace {

constexpr int kChains = 8;        // independent accumulators per thread
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

// Results the compiler cannot discard: a thread stores its chains only if
// their sum is exactly a value the inputs never produce.
__device__ double g_sink_d;
__device__ float g_sink_f;

// In the FP64 kernel each chain has its own multiplier and addend: with one
// shared pair the FP64 unit measured about 8% slower (operand reuse across
// consecutive instructions).  The FP32 units run fastest with the shared pair.
template <typename T>
__global__ void __launch_bounds__(kThreads) fma_kernel(int iters, T a, T b, T* sink) {
  constexpr bool own = sizeof(T) == 8;
  T acc[kChains], ac[kChains], bc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    acc[c] = T(threadIdx.x + c);
    ac[c] = own ? a * (T(1) + T(c) * T(1e-7)) : a;
    bc[c] = own ? b * (T(1) - T(c) * T(1e-3)) : b;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = acc[c] * ac[c] + bc[c];  // one fused multiply-add
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == T(-1.2345)) *sink = s;
}

// op 0: IEEE division, 1: IEEE square root, 2: reciprocal square root
template <int OP>
__global__ void __launch_bounds__(kThreads) special_kernel(int iters, double* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.5 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (OP == 0)
        x[c] = __ddiv_rn(1.25, x[c]) + 1.0;  // stays in [1.5, 1.9]
      else if (OP == 1)
        x[c] = __dsqrt_rn(x[c]) + 0.5;       // converges to ~1.9
      else
        x[c] = rsqrt(x[c]) + 1.0;            // stays in [1.5, 1.9]
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.2345) *sink = s;
}

template <typename K>
cudaError_t time_kernel(K launch, cudaStream_t st, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    launch();  // warm-up (clocks ramp, module load)
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e1);
  }
  cudaEventDestroy(e0);
  return e;
}

}  // namespace

extern "C" bhac_status bhac_measure_peaks(int iters, void* cuda_stream, double out[8]) {
  if (!out || iters < 1 || iters > (1 << 20)) return BHAC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return BHAC_ERR_CUDA;
  const int grid = nsm * kCtasPerSm;
  const double lanes = (double)grid * kThreads * kChains;
  double* sd = nullptr;
  float* sf = nullptr;
  if (cudaGetSymbolAddress((void**)&sd, g_sink_d) != cudaSuccess ||
      cudaGetSymbolAddress((void**)&sf, g_sink_f) != cudaSuccess)
    return BHAC_ERR_CUDA;
  float ms = 0.f;
  cudaError_t e = time_kernel([&] { fma_kernel<double><<<grid, kThreads, 0, st>>>(iters, 0.999999, 1e-7, sd); }, st, &ms);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  out[0] = 2.0 * lanes * iters / (ms * 1e-3);  // FP64 flops/s (fma = 2)
  // FP32: 16x the iterations so the kernel runs long enough to time
  e = time_kernel([&] { fma_kernel<float><<<grid, kThreads, 0, st>>>(16 * iters, 0.999999f, 1e-7f, sf); }, st, &ms);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  out[1] = 2.0 * lanes * 16.0 * iters / (ms * 1e-3);
  const int it_s = iters / 8 > 0 ? iters / 8 : 1;
  e = time_kernel([&] { special_kernel<0><<<grid, kThreads, 0, st>>>(it_s, sd); }, st, &ms);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  out[2] = lanes * it_s / (ms * 1e-3);  // FP64 divisions/s
  e = time_kernel([&] { special_kernel<1><<<grid, kThreads, 0, st>>>(it_s, sd); }, st, &ms);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  out[3] = lanes * it_s / (ms * 1e-3);  // FP64 square roots/s
  e = time_kernel([&] { special_kernel<2><<<grid, kThreads, 0, st>>>(it_s, sd); }, st, &ms);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  out[4] = lanes * it_s / (ms * 1e-3);  // FP64 reciprocal square roots/s
  out[5] = nsm;
  out[6] = grid;
  out[7] = kThreads;
  return BHAC_OK;
}
