// probe.cu - measured fused multiply-add ceilings of the device (FP32
// scalar, FP32 packed pairs, FP64), the compute side of the step's roofline.
//
// Every thread runs NC independent chains a <- a m + k (m just below 1, so
// the chains stay near 1 and never reach a denormal or an overflow) and
// stores nothing unless the final sum equals a value it cannot reach, so the
// kernel moves no memory and the compiler cannot drop the arithmetic.
#include <cuda_runtime.h>

#include "../../include/mrtlb.h"
#include "pair.cuh"

namespace mrtlb {
namespace {

constexpr int NC = 8;          // independent chains per thread
constexpr int THREADS = 256;
constexpr int CTAS_PER_SM = 8; // 2048 threads per SM

template <int KIND>
__global__ void __launch_bounds__(THREADS, CTAS_PER_SM) fma_probe_kernel(double* out, int iters, double m,
                                                                           double k, double never) {
  if (KIND == MRTLB_PEAK_FP64) {
    double a[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) a[c] = 1.0 + c * 1e-3 + threadIdx.x * 1e-6;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < NC; ++c) a[c] = fma(a[c], m, k);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) s += a[c];
    if (s == never) out[0] = s;
  } else if (KIND == MRTLB_PEAK_FP32) {
    float a[NC];
    const float mf = (float)m, kf = (float)k;
#pragma unroll
    for (int c = 0; c < NC; ++c) a[c] = 1.0f + c * 1e-3f + threadIdx.x * 1e-6f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < NC; ++c) a[c] = fmaf(a[c], mf, kf);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) s += a[c];
    if ((double)s == never) out[0] = s;
  } else {
    P2 a[NC];
    const P2 mp((float)m), kp((float)k);
#pragma unroll
    for (int c = 0; c < NC; ++c) a[c] = P2(1.0f + c * 1e-3f + threadIdx.x * 1e-6f, 1.0f - c * 1e-3f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < NC; ++c) a[c] = fma(a[c], mp, kp);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) s += a[c].v.x + a[c].v.y;
    if ((double)s == never) out[0] = s;
  }
}

template <int KIND>
int run_probe(double* tflops) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MRTLB_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    return MRTLB_ERR_CUDA;
  // about 5 ms per launch at the nominal rates
  const int iters = KIND == MRTLB_PEAK_FP64 ? 1024 : KIND == MRTLB_PEAK_FP32 ? 65536 : 32768;
  const double lanes = KIND == MRTLB_PEAK_FP32_PAIR ? 2.0 : 1.0;
  const int grid = nsm * CTAS_PER_SM;
  const double flops = 2.0 * NC * lanes * (double)iters * grid * THREADS;
  double* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MRTLB_OK;
  double best = 0.0;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = MRTLB_ERR_CUDA;
  } else {
    for (int rep = 0; rep < 4 && rc == MRTLB_OK; ++rep) {
      cudaEventRecord(e0, st);
      fma_probe_kernel<KIND><<<grid, THREADS, 0, st>>>(out, iters, 0.999999, 1e-6, -1.0);
      cudaEventRecord(e1, st);
      float ms = 0.0f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = MRTLB_ERR_CUDA;
      } else if (rep > 0 && ms > 0.0f) {
        const double t = flops / (ms * 1e-3) / 1e12;
        if (t > best) best = t;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  if (rc == MRTLB_OK) *tflops = best;
  return rc;
}

}  // namespace
}  // namespace mrtlb

extern "C" int mrtlb_measure_peak(int kind, double* tflops) {
  if (!tflops) return MRTLB_ERR_ARG;
  switch (kind) {
    case MRTLB_PEAK_FP32: return mrtlb::run_probe<MRTLB_PEAK_FP32>(tflops);
    case MRTLB_PEAK_FP32_PAIR: return mrtlb::run_probe<MRTLB_PEAK_FP32_PAIR>(tflops);
    case MRTLB_PEAK_FP64: return mrtlb::run_probe<MRTLB_PEAK_FP64>(tflops);
    default: return MRTLB_ERR_ARG;
  }
}
