// recip_probe.cu - test harness: the step's hand-written reciprocal
// (physics.cuh: the hardware approximation refined by one Newton-Raphson
// step), scalar and on a packed pair, beside CUDA's IEEE division 1.0f / x,
// for a host array of x.  Built and loaded by tests/test_gpu_recip.py.
#include <cuda_runtime.h>

#include "../../paper_1106_0785_gb300/csrc/physics.cuh"

namespace {
__global__ void recip_probe_kernel(const float* x, float* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float a = x[i], b = x[n - 1 - i];
  out[i] = mrtlb::recip(a);
  const mrtlb::P2 r = mrtlb::recip(mrtlb::P2(a, b));  // lane x: x[i], lane y: x[n-1-i]
  out[n + i] = r.v.x;
  out[2 * n + (n - 1 - i)] = r.v.y;
  out[3 * n + i] = 1.0f / a;
}
}  // namespace

// out: 4 * n floats: recip scalar, recip lane x, recip lane y, 1.0f / x
extern "C" int recip_probe(const float* x_host, float* out_host, int n) {
  float *x = nullptr, *out = nullptr;
  if (n < 1 || cudaMalloc(&x, n * sizeof(float)) != cudaSuccess) return 1;
  if (cudaMalloc(&out, 4 * (size_t)n * sizeof(float)) != cudaSuccess) {
    cudaFree(x);
    return 1;
  }
  int rc = cudaMemcpy(x, x_host, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess;
  if (!rc) {
    recip_probe_kernel<<<(n + 255) / 256, 256>>>(x, out, n);
    rc = cudaGetLastError() != cudaSuccess;
  }
  if (!rc) rc = cudaMemcpy(out_host, out, 4 * (size_t)n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess;
  cudaFree(x);
  cudaFree(out);
  return rc;
}
