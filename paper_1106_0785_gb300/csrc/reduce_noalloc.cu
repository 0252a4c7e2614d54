// reduce_noalloc.cu - conservation sums without any device allocation.
//
// mrtlb_reduce_noalloc is the allocation-free variant of the reduction
// behind mrtlb_reduce.  It exists for callers that cannot call cudaMalloc:
// code whose device memory is owned by another allocator with a fixed
// budget (a framework's caching allocator that has reserved the device), or
// a loop that must not pay cudaMalloc's implicit device-wide
// synchronisation.  Its scratch (the FP64 accumulators and the previous
// temperatures for the residual) lives in one file-scope static device
// array, so every GPU that loads this library holds that array until the
// process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mrtlb.h"
#include "physics.cuh"

namespace {

constexpr int kAcc = 8;  // accumulators: sum rho, jx, jy, e; max |dT| (bits); pad

// [0, kAcc): accumulators; [kAcc, kAcc + MRTLB_NOALLOC_MAX_NODES): T_prev
static __device__ __align__(256) double g_noalloc_scratch[kAcc + MRTLB_NOALLOC_MAX_NODES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
// Per device: the CUDA context the entry was set up in, the device address
// of g_noalloc_scratch in that context, the device's SM count, and the grid
// shape of the last call that completed (its temperatures are in T_prev).
// A context created anew (e.g. after cudaDeviceReset) may load the module
// at another address, so the entry is set up again when the context's id
// changes.
struct DeviceEntry {
  unsigned long long ctx_id = 0;
  double* scratch = nullptr;
  int sms = 0;
  int prev_nx = 0, prev_ny = 0;
};
DeviceEntry g_dev[kMaxDevices];

// The driver's id of the calling thread's current context (0 if none):
// cuCtxGetCurrent and cuCtxGetId through the runtime's driver entry points,
// so the library needs no link against the driver library.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)p;
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

template <typename R>
__global__ void reduce_dense_kernel(const R* __restrict__ f, int nx, int ny, double* scratch,
                                    int have_prev) {
  const long long n = (long long)nx * ny;
  double* acc = scratch;
  double* Tprev = scratch + kAcc;
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0, mx = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    double g[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) g[q] = (double)f[q * n + t];
    double rho, jx, jy, e;
    mrtlb::conserved(g, rho, jx, jy, e);
    s0 += rho; s1 += jx; s2 += jy; s3 += e;
    const double T = mrtlb::temperature(rho, jx, jy, e, 1.0 / rho);
    if (have_prev) {
      const double d = fabs(T - Tprev[t]);
      mx = (d > mx || d != d) ? d : mx;
    }
    Tprev[t] = T;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    const double m = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = (m > mx || m != m) ? m : mx;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc + 0, s0);
    atomicAdd(acc + 1, s1);
    atomicAdd(acc + 2, s2);
    atomicAdd(acc + 3, s3);
    atomicMax((unsigned long long*)(acc + 4), (unsigned long long)__double_as_longlong(mx));
  }
}

}  // namespace

extern "C" int mrtlb_reduce_noalloc(const void* f, int nx, int ny, int precision, void* stream,
                                    double out[5]) {
  if (!f || !out || nx < 1 || ny < 1) return MRTLB_ERR_ARG;
  if (precision != MRTLB_FP32 && precision != MRTLB_FP64) return MRTLB_ERR_ARG;
  if ((long long)nx * ny > MRTLB_NOALLOC_MAX_NODES) return MRTLB_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MRTLB_ERR_CUDA;
  const unsigned long long ctx_id = current_context_id();  // 0 before the runtime's first call
  std::lock_guard<std::mutex> lock(g_mutex);  // calls share the array (and T_prev) anyway
  DeviceEntry& d = g_dev[dev];
  if (!d.scratch || ctx_id == 0 || d.ctx_id != ctx_id) {
    // set-up, with the device current: the host-side name of a __device__
    // array is not a device address, so resolve it in this context
    d = DeviceEntry();
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MRTLB_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      return MRTLB_ERR_CUDA;
    d.scratch = (double*)p;
    d.sms = sms;
    d.ctx_id = current_context_id();  // the context the runtime has made current by now
  }
  double* scratch = d.scratch;
  const int have_prev = (d.prev_nx == nx && d.prev_ny == ny) ? 1 : 0;
  // from here until the launch completes T_prev is being rewritten: a failed
  // call leaves no shape to compare against
  d.prev_nx = d.prev_ny = 0;
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the last call's contents: clear the accumulators
  if (cudaMemsetAsync(scratch, 0, kAcc * sizeof(double), st) != cudaSuccess) return MRTLB_ERR_CUDA;
  const long long n = (long long)nx * ny;
  long long blocks = (n + 255) / 256;
  if (blocks > 8LL * d.sms) blocks = 8LL * d.sms;  // 8 blocks of 256 threads per SM, grid-stride beyond
  if (precision == MRTLB_FP64)
    reduce_dense_kernel<double><<<(int)blocks, 256, 0, st>>>((const double*)f, nx, ny, scratch, have_prev);
  else
    reduce_dense_kernel<float><<<(int)blocks, 256, 0, st>>>((const float*)f, nx, ny, scratch, have_prev);
  if (cudaGetLastError() != cudaSuccess) return MRTLB_ERR_CUDA;
  if (cudaMemcpyAsync(out, scratch, 5 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MRTLB_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MRTLB_ERR_CUDA;
  d.prev_nx = nx;
  d.prev_ny = ny;
  return MRTLB_OK;
}
