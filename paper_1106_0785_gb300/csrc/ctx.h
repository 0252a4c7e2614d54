// ctx.h - the library's context (private; shared by the C ABI sources).
#pragma once

#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <string>

#include "../../include/mrtlb.h"
#include "kernels.cuh"
#include "step_tiled.cuh"

using namespace mrtlb;

// A named range on a profiler's host timeline around one library call
// (NVTX; nothing is recorded unless a tool is attached).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

struct mrtlb_adjoint_state;  // adjoint.cu

struct mrtlb_ctx {
  mrtlb_params p{};
  double s[16]{};
  int prec = MRTLB_FP32;
  size_t esize = 4;
  Layout L{};
  Walls walls{};
  Coef<double> c64{};
  Coef<float> c32{};
  size_t state_bytes = 0;
  void* f[2] = {nullptr, nullptr};
  int cur = 0;
  long steps = 0;
  // bumped by every call that changes the state or the rates (a step, set_f,
  // init_equilibrium, bind, load, set_rates, a batched step); the adjoint's
  // backward pass refuses a context changed since its forward pass
  unsigned long long gen = 0;
  long long adj_passes = 0;  // forward passes of the adjoint so far
  cudaStream_t stream = nullptr;
  int kernel = MRTLB_KERNEL_AUTO;
  // library-owned scratch
  int* err = nullptr;            // device error word
  double* acc = nullptr;         // 5 doubles for mrtlb_reduce
  double* Tprev = nullptr;       // [ny][nx] for the residual
  int have_prev = 0;
  void* staging = nullptr;       // dense f or 4 FP64 fields
  size_t staging_bytes = 0;
  TiledPlan plan{};
  // step-kernel timing
  cudaEvent_t* ev = nullptr;
  int ev_cap = 0, ev_used = 0;
  bool timing = false;
  // time loop as CUDA graphs of graph_steps steps, one per starting parity
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_steps = 64;
  mrtlb_adjoint_state* adj = nullptr;  // checkpoints and buffers of the adjoint
  long adj_interval = 0;               // adjoint segment length (0: automatic)
  std::string last_error;
};

void mrtlb_adjoint_free_internal(mrtlb_ctx* c);

