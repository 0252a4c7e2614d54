// step_tiled.cuh - the TMA-fed, row-marching step kernel (host interface).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "kernels.cuh"

// kernel selection (mirrors MRTLB_KERNEL_* in mrtlb.h)
#ifndef MRTLB_KERNEL_AUTO
#define MRTLB_KERNEL_AUTO 0
#define MRTLB_KERNEL_PLAIN 1
#define MRTLB_KERNEL_TILED 2
#endif

namespace mrtlb {

// One column strip per CTA, BX nodes wide; each CTA marches up a segment of
// rows.  Rows arrive by TMA (box = BX + 2*halo columns x 1 row x 16 planes)
// into a ring of shared-memory slots guarded by mbarriers.
struct TiledPlan {
  bool ok = false;
  int esize = 4;
  int bx = 128;        // nodes per strip (threads per CTA)
  int nslot = 6;       // ring depth
  int nstrips = 0, nseg = 0, seglen = 0;
  size_t smem = 0;     // dynamic shared memory per CTA
  CUtensorMap map[2];  // one per state buffer (read side; 64-byte aligned type)
};

// Encode tensor maps for both buffers and choose strips/segments; returns 0
// on success (plan->ok set), nonzero if TMA is unavailable (plain path used).
int plan_tiled(const Layout& L, int esize, void* f0, void* f1, TiledPlan* plan);
// The automatic kernel choice marches only segments of at least this many
// rows (shorter ones spend most of their time filling the row pipeline).
constexpr int kMinMarchRows = 16;
// Choose a segment length for a target number of CTAs.
void plan_segments(const Layout& L, int target_ctas, TiledPlan* plan);
bool tiled_supported(const TiledPlan& plan);
// Row tensor maps (box = bx + 2 halo columns x 1 row x 16 planes) of two
// state buffers; returns 0 on success.
int encode_row_maps(const Layout& L, int esize, void* f0, void* f1, int bx, CUtensorMap out[2]);
bool use_tiled(int which, const TiledPlan& plan, bool fp64);

// One kernel whose bounded wait runs out (sets ERRBIT_TIMEOUT in *err).
void launch_wait_selftest(int* err, cudaStream_t st);

// Launch one step reading buffer `cur` and writing the other one.
template <typename R>
void launch_step_tiled(const TiledPlan& plan, int cur, const Layout& L, const Coef<R>& c, int* err,
                       cudaStream_t st, void* fout);

}  // namespace mrtlb
