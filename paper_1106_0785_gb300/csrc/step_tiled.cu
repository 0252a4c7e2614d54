// step_tiled.cu - TMA-fed row-marching step kernel (the FP32 hot path):
// one CTA per (column strip, row segment) of a single grid.  The device
// side of the march lives in march.cuh.
#include <cuda.h>

#include <cstddef>

#include "march.cuh"
#include "march_pair.cuh"
#include "step_tiled.cuh"

namespace mrtlb {

namespace {

template <typename R, int BX, int NSLOT, int MINB>
__global__ void __launch_bounds__(BX, MINB) step_tiled_kernel(const __grid_constant__ CUtensorMap tmap,
                                                              R* __restrict__ fout, const Layout L,
                                                              const Coef<R> c, int* err, const int seglen) {
  using SM = Smem<R, BX, NSLOT>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int ja = L.j0 + blockIdx.y * seglen;
  const int jb = min(ja + seglen, L.j1);
  if (ja >= jb) return;  // uniform over the CTA
  March<R, BX, NSLOT> m;
  m.slots = reinterpret_cast<R*>(smem_raw);
  m.U = reinterpret_cast<R*>(smem_raw + SM::u_off);
  m.bars = reinterpret_cast<uint64_t*>(smem_raw + SM::bar_off);
  m.map = &tmap;
  m.fout = fout;
  m.err = err;
  m.plane = L.plane;
  m.L = L;
  m.t = threadIdx.x;
  m.kbase = 0;
  if (m.t == 0) {
    for (int s = 0; s < NSLOT; ++s) mbar_init(&m.bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // strips start on multiples of BX so that every TMA box starts on a
  // 16-byte boundary (xoff - HL and BX are multiples of 16 bytes)
  if (m.segment(c, blockIdx.x * BX, ja, jb)) {
    if (m.t == 0) atomicOr(err, ERRBIT_TIMEOUT);
    m.drain();
  }
}

// FP32 with two nodes per thread (march_pair.cuh): BX columns, BX/2 threads,
// 211 registers, four CTAs per SM.  Measured alternatives on GB300: a launch
// bound of five CTAs (168 registers: three warps share an SM sub-partition's
// register file) was 7% slower, 64-column strips with eight one-warp CTAs
// 5% slower.
#ifndef MRTLB_PAIR_MAXNREG
#define MRTLB_PAIR_MAXNREG 0
#endif
template <int BX, int NSLOT, int MINB>
__global__ void
#if MRTLB_PAIR_MAXNREG > 0
    __maxnreg__(MRTLB_PAIR_MAXNREG)
#else
    __launch_bounds__(BX / 2, MINB)
#endif
    step_pair_kernel(const __grid_constant__ CUtensorMap tmap, float* __restrict__ fout, const Layout L,
                     const __grid_constant__ Coef<P2> c, int* err, const int seglen) {
  using SM = PairSmem<BX, NSLOT>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int ja = L.j0 + blockIdx.y * seglen;
  const int jb = min(ja + seglen, L.j1);
  if (ja >= jb) return;  // uniform over the CTA
  PairMarch<BX, NSLOT> m;
  m.slots = reinterpret_cast<float*>(smem_raw);
  m.U = reinterpret_cast<float*>(smem_raw + SM::u_off);
  m.bars = reinterpret_cast<uint64_t*>(smem_raw + SM::bar_off);
  m.map = &tmap;
  m.fout = fout;
  m.err = err;
  m.plane = L.plane;
  m.L = L;
  m.t = threadIdx.x;
  m.kbase = 0;
  if (m.t == 0) {
    for (int s = 0; s < NSLOT; ++s) mbar_init(&m.bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (m.segment(c, blockIdx.x * BX, ja, jb)) {
    if (m.t == 0) atomicOr(err, ERRBIT_TIMEOUT);
    m.drain();
  }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that no
// arrival completes; the wait gives up after its bound and the kernel flags
// ERRBIT_TIMEOUT, as a stalled march would.  No copy is in flight.
__global__ void wait_selftest_kernel(int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) atomicOr(err, ERRBIT_TIMEOUT);
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
  static const EncodeFn fn = [] {  // thread-safe static initialisation
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeFn)p;
    return (EncodeFn) nullptr;
  }();
  return fn;
}

// tile shapes: FP32 128-node strips, 4-slot ring, 4 CTAs per SM;
// FP64 64-node strips (same box bytes), 4-slot ring
template <typename R> struct Tile;
#ifndef MRTLB_PAIR_BX
#define MRTLB_PAIR_BX 128
#endif
template <> struct Tile<float> { static constexpr int BX = MRTLB_PAIR_BX, NSLOT = 4, MINB = 4; };
template <> struct Tile<double> { static constexpr int BX = 64, NSLOT = 4, MINB = 1; };

#ifndef MRTLB_PAIR
#define MRTLB_PAIR 1
#endif
#ifndef MRTLB_PAIR_MINB
#define MRTLB_PAIR_MINB 4
#endif

// The FP32 coefficient block with every constant in both lanes of a pair.
Coef<P2> pair_coef(const Coef<float>& c) {
  static_assert(offsetof(Coef<float>, version) % sizeof(float) == 0, "layout");
  constexpr int n = (int)(offsetof(Coef<float>, version) / sizeof(float));
  static_assert(offsetof(Coef<P2>, version) == n * sizeof(P2), "layout");
  Coef<P2> p;
  const float* src = &c.a1x;
  P2* dst = &p.a1x;
  for (int i = 0; i < n; ++i) dst[i] = P2(src[i]);
  p.version = c.version;
  p.modified = c.modified;
  return p;
}

}  // namespace

void plan_segments(const Layout& L, int target_ctas, TiledPlan* plan) {
  const int nj = L.j1 - L.j0;
  plan->nstrips = (L.i1 + plan->bx - 1) / plan->bx;
  if (plan->nstrips < 1) plan->nstrips = 1;
  int nseg = target_ctas / plan->nstrips;
  if (nseg < 1) nseg = 1;
  int seglen = (nj + nseg - 1) / nseg;
  if (seglen < 8) seglen = 8;
  if (seglen > nj) seglen = nj > 0 ? nj : 1;
  plan->seglen = seglen;
  plan->nseg = (nj + seglen - 1) / seglen;
}

int plan_tiled(const Layout& L, int esize, void* f0, void* f1, TiledPlan* plan) {
  plan->ok = false;
  plan->esize = esize;
  EncodeFn enc = get_encode();
  if (!enc) return 1;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nsm <= 0) nsm = 152;
  int minb;
  if (esize == 4) {
    plan->bx = Tile<float>::BX;
    plan->nslot = Tile<float>::NSLOT;
    plan->smem = Smem<float, Tile<float>::BX, Tile<float>::NSLOT>::bytes;
    minb = Tile<float>::MINB;
  } else {
    plan->bx = Tile<double>::BX;
    plan->nslot = Tile<double>::NSLOT;
    plan->smem = Smem<double, Tile<double>::BX, Tile<double>::NSLOT>::bytes;
    minb = 3;
  }
  const int rc = encode_row_maps(L, esize, f0, f1, plan->bx, plan->map);
  if (rc) return rc;
  // resident CTAs per SM (shared memory and the launch bound); one full wave
  int per_sm = (int)((227 * 1024) / (plan->smem + 1024));
  if (per_sm > minb) per_sm = minb;
  if (esize == 4 && MRTLB_PAIR) {  // the kernel launched for FP32: ask the runtime
    constexpr int BX = Tile<float>::BX, NS = Tile<float>::NSLOT;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_pair_kernel<BX, NS, MRTLB_PAIR_MINB>, BX / 2,
                                                      PairSmem<BX, NS>::bytes) == cudaSuccess && n > 0)
      per_sm = n;
    plan->smem = PairSmem<BX, NS>::bytes;
  }
  if (per_sm < 1) per_sm = 1;
  // the dynamic shared memory of the kernel launch_step_tiled will launch,
  // allowed in the current context (here: once per bind, on the bound
  // device, outside any stream capture)
  {
    const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    constexpr int BXf = Tile<float>::BX, NSf = Tile<float>::NSLOT, MBf = Tile<float>::MINB;
    constexpr int BXd = Tile<double>::BX, NSd = Tile<double>::NSLOT, MBd = Tile<double>::MINB;
    cudaError_t e;
    if (esize == 4 && MRTLB_PAIR)
      e = cudaFuncSetAttribute(step_pair_kernel<BXf, NSf, MRTLB_PAIR_MINB>, A, (int)PairSmem<BXf, NSf>::bytes);
    else if (esize == 4)
      e = cudaFuncSetAttribute(step_tiled_kernel<float, BXf, NSf, MBf>, A, (int)Smem<float, BXf, NSf>::bytes);
    else
      e = cudaFuncSetAttribute(step_tiled_kernel<double, BXd, NSd, MBd>, A, (int)Smem<double, BXd, NSd>::bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return 4;
    }
  }
  // One wave of resident CTAs; for the FP32 march the most waves, up to
  // four, whose segments keep at least kWaveRows rows (each wave then marches
  // a band of rows across the whole width).  Measured on GB300 (ms per step):
  // 4096 x 1024 0.0977 with one wave -> 0.0927 with two (segments of 54 ->
  // 27 rows); 2048 x 2048 0.0984 -> 0.0949 (two); 4096 x 1536 0.146 -> 0.136
  // (two) -> 0.1357 (three); 4096 x 2048 0.205 -> 0.184 (two) -> 0.179
  // (four); 4096 x 4096 0.382 (two) -> 0.356 (four); 3072 x 1024 0.0734 ->
  // 0.0720 (21 rows), but 3000 x 1000 0.0798 -> 0.0810 (20 rows, a ragged
  // last strip); a partial last wave (1.5 waves: 0.118 on 4096 x 1024)
  // leaves SMs idle.
  plan_segments(L, nsm * per_sm, plan);
  if (esize == 4 && MRTLB_PAIR) {
    constexpr int kWaveRows = 24;
    for (int waves = 4; waves >= 2; --waves) {
      TiledPlan more = *plan;
      plan_segments(L, waves * nsm * per_sm, &more);
      if (more.seglen >= kWaveRows) {
        plan->nstrips = more.nstrips;
        plan->nseg = more.nseg;
        plan->seglen = more.seglen;
        break;
      }
    }
  }
  plan->ok = true;
  return 0;
}

int encode_row_maps(const Layout& L, int esize, void* f0, void* f1, int bx, CUtensorMap out[2]) {
  EncodeFn enc = get_encode();
  if (!enc) return 1;
  const int hl = 16 / esize;
  if (((L.xoff - hl) * esize) % 16 != 0 || (bx * esize) % 16 != 0 || bx + 2 * hl > 256) return 3;
  const cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)(L.ny + 2), 16};
  const cuuint64_t strides[2] = {(cuuint64_t)L.pitch * esize, (cuuint64_t)L.plane * esize};
  const cuuint32_t box[3] = {(cuuint32_t)(bx + 2 * hl), 1, 16};
  const cuuint32_t estr[3] = {1, 1, 1};
  void* bufs[2] = {f0, f1};
  for (int b = 0; b < 2; ++b) {
    CUresult r = enc(&out[b], esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                     3, bufs[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return 2;
  }
  return 0;
}

bool tiled_supported(const TiledPlan& plan) { return plan.ok; }

bool use_tiled(int which, const TiledPlan& plan, bool fp64) {
  (void)fp64;
  if (!plan.ok) return false;
  if (which == MRTLB_KERNEL_PLAIN) return false;
  if (which == MRTLB_KERNEL_TILED) return true;
  // AUTO: a march of a few rows is latency-bound (each row waits for its
  // copy); small grids go to the one-thread-per-node kernel
  return plan.seglen >= kMinMarchRows;
}

template <typename R>
void launch_step_tiled(const TiledPlan& plan, int cur, const Layout& L, const Coef<R>& c, int* err,
                       cudaStream_t st, void* fout) {
  constexpr int BX = Tile<R>::BX, NS = Tile<R>::NSLOT, MB = Tile<R>::MINB;
  if (L.i1 <= L.i0 || L.j1 <= L.j0) return;
  dim3 grd(plan.nstrips, plan.nseg);
  if constexpr (sizeof(R) == 4 && MRTLB_PAIR) {
    using SM = PairSmem<BX, NS>;
    step_pair_kernel<BX, NS, MRTLB_PAIR_MINB><<<grd, BX / 2, SM::bytes, st>>>(
        plan.map[cur], (float*)fout, L, pair_coef(reinterpret_cast<const Coef<float>&>(c)), err, plan.seglen);
  } else {
    using SM = Smem<R, BX, NS>;
    step_tiled_kernel<R, BX, NS, MB><<<grd, BX, SM::bytes, st>>>(plan.map[cur], (R*)fout, L, c, err,
                                                                 plan.seglen);
  }
}

void launch_wait_selftest(int* err, cudaStream_t st) { wait_selftest_kernel<<<1, 32, 0, st>>>(err); }

template void launch_step_tiled<float>(const TiledPlan&, int, const Layout&, const Coef<float>&, int*,
                                       cudaStream_t, void*);
template void launch_step_tiled<double>(const TiledPlan&, int, const Layout&, const Coef<double>&, int*,
                                        cudaStream_t, void*);

}  // namespace mrtlb
