// step_tiled.cu - TMA-fed row-marching step kernel (the FP32 hot path).
//
// Work split: CTA (strip s, segment g) advances the nodes x0 <= x < x0 + BX,
// ja <= j < jb; thread t owns column x0 + t.  For output row j it needs
//   * f at (x, j-1), (x, j), (x, j+1)       - kept in registers, rotated;
//   * f at (x-1, j), (x+1, j)                - read from the row-j slot;
//   * u at the four cross neighbours         - computed once per node when
//     its row arrives, (x, j+-1) in registers, (x+-1, j) through a 3-row
//     shared ring (the strip's two halo columns by lanes 0 and 1).
// Rows arrive through cp.async.bulk.tensor (one 3D box = all 16 planes of
// one row plus a 16-byte halo on each side) into NSLOT slots, each with an
// mbarrier; thread 0 refills the slot of row j-1 once every thread is past
// the barrier of iteration j.  Every mbarrier wait is bounded: on expiry
// the CTA agrees (barrier-or) to stop, flags ERRBIT_TIMEOUT, waits (again
// bounded) for its copies still in flight and returns.
#include <cuda.h>

#include "step_tiled.cuh"

namespace mrtlb {

namespace {

constexpr long long kSpinLimit = 1LL << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; true when the phase completed
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long k = 0; k < kSpinLimit; ++k)
    if (mbar_test(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_row(void* dst, const CUtensorMap* map, int x, int y,
                                             uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(0), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <typename R>
struct NodeMac {
  R rho, jx, jy, e, ux, uy, T;
};

template <typename R>
__device__ __forceinline__ NodeMac<R> node_macros(const R g[16]) {
  NodeMac<R> m;
  conserved(g, m.rho, m.jx, m.jy, m.e);
  const R ir = recip(m.rho);
  m.ux = m.jx * ir;
  m.uy = m.jy * ir;
  m.T = temperature(m.rho, m.jx, m.jy, m.e, ir);
  return m;
}

template <typename R, int BX, int NSLOT>
struct Smem {
  static constexpr int HL = 16 / (int)sizeof(R);  // halo columns either side
  static constexpr int BW = BX + 2 * HL;          // box width (elements)
  static constexpr int SLOT = 16 * BW;            // elements per slot
  static constexpr size_t slot_bytes = (size_t)SLOT * sizeof(R);
  static constexpr size_t u_off = (size_t)NSLOT * slot_bytes;
  static constexpr size_t u_bytes = (size_t)3 * 2 * (BX + 2) * sizeof(R);
  static constexpr size_t bar_off = (u_off + u_bytes + 15) & ~(size_t)15;
  static constexpr size_t bytes = bar_off + NSLOT * sizeof(uint64_t);
};

template <typename R, int BX, int NSLOT>
__global__ void __launch_bounds__(BX) step_tiled_kernel(const __grid_constant__ CUtensorMap tmap,
                                                        R* __restrict__ fout, const Layout L,
                                                        const Coef<R> c, int* err, const int seglen) {
  using SM = Smem<R, BX, NSLOT>;
  constexpr int HL = SM::HL, BW = SM::BW, SLOT = SM::SLOT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R* slots = reinterpret_cast<R*>(smem_raw);
  R* U = reinterpret_cast<R*>(smem_raw + SM::u_off);  // [3][2][BX+2]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + SM::bar_off);

  const int t = threadIdx.x;
  // strips start on multiples of BX so that every TMA box starts on a
  // 16-byte boundary (xoff - HL and BX are multiples of 16 bytes)
  const int x0 = blockIdx.x * BX;
  const int x = x0 + t;
  const int ja = L.j0 + blockIdx.y * seglen;
  const int jb = min(ja + seglen, L.j1);
  if (ja >= jb) return;  // uniform over the CTA
  const bool active = x >= L.i0 && x < L.i1;
  const int boxx = L.xoff + x0 - HL;
  const int r_first = ja - 1, r_last = jb;  // grid rows streamed in

  if (t == 0) {
    for (int s = 0; s < NSLOT; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int r) {
    const int k = r - r_first, s = k % NSLOT;
    mbar_expect_tx(&bars[s], (uint32_t)SM::slot_bytes);
    tma_load_row(slots + s * SLOT, &tmap, boxx, r + 1, &bars[s]);
  };
  auto ready = [&](int r) -> bool {
    const int k = r - r_first;
    return mbar_wait(&bars[k % NSLOT], (uint32_t)((k / NSLOT) & 1));
  };
  auto slot_of = [&](int r) -> const R* { return slots + ((r - r_first) % NSLOT) * SLOT; };
  auto urow = [&](int r) -> R* { return U + ((r - r_first) % 3) * 2 * (BX + 2); };

  if (t == 0) {
    for (int k = 0; k < NSLOT && r_first + k <= r_last; ++k) issue(r_first + k);
  }
  int issued_to = min(r_first + NSLOT - 1, r_last);

  // prologue: rows ja-1 and ja
  R fprev[16], fcur[16], fnext[16];
  bool bad = !ready(r_first);
  {
    const R* sl = slot_of(r_first);
#pragma unroll
    for (int q = 0; q < 16; ++q) fprev[q] = sl[q * BW + HL + t];
  }
  bad |= !ready(ja);
  NodeMac<R> mp = node_macros(fprev), mc;
  {
    const R* sl = slot_of(ja);
#pragma unroll
    for (int q = 0; q < 16; ++q) fcur[q] = sl[q * BW + HL + t];
    mc = node_macros(fcur);
    R* u = urow(ja);
    u[t + 1] = mc.ux;
    u[(BX + 2) + t + 1] = mc.uy;
    if (t < 2) {  // halo columns x0-1 (t = 0) and x0+BX (t = 1)
      const int col = (t == 0) ? HL - 1 : HL + BX;
      R g[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) g[q] = sl[q * BW + col];
      const NodeMac<R> mh = node_macros(g);
      const int ui = (t == 0) ? 0 : BX + 1;
      u[ui] = mh.ux;
      u[(BX + 2) + ui] = mh.uy;
    }
  }

  int stopped = 0;
  for (int j = ja; j < jb; ++j) {
    bad |= !ready(j + 1);
    const R* sn = slot_of(j + 1);
#pragma unroll
    for (int q = 0; q < 16; ++q) fnext[q] = sn[q * BW + HL + t];
    const NodeMac<R> mn = node_macros(fnext);
    {
      R* u = urow(j + 1);
      u[t + 1] = mn.ux;
      u[(BX + 2) + t + 1] = mn.uy;
      if (t < 2) {
        const int col = (t == 0) ? HL - 1 : HL + BX;
        R g[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) g[q] = sn[q * BW + col];
        const NodeMac<R> mh = node_macros(g);
        const int ui = (t == 0) ? 0 : BX + 1;
        u[ui] = mh.ux;
        u[(BX + 2) + ui] = mh.uy;
      }
    }
    if (__syncthreads_or(bad)) {
      stopped = 1;
      break;
    }
    // the slot of row j-1 is free: stream in the next row
    if (t == 0 && issued_to < r_last) {
      fence_proxy_async();
      ++issued_to;
      issue(issued_to);
    }
    const R* sc = slot_of(j);
    const R* u = urow(j);
    const R dux_dx = (u[t + 2] - u[t]) * c.inv2dx;
    const R duy_dx = (u[(BX + 2) + t + 2] - u[(BX + 2) + t]) * c.inv2dx;
    const R dux_dy = (mn.ux - mp.ux) * c.inv2dy;
    const R duy_dy = (mn.uy - mp.uy) * c.inv2dy;
    R C[16];
    collision(c, fcur, dux_dx, dux_dy, duy_dx, duy_dy, mc.rho, mc.jx, mc.jy, mc.e, mc.ux, mc.uy, mc.T, C);
    const long long at = L.node(x, j);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const R fc = fcur[q];
      R A = R(0);
      if (vx_of(q) != 0) {
        const R ax = R(vx_of(q)) * c.a1x, bx = R(vx_of(q) * vx_of(q)) * c.b1x;
        const R fe = sc[q * BW + HL + t + 1], fw = sc[q * BW + HL + t - 1];
        A += ax * (fe - fw) - bx * (fe - R(2) * fc + fw);
      }
      if (vy_of(q) != 0) {
        const R ay = R(vy_of(q)) * c.a1y, by = R(vy_of(q) * vy_of(q)) * c.b1y;
        A += ay * (fnext[q] - fprev[q]) - by * (fnext[q] - R(2) * fc + fprev[q]);
      }
      if (active) fout[q * L.plane + at] = fc - A - C[q];
    }
    if (active && (!(mc.rho > R(0)) || !(mc.T > R(0)))) atomicOr(err, ERRBIT_NONPHYSICAL);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      fprev[q] = fcur[q];
      fcur[q] = fnext[q];
    }
    mp = mc;
    mc = mn;
  }
  if (stopped) {
    if (t == 0) {
      atomicOr(err, ERRBIT_TIMEOUT);
      // let copies still in flight land before the CTA's smem goes away
      // (the latest copy of each slot is the only one that can be pending)
      for (int r = max(r_first, issued_to - NSLOT + 1); r <= issued_to; ++r) (void)ready(r);
    }
    __syncthreads();
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
  }
  return fn;
}

template <typename R>
constexpr int tile_bx() { return sizeof(R) == 4 ? 128 : 64; }
template <typename R>
constexpr int tile_nslot() { return sizeof(R) == 4 ? 6 : 4; }

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
  if (esize == 4) {
    plan->bx = tile_bx<float>();
    plan->nslot = tile_nslot<float>();
    plan->smem = Smem<float, tile_bx<float>(), tile_nslot<float>()>::bytes;
  } else {
    plan->bx = tile_bx<double>();
    plan->nslot = tile_nslot<double>();
    plan->smem = Smem<double, tile_bx<double>(), tile_nslot<double>()>::bytes;
  }
  const int hl = 16 / esize;
  if (((L.xoff - hl) * esize) % 16 != 0 || (plan->bx * esize) % 16 != 0) return 3;
  const cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)(L.ny + 2), 16};
  const cuuint64_t strides[2] = {(cuuint64_t)L.pitch * esize, (cuuint64_t)L.plane * esize};
  const cuuint32_t box[3] = {(cuuint32_t)(plan->bx + 2 * hl), 1, 16};
  const cuuint32_t estr[3] = {1, 1, 1};
  void* bufs[2] = {f0, f1};
  for (int b = 0; b < 2; ++b) {
    CUresult r = enc(&plan->map[b], esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                     3, bufs[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return 2;
  }
  // resident CTAs per SM bound by shared memory; aim for one full wave
  int per_sm = (int)((227 * 1024) / (plan->smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  plan_segments(L, nsm * per_sm, plan);
  plan->ok = true;
  return 0;
}

bool tiled_supported(const TiledPlan& plan) { return plan.ok; }

bool use_tiled(int which, const TiledPlan& plan, bool fp64) {
  (void)fp64;
  if (!plan.ok) return false;
  if (which == MRTLB_KERNEL_PLAIN) return false;
  return true;
}

template <typename R>
void launch_step_tiled(const TiledPlan& plan, int cur, const Layout& L, const Coef<R>& c, int* err,
                       cudaStream_t st, void* fout) {
  constexpr int BX = tile_bx<R>(), NS = tile_nslot<R>();
  using SM = Smem<R, BX, NS>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(step_tiled_kernel<R, BX, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)SM::bytes);
    attr = true;
  }
  if (L.i1 <= L.i0 || L.j1 <= L.j0) return;
  dim3 grd(plan.nstrips, plan.nseg);
  step_tiled_kernel<R, BX, NS><<<grd, BX, SM::bytes, st>>>(plan.map[cur], (R*)fout, L, c, err, plan.seglen);
}

template void launch_step_tiled<float>(const TiledPlan&, int, const Layout&, const Coef<float>&, int*,
                                       cudaStream_t, void*);
template void launch_step_tiled<double>(const TiledPlan&, int, const Layout&, const Coef<double>&, int*,
                                        cudaStream_t, void*);

}  // namespace mrtlb
