// march.cuh - device side of the row-marching step (shared by the single-
// instance kernel in step_tiled.cu and the batched kernel in batch.cu).
//
// A CTA owns a strip of BX columns and advances a segment of rows of one
// grid; thread t owns column x0 + t.  For output row j it needs
//   * f at (x, j-1), (x, j), (x, j+1)       - kept in registers;
//   * f at (x-1, j), (x+1, j)                - read from the row-j slot;
//   * u at the four cross neighbours         - computed once per node when
//     its row arrives, (x, j+-1) in registers, (x+-1, j) through a 4-row
//     shared ring (the strip's two halo columns by lanes 0 and 1).
// Rows arrive through cp.async.bulk.tensor (one 3D box = all 16 planes of
// one row plus a 16-byte halo on each side) into NSLOT slots, each with an
// mbarrier; thread 0 refills the slot of row j-1 once every thread is past
// the barrier of iteration j.  The three register rows shift down by copies
// after every row (MRTLB_MARCH_UNROLL3=1 unrolls three rows so that they
// trade roles instead; measured slower on GB300: instruction-cache misses).
// Slot phases run on across the segments a persistent CTA takes in turn
// (kbase counts the rows it has streamed so far).
//
// Every mbarrier wait is bounded (about 2 s of wall clock, read from the
// global timer): on expiry the CTA agrees (barrier-or) to stop and the
// caller flags ERRBIT_TIMEOUT and drains the copies still in flight.
#pragma once

#include <cuda.h>

#include "kernels.cuh"

namespace mrtlb {
namespace {

#ifndef MRTLB_MARCH_UNROLL3
#define MRTLB_MARCH_UNROLL3 0
#endif

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s
constexpr unsigned kSuspendHintNs = 1000000u;                // 1 ms per poll

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
// one poll; the thread may sleep up to the hint waiting for the phase
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait; true when the phase completed
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_test(bar, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
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

template <typename R, int BX, int NSLOT>
struct Smem {
  static_assert((NSLOT & (NSLOT - 1)) == 0 && NSLOT >= 4, "NSLOT: power of two >= 4");
  static constexpr int HL = 16 / (int)sizeof(R);  // halo columns either side
  static constexpr int BW = BX + 2 * HL;          // box width (elements)
  static constexpr int SLOT = 16 * BW;            // elements per slot
  static constexpr int UROW = 2 * (BX + 2);       // u_x, u_y of one row incl. halo
  static constexpr size_t slot_bytes = (size_t)SLOT * sizeof(R);
  static constexpr size_t u_off = (size_t)NSLOT * slot_bytes;
  static constexpr size_t u_bytes = (size_t)4 * UROW * sizeof(R);
  static constexpr size_t bar_off = (u_off + u_bytes + 15) & ~(size_t)15;
  static constexpr size_t bytes = bar_off + NSLOT * sizeof(uint64_t);
};

// Everything one CTA needs while it marches.
template <typename R, int BX, int NSLOT>
struct March {
  using SM = Smem<R, BX, NSLOT>;
  R* slots;
  R* U;
  uint64_t* bars;
  const CUtensorMap* map;
  R* fout;
  int* err;
  long long plane;
  int t, x, boxx, r_first, r_last, issued_to, kbase;
  bool active;
  Layout L;

  __device__ __forceinline__ int k(int r) const { return kbase + r - r_first; }
  __device__ __forceinline__ const R* slot(int r) const { return slots + (k(r) & (NSLOT - 1)) * SM::SLOT; }
  __device__ __forceinline__ R* urow(int r) const { return U + (k(r) & 3) * SM::UROW; }
  __device__ __forceinline__ bool ready(int r) const {
    return mbar_wait(&bars[k(r) & (NSLOT - 1)], (uint32_t)((k(r) / NSLOT) & 1));
  }
  __device__ __forceinline__ void issue(int r) {
    const int s = k(r) & (NSLOT - 1);
    mbar_expect_tx(&bars[s], (uint32_t)SM::slot_bytes);
    tma_load_row(slots + s * SM::SLOT, map, boxx, r + 1, &bars[s]);
  }
  // load own column of row r, its macros, publish u (own + strip halo)
  __device__ __forceinline__ void arrive(int r, R f[16], NodeMac<R>& m) const {
    const R* sl = slot(r);
#pragma unroll
    for (int q = 0; q < 16; ++q) f[q] = sl[q * SM::BW + SM::HL + t];
    m = node_macros(f);
    R* u = urow(r);
    u[t + 1] = m.ux;
    u[(BX + 2) + t + 1] = m.uy;
    if (t < 2) {  // halo columns x0-1 (t = 0) and x0+BX (t = 1)
      const int col = (t == 0) ? SM::HL - 1 : SM::HL + BX;
      R g[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) g[q] = sl[q * SM::BW + col];
      const NodeMac<R> mh = node_macros(g);
      const int ui = (t == 0) ? 0 : BX + 1;
      u[ui] = mh.ux;
      u[(BX + 2) + ui] = mh.uy;
    }
  }
  // one output row j; fp/fc hold rows j-1, j, fn receives row j+1.
  // Returns true if the CTA must stop (a wait expired).
  __device__ __forceinline__ bool row(int j, const Coef<R>& c, const R (&fp)[16], const R (&fc)[16],
                                      R (&fn)[16], const NodeMac<R>& mp, const NodeMac<R>& mc,
                                      NodeMac<R>& mn) {
    const bool bad = !ready(j + 1);
    arrive(j + 1, fn, mn);
    if (__syncthreads_or(bad)) return true;
    // the slot of row j-1 is free: stream in the next row
    if (t == 0 && issued_to < r_last) {
      fence_proxy_async();
      ++issued_to;
      issue(issued_to);
    }
    const R* sc = slot(j);
    const R* u = urow(j);
    const R dux_dx = (u[t + 2] - u[t]) * c.inv2dx;
    const R duy_dx = (u[(BX + 2) + t + 2] - u[(BX + 2) + t]) * c.inv2dx;
    const R dux_dy = (mn.ux - mp.ux) * c.inv2dy;
    const R duy_dy = (mn.uy - mp.uy) * c.inv2dy;
    R C[16];
    collision(c, fc, dux_dx, dux_dy, duy_dx, duy_dy, mc.rho, mc.ir, mc.jx, mc.jy, mc.e, mc.ux, mc.uy,
              mc.T, C);
    R* out = fout + L.node(x, j);
    R vout[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const R fE = (vx_of(q) != 0) ? sc[q * SM::BW + SM::HL + t + 1] : R(0);
      const R fW = (vx_of(q) != 0) ? sc[q * SM::BW + SM::HL + t - 1] : R(0);
      const R v = lw_update(c, q, fc[q], C[q], fE, fW, fn[q], fp[q]);
      if (active) out[q * plane] = v;
      vout[q] = v;
    }
    if (active) {
      const GhostTargets g = ghost_targets(L, x, j);
      if (g.any()) write_ghosts(g, plane, vout, out);
    }
    if (active && (!(mc.rho > R(0)) || !(mc.T > R(0)))) atomicOr(err, ERRBIT_NONPHYSICAL);
    return false;
  }

  // Advance rows [ja, jb) of the strip starting at column x0 (a multiple of
  // BX); rows ja-1 .. jb stream in.  Returns true if a wait expired (the
  // CTA agreed to stop).  Leaves kbase past the rows it streamed.
  __device__ __forceinline__ bool segment(const Coef<R>& c, int x0, int ja, int jb) {
    x = x0 + t;
    active = x >= L.i0 && x < L.i1;
    boxx = L.xoff + x0 - SM::HL;
    r_first = ja - 1;
    r_last = jb;
    if (t == 0)
      for (int kk = 0; kk < NSLOT && r_first + kk <= r_last; ++kk) issue(r_first + kk);
    issued_to = min(r_first + NSLOT - 1, r_last);

    R F0[16], F1[16], F2[16];
    NodeMac<R> M0, M1, M2;
    bool bad = !ready(r_first);
    arrive(r_first, F0, M0);
    bad |= !ready(ja);
    arrive(ja, F1, M1);
    bool stopped = __syncthreads_or(bad);
#if MRTLB_MARCH_UNROLL3
    // rows j-1, j, j+1 live in (F0, F1, F2), then (F1, F2, F0), then (F2, F0, F1)
    for (int j = ja; !stopped && j < jb; j += 3) {
      if ((stopped = row(j, c, F0, F1, F2, M0, M1, M2))) break;
      if (j + 1 >= jb) break;
      if ((stopped = row(j + 1, c, F1, F2, F0, M1, M2, M0))) break;
      if (j + 2 >= jb) break;
      if ((stopped = row(j + 2, c, F2, F0, F1, M2, M0, M1))) break;
    }
#else
    // one body, rows shifted down by register copies
    for (int j = ja; !stopped && j < jb; ++j) {
      if ((stopped = row(j, c, F0, F1, F2, M0, M1, M2))) break;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        F0[q] = F1[q];
        F1[q] = F2[q];
      }
      M0 = M1;
      M1 = M2;
    }
#endif
    if (!stopped) kbase += r_last - r_first + 1;
    return stopped;
  }

  // after a stop: let copies still in flight land before the CTA's smem goes
  // away (the latest copy of each slot is the only one that can be pending)
  __device__ __forceinline__ void drain() {
    if (t == 0)
      for (int r = max(r_first, issued_to - NSLOT + 1); r <= issued_to; ++r) (void)ready(r);
    __syncthreads();
  }
};


}  // namespace
}  // namespace mrtlb
