// march_pair.cuh - the FP32 row march with two nodes per thread.
//
// Same pipeline as march.cuh (one CTA per strip of BX columns and a segment
// of rows; each row arrives by one TMA box into an NSLOT ring with bounded
// mbarrier waits), but thread t owns the adjacent columns x0 + 2t and
// x0 + 2t + 1 and carries both nodes in packed FP32 pairs (pair.cuh), so
// that every add, multiply and fused multiply-add of the per-node templates
// serves two nodes, and shared-memory loads and global stores move 8 bytes.
// Of the x-neighbours of the pair, the inner ones are the pair's own values
// and the outer ones one 4-byte load each.  u of the two strip halo
// columns comes from lanes 0 and 1.  A CTA has BX/2 threads.
//
// Only row j-1 of the pair's columns stays in registers from one row to
// the next: rows j and j+1 are read from their ring slots, and u, 1/rho
// and T of each row go to a 4-row shared ring when the row arrives.  (The
// earlier form kept rows j-1, j, j+1 and their macros in registers and
// shifted them down after every row: 254 registers against 211 now, and
// about 2% slower on GB300.)
#pragma once

#include <cuda.h>

#include "march.cuh"

namespace mrtlb {
namespace {

template <int BX, int NSLOT>
struct PairSmem {
  using S = Smem<float, BX, NSLOT>;  // the same TMA slots as the scalar march
  static constexpr int HL = S::HL, BW = S::BW, SLOT = S::SLOT;
  static constexpr int UW = BX + 4;          // u row: halo x0-1 at 1, column c at 2 + c, x0+BX at BX+2
  static constexpr int UROW = 4 * UW;        // per ring row: u_x, u_y, 1/rho, T
  static constexpr size_t slot_bytes = S::slot_bytes;
  static constexpr size_t u_off = (size_t)NSLOT * slot_bytes;
  static constexpr size_t bar_off = (u_off + (size_t)4 * UROW * sizeof(float) + 15) & ~(size_t)15;
  static constexpr size_t bytes = bar_off + NSLOT * sizeof(uint64_t);
};

template <int BX, int NSLOT>
struct PairMarch {
  using SM = PairSmem<BX, NSLOT>;
  float* slots;
  float* U;
  uint64_t* bars;
  const CUtensorMap* map;
  float* fout;
  int* err;
  long long plane;
  int t, x, boxx, r_first, r_last, issued_to, kbase;
  int pre = 0;  // rows of this segment already issued while the previous one ran
  bool act0, act1;
  Layout L;
  // the next segment (none unless set by the caller): its map, box column,
  // rows, and how many of its rows are issued so far
  const CUtensorMap* nmap = nullptr;
  int nboxx = 0, n_first = 0, n_last = -1, n_issued = 0;

  __device__ __forceinline__ int k(int r) const { return kbase + r - r_first; }
  __device__ __forceinline__ const float* slot(int r) const {
    return slots + (k(r) & (NSLOT - 1)) * SM::SLOT;
  }
  __device__ __forceinline__ float* urow(int r) const { return U + (k(r) & 3) * SM::UROW; }
  __device__ __forceinline__ bool ready(int r) const {
    return mbar_wait(&bars[k(r) & (NSLOT - 1)], (uint32_t)((k(r) / NSLOT) & 1));
  }
  __device__ __forceinline__ void issue_k(int kk, const CUtensorMap* m, int bx, int r) {
    const int s = kk & (NSLOT - 1);
    mbar_expect_tx(&bars[s], (uint32_t)SM::slot_bytes);
    tma_load_row(slots + s * SM::SLOT, m, bx, r + 1, &bars[s]);
  }
  __device__ __forceinline__ void issue(int r) { issue_k(k(r), map, boxx, r); }
  // thread 0, after a barrier: one row into the slot that just became free
  __device__ __forceinline__ void refill() {
    if (issued_to < r_last) {
      fence_proxy_async();
      ++issued_to;
      issue(issued_to);
    } else if (nmap && n_first + n_issued <= n_last) {
      fence_proxy_async();
      const int kk = kbase + (r_last - r_first + 1) + n_issued;
      issue_k(kk, nmap, nboxx, n_first + n_issued);
      ++n_issued;
    }
  }
  // the next segment (tensor map, box column, output rows [ja, jb)), for
  // refill(); call before segment()
  __device__ __forceinline__ void set_next(const CUtensorMap* m, int box_x, int ja, int jb) {
    nmap = m;
    nboxx = box_x;
    n_first = ja - 1;
    n_last = jb;
    n_issued = 0;
  }
  // The pair's own columns of row r into f, and their u, 1/rho and T
  // published to the ring (u also of the strip's two halo columns).
  __device__ __forceinline__ void arrive(int r, P2 f[16]) const {
    const float* sl = slot(r);
#pragma unroll
    for (int q = 0; q < 16; ++q) f[q] = P2(*reinterpret_cast<const float2*>(sl + q * SM::BW + SM::HL + 2 * t));
    const NodeMac<P2> m = node_macros(f);
    float* u = urow(r) + 2 + 2 * t;
    *reinterpret_cast<float2*>(u) = m.ux.v;
    *reinterpret_cast<float2*>(u + SM::UW) = m.uy.v;
    *reinterpret_cast<float2*>(u + 2 * SM::UW) = m.ir.v;
    *reinterpret_cast<float2*>(u + 3 * SM::UW) = m.T.v;
    if (t < 2) {  // halo columns x0-1 (t = 0) and x0+BX (t = 1)
      const int col = (t == 0) ? SM::HL - 1 : SM::HL + BX;
      float g[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) g[q] = sl[q * SM::BW + col];
      const NodeMac<float> mh = node_macros(g);
      float* uh = urow(r) + ((t == 0) ? 1 : BX + 2);
      uh[0] = mh.ux;
      uh[SM::UW] = mh.uy;
    }
  }
  __device__ __forceinline__ static P2 ld2(const float* p) { return P2(*reinterpret_cast<const float2*>(p)); }

  // One output row j for both columns.  Row j-1 of the pair's columns is
  // in fp; row j is read from its slot into fc (the caller's fp of the next
  // row), row j+1 from its slot; rho, j and e are recomputed from the
  // harmonics the collision needs anyway, u, 1/rho and T come from the
  // ring.  Returns true if the CTA must stop (a wait expired).
  __device__ __forceinline__ bool row(int j, const Coef<P2>& c, const P2 (&fp)[16], P2 (&fc)[16]) {
    if (__syncthreads_or(!ready(j + 1))) return true;
    if (t == 0) refill();
    // row j+1's u, 1/rho and T go to the ring in the same block as row j's
    // update (other threads read them only after the next barrier), so that
    // the two interleave
    {
      P2 fn[16];
      arrive(j + 1, fn);
    }
    const float* sc = slot(j);
    const float* sn = slot(j + 1);
    const int o = SM::HL + 2 * t;  // slot column of x
#pragma unroll
    for (int q = 0; q < 16; ++q) fc[q] = ld2(sc + q * SM::BW + o);
    Harm<P2> h;
    harmonics(fc, h);
    P2 rho, jx, jy, e;
    conserved_h(h, rho, jx, jy, e);
    const float* u = urow(j);
    const float* un = urow(j + 1);
    const float* up = urow(j - 1);
    const int ui = 2 + 2 * t;  // ring index of column x
    const P2 ux = ld2(u + ui), uy = ld2(u + SM::UW + ui);
    const P2 ir = ld2(u + 2 * SM::UW + ui), T = ld2(u + 3 * SM::UW + ui);
    const P2 uxE(u[ui + 1], u[ui + 2]), uxW(u[ui - 1], u[ui]);
    const P2 uyE(u[SM::UW + ui + 1], u[SM::UW + ui + 2]), uyW(u[SM::UW + ui - 1], u[SM::UW + ui]);
    const P2 dux_dx = P2((uxE - uxW) * c.inv2dx), duy_dx = P2((uyE - uyW) * c.inv2dx);
    const P2 dux_dy = P2((ld2(un + ui) - ld2(up + ui)) * c.inv2dy);
    const P2 duy_dy = P2((ld2(un + SM::UW + ui) - ld2(up + SM::UW + ui)) * c.inv2dy);
    P2 C[16];
    collision_h(c, h, dux_dx, dux_dy, duy_dx, duy_dy, rho, ir, jx, jy, e, ux, uy, T, C);
    float* out = fout + L.node(x, j);
    P2 vout[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int b = q * SM::BW + o;
      const P2 fE = (vx_of(q) != 0) ? P2(fc[q].v.y, sc[b + 2]) : P2(0.0f);
      const P2 fW = (vx_of(q) != 0) ? P2(sc[b - 1], fc[q].v.x) : P2(0.0f);
      const P2 fN = (vy_of(q) != 0) ? ld2(sn + b) : P2(0.0f);
      vout[q] = lw_update(c, q, fc[q], C[q], fE, fW, fN, fp[q]);
    }
    store_row(j, out, vout);
    const bool bad0 = act0 && (!(rho.v.x > 0.0f) || !(T.v.x > 0.0f));
    const bool bad1 = act1 && (!(rho.v.y > 0.0f) || !(T.v.y > 0.0f));
    if (bad0 || bad1) atomicOr(err, ERRBIT_NONPHYSICAL);
    return false;
  }

  // the row's new values to the output buffer, and to the ghosts they feed
  __device__ __forceinline__ void store_row(int j, float* out, const P2 (&vout)[16]) const {
    if (act0 && act1) {
#pragma unroll
      for (int q = 0; q < 16; ++q) *reinterpret_cast<float2*>(out + q * plane) = vout[q].v;
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if (act0) out[q * plane] = vout[q].v.x;
        if (act1) out[q * plane + 1] = vout[q].v.y;
      }
    }
#ifndef MRTLB_GHOST_GUARD
#define MRTLB_GHOST_GUARD 1
#endif
    // only nodes on the grid's edges have ghosts to write
    if (!MRTLB_GHOST_GUARD || j == 0 || j == L.ny - 1 || x == 0 || x + 1 >= L.nx - 1) {
      const GhostTargets g0 = ghost_targets(L, x, j), g1 = ghost_targets(L, x + 1, j);
      if (act0 && g0.any()) {
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = vout[q].v.x;
        write_ghosts(g0, plane, v, out);
      }
      if (act1 && g1.any()) {
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = vout[q].v.y;
        write_ghosts(g1, plane, v, out + 1);
      }
    }
  }

  // Advance rows [ja, jb) of the strip at x0 (a multiple of BX); as March.
  __device__ __forceinline__ bool segment(const Coef<P2>& c, int x0, int ja, int jb) {
    x = x0 + 2 * t;
    act0 = x >= L.i0 && x < L.i1;
    act1 = x + 1 >= L.i0 && x + 1 < L.i1;
    boxx = L.xoff + x0 - SM::HL;
    r_first = ja - 1;
    r_last = jb;
    // rows the previous segment already put in flight (pre of them); the
    // slots were read through the generic proxy by the previous segment
    if (t == 0) {
      if (pre < NSLOT) fence_proxy_async();
      for (int kk = pre; kk < NSLOT && r_first + kk <= r_last; ++kk) issue(r_first + kk);
    }
    issued_to = min(r_first + max(pre, NSLOT) - 1, r_last);

    P2 FA[16], FB[16];  // rows j-1 (FA) and j (FB) of the pair's columns
    bool bad = !ready(r_first);
    arrive(r_first, FA);
    bad |= !ready(ja);
    arrive(ja, FB);  // (u, 1/rho, T of row ja; its f is read again from the slot)
    bool stopped = __syncthreads_or(bad);
    for (int j = ja; !stopped && j < jb; ++j) {
      if ((stopped = row(j, c, FA, FB))) break;
#pragma unroll
      for (int q = 0; q < 16; ++q) FA[q] = FB[q];
    }
    if (!stopped) kbase += r_last - r_first + 1;
    return stopped;
  }

  // Hand the prefetched rows of the next segment over: call after segment()
  // returned false and before the next segment() (with its L set).
  __device__ __forceinline__ void advance() {
    pre = nmap ? n_issued : 0;
    nmap = nullptr;
    n_issued = 0;
  }

  __device__ __forceinline__ void drain() {
    if (t == 0) {
      // every copy in flight: the current segment's rows and any of the next
      const int klast = (nmap && n_issued > 0) ? kbase + (r_last - r_first + 1) + n_issued - 1 : k(issued_to);
      for (int kk = max(k(r_first), klast - NSLOT + 1); kk <= klast; ++kk)
        (void)mbar_wait(&bars[kk & (NSLOT - 1)], (uint32_t)((kk / NSLOT) & 1));
    }
    __syncthreads();
  }
};

}  // namespace
}  // namespace mrtlb
