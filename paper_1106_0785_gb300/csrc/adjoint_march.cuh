// adjoint_march.cuh - one adjoint step as a single TMA-fed row march.
//
// The adjoint of the step at node p needs, besides B(f)(p) and lambda(p):
// lambda at the four cross neighbours (Lax-Wendroff transpose), u at the
// four neighbours (the strain combinations of the forward collision), and
// the strain-combination adjoints gbar at the four neighbours (the
// modification at r reaches u(p) through its central differences).  The
// two-pass path computes u and gbar into planes first; here they are
// computed per row as the row arrives and kept in a 4-row shared ring, so
// that one kernel reads B(f) and lambda once and writes lambda~ once.
//
// Thread t of a CTA owns column x = x0-2+t: it computes u, 1/rho and gbar
// of that column for every row, and lambda~ of its column if 1 <= t <= SX
// (SX = BX-4 output columns x0-1 .. x0+SX-2; strips start at multiples of
// SX, a multiple of 16 bytes, and overlap by 4 columns so that every
// neighbour an output needs is prepared by a thread of the same CTA).  A CTA
// also owns a segment of output rows [ja, jb) within -1 .. ny.  Rows ja-1 .. jb stream in through
// cp.async.bulk.tensor, one 3D box per row and array (16 planes x BX + 2 HL
// columns starting at x0 - HL, 16-byte aligned):
//   * B(f) rows into an NF-slot ring: row r is read by the prep of r (own
//     and halo columns) and by the core of r (own column);
//   * lambda rows into an NL-slot ring: row r is read by the prep of r and
//     by the cores of rows r-1, r, r+1.
// Rows outside the padded grid (-2 and ny+1) load as zeros (TMA fill) and
// are never used by an advanced node.  Per output row j the CTA:
//   1. waits for row j+1, computes u, 1/rho, gbar of row j+1 for its BX
//      columns into the ring;
//   2. agrees at a barrier (barrier-or of expired waits), refills the slots
//      freed by row j-1 (B(f)) and j-2 (lambda);
//   3. computes lambda~(x, j) from the rings and writes its 16 planes.
// Every mbarrier wait is bounded (march.cuh): on expiry the CTA stops,
// flags ERRBIT_TIMEOUT and lets its copies in flight land.
#pragma once

#include <cuda.h>

#include "adjoint.cuh"
#include "march.cuh"

namespace mrtlb {
namespace {

template <typename R, int BX, int NF, int NL>
struct AdjSmem {
  static constexpr int HL = 16 / (int)sizeof(R);  // halo columns either side of the box
  static constexpr int BW = BX + 2 * HL;          // box width (elements)
  static constexpr int ROW = 16 * BW;             // elements of one row (16 planes)
  static constexpr int SX = BX - 4;               // output columns per strip (strip stride)
  static constexpr int PW = BX;                   // prep columns x0-2 .. x0+BX-3
  static constexpr int NP = 5;                    // u_x, u_y, gbar_shear, gbar_strain, 1/rho
  static constexpr int PROW = NP * PW;
  static constexpr size_t row_bytes = (size_t)ROW * sizeof(R);
  static constexpr size_t l_off = (size_t)NF * row_bytes;
  static constexpr size_t p_off = l_off + (size_t)NL * row_bytes;
  static constexpr size_t bar_off = (p_off + (size_t)4 * PROW * sizeof(R) + 15) & ~(size_t)15;
  static constexpr size_t bytes = bar_off + (size_t)(NF + NL) * sizeof(uint64_t);
};

template <typename R, int BX, int NF, int NL>
struct AdjMarch {
  using SM = AdjSmem<R, BX, NF, NL>;
  R* fs;              // B(f) ring
  R* ls;              // lambda ring
  R* ps;              // prep ring (4 rows)
  uint64_t* fbar;     // one mbarrier per B(f) slot
  uint64_t* lbar;     // one per lambda slot
  const CUtensorMap* fmap;
  const CUtensorMap* lmap;
  R* out;
  Layout L;
  int t, x0, x, boxx, r_first, r_last, f_issued, l_issued;
  bool out_col;  // the thread's column is an output of this strip
  bool colC, colW, colE;  // columns x, x-1, x+1 are advanced (fixed per segment)
  __device__ __forceinline__ bool row_adv(int r) const { return r >= L.j0 && r < L.j1; }

  __device__ __forceinline__ int k(int r) const { return r - r_first; }
  __device__ __forceinline__ const R* frow(int r) const { return fs + (k(r) % NF) * SM::ROW; }
  __device__ __forceinline__ const R* lrow(int r) const { return ls + (k(r) % NL) * SM::ROW; }
  __device__ __forceinline__ R* prow(int r) const { return ps + (k(r) & 3) * SM::PROW; }
  __device__ __forceinline__ bool f_ready(int r) const {
    return mbar_wait(&fbar[k(r) % NF], (uint32_t)((k(r) / NF) & 1));
  }
  __device__ __forceinline__ bool l_ready(int r) const {
    return mbar_wait(&lbar[k(r) % NL], (uint32_t)((k(r) / NL) & 1));
  }
  __device__ __forceinline__ void issue_f(int r) {
    const int s = k(r) % NF;
    mbar_expect_tx(&fbar[s], (uint32_t)SM::row_bytes);
    tma_load_row(fs + s * SM::ROW, fmap, boxx, r + 1, &fbar[s]);
  }
  __device__ __forceinline__ void issue_l(int r) {
    const int s = k(r) % NL;
    mbar_expect_tx(&lbar[s], (uint32_t)SM::row_bytes);
    tma_load_row(ls + s * SM::ROW, lmap, boxx, r + 1, &lbar[s]);
  }
  // thread 0, after a barrier: refill every slot whose row is done
  // (B(f) rows up to `fdone`, lambda rows up to `ldone`)
  __device__ __forceinline__ void refill(int fdone, int ldone) {
    if (t != 0) return;
    const int fto = min(fdone + NF, r_last), lto = min(ldone + NL, r_last);
    if (f_issued < fto || l_issued < lto) fence_proxy_async();
    while (f_issued < fto) issue_f(++f_issued);
    while (l_issued < lto) issue_l(++l_issued);
  }

  // u, 1/rho and gbar of column xc of row r (box column bc) into prep index pi
  __device__ __forceinline__ void prep_col(const AdjCoef<R>& a, const R* fr, const R* lr, R* pr, int xc, int r,
                                          int bc, int pi) const {
    R g[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) g[q] = fr[q * SM::BW + bc];
    R rho, jx, jy, e;
    conserved(g, rho, jx, jy, e);
    const R ir = (rho > R(0)) ? adj_inv(rho) : R(0);  // (rows and columns outside the grid are zero)
    const R ux = jx * ir, uy = jy * ir;
    R gsh = R(0), gst = R(0);
    if (a.c.modified && colC && row_adv(r)) {  // (xc is the thread's own column x)
      R lam[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) lam[q] = lr[q * SM::BW + bc];
      gbar_node(a.c, lam, e - R(0.5) * (jx * ux + jy * uy), ux, uy, gsh, gst);
    }
    pr[pi] = ux;
    pr[SM::PW + pi] = uy;
    pr[2 * SM::PW + pi] = gsh;
    pr[3 * SM::PW + pi] = gst;
    pr[4 * SM::PW + pi] = ir;
  }

  // prep of row r: the thread's own column (box column t-2+HL, prep index t)
  __device__ __forceinline__ void prep(const AdjCoef<R>& a, int r) const {
    prep_col(a, frow(r), lrow(r), prow(r), x, r, SM::HL - 2 + t, t);
  }

  // lambda~ of output node (x, j); the rate gradients of the node go to G
  template <bool RATES, int VER>
  __device__ __forceinline__ void core(const AdjCoef<R>& a, int j, R G[16]) const {
    const Coef<R>& c = a.c;
    const int bc = SM::HL - 2 + t;  // box column of x
    const R* pc = prow(j);
    const R* pn = prow(j + 1);
    const R* pp = prow(j - 1);
    const R* lc = lrow(j);
    const R* ln = lrow(j + 1);
    const R* lp_ = lrow(j - 1);
    const int i1 = t;  // prep index of x
    const R ux = pc[i1], uy = pc[SM::PW + i1];
    R lt[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) lt[q] = R(0);
    // the modification at the neighbours, through u(p)
    R uxb = R(0), uyb = R(0);
    if (c.modified) {
      const int G0 = 2 * SM::PW, G1 = 3 * SM::PW;
      uxb = c.inv2dx * (pc[G0 + i1 - 1] - pc[G0 + i1 + 1]) + c.inv2dy * (pp[G1 + i1] - pn[G1 + i1]);
      uyb = c.inv2dx * (pc[G1 + i1 - 1] - pc[G1 + i1 + 1]) - c.inv2dy * (pp[G0 + i1] - pn[G0 + i1]);
    }
    const bool rC = row_adv(j);
    if (colC && rC) {
      const R* fr = frow(j);
      R g[16], lp[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        g[q] = fr[q * SM::BW + bc];
        lp[q] = lc[q * SM::BW + bc];
      }
      const R shear = (pc[i1 + 1] - pc[i1 - 1]) * c.inv2dx - (pn[SM::PW + i1] - pp[SM::PW + i1]) * c.inv2dy;
      const R strain = (pc[SM::PW + i1 + 1] - pc[SM::PW + i1 - 1]) * c.inv2dx + (pn[i1] - pp[i1]) * c.inv2dy;
      collision_T_node<R, RATES, VER>(a, g, lp, ux, uy, shear, strain, uxb, uyb, lt, G);
    } else if (c.modified) {
      velocity_T(uxb, uyb, ux, uy, pc[4 * SM::PW + i1], lt);
    }
    // neighbours' Lax-Wendroff weights: r = p - e_x (k_E), p + e_x (k_W), p - e_y (k_N), p + e_y (k_S)
    const bool aW = colW && rC, aE = colE && rC;
    const bool aS = colC && row_adv(j - 1), aN = colC && row_adv(j + 1);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (vx_of(q) != 0) {
        if (aW) lt[q] += c.lw[q][0] * lc[q * SM::BW + bc - 1];
        if (aE) lt[q] += c.lw[q][1] * lc[q * SM::BW + bc + 1];
      }
      if (vy_of(q) != 0) {
        if (aS) lt[q] += c.lw[q][2] * lp_[q * SM::BW + bc];
        if (aN) lt[q] += c.lw[q][3] * ln[q * SM::BW + bc];
      }
    }
    {
      R* o = out + L.node(x, j);
#pragma unroll
      for (int q = 0; q < 16; ++q) o[q * L.plane] = lt[q];
    }
  }

  // Output rows [ja, jb) of the strip at x0 (a multiple of BX).  Returns
  // true if a wait expired (the CTA agreed to stop).
  template <bool RATES, int VER>
  __device__ __forceinline__ bool segment(const AdjCoef<R>& a, int ja, int jb, R G[16]) {
    x = x0 - 2 + t;
    out_col = t >= 1 && t <= SM::SX && x <= L.nx;
    colC = x >= L.i0 && x < L.i1;
    colW = x - 1 >= L.i0 && x - 1 < L.i1;
    colE = x + 1 >= L.i0 && x + 1 < L.i1;
    boxx = L.xoff + x0 - SM::HL;
    r_first = ja - 1;
    r_last = jb;
    f_issued = min(r_first + NF - 1, r_last);
    l_issued = min(r_first + NL - 1, r_last);
    if (t == 0) {
      for (int r = r_first; r <= f_issued; ++r) issue_f(r);
      for (int r = r_first; r <= l_issued; ++r) issue_l(r);
    }
    bool bad = !(f_ready(r_first) && l_ready(r_first));
    if (!bad) prep(a, r_first);
    bad |= !(f_ready(ja) && l_ready(ja));
    if (!bad) prep(a, ja);
    if (__syncthreads_or(bad)) return true;
    for (int j = ja; j < jb; ++j) {
      bad = !(f_ready(j + 1) && l_ready(j + 1));
      if (!bad) prep(a, j + 1);
      if (__syncthreads_or(bad)) return true;
      refill(j - 1, j - 2);
      if (out_col) core<RATES, VER>(a, j, G);
    }
    return false;
  }

  // after a stop: let the copies still in flight land before the CTA's
  // shared memory goes away (only the latest copy of each slot can be pending)
  __device__ __forceinline__ void drain() {
    if (t == 0) {
      for (int r = max(r_first, f_issued - NF + 1); r <= f_issued; ++r) (void)f_ready(r);
      for (int r = max(r_first, l_issued - NL + 1); r <= l_issued; ++r) (void)l_ready(r);
    }
    __syncthreads();
  }
};

// One CTA per (strip, row segment): strips x0 = blockIdx.x * SX, output
// rows -1 + blockIdx.y * seglen ... (clipped at ny + 1).
// (FP32: three CTAs per SM, the shared-memory limit, so at most 170 registers)
// VER: the equilibrium version fixed at compile time (1), or 0 to follow the
// coefficients' (the version-2 and -3 transposes then stay out of the
// version-1 kernels: 111 instead of 168 registers in FP32 with the rate
// gradients, and fewer instruction-fetch stalls).
template <typename R, int BX, int NF, int NL, bool RATES, int VER>
__global__ void __launch_bounds__(BX, sizeof(R) == 4 ? 3 : 1)
    adj_march_kernel(const __grid_constant__ CUtensorMap fmap, const __grid_constant__ CUtensorMap lmap,
                     R* __restrict__ out, const Layout L, const __grid_constant__ AdjCoef<R> a, double* gacc,
                     int* err,
                     const int seglen) {
  static_assert(NF >= 3 && NL >= 4, "ring depths: B(f) >= 3, lambda >= 4");
  using SM = AdjSmem<R, BX, NF, NL>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int ja = -1 + (int)blockIdx.y * seglen;
  const int jb = min(ja + seglen, L.ny + 1);
  if (ja >= jb) return;  // uniform over the CTA
  AdjMarch<R, BX, NF, NL> m;
  m.fs = reinterpret_cast<R*>(smem_raw);
  m.ls = reinterpret_cast<R*>(smem_raw + SM::l_off);
  m.ps = reinterpret_cast<R*>(smem_raw + SM::p_off);
  m.fbar = reinterpret_cast<uint64_t*>(smem_raw + SM::bar_off);
  m.lbar = m.fbar + NF;
  m.fmap = &fmap;
  m.lmap = &lmap;
  m.out = out;
  m.L = L;
  m.t = threadIdx.x;
  m.x0 = blockIdx.x * SM::SX;
  if (m.t == 0) {
    for (int s = 0; s < NF + NL; ++s) mbar_init(&m.fbar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  R G[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) G[k] = R(0);
  if (m.template segment<RATES, VER>(a, ja, jb, G)) {
    if (m.t == 0) atomicOr(err, ERRBIT_TIMEOUT);
    m.drain();
  }
  if constexpr (RATES) flush_rate_gradients(G, gacc);
}

}  // namespace
}  // namespace mrtlb
