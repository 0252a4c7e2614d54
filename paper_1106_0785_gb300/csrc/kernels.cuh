// kernels.cuh - device layout and kernel launchers shared by the C ABI.
//
// Device layout of one state buffer (private to the library): 16 planes,
// each (ny + 2) rows of `pitch` elements.  Node (i, j) of the grid sits at
// row j + 1 and column i + xoff; row 0 / ny + 1 and columns xoff - 1 /
// xoff + nx are the one-node ghost layer.  xoff = 128 bytes / element size,
// so every interior row starts on a 128-byte boundary, and the TMA box of a
// tile, which starts 4 elements left of the tile, starts on a 16-byte one.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "physics.cuh"

namespace mrtlb {

enum : int { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_WALL = 2, BC_INFLOW = 3, BC_REFLECT = 4, BC_DIFFUSE = 5 };

// The velocity index of v_q with its x (mirror_x) or y (mirror_y) component
// negated: the plane a reflecting side maps q to.
__host__ __device__ constexpr int mirror_x(int q) {
  int m = q;
  for (int p = 0; p < 16; ++p)
    if (vx_of(p) == -vx_of(q) && vy_of(p) == vy_of(q)) m = p;
  return m;
}
__host__ __device__ constexpr int mirror_y(int q) {
  int m = q;
  for (int p = 0; p < 16; ++p)
    if (vx_of(p) == vx_of(q) && vy_of(p) == -vy_of(q)) m = p;
  return m;
}

// Bits of the device error word.
enum : int { ERRBIT_NONPHYSICAL = 1, ERRBIT_TIMEOUT = 2 };

struct Layout {
  int nx, ny;
  int pitch;          // elements per padded row
  int xoff;           // column of interior node i = 0
  long long plane;    // elements per plane = (ny + 2) * pitch
  int i0, i1, j0, j1; // advanced (non-wall) nodes: [i0, i1) x [j0, j1)
  int bc[4];          // -x, +x, -y, +y (BC_*)
  __host__ __device__ long long node(int i, int j) const {
    return (long long)(j + 1) * pitch + (i + xoff);
  }
};

// Ghost cells that mirror an advanced edge node (x, j): periodic sides
// mirror the opposite edge, zero-gradient outflow and reflecting sides their
// own edge (reflection with the velocity set mirrored across the side).
// A step that writes these from the new values keeps the ghost layer of
// f^{n+1} complete, so the next step needs no separate boundary launch.
// Walls have no ghosts in use; inflow ghosts are constant, filled once in
// every state buffer.  Offsets are relative to node (x, j).
struct GhostTargets {
  bool w[4];
  bool mir[4];  // reflecting side: plane q goes to the mirrored plane
  long long off[4];
  __device__ __forceinline__ bool any() const { return w[0] || w[1] || w[2] || w[3]; }
};

__device__ __forceinline__ GhostTargets ghost_targets(const Layout& L, int x, int j) {
  const bool xl = (x == 0), xr = (x == L.nx - 1), yl = (j == 0), yr = (j == L.ny - 1);
  GhostTargets g;
  // ghost column -1 holds column 0 (outflow, reflect) or column nx-1 (periodic), etc.
  g.w[0] = (xl && (L.bc[0] == BC_OUTFLOW || L.bc[0] == BC_REFLECT)) || (xr && L.bc[0] == BC_PERIODIC);
  g.w[1] = (xr && (L.bc[1] == BC_OUTFLOW || L.bc[1] == BC_REFLECT)) || (xl && L.bc[1] == BC_PERIODIC);
  g.w[2] = (yl && (L.bc[2] == BC_OUTFLOW || L.bc[2] == BC_REFLECT)) || (yr && L.bc[2] == BC_PERIODIC);
  g.w[3] = (yr && (L.bc[3] == BC_OUTFLOW || L.bc[3] == BC_REFLECT)) || (yl && L.bc[3] == BC_PERIODIC);
  for (int s = 0; s < 4; ++s) g.mir[s] = (L.bc[s] == BC_REFLECT);
  g.off[0] = -(long long)x - 1;
  g.off[1] = (long long)(L.nx - x);
  g.off[2] = -(long long)(j + 1) * L.pitch;
  g.off[3] = (long long)(L.ny - j) * L.pitch;
  return g;
}

// Write the 16 new values of a node (plane-0 address `out`) to its ghosts.
template <typename R>
__device__ __forceinline__ void write_ghosts(const GhostTargets& g, long long plane, const R v[16],
                                             R* out) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (!g.w[s]) continue;
    R* p = out + g.off[s];
    if (g.mir[s]) {
#pragma unroll
      for (int q = 0; q < 16; ++q) p[(s < 2 ? mirror_x(q) : mirror_y(q)) * plane] = v[q];
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) p[q * plane] = v[q];
    }
  }
}

struct Walls {
  double ux[4], uy[4], T[4];  // per side: wall or inflow velocity and temperature
  double rho[4];              // inflow density
};

// Boundary cells refilled before every step: NEE wall nodes (ny per x side,
// nx per y side) and diffuse-reflection ghost cells (likewise).
__host__ __device__ inline bool refilled_side(int kind) { return kind == BC_WALL || kind == BC_DIFFUSE; }
__host__ __device__ inline int wall_count(const Layout& L) {
  int n = 0;
  for (int s = 0; s < 4; ++s)
    if (refilled_side(L.bc[s])) n += (s < 2) ? L.ny : L.nx;
  return n;
}

// The wall state's equilibrium at unit density, plane q.
template <typename R>
__device__ __forceinline__ void wall_equilibrium(const Coef<R>& c, R ux, R uy, R T, R e[16]) {
  R eq[16];
  equilibrium(c, R(1), R(1), ux, uy, T + R(0.5) * (ux * ux + uy * uy), ux, uy, T, eq);
  inverse_full(c, eq, e);
}

// Diffuse reflection beside edge node `edge` (plane-0 address) on side s:
// the ghost holds rho_w e_q for velocities entering the fluid and the edge
// value otherwise, rho_w such that the Lax-Wendroff update moves no mass
// across the side: with a_q the ghost's weight in the edge node's update
// and b_q the edge node's in the ghost position's,
//   rho_w = (sum_q b_q f_q - sum_{q not entering} a_q f_q) / sum_{q entering} a_q e_q.
template <typename R>
__device__ __forceinline__ bool entering(int s, int q) {
  return (s == 0) ? vx_of(q) > 0 : (s == 1) ? vx_of(q) < 0 : (s == 2) ? vy_of(q) > 0 : vy_of(q) < 0;
}
template <typename R>
__device__ __forceinline__ void diffuse_weights(const Coef<R>& c, int s, int q, R& a, R& b) {
  const int ga = (s == 0) ? 1 : (s == 1) ? 0 : (s == 2) ? 3 : 2;  // lw index of the ghost neighbour
  a = c.lw[q][ga];
  b = c.lw[q][ga ^ 1];
}
template <typename R>
__device__ __forceinline__ void diffuse_ghost(const Coef<R>& c, const Walls& w, const Layout& L, int s,
                                              const R* edge, R* ghost) {
  R e[16], f[16];
  wall_equilibrium(c, (R)w.ux[s], (R)w.uy[s], (R)w.T[s], e);
  // the flux balance in FP64 from the weights the update uses: in FP32 its
  // rounding would leak mass the same way at every step (e cancels out of
  // the balance, so its own rounding does not)
  double num = 0.0, den = 0.0;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    f[q] = edge[(long long)q * L.plane];
    R a, b;
    diffuse_weights(c, s, q, a, b);
    num += (double)b * (double)f[q];
    if (entering<R>(s, q)) den += (double)a * (double)e[q];
    else num -= (double)a * (double)f[q];
  }
  const double rw = num / den;
#pragma unroll
  for (int q = 0; q < 16; ++q)
    ghost[(long long)q * L.plane] = entering<R>(s, q) ? (R)(rw * (double)e[q]) : f[q];
}

template <typename R>
__device__ __forceinline__ void wall_node(R* f, const Layout& L, const Coef<R>& c, const Walls& w, int k) {
  int side = -1, i = 0, j = 0, ia = 0, ja = 0;
  for (int s = 0; s < 4 && side < 0; ++s) {
    const int n = (s < 2) ? L.ny : L.nx;
    if (!refilled_side(L.bc[s])) continue;
    if (k < n) {
      side = s;
      if (s == 0) { i = 0; j = k; ia = 1; ja = k; }
      if (s == 1) { i = L.nx - 1; j = k; ia = L.nx - 2; ja = k; }
      if (s == 2) { i = k; j = 0; ia = k; ja = 1; }
      if (s == 3) { i = k; j = L.ny - 1; ia = k; ja = L.ny - 2; }
    } else {
      k -= n;
    }
  }
  if (side < 0) return;
  if (L.bc[side] == BC_DIFFUSE) {  // the ghost cell beyond edge node (i, j)
    const long long off = (side == 0) ? -1 : (side == 1) ? 1 : (side == 2) ? -(long long)L.pitch : L.pitch;
    diffuse_ghost(c, w, L, side, f + L.node(i, j), f + L.node(i, j) + off);
    return;
  }
  const long long P = L.plane;
  const long long a = L.node(ia, ja), at = L.node(i, j);
  R g[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) g[q] = f[q * P + a];
  R rho, jx, jy, e;
  conserved(g, rho, jx, jy, e);
  const R ir = R(1) / rho;
  const R ux = jx * ir, uy = jy * ir;
  const R T = temperature(rho, jx, jy, e, ir);
  R eqa[16], eqw[16], d[16], df[16];
  equilibrium(c, rho, ir, jx, jy, e, ux, uy, T, eqa);
  const R uwx = (R)w.ux[side], uwy = (R)w.uy[side], Tw = (R)w.T[side];
  const R ew = rho * (Tw + R(0.5) * (uwx * uwx + uwy * uwy));
  equilibrium(c, rho, ir, rho * uwx, rho * uwy, ew, uwx, uwy, Tw, eqw);
#pragma unroll
  for (int q = 0; q < 16; ++q) d[q] = eqw[q] - eqa[q];
  inverse_full(c, d, df);
#pragma unroll
  for (int q = 0; q < 16; ++q) f[q * P + at] = g[q] + df[q];
}

template <typename R>
void launch_step_plain(const R* fin, R* fout, const Layout& L, const Coef<R>& c, int* err,
                       cudaStream_t st);
template <typename R>
void launch_bc(R* f, const Layout& L, const Coef<R>& c, const Walls& w, cudaStream_t st);
// the inflow sides' fixed ghosts only (state buffers a step writes into)
template <typename R>
void launch_inflow(R* f, const Layout& L, const Coef<R>& c, const Walls& w, cudaStream_t st);
// wall nodes only (the per-step fill; the step kernels keep the ghosts)
template <typename R>
void launch_walls(R* f, const Layout& L, const Coef<R>& c, const Walls& w, cudaStream_t st);
template <typename R>
void launch_pack(const R* dense, R* padded, const Layout& L, cudaStream_t st);
template <typename R>
void launch_unpack(const R* padded, R* dense, const Layout& L, cudaStream_t st);
template <typename R>
void launch_init_eq(const double* rho, const double* ux, const double* uy, const double* T,
                    R* f, const Layout& L, const Coef<double>& c64, cudaStream_t st);
template <typename R>
void launch_macros(const R* f, double* rho, double* ux, double* uy, double* T, const Layout& L,
                   cudaStream_t st);
// acc: 4 FP64 sums + 1 max (as the bit pattern of a non-negative double);
// Tprev: [ny][nx] FP64 temperatures of the previous call (updated in place)
template <typename R>
void launch_reduce(const R* f, double* acc, double* Tprev, int have_prev, const Layout& L,
                   cudaStream_t st);

}  // namespace mrtlb
