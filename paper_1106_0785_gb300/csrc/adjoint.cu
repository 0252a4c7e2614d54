// adjoint.cu - reverse (adjoint) of the time step, checkpointed over K steps.
//
// Forward step, per advanced node r (Sec. II-III as implemented):
//   f1(r) = ft(r) + sum_n k_qn (ft(r + e_n) - ft(r)) - C(ft(r), grad u(r))
// where ft = B(f) is the state with walls refilled (NEE) and ghosts filled.
// Given lambda = dL/df1 (zero at non-advanced nodes) the adjoint step is
//   lambda_prev = B^T J^T lambda,
// gathered per node p of the padded grid:
//   (a) Lax-Wendroff: (1 - sum_n k_qn) lambda_q(p) + sum_n k_qn lambda_q(p - e_n);
//   (b) collision at p: -(dC/df(p))^T lambda(p) (equilibrium, temperature
//       and the modification's local factors rho T u, all through M);
//   (c) the modification at the four neighbours r, through u(p) in their
//       central differences: gbar_shear(r), gbar_strain(r) (dL/d of the two
//       strain combinations at r) from a first pass, then u = j / rho at p.
// B^T adds each ghost's adjoint to the node it mirrors and maps each wall
// node's adjoint through the Jacobian of the NEE fill to its fluid
// neighbour (walls themselves get zero).  Gradients with respect to the
// rates s_5..s_16 accumulate in FP64.
//
// K steps run in segments of S: adjoint_forward keeps the states of the
// last segment in slots (all K states, S = K, when K + 2 states fit in half
// the free memory; else S = ceil(sqrt(K)) with a checkpoint per segment);
// backward recomputes any segment whose states are not held from its
// checkpoint (the context keeps f^K) and runs the adjoint steps through it
// in reverse.  A later forward pass of the same shape reuses the buffers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "adjoint.cuh"
#include "adjoint_march.cuh"
#include "ctx.h"

namespace mrtlb {
namespace {

template <typename R>
__device__ __forceinline__ void load16(const R* f, long long plane, long long at, R g[16]) {
#pragma unroll
  for (int q = 0; q < 16; ++q) g[q] = f[q * plane + at];
}

// Pass 1, every node of [-1, nx] x [-1, ny]: the velocity u = j / rho of
// B(f) into two planes and, at advanced nodes, the adjoints of the two
// strain combinations of the modification (zero elsewhere):
//   gbar_shear  = dL/d(du_x/dx - du_y/dy),  gbar_strain = dL/d(du_y/dx + du_x/dy).
template <typename R>
__global__ void adj_prep_kernel(const R* __restrict__ ft, const R* __restrict__ lam, R* Ux, R* Uy, R* gsh,
                                R* gst, Layout L, AdjCoef<R> a) {
  const int i = -1 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
  const int j = -1 + (int)blockIdx.y;
  if (i > L.nx || ((i < 0 || i >= L.nx) && (j < 0 || j >= L.ny))) return;
  const long long at = L.node(i, j);
  R g[16];
  load16(ft, L.plane, at, g);
  R rho, jx, jy, e;
  conserved(g, rho, jx, jy, e);
  const R ir = (rho > R(0)) ? adj_inv(rho) : R(0);
  const R ux = jx * ir, uy = jy * ir;
  Ux[at] = ux;
  Uy[at] = uy;
  if (!advanced<R>(L, i, j) || !a.c.modified) {
    gsh[at] = R(0);
    gst[at] = R(0);
    return;
  }
  R lb[16];
  load16(lam, L.plane, at, lb);
  R sh, sn;
  gbar_node(a.c, lb, e - R(0.5) * (jx * ux + jy * uy), ux, uy, sh, sn);
  gsh[at] = sh;
  gst[at] = sn;
}

template <typename R>
__device__ __forceinline__ R gbar_at(const R* gb, const Layout& L, int i, int j) {
  if (i < -1 || i > L.nx || j < -1 || j > L.ny) return R(0);
  return gb[L.node(i, j)];
}

// Pass 2: lambda~(p) for one node p of [-1, nx] x [-1, ny] (corners
// excluded); the rate gradients of an advanced node are added to G.
template <typename R, bool RATES>
__device__ __forceinline__ void adj_core_node(const R* __restrict__ ft, const R* __restrict__ lam,
                                              const R* __restrict__ Ux, const R* __restrict__ Uy,
                                              const R* __restrict__ gsh, const R* __restrict__ gst,
                                              R* __restrict__ out, const Layout& L, const AdjCoef<R>& a, int i,
                                              int j, R G[16]) {
  const Coef<R>& c = a.c;
  const long long P = L.plane;
  const long long at = L.node(i, j);
  const R ux = Ux[at], uy = Uy[at];
  R g[16], lt[16];
  load16(ft, P, at, g);
  R rho = R(0);
#pragma unroll
  for (int q = 0; q < 16; ++q) rho += g[q];
  // (ghost rows behind walls are never read by an advanced node and may be empty)
  const R ir = (rho > R(0)) ? adj_inv(rho) : R(0);
#pragma unroll
  for (int q = 0; q < 16; ++q) lt[q] = R(0);
  // (c) the modification at the neighbours, through u(p): with the
  // collision's own u adjoint at an advanced node, else on its own
  R uxb = R(0), uyb = R(0);
  if (c.modified) {
    uxb = c.inv2dx * (gbar_at(gsh, L, i - 1, j) - gbar_at(gsh, L, i + 1, j)) +
          c.inv2dy * (gbar_at(gst, L, i, j - 1) - gbar_at(gst, L, i, j + 1));
    uyb = c.inv2dx * (gbar_at(gst, L, i - 1, j) - gbar_at(gst, L, i + 1, j)) -
          c.inv2dy * (gbar_at(gsh, L, i, j - 1) - gbar_at(gsh, L, i, j + 1));
  }
  if (advanced<R>(L, i, j)) {
    R lp[16];
    load16(lam, P, at, lp);
    const long long aE = at + 1, aW = at - 1, aN = at + L.pitch, aS = at - L.pitch;
    const R shear = (Ux[aE] - Ux[aW]) * c.inv2dx - (Uy[aN] - Uy[aS]) * c.inv2dy;
    const R strain = (Uy[aE] - Uy[aW]) * c.inv2dx + (Ux[aN] - Ux[aS]) * c.inv2dy;
    collision_T_node<R, RATES>(a, g, lp, ux, uy, shear, strain, uxb, uyb, lt, G);
  } else if (c.modified) {
    velocity_T(uxb, uyb, ux, uy, ir, lt);
  }
  // (a) neighbours' Lax-Wendroff weights on p
  const int nbi[4] = {i - 1, i + 1, i, i};  // r = p - e_x (uses kE), p + e_x (kW), p - e_y (kN), p + e_y (kS)
  const int nbj[4] = {j, j, j - 1, j + 1};
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    if (!advanced<R>(L, nbi[n], nbj[n])) continue;
    const long long ar = L.node(nbi[n], nbj[n]);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (n < 2 && vx_of(q) == 0) continue;
      if (n >= 2 && vy_of(q) == 0) continue;
      lt[q] += c.lw[q][n] * lam[q * P + ar];
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) out[q * P + at] = lt[q];
}

#ifndef MRTLB_ADJ_MINB
#define MRTLB_ADJ_MINB 5
#endif

// Persistent over row tiles of 128 nodes (tile t: row -1 + t / tiles_x);
// each thread sums the rate gradients of all its nodes before the warp
// reduction.
template <typename R, bool RATES>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? MRTLB_ADJ_MINB : 2)
    adj_core_kernel(const R* __restrict__ ft, const R* __restrict__ lam, const R* __restrict__ Ux,
                    const R* __restrict__ Uy, const R* __restrict__ gsh, const R* __restrict__ gst,
                    R* __restrict__ out, Layout L, AdjCoef<R> a, double* gacc, int tiles_x, int ntiles) {
  R G[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) G[k] = R(0);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i = -1 + (t % tiles_x) * 128 + (int)threadIdx.x;
    const int j = -1 + t / tiles_x;
    if (i <= L.nx && !((i < 0 || i >= L.nx) && (j < 0 || j >= L.ny)))
      adj_core_node<R, RATES>(ft, lam, Ux, Uy, gsh, gst, out, L, a, i, j, G);
  }
  if constexpr (RATES) flush_rate_gradients(G, gacc);
}

// Adjoint march shapes: 128-column strips (FP32; 64 for FP64, same box
// bytes), 3 B(f) slots and 4 lambda slots: about 71 KB of shared memory,
// three CTAs per SM (measured on GB300 against 4+6, 4+4 slots and 64-,
// 96-, 256-column strips).
#ifndef MRTLB_ADJ_BX
#define MRTLB_ADJ_BX 128
#endif
#ifndef MRTLB_ADJ_NF
#define MRTLB_ADJ_NF 3
#endif
#ifndef MRTLB_ADJ_NL
#define MRTLB_ADJ_NL 4
#endif
template <typename R> struct AdjTile;
template <> struct AdjTile<float> { static constexpr int BX = MRTLB_ADJ_BX, NF = MRTLB_ADJ_NF, NL = MRTLB_ADJ_NL; };
template <> struct AdjTile<double> { static constexpr int BX = 64, NF = 3, NL = 4; };

// B^T, ghosts: every edge node collects the adjoints of the ghost cells that
// copy it (plane q = blockIdx.y); inflow ghosts do not depend on f.  The ghost cells keep their values:
// lambda is only ever read at advanced nodes, and every step overwrites
// the whole padded grid [-1, nx] x [-1, ny].
template <typename R>
__global__ void adj_ghosts_kernel(R* lam, Layout L) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int perim = 2 * L.nx + 2 * L.ny;
  if (t >= perim) return;
  int i, j;
  if (t < L.nx) { i = t; j = 0; }
  else if (t < 2 * L.nx) { i = t - L.nx; j = L.ny - 1; }
  else if (t < 2 * L.nx + L.ny) { i = 0; j = t - 2 * L.nx; }
  else { i = L.nx - 1; j = t - 2 * L.nx - L.ny; }
  // a node on two edges appears twice; let the first appearance do the work
  if (t >= 2 * L.nx && (j == 0 || j == L.ny - 1)) return;
  if (t >= L.nx && t < 2 * L.nx && L.ny == 1) return;
  if (t >= 2 * L.nx + L.ny && L.nx == 1) return;
  const GhostTargets g = ghost_targets(L, i, j);
  if (!g.any()) return;
  const int q = blockIdx.y;
  R* p = lam + L.node(i, j);
  R v = p[(long long)q * L.plane];
  for (int s = 0; s < 4; ++s) {
    if (!g.w[s]) continue;
    // a reflecting side held plane q of the node in the mirrored plane
    const int qg = g.mir[s] ? (s < 2 ? mirror_x(q) : mirror_y(q)) : q;
    v += p[(long long)qg * L.plane + g.off[s]];
  }
  p[(long long)q * L.plane] = v;
}

// B^T, diffuse reflection on side s: the ghost beyond edge node e holds
// g = P f(e) with P linear (diffuse_ghost), so lambda(e) += P^T lambda~(g):
//   lambda(e)_q += [q not entering] lambda~_q + (b_q - [q not entering] a_q) / D * sum_{p entering} e_p lambda~_p.
template <typename R>
__global__ void adj_diffuse_kernel(R* lam, Layout L, Coef<R> c, Walls w, int side) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = (side < 2) ? L.ny : L.nx;
  if (k >= n) return;
  const int i = (side == 0) ? 0 : (side == 1) ? L.nx - 1 : k;
  const int j = (side == 2) ? 0 : (side == 3) ? L.ny - 1 : k;
  const long long off = (side == 0) ? -1 : (side == 1) ? 1 : (side == 2) ? -(long long)L.pitch : L.pitch;
  R* le = lam + L.node(i, j);
  const R* lg = le + off;
  R e[16];
  wall_equilibrium(c, (R)w.ux[side], (R)w.uy[side], (R)w.T[side], e);
  R den = R(0), s_in = R(0);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    if (!entering<R>(side, q)) continue;
    R a, b;
    diffuse_weights(c, side, q, a, b);
    den += a * e[q];
    s_in += e[q] * lg[(long long)q * L.plane];
  }
  const R g = s_in / den;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    R a, b;
    diffuse_weights(c, side, q, a, b);
    const bool in = entering<R>(side, q);
    R add = (b - (in ? R(0) : a)) * g;
    if (!in) add += lg[(long long)q * L.plane];
    le[(long long)q * L.plane] += add;
  }
}

// B^T, walls on one side: the wall node w was NEE(f(a)) of its fluid
// neighbour a: lambda(a) += (dNEE/df(a))^T lambda~(w), lambda(w) = 0.
template <typename R>
__global__ void adj_walls_kernel(R* lam, const R* __restrict__ ft, Layout L, Coef<double> c, Walls w, int side) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = (side < 2) ? L.ny : L.nx;
  if (k >= n) return;
  int i, j, ia, ja;
  if (side == 0) { i = 0; j = k; ia = 1; ja = k; }
  else if (side == 1) { i = L.nx - 1; j = k; ia = L.nx - 2; ja = k; }
  else if (side == 2) { i = k; j = 0; ia = k; ja = 1; }
  else { i = k; j = L.ny - 1; ia = k; ja = L.ny - 2; }
  const long long P = L.plane, aw = L.node(i, j), aa = L.node(ia, ja);
  double v[16], g[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    v[q] = (double)lam[q * P + aw];
    g[q] = (double)ft[q * P + aa];
  }
  double rho, jx, jy, e;
  conserved(g, rho, jx, jy, e);
  const double ir = 1.0 / rho;
  const double ux = jx * ir, uy = jy * ir;
  const double T = temperature(rho, jx, jy, e, ir);
  // NEE(g) = g + M^-1 (eq(rho, rho u_w, e_w, u_w, T_w) - eq(rho, j, e, u, T))
  double db[16];
  inverse_T(c, v, db, true);
  const double uwx = w.ux[side], uwy = w.uy[side], Tw = w.T[side];
  const double kw = Tw + 0.5 * (uwx * uwx + uwy * uwy);
  EqIn<double> xw{rho, ir, rho * uwx, rho * uwy, rho * kw, uwx, uwy, Tw};
  EqIn<double> gw{0, 0, 0, 0, 0, 0, 0, 0};
  equilibrium_T(c, xw, db, gw);
  double rbw = gw.rho - gw.ir * ir * ir + gw.jx * uwx + gw.jy * uwy + gw.e * kw;
  double ndb[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) ndb[q] = -db[q];
  EqIn<double> xa{rho, ir, jx, jy, e, ux, uy, T};
  EqIn<double> ga{0, 0, 0, 0, 0, 0, 0, 0};
  equilibrium_T(c, xa, ndb, ga);
  double rb, jxb, jyb, eb;
  chain_primitive(xa, ga, rb, jxb, jyb, eb);
  rb += rbw;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const double vx = vx_of(q), vy = vy_of(q);
    const double add = v[q] + rb + jxb * vx + jyb * vy + eb * 0.5 * (vx * vx + vy * vy);
    lam[q * P + aa] = (R)((double)lam[q * P + aa] + add);
    lam[q * P + aw] = R(0);
  }
}

// Seed: lambda = (d(rho, u_x, u_y, T)/df)^T (dL/d macros) on every node,
// in the precision of the state.
template <typename R>
__global__ void adj_seed_macros_kernel(const R* __restrict__ ft, const double* __restrict__ seed, R* lam,
                                       Layout L) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= L.nx) return;
  const long long n = (long long)L.nx * L.ny, t = (long long)j * L.nx + i, at = L.node(i, j);
  R g[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) g[q] = ft[q * L.plane + at];
  R rho, jx, jy, e;
  conserved(g, rho, jx, jy, e);
  const R ir = adj_inv(rho);
  EqIn<R> x{rho, ir, jx, jy, e, jx * ir, jy * ir, temperature(rho, jx, jy, e, ir)};
  EqIn<R> gi{(R)seed[t], R(0), R(0), R(0), R(0), (R)seed[n + t], (R)seed[2 * n + t], (R)seed[3 * n + t]};
  R rb, jxb, jyb, eb;
  chain_primitive(x, gi, rb, jxb, jyb, eb);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const R vx = vx_of(q), vy = vy_of(q);
    lam[q * L.plane + at] = rb + jxb * vx + jyb * vy + eb * R(0.5) * (vx * vx + vy * vy);
  }
}

// Dense FP64 [16][ny][nx] <-> padded lambda: mode 0 sets lambda from the
// dense array, 1 writes lambda to it, 2 adds the dense array to lambda.
template <typename R>
__global__ void adj_dense_kernel(R* lam, double* dense, Layout L, int mode) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, q = blockIdx.z;
  if (i >= L.nx) return;
  const long long d = ((long long)q * L.ny + j) * L.nx + i, p = q * L.plane + L.node(i, j);
  if (mode == 1) dense[d] = (double)lam[p];
  else if (mode == 0) lam[p] = (R)dense[d];
  else lam[p] = (R)((double)lam[p] + dense[d]);
}

// dL/d(rho, u_x, u_y, T) of an equilibrium initial state f = M^-1 f^eq from
// dL/df (dense FP64), all in FP64.
__global__ void eq_adjoint_kernel(const double* __restrict__ lamd, const double* __restrict__ rho_in,
                                  const double* __restrict__ ux_in, const double* __restrict__ uy_in,
                                  const double* __restrict__ T_in, double* orho, double* oux, double* ouy,
                                  double* oT, long long n, Coef<double> c) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  double v[16], eqb[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = lamd[q * n + t];
  inverse_T(c, v, eqb, true);
  const double rho = rho_in[t], ux = ux_in[t], uy = uy_in[t], T = T_in[t];
  const double ir = 1.0 / rho, k = T + 0.5 * (ux * ux + uy * uy);
  EqIn<double> x{rho, ir, rho * ux, rho * uy, rho * k, ux, uy, T};
  EqIn<double> g{0, 0, 0, 0, 0, 0, 0, 0};
  equilibrium_T(c, x, eqb, g);
  // inputs of the equilibrium as functions of (rho, u, T)
  orho[t] = g.rho - g.ir * ir * ir + g.jx * ux + g.jy * uy + g.e * k;
  oux[t] = g.ux + g.jx * rho + g.e * rho * ux;
  ouy[t] = g.uy + g.jy * rho + g.e * rho * uy;
  oT[t] = g.T + g.e * rho;
}

}  // namespace
}  // namespace mrtlb

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct mrtlb_adjoint_state {
  long K = 0, S = 0, nseg = 0;
  std::vector<void*> ckpt;   // f^{sS} of every segment s (only when nseg > 1)
  void* seg = nullptr;       // S slots: the states B(f^t) of one segment
  long held = -1;            // the segment whose states the slots hold
  std::vector<TiledPlan> plan;  // per slot: tensor map reading that slot
  bool tiled = false;
  void* lam[2] = {nullptr, nullptr};
  void* gsh = nullptr;       // one padded plane each
  void* gst = nullptr;
  void* ux = nullptr;
  void* uy = nullptr;
  double* gacc = nullptr;
  int core_blocks = 1;       // resident blocks of the core kernel on the device
  size_t bytes = 0;          // device memory held in states
  int kernel = 0;            // the kernel choice the plans were made for
  // the fused adjoint march: read maps of every slot and of both lambdas
  bool march = false;
  std::vector<CUtensorMap> fmap;
  CUtensorMap lmap[2];
  int m_nstrips = 0, m_nseg = 0, m_seglen = 0;
  // the context's generation when the forward pass ended, and the pass's id
  unsigned long long gen = 0;
  long long pass = 0;
};

namespace {

// Blocks of the core kernel that fit on the device at once (its persistent grid).
template <typename R>
int core_resident_blocks() {
#if defined(MRTLB_ADJ_PERSIST) && MRTLB_ADJ_PERSIST == 0
  return 1 << 30;
#else
  int dev = 0, nsm = 1, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, adj_core_kernel<R, true>, 128, 0);
  return std::max(1, nsm) * std::max(1, per);
#endif
}

int afail(mrtlb_ctx* c, int code, const char* msg) {
  c->last_error = msg;
  return code;
}

#define ACK(call, what)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      c->last_error = std::string(what) + ": " + cudaGetErrorString(e_);              \
      return MRTLB_ERR_CUDA;                                                         \
    }                                                                                \
  } while (0)

void release(mrtlb_adjoint_state* a) {
  if (!a) return;
  for (void* p : a->ckpt) cudaFree(p);
  a->ckpt.clear();
  for (void* p : {a->seg, a->lam[0], a->lam[1], a->gsh, a->gst, a->ux, a->uy, (void*)a->gacc})
    if (p) cudaFree(p);
  delete a;
}

template <typename R>
AdjCoef<R> adj_coef(const mrtlb_ctx* c, const Coef<R>& k) {
  AdjCoef<R> a;
  a.c = k;
  for (int q = 0; q < 16; ++q) a.selfw[q] = R(1) - k.lwsum[q];
  const double s5 = c->s[4], s6 = c->s[5], s7 = c->s[6], s8 = c->s[7];
  a.g[0] = (R)(1.0 / s5);
  a.g[1] = (R)(1.0 / s6);
  a.g[2] = (R)(s7 / (s5 * s5));
  a.g[3] = (R)(s7 / (s6 * s6));
  a.g[4] = (R)(s8 / (s5 * s5));
  a.g[5] = (R)(s8 / (s6 * s6));
  return a;
}

template <typename R>
void launch_adj_march(const mrtlb_adjoint_state* a, const Layout& L, const CUtensorMap& fm, const CUtensorMap& lm,
                      R* out, const AdjCoef<R>& ac, int* err, bool rates, cudaStream_t st) {
  constexpr int BX = AdjTile<R>::BX, NF = AdjTile<R>::NF, NL = AdjTile<R>::NL;
  using SM = AdjSmem<R, BX, NF, NL>;
  // (plan_adj_march allowed the kernels' dynamic shared memory in this context)
  dim3 grid(a->m_nstrips, a->m_nseg);
  const bool v1 = ac.c.version == 1;  // (version 1 has its own kernels, without the others' transposes)
  if (rates && v1)
    adj_march_kernel<R, BX, NF, NL, true, 1><<<grid, BX, SM::bytes, st>>>(fm, lm, out, L, ac, a->gacc, err, a->m_seglen);
  else if (rates)
    adj_march_kernel<R, BX, NF, NL, true, 0><<<grid, BX, SM::bytes, st>>>(fm, lm, out, L, ac, a->gacc, err, a->m_seglen);
  else if (v1)
    adj_march_kernel<R, BX, NF, NL, false, 1><<<grid, BX, SM::bytes, st>>>(fm, lm, out, L, ac, a->gacc, err, a->m_seglen);
  else
    adj_march_kernel<R, BX, NF, NL, false, 0><<<grid, BX, SM::bytes, st>>>(fm, lm, out, L, ac, a->gacc, err, a->m_seglen);
}

// one adjoint step: lambda[li] (dL/df^{n+1}) -> lambda[li ^ 1] (dL/df^n),
// ft = B(f^n) in slot n; rates: also sum the rate gradients
template <typename R>
void adjoint_step(mrtlb_ctx* c, mrtlb_adjoint_state* a, long n, int li, const Coef<R>& k, bool rates,
                  cudaStream_t st) {
  const Layout& L = c->L;
  const AdjCoef<R> ac = adj_coef<R>(c, k);
  const R* ft = (const R*)((char*)a->seg + (size_t)n * c->state_bytes);
  const R* lam_in = (const R*)a->lam[li];
  R* lam_out = (R*)a->lam[li ^ 1];
  if (a->march) {
    launch_adj_march<R>(a, L, a->fmap[n], a->lmap[li], lam_out, ac, c->err, rates, st);
  } else {
    dim3 g2((L.nx + 2 + 127) / 128, L.ny + 2);
    adj_prep_kernel<R><<<g2, 128, 0, st>>>(ft, lam_in, (R*)a->ux, (R*)a->uy, (R*)a->gsh, (R*)a->gst, L, ac);
    const int ntiles = (int)(g2.x * g2.y);
    const int grid = std::min(ntiles, a->core_blocks);
    if (rates)
      adj_core_kernel<R, true><<<grid, 128, 0, st>>>(ft, lam_in, (const R*)a->ux, (const R*)a->uy, (const R*)a->gsh,
                                                     (const R*)a->gst, lam_out, L, ac, a->gacc, (int)g2.x, ntiles);
    else
      adj_core_kernel<R, false><<<grid, 128, 0, st>>>(ft, lam_in, (const R*)a->ux, (const R*)a->uy, (const R*)a->gsh,
                                                      (const R*)a->gst, lam_out, L, ac, a->gacc, (int)g2.x, ntiles);
  }
  const int perim = 2 * L.nx + 2 * L.ny;
  adj_ghosts_kernel<R><<<dim3((perim + 127) / 128, 16), 128, 0, st>>>(lam_out, L);
  for (int s = 0; s < 4; ++s) {
    const int nn = (s < 2) ? L.ny : L.nx;
    if (L.bc[s] == BC_DIFFUSE) adj_diffuse_kernel<R><<<(nn + 127) / 128, 128, 0, st>>>(lam_out, L, k, c->walls, s);
    if (L.bc[s] == BC_WALL)
      adj_walls_kernel<R><<<(nn + 127) / 128, 128, 0, st>>>(lam_out, ft, L, c->c64, c->walls, s);
  }
}

// Maps and row segments of the adjoint march; false if it cannot run.
template <typename R>
bool plan_adj_march(mrtlb_ctx* c, mrtlb_adjoint_state* a) {
  constexpr int BX = AdjTile<R>::BX, NF = AdjTile<R>::NF, NL = AdjTile<R>::NL;
  using SM = AdjSmem<R, BX, NF, NL>;
  const Layout& L = c->L;
  const int es = (int)sizeof(R);
  a->fmap.resize((size_t)(a->S + 1) & ~(size_t)1);
  for (long n = 0; n < a->S; n += 2) {
    void* s0 = (char*)a->seg + (size_t)n * c->state_bytes;
    void* s1 = (char*)a->seg + (size_t)std::min(n + 1, a->S - 1) * c->state_bytes;
    if (encode_row_maps(L, es, s0, s1, BX, &a->fmap[n]) != 0) return false;
  }
  if (encode_row_maps(L, es, a->lam[0], a->lam[1], BX, a->lmap) != 0) return false;
  const int b = (int)SM::bytes;
  const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (cudaFuncSetAttribute(adj_march_kernel<R, BX, NF, NL, true, 0>, A, b) != cudaSuccess ||
      cudaFuncSetAttribute(adj_march_kernel<R, BX, NF, NL, false, 0>, A, b) != cudaSuccess ||
      cudaFuncSetAttribute(adj_march_kernel<R, BX, NF, NL, true, 1>, A, b) != cudaSuccess ||
      cudaFuncSetAttribute(adj_march_kernel<R, BX, NF, NL, false, 1>, A, b) != cudaSuccess)
    return false;
  int dev = 0, nsm = 1, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, adj_march_kernel<R, BX, NF, NL, true, 0>, BX, SM::bytes);
  if (per < 1) return false;
  const int rows = L.ny + 2;  // output rows -1 .. ny
  a->m_nstrips = (L.nx + 2 + SM::SX - 1) / SM::SX;
  int nseg = std::max(1, nsm * per / a->m_nstrips);
  a->m_seglen = std::max(8, (rows + nseg - 1) / nseg);
  a->m_nseg = (rows + a->m_seglen - 1) / a->m_seglen;
  return true;
}

template <typename R>
R* slot(const mrtlb_ctx* c, const mrtlb_adjoint_state* a, long n) {
  return (R*)((char*)a->seg + (size_t)n * c->state_bytes);
}

template <typename R>
const Coef<R>& coef_of(const mrtlb_ctx* c) {
  return *reinterpret_cast<const Coef<R>*>(sizeof(R) == 4 ? (const void*)&c->c32 : (const void*)&c->c64);
}

// Run the states of segment sg (t0 = sg S, len steps) through the slots:
// slot n becomes B(f^{t0+n}) (walls refilled, ghosts written through by the
// step that produced it).  Slot 0 must hold f^{t0}.  The last step writes
// into `last` unless it is null (then the segment's final state is not kept).
template <typename R>
void run_segment(mrtlb_ctx* c, mrtlb_adjoint_state* a, long len, const Coef<R>& k, cudaStream_t st, R* last) {
  TraceRange trace_("adjoint_segment");
  for (long n = 0; n < len; ++n) {
    R* fin = slot<R>(c, a, n);
    launch_walls<R>(fin, c->L, coef_of<R>(c), c->walls, st);
    R* fout = (n + 1 < len) ? slot<R>(c, a, n + 1) : last;
    if (!fout) break;
    if (a->tiled) launch_step_tiled<R>(a->plan[n], 0, c->L, k, c->err, st, fout);
    else launch_step_plain<R>(fin, fout, c->L, k, c->err, st);
  }
}

template <typename R>
int backward_impl(mrtlb_ctx* c, const double* dL_dmacros, const double* dL_dfK, double* dL_ds,
                  double* dL_df0) {
  mrtlb_adjoint_state* a = c->adj;
  const Layout& L = c->L;
  cudaStream_t st = c->stream;
  const Coef<R>& k = coef_of<R>(c);
  const size_t sb = c->state_bytes;
  R* lam0 = (R*)a->lam[0];
  R* lam1 = (R*)a->lam[1];
  ACK(cudaMemsetAsync(lam0, 0, sb, st), "clear");
  ACK(cudaMemsetAsync(lam1, 0, sb, st), "clear");
  ACK(cudaMemsetAsync(a->gacc, 0, 16 * sizeof(double), st), "clear");
  // seed on B(f^K)
  R* fK = (R*)c->f[c->cur];
  launch_bc<R>(fK, L, k, c->walls, st);
  dim3 gs((L.nx + 127) / 128, L.ny);
  if (dL_dmacros) adj_seed_macros_kernel<R><<<gs, 128, 0, st>>>(fK, dL_dmacros, lam0, L);
  if (dL_dfK) {  // a direct seed on the state (as mrtlb_get_f returns it); added to the macro seed
    dim3 gd((L.nx + 127) / 128, L.ny, 16);
    adj_dense_kernel<R><<<gd, 128, 0, st>>>(lam0, (double*)dL_dfK, L, dL_dmacros ? 2 : 0);
  }
  // walls of B^T for the seed
  for (int s = 0; s < 4; ++s)
    if (L.bc[s] == BC_WALL) {
      const int n = (s < 2) ? L.ny : L.nx;
      adj_walls_kernel<R><<<(n + 127) / 128, 128, 0, st>>>(lam0, fK, L, c->c64, c->walls, s);
    }
  ACK(cudaGetLastError(), "adjoint seed");
  int li = 0;  // lambda[li] holds dL/df of the latest state reached
  const long K = a->K, S = a->S;
  for (long sgi = a->nseg - 1; sgi >= 0; --sgi) {
    const long t0 = sgi * S;
    const long len = std::min(S, K - t0);
    if (a->held != sgi) {  // recompute the segment's states from its checkpoint
      ACK(cudaMemcpyAsync(a->seg, a->ckpt[sgi], sb, cudaMemcpyDeviceToDevice, st), "restore checkpoint");
      run_segment<R>(c, a, len, k, st, nullptr);
      a->held = sgi;
    }
    for (long n = len - 1; n >= 0; --n) {
      adjoint_step<R>(c, a, n, li, k, dL_ds != nullptr, st);
      li ^= 1;
    }
  }
  ACK(cudaGetLastError(), "adjoint steps");
  if (dL_df0) {
    dim3 gd((L.nx + 127) / 128, L.ny, 16);
    adj_dense_kernel<R><<<gd, 128, 0, st>>>((R*)a->lam[li], dL_df0, L, 1);
  }
  if (dL_ds) ACK(cudaMemcpyAsync(dL_ds, a->gacc, 16 * sizeof(double), cudaMemcpyDeviceToHost, st), "copy grads");
  int h = 0;
  ACK(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, st), "read error word");
  ACK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  if (h & ERRBIT_TIMEOUT) return afail(c, MRTLB_ERR_TIMEOUT, "a bounded device-side wait gave up");
  if (h & ERRBIT_NONPHYSICAL)  // (the gradients of such a run mean nothing)
    return afail(c, MRTLB_ERR_NONPHYSICAL, "a state of the forward pass was non-physical (rho <= 0, T <= 0 or not finite)");
  if (dL_ds)  // the kernels sum the rate gradients without the factor dt
    for (int k = 0; k < 16; ++k) dL_ds[k] *= c->p.dt;
  return MRTLB_OK;
}

// Buffers, tensor maps and launch plans of an adjoint state with S slots
// and nck checkpoints.
template <typename R>
int allocate(mrtlb_ctx* c, mrtlb_adjoint_state* a, long S, long nck) {
  const size_t sb = c->state_bytes;
  cudaStream_t st = c->stream;
  const bool fp64 = sizeof(R) == 8;
  a->S = S;
  a->kernel = c->kernel;
  for (long i = 0; i < nck; ++i) {
    void* p = nullptr;
    ACK(cudaMalloc(&p, sb), "cudaMalloc(checkpoint)");
    a->ckpt.push_back(p);
  }
  ACK(cudaMalloc(&a->seg, sb * (size_t)S), "cudaMalloc(segment)");
  a->bytes = sb * (size_t)(S + nck + 2);
  // the fixed inflow ghosts of every slot (a step writes the other ghosts)
  for (long n = 0; n < S; ++n) launch_inflow<R>(slot<R>(c, a, n), c->L, coef_of<R>(c), c->walls, st);
  for (int b = 0; b < 2; ++b) ACK(cudaMalloc(&a->lam[b], sb), "cudaMalloc(lambda)");
  const size_t pb = (size_t)c->L.plane * c->esize;
  ACK(cudaMalloc(&a->gsh, pb), "cudaMalloc(gbar)");
  ACK(cudaMalloc(&a->gst, pb), "cudaMalloc(gbar)");
  ACK(cudaMalloc(&a->ux, pb), "cudaMalloc(u)");
  ACK(cudaMalloc(&a->uy, pb), "cudaMalloc(u)");
  for (void* q : {a->gsh, a->gst, a->ux, a->uy}) ACK(cudaMemsetAsync(q, 0, pb, st), "clear");
  ACK(cudaMalloc((void**)&a->gacc, 16 * sizeof(double)), "cudaMalloc(grad)");
  a->core_blocks = core_resident_blocks<R>();
  // one read map per slot for the tiled step (the write side is a plain pointer)
  TiledPlan p0;
  plan_tiled(c->L, (int)c->esize, a->seg, a->seg, &p0);
  a->tiled = use_tiled(c->kernel, p0, fp64);
  if (a->tiled) {
    a->plan.resize(S);
    for (long n = 0; n < S; ++n) {
      void* sp = slot<R>(c, a, n);
      if (plan_tiled(c->L, (int)c->esize, sp, sp, &a->plan[n]) != 0) {
        a->tiled = false;
        break;
      }
    }
  }
  a->march = a->tiled && plan_adj_march<R>(c, a);
  return MRTLB_OK;
}

template <typename R>
int forward_impl(mrtlb_ctx* c, long K) {
  const size_t sb = c->state_bytes;
  cudaStream_t st = c->stream;
  mrtlb_adjoint_state* old = c->adj;
  if (old) old->pass = 0;  // until this pass completes, no backward pass is possible
  // segment length: every state when K + 2 states fit in half the free
  // memory (the buffers of a previous forward pass count as free)
  long S = c->adj_interval;
  if (S <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    fr += old ? old->bytes : 0;
    S = ((size_t)(K + 2) * sb <= fr / 2) ? K : (long)std::ceil(std::sqrt((double)K));
  }
  S = std::max(1L, std::min(S, std::max(K, 1L)));
  const long nseg = std::max(1L, (K + S - 1) / S);
  const long nck = (nseg > 1) ? nseg : 0;
  // a previous pass of the same shape keeps its buffers and plans
  mrtlb_adjoint_state* a = old;
  if (!(old && old->S == S && (long)old->ckpt.size() >= nck && old->kernel == c->kernel)) {
    if (old) cudaStreamSynchronize(st);  // (its buffers may still be in use by queued work)
    release(old);
    c->adj = a = new mrtlb_adjoint_state();
    const int rc = allocate<R>(c, a, S, nck);
    if (rc) {  // (no half-built state stays behind for a later pass to reuse)
      cudaGetLastError();  // (reported here; the next launch check must not see it again)
      cudaStreamSynchronize(st);
      release(a);
      c->adj = nullptr;
      return rc;
    }
  }
  a->K = K;
  a->nseg = nseg;
  a->held = -1;
  // all segments but the last: checkpoint, then the context's own time loop
  for (long sg = 0; sg + 1 < a->nseg; ++sg) {
    ACK(cudaMemcpyAsync(a->ckpt[sg], c->f[c->cur], sb, cudaMemcpyDeviceToDevice, st), "store checkpoint");
    const int rc = mrtlb_step(c, S);
    if (rc) return rc;
  }
  // the last segment runs through the slots and stays there for the backward pass
  const long t0 = (a->nseg - 1) * S, len = K - t0;
  if (a->nseg > 1)
    ACK(cudaMemcpyAsync(a->ckpt[a->nseg - 1], c->f[c->cur], sb, cudaMemcpyDeviceToDevice, st), "store checkpoint");
  ACK(cudaMemcpyAsync(a->seg, c->f[c->cur], sb, cudaMemcpyDeviceToDevice, st), "copy state");
  if (len > 0) {
    run_segment<R>(c, a, len, coef_of<R>(c), st, (R*)c->f[c->cur ^ 1]);
    c->cur ^= 1;
    c->steps += len;
    ++c->gen;
  }
  a->held = a->nseg - 1;
  ACK(cudaGetLastError(), "adjoint forward");
  a->gen = c->gen;
  a->pass = ++c->adj_passes;
  return MRTLB_OK;
}

}  // namespace

extern "C" int mrtlb_adjoint_set_interval(mrtlb_ctx* c, long S) {
  if (!c) return MRTLB_ERR_ARG;
  if (S < 0) return afail(c, MRTLB_ERR_ARG, "S < 0");
  c->adj_interval = S;
  return MRTLB_OK;
}

extern "C" int mrtlb_adjoint_forward(mrtlb_ctx* c, long K) {
  TraceRange trace_("mrtlb_adjoint_forward");
  if (!c) return MRTLB_ERR_ARG;
  if (!c->f[0] || !c->f[1]) return afail(c, MRTLB_ERR_STATE, "bind state buffers first");
  if (K < 0) return afail(c, MRTLB_ERR_ARG, "K < 0");
  return (c->prec == MRTLB_FP64) ? forward_impl<double>(c, K) : forward_impl<float>(c, K);
}

extern "C" int mrtlb_adjoint_backward(mrtlb_ctx* c, const double* dL_dmacros, const double* dL_dfK,
                                      double dL_ds[16], double* dL_df0) {
  TraceRange trace_("mrtlb_adjoint_backward");
  if (!c) return MRTLB_ERR_ARG;
  if (!c->adj || c->adj->pass == 0) return afail(c, MRTLB_ERR_STATE, "call mrtlb_adjoint_forward first");
  if (c->adj->gen != c->gen)
    return afail(c, MRTLB_ERR_STATE,
                 "the state or the rates changed since mrtlb_adjoint_forward (a step, set_f, init_equilibrium, "
                 "bind, load, set_rates or a batched step): run the forward pass again");
  if (!dL_dmacros && !dL_dfK) return afail(c, MRTLB_ERR_ARG, "a seed (dL/dmacros or dL/df^K) is required");
  const int rc = (c->prec == MRTLB_FP64) ? backward_impl<double>(c, dL_dmacros, dL_dfK, dL_ds, dL_df0)
                                         : backward_impl<float>(c, dL_dmacros, dL_dfK, dL_ds, dL_df0);
  return rc;
}

extern "C" long long mrtlb_adjoint_pass(const mrtlb_ctx* c) {
  if (!c || !c->adj || c->adj->gen != c->gen) return 0;
  return c->adj->pass;
}

extern "C" int mrtlb_adjoint_release(mrtlb_ctx* c) {
  if (!c) return MRTLB_ERR_ARG;
  if (c->adj) cudaStreamSynchronize(c->stream);
  release(c->adj);
  c->adj = nullptr;
  return MRTLB_OK;
}

extern "C" int mrtlb_equilibrium_adjoint(mrtlb_ctx* c, const double* dL_df, const double* rho,
                                         const double* ux, const double* uy, const double* T,
                                         double* dL_drho, double* dL_dux, double* dL_duy, double* dL_dT) {
  if (!c || !dL_df || !rho || !ux || !uy || !T || !dL_drho || !dL_dux || !dL_duy || !dL_dT)
    return MRTLB_ERR_ARG;
  const long long n = (long long)c->L.nx * c->L.ny;
  eq_adjoint_kernel<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(dL_df, rho, ux, uy, T, dL_drho, dL_dux,
                                                                         dL_duy, dL_dT, n, c->c64);
  ACK(cudaGetLastError(), "equilibrium adjoint");
  ACK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return MRTLB_OK;
}

void mrtlb_adjoint_free_internal(mrtlb_ctx* c) {
  if (c && c->adj) {
    release(c->adj);
    c->adj = nullptr;
  }
}
