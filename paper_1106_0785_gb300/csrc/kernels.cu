// kernels.cu - plain step kernel, boundary fills, layout conversion,
// equilibrium initialisation, macroscopic fields and conservation sums.
#include "kernels.cuh"

namespace mrtlb {

// ---------------------------------------------------------------------------
// Plain step: one thread per advanced node, neighbours read straight from
// global memory (L1/L2 serve the reuse).  Used for the FP64 path and as the
// reference launch shape for the FP32 path.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void node_velocity(const R* __restrict__ f, long long plane, long long at,
                                              R& ux, R& uy) {
  R g[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) g[q] = f[q * plane + at];
  R rho, jx, jy, e;
  conserved(g, rho, jx, jy, e);
  const R r = recip(rho);
  ux = jx * r;
  uy = jy * r;
}

// Thread t takes advanced node t of the row-major enumeration of
// [i0, i1) x [j0, j1), so that every lane of a warp has a node whatever the
// grid's shape (a 4-column grid would leave 28 of 32 lanes idle under a
// 2D block, and FP64 arithmetic costs a warp the same with idle lanes).
template <typename R>
__global__ void __launch_bounds__(128) step_plain_kernel(const R* __restrict__ fin, R* __restrict__ fout,
                                                         Layout L, Coef<R> c, int* err) {
  const int ni = L.i1 - L.i0;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ni * (L.j1 - L.j0)) return;
  const int i = L.i0 + (int)(t % ni);
  const int j = L.j0 + (int)(t / ni);
  const long long P = L.plane;
  const long long at = L.node(i, j);
  const long long E = at + 1, W = at - 1, N = at + L.pitch, S = at - L.pitch;

  R f[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) f[q] = fin[q * P + at];
  R rho, jx, jy, e;
  conserved(f, rho, jx, jy, e);
  const R ir = recip(rho);
  const R ux = jx * ir, uy = jy * ir;
  const R T = temperature(rho, jx, jy, e, ir);

  R uxE, uyE, uxW, uyW, uxN, uyN, uxS, uyS;
  node_velocity(fin, P, E, uxE, uyE);
  node_velocity(fin, P, W, uxW, uyW);
  node_velocity(fin, P, N, uxN, uyN);
  node_velocity(fin, P, S, uxS, uyS);
  const R dux_dx = (uxE - uxW) * c.inv2dx, duy_dx = (uyE - uyW) * c.inv2dx;
  const R dux_dy = (uxN - uxS) * c.inv2dy, duy_dy = (uyN - uyS) * c.inv2dy;

  R C[16];
  collision(c, f, dux_dx, dux_dy, duy_dx, duy_dy, rho, ir, jx, jy, e, ux, uy, T, C);

  R vout[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const R fE = (vx_of(q) != 0) ? fin[q * P + E] : R(0), fW = (vx_of(q) != 0) ? fin[q * P + W] : R(0);
    const R fN = (vy_of(q) != 0) ? fin[q * P + N] : R(0), fS = (vy_of(q) != 0) ? fin[q * P + S] : R(0);
    const R fn = lw_update(c, q, f[q], C[q], fE, fW, fN, fS);
    fout[q * P + at] = fn;
    vout[q] = fn;
  }
  const GhostTargets g = ghost_targets(L, i, j);
  if (g.any()) write_ghosts(g, P, vout, fout + at);
  if (!(rho > R(0)) || !(T > R(0))) atomicOr(err, ERRBIT_NONPHYSICAL);
}

template <typename R>
void launch_step_plain(const R* fin, R* fout, const Layout& L, const Coef<R>& c, int* err,
                       cudaStream_t st) {
  const int ni = L.i1 - L.i0, nj = L.j1 - L.j0;
  if (ni <= 0 || nj <= 0) return;
  // a grid small enough to leave SMs idle takes blocks of fewer threads
  // (the smallest power of two, at least 8, that covers it with one block
  // per SM), so that its latency-bound nodes spread over every SM
  static const int nsm = [] {  // thread-safe static initialisation
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    return n;
  }();
  const long long n = (long long)ni * nj;
  int blk = 8;
  while (blk < 128 && (long long)blk * nsm < n) blk *= 2;
  step_plain_kernel<R><<<(unsigned)((n + blk - 1) / blk), blk, 0, st>>>(fin, fout, L, c, err);
}

// ---------------------------------------------------------------------------
// Boundaries.  Walls first (non-equilibrium extrapolation of Sec. IV A; the
// wall node takes f^eq(rho_a, u_w, T_w) + f_a - f^eq(rho_a, u_a, T_a) from
// its fluid neighbour a), then the ghost layer (periodic copy or
// zero-gradient outflow; behind a wall a copy keeps the ghost finite).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void bc_walls_kernel(R* f, Layout L, Coef<R> c, Walls w) {
  wall_node(f, L, c, w, blockIdx.x * blockDim.x + threadIdx.x);
}

// f^eq of an inflow side's fixed state, plane q.
template <typename R>
__device__ __forceinline__ R inflow_value(const Coef<R>& c, const Walls& w, int side, int q) {
  const R rho = (R)w.rho[side], ux = (R)w.ux[side], uy = (R)w.uy[side], T = (R)w.T[side];
  const R ir = R(1) / rho;
  R eq[16], fe[16];
  equilibrium(c, rho, ir, rho * ux, rho * uy, rho * (T + R(0.5) * (ux * ux + uy * uy)), ux, uy, T, eq);
  inverse_full(c, eq, fe);
  return fe[q];
}

// One ghost value beside side s of a non-periodic side from the edge node
// `edge` (plane-0 address): outflow and walls copy it, reflect takes the
// mirrored plane, inflow the side's fixed equilibrium.
template <typename R>
__device__ __forceinline__ R side_ghost(const Coef<R>& c, const Walls& w, const Layout& L, int s, int q,
                                        const R* edge) {
  if (L.bc[s] == BC_INFLOW) return inflow_value(c, w, s, q);
  if (L.bc[s] == BC_REFLECT) return edge[(long long)(s < 2 ? mirror_x(q) : mirror_y(q)) * L.plane];
  return edge[(long long)q * L.plane];
}

// The ghost layer of f (plane q = blockIdx.y), diffuse sides excepted (the
// wall pass fills those).  only_inflow: just the inflow sides (buffers whose
// other ghosts the steps write).
template <typename R>
__global__ void bc_ghost_kernel(R* f, Layout L, Coef<R> c, Walls w, int only_inflow) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  const long long P = L.plane;
  R* fq = f + q * P;
  if (t < L.ny) {  // x sides, row j = t
    const int j = t;
    const long long row = (long long)(j + 1) * L.pitch;
    const long long first = row + L.xoff, last = row + L.xoff + L.nx - 1;
    if (L.bc[0] == BC_PERIODIC) {
      if (!only_inflow) {
        fq[first - 1] = fq[last];
        fq[last + 1] = fq[first];
      }
    } else {
      if ((!only_inflow && L.bc[0] != BC_DIFFUSE) || L.bc[0] == BC_INFLOW)
        fq[first - 1] = side_ghost(c, w, L, 0, q, f + first);
      if ((!only_inflow && L.bc[1] != BC_DIFFUSE) || L.bc[1] == BC_INFLOW)
        fq[last + 1] = side_ghost(c, w, L, 1, q, f + last);
    }
  }
  if (t < L.nx) {  // y sides, column i = t
    const int i = t;
    const long long first = (long long)1 * L.pitch + L.xoff + i;
    const long long last = (long long)L.ny * L.pitch + L.xoff + i;
    if (L.bc[2] == BC_PERIODIC) {
      if (!only_inflow) {
        fq[first - L.pitch] = fq[last];
        fq[last + L.pitch] = fq[first];
      }
    } else {
      if ((!only_inflow && L.bc[2] != BC_DIFFUSE) || L.bc[2] == BC_INFLOW)
        fq[first - L.pitch] = side_ghost(c, w, L, 2, q, f + first);
      if ((!only_inflow && L.bc[3] != BC_DIFFUSE) || L.bc[3] == BC_INFLOW)
        fq[last + L.pitch] = side_ghost(c, w, L, 3, q, f + last);
    }
  }
}

template <typename R>
void launch_walls(R* f, const Layout& L, const Coef<R>& c, const Walls& w, cudaStream_t st) {
  const int nwall = wall_count(L);
  if (nwall > 0) bc_walls_kernel<R><<<(nwall + 127) / 128, 128, 0, st>>>(f, L, c, w);
}

template <typename R>
void launch_bc(R* f, const Layout& L, const Coef<R>& c, const Walls& w, cudaStream_t st) {
  launch_walls<R>(f, L, c, w, st);
  const int n = (L.nx > L.ny) ? L.nx : L.ny;
  dim3 grd((n + 255) / 256, 16);
  bc_ghost_kernel<R><<<grd, 256, 0, st>>>(f, L, c, w, 0);
}

template <typename R>
void launch_inflow(R* f, const Layout& L, const Coef<R>& c, const Walls& w, cudaStream_t st) {
  bool any = false;
  for (int s = 0; s < 4; ++s) any |= (L.bc[s] == BC_INFLOW);
  if (!any) return;
  const int n = (L.nx > L.ny) ? L.nx : L.ny;
  dim3 grd((n + 255) / 256, 16);
  bc_ghost_kernel<R><<<grd, 256, 0, st>>>(f, L, c, w, 1);
}

// ---------------------------------------------------------------------------
// Dense [16][ny][nx] <-> padded layout.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void pack_kernel(const R* __restrict__ dense, R* __restrict__ padded, Layout L, int to_padded) {
  // grid: x over columns, y over rows, z over planes (no divisions)
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  const int q = blockIdx.z;
  if (i >= L.nx) return;
  const long long d = ((long long)q * L.ny + j) * L.nx + i;
  const long long p = q * L.plane + L.node(i, j);
  if (to_padded) padded[p] = dense[d];
  else ((R*)dense)[d] = padded[p];
}

static int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename R>
void launch_pack(const R* dense, R* padded, const Layout& L, cudaStream_t st) {
  dim3 grd((L.nx + 255) / 256, L.ny, 16);
  pack_kernel<R><<<grd, 256, 0, st>>>(dense, padded, L, 1);
}
template <typename R>
void launch_unpack(const R* padded, R* dense, const Layout& L, cudaStream_t st) {
  dim3 grd((L.nx + 255) / 256, L.ny, 16);
  pack_kernel<R><<<grd, 256, 0, st>>>(dense, (R*)padded, L, 0);
}

// ---------------------------------------------------------------------------
// f = M^-1 f^eq(rho, u, T), computed in FP64.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void init_eq_kernel(const double* __restrict__ rho_in, const double* __restrict__ ux_in,
                               const double* __restrict__ uy_in, const double* __restrict__ T_in,
                               R* __restrict__ f, Layout L, Coef<double> c) {
  const long long n = (long long)L.ny * L.nx;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.nx), j = (int)(t / L.nx);
    const double rho = rho_in[t], ux = ux_in[t], uy = uy_in[t], T = T_in[t];
    const double e = rho * (T + 0.5 * (ux * ux + uy * uy));
    double eq[16], g[16];
    equilibrium(c, rho, 1.0 / rho, rho * ux, rho * uy, e, ux, uy, T, eq);
    inverse_full(c, eq, g);
    const long long at = L.node(i, j);
#pragma unroll
    for (int q = 0; q < 16; ++q) f[q * L.plane + at] = (R)g[q];
  }
}

template <typename R>
void launch_init_eq(const double* rho, const double* ux, const double* uy, const double* T, R* f,
                    const Layout& L, const Coef<double>& c64, cudaStream_t st) {
  const long long n = (long long)L.ny * L.nx;
  init_eq_kernel<R><<<grid_for(n, 128), 128, 0, st>>>(rho, ux, uy, T, f, L, c64);
}

// ---------------------------------------------------------------------------
// rho, u, T in FP64 (Sec. II, R = 1).
// ---------------------------------------------------------------------------
// Moment sums in the storage precision (FP32 states: the same recovery as
// the step, FP32 sums and the compensated temperature numerator), outputs
// in FP64.
template <typename R>
__global__ void macros_kernel(const R* __restrict__ f, double* rho_o, double* ux_o, double* uy_o,
                              double* T_o, Layout L) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= L.nx) return;
  const long long t = (long long)j * L.nx + i;
  const long long at = L.node(i, j);
  R g[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) g[q] = f[q * L.plane + at];
  R rho, jx, jy, e;
  conserved(g, rho, jx, jy, e);
  const R ir = recip(rho);
  if (rho_o) rho_o[t] = (double)rho;
  if (ux_o) ux_o[t] = (double)(jx * ir);
  if (uy_o) uy_o[t] = (double)(jy * ir);
  if (T_o) T_o[t] = (double)temperature(rho, jx, jy, e, ir);
}

template <typename R>
void launch_macros(const R* f, double* rho, double* ux, double* uy, double* T, const Layout& L,
                   cudaStream_t st) {
  dim3 grd((L.nx + 127) / 128, L.ny);
  macros_kernel<R><<<grd, 128, 0, st>>>(f, rho, ux, uy, T, L);
}

// ---------------------------------------------------------------------------
// Conservation sums (FP64) and the max |T - T_prev| residual.
// Warp shuffles, then one atomic per warp.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void reduce_kernel(const R* __restrict__ f, double* acc, double* Tprev, int have_prev,
                              Layout L) {
  const long long n = (long long)L.ny * L.nx;
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0, mx = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.nx), j = (int)(t / L.nx);
    const long long at = L.node(i, j);
    double g[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) g[q] = (double)f[q * L.plane + at];
    double rho, jx, jy, e;
    conserved(g, rho, jx, jy, e);
    s0 += rho; s1 += jx; s2 += jy; s3 += e;
    const double T = temperature(rho, jx, jy, e, 1.0 / rho);
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
    // non-negative doubles order like their bit patterns; NaN maps above inf
    atomicMax((unsigned long long*)(acc + 4), (unsigned long long)__double_as_longlong(mx));
  }
}

template <typename R>
void launch_reduce(const R* f, double* acc, double* Tprev, int have_prev, const Layout& L,
                   cudaStream_t st) {
  const long long n = (long long)L.ny * L.nx;
  reduce_kernel<R><<<grid_for(n, 256), 256, 0, st>>>(f, acc, Tprev, have_prev, L);
}

#define MRTLB_INSTANTIATE(R)                                                                     \
  template void launch_step_plain<R>(const R*, R*, const Layout&, const Coef<R>&, int*,          \
                                     cudaStream_t);                                              \
  template void launch_bc<R>(R*, const Layout&, const Coef<R>&, const Walls&, cudaStream_t); \
  template void launch_walls<R>(R*, const Layout&, const Coef<R>&, const Walls&, cudaStream_t); \
  template void launch_inflow<R>(R*, const Layout&, const Coef<R>&, const Walls&, cudaStream_t); \
  template void launch_pack<R>(const R*, R*, const Layout&, cudaStream_t);                       \
  template void launch_unpack<R>(const R*, R*, const Layout&, cudaStream_t);                     \
  template void launch_init_eq<R>(const double*, const double*, const double*, const double*,    \
                                  R*, const Layout&, const Coef<double>&, cudaStream_t);         \
  template void launch_macros<R>(const R*, double*, double*, double*, double*, const Layout&,    \
                                 cudaStream_t);                                                  \
  template void launch_reduce<R>(const R*, double*, double*, int, const Layout&, cudaStream_t);

MRTLB_INSTANTIATE(float)
MRTLB_INSTANTIATE(double)

}  // namespace mrtlb
