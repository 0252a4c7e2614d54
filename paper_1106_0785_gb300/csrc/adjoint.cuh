// adjoint.cuh - reverse-mode (transpose) arithmetic of the per-node step.
//
// Each function here is the hand-written transpose of a forward function
// in physics.cuh, taking output adjoints ("bar" quantities, dL/d(output))
// and accumulating input adjoints.  The structure of M carries over: the
// transpose of M^-1's inverse butterflies is the forward harmonic butterfly,
// and the transpose of the moment rows is a radial combination per family.
#pragma once

#include "kernels.cuh"
#include "physics.cuh"

namespace mrtlb {

// 1/x as the forward step forms it (FP32: the Newton-refined approximation,
// 5% faster forward + adjoint than the correctly rounded division; FP64: the
// division)
template <typename R>
__device__ __forceinline__ R adj_inv(R x) {
  return recip(x);
}

// transpose of harmonics(): harmonic adjoints -> f adjoints (H^T)
template <typename R>
__device__ __forceinline__ void harmonics_T(const Harm<R>& hb, R fb[16]) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const R S = hb.S[s], X = hb.X[s], Y = hb.Y[s];
    if (s == 0 || s == 2) {  // S = a0+a1+a2+a3, X = a0-a2, Y = a1-a3, Q = a0-a1+a2-a3
      const R Q = hb.Q[s >> 1];
      fb[4 * s + 0] = S + X + Q;
      fb[4 * s + 2] = S - X + Q;
      fb[4 * s + 1] = S + Y - Q;
      fb[4 * s + 3] = S - Y - Q;
    } else {                 // X = b0-b1-b2+b3, Y = b0+b1-b2-b3, P = b0-b1+b2-b3
      const R P = hb.P[s >> 1];
      fb[4 * s + 0] = S + X + Y + P;
      fb[4 * s + 1] = S - X + Y - P;
      fb[4 * s + 2] = S - X - Y + P;
      fb[4 * s + 3] = S + X - Y - P;
    }
  }
}

// transpose of moments(): moment adjoints -> harmonic adjoints (Mom^T)
template <typename R>
__device__ __forceinline__ void moments_T(const R mb[16], Harm<R>& hb) {
  hb.S[0] = mb[0] + R(0.5) * mb[3] + R(0.25) * mb[10] + mb[11];
  hb.S[1] = mb[0] + mb[3] + mb[10] - R(4) * mb[11];
  hb.S[2] = mb[0] + R(2) * mb[3] + R(4) * mb[10] + R(16) * mb[11];
  hb.S[3] = mb[0] + R(4) * mb[3] + R(16) * mb[10] - R(64) * mb[11];
  hb.X[0] = mb[1] + R(0.5) * mb[6] + mb[8] + mb[14];
  hb.X[1] = mb[1] + mb[6] - R(2) * mb[8] - R(4) * mb[14];
  hb.X[2] = R(2) * mb[1] + R(4) * mb[6] + R(8) * mb[8] + R(32) * mb[14];
  hb.X[3] = R(2) * mb[1] + R(8) * mb[6] - R(16) * mb[8] - R(128) * mb[14];
  hb.Y[0] = mb[2] + R(0.5) * mb[7] - mb[9] - mb[15];
  hb.Y[1] = mb[2] + mb[7] + R(2) * mb[9] + R(4) * mb[15];
  hb.Y[2] = R(2) * mb[2] + R(4) * mb[7] - R(8) * mb[9] - R(32) * mb[15];
  hb.Y[3] = R(2) * mb[2] + R(8) * mb[7] + R(16) * mb[9] + R(128) * mb[15];
  hb.Q[0] = mb[4] + mb[12];
  hb.Q[1] = R(4) * mb[4] + R(16) * mb[12];
  hb.P[0] = mb[5] + R(2) * mb[13];
  hb.P[1] = R(4) * mb[5] + R(32) * mb[13];
}

// transpose of inverse_full() (full = true) or inverse_nonconserved()
// (full = false: rows 0..3 of mb are left at zero): f adjoints -> moment adjoints
template <typename R>
__device__ __forceinline__ void inverse_T(const Coef<R>& c, const R fb[16], R mb[16], bool full) {
  Harm<R> h;
  harmonics(fb, h);  // the inverse butterflies transpose to the forward butterflies
#pragma unroll
  for (int k = 0; k < 16; ++k) mb[k] = R(0);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (full) {
      mb[0] += c.invS[s][0] * h.S[s];
      mb[3] += c.invS[s][1] * h.S[s];
      mb[1] += c.invX[s][0] * h.X[s];
      mb[2] += c.invY[s][0] * h.Y[s];
    }
    mb[10] += c.invS[s][2] * h.S[s];
    mb[11] += c.invS[s][3] * h.S[s];
    mb[6] += c.invX[s][1] * h.X[s];
    mb[8] += c.invX[s][2] * h.X[s];
    mb[14] += c.invX[s][3] * h.X[s];
    mb[7] += c.invY[s][1] * h.Y[s];
    mb[9] += c.invY[s][2] * h.Y[s];
    mb[15] += c.invY[s][3] * h.Y[s];
  }
  mb[4] = c.invQ[0][0] * h.Q[0] + c.invQ[1][0] * h.Q[1];
  mb[12] = c.invQ[0][1] * h.Q[0] + c.invQ[1][1] * h.Q[1];
  mb[5] = c.invP[0][0] * h.P[0] + c.invP[1][0] * h.P[1];
  mb[13] = c.invP[0][1] * h.P[0] + c.invP[1][1] * h.P[1];
}

// Adjoints of the inputs of equilibrium() (treated as independent):
// rho, inv_rho, jx, jy, e, ux, uy, T.
template <typename R>
struct EqIn {
  R rho, ir, jx, jy, e, ux, uy, T;
};

// transpose of equilibrium(): eqb[16] (all rows) -> adjoints of its inputs
// (VER: the equilibrium version fixed at compile time, 0 = c.version).
template <typename R, int VER = 0>
__device__ __forceinline__ void equilibrium_T(const Coef<R>& c, const EqIn<R>& x, const R eqb[16],
                                              EqIn<R>& g) {
  const R ux = x.ux, uy = x.uy, ux2 = ux * ux, uy2 = uy * uy, u2 = ux2 + uy2;
  const R p = x.rho * x.T;
  R pb = R(0), u2b = R(0), wb = R(0);
  g.rho += eqb[0];
  g.jx += eqb[1];
  g.jy += eqb[2];
  g.e += eqb[3];
  // 14a: jx ux - jy uy
  g.jx += eqb[4] * ux; g.ux += eqb[4] * x.jx; g.jy -= eqb[4] * uy; g.uy -= eqb[4] * x.jy;
  // 14b: jx uy
  g.jx += eqb[5] * uy; g.uy += eqb[5] * x.jx;
  // 14c, 14d: (e + p) u
  const R ep = x.e + p;
  g.e += eqb[6] * ux + eqb[7] * uy;
  pb += eqb[6] * ux + eqb[7] * uy;
  g.ux += eqb[6] * ep;
  g.uy += eqb[7] * ep;
  // 14e: jx (ux^2 - 3 uy^2)
  g.jx += eqb[8] * (ux2 - R(3) * uy2); g.ux += eqb[8] * x.jx * R(2) * ux; g.uy -= eqb[8] * x.jx * R(6) * uy;
  // 14f: jy (3 ux^2 - uy^2)
  g.jy += eqb[9] * (R(3) * ux2 - uy2); g.ux += eqb[9] * x.jy * R(6) * ux; g.uy -= eqb[9] * x.jy * R(2) * uy;
  // 14g: 2 e^2 ir - rho u2^2 / 4
  g.e += eqb[10] * R(4) * x.e * x.ir;
  g.ir += eqb[10] * R(2) * x.e * x.e;
  g.rho -= eqb[10] * R(0.25) * u2 * u2;
  u2b -= eqb[10] * R(0.5) * x.rho * u2;
  // 14h, 14i with w = 6 e - 2 rho u2
  const R w = R(6) * x.e - R(2) * x.rho * u2;
  wb += eqb[12] * (ux2 - uy2) + eqb[13] * ux * uy;
  g.ux += eqb[12] * w * R(2) * ux + eqb[13] * w * uy;
  g.uy += -eqb[12] * w * R(2) * uy + eqb[13] * w * ux;
  const int ver = VER ? VER : c.version;
  if (ver == 2) {
    const R A = R(-4) + R(10) * x.T + R(5) * ux2 - R(5) * uy2;
    const R B = R(4) - R(10) * x.T + R(5) * ux2 - R(5) * uy2;
    g.rho += eqb[14] * ux * A + eqb[15] * uy * B;
    g.ux += eqb[14] * x.rho * (A + R(10) * ux2) + eqb[15] * x.rho * uy * R(10) * ux;
    g.uy += -eqb[14] * x.rho * ux * R(10) * uy + eqb[15] * x.rho * (B - R(10) * uy2);
    g.T += R(10) * x.rho * (eqb[14] * ux - eqb[15] * uy);
  } else if (ver == 3) {
    // rows 12, 15, 16 of M applied to f_M,q = rho/(2 pi T) exp(-|v_q - u|^2 / 2T):
    // their adjoints go back through the harmonics to f_M, then through
    // d f_M,q = f_M,q (drho / rho + (v_q - u).du / T + (|v_q - u|^2 / 2T^2 - 1/T) dT)
    Harm<R> hb;
    const R sw[4] = {R(1), R(-4), R(16), R(-64)};
    const R xw[4] = {R(1), R(-4), R(32), R(-128)};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      hb.S[s] = eqb[11] * sw[s];
      hb.X[s] = eqb[14] * xw[s];
      hb.Y[s] = -eqb[15] * xw[s];
    }
    hb.Q[0] = hb.Q[1] = hb.P[0] = hb.P[1] = R(0);
    R fmb[16];
    harmonics_T(hb, fmb);
    const R iT = adj_inv(x.T);
    const R pre = x.rho * iT * R(0.15915494309189533576888376337251);  // rho / (2 pi T)
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const R dx = R(vx_of(q)) - ux, dy = R(vy_of(q)) - uy, d2 = dx * dx + dy * dy;
      const R w = fmb[q] * pre * expr(R(-0.5) * iT * d2);
      g.rho += w * x.ir;
      g.ux += w * dx * iT;
      g.uy += w * dy * iT;
      g.T += w * (R(0.5) * d2 * iT * iT - iT);
    }
  }
  // w, u2, p
  g.e += R(6) * wb;
  g.rho -= R(2) * u2 * wb;
  u2b -= R(2) * x.rho * wb;
  g.ux += R(2) * ux * u2b;
  g.uy += R(2) * uy * u2b;
  g.rho += pb * x.T;
  g.T += pb * x.rho;
}

// Chain the adjoints of (rho, ir, jx, jy, e, ux, uy, T) back to the
// conserved moments (rho, jx, jy, e) through ir = 1/rho, u = j ir and
// T = (e rho - |j|^2/2) ir^2, and return dL/dm for rows 0..3.
template <typename R>
__device__ __forceinline__ void chain_primitive(const EqIn<R>& x, const EqIn<R>& g, R& rb, R& jxb, R& jyb,
                                                R& eb) {
  R irb = g.ir;
  jxb = g.jx + g.ux * x.ir;
  jyb = g.jy + g.uy * x.ir;
  irb += g.ux * x.jx + g.uy * x.jy;
  const R N = x.e * x.rho - R(0.5) * (x.jx * x.jx + x.jy * x.jy);
  const R Nb = g.T * x.ir * x.ir;
  irb += g.T * R(2) * N * x.ir;
  eb = g.e + Nb * x.rho;
  rb = g.rho + Nb * x.e - irb * x.ir * x.ir;
  jxb -= Nb * x.jx;
  jyb -= Nb * x.jy;
}

// Coefficients of one adjoint step.
template <typename R>
struct AdjCoef {
  Coef<R> c;
  R selfw[16];  // Lax-Wendroff self weight 1 - sum_n k_qn, in R as the step forms it
  // derivatives of the modification factors dt (s7/s5 - 1), ... divided by
  // dt (the rate gradients are summed without the factor dt, which the host
  // applies to the totals): 1/s5, 1/s6, s7/s5^2, s7/s6^2, s8/s5^2, s8/s6^2
  R g[6];
};

template <typename R>
__device__ __forceinline__ bool advanced(const Layout& L, int i, int j) {
  return i >= L.i0 && i < L.i1 && j >= L.j0 && j < L.j1;
}

// Rows 6 and 7 of inverse_T (all the modification needs): only the X and
// Y harmonics of fb enter them.
template <typename R>
__device__ __forceinline__ void inverse_T_67(const Coef<R>& c, const R fb[16], R& m6, R& m7) {
  m6 = R(0);
  m7 = R(0);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const R a0 = fb[4 * s + 0], a1 = fb[4 * s + 1], a2 = fb[4 * s + 2], a3 = fb[4 * s + 3];
    R X, Y;
    if (s == 0 || s == 2) {
      X = a0 - a2;
      Y = a1 - a3;
    } else {
      X = (a0 + a3) - (a1 + a2);
      Y = (a0 + a1) - (a2 + a3);
    }
    m6 += c.invX[s][1] * X;
    m7 += c.invY[s][1] * Y;
  }
}

// Adjoints of the two strain combinations of the modification at an
// advanced node r with adjoint lambda (dL/dC = -lambda), rho T = P:
//   gsh = dL/d(du_x/dx - du_y/dy),  gst = dL/d(du_y/dx + du_x/dy).
template <typename R>
__device__ __forceinline__ void gbar_node(const Coef<R>& c, const R lam[16], R P, R ux, R uy, R& gsh, R& gst) {
  R c6, c7;
  inverse_T_67(c, lam, c6, c7);
  c6 = -c6;
  c7 = -c7;
  gsh = c6 * c.mod[0] * P * ux + c7 * c.mod[3] * P * uy;
  gst = c6 * c.mod[1] * P * uy + c7 * c.mod[2] * P * ux;
}

// At an advanced node p with state g = B(f)(p), adjoint lp = lambda(p),
// velocity u(p) and the two strain combinations of the forward step:
// lt = (1 - sum_n k_qn) lp_q - (dC/dg)^T lp  (Lax-Wendroff self weight and
// collision transpose, the temperature linearised at T = (e - j.u/2)/rho),
// and the rate gradients of the node added to G[4..15] (RATES = false
// skips them and the moments and equilibria only they need; lt is the same).
// uxb, uyb: the adjoint of u(p) from elsewhere (the modification at the
// neighbours); it joins the collision's own u adjoint and goes back to f
// through u = j / rho with it, which is velocity_T folded into the moments
// (rows 1, v_x, v_y of M).  VER: the equilibrium version fixed at compile
// time (0 = c.version).
template <typename R, bool RATES = true, int VER = 0>
__device__ __forceinline__ void collision_T_node(const AdjCoef<R>& a, const R g[16], const R lp[16], R ux, R uy,
                                                 R shear, R strain, R uxb, R uyb, R lt[16], R G[16]) {
  const Coef<R>& c = a.c;
  R rho, jx, jy, e;
  conserved(g, rho, jx, jy, e);
  const R ir = adj_inv(rho);
  const R T = (e - R(0.5) * (jx * ux + jy * uy)) * ir;
#pragma unroll
  for (int q = 0; q < 16; ++q) lt[q] = a.selfw[q] * lp[q];
  R m[16], eq[16];
  if constexpr (RATES) {
    Harm<R> h;
    harmonics(g, h);
    moments(h, m);
    equilibrium<R, VER>(c, rho, ir, jx, jy, e, ux, uy, T, eq);
  }
  const R Pp = rho * T;
  R Cb[16], cb[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) Cb[q] = -lp[q];
  inverse_T(c, Cb, cb, false);
  R mb[16], eqb[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    mb[k] = (k >= 4) ? c.rate[k] * cb[k] : R(0);
    eqb[k] = (k >= 4) ? -c.rate[k] * cb[k] : R(0);
  }
  EqIn<R> x{rho, ir, jx, jy, e, ux, uy, T};
  EqIn<R> gi{R(0), R(0), R(0), R(0), R(0), uxb, uyb, R(0)};
  if (c.modified) {
    const R Pb = cb[6] * (c.mod[0] * ux * shear + c.mod[1] * uy * strain) +
                 cb[7] * (c.mod[2] * ux * strain + c.mod[3] * uy * shear);
    gi.ux += cb[6] * c.mod[0] * Pp * shear + cb[7] * c.mod[2] * Pp * strain;
    gi.uy += cb[6] * c.mod[1] * Pp * strain + cb[7] * c.mod[3] * Pp * shear;
    gi.rho += Pb * T;
    gi.T += Pb * rho;
  }
  equilibrium_T<R, VER>(c, x, eqb, gi);
  R rb, jxb, jyb, eb;
  chain_primitive(x, gi, rb, jxb, jyb, eb);
  mb[0] += rb;
  mb[1] += jxb;
  mb[2] += jyb;
  mb[3] += eb;
  Harm<R> hb;
  moments_T(mb, hb);
  R fb[16];
  harmonics_T(hb, fb);
#pragma unroll
  for (int q = 0; q < 16; ++q) lt[q] += fb[q];
  // rate gradients over dt: d f1 / d s_k through dt s_k (m_k - eq_k) and
  // the modification factors dt (s7/s5 - 1), ... (dL/dC = -lambda)
  if constexpr (RATES) {
#pragma unroll
    for (int k = 4; k < 16; ++k) G[k] += cb[k] * (m[k] - eq[k]);
    if (c.modified) {
      const R A0 = Pp * ux * shear, A1 = Pp * uy * strain;
      const R A2 = Pp * ux * strain, A3 = Pp * uy * shear;
      G[6] += cb[6] * (A0 * a.g[0] + A1 * a.g[1]);        // 1/s5, 1/s6
      G[7] += cb[7] * (A2 * a.g[1] + A3 * a.g[0]);
      G[4] -= cb[6] * A0 * a.g[2] + cb[7] * A3 * a.g[4];  // s7/s5^2, s8/s5^2
      G[5] -= cb[6] * A1 * a.g[3] + cb[7] * A2 * a.g[5];  // s7/s6^2, s8/s6^2
    }
  }
}

// Adjoint of u = j / rho at p carried to f(p): lt_q += (ub . (v_q - u)) / rho.
template <typename R>
__device__ __forceinline__ void velocity_T(R uxb, R uyb, R ux, R uy, R ir, R lt[16]) {
#pragma unroll
  for (int q = 0; q < 16; ++q) lt[q] += (uxb * (R(vx_of(q)) - ux) + uyb * (R(vy_of(q)) - uy)) * ir;
}

// Sum the rate gradients over the warp; one FP64 atomic per warp and rate.
template <typename R>
__device__ __forceinline__ void flush_rate_gradients(const R G[16], double* gacc) {
#pragma unroll
  for (int k = 4; k < 16; ++k) {
    R v = G[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != R(0)) atomicAdd(gacc + k, (double)v);
  }
}

}  // namespace mrtlb
