// physics.cuh - per-node arithmetic of the MRT FD-LB step (device side).
//
// Everything here is specialised to the paper's D2V16 velocity set (Sec. II,
// Fig. 1) and its SO(2) moment matrix M.  M is never applied as a dense
// 16x16 matrix: its rows are radial polynomials times angular harmonics, so
//   * inside each of the four shells (speed 1, sqrt2, 2, 2sqrt2; four
//     velocities each) a 4-point butterfly gives the angular harmonics
//       axis shells:     S = sum, X = a0-a2, Y = a1-a3, Q = (a0+a2)-(a1+a3)
//       diagonal shells: S = sum, X = (b0+b3)-(b1+b2), Y = (b0+b1)-(b2+b3),
//                        P = (b0+b2)-(b1+b3)
//   * each moment row is a fixed radial combination of one harmonic family
//     over the shells (S: rows 1,4,11,12; X: 2,7,9,15; Y: 3,8,10,16;
//     Q: 5,13; P: 6,14 - the paper's 1-based numbering).
// M^-1 factors the same way: the host inverts each family's small radial
// matrix exactly (rational arithmetic) and passes the columns here.
//
// Indices are 0-based: plane q = paper velocity i = q+1, moment k = paper
// moment k+1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pair.cuh"

namespace mrtlb {

// D2V16 (Fig. 1): order fixed by rows m2 = v_x and m3 = v_y of M.
__host__ __device__ constexpr int vx_of(int q) {
  return (q == 0) ? 1 : (q == 2) ? -1 : (q == 4) ? 1 : (q == 5) ? -1 : (q == 6) ? -1 : (q == 7) ? 1
       : (q == 8) ? 2 : (q == 10) ? -2 : (q == 12) ? 2 : (q == 13) ? -2 : (q == 14) ? -2 : (q == 15) ? 2 : 0;
}
__host__ __device__ constexpr int vy_of(int q) {
  return (q == 1) ? 1 : (q == 3) ? -1 : (q == 4) ? 1 : (q == 5) ? 1 : (q == 6) ? -1 : (q == 7) ? -1
       : (q == 9) ? 2 : (q == 11) ? -2 : (q == 12) ? 2 : (q == 13) ? 2 : (q == 14) ? -2 : (q == 15) ? -2 : 0;
}

// Per-context constants.  The family inverse columns are pre-scaled by the
// inverse-butterfly factors (1/4 for S and Q and 1/2 for X and Y on axis
// shells, 1/4 for everything on diagonal shells).
template <typename R>
struct Coef {
  // Lax-Wendroff (Sec. III): for unit speed along x, a1x = dt/(2dx),
  // b1x = (dt/dx)^2/2; speed-2 velocities use 2*a1x and 4*b1x.
  R a1x, b1x, a1y, b1y;
  R inv2dx, inv2dy;   // 1/(2 dx), 1/(2 dy) for the velocity gradients
  // the same scheme per velocity in neighbour-difference form:
  // f_new = f + kE (f_E - f) + kW (f_W - f) + kN (f_N - f) + kS (f_S - f) - dt C,
  // kE = b_x - a_x, kW = b_x + a_x (a_x = v_x dt/2dx, b_x = (v_x dt/dx)^2/2), same in y
  R lw[16][4];
  R lwsum[16];        // sum_n lw[q][n], exactly (the lw[q][n] lie on a common grid)
  R rate[16];         // dt * s_k (k >= 4 used)
  R mod[4];           // dt*(s7/s5-1), dt*(s7/s6-1), dt*(s8/s6-1), dt*(s8/s5-1)
  R invS[4][4];       // [shell A,B,C,D][family row: k=0,3,10,11]
  R invX[4][4];       // rows k = 1,6,8,14
  R invY[4][4];       // rows k = 2,7,9,15
  R invQ[2][2];       // [shell A,C][rows k = 4,12]
  R invP[2][2];       // [shell B,D][rows k = 5,13]
  int version;        // equilibrium version for k = 11, 14, 15
  int modified;       // 1 = energy-flux modification on
};

template <typename R>
struct Harm {
  R S[4], X[4], Y[4], Q[2], P[2];  // Q: shells A,C; P: shells B,D
};

#define MRTLB_HD __host__ __device__ __forceinline__

template <typename R>
MRTLB_HD void harmonics(const R f[16], Harm<R>& h) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const R a0 = f[4 * s + 0], a1 = f[4 * s + 1], a2 = f[4 * s + 2], a3 = f[4 * s + 3];
    const R p02 = a0 + a2, p13 = a1 + a3;
    h.S[s] = p02 + p13;
    if (s == 0 || s == 2) {  // axis shell
      h.X[s] = a0 - a2;
      h.Y[s] = a1 - a3;
      h.Q[s >> 1] = p02 - p13;
    } else {                 // diagonal shell
      const R p03 = a0 + a3, p12 = a1 + a2;
      h.X[s] = p03 - p12;
      h.Y[s] = (a0 + a1) - (a2 + a3);
      h.P[s >> 1] = p02 - p13;
    }
  }
}

// Moments of one family row from the harmonics (rows of M, Sec. II).
template <typename R>
MRTLB_HD void moments(const Harm<R>& h, R m[16]) {
  const R SA = h.S[0], SB = h.S[1], SC = h.S[2], SD = h.S[3];
  const R XA = h.X[0], XB = h.X[1], XC = h.X[2], XD = h.X[3];
  const R YA = h.Y[0], YB = h.Y[1], YC = h.Y[2], YD = h.Y[3];
  m[0] = (SA + SB) + (SC + SD);
  m[3] = R(0.5) * SA + SB + R(2) * SC + R(4) * SD;
  m[10] = R(0.25) * SA + SB + R(4) * SC + R(16) * SD;
  m[11] = SA - R(4) * SB + R(16) * SC - R(64) * SD;
  m[1] = (XA + XB) + R(2) * (XC + XD);
  m[6] = R(0.5) * XA + XB + R(4) * XC + R(8) * XD;
  m[8] = XA - R(2) * XB + R(8) * XC - R(16) * XD;
  m[14] = XA - R(4) * XB + R(32) * XC - R(128) * XD;
  m[2] = (YA + YB) + R(2) * (YC + YD);
  m[7] = R(0.5) * YA + YB + R(4) * YC + R(8) * YD;
  m[9] = -YA + R(2) * YB - R(8) * YC + R(16) * YD;
  m[15] = -YA + R(4) * YB - R(32) * YC + R(128) * YD;
  m[4] = h.Q[0] + R(4) * h.Q[1];
  m[12] = h.Q[0] + R(16) * h.Q[1];
  m[5] = h.P[0] + R(4) * h.P[1];
  m[13] = R(2) * h.P[0] + R(32) * h.P[1];
}

// Conserved moments only: rho, j_x, j_y, e (rows 1-4 of M), from the
// harmonics or from f.
template <typename R>
MRTLB_HD void conserved_h(const Harm<R>& h, R& rho, R& jx, R& jy, R& e) {
  rho = (h.S[0] + h.S[1]) + (h.S[2] + h.S[3]);
  e = R(0.5) * h.S[0] + h.S[1] + R(2) * h.S[2] + R(4) * h.S[3];
  jx = (h.X[0] + h.X[1]) + R(2) * (h.X[2] + h.X[3]);
  jy = (h.Y[0] + h.Y[1]) + R(2) * (h.Y[2] + h.Y[3]);
}
template <typename R>
MRTLB_HD void conserved(const R f[16], R& rho, R& jx, R& jy, R& e) {
  Harm<R> h;
  harmonics(f, h);
  conserved_h(h, rho, jx, jy, e);
}

// Temperature from the conserved moments (Sec. II with R = 1):
// T = (e rho - |j|^2 / 2) / rho^2.  The numerator, where the kinetic part
// cancels against e behind strong shocks, is formed to about twice FP32
// precision (temperature_compensated; MRTLB_TEMP_COMPENSATED = 0 forms it in
// FP64 from the exact FP64 products of the FP32 moments); the final scaling
// is FP32.
//
// temperature_compensated: N = e rho - (jx^2 + jy^2)/2 to about twice the
// working precision, each product split exactly into its rounded value and
// error (Dekker's TwoProduct in its fused multiply-add form), the two large
// cancellations done with Dekker's Fast2Sum, which is exact when the first
// operand is the larger; here e rho >= (jx^2 + jy^2)/2 whenever T >= 0.
static_assert(sizeof(decltype(fma(1.0f, 1.0f, 1.0f))) == sizeof(float), "fma on floats must stay in FP32");
template <typename R>
MRTLB_HD R temperature_compensated(R rho, R jx, R jy, R e, R inv_rho) {
  const R p = e * rho, ep = fma(e, rho, -p);
  const R hx = R(0.5f) * jx, hy = R(0.5f) * jy;  // exact
  const R a = hx * jx, ea = fma(hx, jx, -a);
  const R b = hy * jy, eb = fma(hy, jy, -b);
  const R s1 = p - a, t1 = (p - s1) - a;
  const R s2 = s1 - b, t2 = (s1 - s2) - b;
  const R num = s2 + ((t1 + t2) + ((ep - ea) - eb));
  return R(num * R(inv_rho * inv_rho));
}
#ifndef MRTLB_TEMP_COMPENSATED
#define MRTLB_TEMP_COMPENSATED 1
#endif
__device__ __forceinline__ float temperature(float rho, float jx, float jy, float e, float inv_rho) {
#if MRTLB_TEMP_COMPENSATED
  return temperature_compensated(rho, jx, jy, e, inv_rho);
#else
  const double j2 = fma((double)jy, (double)jy, (double)jx * (double)jx);
  const double num = fma((double)e, (double)rho, -0.5 * j2);
  return (float)num * (inv_rho * inv_rho);
#endif
}
// (FP64 states: the plain formula)
template <typename R>
MRTLB_HD R temperature_plain(R rho, R jx, R jy, R e, R inv_rho) {
  const R j2 = fma(jy, jy, R(jx * jx));
  return R(fma(e, rho, R(R(-0.5) * j2)) * R(inv_rho * inv_rho));
}
__device__ __forceinline__ double temperature(double rho, double jx, double jy, double e, double inv_rho) {
  return temperature_plain(rho, jx, jy, e, inv_rho);
}

// 1/x: the hardware approximation refined by one Newton-Raphson step
// r <- r (2 - x r), which roughly squares the relative error of the
// approximation (about 2^-22 before the step).
__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r * fmaf(-x, r, 2.0f);
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
// The same three functions on a pair of nodes (pair.cuh): the reciprocal's
// Newton-Raphson step and the compensated numerator run packed; the
// hardware approximation and the exponential run per lane.
__device__ __forceinline__ P2 recip(P2 x) {
  float a, b;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(a) : "f"(x.v.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(b) : "f"(x.v.y));
  const P2 r(a, b);
  return P2(r * fma(-x, r, P2(2.0f)));
}
__device__ __forceinline__ P2 temperature(P2 rho, P2 jx, P2 jy, P2 e, P2 inv_rho) {
  return temperature_compensated(rho, jx, jy, e, inv_rho);
}
__device__ __forceinline__ P2 expr(P2 x) { return P2(expf(x.v.x), expf(x.v.y)); }

// The macroscopic state of one node: the conserved moments, 1/rho, u and T.
template <typename R>
struct NodeMac {
  R rho, ir, jx, jy, e, ux, uy, T;
};
template <typename R>
MRTLB_HD NodeMac<R> node_macros(const R g[16]) {
  NodeMac<R> m;
  conserved(g, m.rho, m.jx, m.jy, m.e);
  m.ir = recip(m.rho);
  m.ux = R(m.jx * m.ir);
  m.uy = R(m.jy * m.ir);
  m.T = temperature(m.rho, m.jx, m.jy, m.e, m.ir);
  return m;
}

// One velocity's Lax-Wendroff update with the collision term,
// f0 + (sum_n k_qn (f_n - f0) - C), given the four neighbours' values.  The
// difference form keeps a uniform region exactly uniform (every f_n - f0
// is an exact zero there); the fused form below (MRTLB_LW_WEIGHTS = 1) takes
// fewer operations but makes the same rounding error at every node of a
// uniform region, which then drifts by about one ulp per step.
#ifndef MRTLB_LW_WEIGHTS
#define MRTLB_LW_WEIGHTS 0
#endif
template <typename R>
MRTLB_HD R lw_update(const Coef<R>& c, int q, R f0, R Cq, R fE, R fW, R fN, R fS) {
#if MRTLB_LW_WEIGHTS
  // (1 - S) f0 - C + sum_n k_qn f_n with S = sum_n k_qn: summed over the
  // nodes of a periodic grid this is sum f0 - sum C exactly whenever S is
  // the exact sum of the stored k_qn, which the coefficient set-up ensures,
  // so it conserves like the difference form with fewer operations.
  R v = fma(-c.lwsum[q], f0, f0) - Cq;
  if (vx_of(q) != 0) {
    v = fma(c.lw[q][0], fE, v);
    v = fma(c.lw[q][1], fW, v);
  }
  if (vy_of(q) != 0) {
    v = fma(c.lw[q][2], fN, v);
    v = fma(c.lw[q][3], fS, v);
  }
#else
  // the increment is summed first and added to f0 once: each partial sum
  // rounds at the increment's own (small) magnitude, and only the final
  // addition at f0's, instead of all five (same operation count)
  R d = -Cq;
  if (vx_of(q) != 0) {
    d += c.lw[q][0] * (fE - f0);
    d += c.lw[q][1] * (fW - f0);
  }
  if (vy_of(q) != 0) {
    d += c.lw[q][2] * (fN - f0);
    d += c.lw[q][3] * (fS - f0);
  }
  const R v = f0 + d;
#endif
  return v;
}

__device__ __forceinline__ float expr(float x) { return expf(x); }
__device__ __forceinline__ double expr(double x) { return exp(x); }

// Equilibrium moments k = 4..15 (Eqs. 14a-14i and the version rule for
// k = 11, 14, 15), given the conserved moments and u, T.
template <typename R, int VER = 0>
MRTLB_HD void equilibrium(const Coef<R>& c, R rho, R inv_rho, R jx, R jy, R e,
                                            R ux, R uy, R T, R eq[16]) {
  const R ux2 = ux * ux, uy2 = uy * uy, u2 = ux2 + uy2;
  const R p = rho * T;
  eq[0] = rho; eq[1] = jx; eq[2] = jy; eq[3] = e;
  eq[4] = jx * ux - jy * uy;                      // 14a (jx^2 - jy^2)/rho
  eq[5] = jx * uy;                                // 14b jx jy / rho
  eq[6] = (e + p) * ux;                           // 14c
  eq[7] = (e + p) * uy;                           // 14d
  eq[8] = jx * (ux2 - R(3) * uy2);                // 14e
  eq[9] = jy * (R(3) * ux2 - uy2);                // 14f
  eq[10] = R(2) * e * e * inv_rho - R(0.25) * rho * u2 * u2;  // 14g
  const R w = R(6) * e - R(2) * rho * u2;
  eq[12] = w * (ux2 - uy2);                       // 14h
  eq[13] = w * ux * uy;                           // 14i
  const int ver = VER ? VER : c.version;          // (VER: fixed at compile time)
  if (ver == 2) {
    eq[11] = R(0);
    eq[14] = rho * ux * (R(-4) + R(10) * T + R(5) * ux2 - R(5) * uy2);
    eq[15] = rho * uy * (R(4) - R(10) * T + R(5) * ux2 - R(5) * uy2);
  } else if (ver == 3) {
    // rows 12, 15, 16 of M applied to rho/(2 pi T) exp(-(v - u)^2 / 2T)
    R fm[16];
    const R pre = rho * recip(R(6.283185307179586476925286766559) * T);
    const R m2T = R(-0.5) * recip(T);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const R dx = R(vx_of(q)) - ux, dy = R(vy_of(q)) - uy;
      fm[q] = pre * expr(m2T * (dx * dx + dy * dy));
    }
    Harm<R> h;
    harmonics(fm, h);
    eq[11] = h.S[0] - R(4) * h.S[1] + R(16) * h.S[2] - R(64) * h.S[3];
    eq[14] = h.X[0] - R(4) * h.X[1] + R(32) * h.X[2] - R(128) * h.X[3];
    eq[15] = -h.Y[0] + R(4) * h.Y[1] - R(32) * h.Y[2] + R(128) * h.Y[3];
  } else {
    eq[11] = R(0); eq[14] = R(0); eq[15] = R(0);
  }
}

// f = M^-1 m for a full moment vector (used for equilibria and walls).
template <typename R>
MRTLB_HD void inverse_full(const Coef<R>& c, const R m[16], R f[16]) {
  R S[4], X[4], Y[4], Q[2], P[2];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    S[s] = c.invS[s][0] * m[0] + c.invS[s][1] * m[3] + c.invS[s][2] * m[10] + c.invS[s][3] * m[11];
    X[s] = c.invX[s][0] * m[1] + c.invX[s][1] * m[6] + c.invX[s][2] * m[8] + c.invX[s][3] * m[14];
    Y[s] = c.invY[s][0] * m[2] + c.invY[s][1] * m[7] + c.invY[s][2] * m[9] + c.invY[s][3] * m[15];
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    Q[s] = c.invQ[s][0] * m[4] + c.invQ[s][1] * m[12];
    P[s] = c.invP[s][0] * m[5] + c.invP[s][1] * m[13];
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const bool axis = (s == 0 || s == 2);
    const R q_or_p = axis ? Q[s >> 1] : P[s >> 1];
    if (axis) {
      const R sp = S[s] + q_or_p, sm = S[s] - q_or_p;
      f[4 * s + 0] = sp + X[s];
      f[4 * s + 2] = sp - X[s];
      f[4 * s + 1] = sm + Y[s];
      f[4 * s + 3] = sm - Y[s];
    } else {
      const R spp = S[s] + q_or_p, smp = S[s] - q_or_p;
      f[4 * s + 0] = spp + (X[s] + Y[s]);
      f[4 * s + 2] = spp - (X[s] + Y[s]);
      f[4 * s + 1] = smp - (X[s] - Y[s]);
      f[4 * s + 3] = smp + (X[s] - Y[s]);
    }
  }
}

// f = M^-1 m for a moment vector whose conserved part m_0..m_3 is zero
// (the collision): the conserved columns of M^-1 are skipped.
template <typename R>
MRTLB_HD void inverse_nonconserved(const Coef<R>& c, const R m[16], R f[16]) {
  R S[4], X[4], Y[4], Q[2], P[2];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    S[s] = c.invS[s][2] * m[10] + c.invS[s][3] * m[11];
    X[s] = c.invX[s][1] * m[6] + c.invX[s][2] * m[8] + c.invX[s][3] * m[14];
    Y[s] = c.invY[s][1] * m[7] + c.invY[s][2] * m[9] + c.invY[s][3] * m[15];
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    Q[s] = c.invQ[s][0] * m[4] + c.invQ[s][1] * m[12];
    P[s] = c.invP[s][0] * m[5] + c.invP[s][1] * m[13];
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (s == 0 || s == 2) {
      const R sp = S[s] + Q[s >> 1], sm = S[s] - Q[s >> 1];
      f[4 * s + 0] = sp + X[s];
      f[4 * s + 2] = sp - X[s];
      f[4 * s + 1] = sm + Y[s];
      f[4 * s + 3] = sm - Y[s];
    } else {
      const R spp = S[s] + P[s >> 1], smp = S[s] - P[s >> 1];
      f[4 * s + 0] = spp + (X[s] + Y[s]);
      f[4 * s + 2] = spp - (X[s] + Y[s]);
      f[4 * s + 1] = smp - (X[s] - Y[s]);
      f[4 * s + 3] = smp + (X[s] - Y[s]);
    }
  }
}

// dt * C = dt * M^-1 c with c_k = s_k (f^_k - f^eq_k) for k >= 4 (the
// conserved components vanish) and the modification of Sec. II added to
// k = 6, 7 (the paper's 7 and 8), from the node's moments, macroscopic
// state and velocity gradients (dux/dx, dux/dy, duy/dx, duy/dy).
// collision_h takes the harmonics of f, collision f itself.
template <typename R>
MRTLB_HD void collision_h(const Coef<R>& c, const Harm<R>& h, R dux_dx, R dux_dy,
                                            R duy_dx, R duy_dy, R rho, R inv_rho, R jx, R jy, R e,
                                            R ux, R uy, R T, R C[16]) {
  R m[16];
  moments(h, m);
  R eq[16];
  equilibrium(c, rho, inv_rho, jx, jy, e, ux, uy, T, eq);
  R cc[16];
#pragma unroll
  for (int k = 4; k < 16; ++k) cc[k] = c.rate[k] * (m[k] - eq[k]);
  if (c.modified) {
    const R p = rho * T;
    const R shear = dux_dx - duy_dy;
    const R strain = duy_dx + dux_dy;
    const R pux = p * ux, puy = p * uy;
    cc[6] += c.mod[0] * pux * shear + c.mod[1] * puy * strain;
    cc[7] += c.mod[2] * pux * strain + c.mod[3] * puy * shear;
  }
  cc[0] = cc[1] = cc[2] = cc[3] = R(0);
  inverse_nonconserved(c, cc, C);
}
template <typename R>
MRTLB_HD void collision(const Coef<R>& c, const R f[16], R dux_dx, R dux_dy,
                                          R duy_dx, R duy_dy, R rho, R inv_rho, R jx, R jy, R e,
                                          R ux, R uy, R T, R C[16]) {
  Harm<R> h;
  harmonics(f, h);
  collision_h(c, h, dux_dx, dux_dy, duy_dx, duy_dy, rho, inv_rho, jx, jy, e, ux, uy, T, C);
}

}  // namespace mrtlb
