/* fdlb_c.c - one time step of the MRT finite-difference lattice Boltzmann
 * model in plain C, FP64 (oracle; TEST INFRASTRUCTURE ONLY).
 *
 * The same method as fdlb.py, written as plain loops for speed on the
 * host: the evolution equation Eq. 3 (Sec. II) with the modified
 * energy-flux relaxation (the two rules after Eq. 16c) on moments 7 and 8,
 * discretised as the amplification matrix G of Sec. III reads: forward
 * Euler in time, per axis a central first difference plus
 * (1/2)(v dt/dx)^2 times the second difference, no x-y cross term:
 *
 *   f^{n+1} = f - sum_a [(v_a dt / 2 d_a)(f(+e_a) - f(-e_a))
 *                        - (1/2)(v_a dt / d_a)^2 (f(+e_a) - 2 f + f(-e_a))] - dt C,
 *   C = M^-1 c,  c_k = s_k (f^_k - f^eq_k) for k >= 5 (1-based), plus the
 *   modification on k = 7, 8 with central differences of the time-n velocity.
 *
 * Equilibria: Eqs. 14a-14i; k = 12, 15, 16 by version (1: zero; 2: the
 * printed polynomials; 3: rows 12, 15, 16 of M applied to
 * rho/(2 pi T) exp(-(v - u)^2 / 2T)).  R = 1 (Sec. IV).
 *
 * Sides (one ghost layer): periodic, zero-gradient outflow (the
 * "extrapolation" of Sec. IV B) and fixed-state inflow (the shock-bubble's
 * post-shock side, Sec. IV B).  Walls and reflecting sides are left to
 * fdlb.py: oracle_step returns -2 for them.
 *
 * M and M^-1 (row-major, 16 x 16) come from the caller (the oracle's exact
 * rationals); the velocity set is Fig. 1's, in the order rows 2-3 of M fix.
 * Arrays are [16][ny][nx], node (i, j) at j * nx + i.  Shares nothing with
 * the CUDA path.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { PERIODIC = 0, OUTFLOW = 1, INFLOW = 3 };

static const double PI = 3.14159265358979323846;

static const int VX[16] = {1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0, 2, -2, -2, 2};
static const int VY[16] = {0, 1, 0, -1, 1, 1, -1, -1, 0, 2, 0, -2, 2, 2, -2, -2};

/* f^eq_hat (16) from the conserved moments (Eqs. 14a-14i and the version rule) */
static void feq_hat(double rho, double jx, double jy, double e, int version, const double *M, double out[16]) {
  const double ux = jx / rho, uy = jy / rho;
  const double T = e / rho - 0.5 * (ux * ux + uy * uy);
  const double jj = jx * jx + jy * jy;
  out[0] = rho;
  out[1] = jx;
  out[2] = jy;
  out[3] = e;
  out[4] = (jx * jx - jy * jy) / rho;                                      /* 14a */
  out[5] = jx * jy / rho;                                                  /* 14b */
  out[6] = (e + rho * T) * jx / rho;                                       /* 14c */
  out[7] = (e + rho * T) * jy / rho;                                       /* 14d */
  out[8] = (jx * jx - 3.0 * jy * jy) * jx / (rho * rho);                   /* 14e */
  out[9] = (3.0 * jx * jx - jy * jy) * jy / (rho * rho);                   /* 14f */
  out[10] = 2.0 * e * e / rho - jj * jj / (4.0 * rho * rho * rho);         /* 14g */
  out[12] = (6.0 * rho * e - 2.0 * jj) * (jx * jx - jy * jy) / (rho * rho * rho); /* 14h */
  out[13] = (6.0 * rho * e - 2.0 * jj) * jx * jy / (rho * rho * rho);      /* 14i */
  if (version == 2) {
    out[11] = 0.0;
    out[14] = rho * ux * (-4.0 + 10.0 * T + 5.0 * ux * ux - 5.0 * uy * uy);
    out[15] = rho * uy * (4.0 - 10.0 * T + 5.0 * ux * ux - 5.0 * uy * uy);
  } else if (version == 3) {
    double fm[16];
    for (int q = 0; q < 16; ++q) {
      const double dx = VX[q] - ux, dy = VY[q] - uy;
      fm[q] = rho / (2.0 * PI * T) * exp(-(dx * dx + dy * dy) / (2.0 * T));
    }
    const int rows[3] = {11, 14, 15};
    for (int r = 0; r < 3; ++r) {
      double acc = 0.0;
      for (int q = 0; q < 16; ++q) acc += M[rows[r] * 16 + q] * fm[q];
      out[rows[r]] = acc;
    }
  } else {
    out[11] = out[14] = out[15] = 0.0;
  }
}

/* f^eq = M^-1 f^eq_hat of a state (rho, u, T) */
static void feq_state(double rho, double ux, double uy, double T, int version, const double *M,
                      const double *Minv, double f[16]) {
  double h[16];
  feq_hat(rho, rho * ux, rho * uy, rho * (T + 0.5 * (ux * ux + uy * uy)), version, M, h);
  for (int q = 0; q < 16; ++q) {
    double acc = 0.0;
    for (int k = 0; k < 16; ++k) acc += Minv[q * 16 + k] * h[k];
    f[q] = acc;
  }
}

/* One step.  kinds[4]: -x, +x, -y, +y; side[4][4]: (ux, uy, T, rho) of an
 * inflow side.  work: at least (16 + 3) (nx + 2)(ny + 2) + 4 nx ny doubles.
 * Returns 0, or -1 for bad arguments, -2 for a side kind not written here. */
int oracle_step(int nx, int ny, double dx, double dy, double dt, const double *s, int version, int modified,
                const int *kinds, const double *side, const double *M, const double *Minv,
                const double *f, double *fout, double *work) {
  if (nx < 1 || ny < 1 || !s || !kinds || !M || !Minv || !f || !fout || !work) return -1;
  for (int a = 0; a < 4; ++a)
    if (kinds[a] != PERIODIC && kinds[a] != OUTFLOW && kinds[a] != INFLOW) return -2;
  if ((kinds[0] == PERIODIC) != (kinds[1] == PERIODIC) || (kinds[2] == PERIODIC) != (kinds[3] == PERIODIC))
    return -1;
  const int NX = nx + 2, NY = ny + 2;
  const long P = (long)NX * NY, n = (long)nx * ny;
  double *g = work;                 /* [16][NY][NX] padded state */
  double *ux = g + 16 * P, *uy = ux + P, *rho_g = uy + P;
  double *grad = rho_g + P;         /* [4][ny][nx]: dux/dx, dux/dy, duy/dx, duy/dy */
  double fin_side[4][16];
  for (int a = 0; a < 4; ++a)
    if (kinds[a] == INFLOW)
      feq_state(side[4 * a + 3], side[4 * a + 0], side[4 * a + 1], side[4 * a + 2], version, M, Minv, fin_side[a]);

  /* ghost layer (Sec. IV sides) */
  for (int q = 0; q < 16; ++q) {
    const double *fq = f + q * n;
    double *gq = g + q * P;
    for (int j = 0; j < ny; ++j) {
      memcpy(gq + (long)(j + 1) * NX + 1, fq + (long)j * nx, sizeof(double) * nx);
      double *row = gq + (long)(j + 1) * NX;
      if (kinds[0] == PERIODIC) {
        row[0] = fq[(long)j * nx + nx - 1];
        row[nx + 1] = fq[(long)j * nx];
      } else {
        row[0] = (kinds[0] == INFLOW) ? fin_side[0][q] : fq[(long)j * nx];
        row[nx + 1] = (kinds[1] == INFLOW) ? fin_side[1][q] : fq[(long)j * nx + nx - 1];
      }
    }
    for (int i = 0; i < nx; ++i) {
      double lo, hi;
      if (kinds[2] == PERIODIC) {
        lo = fq[(long)(ny - 1) * nx + i];
        hi = fq[i];
      } else {
        lo = (kinds[2] == INFLOW) ? fin_side[2][q] : fq[i];
        hi = (kinds[3] == INFLOW) ? fin_side[3][q] : fq[(long)(ny - 1) * nx + i];
      }
      gq[i + 1] = lo;
      gq[(long)(ny + 1) * NX + i + 1] = hi;
    }
    /* corners: not on the cross stencil; kept finite */
    gq[0] = gq[NX + 1];
    gq[NX - 1] = gq[NX + NX - 2];
    gq[(long)(NY - 1) * NX] = gq[(long)(NY - 2) * NX + 1];
    gq[(long)NY * NX - 1] = gq[(long)(NY - 1) * NX - 2];
  }

  /* velocity (and density) on the padded grid: rows 1-3 of M (Sec. II) */
  for (long t = 0; t < P; ++t) {
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int q = 0; q < 16; ++q) {
      const double v = g[q * P + t];
      r += M[0 * 16 + q] * v;
      jx += M[1 * 16 + q] * v;
      jy += M[2 * 16 + q] * v;
    }
    rho_g[t] = r;
    ux[t] = jx / r;
    uy[t] = jy / r;
  }
  /* second-order central differences of u at the interior nodes */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const long c = (long)(j + 1) * NX + i + 1, t = (long)j * nx + i;
      grad[0 * n + t] = (ux[c + 1] - ux[c - 1]) / (2.0 * dx);
      grad[1 * n + t] = (ux[c + NX] - ux[c - NX]) / (2.0 * dy);
      grad[2 * n + t] = (uy[c + 1] - uy[c - 1]) / (2.0 * dx);
      grad[3 * n + t] = (uy[c + NX] - uy[c - NX]) / (2.0 * dy);
    }

  /* collision, advection and the update, node by node */
  double a_x[16], b_x[16], a_y[16], b_y[16];
  for (int q = 0; q < 16; ++q) {
    a_x[q] = VX[q] * dt / (2.0 * dx);
    b_x[q] = 0.5 * (VX[q] * dt / dx) * (VX[q] * dt / dx);
    a_y[q] = VY[q] * dt / (2.0 * dy);
    b_y[q] = 0.5 * (VY[q] * dt / dy) * (VY[q] * dt / dy);
  }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const long c = (long)(j + 1) * NX + i + 1, t = (long)j * nx + i;
      double fl[16], fh[16], eq[16], cc[16];
      for (int q = 0; q < 16; ++q) fl[q] = g[q * P + c];
      for (int k = 0; k < 16; ++k) {
        double acc = 0.0;
        for (int q = 0; q < 16; ++q) acc += M[k * 16 + q] * fl[q];
        fh[k] = acc;
      }
      feq_hat(fh[0], fh[1], fh[2], fh[3], version, M, eq);
      for (int k = 0; k < 16; ++k) cc[k] = (k >= 4) ? s[k] * (fh[k] - eq[k]) : 0.0;
      if (modified) {
        const double r = fh[0], vx = fh[1] / r, vy = fh[2] / r;
        const double T = fh[3] / r - 0.5 * (vx * vx + vy * vy);
        const double rT = r * T;
        const double shear = grad[0 * n + t] - grad[3 * n + t];  /* dux/dx - duy/dy */
        const double strain = grad[2 * n + t] + grad[1 * n + t]; /* duy/dx + dux/dy */
        cc[6] += (s[6] / s[4] - 1.0) * rT * vx * shear + (s[6] / s[5] - 1.0) * rT * vy * strain;
        cc[7] += (s[7] / s[5] - 1.0) * rT * vx * strain + (s[7] / s[4] - 1.0) * rT * vy * shear;
      }
      for (int q = 0; q < 16; ++q) {
        double C = 0.0;
        for (int k = 0; k < 16; ++k) C += Minv[q * 16 + k] * cc[k];
        const double *gq = g + q * P;
        const double f0 = gq[c];
        double A = 0.0;
        if (VX[q] != 0) A += a_x[q] * (gq[c + 1] - gq[c - 1]) - b_x[q] * (gq[c + 1] - 2.0 * f0 + gq[c - 1]);
        if (VY[q] != 0) A += a_y[q] * (gq[c + NX] - gq[c - NX]) - b_y[q] * (gq[c + NX] - 2.0 * f0 + gq[c - NX]);
        fout[q * n + t] = f0 - A - dt * C;
      }
    }
  return 0;
}

/* nsteps steps from f (in place); work as for oracle_step plus 16 nx ny doubles */
int oracle_run(int nx, int ny, double dx, double dy, double dt, const double *s, int version, int modified,
               const int *kinds, const double *side, const double *M, const double *Minv, double *f,
               long nsteps, double *work) {
  const long n = (long)nx * ny;
  double *tmp = work;
  double *w = work + 16 * n;
  for (long k = 0; k < nsteps; ++k) {
    const int rc = oracle_step(nx, ny, dx, dy, dt, s, version, modified, kinds, side, M, Minv, f, tmp, w);
    if (rc) return rc;
    memcpy(f, tmp, sizeof(double) * 16 * n);
  }
  return 0;
}
