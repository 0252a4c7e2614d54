// mrtlb.cu - host side of the C ABI (see include/mrtlb.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "../../include/mrtlb.h"
#include "ctx.h"

using namespace mrtlb;

namespace {

thread_local std::string g_create_error;

// Exact rational arithmetic for the small family inverses (entries of M are
// dyadic rationals, so every intermediate stays small).
struct Frac {
  long long n = 0, d = 1;
  static long long gcd(long long a, long long b) {
    a = a < 0 ? -a : a;
    b = b < 0 ? -b : b;
    while (b) { long long t = a % b; a = b; b = t; }
    return a ? a : 1;
  }
  static Frac make(long long n, long long d) {
    if (d < 0) { n = -n; d = -d; }
    const long long g = gcd(n, d);
    return Frac{n / g, d / g};
  }
  static Frac from_dyadic(double x) {  // exact for dyadic rationals
    long long d = 1;
    while (std::floor(x * d) != x * d && d < (1LL << 40)) d *= 2;
    return make((long long)std::llround(x * d), d);
  }
  Frac operator+(const Frac& o) const { return make(n * o.d + o.n * d, d * o.d); }
  Frac operator-(const Frac& o) const { return make(n * o.d - o.n * d, d * o.d); }
  Frac operator*(const Frac& o) const { return make(n * o.n, d * o.d); }
  Frac operator/(const Frac& o) const { return make(n * o.d, d * o.n); }
  bool zero() const { return n == 0; }
  double val() const { return (double)n / (double)d; }
};

// Gauss-Jordan inverse of an n x n (n <= 4) exact matrix; false if singular.
bool invert(int n, Frac a[4][4], Frac inv[4][4]) {
  Frac m[4][8];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j)
      m[i][j] = (j < n) ? a[i][j] : Frac::make(j - n == i ? 1 : 0, 1);
  for (int col = 0; col < n; ++col) {
    int piv = -1;
    for (int r = col; r < n; ++r)
      if (!m[r][col].zero()) { piv = r; break; }
    if (piv < 0) return false;
    for (int j = 0; j < 2 * n; ++j) { Frac t = m[col][j]; m[col][j] = m[piv][j]; m[piv][j] = t; }
    const Frac p = m[col][col];
    for (int j = 0; j < 2 * n; ++j) m[col][j] = m[col][j] / p;
    for (int r = 0; r < n; ++r) {
      if (r == col || m[r][col].zero()) continue;
      const Frac fac = m[r][col];
      for (int j = 0; j < 2 * n; ++j) m[r][j] = m[r][j] - fac * m[col][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) inv[i][j] = m[i][n + j];
  return true;
}

// Moment rows (0-based k) of each harmonic family and the shells it lives on.
const int kRowsS[4] = {0, 3, 10, 11};
const int kRowsX[4] = {1, 6, 8, 14};
const int kRowsY[4] = {2, 7, 9, 15};
const int kRowsQ[2] = {4, 12};
const int kRowsP[2] = {5, 13};

// Column of the family matrix: the moments of a unit harmonic on one shell,
// taken from the same moments() the kernels use.
void unit_moments(char fam, int shell, double m[16]) {
  Harm<double> h;
  std::memset(&h, 0, sizeof(h));
  if (fam == 'S') h.S[shell] = 1;
  if (fam == 'X') h.X[shell] = 1;
  if (fam == 'Y') h.Y[shell] = 1;
  if (fam == 'Q') h.Q[shell] = 1;
  if (fam == 'P') h.P[shell] = 1;
  moments(h, m);
}

}  // namespace




static int fail(mrtlb_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->last_error = buf;
  else g_create_error = buf;
  return code;
}

static void drop_graphs(mrtlb_ctx* c);

static int cuda_fail(mrtlb_ctx* c, cudaError_t e, const char* what) {
  return fail(c, MRTLB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

// Round the four Lax-Wendroff weights of one velocity to multiples of a
// power of two G >= 2^-mbits sum|k| (so that every weight and any partial
// sum fits an mbits+1-bit significand) and return their sum, which is then
// exact in that precision.  The change to each weight is at most G/2.
static void on_common_grid(double k[4], int mbits, double* sum) {
  double a = 0.0;
  for (int i = 0; i < 4; ++i) a += std::fabs(k[i]);
  *sum = 0.0;
  if (a == 0.0) return;
  const double G = std::ldexp(1.0, (int)std::ceil(std::log2(a)) - mbits);
  for (int i = 0; i < 4; ++i) {
    k[i] = std::nearbyint(k[i] / G) * G;
    *sum += k[i];
  }
}

static int build_coefficients(mrtlb_ctx* c) {
  const mrtlb_params& p = c->p;
  Coef<double>& k = c->c64;
  std::memset(&k, 0, sizeof(k));
  k.a1x = p.dt / (2.0 * p.dx);
  k.b1x = 0.5 * (p.dt / p.dx) * (p.dt / p.dx);
  k.a1y = p.dt / (2.0 * p.dy);
  k.b1y = 0.5 * (p.dt / p.dy) * (p.dt / p.dy);
  k.inv2dx = 1.0 / (2.0 * p.dx);
  k.inv2dy = 1.0 / (2.0 * p.dy);
  for (int q = 0; q < 16; ++q) {
    const double ax = vx_of(q) * k.a1x, bx = vx_of(q) * vx_of(q) * k.b1x;
    const double ay = vy_of(q) * k.a1y, by = vy_of(q) * vy_of(q) * k.b1y;
    k.lw[q][0] = bx - ax;  // east  (x + dx)
    k.lw[q][1] = bx + ax;  // west  (x - dx)
    k.lw[q][2] = by - ay;  // north (y + dy)
    k.lw[q][3] = by + ay;  // south (y - dy)
    on_common_grid(k.lw[q], 52, &k.lwsum[q]);
  }
  for (int q = 0; q < 16; ++q) k.rate[q] = (q >= 4) ? p.dt * c->s[q] : 0.0;
  if (p.modified) {
    const double s5 = c->s[4], s6 = c->s[5], s7 = c->s[6], s8 = c->s[7];
    k.mod[0] = p.dt * (s7 / s5 - 1.0);
    k.mod[1] = p.dt * (s7 / s6 - 1.0);
    k.mod[2] = p.dt * (s8 / s6 - 1.0);
    k.mod[3] = p.dt * (s8 / s5 - 1.0);
  }
  k.version = p.eq_version;
  k.modified = p.modified ? 1 : 0;

  // family matrices F[row][shell] and their exact inverses
  struct Fam { char name; int n; const int* rows; int shells[4]; };
  const Fam fams[5] = {{'S', 4, kRowsS, {0, 1, 2, 3}}, {'X', 4, kRowsX, {0, 1, 2, 3}},
                       {'Y', 4, kRowsY, {0, 1, 2, 3}}, {'Q', 2, kRowsQ, {0, 2, 0, 0}},
                       {'P', 2, kRowsP, {1, 3, 0, 0}}};
  for (const Fam& fm : fams) {
    Frac F[4][4], Fi[4][4];
    for (int col = 0; col < fm.n; ++col) {
      double m[16];
      unit_moments(fm.name, col, m);
      for (int r = 0; r < fm.n; ++r) F[r][col] = Frac::from_dyadic(m[fm.rows[r]]);
    }
    if (!invert(fm.n, F, Fi)) return fail(c, MRTLB_ERR_SINGULAR, "family %c of M is singular", fm.name);
    for (int sh = 0; sh < fm.n; ++sh) {
      const int shell = fm.shells[sh];
      const bool axis = (shell == 0 || shell == 2);
      double scale = 0.25;
      if (axis && (fm.name == 'X' || fm.name == 'Y')) scale = 0.5;
      for (int r = 0; r < fm.n; ++r) {
        const double v = scale * Fi[sh][r].val();
        if (fm.name == 'S') k.invS[sh][r] = v;
        if (fm.name == 'X') k.invX[sh][r] = v;
        if (fm.name == 'Y') k.invY[sh][r] = v;
        if (fm.name == 'Q') k.invQ[sh][r] = v;
        if (fm.name == 'P') k.invP[sh][r] = v;
      }
    }
  }
  // self-check: the factorised M^-1 M is the identity
  for (int q = 0; q < 16; ++q) {
    double e[16] = {0}, m[16], back[16];
    e[q] = 1.0;
    Harm<double> h;
    harmonics(e, h);
    moments(h, m);
    inverse_full(k, m, back);
    for (int r = 0; r < 16; ++r)
      if (std::fabs(back[r] - (r == q ? 1.0 : 0.0)) > 1e-14)
        return fail(c, MRTLB_ERR_SINGULAR, "factorised inverse of M failed its check");
  }
  // FP32 copy
  Coef<float>& f = c->c32;
  f.a1x = (float)k.a1x; f.b1x = (float)k.b1x; f.a1y = (float)k.a1y; f.b1y = (float)k.b1y;
  f.inv2dx = (float)k.inv2dx; f.inv2dy = (float)k.inv2dy;
  for (int q = 0; q < 16; ++q) {
    double w[4] = {k.lw[q][0], k.lw[q][1], k.lw[q][2], k.lw[q][3]}, sum;
    on_common_grid(w, 23, &sum);
    for (int a = 0; a < 4; ++a) f.lw[q][a] = (float)w[a];
    f.lwsum[q] = (float)sum;
  }
  for (int q = 0; q < 16; ++q) f.rate[q] = (float)k.rate[q];
  for (int q = 0; q < 4; ++q) f.mod[q] = (float)k.mod[q];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      f.invS[a][b] = (float)k.invS[a][b];
      f.invX[a][b] = (float)k.invX[a][b];
      f.invY[a][b] = (float)k.invY[a][b];
    }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      f.invQ[a][b] = (float)k.invQ[a][b];
      f.invP[a][b] = (float)k.invP[a][b];
    }
  f.version = k.version;
  f.modified = k.modified;
  return MRTLB_OK;
}

extern "C" int mrtlb_create(const mrtlb_params* params, mrtlb_ctx** out) {
  mrtlb_ctx* c = nullptr;
  g_create_error.clear();
  if (!out) return fail(nullptr, MRTLB_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!params) return fail(nullptr, MRTLB_ERR_ARG, "params is NULL");
  const mrtlb_params& p = *params;
  if (p.nvel != 16) return fail(nullptr, MRTLB_ERR_UNSUPPORTED, "nvel = %d; only the 16-velocity set of the paper is supported", p.nvel);
  if (!p.v || !p.M) return fail(nullptr, MRTLB_ERR_ARG, "v and M are required");
  for (int q = 0; q < 16; ++q)
    if (p.v[2 * q] != (double)vx_of(q) || p.v[2 * q + 1] != (double)vy_of(q))
      return fail(nullptr, MRTLB_ERR_UNSUPPORTED, "velocity %d is not the paper's D2V16 velocity", q + 1);
  for (int q = 0; q < 16; ++q) {
    double e[16] = {0}, m[16];
    e[q] = 1.0;
    Harm<double> h;
    harmonics(e, h);
    moments(h, m);
    for (int k = 0; k < 16; ++k)
      if (p.M[k * 16 + q] != m[k])
        return fail(nullptr, MRTLB_ERR_UNSUPPORTED, "M[%d][%d] = %g differs from the paper's %g", k + 1, q + 1, p.M[k * 16 + q], m[k]);
  }
  if (p.nx < 1 || p.ny < 1 || p.ny > 65535)
    return fail(nullptr, MRTLB_ERR_ARG, "grid %d x %d (need nx >= 1, 1 <= ny <= 65535)", p.nx, p.ny);
  if (!(p.dx > 0) || !(p.dy > 0) || !(p.dt > 0)) return fail(nullptr, MRTLB_ERR_ARG, "dx, dy, dt must be positive");
  if (p.eq_version < 1 || p.eq_version > 3) return fail(nullptr, MRTLB_ERR_ARG, "eq_version %d", p.eq_version);
  if (p.precision != MRTLB_FP32 && p.precision != MRTLB_FP64) return fail(nullptr, MRTLB_ERR_ARG, "precision %d", p.precision);
  for (int s = 0; s < 4; ++s)
    if (p.bc[s].kind < 0 || p.bc[s].kind > 5) return fail(nullptr, MRTLB_ERR_ARG, "bc[%d].kind = %d", s, p.bc[s].kind);
  for (int a = 0; a < 2; ++a) {
    const int k0 = p.bc[2 * a].kind, k1 = p.bc[2 * a + 1].kind;
    if ((k0 == MRTLB_BC_PERIODIC) != (k1 == MRTLB_BC_PERIODIC))
      return fail(nullptr, MRTLB_ERR_ARG, "periodic sides must come in pairs");
  }
  const bool xwall = p.bc[0].kind == MRTLB_BC_WALL_NEE || p.bc[1].kind == MRTLB_BC_WALL_NEE;
  const bool ywall = p.bc[2].kind == MRTLB_BC_WALL_NEE || p.bc[3].kind == MRTLB_BC_WALL_NEE;
  if (xwall && ywall) return fail(nullptr, MRTLB_ERR_UNSUPPORTED, "walls on one axis only");
  if (xwall && p.nx < 3) return fail(nullptr, MRTLB_ERR_ARG, "walls along x need nx >= 3");
  if (ywall && p.ny < 3) return fail(nullptr, MRTLB_ERR_ARG, "walls along y need ny >= 3");
  for (int s = 0; s < 4; ++s) {
    if (p.bc[s].kind == MRTLB_BC_WALL_NEE && !(p.bc[s].T > 0))
      return fail(nullptr, MRTLB_ERR_ARG, "wall temperature on side %d must be positive", s);
    if (p.bc[s].kind == MRTLB_BC_DIFFUSE && !(p.bc[s].T > 0))
      return fail(nullptr, MRTLB_ERR_ARG, "diffuse wall temperature on side %d must be positive", s);
    if (p.bc[s].kind == MRTLB_BC_INFLOW && (!(p.bc[s].T > 0) || !(p.bc[s].rho > 0)))
      return fail(nullptr, MRTLB_ERR_ARG, "inflow density and temperature on side %d must be positive", s);
  }
  // Lax-Wendroff stability: Courant number of the fastest axis speed (2)
  const double cfl = 2.0 * p.dt / (p.dx < p.dy ? p.dx : p.dy);
  if (cfl > 1.0) return fail(nullptr, MRTLB_ERR_ARG, "CFL number 2 dt / min(dx, dy) = %g exceeds 1", cfl);

  c = new mrtlb_ctx();
  c->p = p;
  c->p.v = nullptr;
  c->p.M = nullptr;
  c->p.s = nullptr;
  if (p.s) {
    for (int q = 0; q < 16; ++q) c->s[q] = p.s[q];
  } else {
    for (int q = 0; q < 16; ++q) c->s[q] = p.s_other;
    c->s[4] = c->s[5] = p.s_visc;
    c->s[6] = c->s[7] = p.Pr * p.s_visc;
  }
  for (int q = 4; q < 16; ++q) {
    if (!(c->s[q] >= 0) || c->s[q] * p.dt > 2.0) {
      const double sv = c->s[q];
      delete c;
      return fail(nullptr, MRTLB_ERR_ARG, "s_%d = %g: need 0 <= s dt <= 2 (forward-Euler relaxation limit)", q + 1, sv);
    }
  }
  if (p.modified && (!(c->s[4] > 0) || !(c->s[5] > 0))) {
    delete c;
    return fail(nullptr, MRTLB_ERR_ARG, "the modified collision needs s5, s6 > 0");
  }
  c->prec = p.precision;
  c->esize = (p.precision == MRTLB_FP64) ? 8 : 4;
  c->stream = (cudaStream_t)p.stream;
  Layout& L = c->L;
  L.nx = p.nx;
  L.ny = p.ny;
  L.xoff = (int)(128 / c->esize);
  const int align = (int)(128 / c->esize);
  L.pitch = ((L.xoff + p.nx + 4 + align - 1) / align) * align;
  L.plane = (long long)(p.ny + 2) * L.pitch;
  for (int s = 0; s < 4; ++s) L.bc[s] = p.bc[s].kind;
  L.i0 = (p.bc[0].kind == MRTLB_BC_WALL_NEE) ? 1 : 0;
  L.i1 = p.nx - ((p.bc[1].kind == MRTLB_BC_WALL_NEE) ? 1 : 0);
  L.j0 = (p.bc[2].kind == MRTLB_BC_WALL_NEE) ? 1 : 0;
  L.j1 = p.ny - ((p.bc[3].kind == MRTLB_BC_WALL_NEE) ? 1 : 0);
  for (int s = 0; s < 4; ++s) {
    c->walls.ux[s] = p.bc[s].ux;
    c->walls.uy[s] = p.bc[s].uy;
    c->walls.T[s] = p.bc[s].T;
    c->walls.rho[s] = p.bc[s].rho;
  }
  c->state_bytes = (size_t)16 * (size_t)L.plane * c->esize;
  const int rc = build_coefficients(c);
  if (rc != MRTLB_OK) {
    g_create_error = c->last_error;
    delete c;
    return rc;
  }
  *out = c;
  return MRTLB_OK;
}

extern "C" int mrtlb_state_bytes(const mrtlb_ctx* c, size_t* bytes) {
  if (!c || !bytes) return MRTLB_ERR_ARG;
  *bytes = c->state_bytes;
  return MRTLB_OK;
}

static int ensure_scratch(mrtlb_ctx* c) {
  if (!c->err) {
    CK(cudaMalloc((void**)&c->err, 256), "cudaMalloc(error word)");
    CK(cudaMemsetAsync(c->err, 0, 256, c->stream), "cudaMemsetAsync");
  }
  if (!c->acc) CK(cudaMalloc((void**)&c->acc, 8 * sizeof(double)), "cudaMalloc(accumulators)");
  return MRTLB_OK;
}

// The device address of a host buffer the GPU reaches directly (page-locked
// memory mapped into the device's address space), else null: such buffers
// are read or written by the kernels themselves over the host link, with
// no staging copy.
static void* mapped_host(const void* host) {
  cudaPointerAttributes a;
  if (!host || cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost) ? a.devicePointer : nullptr;
}

static int ensure_staging(mrtlb_ctx* c, size_t bytes) {
  if (c->staging_bytes >= bytes) return MRTLB_OK;
  if (c->staging) {
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    cudaFree(c->staging);
    c->staging = nullptr;
    c->staging_bytes = 0;
  }
  CK(cudaMalloc(&c->staging, bytes), "cudaMalloc(staging)");
  c->staging_bytes = bytes;
  return MRTLB_OK;
}

extern "C" int mrtlb_bind(mrtlb_ctx* c, void* f_a, void* f_b, size_t bytes) {
  if (!c) return MRTLB_ERR_ARG;
  if (!f_a || !f_b || f_a == f_b) return fail(c, MRTLB_ERR_ARG, "two distinct state buffers are required");
  if (bytes < c->state_bytes) return fail(c, MRTLB_ERR_ARG, "state buffer of %zu bytes, need %zu", bytes, c->state_bytes);
  if (((uintptr_t)f_a & 255) || ((uintptr_t)f_b & 255)) return fail(c, MRTLB_ERR_ARG, "state buffers must be 256-byte aligned");
  c->f[0] = f_a;
  c->f[1] = f_b;
  c->cur = 0;
  ++c->gen;
  c->steps = 0;
  c->have_prev = 0;
  int rc = ensure_scratch(c);
  if (rc) return rc;
  CK(cudaMemsetAsync(f_a, 0, c->state_bytes, c->stream), "cudaMemsetAsync");
  CK(cudaMemsetAsync(f_b, 0, c->state_bytes, c->stream), "cudaMemsetAsync");
  drop_graphs(c);
  rc = plan_tiled(c->L, (int)c->esize, c->f[0], c->f[1], &c->plan);
  if (rc) return fail(c, MRTLB_ERR_CUDA, "tensor-map set-up failed (%d)", rc);
  return MRTLB_OK;
}

static bool bound(mrtlb_ctx* c) { return c && c->f[0] && c->f[1]; }

// The boundary fill of f; the fixed inflow ghosts go into both state
// buffers, since a step writes every other ghost of its output itself.
static void enqueue_bc(mrtlb_ctx* c, void* f) {
  TraceRange trace_("bc_fill");
  if (c->prec == MRTLB_FP64) launch_bc<double>((double*)f, c->L, c->c64, c->walls, c->stream);
  else launch_bc<float>((float*)f, c->L, c->c32, c->walls, c->stream);
  for (int b = 0; b < 2; ++b) {
    if (!c->f[b] || c->f[b] == f) continue;
    if (c->prec == MRTLB_FP64) launch_inflow<double>((double*)c->f[b], c->L, c->c64, c->walls, c->stream);
    else launch_inflow<float>((float*)c->f[b], c->L, c->c32, c->walls, c->stream);
  }
}

static int check_launch(mrtlb_ctx* c, const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  return MRTLB_OK;
}

extern "C" int mrtlb_init_equilibrium(mrtlb_ctx* c, const double* rho, const double* ux,
                                      const double* uy, const double* T, int on_device) {
  if (!bound(c)) return c ? fail(c, MRTLB_ERR_STATE, "bind state buffers first") : MRTLB_ERR_ARG;
  if (!rho || !ux || !uy || !T) return fail(c, MRTLB_ERR_ARG, "all four fields are required");
  const size_t n = (size_t)c->L.nx * c->L.ny;
  const double *r = rho, *a = ux, *b = uy, *t = T;
  if (!on_device) {
    int rc = ensure_staging(c, 4 * n * sizeof(double));
    if (rc) return rc;
    double* s = (double*)c->staging;
    CK(cudaMemcpyAsync(s, rho, n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy rho");
    CK(cudaMemcpyAsync(s + n, ux, n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy ux");
    CK(cudaMemcpyAsync(s + 2 * n, uy, n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy uy");
    CK(cudaMemcpyAsync(s + 3 * n, T, n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy T");
    r = s; a = s + n; b = s + 2 * n; t = s + 3 * n;
  }
  c->cur = 0;
  ++c->gen;
  CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), "clear error word");  // a new run
  if (c->prec == MRTLB_FP64) launch_init_eq<double>(r, a, b, t, (double*)c->f[0], c->L, c->c64, c->stream);
  else launch_init_eq<float>(r, a, b, t, (float*)c->f[0], c->L, c->c64, c->stream);
  enqueue_bc(c, c->f[0]);
  c->steps = 0;
  c->have_prev = 0;
  if (!on_device) CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return check_launch(c, "init_equilibrium");
}

// one step reading buffer `cur` (walls refilled, then the step kernel)
static void enqueue_one(mrtlb_ctx* c, int cur, cudaStream_t st, bool timed) {
  const bool tiled = use_tiled(c->kernel, c->plan, c->prec == MRTLB_FP64);
  void* fin = c->f[cur];
  void* fout = c->f[cur ^ 1];
  // (ghosts of fin were written through by the previous step)
  if (c->prec == MRTLB_FP64) launch_walls<double>((double*)fin, c->L, c->c64, c->walls, st);
  else launch_walls<float>((float*)fin, c->L, c->c32, c->walls, st);
  if (timed) cudaEventRecord(c->ev[2 * c->ev_used], st);
  if (c->prec == MRTLB_FP64) {
    if (tiled) launch_step_tiled<double>(c->plan, cur, c->L, c->c64, c->err, st, fout);
    else launch_step_plain<double>((const double*)fin, (double*)fout, c->L, c->c64, c->err, st);
  } else {
    if (tiled) launch_step_tiled<float>(c->plan, cur, c->L, c->c32, c->err, st, fout);
    else launch_step_plain<float>((const float*)fin, (float*)fout, c->L, c->c32, c->err, st);
  }
  if (timed) {
    cudaEventRecord(c->ev[2 * c->ev_used + 1], st);
    ++c->ev_used;
  }
}

static void drop_graphs(mrtlb_ctx* c) {
  for (int p = 0; p < 2; ++p)
    if (c->graph[p]) {
      cudaGraphExecDestroy(c->graph[p]);
      c->graph[p] = nullptr;
    }
}

// capture graph_steps steps starting at parity p; false if capture is not possible
static bool ensure_graph(mrtlb_ctx* c, int p) {
  if (c->graph[p]) return true;
  if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) return false;
  if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  int cur = p;
  for (int k = 0; k < c->graph_steps; ++k) {
    enqueue_one(c, cur, c->cap, false);
    cur ^= 1;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(c->cap, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return false;
  }
  const bool ok = cudaGraphInstantiate(&c->graph[p], g, 0) == cudaSuccess;
  cudaGraphDestroy(g);
  if (!ok) {
    c->graph[p] = nullptr;
    cudaGetLastError();
  }
  return ok;
}

static int enqueue_steps(mrtlb_ctx* c, long nsteps) {
  long n = 0;
  // runs of graph_steps steps replay as CUDA graphs (not while timing kernels)
  while (!c->timing && c->graph_steps > 0 && nsteps - n >= c->graph_steps && ensure_graph(c, c->cur)) {
    const cudaError_t e = cudaGraphLaunch(c->graph[c->cur], c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
    n += c->graph_steps;
    if (c->graph_steps & 1) c->cur ^= 1;
  }
  for (; n < nsteps; ++n) {
    enqueue_one(c, c->cur, c->stream, c->timing && c->ev_used < c->ev_cap);
    c->cur ^= 1;
  }
  c->steps += nsteps;
  if (nsteps > 0) ++c->gen;
  return check_launch(c, "step");
}

extern "C" int mrtlb_step(mrtlb_ctx* c, long nsteps) {
  TraceRange trace_("mrtlb_step");
  if (!bound(c)) return c ? fail(c, MRTLB_ERR_STATE, "bind state buffers first") : MRTLB_ERR_ARG;
  if (nsteps < 0) return fail(c, MRTLB_ERR_ARG, "nsteps < 0");
  return enqueue_steps(c, nsteps);
}

static int sync_and_check(mrtlb_ctx* c) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read error word");
  CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (h & ERRBIT_TIMEOUT) return fail(c, MRTLB_ERR_TIMEOUT, "a bounded device-side wait gave up");
  if (h & ERRBIT_NONPHYSICAL)
    return fail(c, MRTLB_ERR_NONPHYSICAL, "non-physical state (rho <= 0, T <= 0 or non-finite) met by a step");
  return MRTLB_OK;
}

extern "C" int mrtlb_sync(mrtlb_ctx* c) {
  if (!bound(c)) return c ? fail(c, MRTLB_ERR_STATE, "bind state buffers first") : MRTLB_ERR_ARG;
  return sync_and_check(c);
}

extern "C" int mrtlb_selftest_wait(mrtlb_ctx* c) {
  if (!bound(c)) return c ? fail(c, MRTLB_ERR_STATE, "bind state buffers first") : MRTLB_ERR_ARG;
  int rc = sync_and_check(c);
  if (rc) return rc;  // an error from earlier work comes first
  launch_wait_selftest(c->err, c->stream);
  rc = check_launch(c, "wait self-test");
  if (rc) return rc;
  rc = sync_and_check(c);
  CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), "clear error word");
  CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return rc;
}

extern "C" int mrtlb_macros(mrtlb_ctx* c, double* rho, double* ux, double* uy, double* T, int on_device) {
  TraceRange trace_("mrtlb_macros");
  if (!bound(c)) return c ? fail(c, MRTLB_ERR_STATE, "bind state buffers first") : MRTLB_ERR_ARG;
  const size_t n = (size_t)c->L.nx * c->L.ny;
  void* f = c->f[c->cur];
  enqueue_bc(c, f);  // wall nodes follow the current neighbours
  double* d[4] = {rho, ux, uy, T};
  double* dd[4] = {rho, ux, uy, T};
  bool direct = !on_device;
  if (!on_device) {
    for (int k = 0; k < 4; ++k)
      if (d[k] && !(dd[k] = (double*)mapped_host(d[k]))) direct = false;
  }
  if (!on_device && !direct) {
    int rc = ensure_staging(c, 4 * n * sizeof(double));
    if (rc) return rc;
    for (int k = 0; k < 4; ++k) dd[k] = d[k] ? (double*)c->staging + k * n : nullptr;
  }
  if (c->prec == MRTLB_FP64) launch_macros<double>((const double*)f, dd[0], dd[1], dd[2], dd[3], c->L, c->stream);
  else launch_macros<float>((const float*)f, dd[0], dd[1], dd[2], dd[3], c->L, c->stream);
  int rc = check_launch(c, "macros");
  if (rc) return rc;
  if (!on_device && !direct)
    for (int k = 0; k < 4; ++k)
      if (d[k]) CK(cudaMemcpyAsync(d[k], dd[k], n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy macros");
  return sync_and_check(c);
}

extern "C" int mrtlb_reduce(mrtlb_ctx* c, double out[5]) {
  TraceRange trace_("mrtlb_reduce");
  if (!bound(c)) return c ? fail(c, MRTLB_ERR_STATE, "bind state buffers first") : MRTLB_ERR_ARG;
  if (!out) return fail(c, MRTLB_ERR_ARG, "out is NULL");
  const size_t n = (size_t)c->L.nx * c->L.ny;
  if (!c->Tprev) CK(cudaMalloc((void**)&c->Tprev, n * sizeof(double)), "cudaMalloc(Tprev)");
  void* f = c->f[c->cur];
  enqueue_bc(c, f);
  CK(cudaMemsetAsync(c->acc, 0, 5 * sizeof(double), c->stream), "cudaMemsetAsync");
  if (c->prec == MRTLB_FP64) launch_reduce<double>((const double*)f, c->acc, c->Tprev, c->have_prev, c->L, c->stream);
  else launch_reduce<float>((const float*)f, c->acc, c->Tprev, c->have_prev, c->L, c->stream);
  int rc = check_launch(c, "reduce");
  if (rc) return rc;
  CK(cudaMemcpyAsync(out, c->acc, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy sums");
  rc = sync_and_check(c);
  // T_prev holds this call's temperatures unless the device work itself
  // failed (a latched non-physical state or expired wait still let it run)
  c->have_prev = (rc == MRTLB_OK || rc == MRTLB_ERR_NONPHYSICAL || rc == MRTLB_ERR_TIMEOUT) ? 1 : 0;
  return rc;
}

extern "C" int mrtlb_get_f(mrtlb_ctx* c, void* f, int on_device) {
  TraceRange trace_("mrtlb_get_f");
  if (!bound(c)) return c ? fail(c, MRTLB_ERR_STATE, "bind state buffers first") : MRTLB_ERR_ARG;
  if (!f) return fail(c, MRTLB_ERR_ARG, "f is NULL");
  const size_t bytes = (size_t)16 * c->L.nx * c->L.ny * c->esize;
  void* cur = c->f[c->cur];
  enqueue_bc(c, cur);
  void* dst = f;
  void* direct = on_device ? nullptr : mapped_host(f);
  if (direct) {
    dst = direct;
  } else if (!on_device) {
    int rc = ensure_staging(c, bytes);
    if (rc) return rc;
    dst = c->staging;
  }
  if (c->prec == MRTLB_FP64) launch_unpack<double>((const double*)cur, (double*)dst, c->L, c->stream);
  else launch_unpack<float>((const float*)cur, (float*)dst, c->L, c->stream);
  int rc = check_launch(c, "get_f");
  if (rc) return rc;
  if (!on_device && !direct) CK(cudaMemcpyAsync(f, dst, bytes, cudaMemcpyDeviceToHost, c->stream), "copy f");
  return sync_and_check(c);
}

extern "C" int mrtlb_set_f(mrtlb_ctx* c, const void* f, int on_device) {
  TraceRange trace_("mrtlb_set_f");
  if (!bound(c)) return c ? fail(c, MRTLB_ERR_STATE, "bind state buffers first") : MRTLB_ERR_ARG;
  if (!f) return fail(c, MRTLB_ERR_ARG, "f is NULL");
  const size_t bytes = (size_t)16 * c->L.nx * c->L.ny * c->esize;
  const void* src = f;
  const void* direct = on_device ? nullptr : mapped_host(f);
  if (direct) {
    src = direct;
  } else if (!on_device) {
    int rc = ensure_staging(c, bytes);
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->staging, f, bytes, cudaMemcpyHostToDevice, c->stream), "copy f");
    src = c->staging;
  }
  c->cur = 0;
  ++c->gen;
  CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), "clear error word");  // a new run
  if (c->prec == MRTLB_FP64) launch_pack<double>((const double*)src, (double*)c->f[0], c->L, c->stream);
  else launch_pack<float>((const float*)src, (float*)c->f[0], c->L, c->stream);
  enqueue_bc(c, c->f[0]);
  c->steps = 0;
  c->have_prev = 0;
  if (!on_device) CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return check_launch(c, "set_f");
}

extern "C" long mrtlb_step_count(const mrtlb_ctx* c) { return c ? c->steps : -1; }

extern "C" int mrtlb_set_rates(mrtlb_ctx* c, const double* s) {
  if (!c || !s) return MRTLB_ERR_ARG;
  for (int q = 4; q < 16; ++q)
    if (!(s[q] >= 0) || s[q] * c->p.dt > 2.0)
      return fail(c, MRTLB_ERR_ARG, "s_%d = %g: need 0 <= s dt <= 2", q + 1, s[q]);
  if (c->p.modified && (!(s[4] > 0) || !(s[5] > 0)))
    return fail(c, MRTLB_ERR_ARG, "the modified collision needs s5, s6 > 0");
  if (c->f[0]) {
    const cudaError_t e = cudaStreamSynchronize(c->stream);  // queued steps use the old rates
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  }
  for (int q = 0; q < 16; ++q) c->s[q] = s[q];
  ++c->gen;
  drop_graphs(c);  // captured launches hold the old coefficients
  return build_coefficients(c);
}

extern "C" int mrtlb_get_rates(const mrtlb_ctx* c, double* s) {
  if (!c || !s) return MRTLB_ERR_ARG;
  for (int q = 0; q < 16; ++q) s[q] = c->s[q];
  return MRTLB_OK;
}

static void free_events(mrtlb_ctx* c) {
  for (int k = 0; k < 2 * c->ev_cap; ++k) cudaEventDestroy(c->ev[k]);
  delete[] c->ev;
  c->ev = nullptr;
  c->ev_cap = c->ev_used = 0;
}

extern "C" int mrtlb_timing_begin(mrtlb_ctx* c, int max_launches) {
  if (!c) return MRTLB_ERR_ARG;
  if (max_launches < 1) return fail(c, MRTLB_ERR_ARG, "max_launches < 1");
  if (c->ev_cap < max_launches) {
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    free_events(c);
    c->ev = new cudaEvent_t[2 * (size_t)max_launches];
    for (int k = 0; k < 2 * max_launches; ++k) CK(cudaEventCreate(&c->ev[k]), "cudaEventCreate");
    c->ev_cap = max_launches;
  }
  c->ev_used = 0;
  c->timing = true;
  return MRTLB_OK;
}

extern "C" int mrtlb_timing_end(mrtlb_ctx* c, double* kernel_ms, long* launches) {
  if (!c || !kernel_ms || !launches) return MRTLB_ERR_ARG;
  c->timing = false;
  CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  double total = 0.0;
  for (int k = 0; k < c->ev_used; ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]), "cudaEventElapsedTime");
    total += ms;
  }
  *kernel_ms = total;
  *launches = c->ev_used;
  return MRTLB_OK;
}

extern "C" int mrtlb_launches_per_step(const mrtlb_ctx* c) {
  if (!c) return MRTLB_ERR_ARG;
  int n = 1;  // the step (it writes the ghost layer through)
  for (int s = 0; s < 4; ++s)
    if (refilled_side(c->L.bc[s])) { ++n; break; }  // + the wall and diffuse-ghost fill
  return n;
}

extern "C" int mrtlb_set_kernel(mrtlb_ctx* c, int which) {
  if (!c) return MRTLB_ERR_ARG;
  if (which < MRTLB_KERNEL_AUTO || which > MRTLB_KERNEL_TILED) return fail(c, MRTLB_ERR_ARG, "kernel %d", which);
  if (which == MRTLB_KERNEL_TILED && !tiled_supported(c->plan))
    return fail(c, MRTLB_ERR_UNSUPPORTED, "the tiled kernel is not available for this grid/binding");
  c->kernel = which;
  drop_graphs(c);
  return MRTLB_OK;
}

extern "C" const char* mrtlb_last_error(const mrtlb_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->last_error.c_str();
}

extern "C" void mrtlb_destroy(mrtlb_ctx* c) {
  if (!c) return;
  if (c->err || c->acc || c->staging || c->Tprev) cudaStreamSynchronize(c->stream);
  if (c->err) cudaFree(c->err);
  if (c->acc) cudaFree(c->acc);
  if (c->Tprev) cudaFree(c->Tprev);
  if (c->staging) cudaFree(c->staging);
  if (c->ev) free_events(c);
  drop_graphs(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  mrtlb_adjoint_free_internal(c);
  delete c;
}
