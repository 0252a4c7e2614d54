// step_flops.cu - counts the floating-point operations of one node update of
// the FP32 step, by running the kernel's own per-node templates (physics.cuh)
// on the host with an operation-counting number type.  The sequence is the
// one the row march executes per node: the macroscopic state when the row
// arrives, the velocity gradients, the harmonics and conserved moments again
// for the collision, the modified collision (equilibrium version 1), and the
// Lax-Wendroff update of the 16 velocities.  A sign change counts nothing (it
// folds into the next operation), a fused multiply-add two, the reciprocal's
// hardware approximation one special-function operation (not a flop), an
// FP64 division one.  Prints one JSON object with the FP32 and the FP64
// step's counts.
#include <cstdio>

#include "../../paper_1106_0785_gb300/csrc/physics.cuh"

namespace cnt {
long long n_add = 0, n_mul = 0, n_fma = 0, n_sfu = 0, n_div = 0;
bool fp64 = false;  // count the FP64 step's forms of 1/rho and T
struct Num {
  double v;
  Num() = default;
  Num(double x) : v(x) {}
};
inline Num operator+(Num a, Num b) { ++n_add; return Num(a.v + b.v); }
inline Num operator-(Num a, Num b) { ++n_add; return Num(a.v - b.v); }
inline Num operator-(Num a) { return Num(-a.v); }
inline Num operator*(Num a, Num b) { ++n_mul; return Num(a.v * b.v); }
inline Num& operator+=(Num& a, Num b) { return a = a + b; }
inline Num& operator-=(Num& a, Num b) { return a = a - b; }
inline Num fma(Num a, Num b, Num c) { ++n_fma; return Num(a.v * b.v + c.v); }
// 1/x as the kernels form it: FP32 approximation, then r (2 - x r); FP64
// one division
inline Num recip(Num x) {
  if (fp64) {
    ++n_div;
    return Num(1.0 / x.v);
  }
  ++n_sfu;
  const Num r(1.0 / x.v);
  return r * fma(-x, r, Num(2.0));
}
inline Num temperature(Num rho, Num jx, Num jy, Num e, Num ir) {
  return fp64 ? mrtlb::temperature_plain(rho, jx, jy, e, ir) : mrtlb::temperature_compensated(rho, jx, jy, e, ir);
}
inline Num expr(Num x) { ++n_sfu; return x; }
long long flops() { return n_add + n_mul + 2 * n_fma + n_div; }
void reset() { n_add = n_mul = n_fma = n_sfu = n_div = 0; }
}  // namespace cnt

// One node update; prints its counts as a JSON object.
static void count_step(const char* name) {
  using cnt::Num;
  using namespace mrtlb;
  cnt::reset();
  Coef<Num> c;
  Num* fields = &c.a1x;
  const int nf = (int)(offsetof(Coef<Num>, version) / sizeof(Num));
  for (int i = 0; i < nf; ++i) fields[i] = Num(0.01 * (i + 1));
  c.version = 1;
  c.modified = 1;
  Num f[16], fE[16], fW[16], fN[16], fS[16];
  for (int q = 0; q < 16; ++q) f[q] = fE[q] = fW[q] = fN[q] = fS[q] = Num(0.1 + 0.01 * q);
  const Num uE(0.1), uW(0.2), uN(0.3), uS(0.4);

  // the row's arrival: rho, j, e, 1/rho, u, T
  const NodeMac<Num> m = node_macros(f);
  const long long arrive = cnt::flops();
  // velocity gradients (central differences)
  const Num dux_dx = (uE - uW) * c.inv2dx, duy_dx = (uE - uW) * c.inv2dx;
  const Num dux_dy = (uN - uS) * c.inv2dy, duy_dy = (uN - uS) * c.inv2dy;
  // the collision, from the harmonics and conserved moments formed again
  Harm<Num> h;
  harmonics(f, h);
  Num rho, jx, jy, e;
  conserved_h(h, rho, jx, jy, e);
  Num C[16];
  collision_h(c, h, dux_dx, dux_dy, duy_dx, duy_dy, rho, m.ir, jx, jy, e, m.ux, m.uy, m.T, C);
  const long long collide = cnt::flops() - arrive;
  Num sum(0.0);
  for (int q = 0; q < 16; ++q) sum.v += lw_update(c, q, f[q], C[q], fE[q], fW[q], fN[q], fS[q]).v;
  const long long advect = cnt::flops() - arrive - collide;
  std::printf("\"%s\": {\"arrive\": %lld, \"collide\": %lld, \"advect\": %lld, \"total\": %lld, "
              "\"adds\": %lld, \"muls\": %lld, \"fmas\": %lld, \"divs\": %lld, \"sfu\": %lld, \"finite\": %d}",
              name, arrive, collide, advect, cnt::flops(), cnt::n_add, cnt::n_mul, cnt::n_fma, cnt::n_div,
              cnt::n_sfu, sum.v == sum.v ? 1 : 0);
}

int main() {
  std::printf("{");
  cnt::fp64 = false;
  count_step("fp32");
  std::printf(", ");
  cnt::fp64 = true;
  count_step("fp64");
  std::printf("}\n");
  return 0;
}
