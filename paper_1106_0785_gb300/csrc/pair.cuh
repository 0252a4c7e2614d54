// pair.cuh - two FP32 lattice nodes in one 64-bit register pair.
//
// Blackwell executes FP32 add, multiply and fused multiply-add on packed
// pairs (one instruction for two lanes).  P2 holds the same quantity of two
// neighbouring nodes; its operators make the per-node templates of
// physics.cuh run on both nodes at once.  A product is kept lazy (P2Mul) so
// that a * b + c, c + a * b, a * b - c and c - a * b each become one packed
// fused multiply-add, as the compiler would contract the scalar forms.
// Every lane is rounded exactly as the scalar FP32 arithmetic rounds it.
#pragma once

#include <cuda_runtime.h>

namespace mrtlb {

struct P2 {
  float2 v;
  P2() = default;
  __host__ __device__ __forceinline__ P2(float s) : v(make_float2(s, s)) {}
  __host__ __device__ __forceinline__ P2(float a, float b) : v(make_float2(a, b)) {}
  __host__ __device__ __forceinline__ explicit P2(float2 a) : v(a) {}
};

__device__ __forceinline__ P2 p2_add(P2 a, P2 b) { return P2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ P2 p2_mul(P2 a, P2 b) { return P2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ P2 p2_fma(P2 a, P2 b, P2 c) { return P2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ P2 operator-(P2 a) { return P2(make_float2(-a.v.x, -a.v.y)); }

struct P2Mul {
  P2 a, b;
  __device__ __forceinline__ operator P2() const { return p2_mul(a, b); }
};

__device__ __forceinline__ P2Mul operator*(P2 a, P2 b) { return P2Mul{a, b}; }
__device__ __forceinline__ P2Mul operator*(P2Mul m, P2 b) { return P2Mul{P2(m), b}; }
__device__ __forceinline__ P2Mul operator*(P2 a, P2Mul m) { return P2Mul{a, P2(m)}; }
__device__ __forceinline__ P2Mul operator*(P2Mul m, P2Mul n) { return P2Mul{P2(m), P2(n)}; }
__device__ __forceinline__ P2Mul operator-(P2Mul m) { return P2Mul{-m.a, m.b}; }

__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return p2_add(a, b); }
__device__ __forceinline__ P2 operator-(P2 a, P2 b) { return p2_add(a, -b); }
__device__ __forceinline__ P2 operator+(P2Mul m, P2 c) { return p2_fma(m.a, m.b, c); }
__device__ __forceinline__ P2 operator+(P2 c, P2Mul m) { return p2_fma(m.a, m.b, c); }
__device__ __forceinline__ P2 operator-(P2Mul m, P2 c) { return p2_fma(m.a, m.b, -c); }
__device__ __forceinline__ P2 operator-(P2 c, P2Mul m) { return p2_fma(-m.a, m.b, c); }
__device__ __forceinline__ P2 operator+(P2Mul m, P2Mul n) { return p2_fma(m.a, m.b, P2(n)); }
__device__ __forceinline__ P2 operator-(P2Mul m, P2Mul n) { return p2_fma(m.a, m.b, -P2(n)); }

__device__ __forceinline__ P2& operator+=(P2& a, P2 b) { return a = a + b; }
__device__ __forceinline__ P2& operator+=(P2& a, P2Mul m) { return a = a + m; }
__device__ __forceinline__ P2& operator-=(P2& a, P2 b) { return a = a - b; }
__device__ __forceinline__ P2& operator-=(P2& a, P2Mul m) { return a = a - m; }
__device__ __forceinline__ P2& operator*=(P2& a, P2 b) { return a = P2(a * b); }

using ::fma;  // keep the scalar overloads visible beside the pair one
__device__ __forceinline__ P2 fma(P2 a, P2 b, P2 c) { return p2_fma(a, b, c); }

}  // namespace mrtlb
