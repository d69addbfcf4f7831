// Device-side building blocks of the gradsolve-gb300 hot path: explicit-
// rounding arithmetic, the problem registry (f, J^T v, f_theta^T v written out
// by hand per problem), the Tsit5 tableau and step, and the warp-level helpers
// of the persistent kernels.
//
// Every floating-point operation of the solver arithmetic is written with an
// explicitly rounded intrinsic (fma_, mul_, add_, sub_). The compiler can then
// neither contract nor reassociate it, so every kernel that instantiates this
// code (with or without save-state output, record or reverse) performs the
// same roundings in the same order: the mesh a record produces and the states
// a reverse sweep recomputes do not depend on which kernel ran.
//
// One trajectory per lane, state in registers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gs {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int KMAX = 32;  // largest checkpoint interval (accepted steps per record segment)

enum : int { TRAJ_OK = 0, TRAJ_MAXSTEPS = 1, TRAJ_DT_UNDERFLOW = 2, TRAJ_NONFINITE = 3, TRAJ_SINGULAR = 4 };

// ---------------------------------------------------------------------------
// Explicitly rounded arithmetic (round to nearest even), FP64 and FP32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }

// ---------------------------------------------------------------------------
// FP32 <-> FP64 conversions on the integer ALU. GB300 executes the hardware
// conversion instructions on its FP64 pipe (2 lanes per clock per SM), which
// the FP32-mixed form otherwise spends on format changes; these rebuild the
// IEEE-754 encodings with integer operations instead. to_d is exact for every
// float (subnormals flush to zero); to_f truncates the mantissa (round toward
// zero), flushes values below the float normal range to zero and saturates
// to infinity above it. Both are identities when R = double.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double to_d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint64_t s = (uint64_t)(u & 0x80000000u) << 32;
  const uint64_t ed = (e == 0u) ? 0u : (e == 0xffu ? 0x7ffu : e + 896u);
  const uint64_t m = (e == 0u) ? 0u : (uint64_t)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(s | (ed << 52) | m));
}
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ float to_f(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t s = (uint32_t)(b >> 32) & 0x80000000u;
  const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
  const uint32_t m = (uint32_t)(b >> 29) & 0x7fffffu;
  uint32_t r = s | ((e - 896u) << 23) | m;                   // normal range: e in [897, 1150]
  r = (e < 897u) ? s : r;                                     // underflow: signed zero
  r = (e > 1150u) ? (s | 0x7f800000u | (e == 0x7ffu && (b << 12) ? 0x400000u : 0u)) : r;  // inf / nan
  return __uint_as_float(r);
}
// Order tests on FP64 values done on the integer ALU: for IEEE doubles that
// are >= +0 (or NaN), the bit patterns order exactly as the values do, and NaN
// patterns lie above +inf.
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ unsigned long long abs_bits(double x) { return dbits(x) & 0x7fffffffffffffffull; }
__device__ __forceinline__ double max_abs(double a, double b) {  // max(|a|, |b|) for finite or inf a, b
  const unsigned long long ua = abs_bits(a), ub = abs_bits(b);
  return __longlong_as_double((long long)(ua > ub ? ua : ub));
}
// Order key of any non-NaN double as a signed 64-bit integer: negative values
// get their magnitude bits flipped, so key(a) < key(b) iff a < b (with -0 just
// below +0). Equality of two doubles that are not zero or NaN is equality of
// their bits. The solver's time comparisons (end of span, save times) run on
// the integer ALU this way.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool same_time(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b);
}
constexpr unsigned long long DBITS_ONE = 0x3ff0000000000000ull;  // 1.0
constexpr unsigned long long DBITS_INF = 0x7ff0000000000000ull;  // +inf
__device__ __forceinline__ bool le_one(double q) { return dbits(q) <= DBITS_ONE; }      // q >= 0: q <= 1, NaN false
__device__ __forceinline__ bool finite_nonneg(double q) { return dbits(q) < DBITS_INF; }  // q >= 0 finite
__device__ __forceinline__ bool positive(double q) { return dbits(q) != 0ull && dbits(q) < 0x8000000000000000ull; }
__device__ __forceinline__ bool finite_d(double x) { return abs_bits(x) < DBITS_INF; }  // not inf or NaN

// The loss sum_s ||y(t_s)||^2 of one trajectory, accumulated in FP64.
__device__ __forceinline__ double acc_loss(double loss, double v) { return add_(loss, v); }
__device__ __forceinline__ double acc_loss(double loss, float v) { return add_(loss, to_d(v)); }

template <class R>
__device__ __forceinline__ R to_r(double x);
template <>
__device__ __forceinline__ double to_r<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_r<float>(double x) { return to_f(x); }

// ---------------------------------------------------------------------------
// Problems (paper Appendix A). Each provides
//   f(y, p, o):           o = f(y, theta)
//   vjp(y, p, v, yb, pb): yb = J(y)^T v,  pb += (df/dtheta)^T v
// with the analytic derivatives of the printed right-hand sides, and the
// operation counts (FP64 instructions; an FMA is one instruction, two flops)
// F_OPS / F_FLOPS and VJP_OPS / VJP_FLOPS used for the algorithmic flop count.
// ---------------------------------------------------------------------------
struct Lorenz {  // sigma (y - x), x (rho - z) - y, x y - beta z; theta = (sigma, rho, beta)
  static constexpr int D = 3, NP = 3;
  template <class R>
  __device__ __forceinline__ static void f(const R (&y)[D], const R (&p)[NP], R (&o)[D]) {
    o[0] = mul_(p[0], sub_(y[1], y[0]));
    o[1] = fma_(y[0], sub_(p[1], y[2]), -y[1]);
    o[2] = fma_(y[0], y[1], -mul_(p[2], y[2]));
  }
  template <class R>
  __device__ __forceinline__ static void vjp(const R (&y)[D], const R (&p)[NP], const R (&v)[D], R (&yb)[D],
                                             R (&pb)[NP]) {
    // J = [[-sigma, sigma, 0], [rho - z, -1, -x], [y, x, -beta]]
    yb[0] = fma_(sub_(p[1], y[2]), v[1], fma_(y[1], v[2], -mul_(p[0], v[0])));
    yb[1] = fma_(p[0], v[0], fma_(y[0], v[2], -v[1]));
    yb[2] = -fma_(y[0], v[1], mul_(p[2], v[2]));
    pb[0] = fma_(sub_(y[1], y[0]), v[0], pb[0]);
    pb[1] = fma_(y[0], v[1], pb[1]);
    pb[2] = fma_(-y[2], v[2], pb[2]);
  }
  // Tangent: o = J(y) yd + (df/dtheta) pd.
  template <class R>
  __device__ __forceinline__ static void jvp(const R (&y)[D], const R (&p)[NP], const R (&yd)[D], const R (&pd)[NP],
                                             R (&o)[D]) {
    o[0] = fma_(pd[0], sub_(y[1], y[0]), mul_(p[0], sub_(yd[1], yd[0])));
    o[1] = fma_(yd[0], sub_(p[1], y[2]), fma_(y[0], sub_(pd[1], yd[2]), -yd[1]));
    o[2] = fma_(yd[0], y[1], fma_(y[0], yd[1], -fma_(pd[2], y[2], mul_(p[2], yd[2]))));
  }
};

struct VanDerPol {  // x' = v, v' = mu ((1 - x^2) v - x); theta = (mu)
  static constexpr int D = 2, NP = 1;
  template <class R>
  __device__ __forceinline__ static void f(const R (&y)[D], const R (&p)[NP], R (&o)[D]) {
    o[0] = y[1];
    o[1] = mul_(p[0], fma_(fma_(-y[0], y[0], R(1)), y[1], -y[0]));
  }
  template <class R>
  __device__ __forceinline__ static void vjp(const R (&y)[D], const R (&p)[NP], const R (&v)[D], R (&yb)[D],
                                             R (&pb)[NP]) {
    // J = [[0, 1], [mu (-2 x v - 1), mu (1 - x^2)]]
    const R w = fma_(-y[0], y[0], R(1));
    const R mv = mul_(p[0], v[1]);
    yb[0] = -mul_(mv, fma_(add_(y[0], y[0]), y[1], R(1)));
    yb[1] = fma_(mv, w, v[0]);
    pb[0] = fma_(fma_(w, y[1], -y[0]), v[1], pb[0]);
  }
  template <class R>
  __device__ __forceinline__ static void jvp(const R (&y)[D], const R (&p)[NP], const R (&yd)[D], const R (&pd)[NP],
                                             R (&o)[D]) {
    const R w = fma_(-y[0], y[0], R(1));
    const R g = fma_(w, y[1], -y[0]);                                              // (1 - x^2) v - x
    const R gd = fma_(w, yd[1], fma_(mul_(-add_(y[0], y[0]), yd[0]), y[1], -yd[0]));  // its tangent
    o[0] = yd[1];
    o[1] = fma_(pd[0], g, mul_(p[0], gd));
  }
};

struct Linear2 {  // y' = A y, A = [[p0, p1], [p2, p3]]
  static constexpr int D = 2, NP = 4;
  template <class R>
  __device__ __forceinline__ static void f(const R (&y)[D], const R (&p)[NP], R (&o)[D]) {
    o[0] = fma_(p[0], y[0], mul_(p[1], y[1]));
    o[1] = fma_(p[2], y[0], mul_(p[3], y[1]));
  }
  template <class R>
  __device__ __forceinline__ static void vjp(const R (&y)[D], const R (&p)[NP], const R (&v)[D], R (&yb)[D],
                                             R (&pb)[NP]) {
    yb[0] = fma_(p[0], v[0], mul_(p[2], v[1]));
    yb[1] = fma_(p[1], v[0], mul_(p[3], v[1]));
    pb[0] = fma_(y[0], v[0], pb[0]);
    pb[1] = fma_(y[1], v[0], pb[1]);
    pb[2] = fma_(y[0], v[1], pb[2]);
    pb[3] = fma_(y[1], v[1], pb[3]);
  }
  // Dense J (row-major, J[c][a] = d f_c / d y_a) and the gradient of
  // g = r^T J(y, theta) u: gy += dg/dy, gp += dg/dtheta (J = A: no y term).
  template <class R>
  __device__ __forceinline__ static void jac(const R (&y)[D], const R (&p)[NP], R (&J)[D][D]) {
    J[0][0] = p[0]; J[0][1] = p[1];
    J[1][0] = p[2]; J[1][1] = p[3];
  }
  template <class R>
  __device__ __forceinline__ static void jac_contract(const R (&y)[D], const R (&p)[NP], const R (&r)[D],
                                                      const R (&u)[D], R (&gy)[D], R (&gp)[NP]) {
    gp[0] = fma_(r[0], u[0], gp[0]);
    gp[1] = fma_(r[0], u[1], gp[1]);
    gp[2] = fma_(r[1], u[0], gp[2]);
    gp[3] = fma_(r[1], u[1], gp[3]);
  }
  template <class R>
  __device__ __forceinline__ static void jvp(const R (&y)[D], const R (&p)[NP], const R (&yd)[D], const R (&pd)[NP],
                                             R (&o)[D]) {
    o[0] = fma_(p[0], yd[0], fma_(p[1], yd[1], fma_(pd[0], y[0], mul_(pd[1], y[1]))));
    o[1] = fma_(p[2], yd[0], fma_(p[3], yd[1], fma_(pd[2], y[0], mul_(pd[3], y[1]))));
  }
  // Directional derivative of the Jacobian applied to u: o = (dJ/dy[yd] + dJ/dtheta[pd]) u.
  template <class R>
  __device__ __forceinline__ static void jac_dir(const R (&y)[D], const R (&p)[NP], const R (&yd)[D],
                                                 const R (&pd)[NP], const R (&u)[D], R (&o)[D]) {
    o[0] = fma_(pd[0], u[0], mul_(pd[1], u[1]));
    o[1] = fma_(pd[2], u[0], mul_(pd[3], u[1]));
  }
};

// Robertson (Appendix A): y1' = -k1 y1 + k3 y2 y3, y2' = k1 y1 - k3 y2 y3 - k2 y2^2,
// y3' = k2 y2^2; theta = (k1, k2, k3).
struct Robertson {
  static constexpr int D = 3, NP = 3;
  template <class R>
  __device__ __forceinline__ static void f(const R (&y)[D], const R (&p)[NP], R (&o)[D]) {
    const R a = mul_(p[0], y[0]);
    const R b = mul_(mul_(p[2], y[1]), y[2]);
    const R c = mul_(mul_(p[1], y[1]), y[1]);
    o[0] = sub_(b, a);
    o[1] = sub_(sub_(a, b), c);
    o[2] = c;
  }
  template <class R>
  __device__ __forceinline__ static void vjp(const R (&y)[D], const R (&p)[NP], const R (&v)[D], R (&yb)[D],
                                             R (&pb)[NP]) {
    const R d01 = sub_(v[1], v[0]), d21 = sub_(v[2], v[1]);
    yb[0] = mul_(p[0], d01);
    yb[1] = fma_(mul_(p[2], y[2]), -d01, mul_(add_(p[1], p[1]), mul_(y[1], d21)));
    yb[2] = mul_(mul_(p[2], y[1]), -d01);
    pb[0] = fma_(y[0], d01, pb[0]);
    pb[1] = fma_(mul_(y[1], y[1]), d21, pb[1]);
    pb[2] = fma_(mul_(y[1], y[2]), -d01, pb[2]);
  }
  template <class R>
  __device__ __forceinline__ static void jac(const R (&y)[D], const R (&p)[NP], R (&J)[D][D]) {
    const R k3y1 = mul_(p[2], y[1]), k3y2 = mul_(p[2], y[2]), k2y1x2 = mul_(add_(p[1], p[1]), y[1]);
    J[0][0] = -p[0]; J[0][1] = k3y2;               J[0][2] = k3y1;
    J[1][0] = p[0];  J[1][1] = -add_(k3y2, k2y1x2); J[1][2] = -k3y1;
    J[2][0] = R(0);  J[2][1] = k2y1x2;             J[2][2] = R(0);
  }
  template <class R>
  __device__ __forceinline__ static void jac_contract(const R (&y)[D], const R (&p)[NP], const R (&r)[D],
                                                      const R (&u)[D], R (&gy)[D], R (&gp)[NP]) {
    // g = r^T J u; J depends on y2, y3 (1-based) and linearly on k.
    const R r01 = sub_(r[0], r[1]), r21 = sub_(r[2], r[1]);
    gy[1] = fma_(mul_(p[2], u[2]), r01, fma_(mul_(add_(p[1], p[1]), u[1]), r21, gy[1]));
    gy[2] = fma_(mul_(p[2], u[1]), r01, gy[2]);
    gp[0] = fma_(u[0], -r01, gp[0]);
    gp[1] = fma_(mul_(add_(y[1], y[1]), u[1]), r21, gp[1]);
    gp[2] = fma_(fma_(y[2], u[1], mul_(y[1], u[2])), r01, gp[2]);
  }
  template <class R>
  __device__ __forceinline__ static void jvp(const R (&y)[D], const R (&p)[NP], const R (&yd)[D], const R (&pd)[NP],
                                             R (&o)[D]) {
    const R ad = fma_(pd[0], y[0], mul_(p[0], yd[0]));                                       // d(k1 y1)
    const R bd = fma_(mul_(pd[2], y[1]), y[2], mul_(p[2], fma_(yd[1], y[2], mul_(y[1], yd[2]))));  // d(k3 y2 y3)
    const R cd = fma_(mul_(pd[1], y[1]), y[1], mul_(add_(p[1], p[1]), mul_(y[1], yd[1])));        // d(k2 y2^2)
    o[0] = sub_(bd, ad);
    o[1] = sub_(sub_(ad, bd), cd);
    o[2] = cd;
  }
  template <class R>
  __device__ __forceinline__ static void jac_dir(const R (&y)[D], const R (&p)[NP], const R (&yd)[D],
                                                 const R (&pd)[NP], const R (&u)[D], R (&o)[D]) {
    const R e = fma_(pd[2], y[2], mul_(p[2], yd[2]));                   // d(k3 y3)
    const R g = fma_(pd[2], y[1], mul_(p[2], yd[1]));                   // d(k3 y2)
    const R q = mul_(R(2), fma_(pd[1], y[1], mul_(p[1], yd[1])));       // d(2 k2 y2)
    o[0] = fma_(-pd[0], u[0], fma_(e, u[1], mul_(g, u[2])));
    o[1] = fma_(pd[0], u[0], fma_(-add_(e, q), u[1], -mul_(g, u[2])));
    o[2] = mul_(q, u[1]);
  }
};

// HIRES (Appendix A), the 12 distinct literal constants as parameters
// p0..p11 = (1.71, 0.43, 8.32, 0.0007, 8.75, 10.03, 0.035, 1.12, 1.745, 280,
// 0.69, 1.81), each shared wherever it appears.
struct Hires {
  static constexpr int D = 8, NP = 12;
  template <class R>
  __device__ __forceinline__ static void f(const R (&y)[D], const R (&p)[NP], R (&o)[D]) {
    const R w = mul_(mul_(p[9], y[5]), y[7]);
    o[0] = add_(fma_(p[2], y[2], fma_(p[1], y[1], -mul_(p[0], y[0]))), p[3]);
    o[1] = fma_(p[0], y[0], -mul_(p[4], y[1]));
    o[2] = fma_(p[6], y[4], fma_(p[1], y[3], -mul_(p[5], y[2])));
    o[3] = fma_(p[2], y[1], fma_(p[0], y[2], -mul_(p[7], y[3])));
    o[4] = fma_(p[1], add_(y[5], y[6]), -mul_(p[8], y[4]));
    o[5] = sub_(fma_(p[10], add_(y[3], y[6]), fma_(p[0], y[4], -mul_(p[1], y[5]))), w);
    o[6] = fma_(-p[11], y[6], w);
    o[7] = fma_(p[11], y[6], -w);
  }
  template <class R>
  __device__ __forceinline__ static void vjp(const R (&y)[D], const R (&p)[NP], const R (&v)[D], R (&yb)[D],
                                             R (&pb)[NP]) {
    const R d10 = sub_(v[1], v[0]);
    const R s = sub_(sub_(v[6], v[5]), v[7]);  // v6 - v5 - v7
    const R d76 = sub_(v[7], v[6]);
    yb[0] = mul_(p[0], d10);
    yb[1] = fma_(p[1], v[0], fma_(p[2], v[3], -mul_(p[4], v[1])));
    yb[2] = fma_(p[2], v[0], fma_(p[0], v[3], -mul_(p[5], v[2])));
    yb[3] = fma_(p[1], v[2], fma_(p[10], v[5], -mul_(p[7], v[3])));
    yb[4] = fma_(p[6], v[2], fma_(p[0], v[5], -mul_(p[8], v[4])));
    yb[5] = fma_(p[1], sub_(v[4], v[5]), mul_(mul_(p[9], y[7]), s));
    yb[6] = fma_(p[1], v[4], fma_(p[10], v[5], mul_(p[11], d76)));
    yb[7] = mul_(mul_(p[9], y[5]), s);
    pb[0] = fma_(y[0], d10, fma_(y[2], v[3], fma_(y[4], v[5], pb[0])));
    pb[1] = fma_(y[1], v[0], fma_(y[3], v[2], fma_(add_(y[5], y[6]), v[4], fma_(-y[5], v[5], pb[1]))));
    pb[2] = fma_(y[2], v[0], fma_(y[1], v[3], pb[2]));
    pb[3] = add_(v[0], pb[3]);
    pb[4] = fma_(-y[1], v[1], pb[4]);
    pb[5] = fma_(-y[2], v[2], pb[5]);
    pb[6] = fma_(y[4], v[2], pb[6]);
    pb[7] = fma_(-y[3], v[3], pb[7]);
    pb[8] = fma_(-y[4], v[4], pb[8]);
    pb[9] = fma_(mul_(y[5], y[7]), s, pb[9]);
    pb[10] = fma_(add_(y[3], y[6]), v[5], pb[10]);
    pb[11] = fma_(y[6], d76, pb[11]);
  }
  template <class R>
  __device__ __forceinline__ static void jac(const R (&y)[D], const R (&p)[NP], R (&J)[D][D]) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) J[i][j] = R(0);
    const R p9y7 = mul_(p[9], y[7]), p9y5 = mul_(p[9], y[5]);
    J[0][0] = -p[0]; J[0][1] = p[1]; J[0][2] = p[2];
    J[1][0] = p[0];  J[1][1] = -p[4];
    J[2][2] = -p[5]; J[2][3] = p[1]; J[2][4] = p[6];
    J[3][1] = p[2];  J[3][2] = p[0]; J[3][3] = -p[7];
    J[4][4] = -p[8]; J[4][5] = p[1]; J[4][6] = p[1];
    J[5][3] = p[10]; J[5][4] = p[0]; J[5][5] = -add_(p9y7, p[1]); J[5][6] = p[10]; J[5][7] = -p9y5;
    J[6][5] = p9y7;  J[6][6] = -p[11]; J[6][7] = p9y5;
    J[7][5] = -p9y7; J[7][6] = p[11];  J[7][7] = -p9y5;
  }
  template <class R>
  __device__ __forceinline__ static void jac_contract(const R (&y)[D], const R (&p)[NP], const R (&r)[D],
                                                      const R (&u)[D], R (&gy)[D], R (&gp)[NP]) {
    // g = r^T J u: the y-dependent entries are p9 y8 and p9 y6 (1-based) in rows 6..8.
    const R s = sub_(sub_(r[6], r[5]), r[7]);  // r6 - r5 - r7
    gy[5] = fma_(mul_(p[9], u[7]), s, gy[5]);
    gy[7] = fma_(mul_(p[9], u[5]), s, gy[7]);
    gp[0] = fma_(sub_(r[1], r[0]), u[0], fma_(r[3], u[2], fma_(r[5], u[4], gp[0])));
    gp[1] = fma_(r[0], u[1], fma_(r[2], u[3], fma_(r[4], add_(u[5], u[6]), fma_(-r[5], u[5], gp[1]))));
    gp[2] = fma_(r[0], u[2], fma_(r[3], u[1], gp[2]));
    gp[4] = fma_(-r[1], u[1], gp[4]);
    gp[5] = fma_(-r[2], u[2], gp[5]);
    gp[6] = fma_(r[2], u[4], gp[6]);
    gp[7] = fma_(-r[3], u[3], gp[7]);
    gp[8] = fma_(-r[4], u[4], gp[8]);
    gp[9] = fma_(fma_(y[7], u[5], mul_(y[5], u[7])), s, gp[9]);
    gp[10] = fma_(r[5], add_(u[3], u[6]), gp[10]);
    gp[11] = fma_(u[6], sub_(r[7], r[6]), gp[11]);
  }
  template <class R>
  __device__ __forceinline__ static void jvp(const R (&y)[D], const R (&p)[NP], const R (&yd)[D], const R (&pd)[NP],
                                             R (&o)[D]) {
    // each bilinear term p_i y_j contributes pd_i y_j + p_i yd_j; w = p9 y5 y7 (0-based)
    auto dl = [](R pp, R ppd, R yy, R yyd) { return fma_(ppd, yy, mul_(pp, yyd)); };
    const R wd = fma_(mul_(pd[9], y[5]), y[7], mul_(p[9], fma_(yd[5], y[7], mul_(y[5], yd[7]))));
    o[0] = add_(sub_(add_(dl(p[2], pd[2], y[2], yd[2]), dl(p[1], pd[1], y[1], yd[1])), dl(p[0], pd[0], y[0], yd[0])),
                pd[3]);
    o[1] = sub_(dl(p[0], pd[0], y[0], yd[0]), dl(p[4], pd[4], y[1], yd[1]));
    o[2] = sub_(add_(dl(p[6], pd[6], y[4], yd[4]), dl(p[1], pd[1], y[3], yd[3])), dl(p[5], pd[5], y[2], yd[2]));
    o[3] = sub_(add_(dl(p[2], pd[2], y[1], yd[1]), dl(p[0], pd[0], y[2], yd[2])), dl(p[7], pd[7], y[3], yd[3]));
    o[4] = sub_(dl(p[1], pd[1], add_(y[5], y[6]), add_(yd[5], yd[6])), dl(p[8], pd[8], y[4], yd[4]));
    o[5] = sub_(sub_(add_(dl(p[10], pd[10], add_(y[3], y[6]), add_(yd[3], yd[6])), dl(p[0], pd[0], y[4], yd[4])),
                     dl(p[1], pd[1], y[5], yd[5])),
                wd);
    const R z = dl(p[11], pd[11], y[6], yd[6]);
    o[6] = sub_(wd, z);
    o[7] = sub_(z, wd);
  }
  template <class R>
  __device__ __forceinline__ static void jac_dir(const R (&y)[D], const R (&p)[NP], const R (&yd)[D],
                                                 const R (&pd)[NP], const R (&u)[D], R (&o)[D]) {
    const R a = fma_(pd[9], y[7], mul_(p[9], yd[7]));  // d(p9 y7)
    const R b = fma_(pd[9], y[5], mul_(p[9], yd[5]));  // d(p9 y5)
    o[0] = fma_(-pd[0], u[0], fma_(pd[1], u[1], mul_(pd[2], u[2])));
    o[1] = fma_(pd[0], u[0], -mul_(pd[4], u[1]));
    o[2] = fma_(-pd[5], u[2], fma_(pd[1], u[3], mul_(pd[6], u[4])));
    o[3] = fma_(pd[2], u[1], fma_(pd[0], u[2], -mul_(pd[7], u[3])));
    o[4] = fma_(-pd[8], u[4], mul_(pd[1], add_(u[5], u[6])));
    o[5] = fma_(pd[10], add_(u[3], u[6]), fma_(pd[0], u[4], fma_(-add_(a, pd[1]), u[5], -mul_(b, u[7]))));
    o[6] = fma_(a, u[5], fma_(-pd[11], u[6], mul_(b, u[7])));
    o[7] = fma_(-a, u[5], fma_(pd[11], u[6], -mul_(b, u[7])));
  }
};

// ---------------------------------------------------------------------------
// Tsit5 (Tsitouras 2011, Table 1): 7 stages, FSAL (b = row 7 of A, b_7 = 0).
// ---------------------------------------------------------------------------
namespace tsit5 {
__host__ __device__ constexpr double A(int i, int j) {
  // 0-based stage i (1..6), column j < i
  return (i == 1 && j == 0)   ? 0.161
         : (i == 2 && j == 0) ? -0.008480655492356989
         : (i == 2 && j == 1) ? 0.335480655492357
         : (i == 3 && j == 0) ? 2.897153057105493
         : (i == 3 && j == 1) ? -6.359448489975075
         : (i == 3 && j == 2) ? 4.3622954328695815
         : (i == 4 && j == 0) ? 5.325864828439257
         : (i == 4 && j == 1) ? -11.748883564062828
         : (i == 4 && j == 2) ? 7.4955393428898365
         : (i == 4 && j == 3) ? -0.09249506636175525
         : (i == 5 && j == 0) ? 5.86145544294642
         : (i == 5 && j == 1) ? -12.92096931784711
         : (i == 5 && j == 2) ? 8.159367898576159
         : (i == 5 && j == 3) ? -0.071584973281401
         : (i == 5 && j == 4) ? -0.028269050394068383
         : (i == 6 && j == 0) ? 0.09646076681806523
         : (i == 6 && j == 1) ? 0.01
         : (i == 6 && j == 2) ? 0.4798896504144996
         : (i == 6 && j == 3) ? 1.379008574103742
         : (i == 6 && j == 4) ? -3.290069515436081
         : (i == 6 && j == 5) ? 2.324710524099774
                              : 0.0;
}
__host__ __device__ constexpr double B(int j) { return A(6, j); }
__host__ __device__ constexpr double Bhat(int j) {
  return j == 0   ? 0.09468075576583945
         : j == 1 ? 0.009183565540343
         : j == 2 ? 0.4877705284247616
         : j == 3 ? 1.234297566930479
         : j == 4 ? -2.707712349983525
         : j == 5 ? 1.866628418170587
                  : 1.0 / 66.0;
}
__host__ __device__ constexpr double Btilde(int j) { return B(j) - Bhat(j); }  // error weights
}  // namespace tsit5

// Problems with a shared network (they declare kWeights).
template <class Pb, class = void>
struct HasNet : std::false_type {};
template <class Pb>
struct HasNet<Pb, std::void_t<decltype(Pb::kWeights)>> : std::true_type {};

// Stage inputs Y[0..6] of one Tsit5 step from y with size h (Y[0] = y,
// Y[6] = y_new by FSAL) and stage slopes K[0..KN-1]. K[0] must hold f(y).
// KN = 7 also evaluates k7 = f(y_new) for the error estimate and FSAL.
template <class Pb, class R, int KN>
__device__ __forceinline__ void tsit5_stages(const R (&y)[Pb::D], const R (&p)[Pb::NP], R h, R (&Y)[7][Pb::D],
                                             R (&K)[7][Pb::D]) {
  constexpr int D = Pb::D;
#pragma unroll
  for (int c = 0; c < D; ++c) Y[0][c] = y[c];
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    // FP32 (not the network problems, whose register budget it upsets): components 0, 1 as FP32x2
    constexpr bool PACK = std::is_same<R, float>::value && D >= 2 && !HasNet<Pb>::value;
    if constexpr (PACK) {
      // the same per-component IEEE operations, two components per instruction
      float2 s = __fmul2_rn(make_float2(tsit5::A(i, 0), tsit5::A(i, 0)), make_float2(K[0][0], K[0][1]));
#pragma unroll
      for (int j = 1; j < i; ++j)
        s = __ffma2_rn(make_float2(tsit5::A(i, j), tsit5::A(i, j)), make_float2(K[j][0], K[j][1]), s);
      const float2 yy = __ffma2_rn(make_float2(h, h), s, make_float2(y[0], y[1]));
      Y[i][0] = yy.x;
      Y[i][1] = yy.y;
    }
#pragma unroll
    for (int c = PACK ? 2 : 0; c < D; ++c) {
      R s = mul_(R(tsit5::A(i, 0)), K[0][c]);
#pragma unroll
      for (int j = 1; j < i; ++j) s = fma_(R(tsit5::A(i, j)), K[j][c], s);
      Y[i][c] = fma_(h, s, y[c]);
    }
    if (i < 6 || KN == 7) Pb::f(Y[i], p, K[i]);
  }
}

// Embedded error estimate e = y_new - yhat_new = h sum_j (b_j - bhat_j) k_j.
template <class Pb, class R>
__device__ __forceinline__ void tsit5_error(const R (&K)[7][Pb::D], R h, R (&e)[Pb::D]) {
  // FP32: components 0, 1 as FP32x2 (the same per-component IEEE operations)
  constexpr bool PACK = std::is_same<R, float>::value && Pb::D >= 2 && !HasNet<Pb>::value;
  if constexpr (PACK) {
    float2 s = __fmul2_rn(make_float2(tsit5::Btilde(0), tsit5::Btilde(0)), make_float2(K[0][0], K[0][1]));
#pragma unroll
    for (int j = 1; j < 7; ++j)
      s = __ffma2_rn(make_float2(tsit5::Btilde(j), tsit5::Btilde(j)), make_float2(K[j][0], K[j][1]), s);
    const float2 e2 = __fmul2_rn(make_float2(h, h), s);
    e[0] = e2.x;
    e[1] = e2.y;
  }
#pragma unroll
  for (int c = PACK ? 2 : 0; c < Pb::D; ++c) {
    R s = mul_(R(tsit5::Btilde(0)), K[0][c]);
#pragma unroll
    for (int j = 1; j < 7; ++j) s = fma_(R(tsit5::Btilde(j)), K[j][c], s);
    e[c] = mul_(h, s);
  }
}

// Forward mode of one Tsit5 step with h held as data: y_new (the same
// arithmetic as tsit5_stages) and, for each of ND tangent directions
// (yd, pd), yd_new = dPhi/dy yd + dPhi/dtheta pd, from the stage tangents
// Yd_i = yd + h sum_j a_ij Kd_j, Kd_i = J(Y_i) Yd_i + f_theta(Y_i) pd.
template <class Pb, int ND>
__device__ __forceinline__ void tsit5_tangent(const double (&y)[Pb::D], const double (&yd)[ND][Pb::D],
                                              const double (&p)[Pb::NP], const double (&pd)[ND][Pb::NP], double h,
                                              double (&yn)[Pb::D], double (&ydn)[ND][Pb::D]) {
  constexpr int D = Pb::D;
  double K[6][D], Kd[6][ND][D];
  Pb::f(y, p, K[0]);
#pragma unroll
  for (int q = 0; q < ND; ++q) Pb::jvp(y, p, yd[q], pd[q], Kd[0][q]);
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    double Y[D], Yd[ND][D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double s = mul_(tsit5::A(i, 0), K[0][c]);
#pragma unroll
      for (int j = 1; j < i; ++j) s = fma_(tsit5::A(i, j), K[j][c], s);
      Y[c] = fma_(h, s, y[c]);
    }
#pragma unroll
    for (int q = 0; q < ND; ++q)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double s = mul_(tsit5::A(i, 0), Kd[0][q][c]);
#pragma unroll
        for (int j = 1; j < i; ++j) s = fma_(tsit5::A(i, j), Kd[j][q][c], s);
        Yd[q][c] = fma_(h, s, yd[q][c]);
      }
    if (i < 6) {
      Pb::f(Y, p, K[i]);
#pragma unroll
      for (int q = 0; q < ND; ++q) Pb::jvp(Y, p, Yd[q], pd[q], Kd[i][q]);
    } else {
#pragma unroll
      for (int c = 0; c < D; ++c) yn[c] = Y[c];
#pragma unroll
      for (int q = 0; q < ND; ++q)
#pragma unroll
        for (int c = 0; c < D; ++c) ydn[q][c] = Yd[q][c];
    }
  }
}

// Reverse of one Tsit5 step over its recomputed stage inputs Y[0..5]:
// given the cotangent c of y_new returns v = dL/dy (the cotangent of y) and
// accumulates dL/dtheta. kbar_j = h (b_j c + sum_{m>j} a_mj Ybar_m),
// Ybar_j = J(Y_j)^T kbar_j, theta_bar += f_theta(Y_j)^T kbar_j,
// v = c + sum_j Ybar_j.
template <class Pb, class R, class RB>
__device__ __forceinline__ void tsit5_reverse(const R (&Y)[7][Pb::D], const R (&p)[Pb::NP], R h, const R (&c)[Pb::D],
                                              R (&v)[Pb::D], RB& pbacc) {
  constexpr int D = Pb::D;
  // acc[l] = sum over the stages m already reversed of a_ml Ybar_m; stage 6 (the
  // first one reversed) starts every sum, so no zero is ever added.
  R acc[6][D];
#pragma unroll
  for (int q = 0; q < D; ++q) v[q] = c[q];
  // FP32 (not the network problems): components 0, 1 as FP32x2, the same
  // per-component IEEE operations
  constexpr bool PACK = std::is_same<R, float>::value && D >= 2 && !HasNet<Pb>::value;
  constexpr int Q0 = PACK ? 2 : 0;  // first component done one at a time
#pragma unroll
  for (int j = 5; j >= 0; --j) {
    R kb[D], yb[D];
    if constexpr (PACK) {
      const float2 bb = make_float2(tsit5::B(j), tsit5::B(j)), hh = make_float2(h, h), cc = make_float2(c[0], c[1]);
      const float2 k2 = (j == 5) ? __fmul2_rn(hh, __fmul2_rn(bb, cc))
                                 : __fmul2_rn(hh, __ffma2_rn(bb, cc, make_float2(acc[j][0], acc[j][1])));
      kb[0] = k2.x;
      kb[1] = k2.y;
    }
#pragma unroll
    for (int q = Q0; q < D; ++q)
      kb[q] = (j == 5) ? mul_(h, mul_(R(tsit5::B(j)), c[q])) : mul_(h, fma_(R(tsit5::B(j)), c[q], acc[j][q]));
    pbacc.template vjp<Pb>(Y[j], p, kb, yb);
    if constexpr (PACK) {
      const float2 v2 = __fadd2_rn(make_float2(v[0], v[1]), make_float2(yb[0], yb[1]));
      v[0] = v2.x;
      v[1] = v2.y;
    }
#pragma unroll
    for (int q = Q0; q < D; ++q) v[q] = add_(v[q], yb[q]);
#pragma unroll
    for (int l = 0; l < j; ++l) {
      if constexpr (PACK) {
        const float2 aa = make_float2(tsit5::A(j, l), tsit5::A(j, l)), y2 = make_float2(yb[0], yb[1]);
        const float2 a2 = (j == 5) ? __fmul2_rn(aa, y2) : __ffma2_rn(aa, y2, make_float2(acc[l][0], acc[l][1]));
        acc[l][0] = a2.x;
        acc[l][1] = a2.y;
      }
#pragma unroll
      for (int q = Q0; q < D; ++q)
        acc[l][q] = (j == 5) ? mul_(R(tsit5::A(j, l)), yb[q]) : fma_(R(tsit5::A(j, l)), yb[q], acc[l][q]);
    }
  }
  pbacc.flush();
}

// ---------------------------------------------------------------------------
// Verner7: Verner's "efficient" seventh-order pair with a sixth-order embedded
// formula (J. H. Verner, Numer. Algorithms 53 (2010) 383-396), the pair the
// paper cites for its higher-order engine (Sec. 5). The 7th-order solution
// uses stages 1..9 (c_9 = 1); stage 10 (c_10 = 1) feeds only the 6th-order
// embedded formula; a_i2 = 0 from stage 4 on and b_2 = b_3 = 0. Not FSAL:
// each step evaluates f(y). Coefficients to 40 significant digits as
// published (each rounds to the nearest double at compile time).
// ---------------------------------------------------------------------------
namespace vern7 {
__host__ __device__ constexpr double A(int i, int j) {
  // 0-based stage i (1..9), column j < i
  return (i == 1 && j == 0) ? 0.005
         : (i == 2 && j == 0) ? -1.076790123456790123456790123456790123457
         : (i == 2 && j == 1) ? 1.185679012345679012345679012345679012346
         : (i == 3 && j == 0) ? 0.04083333333333333333333333333333333333333
         : (i == 3 && j == 2) ? 0.1225
         : (i == 4 && j == 0) ? 0.6389139236255726780508121615993336109954
         : (i == 4 && j == 2) ? -2.455672638223656809662640566430653894211
         : (i == 4 && j == 3) ? 2.272258714598084131611828404831320283215
         : (i == 5 && j == 0) ? -2.661577375018757131119259297861818119279
         : (i == 5 && j == 2) ? 10.80451388645613769565396655365532838482
         : (i == 5 && j == 3) ? -8.353914657396199411968048547819291691541
         : (i == 5 && j == 4) ? 0.8204875949566569791420417341743839209619
         : (i == 6 && j == 0) ? 6.067741434696770992718360183877276714679
         : (i == 6 && j == 2) ? -24.71127363591108579734203485290746001803
         : (i == 6 && j == 3) ? 20.42751793078889394045773111748346612697
         : (i == 6 && j == 4) ? -1.906157978816647150624096784352757010879
         : (i == 6 && j == 5) ? 1.006172249242068014790040335899474187268
         : (i == 7 && j == 0) ? 12.05467007625320299509109452892778311648
         : (i == 7 && j == 2) ? -49.75478495046898932807257615331444758322
         : (i == 7 && j == 3) ? 41.14288863860467663259698416710157354209
         : (i == 7 && j == 4) ? -4.461760149974004185641911603484815375051
         : (i == 7 && j == 5) ? 2.042334822239174959821717077708608543738
         : (i == 7 && j == 6) ? -0.09834843665406107379530801693870224403537
         : (i == 8 && j == 0) ? 10.13814652288180787641845141981689030769
         : (i == 8 && j == 2) ? -42.64113603171750214622846006736635730625
         : (i == 8 && j == 3) ? 35.76384003992257007135021178023160054034
         : (i == 8 && j == 4) ? -4.348022840392907653340370296908245943710
         : (i == 8 && j == 5) ? 2.009862268377035895441943593011827554771
         : (i == 8 && j == 6) ? 0.3487490460338272405953822853053145879140
         : (i == 8 && j == 7) ? -0.2714390051048312842371587140910297407572
         : (i == 9 && j == 0) ? -45.03007203429867712435322405073769635151
         : (i == 9 && j == 2) ? 187.3272437654588840752418206154201997384
         : (i == 9 && j == 3) ? -154.0288236935018690596728621034510402582
         : (i == 9 && j == 4) ? 18.56465306347536233859492332958439136765
         : (i == 9 && j == 5) ? -7.141809679295078854925420496823551192821
         : (i == 9 && j == 6) ? 1.308808578161378625114762706007696696508
                              : 0.0;
}
__host__ __device__ constexpr double B(int j) {
  return j == 0 ? 0.04715561848627222170431765108838175679569
         : j == 3 ? 0.2575056429843415189596436101037687580986
         : j == 4 ? 0.2621665397741262047713863095764527711129
         : j == 5 ? 0.1521609265673855740323133199165117535523
         : j == 6 ? 0.4939969170032484246907175893227876844296
         : j == 7 ? -0.2943031171403250441557244744092703429139
         : j == 8 ? 0.08131747232495109999734599440136761892478
                  : 0.0;
}
__host__ __device__ constexpr double Bhat(int j) {
  return j == 0 ? 0.04460860660634117628731817597479197781432
         : j == 3 ? 0.2671640378571372680509102260943837899738
         : j == 4 ? 0.2201018300177293019979715776650753096323
         : j == 5 ? 0.2188431703143156830983120833512893824578
         : j == 6 ? 0.2289871705411202883378173889763552365362
         : j == 9 ? 0.02029518466335628222767054793810430358554
                  : 0.0;
}
__host__ __device__ constexpr double Btilde(int j) { return B(j) - Bhat(j); }  // error weights
}  // namespace vern7

// Stages of one Verner7 step from y with size h: stage inputs Y[0..NS-1]
// (Y[0] = y) and slopes K[0..NS-1], K[i] = f(Y[i]). NS = 9 gives what y_new
// needs; NS = 10 adds stage 10 for the error estimate. Zero coefficients are
// skipped.
template <class Pb, class R, int NS>
__device__ __forceinline__ void vern7_stages(const R (&y)[Pb::D], const R (&p)[Pb::NP], R h, R (&Y)[NS][Pb::D],
                                             R (&K)[NS][Pb::D]) {
  constexpr int D = Pb::D;
#pragma unroll
  for (int c = 0; c < D; ++c) Y[0][c] = y[c];
  Pb::f(y, p, K[0]);
#pragma unroll
  for (int i = 1; i < NS; ++i) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      R s = mul_(R(vern7::A(i, 0)), K[0][c]);
#pragma unroll
      for (int j = 1; j < i; ++j)
        if (vern7::A(i, j) != 0.0) s = fma_(R(vern7::A(i, j)), K[j][c], s);
      Y[i][c] = fma_(h, s, y[c]);
    }
    Pb::f(Y[i], p, K[i]);
  }
}

// y_new = y + h sum_{j<9} b_j k_j.
template <class Pb, class R, int NS>
__device__ __forceinline__ void vern7_update(const R (&y)[Pb::D], const R (&K)[NS][Pb::D], R h, R (&yn)[Pb::D]) {
#pragma unroll
  for (int c = 0; c < Pb::D; ++c) {
    R s = mul_(R(vern7::B(0)), K[0][c]);
#pragma unroll
    for (int j = 1; j < 9; ++j)
      if (vern7::B(j) != 0.0) s = fma_(R(vern7::B(j)), K[j][c], s);
    yn[c] = fma_(h, s, y[c]);
  }
}

// Embedded error estimate e = h sum_j (b_j - bhat_j) k_j (stages 2 and 3 have zero weight).
template <class Pb, class R>
__device__ __forceinline__ void vern7_error(const R (&K)[10][Pb::D], R h, R (&e)[Pb::D]) {
#pragma unroll
  for (int c = 0; c < Pb::D; ++c) {
    R s = mul_(R(vern7::Btilde(0)), K[0][c]);
#pragma unroll
    for (int j = 1; j < 10; ++j)
      if (vern7::Btilde(j) != 0.0) s = fma_(R(vern7::Btilde(j)), K[j][c], s);
    e[c] = mul_(h, s);
  }
}

// Forward mode of one Verner7 step with h held as data: y_new (the arithmetic
// of vern7_stages + vern7_update over nine stages) and, for each of ND tangent
// directions (yd, pd), yd_new from the stage tangents
// Yd_i = yd + h sum_j a_ij Kd_j, Kd_i = J(Y_i) Yd_i + f_theta(Y_i) pd.
template <class Pb, int ND>
__device__ __forceinline__ void vern7_tangent(const double (&y)[Pb::D], const double (&yd)[ND][Pb::D],
                                              const double (&p)[Pb::NP], const double (&pd)[ND][Pb::NP], double h,
                                              double (&yn)[Pb::D], double (&ydn)[ND][Pb::D]) {
  constexpr int D = Pb::D;
  double K[9][D], Kd[9][ND][D];
  Pb::f(y, p, K[0]);
#pragma unroll
  for (int q = 0; q < ND; ++q) Pb::jvp(y, p, yd[q], pd[q], Kd[0][q]);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    double Y[D], Yd[ND][D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double s = mul_(vern7::A(i, 0), K[0][c]);
#pragma unroll
      for (int j = 1; j < i; ++j)
        if (vern7::A(i, j) != 0.0) s = fma_(vern7::A(i, j), K[j][c], s);
      Y[c] = fma_(h, s, y[c]);
    }
#pragma unroll
    for (int q = 0; q < ND; ++q)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double s = mul_(vern7::A(i, 0), Kd[0][q][c]);
#pragma unroll
        for (int j = 1; j < i; ++j)
          if (vern7::A(i, j) != 0.0) s = fma_(vern7::A(i, j), Kd[j][q][c], s);
        Yd[q][c] = fma_(h, s, yd[q][c]);
      }
    Pb::f(Y, p, K[i]);
#pragma unroll
    for (int q = 0; q < ND; ++q) Pb::jvp(Y, p, Yd[q], pd[q], Kd[i][q]);
  }
  vern7_update<Pb, double, 9>(y, K, h, yn);
#pragma unroll
  for (int q = 0; q < ND; ++q)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double s = mul_(vern7::B(0), Kd[0][q][c]);
#pragma unroll
      for (int j = 1; j < 9; ++j)
        if (vern7::B(j) != 0.0) s = fma_(vern7::B(j), Kd[j][q][c], s);
      ydn[q][c] = fma_(h, s, yd[q][c]);
    }
}

// Reverse of one Verner7 step over its stage inputs Y[0..8]: given
// the cotangent c of y_new returns v = dL/dy and accumulates dL/dtheta.
// kbar_j = h (b_j c + sum_{m>j} a_mj Ybar_m), Ybar_j = J(Y_j)^T kbar_j,
// theta_bar += f_theta(Y_j)^T kbar_j, v = c + sum_j Ybar_j. acc[l] holds
// sum over the stages already reversed of a_ml Ybar_m; stage 9 starts it.
template <class Pb, class R, int NY, class RB>
__device__ __forceinline__ void vern7_reverse(const R (&Y)[NY][Pb::D], const R (&p)[Pb::NP], R h, const R (&c)[Pb::D],
                                              R (&v)[Pb::D], RB& pbacc) {
  static_assert(NY >= 9, "the reverse reads stage inputs Y[0..8]");
  constexpr int D = Pb::D;
  R acc[8][D];
#pragma unroll
  for (int q = 0; q < D; ++q) v[q] = c[q];
#pragma unroll
  for (int j = 8; j >= 0; --j) {
    R kb[D], yb[D];
#pragma unroll
    for (int q = 0; q < D; ++q) {
      if (j == 8)
        kb[q] = mul_(h, mul_(R(vern7::B(j)), c[q]));
      else if (vern7::B(j) == 0.0)
        kb[q] = mul_(h, acc[j][q]);
      else
        kb[q] = mul_(h, fma_(R(vern7::B(j)), c[q], acc[j][q]));
    }
    pbacc.template vjp<Pb>(Y[j], p, kb, yb);
#pragma unroll
    for (int q = 0; q < D; ++q) v[q] = add_(v[q], yb[q]);
#pragma unroll
    for (int l = 0; l < j; ++l) {
      // column l of row j: the first nonzero entry met (largest j) starts acc[l]
      if (vern7::A(j, l) == 0.0) continue;
      bool first = true;
#pragma unroll
      for (int m = 8; m > j; --m)
        if (vern7::A(m, l) != 0.0) first = false;
#pragma unroll
      for (int q = 0; q < D; ++q)
        acc[l][q] = first ? mul_(R(vern7::A(j, l)), yb[q]) : fma_(R(vern7::A(j, l)), yb[q], acc[l][q]);
    }
  }
  pbacc.flush();
}

// Parameter-gradient accumulators: plain (FP64) and compensated (FP32-mixed,
// Neumaier's variant of Kahan summation).
// vjp<Pb>(y, p, v, yb): yb = J(y)^T v and accumulates f_theta(y)^T v;
// flush(): called once at the end of each unit's reverse (the compensated form
// sums a unit's stage contributions plainly and adds the unit's total to the
// running sum with compensation).
template <int NP>
struct PlainAcc {
  double s[NP];
  __device__ void zero() {
#pragma unroll
    for (int q = 0; q < NP; ++q) s[q] = 0.0;
  }
  template <class Pb>
  __device__ __forceinline__ void vjp(const double (&y)[Pb::D], const double (&p)[NP], const double (&v)[Pb::D],
                                      double (&yb)[Pb::D]) {
    Pb::vjp(y, p, v, yb, s);  // FP64: accumulate straight into the sums
  }
  // gy += d/dy (r^T J(y) u), theta_bar += d/dtheta (r^T J u)
  template <class Pb>
  __device__ __forceinline__ void jac_contract(const double (&y)[Pb::D], const double (&p)[NP],
                                               const double (&r)[Pb::D], const double (&u)[Pb::D],
                                               double (&gy)[Pb::D]) {
    Pb::jac_contract(y, p, r, u, gy, s);
  }
  __device__ __forceinline__ void flush() {}
  __device__ double get(int q) const { return s[q]; }
};
template <int NP>
struct CompensatedAcc {
  float s[NP], comp[NP], u[NP];  // running sum, its compensation, this unit's partial
  __device__ void zero() {
#pragma unroll
    for (int q = 0; q < NP; ++q) s[q] = comp[q] = u[q] = 0.0f;
  }
  template <class Pb>
  __device__ __forceinline__ void vjp(const float (&y)[Pb::D], const float (&p)[NP], const float (&v)[Pb::D],
                                      float (&yb)[Pb::D]) {
    Pb::vjp(y, p, v, yb, u);
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const float x = u[q], t = add_(s[q], x);
      comp[q] = add_(comp[q], (fabsf(s[q]) >= fabsf(x)) ? add_(sub_(s[q], t), x) : add_(sub_(x, t), s[q]));
      s[q] = t;
      u[q] = 0.0f;
    }
  }
  __device__ double get(int q) const { return (double)s[q] + (double)comp[q] + (double)u[q]; }
};

// ---------------------------------------------------------------------------
// Step-size control (FP64 for t, h and the error test).
// ---------------------------------------------------------------------------

// Hardware base-2 logarithm and exponential (PTX lg2.approx / ex2.approx).
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Weighted RMS error test of the paper's Sec. 2.1, as a mean square:
// q = (1/D) sum_c (e_c / (atol + rtol max(|y_c|, |ynew_c|)))^2; accept iff q <= 1.
// Each ratio is formed to FP32 accuracy (relative error below 1e-6 in q) and
// the squares are summed in FP64: q decides accept / reject and scales the
// next step, and never enters the accepted solution. The FP64 error e is
// computed in FP64 (its terms cancel); the ratio's scale and reciprocal run on
// the FP32 pipe with the bit-level conversions, leaving one FP64 FMA per
// component. Components whose scale or state lies outside the range where
// that is accurate (scale below 1e-30, |y| above 1e30) take the FP64 division.
template <int D>
__device__ __forceinline__ double err_meansq(const double (&e)[D], const double (&y)[D], const double (&yn)[D],
                                             double rtol, double atol, float rt, float at) {
  constexpr unsigned long long BITS_1E30 = 0x46293e5939a08ceaull;  // 1e30
  double q = 0.0;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const double m = max_abs(y[c], yn[c]);
    const float sc = fmaf(rt, to_f(m), at);
    double r;
    if (dbits(m) < BITS_1E30 && sc >= 1e-30f) {
      r = to_d(__fmul_rn(to_f(e[c]), __frcp_rn(sc)));
    } else {
      r = e[c] / fma_(rtol, m, atol);
    }
    q = fma_(r, r, q);
  }
  return mul_(q, 1.0 / D);
}
// FP32-mixed form: the error, y and y_new are FP32 stage values, so the whole
// norm is formed in FP32: each ratio e_c / sc_c (scale with an IEEE
// reciprocal), the sum of squares and the mean (relative error ~1e-7, below
// the 1e-6 the ratios already carry). A ratio beyond 1e18 is clamped there so
// that the square stays finite (any error that large gives the controller's
// minimum factor either way); a NaN passes through. No FP64 instruction.
template <int D>
__device__ __forceinline__ double err_meansq(const float (&e)[D], const float (&y)[D], const float (&yn)[D],
                                             double, double, float rt, float at) {
  float q = 0.0f;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const float sc = fmaf(rt, fmaxf(fabsf(y[c]), fabsf(yn[c])), at);
    float r = __fmul_rn(e[c], __frcp_rn(sc));
    r = (fabsf(r) > 1e18f) ? 1e18f : r;
    q = __fmaf_rn(r, r, q);
  }
  return to_d(__fmul_rn(q, 1.0f / D));
}

// Integral-controller factor from the mean-square error q = err^2, for an
// error estimate of lower order Q: clamp(0.9 err^(-1/(Q+1)), 0.2, 10) =
// clamp(0.9 q^(-1/(2(Q+1))), 0.2, 10) (Q = 4: Tsit5, Rodas5P; Q = 2:
// Rosenbrock23); q = 0 gives 10. FP32 with the hardware log2 / exp2: the factor
// only scales the next trial step.
template <int Q>
__device__ __forceinline__ float ctrl_factor(double q) {
  constexpr float EXPO = -0.5f / (Q + 1);
  if (!positive(q)) return 10.0f;
  const float f = __fmul_rn(0.9f, ex2_approx(__fmul_rn(EXPO, lg2_approx(to_f(q)))));
  return fminf(10.0f, fmaxf(0.2f, f));
}

// Starting step: the algorithm of Hairer, Norsett & Wanner, Vol. I, Sec. II.4
// (the method's order p, the weighted RMS norm, one explicit Euler probe),
// evaluated in FP32 from y0, theta and f(y0): it only picks the first trial
// step. Returns a non-finite value if the inputs overflow FP32.
template <class Pb, int ORDER>
__device__ __forceinline__ double initial_step_f32(const float (&y0)[Pb::D], const float (&p)[Pb::NP],
                                                   const float (&f0)[Pb::D], double t0, double t1, double rtol,
                                                   double atol) {
  constexpr int D = Pb::D;
  float sc[D], y1[D], f1[D];
  const float rt = (float)rtol, at = (float)atol, span = (float)(t1 - t0);
  float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    sc[c] = fmaf(rt, fabsf(y0[c]), at);
    const float r0 = y0[c] / sc[c], r1 = f0[c] / sc[c];
    d0 = fmaf(r0, r0, d0);
    d1 = fmaf(r1, r1, d1);
  }
  d0 = sqrtf(d0 / D);
  d1 = sqrtf(d1 / D);
  float h0 = (d0 < 1e-5f || d1 < 1e-5f) ? 1e-6f : 0.01f * d0 / d1;
  h0 = fminf(h0, span);
#pragma unroll
  for (int c = 0; c < D; ++c) y1[c] = fmaf(h0, f0[c], y0[c]);
  Pb::f(y1, p, f1);
  float d2 = 0.0f;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const float r = (f1[c] - f0[c]) / sc[c];
    d2 = fmaf(r, r, d2);
  }
  d2 = sqrtf(d2 / D) / h0;
  const float dm = fmaxf(d1, d2);
  const float h1 =
      (dm <= 1e-15f) ? fmaxf(1e-6f, h0 * 1e-3f) : ex2_approx(lg2_approx(0.01f / dm) * (1.0f / (ORDER + 1)));
  return (double)fminf(fminf(100.0f * h0, h1), span);
}

// ---------------------------------------------------------------------------
// FP64 step control (GS_CONTROL_FP64): the error norm, the accept test, the
// controller factor and the starting step evaluated in FP64 (the paper's
// Sec. 2.1 norm and accept test; Hairer, Norsett & Wanner I, Sec. II.4 for the
// starting step). The record works with the mean square m of the scaled error
// instead of err = sqrt(m): the accept test is the exact equivalent of
// sqrt(m) <= 1. Reciprocals and the controller's root come from
// single-precision estimates refined by one FP64 Newton step, to about 1e-14
// and 1e-12 relative: far below the ~1e-7 relative difference that the
// rounding of the stage sums already makes in the error estimate of two codes
// (the error estimate cancels), so the mesh follows a plain CPU evaluation of
// the same rule up to that rounding.
// ---------------------------------------------------------------------------

// Bit patterns of positive doubles order as their values: range tests and
// clamps of positive values run on the integer pipe.
constexpr unsigned long long DBITS_1EM30 = 0x39b4484bfeebc2a0ull;  // 1e-30
constexpr unsigned long long DBITS_1E30 = 0x46293e5939a08ceaull;   // 1e30
constexpr unsigned long long DBITS_0P2 = 0x3fc999999999999aull;    // 0.2
constexpr unsigned long long DBITS_TEN = 0x4024000000000000ull;    // 10
__device__ __forceinline__ double clamp_pos_bits(double x, unsigned long long lo, unsigned long long hi) {
  const unsigned long long b = dbits(x);  // x > 0
  return __longlong_as_double((long long)(b < lo ? lo : (b > hi ? hi : b)));
}

// 1/x for 1e-30 < |x| < 1e30: the correctly rounded single-precision
// reciprocal (relative error <= 2^-24) and one Newton step x0 + x0 (1 - x x0),
// which squares the relative error; IEEE division outside that range.
__device__ __forceinline__ double rcp_f64(double x) {
  const unsigned long long ax = abs_bits(x);
  if (!(ax > DBITS_1EM30 && ax < DBITS_1E30)) return __ddiv_rn(1.0, x);
  const double x0 = (double)__frcp_rn((float)x);
  return fma_(x0, fma_(-x, x0, 1.0), x0);
}

// m = (1/D) sum_c (e_c / (atol + rtol max(|y_c|, |ynew_c|)))^2 (err = sqrt(m));
// the scale with one rounding (a fused multiply-add).
template <int D, class R>
__device__ __forceinline__ double err_meansq_f64(const R (&e)[D], const R (&y)[D], const R (&yn)[D], double rtol,
                                                 double atol) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const double sc = fma_(rtol, max_abs(to_d(y[c]), to_d(yn[c])), atol);
    const double r = mul_(to_d(e[c]), rcp_f64(sc));
    s = fma_(r, r, s);
  }
  return mul_(s, 1.0 / D);
}

// sqrt(m) <= 1 with sqrt correctly rounded: m <= 1 + 2^-52 (the square root of
// the next double after 1 rounds back to 1; of the one after that, it does not).
// NaN rejects.
__device__ __forceinline__ bool rms_le_one(double m) { return dbits(m) <= DBITS_ONE + 1ull; }

template <int K>
__device__ __forceinline__ double ipow_(double y) {  // y^K by repeated squaring
  if constexpr (K == 1)
    return y;
  else if constexpr (K % 2 == 0) {
    const double h = ipow_<K / 2>(y);
    return mul_(h, h);
  } else
    return mul_(ipow_<K - 1>(y), y);
}

// Controller factor from the mean square m: clamp(0.9 m^(-1/K), 0.2, 10), K =
// 2(Q+1), i.e. 0.9 err^(-1/(Q+1)); m = 0 gives 10. m^(-1/K) is the positive
// root of g(y) = m y^K - 1: Newton's method, y <- y + y (1 - m y^K) / K, from a
// single-precision estimate (relative error ~3e-7); the step squares the error
// and scales it by about (K+1)/2, to ~5e-13 (checked over m in [1e-12, 1e7]).
// Outside [1e-30, 1e30] the factor is clamped whatever m is, so m is held to
// that range first.
template <int Q>
__device__ __forceinline__ double ctrl_factor_ms_f64(double m) {  // m >= 0, not NaN
  constexpr int K = 2 * (Q + 1);
  if (!positive(m)) return 10.0;
  const double mc = clamp_pos_bits(m, DBITS_1EM30, DBITS_1E30);
  double y = (double)exp2f(log2f((float)mc) * (-1.0f / K));
  y = fma_(y, mul_(fma_(-mc, ipow_<K>(y), 1.0), 1.0 / K), y);
  return clamp_pos_bits(mul_(0.9, y), DBITS_0P2, DBITS_TEN);
}

// RMS of v_c / sc_c.
template <int D>
__device__ __forceinline__ double rms_scaled_f64(const double (&v)[D], const double (&sc)[D]) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const double r = __ddiv_rn(v[c], sc[c]);
    s = add_(s, mul_(r, r));
  }
  return __dsqrt_rn(__ddiv_rn(s, (double)D));
}

// Starting step (Hairer, Norsett & Wanner I, Sec. II.4) in FP64 from y0, theta
// and f(y0): d0 = ||y0||, d1 = ||f0||, h0 = 0.01 d0 / d1 (1e-6 if either is
// below 1e-5), one explicit Euler probe y1 = y0 + h0 f0, d2 = ||f(y1) - f0|| / h0,
// h1 = (0.01 / max(d1, d2))^(1/(p+1)) (max(1e-6, 1e-3 h0) if that max is at most
// 1e-15), h = min(100 h0, h1, t1 - t0); the norm is the weighted RMS with
// scale atol + rtol |y0_c|.
template <class Pb, int ORDER>
__device__ __forceinline__ double initial_step_f64(const double (&y0)[Pb::D], const double (&p)[Pb::NP],
                                                   const double (&f0)[Pb::D], double t0, double t1, double rtol,
                                                   double atol) {
  constexpr int D = Pb::D;
  double sc[D], y1[D], f1[D], df[D];
#pragma unroll
  for (int c = 0; c < D; ++c) sc[c] = add_(atol, mul_(rtol, fabs(y0[c])));
  const double d0 = rms_scaled_f64<D>(y0, sc), d1 = rms_scaled_f64<D>(f0, sc);
  const double span = sub_(t1, t0);
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : __ddiv_rn(mul_(0.01, d0), d1);
  h0 = fmin(h0, span);
#pragma unroll
  for (int c = 0; c < D; ++c) y1[c] = add_(y0[c], mul_(h0, f0[c]));
  Pb::f(y1, p, f1);
#pragma unroll
  for (int c = 0; c < D; ++c) df[c] = sub_(f1[c], f0[c]);
  const double d2 = __ddiv_rn(rms_scaled_f64<D>(df, sc), h0);
  const double dm = fmax(d1, d2);
  const double h1 = (dm <= 1e-15) ? fmax(1e-6, mul_(h0, 1e-3)) : pow(__ddiv_rn(0.01, dm), 1.0 / (ORDER + 1));
  return fmin(fmin(mul_(100.0, h0), h1), span);
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Warp-aggregated ticket: every lane with `want` gets a distinct value of
// *ctr (post-increment), with one atomic per warp. Must be called by all 32
// lanes together.
__device__ __forceinline__ long long warp_ticket(unsigned long long* ctr, bool want) {
  const unsigned mask = __ballot_sync(FULL_MASK, want);
  if (mask == 0u) return -1;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane_id() == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
  base = __shfl_sync(FULL_MASK, base, leader);
  const int rank = __popc(mask & ((1u << lane_id()) - 1u));
  return want ? (long long)(base + rank) : -1;
}

}  // namespace gs
