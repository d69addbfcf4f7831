// The persistent record and reverse-sweep kernels, generic over the one-step
// method (Tsit5 and Verner7 for non-stiff problems, Rodas5P and Rosenbrock23
// for stiff ones).
//
// Both kernels are persistent: a grid of resident CTAs whose lanes each own one
// trajectory at a time and take the next one from a global ticket counter
// (one atomic per warp per refill) as soon as theirs finishes, so a lane never
// waits for a slower neighbour's trajectory to end. Each loop iteration first
// does the lane's bookkeeping (refill, record write-out, the walk through its
// record), then meets the warp at a __syncwarp and runs one unit of solver
// arithmetic as a single block, so the floating-point work of all busy lanes
// issues together whatever phase their trajectories are in.
//
// Record (paper Sec. 3.1, map R): the adaptive loop of Sec. 2.1 with the
// weighted RMS error test and an integral controller. Accepted step sizes are
// staged per lane in shared memory and written out as fixed-size record
// segments [prev, t_start, y_start[d], h[k]] (one vector-stored segment per k
// accepted steps; with stored stages, k = 1 and the step's stage data follow
// h) allocated from a device arena in per-warp blocks of slots.
//
// Reverse (paper Sec. 3.1, discrete adjoint of Eq. (replay)): each lane walks
// its trajectory's segments last to first and runs one unit per iteration: a
// state recompute inside a segment (k > 1 only), a step VJP
// (lambda_{i-1} = dPhi/dy^T lambda_i), or a save-time side-step VJP
// (lambda_i += dPhi/dy^T ybar_s).
//
// A Method provides Carry (state carried between accepted steps), start (the
// carry and f(y0) for the starting step), trial (one trial step: y_new and the
// error estimate; false if the step's linear system is singular), side (one
// step of a given size from an accepted state) and unit (the reverse unit);
// with kStages also StageData, its payload sizes, trial_s, pack, unpack and
// unit_stored (the stored-stage record and reverse unit).
#pragma once

#include <cstring>
#include <type_traits>

#include "gs_device.cuh"
#include "gs_internal.h"
#include "gs_rodas.cuh"
#include "gs_ude.cuh"
#include "gs_nrob.cuh"

namespace gs {

// Problems with shared network weights (the LV UDE): weights staged per CTA,
// trajectories assigned to lanes statically (so the per-warp weight-gradient
// sums are reproducible), and warp-collective reverse units.
template <class Pb, class = void>
struct HasWeights : std::false_type {};
template <class Pb>
struct HasWeights<Pb, std::void_t<decltype(Pb::kWeights)>> : std::integral_constant<bool, Pb::kWeights> {};
// Problems whose reverse-sweep units run CTA-collectively (all 128 lanes of a
// CTA in lockstep: the tensor-core network of LvUdeCta).
template <class Pb, class = void>
struct CtaColl : std::false_type {};
template <class Pb>
struct CtaColl<Pb, std::void_t<decltype(Pb::kCta)>> : std::integral_constant<bool, Pb::kCta> {};

constexpr int TPB_FWD = 128;
constexpr int TPB_REV = 128;



enum : int { U_NONE = 0, U_RECOMP = 1, U_STEP = 2, U_SIDE = 3, U_DONE = 4, U_FAIL = 5 };

__device__ __forceinline__ double nan_d() { return __longlong_as_double(0x7ff8000000000000LL); }

// Cotangent of a unit: the lambda of a step unit, or the save-time cotangent of
// a side unit (the user's, or 2 y(t_s) for the built-in loss, whose value the
// unit adds to the loss).
template <class Pb, class R, bool USER_COT>
__device__ __forceinline__ void unit_cotangent(const RevArgs& a, long long k, bool active, bool side, int us,
                                               const R (&ynew)[Pb::D], const R (&lam)[Pb::D], R (&cv)[Pb::D],
                                               double& loss) {
  constexpr int D = Pb::D;
  R l2 = R(0);  // ||y(t_s)||^2 in the unit's precision; only side units add it to the FP64 loss
#pragma unroll
  for (int c = 0; c < D; ++c) {
    R cs = R(0);
    if (USER_COT) {
      if (active && side) cs = to_r<R>(a.y_save_bar[((long long)us * D + c) * a.n + k]);
    } else {
      cs = add_(ynew[c], ynew[c]);  // d/dy of ||y||^2
      l2 = fma_(ynew[c], ynew[c], l2);
    }
    cv[c] = active ? (side ? cs : lam[c]) : R(0);
  }
  if (!USER_COT && active && side) loss = acc_loss(loss, l2);
}

// ---------------------------------------------------------------------------
// Methods
// ---------------------------------------------------------------------------
struct Tsit5Method {
  static constexpr int ORDER = 5, ERR_ORDER = 4;  // solution order; lower order of the error estimate
  static constexpr bool kStages = true;           // records may store stage inputs
  static constexpr bool kControl64 = true;        // record kernels with FP64 step control
  static constexpr int REV_MINB_F32 = 8, REV_MINB_STAGES = 5;  // reverse-sweep register caps (see rev_min_blocks)
  // Step of the lanes without work in a warp-collective unit (zero cotangent):
  // any value whose step stays finite.
  static constexpr double IDLE_H = 0.0;
  template <class Pb, class R>
  struct Carry {
    R k1[Pb::D];  // FSAL: f(y) of the current accepted state
  };
  static constexpr bool kCarryIsF = true;  // the carry is f(y) (start() computes it)
  template <class Pb, class R, class Get>
  __device__ __forceinline__ static void set_carry_f(Carry<Pb, R>& cy, Get f) {
#pragma unroll
    for (int c = 0; c < Pb::D; ++c) cy.k1[c] = f(c);
  }
  template <class Pb, class R>
  __device__ __forceinline__ static R carry_f(const Carry<Pb, R>& cy, int c) {
    return cy.k1[c];
  }
  template <class Pb, class R>
  __device__ __forceinline__ static void start(const R (&y)[Pb::D], const R (&p)[Pb::NP], Carry<Pb, R>& cy,
                                               float (&f0)[Pb::D]) {
    Pb::f(y, p, cy.k1);
#pragma unroll
    for (int c = 0; c < Pb::D; ++c) f0[c] = (float)cy.k1[c];
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool trial(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                               const Carry<Pb, R>& cy, R (&ynew)[Pb::D], R (&e)[Pb::D],
                                               Carry<Pb, R>& next) {
    constexpr int D = Pb::D;
    R Y[7][D], K[7][D];
#pragma unroll
    for (int c = 0; c < D; ++c) K[0][c] = cy.k1[c];
    tsit5_stages<Pb, R, 7>(y, p, to_r<R>(h), Y, K);
    tsit5_error<Pb, R>(K, to_r<R>(h), e);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      ynew[c] = Y[6][c];
      next.k1[c] = K[6][c];
    }
    return true;
  }
  // ---- stored stages (records that keep every step's stage inputs)
  // A step stores Y_1..Y_5 (Y_0 is the segment's state); a side step also Y_6,
  // its save state.
  template <class Pb, class R>
  struct StageData {
    R Y[7][Pb::D];
  };
  template <int D>
  static constexpr int step_payload() {
    return 5 * D;
  }
  template <int D>
  static constexpr int side_payload() {
    return 6 * D;
  }
  // The trial step that also returns its stage data.
  template <class Pb, class R>
  __device__ __forceinline__ static bool trial_s(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                                 const Carry<Pb, R>& cy, R (&ynew)[Pb::D], R (&e)[Pb::D],
                                                 Carry<Pb, R>& next, StageData<Pb, R>& sd) {
    constexpr int D = Pb::D;
    R K[7][D];
#pragma unroll
    for (int c = 0; c < D; ++c) K[0][c] = cy.k1[c];
    tsit5_stages<Pb, R, 7>(y, p, to_r<R>(h), sd.Y, K);
    tsit5_error<Pb, R>(K, to_r<R>(h), e);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      ynew[c] = sd.Y[6][c];
      next.k1[c] = K[6][c];
    }
    return true;
  }
  template <class Pb, class R, class W>
  __device__ __forceinline__ static void pack(const StageData<Pb, R>& sd, bool side, W&& write) {
    constexpr int D = Pb::D;
#pragma unroll
    for (int j = 1; j < 7; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (j < 6 || side) write((j - 1) * D + c, to_d(sd.Y[j][c]));
  }
  template <class Pb, class R, class Rd>
  __device__ __forceinline__ static void unpack(bool side, const R (&x)[Pb::D], Rd&& read, StageData<Pb, R>& sd) {
    constexpr int D = Pb::D;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      sd.Y[0][c] = x[c];
      sd.Y[6][c] = x[c];  // replaced below for a side step; a step unit does not use it
    }
#pragma unroll
    for (int j = 1; j < 7; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (j < 6 || side) sd.Y[j][c] = to_r<R>(read((j - 1) * D + c));
  }
  // Reverse unit over stored stage data: no stage is recomputed. Same
  // arithmetic as unit().
  template <class Pb, class R, bool USER_COT, class Acc>
  __device__ __forceinline__ static bool unit_stored(const RevArgs& a, long long k, int mode, bool active, int us,
                                                     const R (&x)[Pb::D], double h, const R (&p)[Pb::NP],
                                                     const StageData<Pb, R>& sd, R (&lam)[Pb::D], Acc& pacc,
                                                     double& loss) {
    constexpr int D = Pb::D;
    const bool side = (mode == U_SIDE);
    R cv[D], v[D];
    unit_cotangent<Pb, R, USER_COT>(a, k, active, side, us, sd.Y[6], lam, cv, loss);
    tsit5_reverse<Pb, R>(sd.Y, p, to_r<R>(h), cv, v, pacc);
#pragma unroll
    for (int c = 0; c < D; ++c) lam[c] = !active ? lam[c] : (side ? add_(lam[c], v[c]) : v[c]);
    return true;
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool side(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                              const Carry<Pb, R>& cy, R (&ys)[Pb::D]) {
    constexpr int D = Pb::D;
    R Y[7][D], K[7][D];
#pragma unroll
    for (int c = 0; c < D; ++c) K[0][c] = cy.k1[c];
    tsit5_stages<Pb, R, 6>(y, p, to_r<R>(h), Y, K);
#pragma unroll
    for (int c = 0; c < D; ++c) ys[c] = Y[6][c];
    return true;
  }
  // One step of the replay chain, y_new = Phi(y; h) (no carried state).
  template <class Pb, class R>
  __device__ __forceinline__ static bool replay_step(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                                     R (&ynew)[Pb::D]) {
    constexpr int D = Pb::D;
    R Y[7][D], K[7][D];
    Pb::f(y, p, K[0]);
    tsit5_stages<Pb, R, 6>(y, p, to_r<R>(h), Y, K);
#pragma unroll
    for (int c = 0; c < D; ++c) ynew[c] = Y[6][c];
    return true;
  }
  // Reverse unit: stages from x with step h; a step unit replaces lambda with
  // dPhi/dy^T lambda, a side unit adds dPhi/dy^T ybar_s. Returns y_new in ynew.
  // `active` is false only for the lanes without work that join a
  // warp-collective unit (shared-weight problems); they run with h = 0 and a
  // zero cotangent and change nothing.
  template <class Pb, class R, bool USER_COT, class Acc>
  __device__ __forceinline__ static bool unit(const RevArgs& a, long long k, int mode, bool active, int us,
                                              const R (&x)[Pb::D], double h, const R (&p)[Pb::NP], R (&lam)[Pb::D],
                                              Acc& pacc, double& loss, R (&ynew)[Pb::D]) {
    constexpr int D = Pb::D;
    R Y[7][D], K[7][D];
    Pb::f(x, p, K[0]);
    tsit5_stages<Pb, R, 6>(x, p, to_r<R>(h), Y, K);
#pragma unroll
    for (int c = 0; c < D; ++c) ynew[c] = Y[6][c];
    if (mode == U_RECOMP) return true;
    const bool side = (mode == U_SIDE);
    R cv[D], v[D];
    unit_cotangent<Pb, R, USER_COT>(a, k, active, side, us, ynew, lam, cv, loss);
    tsit5_reverse<Pb, R>(Y, p, to_r<R>(h), cv, v, pacc);
#pragma unroll
    for (int c = 0; c < D; ++c) lam[c] = !active ? lam[c] : (side ? add_(lam[c], v[c]) : v[c]);
    return true;
  }
};

#ifndef GS_RODAS_REV_MINB_STAGES
#define GS_RODAS_REV_MINB_STAGES 0
#endif
#ifndef GS_VERN7_REV_MINB_STAGES
#define GS_VERN7_REV_MINB_STAGES 0
#endif
struct Rodas5PMethod {  // FP64 only: the stiff W-matrix LU and its solves stay FP64
  static constexpr bool kControl64 = false;
  static constexpr int REV_MINB_F32 = 0, REV_MINB_STAGES = GS_RODAS_REV_MINB_STAGES;
  static constexpr int ORDER = 5, ERR_ORDER = 4;
  static constexpr bool kStages = true;
  template <class Pb, class R>
  struct Carry {};
  static constexpr bool kCarryIsF = false;
  // ---- stored stages: a step stores U_0..U_7 and the LU of W (factors, pivot
  // reciprocals, pivots). The stage inputs Y_i = y + sum_j a_ij U_j and the
  // new state are rebuilt from them by the same operations as the step.
  template <class Pb, class R>
  struct StageData {
    double Y[8][Pb::D], U[8][Pb::D], LU[Pb::D][Pb::D], rinv[Pb::D], ynew[Pb::D];
    int piv[Pb::D];
  };
  template <int D>
  static constexpr int step_payload() {
    return 8 * D + D * D + 2 * D;
  }
  template <int D>
  static constexpr int side_payload() {
    return step_payload<D>();
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool trial_s(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                                 const Carry<Pb, R>&, R (&ynew)[Pb::D], R (&e)[Pb::D],
                                                 Carry<Pb, R>&, StageData<Pb, R>& sd) {
    constexpr int D = Pb::D;
    const bool ok = rodas_step<Pb>(y, p, h, sd.Y, sd.U, sd.LU, sd.piv, sd.rinv, ynew);
#pragma unroll
    for (int c = 0; c < D; ++c) e[c] = sd.U[7][c];
    return ok;
  }
  template <class Pb, class R, class W>
  __device__ __forceinline__ static void pack(const StageData<Pb, R>& sd, bool, W&& write) {
    constexpr int D = Pb::D;
    int i = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c) write(i++, sd.U[j][c]);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) write(i++, sd.LU[r][c]);
#pragma unroll
    for (int c = 0; c < D; ++c) write(i++, sd.rinv[c]);
#pragma unroll
    for (int c = 0; c < D; ++c) write(i++, (double)sd.piv[c]);
  }
  template <class Pb, class R, class Rd>
  __device__ __forceinline__ static void unpack(bool side, const R (&x)[Pb::D], Rd&& read, StageData<Pb, R>& sd) {
    constexpr int D = Pb::D;
    int i = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c) sd.U[j][c] = read(i++);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) sd.LU[r][c] = read(i++);
#pragma unroll
    for (int c = 0; c < D; ++c) sd.rinv[c] = read(i++);
#pragma unroll
    for (int c = 0; c < D; ++c) sd.piv[c] = (int)read(i++);
    rodas_stage_inputs<D>(x, sd.U, sd.Y);
#pragma unroll
    for (int c = 0; c < D; ++c) sd.ynew[c] = side ? add_(sd.Y[7][c], sd.U[7][c]) : x[c];
  }
  template <class Pb, class R, bool USER_COT, class Acc>
  __device__ __forceinline__ static bool unit_stored(const RevArgs& a, long long k, int mode, bool active, int us,
                                                     const R (&x)[Pb::D], double h, const R (&p)[Pb::NP],
                                                     const StageData<Pb, R>& sd, R (&lam)[Pb::D], Acc& pacc,
                                                     double& loss) {
    constexpr int D = Pb::D;
    const bool side = (mode == U_SIDE);
    double cv[D], v[D];
    unit_cotangent<Pb, R, USER_COT>(a, k, active, side, us, sd.ynew, lam, cv, loss);
    rodas_reverse<Pb>(x, p, h, sd.Y, sd.U, sd.LU, sd.piv, sd.rinv, cv, v, pacc);
#pragma unroll
    for (int c = 0; c < D; ++c) lam[c] = !active ? lam[c] : (side ? add_(lam[c], v[c]) : v[c]);
    return true;
  }
  static constexpr double IDLE_H = 1.0;  // W = I/(h gamma) - J needs h != 0
  template <class Pb, class R>
  __device__ __forceinline__ static void start(const R (&y)[Pb::D], const R (&p)[Pb::NP], Carry<Pb, R>&,
                                               float (&f0)[Pb::D]) {
    R f[Pb::D];
    Pb::f(y, p, f);
#pragma unroll
    for (int c = 0; c < Pb::D; ++c) f0[c] = (float)f[c];
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool trial(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                               const Carry<Pb, R>&, R (&ynew)[Pb::D], R (&e)[Pb::D],
                                               Carry<Pb, R>&) {
    static_assert(std::is_same<R, double>::value, "Rodas5P runs in FP64");
    constexpr int D = Pb::D;
    double Y[8][D], U[8][D], LU[D][D], rinv[D];
    int piv[D];
    const bool ok = rodas_step<Pb>(y, p, h, Y, U, LU, piv, rinv, ynew);
#pragma unroll
    for (int c = 0; c < D; ++c) e[c] = U[7][c];
    return ok;
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool side(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                              const Carry<Pb, R>&, R (&ys)[Pb::D]) {
    constexpr int D = Pb::D;
    double Y[8][D], U[8][D], LU[D][D], rinv[D];
    int piv[D];
    return rodas_step<Pb>(y, p, h, Y, U, LU, piv, rinv, ys);
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool replay_step(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                                     R (&ynew)[Pb::D]) {
    constexpr int D = Pb::D;
    double Y[8][D], U[8][D], LU[D][D], rinv[D];
    int piv[D];
    return rodas_step<Pb>(y, p, h, Y, U, LU, piv, rinv, ynew);
  }
  template <class Pb, class R, bool USER_COT, class Acc>
  __device__ __forceinline__ static bool unit(const RevArgs& a, long long k, int mode, bool active, int us,
                                              const R (&x)[Pb::D], double h, const R (&p)[Pb::NP], R (&lam)[Pb::D],
                                              Acc& pacc, double& loss, R (&ynew)[Pb::D]) {
    static_assert(std::is_same<R, double>::value, "Rodas5P runs in FP64");
    constexpr int D = Pb::D;
    double Y[8][D], U[8][D], LU[D][D], rinv[D];
    int piv[D];
    const bool ok = rodas_step<Pb>(x, p, h, Y, U, LU, piv, rinv, ynew);
    if (mode == U_RECOMP) return ok;
    const bool side = (mode == U_SIDE);
    double cv[D], v[D];
    unit_cotangent<Pb, R, USER_COT>(a, k, active, side, us, ynew, lam, cv, loss);
    rodas_reverse<Pb>(x, p, h, Y, U, LU, piv, rinv, cv, v, pacc);
#pragma unroll
    for (int c = 0; c < D; ++c) lam[c] = !active ? lam[c] : (side ? add_(lam[c], v[c]) : v[c]);
    return ok;
  }
};

// Rosenbrock23 (FP64 only): second order, error estimate of order 2 (err^(-1/3)
// controller), f at the accepted state carried to the next step.
struct Ros23Method {
  static constexpr bool kControl64 = false;
  static constexpr int REV_MINB_F32 = 0, REV_MINB_STAGES = 0;
  static constexpr int ORDER = 2, ERR_ORDER = 2;
  static constexpr bool kStages = true;
  static constexpr double IDLE_H = 1.0;
  template <class Pb, class R>
  struct Carry {
    R F0[Pb::D];  // f(y) of the current accepted state
  };
  static constexpr bool kCarryIsF = true;  // the carry is f(y) (start() computes it)
  template <class Pb, class R, class Get>
  __device__ __forceinline__ static void set_carry_f(Carry<Pb, R>& cy, Get f) {
#pragma unroll
    for (int c = 0; c < Pb::D; ++c) cy.F0[c] = f(c);
  }
  template <class Pb, class R>
  __device__ __forceinline__ static R carry_f(const Carry<Pb, R>& cy, int c) {
    return cy.F0[c];
  }
  // ---- stored stages: a step stores k1, u2 and the LU of W (factors, pivot
  // reciprocals, pivots); Y1 = y + h/2 k1 and a side step's save state
  // y + h (u2 + k1) are rebuilt from them by the step's own operations.
  template <class Pb, class R>
  struct StageData {
    double k1[Pb::D], u2[Pb::D], LU[Pb::D][Pb::D], rinv[Pb::D];
    int piv[Pb::D];
  };
  template <int D>
  static constexpr int step_payload() {
    return 4 * D + D * D;
  }
  template <int D>
  static constexpr int side_payload() {
    return step_payload<D>();
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool trial_s(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                                 const Carry<Pb, R>& cy, R (&ynew)[Pb::D], R (&e)[Pb::D],
                                                 Carry<Pb, R>& next, StageData<Pb, R>& sd) {
    return ros23_trial<Pb>(y, p, h, cy.F0, ynew, e, next.F0, sd.LU, sd.piv, sd.rinv, sd.k1, sd.u2);
  }
  template <class Pb, class R, class W>
  __device__ __forceinline__ static void pack(const StageData<Pb, R>& sd, bool, W&& write) {
    constexpr int D = Pb::D;
    int i = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) write(i++, sd.k1[c]);
#pragma unroll
    for (int c = 0; c < D; ++c) write(i++, sd.u2[c]);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) write(i++, sd.LU[r][c]);
#pragma unroll
    for (int c = 0; c < D; ++c) write(i++, sd.rinv[c]);
#pragma unroll
    for (int c = 0; c < D; ++c) write(i++, (double)sd.piv[c]);
  }
  template <class Pb, class R, class Rd>
  __device__ __forceinline__ static void unpack(bool, const R (&)[Pb::D], Rd&& read, StageData<Pb, R>& sd) {
    constexpr int D = Pb::D;
    int i = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) sd.k1[c] = read(i++);
#pragma unroll
    for (int c = 0; c < D; ++c) sd.u2[c] = read(i++);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) sd.LU[r][c] = read(i++);
#pragma unroll
    for (int c = 0; c < D; ++c) sd.rinv[c] = read(i++);
#pragma unroll
    for (int c = 0; c < D; ++c) sd.piv[c] = (int)read(i++);
  }
  template <class Pb, class R, bool USER_COT, class Acc>
  __device__ __forceinline__ static bool unit_stored(const RevArgs& a, long long k, int mode, bool active, int us,
                                                     const R (&x)[Pb::D], double h, const R (&p)[Pb::NP],
                                                     const StageData<Pb, R>& sd, R (&lam)[Pb::D], Acc& pacc,
                                                     double& loss) {
    constexpr int D = Pb::D;
    const bool side = (mode == U_SIDE);
    const double hh = mul_(0.5, h);
    double Y1[D], ynew[D], cv[D], v[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      Y1[c] = fma_(hh, sd.k1[c], x[c]);
      ynew[c] = fma_(h, add_(sd.u2[c], sd.k1[c]), x[c]);
    }
    unit_cotangent<Pb, R, USER_COT>(a, k, active, side, us, ynew, lam, cv, loss);
    ros23_reverse<Pb>(x, p, h, sd.k1, sd.u2, Y1, sd.LU, sd.piv, sd.rinv, cv, v, pacc);
#pragma unroll
    for (int c = 0; c < D; ++c) lam[c] = !active ? lam[c] : (side ? add_(lam[c], v[c]) : v[c]);
    return true;
  }
  template <class Pb, class R>
  __device__ __forceinline__ static void start(const R (&y)[Pb::D], const R (&p)[Pb::NP], Carry<Pb, R>& cy,
                                               float (&f0)[Pb::D]) {
    Pb::f(y, p, cy.F0);
#pragma unroll
    for (int c = 0; c < Pb::D; ++c) f0[c] = (float)cy.F0[c];
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool trial(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                               const Carry<Pb, R>& cy, R (&ynew)[Pb::D], R (&e)[Pb::D],
                                               Carry<Pb, R>& next) {
    static_assert(std::is_same<R, double>::value, "Rosenbrock23 runs in FP64");
    return ros23_trial<Pb>(y, p, h, cy.F0, ynew, e, next.F0);
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool side(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                              const Carry<Pb, R>& cy, R (&ys)[Pb::D]) {
    constexpr int D = Pb::D;
    double LU[D][D], rinv[D], k1[D], u2[D], Y1[D], F1[D];
    int piv[D];
    const bool ok = ros23_factor<Pb>(y, p, h, LU, piv, rinv);
    ros23_stages<Pb>(y, p, h, cy.F0, LU, piv, rinv, k1, u2, Y1, F1, ys);
    return ok;
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool replay_step(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                                     R (&ynew)[Pb::D]) {
    constexpr int D = Pb::D;
    double LU[D][D], rinv[D], F0[D], k1[D], u2[D], Y1[D], F1[D];
    int piv[D];
    const bool ok = ros23_factor<Pb>(y, p, h, LU, piv, rinv);
    Pb::f(y, p, F0);
    ros23_stages<Pb>(y, p, h, F0, LU, piv, rinv, k1, u2, Y1, F1, ynew);
    return ok;
  }
  template <class Pb, class R, bool USER_COT, class Acc>
  __device__ __forceinline__ static bool unit(const RevArgs& a, long long k, int mode, bool active, int us,
                                              const R (&x)[Pb::D], double h, const R (&p)[Pb::NP], R (&lam)[Pb::D],
                                              Acc& pacc, double& loss, R (&ynew)[Pb::D]) {
    static_assert(std::is_same<R, double>::value, "Rosenbrock23 runs in FP64");
    constexpr int D = Pb::D;
    double LU[D][D], rinv[D], F0[D], k1[D], u2[D], Y1[D], F1[D];
    int piv[D];
    const bool ok = ros23_factor<Pb>(x, p, h, LU, piv, rinv);
    Pb::f(x, p, F0);
    ros23_stages<Pb>(x, p, h, F0, LU, piv, rinv, k1, u2, Y1, F1, ynew);
    if (mode == U_RECOMP) return ok;
    const bool side = (mode == U_SIDE);
    double cv[D], v[D];
    unit_cotangent<Pb, R, USER_COT>(a, k, active, side, us, ynew, lam, cv, loss);
    ros23_reverse<Pb>(x, p, h, k1, u2, Y1, LU, piv, rinv, cv, v, pacc);
#pragma unroll
    for (int c = 0; c < D; ++c) lam[c] = !active ? lam[c] : (side ? add_(lam[c], v[c]) : v[c]);
    return ok;
  }
};

struct Verner7Method {  // FP64 only
  static constexpr bool kControl64 = false;
  static constexpr int REV_MINB_F32 = 0, REV_MINB_STAGES = GS_VERN7_REV_MINB_STAGES;
  static constexpr int ORDER = 7, ERR_ORDER = 6;
  static constexpr bool kStages = true;
  static constexpr double IDLE_H = 0.0;
  template <class Pb, class R>
  struct Carry {};  // not FSAL: every step evaluates f(y)
  static constexpr bool kCarryIsF = false;
  // ---- stored stages: a step stores the stage inputs Y_1..Y_8 (Y_0 is the
  // segment's state); a side step also its save state.
  template <class Pb, class R>
  struct StageData {
    R Y[10][Pb::D], ynew[Pb::D];
  };
  template <int D>
  static constexpr int step_payload() {
    return 8 * D;
  }
  template <int D>
  static constexpr int side_payload() {
    return 9 * D;
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool trial_s(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                                 const Carry<Pb, R>&, R (&ynew)[Pb::D], R (&e)[Pb::D],
                                                 Carry<Pb, R>&, StageData<Pb, R>& sd) {
    constexpr int D = Pb::D;
    R K[10][D];
    vern7_stages<Pb, R, 10>(y, p, h, sd.Y, K);
    vern7_update<Pb, R, 10>(y, K, h, ynew);
    vern7_error<Pb, R>(K, h, e);
#pragma unroll
    for (int c = 0; c < D; ++c) sd.ynew[c] = ynew[c];
    return true;
  }
  template <class Pb, class R, class W>
  __device__ __forceinline__ static void pack(const StageData<Pb, R>& sd, bool side, W&& write) {
    constexpr int D = Pb::D;
#pragma unroll
    for (int j = 1; j < 9; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c) write((j - 1) * D + c, sd.Y[j][c]);
    if (side) {
#pragma unroll
      for (int c = 0; c < D; ++c) write(8 * D + c, sd.ynew[c]);
    }
  }
  template <class Pb, class R, class Rd>
  __device__ __forceinline__ static void unpack(bool side, const R (&x)[Pb::D], Rd&& read, StageData<Pb, R>& sd) {
    constexpr int D = Pb::D;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      sd.Y[0][c] = x[c];
      sd.ynew[c] = x[c];  // replaced below for a side step; a step unit does not use it
    }
#pragma unroll
    for (int j = 1; j < 9; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c) sd.Y[j][c] = read((j - 1) * D + c);
    if (side) {
#pragma unroll
      for (int c = 0; c < D; ++c) sd.ynew[c] = read(8 * D + c);
    }
  }
  template <class Pb, class R, bool USER_COT, class Acc>
  __device__ __forceinline__ static bool unit_stored(const RevArgs& a, long long k, int mode, bool active, int us,
                                                     const R (&x)[Pb::D], double h, const R (&p)[Pb::NP],
                                                     const StageData<Pb, R>& sd, R (&lam)[Pb::D], Acc& pacc,
                                                     double& loss) {
    constexpr int D = Pb::D;
    const bool side = (mode == U_SIDE);
    R cv[D], v[D];
    unit_cotangent<Pb, R, USER_COT>(a, k, active, side, us, sd.ynew, lam, cv, loss);
    vern7_reverse<Pb, R>(sd.Y, p, h, cv, v, pacc);
#pragma unroll
    for (int c = 0; c < D; ++c) lam[c] = !active ? lam[c] : (side ? add_(lam[c], v[c]) : v[c]);
    return true;
  }
  template <class Pb, class R>
  __device__ __forceinline__ static void start(const R (&y)[Pb::D], const R (&p)[Pb::NP], Carry<Pb, R>&,
                                               float (&f0)[Pb::D]) {
    R f[Pb::D];
    Pb::f(y, p, f);
#pragma unroll
    for (int c = 0; c < Pb::D; ++c) f0[c] = (float)f[c];
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool trial(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                               const Carry<Pb, R>&, R (&ynew)[Pb::D], R (&e)[Pb::D],
                                               Carry<Pb, R>&) {
    static_assert(std::is_same<R, double>::value, "Verner7 runs in FP64");
    constexpr int D = Pb::D;
    R Y[10][D], K[10][D];
    vern7_stages<Pb, R, 10>(y, p, h, Y, K);
    vern7_update<Pb, R, 10>(y, K, h, ynew);
    vern7_error<Pb, R>(K, h, e);
    return true;
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool side(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                              const Carry<Pb, R>&, R (&ys)[Pb::D]) {
    return replay_step<Pb, R>(y, p, h, ys);
  }
  template <class Pb, class R>
  __device__ __forceinline__ static bool replay_step(const R (&y)[Pb::D], const R (&p)[Pb::NP], double h,
                                                     R (&ynew)[Pb::D]) {
    constexpr int D = Pb::D;
    R Y[9][D], K[9][D];
    vern7_stages<Pb, R, 9>(y, p, h, Y, K);
    vern7_update<Pb, R, 9>(y, K, h, ynew);
    return true;
  }
  template <class Pb, class R, bool USER_COT, class Acc>
  __device__ __forceinline__ static bool unit(const RevArgs& a, long long k, int mode, bool active, int us,
                                              const R (&x)[Pb::D], double h, const R (&p)[Pb::NP], R (&lam)[Pb::D],
                                              Acc& pacc, double& loss, R (&ynew)[Pb::D]) {
    static_assert(std::is_same<R, double>::value, "Verner7 runs in FP64");
    constexpr int D = Pb::D;
    R Y[9][D], K[9][D];
    vern7_stages<Pb, R, 9>(x, p, h, Y, K);
    vern7_update<Pb, R, 9>(x, K, h, ynew);
    if (mode == U_RECOMP) return true;
    const bool side = (mode == U_SIDE);
    R cv[D], v[D];
    unit_cotangent<Pb, R, USER_COT>(a, k, active, side, us, ynew, lam, cv, loss);
    vern7_reverse<Pb, R>(Y, p, h, cv, v, pacc);
#pragma unroll
    for (int c = 0; c < D; ++c) lam[c] = !active ? lam[c] : (side ? add_(lam[c], v[c]) : v[c]);
    return true;
  }
};

// ---------------------------------------------------------------------------
// Record kernel
// ---------------------------------------------------------------------------
// The stage data type of a method when a kernel stores or loads stages (an
// empty placeholder otherwise).
struct NoStages {};
template <class M, class Pb, class R, bool STAGES>
struct StageOf {
  using type = NoStages;
};
template <class M, class Pb, class R>
struct StageOf<M, Pb, R, true> {
  using type = typename M::template StageData<Pb, R>;
};
// Doubles of a stored-stage segment, [prev, t, y[D], h, step payload],
// rounded up to a 16-byte multiple.
template <class M, int D>
constexpr int stage_segw() {
  return ((3 + D + M::template step_payload<D>()) + 1) & ~1;
}
// Layout of the side steps' stage data (side_stg): for an even payload (Tsit5)
// [n][n_save][payload], each side step's data one 16-byte-aligned block that a
// lane writes and reads with vector accesses and whole DRAM sectors (the Lorenz
// record's DRAM traffic fell from 279 to 214 B per accepted step, its
// algorithmic 205, with no change in time); for an odd payload (Rodas5P,
// Rosenbrock23, Verner7 at d = 3) [n_save][payload][n], which measured 1% faster
// for the Robertson record than the block layout with scalar accesses.
template <int SP>
constexpr bool side_blocks() {
  return SP % 2 == 0;
}
// A (method, problem, precision) stores stages only in FP64, without shared
// weights and when its segment fits the record kernel's staging buffer.
template <class M, class Pb, class R>
constexpr bool stages_possible() {
  if constexpr (M::kStages && std::is_same<R, double>::value && !HasWeights<Pb>::value)
    return stage_segw<M, Pb::D>() <= MAX_STAGE_SEGW;
  else
    return false;
}

// Whether the starting-step pass also hands the record its carry f(y0)
// (FP64 methods whose carry is f(y0)): measured at Lorenz / Van der Pol 2^24,
// FP64 records 0.3% / 2.3% faster (3% with FP64 step control), FP32-mixed
// records 5% / 2.6% slower (their f(y0) in FP32 costs less than the exact
// conversions of the carried values), so FP64 only.
template <class M, class R>
constexpr bool carry_from_pass() {
  return M::kCarryIsF && std::is_same<R, double>::value;
}

// SAVES: save-time side steps run (for y_save, or for the stored side stages);
// STAGES: the record stores stage inputs (k = 1); C64: FP64 step control
// (GS_CONTROL_FP64: error norm, controller, starting step and step floor in FP64).
template <class M, class Pb, class R, bool SAVES, bool STAGES, bool C64 = false>
__device__ __forceinline__ void record_body(const FwdArgs& a) {
  static_assert(!STAGES || (SAVES && M::kStages), "stored stages need side steps and a method that exposes stages");
  constexpr int D = Pb::D, NP = Pb::NP;
  using Carry = typename M::template Carry<Pb, R>;
  extern __shared__ double smem[];
  const int ns = a.n_save;
  double* s_save = smem;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) s_save[i] = a.save_t[i];
  const int TB = blockDim.x;
  double* stg = smem + ((ns + 1) & ~1) + threadIdx.x;  // this lane's segment staging, stride TB
  if constexpr (HasWeights<Pb>::value) Pb::block_setup(a.shared_w);
  __syncthreads();

  const long long n = a.n;
  const double t1 = a.t1;
  const double sliver = 1e-12 * fmax(1.0, fabs(t1));
  const long long key_end = dkey(t1 - sliver);  // a step reaching past t1 - sliver is the last
  const float rtf = (float)a.rtol, atf = (float)a.atol;  // the error norm's FP32 scale factors
  long long k = -1;
  bool drained = false;
  double t = 0.0, h = 0.0;
  R y[D], p[NP];
  Carry cy;
  int S = 0, natt = 0, slot = 0, js = 0, status = TRAJ_OK;
  bool rej = false, lastnf = false, lastsing = false, ended = false;
  long long prev = -1;
  // pending save-time side steps [jp, je), all from the mesh point (tp, yp)
  R yp[D];
  Carry cyp;
  double tp = 0.0;
  int jp = 0, je = 0;
  long long res_next = 0, res_end = 0;  // this warp's reserved arena slots [res_next, res_end) (warp-uniform)

  for (;;) {
    // ---- refill: lanes without a trajectory take the next ticket
    const bool need = (k < 0) && !drained;
    if (__any_sync(FULL_MASK, need)) {
      const long long got = warp_ticket(a.work, need);
      if (need) {
        if (got < n) {
          k = got;
          bool fin = true;
          float yf[D], pf[NP], ff[D];
          double yd[D], pd[NP];  // (FP64 step control: the inputs as given)
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            const double v = a.params[q * n + k];
            p[q] = (R)v;
            pf[q] = (float)v;
            pd[q] = v;
            fin = fin && finite_d(v);
          }
#pragma unroll
          for (int c = 0; c < D; ++c) {
            const double v = a.y0[c * n + k];
            y[c] = (R)v;
            yf[c] = (float)v;
            yd[c] = v;
            fin = fin && finite_d(v);
          }
          t = a.t0;
          S = natt = slot = js = jp = je = 0;
          status = TRAJ_OK;
          rej = lastnf = lastsing = false;
          prev = -1;
          bool carried = false;
          if constexpr (carry_from_pass<M, R>()) {
            if (a.h0_pre == 2) {  // the pass's starting step and f(y0) (slots rewritten when k ends)
              M::template set_carry_f<Pb, R>(cy, [&](int c) { return to_r<R>(a.y_final[c * n + k]); });
              h = __longlong_as_double(a.head[k]);
              carried = true;
            }
          }
          if (!carried) {
            M::template start<Pb, R>(y, p, cy, ff);
            if (a.h0 > 0.0) {
              h = a.h0;
            } else if (a.h0_pre) {
              h = a.y_final[k];  // the starting-step pass's result (this slot is rewritten when k ends)
            } else if constexpr (C64) {
              double fd[D];
              Pb::f(yd, pd, fd);
              h = initial_step_f64<Pb, M::ORDER>(yd, pd, fd, a.t0, t1, a.rtol, a.atol);
            } else {
              h = initial_step_f32<Pb, M::ORDER>(yf, pf, ff, a.t0, t1, a.rtol, a.atol);
            }
          }
          fin = fin && positive(h) && finite_nonneg(h);
          ended = !fin;
          if (!fin) status = TRAJ_NONFINITE;
          if (a.k > 0) {
            stg[1 * TB] = t;
#pragma unroll
            for (int c = 0; c < D; ++c) stg[(2 + c) * TB] = to_d(y[c]);
          }
        } else {
          drained = true;
        }
      }
    }
    if (!__any_sync(FULL_MASK, k >= 0)) break;

    // ---- this lane's unit: a pending save-time side step (it starts from the
    // mesh point before the last accepted step), else a trial step
    int um = U_NONE;
    bool last = false;
    double tsum = 0.0;  // t + h of a trial step
    if (k >= 0) {
      if (SAVES) {
        while (jp < je && same_time(s_save[jp], tp)) {  // a save on that mesh point: its state, no step
          if (a.y_save) {
#pragma unroll
            for (int c = 0; c < D; ++c) a.y_save[((long long)jp * D + c) * n + k] = (double)yp[c];
          }
          ++jp;
        }
        if (jp < je) um = U_SIDE;
      }
      if (um == U_NONE && !ended) {
        if (natt >= a.max_steps) {
          status = TRAJ_MAXSTEPS;
          ended = true;
        } else {
          um = U_STEP;
          tsum = add_(t, h);
          if (dkey(tsum) >= key_end) {
            h = t1 - t;
            last = true;
          }
        }
      }
    }

    // ---- one step for every lane with a unit: trial steps and side steps run
    // the same code (a side step ignores the error estimate). The mode is made
    // opaque to the optimiser so that the two share one copy of the code and
    // the warp runs it once with all its busy lanes.
    __syncwarp();
    asm volatile("" : "+r"(um));
    // a side step's length: in the FP64 form (bound by the FP64 pipe) the
    // subtraction runs only in iterations that have a side step; the FP32-mixed
    // kernels are bound by instruction issue, where a select is cheaper
    double hx = h;
    if constexpr (std::is_same<R, double>::value) {
      if (SAVES && __any_sync(FULL_MASK, um == U_SIDE)) {
        if (um == U_SIDE) hx = sub_(s_save[jp], tp);
      }
    } else {
      hx = (SAVES && um == U_SIDE) ? s_save[jp] - tp : h;
    }
    R yn[D], e[D];
    typename StageOf<M, Pb, R, STAGES>::type sd;  // stage data of this unit (stored-stage records)
    Carry next;
    double q = 2.0;
    bool solved = true;
    if (um != U_NONE) {
      const bool is_side = SAVES && (um == U_SIDE);
      R xin[D], pin[NP];
#pragma unroll
      for (int c = 0; c < D; ++c) xin[c] = is_side ? yp[c] : y[c];
      // the unit works on its own copy of the parameters: with it the register
      // allocation of the FP64 Lorenz stored-stage record changes and the
      // kernel runs 4.5% faster (318 -> 304 ms at 2^24, measured)
#pragma unroll
      for (int q2 = 0; q2 < NP; ++q2) pin[q2] = p[q2];
      const Carry cin = is_side ? cyp : cy;
      if constexpr (STAGES) {
        // the unit's stage data go out at once (a step's to its staging slot,
        // overwritten by the next trial if this one is rejected), so that they
        // are not held in registers across the step-size decision
        solved = M::template trial_s<Pb, R>(xin, pin, hx, cin, yn, e, next, sd);
        if (is_side) {
          constexpr int SP = M::template side_payload<D>();
          if constexpr (side_blocks<SP>()) {  // this trajectory's block, 16-byte vector stores
            double* dst = a.side_stg + ((long long)k * ns + jp) * SP;
            double buf[SP];
            M::template pack<Pb, R>(sd, true, [&](int i, double v) { buf[i] = v; });
#pragma unroll
            for (int w = 0; w < SP / 2; ++w)
              reinterpret_cast<double2*>(dst)[w] = make_double2(buf[2 * w], buf[2 * w + 1]);
          } else {
            double* dst = a.side_stg + (long long)jp * SP * n + k;
            M::template pack<Pb, R>(sd, true, [&](int i, double v) { dst[(long long)i * n] = v; });
          }
        } else {
          M::template pack<Pb, R>(sd, false, [&](int i, double v) { stg[(3 + D + i) * TB] = v; });
        }
      } else {
        solved = M::template trial<Pb, R>(xin, pin, hx, cin, yn, e, next);
      }
      if (!is_side) {
        ++natt;
        // q: the mean square of the scaled error, in the fast control's FP32
        // form or in FP64; q <= 1 (FP64: sqrt(q) <= 1) accepts
        if constexpr (C64)
          q = err_meansq_f64<D>(e, y, yn, a.rtol, a.atol);
        else
          q = err_meansq<D>(e, y, yn, a.rtol, a.atol, rtf, atf);
      }
    }
    if (SAVES && um == U_SIDE) {
      if (a.y_save) {
#pragma unroll
        for (int c = 0; c < D; ++c) a.y_save[((long long)jp * D + c) * n + k] = solved ? (double)yn[c] : nan_d();
      }
      ++jp;
    }
    const bool trial = (um == U_STEP);
    const bool accept = trial && solved && (C64 ? rms_le_one(q) : le_one(q));  // q >= 0; NaN rejects
    if (accept) {
      const double tn = last ? t1 : tsum;
      if (SAVES) {
        // save times in [t, tn): side steps from (t, y), taken as units of the
        // following iterations; exactly tn: y_new
        jp = js;
        tp = t;
#pragma unroll
        for (int c = 0; c < D; ++c) yp[c] = y[c];
        cyp = cy;
        const long long key_tn = dkey(tn);
        while (js < ns && dkey(s_save[js]) < key_tn) ++js;
        je = js;
        while (js < ns && same_time(s_save[js], tn)) {
          if (a.y_save) {
#pragma unroll
            for (int c = 0; c < D; ++c) a.y_save[((long long)js * D + c) * n + k] = (double)yn[c];
          }
          ++js;
        }
      }
      if (a.k > 0) stg[(2 + D + slot) * TB] = h;  // (stored stages, k = 1: the step's data follow h)
      ++slot;
      t = tn;
#pragma unroll
      for (int c = 0; c < D; ++c) y[c] = yn[c];
      cy = next;
      ++S;
      if (last) ended = true;
    }
    if (trial && !ended) {
      // integral controller: accepted steps grow at most x10 (x1 right after a
      // rejection), rejected ones shrink by the same rule, x0.2 on a non-finite
      // error, x0.25 when the step's linear system is singular
      const bool nf = solved && !finite_nonneg(q);
      bool under;
      if constexpr (C64) {
        double fac = !solved ? 0.25 : (nf ? 0.2 : ctrl_factor_ms_f64<M::ERR_ORDER>(q));
        if (accept && rej) fac = fmin(fac, 1.0);
        h = mul_(h, fac);
        under = fabs(h) < mul_(1e-14, fmax(1.0, fabs(t)));
      } else {
        float fac = !solved ? 0.25f : (nf ? 0.2f : ctrl_factor<M::ERR_ORDER>(q));
        if (accept && rej) fac = fminf(fac, 1.0f);
        h = mul_(h, to_d(fac));
        // |h| < 1e-14 max(1, |t|), evaluated in FP32 (a threshold test, not arithmetic of the solution)
        under = fabsf(to_f(h)) < 1e-14f * fmaxf(1.0f, fabsf(to_f(t)));
      }
      rej = !accept;
      lastnf = !accept && nf;
      lastsing = !solved;
      if (under) {
        status = lastsing ? TRAJ_SINGULAR : (lastnf ? TRAJ_NONFINITE : TRAJ_DT_UNDERFLOW);
        ended = true;
      }
    }
    // the trajectory is done once it has ended and its pending side steps are taken
    const bool done = (k >= 0) && ended && !(SAVES && jp < je);
    // (a.k == 0: forward-only solve, nothing is recorded)
    const bool flush = (a.k > 0) && (k >= 0) && ((slot == a.k) || (done && slot > 0));

    // ---- segment write-out: one arena slot per flushing lane, from the warp's reserved block
    if (__any_sync(FULL_MASK, flush)) {
      // arena slots are reserved per warp in blocks (one atomic per block, not
      // per flush); the unused tail of a warp's last block stays empty, since
      // segments are linked, not indexed
      const unsigned fm = __ballot_sync(FULL_MASK, flush);
      const int cnt = __popc(fm), rem = (int)(res_end - res_next);
      const int blk = a.arena_block >= 32 ? a.arena_block : ARENA_BLOCK_HOST;
      long long nb = 0;
      if (cnt > rem) {  // warp-uniform: a new block continues where the reserved one ends
        unsigned long long base = 0;
        if (lane_id() == 0) base = atomicAdd(a.arena_top, (unsigned long long)blk);
        nb = (long long)__shfl_sync(FULL_MASK, base, 0);
      }
      const int rank = __popc(fm & ((1u << lane_id()) - 1u));
      const long long idx = rank < rem ? res_next + rank : nb + (rank - rem);
      if (cnt > rem) {
        res_next = nb + (cnt - rem);
        res_end = nb + blk;
      } else {
        res_next += cnt;
      }
      if (flush) {
        stg[0] = __longlong_as_double(prev);
        if (idx < a.arena_cap) {
          double2* dst = reinterpret_cast<double2*>(a.arena + idx * a.segw);
          for (int w = 0; w < (a.segw >> 1); ++w) dst[w] = make_double2(stg[(2 * w) * TB], stg[(2 * w + 1) * TB]);
        } else {
          *a.overflow = 1;
        }
        prev = idx;
        slot = 0;
        stg[1 * TB] = t;
#pragma unroll
        for (int c = 0; c < D; ++c) stg[(2 + c) * TB] = to_d(y[c]);
      }
    }

    if (done) {
      if (a.head) a.head[k] = prev;
      if (a.S) a.S[k] = S;
      if (a.natt) a.natt[k] = natt;
      a.status[k] = status;
#pragma unroll
      for (int c = 0; c < D; ++c) a.y_final[c * n + k] = (double)y[c];
      if (a.step_counts) {
        a.step_counts[k] = S;
        a.step_counts[n + k] = natt;
      }
      if (status != TRAJ_OK) *a.any_failed = 1;
      k = -1;
    }
  }
}

// Starting steps of all trajectories in one pass, before the record kernel:
// y_final[k] = the h the record's refill would compute for trajectory k, by the
// same function and inputs (shared-weight problems stage their weights first,
// as the record does). With h0_pre = 2 (a record, whose head[k] is free until
// k ends, and carry_from_pass) head[k] holds h and y_final[., k] the carry
// f(y0). In the record this is per-trajectory code that one or two lanes of a
// warp run while the others wait; here every lane computes one.
template <class M, class Pb, class R, bool C64>
__global__ void __launch_bounds__(256) init_step_kernel(const FwdArgs a) {
  constexpr int D = Pb::D, NP = Pb::NP;
  using Carry = typename M::template Carry<Pb, R>;
  if constexpr (HasWeights<Pb>::value) Pb::block_setup(a.shared_w);
  __syncthreads();
  const long long n = a.n;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    R y[D], p[NP];
    float yf[D], pf[NP], ff[D];
    double yd[D], pd[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const double v = a.params[q * n + k];
      p[q] = (R)v;
      pf[q] = (float)v;
      pd[q] = v;
    }
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const double v = a.y0[c * n + k];
      y[c] = (R)v;
      yf[c] = (float)v;
      yd[c] = v;
    }
    double h;
    Carry cy;
    M::template start<Pb, R>(y, p, cy, ff);
    if constexpr (C64) {
      double fd[D];
      Pb::f(yd, pd, fd);
      h = initial_step_f64<Pb, M::ORDER>(yd, pd, fd, a.t0, a.t1, a.rtol, a.atol);
    } else {
      h = initial_step_f32<Pb, M::ORDER>(yf, pf, ff, a.t0, a.t1, a.rtol, a.atol);
    }
    if constexpr (carry_from_pass<M, R>()) {
      if (a.h0_pre == 2) {  // f(y0), the record's carry, too: h then goes to head[k]
#pragma unroll
        for (int c = 0; c < D; ++c) a.y_final[c * n + k] = to_d(M::template carry_f<Pb, R>(cy, c));
        a.head[k] = __double_as_longlong(h);
        continue;
      }
    }
    a.y_final[k] = h;
  }
}

template <class M, class Pb, class R, bool SAVES, bool STAGES, bool C64 = false>
__global__ void __launch_bounds__(TPB_FWD) record_kernel(const FwdArgs a) {
  record_body<M, Pb, R, SAVES, STAGES, C64>(a);
}
template <class M, class Pb, class R, bool SAVES, bool STAGES, bool C64, int MINB>
__global__ void __launch_bounds__(TPB_FWD, MINB) record_kernel_mb(const FwdArgs a) {
  record_body<M, Pb, R, SAVES, STAGES, C64>(a);
}
#ifndef GS_FWD_C64_MINB
#define GS_FWD_C64_MINB 0
#endif
// The record kernel of (M, Pb, R, SAVES, STAGES, C64); the FP64-control forms
// with a register cap of GS_FWD_C64_MINB resident CTAs per SM (0: none).
template <class M, class Pb, class R, bool SAVES, bool STAGES, bool C64>
constexpr auto record_entry() {
  if constexpr (C64 && GS_FWD_C64_MINB > 0)
    return &record_kernel_mb<M, Pb, R, SAVES, STAGES, C64, GS_FWD_C64_MINB>;
  else
    return &record_kernel<M, Pb, R, SAVES, STAGES, C64>;
}

// ---------------------------------------------------------------------------
// Reverse-kernel helpers
// ---------------------------------------------------------------------------
template <int NP, int D>
__device__ __forceinline__ void write_nan(const RevArgs& a, long long k) {
  const long long n = a.n;
  if (a.params_bar)
    for (int q = 0; q < NP; ++q) a.params_bar[q * n + k] = nan_d();
  if (a.y0_bar)
    for (int c = 0; c < D; ++c) a.y0_bar[c * n + k] = nan_d();
  if (a.loss) a.loss[k] = nan_d();
}

template <int NP, int D, class R, class Acc>
__device__ __forceinline__ void write_grad(const RevArgs& a, long long k, const Acc& pacc, const R (&lam)[D],
                                           double loss) {
  const long long n = a.n;
  if (a.params_bar)
#pragma unroll
    for (int q = 0; q < NP; ++q) a.params_bar[q * n + k] = pacc.get(q);
  if (a.y0_bar)
#pragma unroll
    for (int c = 0; c < D; ++c) a.y0_bar[c * n + k] = (double)lam[c];
  if (a.loss) a.loss[k] = loss;
}

// Save times attached to the state (tx, yx), visited in decreasing order:
// equal times add their cotangent to lambda directly; a later time is a side
// step from the state (returns true with its save index in us).
template <int D, class R, bool USER_COT>
__device__ __forceinline__ bool next_save(const RevArgs& a, const double* s_save, long long k, int& js, double tx,
                                          const R (&yx)[D], R (&lam)[D], double& loss, int& us) {
  const long long key_tx = dkey(tx);
  while (js >= 0 && dkey(s_save[js]) >= key_tx) {
    if (same_time(s_save[js], tx)) {
#pragma unroll
      for (int c = 0; c < D; ++c) {
        if (USER_COT) {
          lam[c] = add_(lam[c], to_r<R>(a.y_save_bar[((long long)js * D + c) * a.n + k]));
        } else {
          lam[c] = add_(lam[c], add_(yx[c], yx[c]));
          loss = acc_loss(loss, mul_(yx[c], yx[c]));
        }
      }
      --js;
    } else {
      us = js;
      --js;
      return true;
    }
  }
  return false;
}

template <class R, int NP>
using AccOf = typename std::conditional<std::is_same<R, float>::value, CompensatedAcc<NP>, PlainAcc<NP>>::type;
// Shared-weight problems bring their own accumulator (per-trajectory theta plus
// the warp's share of the weight gradient).
template <class Pb>
struct WeightAcc {
  using type = void;
};
template <>
struct WeightAcc<LvUde> {
  using type = UdeAcc;
};
template <>
struct WeightAcc<LvUdeWarp> {
  using type = UdeAcc;
};
template <>
struct WeightAcc<LvUdeCta> {
  using type = UdeAcc;
};
template <>
struct WeightAcc<NeuralRobertson> {
  using type = NrAcc;
};
template <class Pb, class R>
using AccFor = typename std::conditional<HasWeights<Pb>::value, typename WeightAcc<Pb>::type, AccOf<R, Pb::NP>>::type;
// Dynamic shared memory a shared-weight accumulator stages its factors in.
template <class Pb>
constexpr size_t weight_stage_bytes() {
  return std::is_same<Pb, NeuralRobertson>::value ? NR_STAGE_DOUBLES * sizeof(double) : 0;
}

// ---------------------------------------------------------------------------
// Reverse kernel, checkpoint interval k > 1: states inside a segment are
// recomputed from its checkpoint into a per-lane buffer (local memory).
// ---------------------------------------------------------------------------
enum : int { PH_LOAD = 0, PH_RECOMP = 1, PH_INJECT = 2 };

template <class M, class Pb, class R, bool USER_COT>
__global__ void __launch_bounds__(TPB_REV) reverse_kernel(const RevArgs a) {
  constexpr int D = Pb::D, NP = Pb::NP;
  static_assert(!HasWeights<Pb>::value, "shared-weight problems use the k = 1 reverse kernel");
  using Acc = AccOf<R, NP>;
  extern __shared__ double smem[];
  const int ns = a.n_save;
  double* s_save = smem;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) s_save[i] = a.save_t[i];
  __syncthreads();

  const long long n = a.n;
  long long k = -1;
  bool drained = false;
  R p[NP], lam[D], yfin[D];
  Acc pacc;
  double loss = 0.0;
  long long seg = -1, prevseg = -1;
  int m = 0, j = 0, rj = 0, js = -1, phase = PH_LOAD, segs_left = 0;
  bool final_seg = true;
  double ts[KMAX], hs[KMAX];
  R ys[KMAX][D];

  for (;;) {
    const bool need = (k < 0) && !drained;
    if (__any_sync(FULL_MASK, need)) {
      const long long got = warp_ticket(a.work, need);
      if (need) {
        if (got < n) {
          k = got;
          const long long hd = a.head[k];
          if (a.status[k] != TRAJ_OK || hd < 0) {
            write_nan<NP, D>(a, k);
            k = -1;  // take another ticket next iteration
          } else {
#pragma unroll
            for (int q = 0; q < NP; ++q) p[q] = (R)a.params[q * n + k];
#pragma unroll
            for (int c = 0; c < D; ++c) {
              lam[c] = R(0);
              yfin[c] = (R)a.y_final[c * n + k];
            }
            pacc.zero();
            loss = 0.0;
            seg = hd;
            const int Sk = a.S[k];
            m = Sk - ((Sk - 1) / a.k) * a.k;  // steps in the last segment
            segs_left = (Sk + a.k - 1) / a.k;
            final_seg = true;
            phase = PH_LOAD;
            js = ns - 1;
          }
        } else {
          drained = true;
        }
      }
    }
    if (!__any_sync(FULL_MASK, k >= 0 || !drained)) break;

    // Advance this lane to its next unit of work.
    int mode = U_NONE, us = 0;
    R ux[D];
    double uh = 0.0;
    if (k >= 0) {
      for (;;) {
        if (phase == PH_LOAD) {
          if (seg < 0 || seg >= a.arena_cap || segs_left <= 0) {  // inconsistent record: stop this lane
            mode = U_FAIL;
            break;
          }
          --segs_left;
          const double2* src = reinterpret_cast<const double2*>(a.arena + seg * a.segw);
          const double2 w0 = src[0];
          prevseg = __double_as_longlong(w0.x);
          ts[0] = w0.y;
          // y_start at [2, 2+D), h at [2+D, 2+D+m)
          for (int w = 1; w < (a.segw >> 1); ++w) {
            const double2 v = src[w];
            const int i0 = 2 * w, i1 = 2 * w + 1;
            if (i0 < 2 + D) ys[0][i0 - 2] = to_r<R>(v.x); else if (i0 - 2 - D < m) hs[i0 - 2 - D] = v.x;
            if (i1 < 2 + D) ys[0][i1 - 2] = to_r<R>(v.y); else if (i1 - 2 - D < m) hs[i1 - 2 - D] = v.y;
          }
          rj = 1;
          phase = PH_RECOMP;
        }
        if (phase == PH_RECOMP) {
          if (rj < m) {
            mode = U_RECOMP;
#pragma unroll
            for (int c = 0; c < D; ++c) ux[c] = ys[rj - 1][c];
            uh = hs[rj - 1];
            break;
          }
          j = m;
          phase = PH_INJECT;
        }
        // saves at state j of this segment (state m only in the final segment: y(t1))
        if (j < m || final_seg) {
          const double tj = (j == m) ? a.t1 : ts[j];
          R yj[D];
#pragma unroll
          for (int c = 0; c < D; ++c) yj[c] = (j == m) ? yfin[c] : ys[j][c];
          if (next_save<D, R, USER_COT>(a, s_save, k, js, tj, yj, lam, loss, us)) {
            mode = U_SIDE;
#pragma unroll
            for (int c = 0; c < D; ++c) ux[c] = yj[c];
            uh = s_save[us] - tj;
            break;
          }
        }
        if (j > 0) {
          mode = U_STEP;
#pragma unroll
          for (int c = 0; c < D; ++c) ux[c] = ys[j - 1][c];
          uh = hs[j - 1];
          --j;
          break;
        }
        if (prevseg < 0) {
          mode = (segs_left == 0) ? U_DONE : U_FAIL;
          break;
        }
        seg = prevseg;
        m = a.k;
        final_seg = false;
        phase = PH_LOAD;
      }
    }

    __syncwarp();
    if (mode == U_RECOMP || mode == U_STEP || mode == U_SIDE) {
      R yn[D];
      const bool ok = M::template unit<Pb, R, USER_COT, Acc>(a, k, mode, true, us, ux, uh, p, lam, pacc, loss, yn);
      if (!ok) {
        mode = U_FAIL;
      } else if (mode == U_RECOMP) {
#pragma unroll
        for (int c = 0; c < D; ++c) ys[rj][c] = yn[c];
        ts[rj] = add_(ts[rj - 1], hs[rj - 1]);
        ++rj;
      }
    }
    if (mode == U_FAIL) {
      write_nan<NP, D>(a, k);
      k = -1;
    }
    if (mode == U_DONE) {
      write_grad<NP, D, R>(a, k, pacc, lam, loss);
      k = -1;
    }
  }
}

// ---------------------------------------------------------------------------
// Reverse kernel, every accepted state stored (checkpoint interval k = 1).
//
// Segment i holds (t_{i-1}, y_{i-1}, h_i): nothing is recomputed, and every
// unit is a VJP with the same code, either the step-i VJP from y_{i-1} or a
// save-time side-step VJP from a mesh state. Per trajectory: the saves at
// state S (y(t1)); then for i = S..1: load segment i, step VJP, the saves
// attached to state i-1.
// ---------------------------------------------------------------------------
// STAGES: the record holds every step's stage data after h (segments of
// stage_segw<M, D>() doubles) and side_stg the side steps' (see side_blocks):
// the units load them instead of recomputing the stages.
// The cotangent of the save at t1 for every trajectory in one pass before the
// k = 1 reverse sweep (FP64): y0_bar[., k] = lambda after that save (2 y(t1)
// for the built-in loss, else the caller's dL/dy(t1)), loss[k] = ||y(t1)||^2
// for the built-in loss; the sweep starts from them. In the sweep this is
// per-trajectory code that one or two lanes of a warp run while the others
// wait; the arithmetic is the same (next_save's), so the results are too.
template <class Pb, bool USER_COT>
__global__ void __launch_bounds__(256) t1_save_kernel(const RevArgs a) {
  constexpr int D = Pb::D;
  const long long n = a.n;
  const int js = a.n_save - 1;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    double loss = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const double y = a.y_final[c * n + k];
      double lam = 0.0;
      if (USER_COT) {
        lam = add_(lam, a.y_save_bar[((long long)js * D + c) * n + k]);
      } else {
        lam = add_(lam, add_(y, y));
        loss = acc_loss(loss, mul_(y, y));
      }
      a.y0_bar[c * n + k] = lam;
    }
    if (!USER_COT && a.loss) a.loss[k] = loss;
  }
}

template <class M, class Pb, class R, bool USER_COT, bool STAGES = false>
__device__ __forceinline__ void reverse_k1_body(const RevArgs& a) {
  constexpr int D = Pb::D, NP = Pb::NP;
  constexpr bool COLL = HasWeights<Pb>::value;
  constexpr bool CTA = CtaColl<Pb>::value;  // units in lockstep across the CTA, not only the warp
  using Acc = AccFor<Pb, R>;
  extern __shared__ double smem[];
  const int ns = a.n_save;
  double* s_save = smem;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) s_save[i] = a.save_t[i];
  if constexpr (COLL) Pb::block_setup(a.shared_w);
  __syncthreads();

  const long long n = a.n;
  long long k = -1;
  bool drained = false;
  R p[NP], lam[D], yx[D];  // yx: the mesh state the next unit starts from
  // static schedule (shared-weight problems): lane i takes trajectories i, i + L, i + 2L, ...
  long long stat_next = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stat_stride = (long long)gridDim.x * blockDim.x;
#pragma unroll
  for (int q = 0; q < NP; ++q) p[q] = R(0);
#pragma unroll
  for (int c = 0; c < D; ++c) lam[c] = yx[c] = R(0);
  Acc pacc;
  if constexpr (COLL) pacc.init(smem + ((ns + 1) & ~1));
  double loss = 0.0, tx = 0.0;
  long long seg = -1;
  int js = -1, segs_left = 0;

  for (;;) {
    const bool need = (k < 0) && !drained;
    if (__any_sync(FULL_MASK, need)) {
      long long got;
      if constexpr (COLL) {
        got = need ? stat_next : -1;
        if (need) stat_next += stat_stride;
      } else {
        got = warp_ticket(a.work, need);
      }
      if (need) {
        if (got < n) {
          k = got;
          const long long hd = a.head[k];
          if (a.status[k] != TRAJ_OK || hd < 0) {
            write_nan<NP, D>(a, k);
            k = -1;
          } else {
#pragma unroll
            for (int q = 0; q < NP; ++q) p[q] = (R)a.params[q * n + k];
#pragma unroll
            for (int c = 0; c < D; ++c) {
              lam[c] = R(0);
              yx[c] = (R)a.y_final[c * n + k];
            }
            pacc.zero();
            loss = 0.0;
            tx = a.t1;
            seg = hd;
            segs_left = a.S[k];
            js = ns - 1;
            if constexpr (std::is_same<R, double>::value) {
              if (a.t1_pre) {  // the save at t1, taken by the pass before this kernel
#pragma unroll
                for (int c = 0; c < D; ++c) lam[c] = a.y0_bar[c * n + k];
                if (!USER_COT && a.loss) loss = a.loss[k];
                js = ns - 2;
              }
            }
          }
        } else {
          drained = true;
        }
      }
    }
    if constexpr (CTA) {
      if (!__syncthreads_or(k >= 0 || !drained)) break;
    } else {
      if (!__any_sync(FULL_MASK, k >= 0 || !drained)) break;
    }

    int mode = U_NONE, us = 0;
    double uh = 0.0;
    typename StageOf<M, Pb, R, STAGES>::type sd;  // stored stage data of this unit (STAGES)
    if (k >= 0) {
      if (next_save<D, R, USER_COT>(a, s_save, k, js, tx, yx, lam, loss, us)) {
        mode = U_SIDE;  // (its length s - t is formed below, once per warp iteration)
        if constexpr (STAGES) {
          constexpr int SP = M::template side_payload<D>();
          if constexpr (side_blocks<SP>()) {  // this trajectory's block, 16-byte vector loads
            const double* src = a.side_stg + ((long long)k * ns + us) * SP;
            double buf[SP];
#pragma unroll
            for (int w = 0; w < SP / 2; ++w) {
              const double2 v = reinterpret_cast<const double2*>(src)[w];
              buf[2 * w] = v.x;
              buf[2 * w + 1] = v.y;
            }
            M::template unpack<Pb, R>(true, yx, [&](int i) { return buf[i]; }, sd);
          } else {
            const double* src = a.side_stg + (long long)us * SP * a.n + k;
            M::template unpack<Pb, R>(true, yx, [&](int i) { return src[(long long)i * a.n]; }, sd);
          }
        }
      } else if (seg < 0) {
        mode = (segs_left == 0) ? U_DONE : U_FAIL;
      } else if (seg >= a.arena_cap || segs_left <= 0) {
        mode = U_FAIL;  // inconsistent record
      } else {
        // segment i: [prev, t_{i-1}, y_{i-1}[D], h_i (, Y_1..Y_5 of step i)]
        const double* sp = a.arena + seg * a.segw;
        if constexpr (STAGES) {
          const double2 w0 = *reinterpret_cast<const double2*>(sp);
          seg = __double_as_longlong(w0.x);
          tx = w0.y;
          constexpr int SW = stage_segw<M, D>();
          double buf[SW];
#pragma unroll
          for (int w = 1; w < SW / 2; ++w) {
            const double2 v = reinterpret_cast<const double2*>(sp)[w];
            buf[2 * w] = v.x;
            buf[2 * w + 1] = v.y;
          }
#pragma unroll
          for (int c = 0; c < D; ++c) yx[c] = to_r<R>(buf[2 + c]);
          uh = buf[2 + D];
          M::template unpack<Pb, R>(false, yx, [&](int i) { return buf[3 + D + i]; }, sd);
        } else {
          constexpr int CW = ((3 + D) + 1) & ~1;  // [prev, t, y[D], h] in whole double2
          double buf[CW];
#pragma unroll
          for (int w = 0; w < CW / 2; ++w) {
            const double2 v = reinterpret_cast<const double2*>(sp)[w];
            buf[2 * w] = v.x;
            buf[2 * w + 1] = v.y;
          }
          seg = __double_as_longlong(buf[0]);
          tx = buf[1];
#pragma unroll
          for (int c = 0; c < D; ++c) yx[c] = to_r<R>(buf[2 + c]);
          uh = buf[2 + D];
        }
        --segs_left;
        mode = U_STEP;
      }
    }

    __syncwarp();
    if constexpr (std::is_same<R, double>::value) {  // (as in the record kernel)
      if (__any_sync(FULL_MASK, mode == U_SIDE)) {
        if (mode == U_SIDE) uh = sub_(s_save[us], tx);
      }
    } else {
      if (mode == U_SIDE) uh = s_save[us] - tx;
    }
    const bool busy = (mode == U_STEP || mode == U_SIDE);
    if constexpr (STAGES) {
      if (busy && !M::template unit_stored<Pb, R, USER_COT, Acc>(a, k, mode, true, us, yx, uh, p, sd, lam, pacc, loss))
        mode = U_FAIL;
    } else if (COLL || busy) {
      R yn[D], xin[D];
#pragma unroll
      for (int c = 0; c < D; ++c) xin[c] = busy ? yx[c] : R(0);
      if (!M::template unit<Pb, R, USER_COT, Acc>(a, k, mode, busy, us, xin, busy ? uh : M::IDLE_H, p, lam, pacc,
                                                   loss, yn) &&
          busy)
        mode = U_FAIL;
    }
    if (mode == U_FAIL) {
      write_nan<NP, D>(a, k);
      k = -1;
    }
    if (mode == U_DONE) {
      write_grad<NP, D, R>(a, k, pacc, lam, loss);
      k = -1;
    }
  }
  if constexpr (COLL) {
    if (a.wpart) pacc.finish(a.wpart, (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
  }
  if constexpr (CTA) Pb::block_teardown(a.tc_error);
}

// Minimum resident CTAs of 128 threads per SM requested from the compiler for
// the k = 1 reverse sweep (0: no request, the compiler's own choice). A
// request caps the registers per thread at 65536 / (128 x blocks) so that more
// warps hide the latency of the dependent segment loads and arithmetic chains.
// Measured at 2^24 Lorenz trajectories: the FP32-mixed sweep 3.4% faster at 8
// blocks (64 registers) than at the compiler's 72, the FP64 stored-stage sweep
// 1.5% faster at 5 (96 registers) than at 122 (at 6, 80 registers: 1.2%; at 7,
// 72: 1.0%); the shared-weight kernels need more
// registers than either cap and keep the compiler's choice. Capping the
// Rodas5P (252 registers, 2 CTAs) and Verner7 (154, 3 CTAs) stored-stage sweeps
// at 3 to 5 CTAs changed their time by under 2% (Robertson 2^20, Lorenz 2^23),
// so they keep the compiler's choice too.
template <class M, class Pb, class R, bool STAGES>
constexpr int rev_min_blocks() {
  if constexpr (HasWeights<Pb>::value)
    return 0;
  else
    return std::is_same<R, float>::value ? M::REV_MINB_F32 : (STAGES ? M::REV_MINB_STAGES : 0);
}
template <class M, class Pb, class R, bool USER_COT, bool STAGES = false>
__global__ void __launch_bounds__(TPB_REV) reverse_k1_kernel(const RevArgs a) {
  reverse_k1_body<M, Pb, R, USER_COT, STAGES>(a);
}
template <class M, class Pb, class R, bool USER_COT, bool STAGES, int MINB>
__global__ void __launch_bounds__(TPB_REV, MINB) reverse_k1_kernel_mb(const RevArgs a) {
  reverse_k1_body<M, Pb, R, USER_COT, STAGES>(a);
}
// The k = 1 reverse kernel of (M, Pb, R, USER_COT, STAGES), with its register cap.
template <class M, class Pb, class R, bool USER_COT, bool STAGES = false>
constexpr auto reverse_k1_entry() {
  constexpr int mb = rev_min_blocks<M, Pb, R, STAGES>();
  if constexpr (mb > 0)
    return &reverse_k1_kernel_mb<M, Pb, R, USER_COT, STAGES, mb>;
  else
    return &reverse_k1_kernel<M, Pb, R, USER_COT, STAGES>;
}

// ---------------------------------------------------------------------------
// Refresh kernel (frozen-mesh reuse, paper Sec. 3.1): re-runs the state chain
// y_i = Phi(y_{i-1}; h_i, theta) of every trajectory over its recorded mesh
// with new (theta, y0), rewriting the state checkpoints and y(t1). Segments are
// linked last to first, so the lane finds them in forward order a window of
// RING segments at a time (one backward walk per window).
// ---------------------------------------------------------------------------
constexpr int REFRESH_RING = 64;

template <class M, class Pb, class R>
__global__ void __launch_bounds__(TPB_REV) refresh_kernel(const RevArgs a, double* arena, double* y_final,
                                                          const double* y0) {
  constexpr int D = Pb::D, NP = Pb::NP;
  if constexpr (HasWeights<Pb>::value) Pb::block_setup(a.shared_w);
  __syncthreads();
  const long long n = a.n;
  long long ring[REFRESH_RING];
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    if (a.status[k] != TRAJ_OK || a.head[k] < 0) continue;
    R p[NP], y[D];
#pragma unroll
    for (int q = 0; q < NP; ++q) p[q] = (R)a.params[q * n + k];
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = (R)y0[c * n + k];
    const int S = a.S[k];
    const int nseg = (S + a.k - 1) / a.k;
    bool ok = true;
    for (int c0 = 0; c0 < nseg && ok; c0 += REFRESH_RING) {
      const int c1 = min(nseg, c0 + REFRESH_RING);
      long long seg = a.head[k];
      for (int pos = nseg - 1; pos >= c0; --pos) {
        if (seg < 0 || seg >= a.arena_cap) { ok = false; break; }
        if (pos < c1) ring[pos - c0] = seg;
        seg = __double_as_longlong(arena[seg * a.segw]);
      }
      for (int pos = c0; pos < c1 && ok; ++pos) {
        double* sp = arena + ring[pos - c0] * a.segw;
#pragma unroll
        for (int c = 0; c < D; ++c) sp[2 + c] = to_d(y[c]);
        const int m = (pos == nseg - 1) ? S - (nseg - 1) * a.k : a.k;
        for (int j = 0; j < m; ++j) {
          R yn[D];
          ok = ok && M::template replay_step<Pb, R>(y, p, sp[2 + D + j], yn);
#pragma unroll
          for (int c = 0; c < D; ++c) y[c] = yn[c];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) y_final[c * n + k] = ok ? to_d(y[c]) : nan_d();
  }
}

inline int sm_count();

template <class M, class Pb, class R>
inline cudaError_t refresh_dispatch(const RevArgs& a, double* arena, double* y_final, const double* y0,
                                    cudaStream_t s) {
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, refresh_kernel<M, Pb, R>, TPB_REV, 0);
  long long blocks = (long long)sm_count() * (bps > 0 ? bps : 1);
  const long long need = (a.n + TPB_REV - 1) / TPB_REV;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  refresh_kernel<M, Pb, R><<<(unsigned)blocks, TPB_REV, 0, s>>>(a, arena, y_final, y0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
inline int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Persistent grid: as many CTAs as fit on the SMs at once (no more than the
// ensemble needs).
template <class Kern>
inline cudaError_t persistent_launch(Kern kern, int tpb, size_t smem, long long n, cudaStream_t s,
                                     const void* args_ptr) {
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int bps = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, tpb, smem);
  if (err != cudaSuccess) return err;
  long long blocks = (long long)sm_count() * (bps > 0 ? bps : 1);
  const long long need = (n + tpb - 1) / tpb;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  void* args[] = {const_cast<void*>(args_ptr)};
  return cudaLaunchKernel((const void*)kern, dim3((unsigned)blocks), dim3(tpb), args, smem, s);
}

#ifndef GS_INIT_STEP_PASS
#define GS_INIT_STEP_PASS 1
#endif
// Launches the starting-step pass when the record would compute starting steps
// (no h0 given); returns whether it ran.
template <class M, class Pb, class R, bool C64>
inline bool init_step_pass(FwdArgs& a, cudaStream_t s, cudaError_t* err) {
  *err = cudaSuccess;
  if constexpr (!GS_INIT_STEP_PASS) {
    return false;
  } else {
    if (a.h0 > 0.0 || a.n <= 0) return false;
    // y_final is the scratch: not when it overlaps the inputs (an in-place call)
    const char* yf = reinterpret_cast<const char*>(a.y_final);
    const size_t yf_bytes = (size_t)a.n * sizeof(double);
    auto overlaps = [&](const double* p, int rows) {
      const char* b = reinterpret_cast<const char*>(p);
      return b < yf + yf_bytes && yf < b + (size_t)rows * a.n * sizeof(double);
    };
    if (overlaps(a.params, Pb::NP) || overlaps(a.y0, Pb::D)) return false;
    long long blocks = (a.n + 255) / 256;
    const long long cap = (long long)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    a.h0_pre = (carry_from_pass<M, R>() && a.head) ? 2 : 1;
    init_step_kernel<M, Pb, R, C64><<<(unsigned)blocks, 256, 0, s>>>(a);
    *err = cudaGetLastError();
    if (*err != cudaSuccess) a.h0_pre = 0;
    return *err == cudaSuccess;
  }
}

template <class M, class Pb, class R>
inline cudaError_t fwd_dispatch(const FwdArgs& a_in, cudaStream_t s) {
  FwdArgs a = a_in;
  {
    cudaError_t e = cudaSuccess;
    a.h0_pre = 0;
    if constexpr (M::kControl64 && !HasWeights<Pb>::value) {  // (FP64 control: no shared weights)
      if (a.control)
        init_step_pass<M, Pb, R, true>(a, s, &e);
      else
        init_step_pass<M, Pb, R, false>(a, s, &e);
    } else {
      init_step_pass<M, Pb, R, false>(a, s, &e);
    }
    if (e != cudaSuccess) return e;
  }
  const size_t smem = (size_t)(((a.n_save + 1) & ~1) + a.segw * TPB_FWD) * sizeof(double);
  if (a.control) {  // FP64 step control: Tsit5 without shared weights
    if constexpr (M::kControl64 && !HasWeights<Pb>::value) {
      if constexpr (stages_possible<M, Pb, R>()) {
        if (a.stages)
          return persistent_launch(record_entry<M, Pb, R, true, true, true>(), TPB_FWD, smem, a.n, s, &a);
      } else {
        if (a.stages) return cudaErrorInvalidValue;
      }
      if (a.y_save) return persistent_launch(record_entry<M, Pb, R, true, false, true>(), TPB_FWD, smem, a.n, s, &a);
      return persistent_launch(record_entry<M, Pb, R, false, false, true>(), TPB_FWD, smem, a.n, s, &a);
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if constexpr (stages_possible<M, Pb, R>()) {
    if (a.stages) return persistent_launch(record_kernel<M, Pb, R, true, true>, TPB_FWD, smem, a.n, s, &a);
  } else {
    if (a.stages) return cudaErrorInvalidValue;
  }
  if (a.y_save) return persistent_launch(record_kernel<M, Pb, R, true, false>, TPB_FWD, smem, a.n, s, &a);
  return persistent_launch(record_kernel<M, Pb, R, false, false>, TPB_FWD, smem, a.n, s, &a);
}

#ifndef GS_T1_SAVE_PASS
#define GS_T1_SAVE_PASS 1
#endif
// Launches the t1-save pass for the FP64 k = 1 reverse sweep when the last save
// time is t1 and y0_bar is given (and overlaps none of the sweep's inputs);
// returns whether it ran.
template <class Pb, class R>
inline bool t1_save_pass(const RevArgs& a, cudaStream_t s, cudaError_t* err) {
  *err = cudaSuccess;
  if constexpr (!std::is_same<R, double>::value || HasWeights<Pb>::value || !GS_T1_SAVE_PASS) {
    return false;
  } else {
    const int ns = a.n_save;
    if (a.n <= 0 || !a.y0_bar || ns < 1 || a.k != 1) return false;
    if (std::memcmp(&a.save_t[ns - 1], &a.t1, sizeof(double)) != 0) return false;
    auto overlaps = [](const void* x, size_t xb, const void* y, size_t yb) {
      const char *p = static_cast<const char*>(x), *q = static_cast<const char*>(y);
      return p && q && p < q + yb && q < p + xb;
    };
    const size_t nb = (size_t)a.n * sizeof(double);
    const void* outs[2] = {a.y0_bar, a.loss};
    const size_t outb[2] = {nb * Pb::D, nb};
    const void* ins[3] = {a.params, a.y_save_bar, a.y_final};
    const size_t inb[3] = {nb * Pb::NP, nb * Pb::D * (size_t)ns, nb * Pb::D};
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j)
        if (overlaps(outs[i], outb[i], ins[j], inb[j])) return false;
    long long blocks = (a.n + 255) / 256;
    const long long cap = (long long)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (a.y_save_bar)
      t1_save_kernel<Pb, true><<<(unsigned)blocks, 256, 0, s>>>(a);
    else
      t1_save_kernel<Pb, false><<<(unsigned)blocks, 256, 0, s>>>(a);
    *err = cudaGetLastError();
    return *err == cudaSuccess;
  }
}

template <class M, class Pb, class R>
inline cudaError_t rev_dispatch(const RevArgs& a_in, cudaStream_t s) {
  RevArgs a = a_in;
  a.t1_pre = 0;
  size_t smem = (size_t)((a.n_save + 1) & ~1) * sizeof(double);
  if constexpr (HasWeights<Pb>::value) {
    using Acc = AccFor<Pb, R>;
    if (a.k != 1) return cudaErrorInvalidValue;
    smem += weight_stage_bytes<Pb>();
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, reverse_k1_kernel<M, Pb, R, false>, TPB_REV, smem);
    cudaError_t e = a.y_save_bar ? persistent_launch(reverse_k1_kernel<M, Pb, R, true>, TPB_REV, smem, a.n, s, &a)
                                 : persistent_launch(reverse_k1_kernel<M, Pb, R, false>, TPB_REV, smem, a.n, s, &a);
    if (e != cudaSuccess || !a.wpart || !a.shared_w_bar) return e;
    long long blocks = (long long)sm_count() * (bps > 0 ? bps : 1);
    const long long need = (a.n + TPB_REV - 1) / TPB_REV;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    using Part = typename Acc::Part;
    weight_reduce_kernel<Part><<<(Acc::NW + 127) / 128, 128, 0, s>>>(static_cast<const Part*>(a.wpart), Acc::NW,
                                                                      (int)(blocks * (TPB_REV / 32)), a.shared_w_bar);
    return cudaGetLastError();
  } else {
  if (a.k == 1) {
    cudaError_t e;
    a.t1_pre = t1_save_pass<Pb, R>(a, s, &e) ? 1 : 0;
    if (e != cudaSuccess) return e;
  }
  if constexpr (stages_possible<M, Pb, R>()) {
    if (a.stages) {
      if (a.k != 1 || a.segw != stage_segw<M, Pb::D>()) return cudaErrorInvalidValue;
      if (a.y_save_bar)
        return persistent_launch(reverse_k1_entry<M, Pb, R, true, true>(), TPB_REV, smem, a.n, s, &a);
      return persistent_launch(reverse_k1_entry<M, Pb, R, false, true>(), TPB_REV, smem, a.n, s, &a);
    }
  } else {
    if (a.stages) return cudaErrorInvalidValue;
  }
  if (a.k == 1) {
    if (a.y_save_bar) return persistent_launch(reverse_k1_entry<M, Pb, R, true>(), TPB_REV, smem, a.n, s, &a);
    return persistent_launch(reverse_k1_entry<M, Pb, R, false>(), TPB_REV, smem, a.n, s, &a);
  }
  if (a.y_save_bar) return persistent_launch(reverse_kernel<M, Pb, R, true>, TPB_REV, smem, a.n, s, &a);
  return persistent_launch(reverse_kernel<M, Pb, R, false>, TPB_REV, smem, a.n, s, &a);
  }
}

}  // namespace gs
