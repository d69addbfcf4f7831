// Rodas5P (Steinebach 2023): the stiff one-step map of the paper's Sec. 3.2,
// its per-lane dense LU, and the discrete adjoint of one step.
//
// Transformed Rosenbrock form, with W = I/(h gamma) - J(y):
//   W U_i = f(y + sum_{j<i} a_ij U_j) + (1/h) sum_{j<i} C_ij U_j,  i = 1..8,
//   y_new = y + sum_j m_j U_j,
// stiffly accurate: rows 7 and 8 of a extend row 6 by ones and m = (a_8., 1),
// so y_new = Y_8 + U_8 and the embedded solution is Y_8 = y_new - U_8 (error
// estimate U_8). All problems here are autonomous (no df/dt term).
#pragma once

#include "gs_device.cuh"

namespace gs {
namespace rodas {

constexpr double GAMMA = 0.21193756319429014;

__host__ __device__ constexpr double A6(int j) {  // row 6 (1-based), extended into rows 7 and 8
  return j == 0   ? -7.502846399306121
         : j == 1 ? 2.561846144803919
         : j == 2 ? -11.627539656261098
         : j == 3 ? -0.18268767659942256
         : j == 4 ? 0.030198172008377946
                  : 0.0;
}
// a_ij, 0-based stage i (1..7), j < i.
__host__ __device__ constexpr double a(int i, int j) {
  return (i == 1 && j == 0)   ? 3.0
         : (i == 2 && j == 0) ? 2.849394379747939
         : (i == 2 && j == 1) ? 0.45842242204463923
         : (i == 3 && j == 0) ? -6.954028509809101
         : (i == 3 && j == 1) ? 2.489845061869568
         : (i == 3 && j == 2) ? -10.358996098473584
         : (i == 4 && j == 0) ? 2.8029986275628964
         : (i == 4 && j == 1) ? 0.5072464736228206
         : (i == 4 && j == 2) ? -0.3988312541770524
         : (i == 4 && j == 3) ? -0.04721187230404641
         : (i == 5 && j < 5)  ? A6(j)
         : (i == 6 && j < 5)  ? A6(j)
         : (i == 6 && j == 5) ? 1.0
         : (i == 7 && j < 5)  ? A6(j)
         : (i == 7 && j == 5) ? 1.0
         : (i == 7 && j == 6) ? 1.0
                              : 0.0;
}
__host__ __device__ constexpr double C(int i, int j) {
  return (i == 1 && j == 0)   ? -14.155112264123755
         : (i == 2 && j == 0) ? -17.97296035885952
         : (i == 2 && j == 1) ? -2.859693295451294
         : (i == 3 && j == 0) ? 147.12150275711716
         : (i == 3 && j == 1) ? -1.41221402718213
         : (i == 3 && j == 2) ? 71.68940251302358
         : (i == 4 && j == 0) ? 165.43517024871676
         : (i == 4 && j == 1) ? -0.4592823456491126
         : (i == 4 && j == 2) ? 42.90938336958603
         : (i == 4 && j == 3) ? -5.961986721573306
         : (i == 5 && j == 0) ? 24.854864614690072
         : (i == 5 && j == 1) ? -3.0009227002832186
         : (i == 5 && j == 2) ? 47.4931110020768
         : (i == 5 && j == 3) ? 5.5814197821558125
         : (i == 5 && j == 4) ? -0.6610691825249471
         : (i == 6 && j == 0) ? 30.91273214028599
         : (i == 6 && j == 1) ? -3.1208243349937974
         : (i == 6 && j == 2) ? 77.79954646070892
         : (i == 6 && j == 3) ? 34.28646028294783
         : (i == 6 && j == 4) ? -19.097331116725623
         : (i == 6 && j == 5) ? -28.087943162872662
         : (i == 7 && j == 0) ? 37.80277123390563
         : (i == 7 && j == 1) ? -3.2571969029072276
         : (i == 7 && j == 2) ? 112.26918849496327
         : (i == 7 && j == 3) ? 66.9347231244047
         : (i == 7 && j == 4) ? -40.06618937091002
         : (i == 7 && j == 5) ? -54.66780262877968
         : (i == 7 && j == 6) ? -9.48861652309627
                              : 0.0;
}
__host__ __device__ constexpr double m(int j) { return j < 7 ? a(7, j) : 1.0; }

}  // namespace rodas

// ---------------------------------------------------------------------------
// Dense LU with partial pivoting (Doolittle; ties pick the lowest row index),
// fully unrolled and branch-free: row swaps are selects, so the matrix stays
// in registers. piv[k] is the row swapped with row k at column k; rinv[k] is
// 1 / U_kk. Returns false on an exactly zero pivot.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ bool lu_factor(double (&A)[D][D], int (&piv)[D], double (&rinv)[D]) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    int pr = k;
    double best = fabs(A[k][k]);
#pragma unroll
    for (int i = k + 1; i < D; ++i) {
      const double v = fabs(A[i][k]);
      const bool gt = v > best;
      best = gt ? v : best;
      pr = gt ? i : pr;
    }
    piv[k] = pr;
    ok = ok && (best != 0.0);
#pragma unroll
    for (int i = k + 1; i < D; ++i) {
      const bool sw = (i == pr);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const double t = A[k][j];
        A[k][j] = sw ? A[i][j] : t;
        A[i][j] = sw ? t : A[i][j];
      }
    }
    rinv[k] = 1.0 / A[k][k];
#pragma unroll
    for (int i = k + 1; i < D; ++i) {
      const double l = mul_(A[i][k], rinv[k]);
      A[i][k] = l;
#pragma unroll
      for (int j = k + 1; j < D; ++j) A[i][j] = fma_(-l, A[k][j], A[i][j]);
    }
  }
  return ok;
}

// Solve W x = b with the factors (apply the row swaps, then L and U).
template <int D>
__device__ __forceinline__ void lu_solve(const double (&LU)[D][D], const int (&piv)[D], const double (&rinv)[D],
                                         const double (&b)[D], double (&x)[D]) {
  double z[D];
#pragma unroll
  for (int i = 0; i < D; ++i) z[i] = b[i];
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int i = k + 1; i < D; ++i) {
      const bool sw = (i == piv[k]);
      const double t = z[k];
      z[k] = sw ? z[i] : t;
      z[i] = sw ? t : z[i];
    }
  }
#pragma unroll
  for (int i = 1; i < D; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) z[i] = fma_(-LU[i][j], z[j], z[i]);
#pragma unroll
  for (int i = D - 1; i >= 0; --i) {
    double s = z[i];
#pragma unroll
    for (int j = i + 1; j < D; ++j) s = fma_(-LU[i][j], x[j], s);
    x[i] = mul_(s, rinv[i]);
  }
}

// Solve W^T x = b: U^T w = b, L^T v = w, then undo the row swaps in reverse.
template <int D>
__device__ __forceinline__ void lu_solve_t(const double (&LU)[D][D], const int (&piv)[D], const double (&rinv)[D],
                                           const double (&b)[D], double (&x)[D]) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = b[i];
#pragma unroll
    for (int j = 0; j < i; ++j) s = fma_(-LU[j][i], x[j], s);
    x[i] = mul_(s, rinv[i]);
  }
#pragma unroll
  for (int i = D - 2; i >= 0; --i)
#pragma unroll
    for (int j = i + 1; j < D; ++j) x[i] = fma_(-LU[j][i], x[j], x[i]);
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
#pragma unroll
    for (int i = k + 1; i < D; ++i) {
      const bool sw = (i == piv[k]);
      const double t = x[k];
      x[k] = sw ? x[i] : t;
      x[i] = sw ? t : x[i];
    }
  }
}

// One Rodas5P step from y with size h: stage inputs Y[0..7], stage solutions
// U[0..7], the LU of W, y_new and the error estimate U[7]. false if W is singular.
// Stage input Y_i = y + sum_{j<i} a_ij U_j, in a fixed order (the step and
// the stored-stage reverse build it the same way).
template <int D>
__device__ __forceinline__ void rodas_stage_input(int i, const double (&y)[D], const double (&U)[8][D],
                                                  double (&Yi)[D]) {
#pragma unroll
  for (int c = 0; c < D; ++c) {
    double s = y[c];
#pragma unroll
    for (int j = 0; j < i; ++j) s = fma_(rodas::a(i, j), U[j][c], s);
    Yi[c] = s;
  }
}
template <int D>
__device__ __forceinline__ void rodas_stage_inputs(const double (&y)[D], const double (&U)[8][D],
                                                   double (&Y)[8][D]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) rodas_stage_input<D>(i, y, U, Y[i]);
}

template <class Pb>
__device__ __forceinline__ bool rodas_step(const double (&y)[Pb::D], const double (&p)[Pb::NP], double h,
                                           double (&Y)[8][Pb::D], double (&U)[8][Pb::D], double (&LU)[Pb::D][Pb::D],
                                           int (&piv)[Pb::D], double (&rinv)[Pb::D], double (&ynew)[Pb::D]) {
  constexpr int D = Pb::D;
  Pb::jac(y, p, LU);
  const double inv_hg = 1.0 / mul_(h, rodas::GAMMA);
  const double inv_h = 1.0 / h;
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) LU[i][j] = -LU[i][j];
    LU[i][i] = add_(LU[i][i], inv_hg);
  }
  const bool ok = lu_factor<D>(LU, piv, rinv);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    double F[D], Rhs[D];
    rodas_stage_input<D>(i, y, U, Y[i]);
    Pb::f(Y[i], p, F);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (i == 0) {
        Rhs[c] = F[c];
      } else {
        double s = mul_(rodas::C(i, 0), U[0][c]);
#pragma unroll
        for (int j = 1; j < i; ++j) s = fma_(rodas::C(i, j), U[j][c], s);
        Rhs[c] = fma_(inv_h, s, F[c]);
      }
    }
    lu_solve<D>(LU, piv, rinv, Rhs, U[i]);
  }
#pragma unroll
  for (int c = 0; c < D; ++c) ynew[c] = add_(Y[7][c], U[7][c]);
  return ok;
}

// Forward mode of one Rodas5P step with h held as data: y_new (the arithmetic
// of rodas_step) and, for each of ND tangent directions (yd, pd),
//   W Ud_i = Fd_i + (1/h) sum_{j<i} C_ij Ud_j + Jd U_i,
//   Fd_i = J(Y_i) Yd_i + f_theta(Y_i) pd,  Yd_i = yd + sum_{j<i} a_ij Ud_j,
// where Jd = dJ(y)[yd, pd] (W = I/(h gamma) - J(y), so dW = -Jd), and
// yd_new = Yd_8 + Ud_8. false if W is singular.
template <class Pb, int ND>
__device__ __forceinline__ bool rodas_tangent(const double (&y)[Pb::D], const double (&yd)[ND][Pb::D],
                                              const double (&p)[Pb::NP], const double (&pd)[ND][Pb::NP], double h,
                                              double (&yn)[Pb::D], double (&ydn)[ND][Pb::D]) {
  constexpr int D = Pb::D;
  double LU[D][D], rinv[D], U[8][D], Ud[8][ND][D];
  int piv[D];
  Pb::jac(y, p, LU);
  const double inv_hg = 1.0 / mul_(h, rodas::GAMMA);
  const double inv_h = 1.0 / h;
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) LU[i][j] = -LU[i][j];
    LU[i][i] = add_(LU[i][i], inv_hg);
  }
  const bool ok = lu_factor<D>(LU, piv, rinv);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    double Y[D], F[D], Rhs[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double s = y[c];
#pragma unroll
      for (int j = 0; j < i; ++j) s = fma_(rodas::a(i, j), U[j][c], s);
      Y[c] = s;
    }
    Pb::f(Y, p, F);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (i == 0) {
        Rhs[c] = F[c];
      } else {
        double s = mul_(rodas::C(i, 0), U[0][c]);
#pragma unroll
        for (int j = 1; j < i; ++j) s = fma_(rodas::C(i, j), U[j][c], s);
        Rhs[c] = fma_(inv_h, s, F[c]);
      }
    }
    lu_solve<D>(LU, piv, rinv, Rhs, U[i]);
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      double Yd[D], Fd[D], JdU[D], Rd[D];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double s = yd[q][c];
#pragma unroll
        for (int j = 0; j < i; ++j) s = fma_(rodas::a(i, j), Ud[j][q][c], s);
        Yd[c] = s;
      }
      Pb::jvp(Y, p, Yd, pd[q], Fd);
      Pb::jac_dir(y, p, yd[q], pd[q], U[i], JdU);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        if (i == 0) {
          Rd[c] = add_(Fd[c], JdU[c]);
        } else {
          double s = mul_(rodas::C(i, 0), Ud[0][q][c]);
#pragma unroll
          for (int j = 1; j < i; ++j) s = fma_(rodas::C(i, j), Ud[j][q][c], s);
          Rd[c] = add_(fma_(inv_h, s, Fd[c]), JdU[c]);
        }
      }
      lu_solve<D>(LU, piv, rinv, Rd, Ud[i][q]);
      if (i == 7) {
#pragma unroll
        for (int c = 0; c < D; ++c) ydn[q][c] = add_(Yd[c], Ud[7][q][c]);
      }
    }
    if (i == 7) {
#pragma unroll
      for (int c = 0; c < D; ++c) yn[c] = add_(Y[c], U[7][c]);
    }
  }
  return ok;
}

// Reverse of one Rodas5P step (h held as data) over its recomputed stages:
// given the cotangent lam of y_new, returns v = dL/dy and accumulates dL/dtheta.
//   Ubar_j = m_j lam;  for i = 8..1: Rbar_i = W^{-T} Ubar_i,
//   Ubar_j += (C_ij / h) Rbar_i, Ybar_i = J(Y_i)^T Rbar_i, theta_bar += f_theta(Y_i)^T Rbar_i,
//   v += Ybar_i, Ubar_j += a_ij Ybar_i;
// and W = I/(h gamma) - J(y) gives dL/dJ = sum_i Rbar_i U_i^T, contracted through
// J(y, theta): v += d/dy (Rbar_i^T J U_i), theta_bar += d/dtheta (Rbar_i^T J U_i).
template <class Pb, class Acc>
__device__ __forceinline__ void rodas_reverse(const double (&y)[Pb::D], const double (&p)[Pb::NP], double h,
                                              const double (&Y)[8][Pb::D], const double (&U)[8][Pb::D],
                                              const double (&LU)[Pb::D][Pb::D], const int (&piv)[Pb::D],
                                              const double (&rinv)[Pb::D], const double (&lam)[Pb::D],
                                              double (&v)[Pb::D], Acc& pacc) {
  constexpr int D = Pb::D;
  const double inv_h = 1.0 / h;
  double Ub[8][D];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int c = 0; c < D; ++c) Ub[j][c] = (j == 7) ? lam[c] : mul_(rodas::m(j), lam[c]);
#pragma unroll
  for (int c = 0; c < D; ++c) v[c] = lam[c];
#pragma unroll
  for (int i = 7; i >= 0; --i) {
    double Rb[D], Yb[D], Rh[D];
    lu_solve_t<D>(LU, piv, rinv, Ub[i], Rb);
#pragma unroll
    for (int c = 0; c < D; ++c) Rh[c] = mul_(inv_h, Rb[c]);
#pragma unroll
    for (int j = 0; j < i; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c) Ub[j][c] = fma_(rodas::C(i, j), Rh[c], Ub[j][c]);
    pacc.template vjp<Pb>(Y[i], p, Rb, Yb);
#pragma unroll
    for (int c = 0; c < D; ++c) v[c] = add_(v[c], Yb[c]);
#pragma unroll
    for (int j = 0; j < i; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c) Ub[j][c] = fma_(rodas::a(i, j), Yb[c], Ub[j][c]);
    pacc.template jac_contract<Pb>(y, p, Rb, U[i], v);
  }
}

// ---------------------------------------------------------------------------
// Rosenbrock23 (Shampine & Reichelt 1997, the ode23s formulas; the paper's
// second-order stiff method, Sec. 3.2), autonomous f, W = I - h d J(y):
//   k1 = W^{-1} F0 (F0 = f(y)),  Y1 = y + h/2 k1,  F1 = f(Y1),
//   u2 = W^{-1} (F1 - k1),  k2 = u2 + k1,  y_new = y + h k2,
//   F2 = f(y_new),  k3 = W^{-1} (F2 - e32 (k2 - F1) - 2 (k1 - F0)),
//   e = h/6 (k1 - 2 k2 + k3);  d = 1/(2 + sqrt 2), e32 = 6 + sqrt 2.
// F2 is f at the next accepted state (first-same-as-last).
// ---------------------------------------------------------------------------
namespace ros23 {
constexpr double DC = 0.2928932188134525;   // 1 / (2 + sqrt 2)
constexpr double E32 = 7.414213562373095;   // 6 + sqrt 2
}  // namespace ros23

// W = I - h d J(y), factored. false if singular.
template <class Pb>
__device__ __forceinline__ bool ros23_factor(const double (&y)[Pb::D], const double (&p)[Pb::NP], double h,
                                             double (&LU)[Pb::D][Pb::D], int (&piv)[Pb::D], double (&rinv)[Pb::D]) {
  constexpr int D = Pb::D;
  Pb::jac(y, p, LU);
  const double mhd = -mul_(h, ros23::DC);
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) LU[i][j] = mul_(mhd, LU[i][j]);
    LU[i][i] = add_(LU[i][i], 1.0);
  }
  return lu_factor<D>(LU, piv, rinv);
}

// The replay map with its stage quantities: k1, u2, Y1, F1 and y_new, from
// y, F0 = f(y) and the factored W.
template <class Pb>
__device__ __forceinline__ void ros23_stages(const double (&y)[Pb::D], const double (&p)[Pb::NP], double h,
                                             const double (&F0)[Pb::D], const double (&LU)[Pb::D][Pb::D],
                                             const int (&piv)[Pb::D], const double (&rinv)[Pb::D],
                                             double (&k1)[Pb::D], double (&u2)[Pb::D], double (&Y1)[Pb::D],
                                             double (&F1)[Pb::D], double (&ynew)[Pb::D]) {
  constexpr int D = Pb::D;
  lu_solve<D>(LU, piv, rinv, F0, k1);
  const double hh = mul_(0.5, h);
#pragma unroll
  for (int c = 0; c < D; ++c) Y1[c] = fma_(hh, k1[c], y[c]);
  Pb::f(Y1, p, F1);
  double r[D];
#pragma unroll
  for (int c = 0; c < D; ++c) r[c] = sub_(F1[c], k1[c]);
  lu_solve<D>(LU, piv, rinv, r, u2);
#pragma unroll
  for (int c = 0; c < D; ++c) ynew[c] = fma_(h, add_(u2[c], k1[c]), y[c]);
}

// Trial step of the record: y_new, the error estimate e and F2 = f(y_new), and
// the step's factored W and stage solutions k1, u2 (what a stored-stage record
// keeps).
template <class Pb>
__device__ __forceinline__ bool ros23_trial(const double (&y)[Pb::D], const double (&p)[Pb::NP], double h,
                                            const double (&F0)[Pb::D], double (&ynew)[Pb::D], double (&e)[Pb::D],
                                            double (&F2)[Pb::D], double (&LU)[Pb::D][Pb::D], int (&piv)[Pb::D],
                                            double (&rinv)[Pb::D], double (&k1)[Pb::D], double (&u2)[Pb::D]) {
  constexpr int D = Pb::D;
  double Y1[D], F1[D], r[D], k3[D];
  const bool ok = ros23_factor<Pb>(y, p, h, LU, piv, rinv);
  ros23_stages<Pb>(y, p, h, F0, LU, piv, rinv, k1, u2, Y1, F1, ynew);
  Pb::f(ynew, p, F2);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const double k2 = add_(u2[c], k1[c]);
    r[c] = fma_(-ros23::E32, sub_(k2, F1[c]), fma_(-2.0, sub_(k1[c], F0[c]), F2[c]));
  }
  lu_solve<D>(LU, piv, rinv, r, k3);
  const double h6 = h / 6.0;
#pragma unroll
  for (int c = 0; c < D; ++c) e[c] = mul_(h6, add_(fma_(-2.0, add_(u2[c], k1[c]), k1[c]), k3[c]));
  return ok;
}
template <class Pb>
__device__ __forceinline__ bool ros23_trial(const double (&y)[Pb::D], const double (&p)[Pb::NP], double h,
                                            const double (&F0)[Pb::D], double (&ynew)[Pb::D], double (&e)[Pb::D],
                                            double (&F2)[Pb::D]) {
  constexpr int D = Pb::D;
  double LU[D][D], rinv[D], k1[D], u2[D];
  int piv[D];
  return ros23_trial<Pb>(y, p, h, F0, ynew, e, F2, LU, piv, rinv, k1, u2);
}

// Reverse of one Rosenbrock23 step (h held as data): given lam = dL/dy_new,
// returns v = dL/dy and accumulates dL/dtheta:
//   k2bar = h lam, r2bar = W^{-T} k2bar, F1bar = r2bar, k1bar = k2bar - r2bar,
//   Y1bar = J(Y1)^T r2bar (theta_bar += f_theta(Y1)^T r2bar), k1bar += h/2 Y1bar,
//   r1bar = W^{-T} k1bar, v = lam + Y1bar + J(y)^T r1bar (theta_bar += f_theta(y)^T r1bar),
// and dL/dJ = h d (r1bar k1^T + r2bar u2^T) contracted through J(y, theta).
template <class Pb, class Acc>
__device__ __forceinline__ void ros23_reverse(const double (&y)[Pb::D], const double (&p)[Pb::NP], double h,
                                              const double (&k1)[Pb::D], const double (&u2)[Pb::D],
                                              const double (&Y1)[Pb::D], const double (&LU)[Pb::D][Pb::D],
                                              const int (&piv)[Pb::D], const double (&rinv)[Pb::D],
                                              const double (&lam)[Pb::D], double (&v)[Pb::D], Acc& pacc) {
  constexpr int D = Pb::D;
  double k2b[D], r2b[D], k1b[D], r1b[D], Y1b[D], y0b[D];
#pragma unroll
  for (int c = 0; c < D; ++c) k2b[c] = mul_(h, lam[c]);
  lu_solve_t<D>(LU, piv, rinv, k2b, r2b);
  pacc.template vjp<Pb>(Y1, p, r2b, Y1b);
  const double hh = mul_(0.5, h);
#pragma unroll
  for (int c = 0; c < D; ++c) k1b[c] = fma_(hh, Y1b[c], sub_(k2b[c], r2b[c]));
  lu_solve_t<D>(LU, piv, rinv, k1b, r1b);
  pacc.template vjp<Pb>(y, p, r1b, y0b);
#pragma unroll
  for (int c = 0; c < D; ++c) v[c] = add_(add_(lam[c], Y1b[c]), y0b[c]);
  const double hd = mul_(h, ros23::DC);
  double r1s[D], r2s[D];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    r1s[c] = mul_(hd, r1b[c]);
    r2s[c] = mul_(hd, r2b[c]);
  }
  pacc.template jac_contract<Pb>(y, p, r1s, k1, v);
  pacc.template jac_contract<Pb>(y, p, r2s, u2, v);
}

// Forward mode of one Rosenbrock23 step (h held as data), ND directions:
//   Jd = dJ(y)[yd, pd], dW = -h d Jd;
//   kd1 = W^{-1} (Fd0 + h d Jd k1),  Fd0 = J(y) yd + f_theta(y) pd;
//   Yd1 = yd + h/2 kd1,  Fd1 = J(Y1) Yd1 + f_theta(Y1) pd;
//   ud2 = W^{-1} (Fd1 - kd1 + h d Jd u2);  yd_new = yd + h (ud2 + kd1).
template <class Pb, int ND>
__device__ __forceinline__ bool ros23_tangent(const double (&y)[Pb::D], const double (&yd)[ND][Pb::D],
                                              const double (&p)[Pb::NP], const double (&pd)[ND][Pb::NP], double h,
                                              double (&yn)[Pb::D], double (&ydn)[ND][Pb::D]) {
  constexpr int D = Pb::D;
  double LU[D][D], rinv[D], F0[D], k1[D], u2[D], Y1[D], F1[D];
  int piv[D];
  const bool ok = ros23_factor<Pb>(y, p, h, LU, piv, rinv);
  Pb::f(y, p, F0);
  ros23_stages<Pb>(y, p, h, F0, LU, piv, rinv, k1, u2, Y1, F1, yn);
  const double hd = mul_(h, ros23::DC), hh = mul_(0.5, h);
#pragma unroll
  for (int q = 0; q < ND; ++q) {
    double Fd[D], JdU[D], r[D], kd1[D], Yd1[D], ud2[D];
    Pb::jvp(y, p, yd[q], pd[q], Fd);
    Pb::jac_dir(y, p, yd[q], pd[q], k1, JdU);
#pragma unroll
    for (int c = 0; c < D; ++c) r[c] = fma_(hd, JdU[c], Fd[c]);
    lu_solve<D>(LU, piv, rinv, r, kd1);
#pragma unroll
    for (int c = 0; c < D; ++c) Yd1[c] = fma_(hh, kd1[c], yd[q][c]);
    Pb::jvp(Y1, p, Yd1, pd[q], Fd);
    Pb::jac_dir(y, p, yd[q], pd[q], u2, JdU);
#pragma unroll
    for (int c = 0; c < D; ++c) r[c] = fma_(hd, JdU[c], sub_(Fd[c], kd1[c]));
    lu_solve<D>(LU, piv, rinv, r, ud2);
#pragma unroll
    for (int c = 0; c < D; ++c) ydn[q][c] = fma_(h, add_(ud2[c], kd1[c]), yd[q][c]);
  }
  return ok;
}

}  // namespace gs
