// gradsolve oracle: a plain, slow, obviously correct FP64 CPU implementation of
// the record-and-replay gradient of an ensemble of ODE trajectories.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load
// this file; only the tests, the smoke check and the CPU-baseline leg of the
// benchmark use it. It shares no code, header, table or constant with the CUDA
// library: every coefficient below is typed here from the method's publication.
//
// What it computes (paper, Sec. 3.1 "The construction", Eq. (replay)):
//   record  R:  an adaptive solve that keeps the accepted step sizes {h_i};
//   replay  Psi: the fixed chain y_i = Phi(y_{i-1}; h_i, theta), i = 1..S,
//               with h held as data (stop-gradient);
//   gradient:   the exact reverse-mode derivative of the replay's loss with
//               respect to theta and y0 (the discrete adjoint).
//
// Derivatives of the right-hand side (J = df/dy, df/dtheta and the second
// derivative contractions the stiff adjoint needs) are taken by forward-mode
// dual numbers applied to f itself, so the only hand-typed model code is f,
// exactly as printed in the paper's Appendix A ("Benchmark problem definitions").
//
// Parity pins: see tests/test_oracle_*.py (order conditions, closed-form linear
// replay, complex-step gradients, finite differences, invariants, Rosenbrock23's
// stability function and error estimate, the neural term's weight derivatives;
// the starting step and the controller against scipy's implementations of the
// same textbook rules, for Tsit5 and Verner7, and for the two Rosenbrock
// methods with scipy's driver stepping with this file's Rosenbrock step; with
// planted mistakes caught).
//
// Parity unpinned (no value outside this file fixes them; they only shape the
// mesh, which the gradient treats as data): the end-of-span sliver 1e-12, the
// quartered step after a singular linear system, and Rodas5P's coefficients
// beyond what its order conditions and stiff accuracy fix.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------- scalars
inline double tanh_(double x) { return std::tanh(x); }

template <class T> struct Dual {
  T v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(const T& v_, const T& d_) : v(v_), d(d_) {}
};
template <class T> Dual<T> operator+(const Dual<T>& a, const Dual<T>& b) { return {a.v + b.v, a.d + b.d}; }
template <class T> Dual<T> operator-(const Dual<T>& a, const Dual<T>& b) { return {a.v - b.v, a.d - b.d}; }
template <class T> Dual<T> operator-(const Dual<T>& a) { return {-a.v, -a.d}; }
template <class T> Dual<T> operator*(const Dual<T>& a, const Dual<T>& b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T> Dual<T> operator/(const Dual<T>& a, const Dual<T>& b) {
  T q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <class T> Dual<T> operator+(const Dual<T>& a, double b) { return a + Dual<T>(b); }
template <class T> Dual<T> operator+(double a, const Dual<T>& b) { return Dual<T>(a) + b; }
template <class T> Dual<T> operator-(const Dual<T>& a, double b) { return a - Dual<T>(b); }
template <class T> Dual<T> operator-(double a, const Dual<T>& b) { return Dual<T>(a) - b; }
template <class T> Dual<T> operator*(const Dual<T>& a, double b) { return {a.v * b, a.d * b}; }
template <class T> Dual<T> operator*(double a, const Dual<T>& b) { return {b.v * a, b.d * a}; }
template <class T> Dual<T> operator/(const Dual<T>& a, double b) { return a / Dual<T>(b); }
template <class T> Dual<T>& operator+=(Dual<T>& a, const Dual<T>& b) { a = a + b; return a; }
template <class T> Dual<T>& operator-=(Dual<T>& a, const Dual<T>& b) { a = a - b; return a; }
template <class T> Dual<T> tanh_(const Dual<T>& a) {
  T t = tanh_(a.v);
  return {t, a.d * (1.0 - t * t)};
}

inline double val(double x) { return x; }
template <class T> double val(const Dual<T>& x) { return val(x.v); }

// ---------------------------------------------------------------- problems
// Problem ids (match the C-ABI's numbering; the numbers are the interface).
enum { P_LORENZ = 0, P_VDP = 1, P_ROBERTSON = 2, P_HIRES = 3, P_LINEAR = 4, P_LV_UDE = 5, P_NROB = 6 };
constexpr int DMAX = 8;
constexpr int PMAX = 12;
// LV UDE network: 2 -> 16 -> 16 -> 2, tanh hidden, linear output.
// Flat weight layout: W1[16][2], b1[16], W2[16][16], b2[16], W3[2][16], b3[2] = 354.
constexpr int UDE_H = 16;
constexpr int UDE_NW = UDE_H * 2 + UDE_H + UDE_H * UDE_H + UDE_H + 2 * UDE_H + 2;
// Robertson neural right-hand side (paper Appendix A): MLP 3 -> 16 -> 16 -> 1,
// tanh hidden, softplus output. Flat layout: W1[16][3], b1[16], W2[16][16],
// b2[16], W3[16], b3 = 353.
constexpr int NR_NW = UDE_H * 3 + UDE_H + UDE_H * UDE_H + UDE_H + UDE_H + 1;

int dim_of(int pid) {
  switch (pid) {
    case P_LORENZ: return 3;
    case P_VDP: return 2;
    case P_ROBERTSON: return 3;
    case P_HIRES: return 8;
    case P_LINEAR: return 2;
    case P_LV_UDE: return 2;
    case P_NROB: return 3;
  }
  return -1;
}
int npar_of(int pid) {
  switch (pid) {
    case P_LORENZ: return 3;
    case P_VDP: return 1;
    case P_ROBERTSON: return 3;
    case P_HIRES: return 12;
    case P_LINEAR: return 4;
    case P_LV_UDE: return 2;
    case P_NROB: return 2;  // k1, k3
  }
  return -1;
}
int stiff_of(int pid) { return (pid == P_ROBERTSON || pid == P_HIRES || pid == P_NROB) ? 1 : 0; }
int nshared_of(int pid) { return pid == P_LV_UDE ? UDE_NW : (pid == P_NROB ? NR_NW : 0); }

// softplus(x) = log(1 + e^x) and its derivative, the logistic function, for
// plain and dual numbers.
inline double sigmoid_(double x) { return 1.0 / (1.0 + std::exp(-x)); }
inline double softplus_(double x) { return x > 0.0 ? x + std::log1p(std::exp(-x)) : std::log1p(std::exp(x)); }
template <class T> Dual<T> sigmoid_(const Dual<T>& a) {
  const T s = sigmoid_(a.v);
  return {s, a.d * (s * (1.0 - s))};
}
template <class T> Dual<T> softplus_(const Dual<T>& a) { return {softplus_(a.v), a.d * sigmoid_(a.v)}; }

// The neural term NN(y) of the Robertson neural right-hand side.
template <class T, class TW>
T nr_mlp(const T* y, const TW* w) {
  const TW* W1 = w;
  const TW* b1 = W1 + UDE_H * 3;
  const TW* W2 = b1 + UDE_H;
  const TW* b2 = W2 + UDE_H * UDE_H;
  const TW* W3 = b2 + UDE_H;
  const TW* b3 = W3 + UDE_H;
  T h1[UDE_H], h2[UDE_H];
  for (int i = 0; i < UDE_H; ++i)
    h1[i] = tanh_(T(b1[i]) + T(W1[i * 3]) * y[0] + T(W1[i * 3 + 1]) * y[1] + T(W1[i * 3 + 2]) * y[2]);
  for (int i = 0; i < UDE_H; ++i) {
    T s = T(b2[i]);
    for (int j = 0; j < UDE_H; ++j) s = s + T(W2[i * UDE_H + j]) * h1[j];
    h2[i] = tanh_(s);
  }
  T z = T(b3[0]);
  for (int j = 0; j < UDE_H; ++j) z = z + T(W3[j]) * h2[j];
  return softplus_(z);
}

// Shared MLP of the LV UDE (2-16-16-2, tanh, linear output).
template <class T, class TW>
void ude_mlp(const T* x, const TW* w, T* out) {
  const TW* W1 = w;
  const TW* b1 = W1 + UDE_H * 2;
  const TW* W2 = b1 + UDE_H;
  const TW* b2 = W2 + UDE_H * UDE_H;
  const TW* W3 = b2 + UDE_H;
  const TW* b3 = W3 + 2 * UDE_H;
  T h1[UDE_H], h2[UDE_H];
  for (int i = 0; i < UDE_H; ++i) h1[i] = tanh_(T(b1[i]) + T(W1[i * 2 + 0]) * x[0] + T(W1[i * 2 + 1]) * x[1]);
  for (int i = 0; i < UDE_H; ++i) {
    T s = T(b2[i]);
    for (int j = 0; j < UDE_H; ++j) s = s + T(W2[i * UDE_H + j]) * h1[j];
    h2[i] = tanh_(s);
  }
  for (int i = 0; i < 2; ++i) {
    T s = T(b3[i]);
    for (int j = 0; j < UDE_H; ++j) s = s + T(W3[i * UDE_H + j]) * h2[j];
    out[i] = s;
  }
}

// f(y, theta): the right-hand sides of the paper's Appendix A (and the LV UDE).
// HIRES: its 12 distinct literal constants, in order of first appearance, are the
// 12 parameters (1.71, 0.43, 8.32, 0.0007, 8.75, 10.03, 0.035, 1.12, 1.745, 280,
// 0.69, 1.81); each literal is one shared parameter wherever it appears.
// LINEAR: dy/dt = A y with A = [[p0, p1], [p2, p3]] (closed-form test problem).
template <class T, class TW>
void rhs(int pid, const T* y, const T* p, const TW* w, T* f) {
  switch (pid) {
    case P_LORENZ:
      f[0] = p[0] * (y[1] - y[0]);
      f[1] = y[0] * (p[1] - y[2]) - y[1];
      f[2] = y[0] * y[1] - p[2] * y[2];
      break;
    case P_VDP:
      f[0] = y[1];
      f[1] = p[0] * ((1.0 - y[0] * y[0]) * y[1] - y[0]);
      break;
    case P_ROBERTSON:
      f[0] = -p[0] * y[0] + p[2] * y[1] * y[2];
      f[1] = p[0] * y[0] - p[2] * y[1] * y[2] - p[1] * y[1] * y[1];
      f[2] = p[1] * y[1] * y[1];
      break;
    case P_HIRES:
      f[0] = -p[0] * y[0] + p[1] * y[1] + p[2] * y[2] + p[3];
      f[1] = p[0] * y[0] - p[4] * y[1];
      f[2] = -p[5] * y[2] + p[1] * y[3] + p[6] * y[4];
      f[3] = p[2] * y[1] + p[0] * y[2] - p[7] * y[3];
      f[4] = -p[8] * y[4] + p[1] * y[5] + p[1] * y[6];
      f[5] = -p[9] * y[5] * y[7] + p[10] * y[3] + p[0] * y[4] - p[1] * y[5] + p[10] * y[6];
      f[6] = p[9] * y[5] * y[7] - p[11] * y[6];
      f[7] = -p[9] * y[5] * y[7] + p[11] * y[6];
      break;
    case P_LINEAR:
      f[0] = p[0] * y[0] + p[1] * y[1];
      f[1] = p[2] * y[0] + p[3] * y[1];
      break;
    case P_LV_UDE: {
      T nn[2];
      ude_mlp(y, w, nn);
      f[0] = p[0] * y[0] - nn[0];
      f[1] = -p[1] * y[1] + nn[1];
      break;
    }
    case P_NROB: {  // Robertson with k2 y2^2 replaced by NN(y) in its sink and source; p = (k1, k3)
      const T nn = nr_mlp(y, w);
      f[0] = -p[0] * y[0] + p[1] * y[1] * y[2];
      f[1] = p[0] * y[0] - p[1] * y[1] * y[2] - nn;
      f[2] = nn;
      break;
    }
  }
}

// The problem as the solvers see it: dimensions plus the per-trajectory data.
struct Prob {
  int pid, d, P;
  const double* w;  // shared UDE weights (nullptr otherwise)
};

template <class T>
void f_eval(const Prob& pr, const T* y, const T* p, T* f) { rhs<T, double>(pr.pid, y, p, pr.w, f); }

// J[c][a] = d f_c / d y_a by forward-mode dual numbers.
template <class T>
void jac_y(const Prob& pr, const T* y, const T* p, T J[DMAX][DMAX]) {
  using D = Dual<T>;
  D yd[DMAX], pd[PMAX], fd[DMAX];
  for (int q = 0; q < pr.P; ++q) pd[q] = D(p[q], T(0.0));
  for (int a = 0; a < pr.d; ++a) {
    for (int b = 0; b < pr.d; ++b) yd[b] = D(y[b], T(a == b ? 1.0 : 0.0));
    f_eval(pr, yd, pd, fd);
    for (int c = 0; c < pr.d; ++c) J[c][a] = fd[c].d;
  }
}
// Fp[c][q] = d f_c / d theta_q.
template <class T>
void jac_p(const Prob& pr, const T* y, const T* p, T Fp[DMAX][PMAX]) {
  using D = Dual<T>;
  D yd[DMAX], pd[PMAX], fd[DMAX];
  for (int b = 0; b < pr.d; ++b) yd[b] = D(y[b], T(0.0));
  for (int q = 0; q < pr.P; ++q) {
    for (int r = 0; r < pr.P; ++r) pd[r] = D(p[r], T(q == r ? 1.0 : 0.0));
    f_eval(pr, yd, pd, fd);
    for (int c = 0; c < pr.d; ++c) Fp[c][q] = fd[c].d;
  }
}
// Second-derivative contractions g(y, theta) = r^T J(y, theta) u:
//   gy[b] = d g / d y_b,  gp[q] = d g / d theta_q   (nested dual numbers).
void jac_contract_grad(const Prob& pr, const double* y, const double* p, const double* r, const double* u,
                       double* gy, double* gp) {
  using D1 = Dual<double>;
  using D2 = Dual<D1>;
  D2 yd[DMAX], pd[PMAX], fd[DMAX];
  // Inner tangent (epsilon) along u in y; outer tangent (eta) along a unit vector.
  for (int b = 0; b < pr.d + pr.P; ++b) {
    for (int a = 0; a < pr.d; ++a)
      yd[a] = D2(D1(y[a], u[a]), D1(b == a ? 1.0 : 0.0, 0.0));
    for (int q = 0; q < pr.P; ++q)
      pd[q] = D2(D1(p[q], 0.0), D1(b == pr.d + q ? 1.0 : 0.0, 0.0));
    rhs<D2, double>(pr.pid, yd, pd, pr.w, fd);
    double g = 0.0;
    for (int c = 0; c < pr.d; ++c) g += r[c] * fd[c].d.d;  // d/deta d/deps (r . f)
    if (b < pr.d) gy[b] = g; else gp[b - pr.d] = g;
  }
}

// Shared-weight VJP of the UDE: wbar[k] += sum_c v_c d f_c / d w_k at (y, p).
// Reverse mode written out by hand for the tiny MLP (f_0 = a x - nn_0,
// f_1 = -d y + nn_1, so the output cotangent is (-v_0, v_1)).
void ude_w_vjp(const double* y, const double* w, const double* v, double* wbar) {
  const double* W1 = w;
  const double* b1 = W1 + UDE_H * 2;
  const double* W2 = b1 + UDE_H;
  const double* b2 = W2 + UDE_H * UDE_H;
  const double* W3 = b2 + UDE_H;
  double* gW1 = wbar;
  double* gb1 = gW1 + UDE_H * 2;
  double* gW2 = gb1 + UDE_H;
  double* gb2 = gW2 + UDE_H * UDE_H;
  double* gW3 = gb2 + UDE_H;
  double* gb3 = gW3 + 2 * UDE_H;
  double h1[UDE_H], h2[UDE_H];
  for (int i = 0; i < UDE_H; ++i) h1[i] = std::tanh(b1[i] + W1[i * 2] * y[0] + W1[i * 2 + 1] * y[1]);
  for (int i = 0; i < UDE_H; ++i) {
    double s = b2[i];
    for (int j = 0; j < UDE_H; ++j) s += W2[i * UDE_H + j] * h1[j];
    h2[i] = std::tanh(s);
  }
  double go[2] = {-v[0], v[1]};
  double gh2[UDE_H] = {0}, gh1[UDE_H] = {0};
  for (int i = 0; i < 2; ++i) {
    gb3[i] += go[i];
    for (int j = 0; j < UDE_H; ++j) { gW3[i * UDE_H + j] += go[i] * h2[j]; gh2[j] += go[i] * W3[i * UDE_H + j]; }
  }
  for (int i = 0; i < UDE_H; ++i) {
    double gs = gh2[i] * (1.0 - h2[i] * h2[i]);
    gb2[i] += gs;
    for (int j = 0; j < UDE_H; ++j) { gW2[i * UDE_H + j] += gs * h1[j]; gh1[j] += gs * W2[i * UDE_H + j]; }
  }
  for (int i = 0; i < UDE_H; ++i) {
    double gs = gh1[i] * (1.0 - h1[i] * h1[i]);
    gb1[i] += gs;
    gW1[i * 2 + 0] += gs * y[0];
    gW1[i * 2 + 1] += gs * y[1];
  }
}

// Shared-weight VJP of the neural Robertson term: wbar[k] += c dNN/dw_k at y,
// reverse mode written out by hand. Templated so that, run on dual numbers
// y = y0 + eps u, the eps-parts of wbar are c d/dw (grad_y NN . u): the
// weight derivative of the Jacobian contraction the stiff adjoint needs.
template <class T>
void nr_w_vjp(const T* y, const double* w, T c, T* wbar) {
  const double* W1 = w;
  const double* b1 = W1 + UDE_H * 3;
  const double* W2 = b1 + UDE_H;
  const double* b2 = W2 + UDE_H * UDE_H;
  const double* W3 = b2 + UDE_H;
  const double* b3 = W3 + UDE_H;
  T* gW1 = wbar;
  T* gb1 = gW1 + UDE_H * 3;
  T* gW2 = gb1 + UDE_H;
  T* gb2 = gW2 + UDE_H * UDE_H;
  T* gW3 = gb2 + UDE_H;
  T* gb3 = gW3 + UDE_H;
  T h1[UDE_H], h2[UDE_H];
  for (int i = 0; i < UDE_H; ++i)
    h1[i] = tanh_(T(b1[i]) + W1[i * 3] * y[0] + W1[i * 3 + 1] * y[1] + W1[i * 3 + 2] * y[2]);
  for (int i = 0; i < UDE_H; ++i) {
    T s = T(b2[i]);
    for (int j = 0; j < UDE_H; ++j) s = s + W2[i * UDE_H + j] * h1[j];
    h2[i] = tanh_(s);
  }
  T z = T(b3[0]);
  for (int j = 0; j < UDE_H; ++j) z = z + W3[j] * h2[j];
  const T gz = c * sigmoid_(z);
  gb3[0] += gz;
  T gh1[UDE_H];
  for (int j = 0; j < UDE_H; ++j) gh1[j] = T(0.0);
  for (int i = 0; i < UDE_H; ++i) {
    gW3[i] += gz * h2[i];
    const T gs = (gz * W3[i]) * (1.0 - h2[i] * h2[i]);
    gb2[i] += gs;
    for (int j = 0; j < UDE_H; ++j) {
      gW2[i * UDE_H + j] += gs * h1[j];
      gh1[j] += gs * W2[i * UDE_H + j];
    }
  }
  for (int i = 0; i < UDE_H; ++i) {
    const T gs = gh1[i] * (1.0 - h1[i] * h1[i]);
    gb1[i] += gs;
    for (int a = 0; a < 3; ++a) gW1[i * 3 + a] += gs * y[a];
  }
}

// Shared-weight VJP of f for the problems with shared weights.
void w_vjp(const Prob& pr, const double* y, const double* v, double* wbar) {
  if (pr.pid == P_LV_UDE) ude_w_vjp(y, pr.w, v, wbar);
  if (pr.pid == P_NROB) nr_w_vjp<double>(y, pr.w, v[2] - v[1], wbar);
}
// Shared-weight gradient of g = r^T J(y, w) u (stiff adjoint): only the neural
// term depends on w, through (r_3 - r_2) grad_y NN . u (1-based rows).
void w_contract(const Prob& pr, const double* y, const double* r, const double* u, double* wbar) {
  if (pr.pid != P_NROB) return;
  using D = Dual<double>;
  D yd[3], gd[NR_NW];
  for (int a = 0; a < 3; ++a) yd[a] = D(y[a], u[a]);
  for (int k = 0; k < NR_NW; ++k) gd[k] = D(0.0, 0.0);
  nr_w_vjp<D>(yd, pr.w, D(r[2] - r[1], 0.0), gd);
  for (int k = 0; k < NR_NW; ++k) wbar[k] += gd[k].d;
}

// ---------------------------------------------------------------- tableaus
// Tsit5: the 5(4) pair of Tsitouras (2011), Table 1. The first column follows
// from the row-sum condition c_i = sum_j a_ij, as in that construction.
struct Tsit5Tab {
  double c[7], A[7][7], b[7], bhat[7];
  Tsit5Tab() {
    std::memset(this, 0, sizeof(*this));
    c[1] = 0.161; c[2] = 0.327; c[3] = 0.9; c[4] = 0.9800255409045097; c[5] = 1.0; c[6] = 1.0;
    A[2][1] = 0.335480655492357;
    A[3][1] = -6.359448489975075; A[3][2] = 4.3622954328695815;
    A[4][1] = -11.748883564062828; A[4][2] = 7.4955393428898365; A[4][3] = -0.09249506636175525;
    A[5][1] = -12.92096931784711; A[5][2] = 8.159367898576159; A[5][3] = -0.071584973281401;
    A[5][4] = -0.028269050394068383;
    A[6][0] = 0.09646076681806523; A[6][1] = 0.01; A[6][2] = 0.4798896504144996;
    A[6][3] = 1.379008574103742; A[6][4] = -3.290069515436081; A[6][5] = 2.324710524099774;
    for (int i = 1; i < 6; ++i) {
      double s = 0.0;
      for (int j = 1; j < i; ++j) s += A[i][j];
      A[i][0] = c[i] - s;
    }
    for (int j = 0; j < 7; ++j) b[j] = A[6][j];  // FSAL: the last stage is evaluated at y_new
    bhat[0] = 0.09468075576583945; bhat[1] = 0.009183565540343; bhat[2] = 0.4877705284247616;
    bhat[3] = 1.234297566930479; bhat[4] = -2.707712349983525; bhat[5] = 1.866628418170587;
    bhat[6] = 1.0 / 66.0;
  }
};
const Tsit5Tab& tsit5() { static Tsit5Tab t; return t; }

// Rodas5P (Steinebach 2023), in the transformed Rosenbrock form
//   (I/(h gamma) - J) U_i = f(y + sum_{j<i} a_ij U_j) + sum_{j<i} (C_ij / h) U_j,
//   y_new = y + sum_j m_j U_j,
// stiffly accurate: rows 7 and 8 of a extend row 6 by ones, m = (a_8*, 1), and
// the embedded solution is y_new - U_8.
struct RodasTab {
  double gamma, a[8][8], C[8][8], m[8];
  RodasTab() {
    std::memset(this, 0, sizeof(*this));
    gamma = 0.21193756319429014;
    a[1][0] = 3.0;
    a[2][0] = 2.849394379747939; a[2][1] = 0.45842242204463923;
    a[3][0] = -6.954028509809101; a[3][1] = 2.489845061869568; a[3][2] = -10.358996098473584;
    a[4][0] = 2.8029986275628964; a[4][1] = 0.5072464736228206; a[4][2] = -0.3988312541770524;
    a[4][3] = -0.04721187230404641;
    a[5][0] = -7.502846399306121; a[5][1] = 2.561846144803919; a[5][2] = -11.627539656261098;
    a[5][3] = -0.18268767659942256; a[5][4] = 0.030198172008377946;
    for (int j = 0; j < 5; ++j) { a[6][j] = a[5][j]; a[7][j] = a[5][j]; }
    a[6][5] = 1.0; a[7][5] = 1.0; a[7][6] = 1.0;
    C[1][0] = -14.155112264123755;
    C[2][0] = -17.97296035885952; C[2][1] = -2.859693295451294;
    C[3][0] = 147.12150275711716; C[3][1] = -1.41221402718213; C[3][2] = 71.68940251302358;
    C[4][0] = 165.43517024871676; C[4][1] = -0.4592823456491126; C[4][2] = 42.90938336958603;
    C[4][3] = -5.961986721573306;
    C[5][0] = 24.854864614690072; C[5][1] = -3.0009227002832186; C[5][2] = 47.4931110020768;
    C[5][3] = 5.5814197821558125; C[5][4] = -0.6610691825249471;
    C[6][0] = 30.91273214028599; C[6][1] = -3.1208243349937974; C[6][2] = 77.79954646070892;
    C[6][3] = 34.28646028294783; C[6][4] = -19.097331116725623; C[6][5] = -28.087943162872662;
    C[7][0] = 37.80277123390563; C[7][1] = -3.2571969029072276; C[7][2] = 112.26918849496327;
    C[7][3] = 66.9347231244047; C[7][4] = -40.06618937091002; C[7][5] = -54.66780262877968;
    C[7][6] = -9.48861652309627;
    for (int j = 0; j < 7; ++j) m[j] = a[7][j];
    m[7] = 1.0;
  }
};
const RodasTab& rodas() { static RodasTab t; return t; }

// Verner7: Verner's "efficient" seventh-order explicit pair with a
// sixth-order embedded formula (J. H. Verner, Numerically optimal Runge-Kutta
// pairs with interpolants, Numer. Algorithms 53 (2010) 383-396), the pair the
// paper cites for its higher-order engine (Sec. 5). 10 stages, not FSAL: the
// 7th-order solution uses stages 1..9 (c_9 = 1), stage 10 (c_10 = 1) enters
// only the 6th-order formula; a_i2 = 0 from stage 4 on and b_2 = b_3 = 0.
// Coefficients to 40 significant digits as published (the compiler rounds each
// to the nearest double). Zero-based indices below.
struct Vern7Tab {
  double c[10], A[10][10], b[10], bhat[10];
  Vern7Tab() {
    std::memset(this, 0, sizeof(*this));
    c[1] = 0.005;
    c[2] = 0.1088888888888888888888888888888888888889;
    c[3] = 0.1633333333333333333333333333333333333333;
    c[4] = 0.4555;
    c[5] = 0.6095094489978381317087004421486024949638;
    c[6] = 0.884;
    c[7] = 0.925;
    c[8] = 1.0;
    c[9] = 1.0;
    A[1][0] = 0.005;
    A[2][0] = -1.076790123456790123456790123456790123457;
    A[2][1] = 1.185679012345679012345679012345679012346;
    A[3][0] = 0.04083333333333333333333333333333333333333;
    A[3][2] = 0.1225;
    A[4][0] = 0.6389139236255726780508121615993336109954;
    A[4][2] = -2.455672638223656809662640566430653894211;
    A[4][3] = 2.272258714598084131611828404831320283215;
    A[5][0] = -2.661577375018757131119259297861818119279;
    A[5][2] = 10.80451388645613769565396655365532838482;
    A[5][3] = -8.353914657396199411968048547819291691541;
    A[5][4] = 0.8204875949566569791420417341743839209619;
    A[6][0] = 6.067741434696770992718360183877276714679;
    A[6][2] = -24.71127363591108579734203485290746001803;
    A[6][3] = 20.42751793078889394045773111748346612697;
    A[6][4] = -1.906157978816647150624096784352757010879;
    A[6][5] = 1.006172249242068014790040335899474187268;
    A[7][0] = 12.05467007625320299509109452892778311648;
    A[7][2] = -49.75478495046898932807257615331444758322;
    A[7][3] = 41.14288863860467663259698416710157354209;
    A[7][4] = -4.461760149974004185641911603484815375051;
    A[7][5] = 2.042334822239174959821717077708608543738;
    A[7][6] = -0.09834843665406107379530801693870224403537;
    A[8][0] = 10.13814652288180787641845141981689030769;
    A[8][2] = -42.64113603171750214622846006736635730625;
    A[8][3] = 35.76384003992257007135021178023160054034;
    A[8][4] = -4.348022840392907653340370296908245943710;
    A[8][5] = 2.009862268377035895441943593011827554771;
    A[8][6] = 0.3487490460338272405953822853053145879140;
    A[8][7] = -0.2714390051048312842371587140910297407572;
    A[9][0] = -45.03007203429867712435322405073769635151;
    A[9][2] = 187.3272437654588840752418206154201997384;
    A[9][3] = -154.0288236935018690596728621034510402582;
    A[9][4] = 18.56465306347536233859492332958439136765;
    A[9][5] = -7.141809679295078854925420496823551192821;
    A[9][6] = 1.308808578161378625114762706007696696508;
    b[0] = 0.04715561848627222170431765108838175679569;
    b[3] = 0.2575056429843415189596436101037687580986;
    b[4] = 0.2621665397741262047713863095764527711129;
    b[5] = 0.1521609265673855740323133199165117535523;
    b[6] = 0.4939969170032484246907175893227876844296;
    b[7] = -0.2943031171403250441557244744092703429139;
    b[8] = 0.08131747232495109999734599440136761892478;
    bhat[0] = 0.04460860660634117628731817597479197781432;
    bhat[3] = 0.2671640378571372680509102260943837899738;
    bhat[4] = 0.2201018300177293019979715776650753096323;
    bhat[5] = 0.2188431703143156830983120833512893824578;
    bhat[6] = 0.2289871705411202883378173889763552365362;
    bhat[9] = 0.02029518466335628222767054793810430358554;
  }
};
const Vern7Tab& vern7() { static Vern7Tab t; return t; }

enum { M_TSIT5 = 1, M_RODAS5P = 2, M_ROS23 = 3, M_VERN7 = 4 };
enum { TRAJ_OK = 0, TRAJ_MAXSTEPS = 1, TRAJ_DT_UNDERFLOW = 2, TRAJ_NONFINITE = 3, TRAJ_SINGULAR = 4 };

// ---------------------------------------------------------------- Tsit5 step
// One explicit step (paper Eqs. (stages) and (update)) from y with size h:
// stage inputs Ys[j], stages K[j], y_new, and the embedded difference
// e = y_new - yhat_new = h sum_j (b_j - bhat_j) k_j.
template <class T>
void tsit5_step(const Prob& pr, const T* y, const T* p, double h, T Ys[7][DMAX], T K[7][DMAX], T* ynew, T* err) {
  const Tsit5Tab& tb = tsit5();
  const int d = pr.d;
  for (int i = 0; i < 7; ++i) {
    for (int c = 0; c < d; ++c) {
      T s = T(0.0);
      for (int j = 0; j < i; ++j) s = s + tb.A[i][j] * K[j][c];
      Ys[i][c] = y[c] + h * s;
    }
    f_eval(pr, Ys[i], p, K[i]);
  }
  for (int c = 0; c < d; ++c) {
    T s = T(0.0), e = T(0.0);
    for (int j = 0; j < 7; ++j) {
      s = s + tb.b[j] * K[j][c];
      e = e + (tb.b[j] - tb.bhat[j]) * K[j][c];
    }
    ynew[c] = y[c] + h * s;
    if (err) err[c] = h * e;
  }
}

// Reverse of one Tsit5 step (textbook reverse mode of the stage recursion):
// given lam = dL/dy_new, returns ybar = dL/dy and adds dL/dtheta to pbar.
// kbar_j = h (b_j lam + sum_{m>j} a_mj Ybar_m),  Ybar_j = J(Y_j)^T kbar_j,
// pbar += f_theta(Y_j)^T kbar_j,  ybar = lam + sum_j Ybar_j.
void tsit5_step_vjp(const Prob& pr, const double* y, const double* p, double h, const double* lam,
                    double* ybar, double* pbar, double* wbar) {
  const Tsit5Tab& tb = tsit5();
  const int d = pr.d, P = pr.P;
  double Ys[7][DMAX], K[7][DMAX], yn[DMAX];
  tsit5_step(pr, y, p, h, Ys, K, yn, (double*)nullptr);
  double Ybar[7][DMAX] = {{0}};
  for (int j = 6; j >= 0; --j) {
    double kbar[DMAX];
    for (int c = 0; c < d; ++c) {
      double s = tb.b[j] * lam[c];
      for (int m = j + 1; m < 7; ++m) s += tb.A[m][j] * Ybar[m][c];
      kbar[c] = h * s;
    }
    double J[DMAX][DMAX], Fp[DMAX][PMAX];
    jac_y(pr, Ys[j], p, J);
    jac_p(pr, Ys[j], p, Fp);
    for (int a = 0; a < d; ++a) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s += J[c][a] * kbar[c];
      Ybar[j][a] = s;
    }
    for (int q = 0; q < P; ++q) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s += Fp[c][q] * kbar[c];
      pbar[q] += s;
    }
    if (wbar) w_vjp(pr, Ys[j], kbar, wbar);
  }
  for (int c = 0; c < d; ++c) {
    double s = lam[c];
    for (int j = 0; j < 7; ++j) s += Ybar[j][c];
    ybar[c] = s;
  }
}

// ---------------------------------------------------------------- Verner7 step
// One explicit step of the 7(6) pair: stage inputs Ys[j] and stages K[j]
// (j = 0..9), y_new = y + h sum_j b_j k_j over stages 1..9 and the embedded
// difference e = h sum_j (b_j - bhat_j) k_j, which needs stage 10.
template <class T>
void vern7_step(const Prob& pr, const T* y, const T* p, double h, T Ys[10][DMAX], T K[10][DMAX], T* ynew, T* err) {
  const Vern7Tab& tb = vern7();
  const int d = pr.d;
  const int ns = err ? 10 : 9;
  for (int i = 0; i < ns; ++i) {
    for (int c = 0; c < d; ++c) {
      T s = T(0.0);
      for (int j = 0; j < i; ++j) s = s + tb.A[i][j] * K[j][c];
      Ys[i][c] = y[c] + h * s;
    }
    f_eval(pr, Ys[i], p, K[i]);
  }
  for (int c = 0; c < d; ++c) {
    T s = T(0.0), e = T(0.0);
    for (int j = 0; j < 9; ++j) s = s + tb.b[j] * K[j][c];
    ynew[c] = y[c] + h * s;
    if (err) {
      for (int j = 0; j < 10; ++j) e = e + (tb.b[j] - tb.bhat[j]) * K[j][c];
      err[c] = h * e;
    }
  }
}

// Reverse of one Verner7 step, as for Tsit5 over the nine stages that y_new
// depends on: kbar_j = h (b_j lam + sum_{m>j} a_mj Ybar_m), Ybar_j = J(Y_j)^T kbar_j,
// pbar += f_theta(Y_j)^T kbar_j, ybar = lam + sum_j Ybar_j.
void vern7_step_vjp(const Prob& pr, const double* y, const double* p, double h, const double* lam,
                    double* ybar, double* pbar, double* wbar) {
  const Vern7Tab& tb = vern7();
  const int d = pr.d, P = pr.P;
  double Ys[10][DMAX], K[10][DMAX], yn[DMAX];
  vern7_step(pr, y, p, h, Ys, K, yn, (double*)nullptr);
  double Ybar[9][DMAX] = {{0}};
  for (int j = 8; j >= 0; --j) {
    double kbar[DMAX];
    for (int c = 0; c < d; ++c) {
      double s = tb.b[j] * lam[c];
      for (int m = j + 1; m < 9; ++m) s += tb.A[m][j] * Ybar[m][c];
      kbar[c] = h * s;
    }
    double J[DMAX][DMAX], Fp[DMAX][PMAX];
    jac_y(pr, Ys[j], p, J);
    jac_p(pr, Ys[j], p, Fp);
    for (int a = 0; a < d; ++a) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s += J[c][a] * kbar[c];
      Ybar[j][a] = s;
    }
    for (int q = 0; q < P; ++q) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s += Fp[c][q] * kbar[c];
      pbar[q] += s;
    }
    if (wbar) w_vjp(pr, Ys[j], kbar, wbar);
  }
  for (int c = 0; c < d; ++c) {
    double s = lam[c];
    for (int j = 0; j < 9; ++j) s += Ybar[j][c];
    ybar[c] = s;
  }
}

// ---------------------------------------------------------------- dense LU
// Doolittle LU with partial pivoting; ties pick the lowest row index.
// Returns false on an exactly zero pivot.
template <class T>
bool lu_factor(int n, T A[DMAX][DMAX], int* perm) {
  for (int i = 0; i < n; ++i) perm[i] = i;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = std::fabs(val(A[k][k]));
    for (int i = k + 1; i < n; ++i) {
      double v = std::fabs(val(A[i][k]));
      if (v > best) { best = v; piv = i; }
    }
    if (best == 0.0) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k][j], A[piv][j]);
      std::swap(perm[k], perm[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      A[i][k] = A[i][k] / A[k][k];
      for (int j = k + 1; j < n; ++j) A[i][j] = A[i][j] - A[i][k] * A[k][j];
    }
  }
  return true;
}
// Solve (P^T L U) x = b, i.e. L U x = P b.
template <class T>
void lu_solve(int n, T LU[DMAX][DMAX], const int* perm, const T* b, T* x) {
  T z[DMAX];
  for (int i = 0; i < n; ++i) {
    T s = b[perm[i]];
    for (int j = 0; j < i; ++j) s = s - LU[i][j] * z[j];
    z[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    T s = z[i];
    for (int j = i + 1; j < n; ++j) s = s - LU[i][j] * x[j];
    x[i] = s / LU[i][i];
  }
}
// Solve W^T x = b with W = P^T L U:  U^T w = b, L^T v = w, x = P^T v.
void lu_solve_t(int n, double LU[DMAX][DMAX], const int* perm, const double* b, double* x) {
  double w[DMAX], v[DMAX];
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int j = 0; j < i; ++j) s -= LU[j][i] * w[j];
    w[i] = s / LU[i][i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = w[i];
    for (int j = i + 1; j < n; ++j) s -= LU[j][i] * v[j];
    v[i] = s;
  }
  for (int i = 0; i < n; ++i) x[perm[i]] = v[i];
}

// ---------------------------------------------------------------- Rodas5P step
// One Rosenbrock step (paper Sec. 3.2: each stage solves with I - gamma h J,
// here in the transformed form W = I/(h gamma) - J with J = J(y)). Outputs the
// stage inputs Ys, stage solutions U, y_new, and the error estimate e = U_8.
// Returns false if W is singular.
template <class T>
bool rodas_step(const Prob& pr, const T* y, const T* p, double h, T Ys[8][DMAX], T U[8][DMAX], T* ynew, T* err,
                T LU[DMAX][DMAX], int* perm) {
  const RodasTab& tb = rodas();
  const int d = pr.d;
  T J[DMAX][DMAX];
  jac_y(pr, y, p, J);
  const double inv_hg = 1.0 / (h * tb.gamma);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) LU[i][j] = (i == j ? T(inv_hg) : T(0.0)) - J[i][j];
  if (!lu_factor(d, LU, perm)) return false;
  for (int i = 0; i < 8; ++i) {
    T F[DMAX], R[DMAX];
    for (int c = 0; c < d; ++c) {
      T s = T(0.0);
      for (int j = 0; j < i; ++j) s = s + tb.a[i][j] * U[j][c];
      Ys[i][c] = y[c] + s;
    }
    f_eval(pr, Ys[i], p, F);
    for (int c = 0; c < d; ++c) {
      T s = T(0.0);
      for (int j = 0; j < i; ++j) s = s + (tb.C[i][j] / h) * U[j][c];
      R[c] = F[c] + s;
    }
    lu_solve(d, LU, perm, R, U[i]);
  }
  for (int c = 0; c < d; ++c) {
    T s = T(0.0);
    for (int j = 0; j < 8; ++j) s = s + tb.m[j] * U[j][c];
    ynew[c] = y[c] + s;
    if (err) err[c] = U[7][c];
  }
  return true;
}

// Reverse of one Rodas5P step with h as data (linear-solve adjoint, paper
// Sec. 3.2): Rbar_i = W^{-T} Ubar_i; Ubar_j += (C_ij/h) Rbar_i; Ybar_i =
// J(Y_i)^T Rbar_i; Ubar_j += a_ij Ybar_i; and the Jacobian cotangent
// Jbar = sum_i Rbar_i U_i^T contracted through J(y, theta).
bool rodas_step_vjp(const Prob& pr, const double* y, const double* p, double h, const double* lam,
                    double* ybar, double* pbar, double* wbar) {
  const RodasTab& tb = rodas();
  const int d = pr.d, P = pr.P;
  double Ys[8][DMAX], U[8][DMAX], yn[DMAX], LU[DMAX][DMAX];
  int perm[DMAX];
  if (!rodas_step(pr, y, p, h, Ys, U, yn, (double*)nullptr, LU, perm)) return false;
  double Ubar[8][DMAX], Rbar[8][DMAX];
  for (int j = 0; j < 8; ++j)
    for (int c = 0; c < d; ++c) Ubar[j][c] = tb.m[j] * lam[c];
  for (int c = 0; c < d; ++c) ybar[c] = lam[c];
  for (int i = 7; i >= 0; --i) {
    lu_solve_t(d, LU, perm, Ubar[i], Rbar[i]);
    for (int j = 0; j < i; ++j)
      for (int c = 0; c < d; ++c) Ubar[j][c] += (tb.C[i][j] / h) * Rbar[i][c];
    double J[DMAX][DMAX], Fp[DMAX][PMAX], Yb[DMAX];
    jac_y(pr, Ys[i], p, J);
    jac_p(pr, Ys[i], p, Fp);
    for (int a = 0; a < d; ++a) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s += J[c][a] * Rbar[i][c];
      Yb[a] = s;
    }
    for (int q = 0; q < P; ++q) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s += Fp[c][q] * Rbar[i][c];
      pbar[q] += s;
    }
    if (wbar) w_vjp(pr, Ys[i], Rbar[i], wbar);
    for (int c = 0; c < d; ++c) ybar[c] += Yb[c];
    for (int j = 0; j < i; ++j)
      for (int c = 0; c < d; ++c) Ubar[j][c] += tb.a[i][j] * Yb[c];
  }
  // W = I/(h gamma) - J(y): dL/dJ = -dL/dW = sum_i Rbar_i U_i^T.
  for (int i = 0; i < 8; ++i) {
    double gy[DMAX], gp[PMAX];
    jac_contract_grad(pr, y, p, Rbar[i], U[i], gy, gp);
    if (wbar) w_contract(pr, y, Rbar[i], U[i], wbar);
    for (int c = 0; c < d; ++c) ybar[c] += gy[c];
    for (int q = 0; q < P; ++q) pbar[q] += gp[q];
  }
  return true;
}

// ---------------------------------------------------------------- Rosenbrock23
// The second-order linearly implicit method of Shampine & Reichelt (1997), the
// formulas of MATLAB's ode23s, for autonomous f (paper Sec. 3.2, its stiff
// default for the fused kernels), with W = I - h d J(y):
//   F0 = f(y),                  k1 = W^{-1} F0,
//   F1 = f(y + h/2 k1),         k2 = W^{-1} (F1 - k1) + k1,
//   y_new = y + h k2,
//   F2 = f(y_new),              k3 = W^{-1} (F2 - e32 (k2 - F1) - 2 (k1 - F0)),
//   e = h/6 (k1 - 2 k2 + k3),
// with d = 1/(2 + sqrt 2) and e32 = 6 + sqrt 2. Outputs k1, u2 = W^{-1}(F1 - k1)
// (so k2 = u2 + k1), the stage input Y1 = y + h/2 k1 and the LU of W.
const double ROS23_D = 1.0 / (2.0 + std::sqrt(2.0));
const double ROS23_E32 = 6.0 + std::sqrt(2.0);

template <class T>
bool ros23_step(const Prob& pr, const T* y, const T* p, double h, T* ynew, T* err, T* k1, T* u2, T* Y1,
                T LU[DMAX][DMAX], int* perm) {
  const int d = pr.d;
  T J[DMAX][DMAX];
  jac_y(pr, y, p, J);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) LU[i][j] = (i == j ? T(1.0) : T(0.0)) - (h * ROS23_D) * J[i][j];
  if (!lu_factor(d, LU, perm)) return false;
  T F0[DMAX], F1[DMAX], r[DMAX], k2[DMAX];
  f_eval(pr, y, p, F0);
  lu_solve(d, LU, perm, F0, k1);
  for (int c = 0; c < d; ++c) Y1[c] = y[c] + (0.5 * h) * k1[c];
  f_eval(pr, Y1, p, F1);
  for (int c = 0; c < d; ++c) r[c] = F1[c] - k1[c];
  lu_solve(d, LU, perm, r, u2);
  for (int c = 0; c < d; ++c) {
    k2[c] = u2[c] + k1[c];
    ynew[c] = y[c] + h * k2[c];
  }
  if (err) {
    T F2[DMAX], k3[DMAX];
    f_eval(pr, ynew, p, F2);
    for (int c = 0; c < d; ++c) r[c] = F2[c] - ROS23_E32 * (k2[c] - F1[c]) - 2.0 * (k1[c] - F0[c]);
    lu_solve(d, LU, perm, r, k3);
    for (int c = 0; c < d; ++c) err[c] = (h / 6.0) * (k1[c] - 2.0 * k2[c] + k3[c]);
  }
  return true;
}

// Reverse of one Rosenbrock23 step with h as data: with lam = dL/dy_new,
//   k2bar = h lam;  r2bar = W^{-T} k2bar (u2 = W^{-1} r2, r2 = F1 - k1);
//   F1bar = r2bar;  k1bar = k2bar - r2bar;
//   Y1bar = J(Y1)^T F1bar, theta_bar += f_theta(Y1)^T F1bar;
//   k1bar += h/2 Y1bar;  r1bar = W^{-T} k1bar (k1 = W^{-1} F0);
//   ybar = lam + Y1bar + J(y)^T r1bar, theta_bar += f_theta(y)^T r1bar;
// and W = I - h d J(y) gives dL/dJ = h d (r1bar k1^T + r2bar u2^T), contracted
// through J(y, theta).
bool ros23_step_vjp(const Prob& pr, const double* y, const double* p, double h, const double* lam, double* ybar,
                    double* pbar, double* wbar) {
  const int d = pr.d, P = pr.P;
  double yn[DMAX], k1[DMAX], u2[DMAX], Y1[DMAX], LU[DMAX][DMAX];
  int perm[DMAX];
  if (!ros23_step(pr, y, p, h, yn, (double*)nullptr, k1, u2, Y1, LU, perm)) return false;
  double k2b[DMAX], r2b[DMAX], k1b[DMAX], r1b[DMAX];
  for (int c = 0; c < d; ++c) k2b[c] = h * lam[c];
  lu_solve_t(d, LU, perm, k2b, r2b);
  auto vjp_at = [&](const double* x, const double* v, double* xb) {  // xb = J(x)^T v; pbar += f_theta(x)^T v
    double J[DMAX][DMAX], Fp[DMAX][PMAX];
    jac_y(pr, x, p, J);
    jac_p(pr, x, p, Fp);
    for (int a = 0; a < d; ++a) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s += J[c][a] * v[c];
      xb[a] = s;
    }
    for (int q = 0; q < P; ++q) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s += Fp[c][q] * v[c];
      pbar[q] += s;
    }
    if (wbar) w_vjp(pr, x, v, wbar);
  };
  double Y1b[DMAX], y0b[DMAX];
  vjp_at(Y1, r2b, Y1b);
  for (int c = 0; c < d; ++c) k1b[c] = k2b[c] - r2b[c] + (0.5 * h) * Y1b[c];
  lu_solve_t(d, LU, perm, k1b, r1b);
  vjp_at(y, r1b, y0b);
  for (int c = 0; c < d; ++c) ybar[c] = lam[c] + Y1b[c] + y0b[c];
  double r1s[DMAX], r2s[DMAX];
  for (int c = 0; c < d; ++c) {
    r1s[c] = (h * ROS23_D) * r1b[c];
    r2s[c] = (h * ROS23_D) * r2b[c];
  }
  double gy[DMAX], gp[PMAX];
  jac_contract_grad(pr, y, p, r1s, k1, gy, gp);
  if (wbar) w_contract(pr, y, r1s, k1, wbar);
  for (int c = 0; c < d; ++c) ybar[c] += gy[c];
  for (int q = 0; q < P; ++q) pbar[q] += gp[q];
  jac_contract_grad(pr, y, p, r2s, u2, gy, gp);
  if (wbar) w_contract(pr, y, r2s, u2, wbar);
  for (int c = 0; c < d; ++c) ybar[c] += gy[c];
  for (int q = 0; q < P; ++q) pbar[q] += gp[q];
  return true;
}

// Generic one-step map Phi(y; h) for the chosen method.
template <class T>
bool phi_step(int method, const Prob& pr, const T* y, const T* p, double h, T* ynew) {
  if (method == M_TSIT5) {
    T Ys[7][DMAX], K[7][DMAX];
    tsit5_step(pr, y, p, h, Ys, K, ynew, (T*)nullptr);
    return true;
  }
  if (method == M_ROS23) {
    T k1[DMAX], u2[DMAX], Y1[DMAX], LU[DMAX][DMAX];
    int perm[DMAX];
    return ros23_step(pr, y, p, h, ynew, (T*)nullptr, k1, u2, Y1, LU, perm);
  }
  if (method == M_VERN7) {
    T Ys[10][DMAX], K[10][DMAX];
    vern7_step(pr, y, p, h, Ys, K, ynew, (T*)nullptr);
    return true;
  }
  T Ys[8][DMAX], U[8][DMAX], LU[DMAX][DMAX];
  int perm[DMAX];
  return rodas_step(pr, y, p, h, Ys, U, ynew, (T*)nullptr, LU, perm);
}
bool phi_step_vjp(int method, const Prob& pr, const double* y, const double* p, double h, const double* lam,
                  double* ybar, double* pbar, double* wbar) {
  if (method == M_TSIT5) { tsit5_step_vjp(pr, y, p, h, lam, ybar, pbar, wbar); return true; }
  if (method == M_ROS23) return ros23_step_vjp(pr, y, p, h, lam, ybar, pbar, wbar);
  if (method == M_VERN7) { vern7_step_vjp(pr, y, p, h, lam, ybar, pbar, wbar); return true; }
  return rodas_step_vjp(pr, y, p, h, lam, ybar, pbar, wbar);
}
// Order of the method's solution (the starting step) and the lower order q of its
// error estimate (the controller exponent 1/(q+1)): Tsit5 and Rodas5P 5 and 4,
// Rosenbrock23 2 and 2, Verner7 7 and 6.
int method_order(int method) { return method == M_ROS23 ? 2 : (method == M_VERN7 ? 7 : 5); }
int method_err_order(int method) { return method == M_ROS23 ? 2 : (method == M_VERN7 ? 6 : 4); }

// ---------------------------------------------------------------- record
// Weighted RMS norm of the paper's Sec. 2.1: sqrt(mean_c (e_c / (atol + rtol max(|y_c|, |ynew_c|)))^2).
double err_norm(int d, const double* e, const double* y, const double* yn, double rtol, double atol) {
  double s = 0.0;
  for (int c = 0; c < d; ++c) {
    double sc = atol + rtol * std::max(std::fabs(y[c]), std::fabs(yn[c]));
    double r = e[c] / sc;
    s += r * r;
  }
  return std::sqrt(s / d);
}
double rms_scaled(int d, const double* v, const double* sc) {
  double s = 0.0;
  for (int c = 0; c < d; ++c) { double r = v[c] / sc[c]; s += r * r; }
  return std::sqrt(s / d);
}

// Starting step: the algorithm of Hairer, Norsett & Wanner, Vol. I, Sec. II.4,
// with the method's order p, the same weighted RMS norm, and one explicit Euler probe.
double initial_step(const Prob& pr, const double* y0, const double* p, double t0, double t1, double rtol,
                    double atol, int order = 5) {
  const int d = pr.d;
  double f0[DMAX], sc[DMAX], y1[DMAX], f1[DMAX], df[DMAX];
  f_eval(pr, y0, p, f0);
  for (int c = 0; c < d; ++c) sc[c] = atol + rtol * std::fabs(y0[c]);
  double d0 = rms_scaled(d, y0, sc), d1 = rms_scaled(d, f0, sc);
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  h0 = std::min(h0, t1 - t0);
  for (int c = 0; c < d; ++c) y1[c] = y0[c] + h0 * f0[c];
  f_eval(pr, y1, p, f1);
  for (int c = 0; c < d; ++c) df[c] = f1[c] - f0[c];
  double d2 = rms_scaled(d, df, sc) / h0;
  double dm = std::max(d1, d2);
  double h1 = (dm <= 1e-15) ? std::max(1e-6, h0 * 1e-3) : std::pow(0.01 / dm, 1.0 / (order + 1));
  return std::min(std::min(100.0 * h0, h1), t1 - t0);
}

// Step-size factor of the integral controller: clamp(0.9 err^(-1/(q+1)), 0.2, 10)
// with q the lower order of the error estimate (4 for Tsit5 and Rodas5P, so
// err^(-1/5); 2 for Rosenbrock23, err^(-1/3)); err = 0 gives 10.
double ctrl_factor(double err, int q = 4) {
  if (!(err > 0.0)) return 10.0;
  double f = 0.9 * std::pow(err, -1.0 / (q + 1));
  return std::min(10.0, std::max(0.2, f));
}

struct RecordOut {
  std::vector<double> h;
  int64_t n_att = 0;
  int status = TRAJ_OK;
};

// The record map R (paper Sec. 3.1): an ordinary adaptive solve that keeps the
// accepted step sizes. Save-time states are one extra step from the preceding
// mesh point (paper Sec. 3.4); they do not alter the mesh.
RecordOut record_one(int method, const Prob& pr, const double* y0, const double* p, double t0, double t1,
                     const double* save_t, int ns, double rtol, double atol, int64_t max_steps, double h_init,
                     double* y_save /*[ns][d] or null*/) {
  const int d = pr.d;
  RecordOut out;
  double y[DMAX], yn[DMAX], e[DMAX];
  for (int c = 0; c < d; ++c) y[c] = y0[c];
  double t = t0;
  double h = h_init > 0.0 ? h_init : initial_step(pr, y0, p, t0, t1, rtol, atol, method_order(method));
  const double sliver = 1e-12 * std::max(1.0, std::fabs(t1));
  bool reject_prev = false, last_nonfinite = false;
  int js = 0;
  for (int c = 0; c < d; ++c)
    if (!std::isfinite(y0[c])) { out.status = TRAJ_NONFINITE; return out; }
  for (int q = 0; q < pr.P; ++q)
    if (!std::isfinite(p[q])) { out.status = TRAJ_NONFINITE; return out; }
  if (!std::isfinite(h)) { out.status = TRAJ_NONFINITE; return out; }
  for (;;) {
    if (out.n_att >= max_steps) { out.status = TRAJ_MAXSTEPS; return out; }
    bool last = false;
    if (t + h >= t1 - sliver) { h = t1 - t; last = true; }
    ++out.n_att;
    bool ok;
    if (method == M_TSIT5) {
      double Ys[7][DMAX], K[7][DMAX];
      tsit5_step(pr, y, p, h, Ys, K, yn, e);
      ok = true;
    } else if (method == M_ROS23) {
      double k1[DMAX], u2[DMAX], Y1[DMAX], LU[DMAX][DMAX];
      int perm[DMAX];
      ok = ros23_step(pr, y, p, h, yn, e, k1, u2, Y1, LU, perm);
    } else if (method == M_VERN7) {
      double Ys[10][DMAX], K[10][DMAX];
      vern7_step(pr, y, p, h, Ys, K, yn, e);
      ok = true;
    } else {
      double Ys[8][DMAX], U[8][DMAX], LU[DMAX][DMAX];
      int perm[DMAX];
      ok = rodas_step(pr, y, p, h, Ys, U, yn, e, LU, perm);
    }
    if (!ok) {  // singular W: a failed trial with a quartered step
      h = h * 0.25;
      reject_prev = true;
      if (std::fabs(h) < 1e-14 * std::max(1.0, std::fabs(t))) { out.status = TRAJ_SINGULAR; return out; }
      continue;
    }
    double err = err_norm(d, e, y, yn, rtol, atol);
    if (std::isfinite(err) && err <= 1.0) {
      double t_new = last ? t1 : t + h;
      // Save times in [t, t_new): one extra step from y; exactly t_new: y_new.
      while (js < ns && save_t[js] < t_new) {
        if (y_save) {
          double hs = save_t[js] - t;
          if (hs == 0.0) {
            for (int c = 0; c < d; ++c) y_save[js * d + c] = y[c];
          } else {
            phi_step(method, pr, y, p, hs, y_save + js * d);
          }
        }
        ++js;
      }
      while (js < ns && save_t[js] == t_new) {
        if (y_save) for (int c = 0; c < d; ++c) y_save[js * d + c] = yn[c];
        ++js;
      }
      out.h.push_back(h);
      t = t_new;
      for (int c = 0; c < d; ++c) y[c] = yn[c];
      if (last) return out;
      double fac = ctrl_factor(err, method_err_order(method));
      if (reject_prev) fac = std::min(fac, 1.0);
      reject_prev = false;
      last_nonfinite = false;
      h = h * fac;
    } else {
      last_nonfinite = !std::isfinite(err);
      double fac = last_nonfinite ? 0.2 : ctrl_factor(err, method_err_order(method));
      h = h * fac;
      reject_prev = true;
    }
    if (std::fabs(h) < 1e-14 * std::max(1.0, std::fabs(t))) {
      out.status = last_nonfinite ? TRAJ_NONFINITE : TRAJ_DT_UNDERFLOW;
      return out;
    }
  }
}

// ---------------------------------------------------------------- replay
// Mesh times t_i = t_{i-1} + h_i (i < S), t_S = t1 exactly (the record's rule).
void mesh_times(double t0, double t1, const double* h, int64_t S, std::vector<double>& ts) {
  ts.assign(S + 1, 0.0);
  ts[0] = t0;
  for (int64_t i = 1; i <= S; ++i) ts[i] = (i == S) ? t1 : ts[i - 1] + h[i - 1];
}
// i(s) = max{ i : t_i <= t_s } for each save time.
void save_index(const std::vector<double>& ts, const double* save_t, int ns, std::vector<int64_t>& is) {
  is.assign(ns, 0);
  const int64_t S = (int64_t)ts.size() - 1;
  for (int s = 0; s < ns; ++s) {
    int64_t i = 0;
    while (i < S && ts[i + 1] <= save_t[s]) ++i;
    is[s] = i;
  }
}

// Forward replay (Eq. (replay)) on a given mesh, templated for dual-number JVPs.
// Returns the save-time states and the built-in loss sum_s ||y(t_s)||^2.
template <class T>
bool replay_forward(int method, const Prob& pr, const T* y0, const T* p, double t0, double t1, const double* save_t,
                    int ns, const double* h, int64_t S, T* y_save, T* loss) {
  const int d = pr.d;
  std::vector<double> ts;
  std::vector<int64_t> is;
  mesh_times(t0, t1, h, S, ts);
  save_index(ts, save_t, ns, is);
  std::vector<T> ys((S + 1) * d);
  for (int c = 0; c < d; ++c) ys[c] = y0[c];
  for (int64_t i = 1; i <= S; ++i)
    if (!phi_step(method, pr, &ys[(i - 1) * d], p, h[i - 1], &ys[i * d])) return false;
  T L = T(0.0);
  for (int s = 0; s < ns; ++s) {
    const T* yi = &ys[is[s] * d];
    double hs = save_t[s] - ts[is[s]];
    if (hs == 0.0) {
      for (int c = 0; c < d; ++c) y_save[s * d + c] = yi[c];
    } else if (!phi_step(method, pr, yi, p, hs, y_save + s * d)) {
      return false;
    }
    for (int c = 0; c < d; ++c) L = L + y_save[s * d + c] * y_save[s * d + c];
  }
  *loss = L;
  return true;
}

// Discrete adjoint of the replay (paper Sec. 3.1): the exact reverse-mode
// derivative of the chain with h held as data. ybar_save = dL/dy(t_s) if given,
// else the built-in loss's 2 y(t_s).
bool replay_grad(int method, const Prob& pr, const double* y0, const double* p, double t0, double t1,
                 const double* save_t, int ns, const double* h, int64_t S, const double* ybar_save, double* y_save,
                 double* loss, double* pbar, double* y0bar, double* wbar) {
  const int d = pr.d, P = pr.P;
  std::vector<double> ts;
  std::vector<int64_t> is;
  mesh_times(t0, t1, h, S, ts);
  save_index(ts, save_t, ns, is);
  std::vector<double> ys((S + 1) * d);
  for (int c = 0; c < d; ++c) ys[c] = y0[c];
  for (int64_t i = 1; i <= S; ++i)
    if (!phi_step(method, pr, &ys[(i - 1) * d], p, h[i - 1], &ys[i * d])) return false;
  double L = 0.0;
  for (int s = 0; s < ns; ++s) {
    const double* yi = &ys[is[s] * d];
    double hs = save_t[s] - ts[is[s]];
    if (hs == 0.0) {
      for (int c = 0; c < d; ++c) y_save[s * d + c] = yi[c];
    } else if (!phi_step(method, pr, yi, p, hs, y_save + s * d)) {
      return false;
    }
    for (int c = 0; c < d; ++c) L += y_save[s * d + c] * y_save[s * d + c];
  }
  *loss = L;
  for (int q = 0; q < P; ++q) pbar[q] = 0.0;
  double lam[DMAX] = {0};
  for (int64_t i = S; i >= 0; --i) {
    // cotangents of the save-time states attached to mesh point i
    for (int s = 0; s < ns; ++s) {
      if (is[s] != i) continue;
      double cb[DMAX];
      for (int c = 0; c < d; ++c) cb[c] = ybar_save ? ybar_save[s * d + c] : 2.0 * y_save[s * d + c];
      double hs = save_t[s] - ts[i];
      if (hs == 0.0) {
        for (int c = 0; c < d; ++c) lam[c] += cb[c];
      } else {
        double v[DMAX];
        if (!phi_step_vjp(method, pr, &ys[i * d], p, hs, cb, v, pbar, wbar)) return false;
        for (int c = 0; c < d; ++c) lam[c] += v[c];
      }
    }
    if (i > 0) {
      double v[DMAX];
      if (!phi_step_vjp(method, pr, &ys[(i - 1) * d], p, h[i - 1], lam, v, pbar, wbar)) return false;
      for (int c = 0; c < d; ++c) lam[c] = v[c];
    }
  }
  for (int c = 0; c < d; ++c) y0bar[c] = lam[c];
  return true;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F&& fn) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (nthreads > n) nthreads = (int)std::max<int64_t>(1, n);
  if (nthreads == 1) { for (int64_t i = 0; i < n; ++i) fn(i, 0); return; }
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] {
      for (int64_t i = t; i < n; i += nthreads) fn(i, t);
    });
  for (auto& x : th) x.join();
}

int resolve_method(int pid, int method) {
  if (method == 0) return stiff_of(pid) ? M_RODAS5P : M_TSIT5;
  return method;
}

}  // namespace

// ================================================================ C interface
// Array layouts are per trajectory (AoS): params[n][P], y0[n][d],
// y_save[n][ns][d]; the mesh is ragged: h[offsets[k] .. offsets[k+1]).
extern "C" {

int or_problem_info(int pid, int* d, int* P, int* stiff, int* n_shared) {
  if (dim_of(pid) < 0) return 1;
  *d = dim_of(pid);
  *P = npar_of(pid);
  *stiff = stiff_of(pid);
  *n_shared = nshared_of(pid);
  return 0;
}

// Coefficients, exported for the order-condition tests.
// method 1: A[7*7], b[7], bhat[7], c[7]; method 2: a[8*8], C[8*8], m[8], gamma;
// method 4: A[10*10], b[10], bhat[10], c[10].
int or_tableau(int method, double* A, double* b, double* bhat_or_C, double* c_or_gamma) {
  if (method == M_TSIT5) {
    const Tsit5Tab& t = tsit5();
    for (int i = 0; i < 7; ++i) {
      for (int j = 0; j < 7; ++j) A[i * 7 + j] = t.A[i][j];
      b[i] = t.b[i];
      bhat_or_C[i] = t.bhat[i];
      c_or_gamma[i] = t.c[i];
    }
    return 0;
  }
  if (method == M_VERN7) {
    const Vern7Tab& t = vern7();
    for (int i = 0; i < 10; ++i) {
      for (int j = 0; j < 10; ++j) A[i * 10 + j] = t.A[i][j];
      b[i] = t.b[i];
      bhat_or_C[i] = t.bhat[i];
      c_or_gamma[i] = t.c[i];
    }
    return 0;
  }
  if (method == M_RODAS5P) {
    const RodasTab& t = rodas();
    for (int i = 0; i < 8; ++i) {
      for (int j = 0; j < 8; ++j) { A[i * 8 + j] = t.a[i][j]; bhat_or_C[i * 8 + j] = t.C[i][j]; }
      b[i] = t.m[i];
    }
    *c_or_gamma = t.gamma;
    return 0;
  }
  return 1;
}

// Record: adaptive solve per trajectory. mesh_out[k * mesh_cap + i] = h_{i+1};
// S_out[k] accepted steps (-1 if mesh_cap was too small), n_att_out attempts.
int or_record(int pid, int method, int64_t n, const double* params, const double* y0, const double* w, double t0,
              double t1, const double* save_t, int ns, double rtol, double atol, int64_t max_steps, double h_init,
              int64_t mesh_cap, int64_t* S_out, double* mesh_out, int64_t* n_att_out, double* y_save,
              int32_t* status, int nthreads) {
  if (dim_of(pid) < 0) return 1;
  Prob pr{pid, dim_of(pid), npar_of(pid), w};
  method = resolve_method(pid, method);
  parallel_for(n, nthreads, [&](int64_t k, int) {
    RecordOut r = record_one(method, pr, y0 + k * pr.d, params + k * pr.P, t0, t1, save_t, ns, rtol, atol,
                             max_steps, h_init, y_save ? y_save + k * ns * pr.d : nullptr);
    status[k] = r.status;
    n_att_out[k] = r.n_att;
    if ((int64_t)r.h.size() > mesh_cap) {
      S_out[k] = -1;
    } else {
      S_out[k] = (int64_t)r.h.size();
      for (size_t i = 0; i < r.h.size(); ++i) mesh_out[k * mesh_cap + i] = r.h[i];
    }
  });
  return 0;
}

// Replay + discrete adjoint on a given ragged mesh. ybar_save may be null
// (built-in loss). wbar (shared-weight problems) receives the ensemble sum, accumulated in
// trajectory order.
int or_replay_grad(int pid, int method, int64_t n, const double* params, const double* y0, const double* w,
                   double t0, double t1, const double* save_t, int ns, const int64_t* offsets, const double* h,
                   const double* ybar_save, double* loss, double* y_save, double* pbar, double* y0bar, double* wbar,
                   int32_t* ok, int nthreads) {
  if (dim_of(pid) < 0) return 1;
  Prob pr{pid, dim_of(pid), npar_of(pid), w};
  method = resolve_method(pid, method);
  const int nw = wbar ? nshared_of(pid) : 0;
  std::vector<double> wpart(nw ? (size_t)n * nw : 0, 0.0);
  parallel_for(n, nthreads, [&](int64_t k, int) {
    double* wb = nw ? &wpart[(size_t)k * nw] : nullptr;
    bool good = replay_grad(method, pr, y0 + k * pr.d, params + k * pr.P, t0, t1, save_t, ns, h + offsets[k],
                            offsets[k + 1] - offsets[k], ybar_save ? ybar_save + k * ns * pr.d : nullptr,
                            y_save + k * ns * pr.d, loss + k, pbar + k * pr.P, y0bar + k * pr.d, wb);
    ok[k] = good ? 1 : 0;
  });
  if (nw) {
    for (int j = 0; j < nw; ++j) wbar[j] = 0.0;
    for (int64_t k = 0; k < n; ++k)
      for (int j = 0; j < nw; ++j) wbar[j] += wpart[(size_t)k * nw + j];
  }
  return 0;
}

// Forward-mode (dual-number) derivative of the replay along (params_dot, y0_dot):
// returns loss_dot[k] = d loss_k and y_save_dot.
int or_replay_jvp(int pid, int method, int64_t n, const double* params, const double* y0, const double* w,
                  double t0, double t1, const double* save_t, int ns, const int64_t* offsets, const double* h,
                  const double* params_dot, const double* y0_dot, double* loss, double* loss_dot,
                  double* y_save_dot, int nthreads) {
  if (dim_of(pid) < 0) return 1;
  Prob pr{pid, dim_of(pid), npar_of(pid), w};
  method = resolve_method(pid, method);
  using D = Dual<double>;
  parallel_for(n, nthreads, [&](int64_t k, int) {
    D yd[DMAX], pd[PMAX], L;
    for (int c = 0; c < pr.d; ++c) yd[c] = D(y0[k * pr.d + c], y0_dot[k * pr.d + c]);
    for (int q = 0; q < pr.P; ++q) pd[q] = D(params[k * pr.P + q], params_dot[k * pr.P + q]);
    std::vector<D> ysv((size_t)ns * pr.d);
    replay_forward(method, pr, yd, pd, t0, t1, save_t, ns, h + offsets[k], offsets[k + 1] - offsets[k],
                   ysv.data(), &L);
    loss[k] = L.v;
    loss_dot[k] = L.d;
    for (int i = 0; i < ns * pr.d; ++i) y_save_dot[k * ns * pr.d + i] = ysv[i].d;
  });
  return 0;
}

// One step of the method from each y (h per trajectory), for direct tests.
int or_step(int pid, int method, int64_t n, const double* params, const double* y, const double* w,
            const double* h, double* ynew, double* err) {
  if (dim_of(pid) < 0) return 1;
  Prob pr{pid, dim_of(pid), npar_of(pid), w};
  method = resolve_method(pid, method);
  for (int64_t k = 0; k < n; ++k) {
    const double* yk = y + k * pr.d;
    const double* pk = params + k * pr.P;
    if (method == M_TSIT5) {
      double Ys[7][DMAX], K[7][DMAX];
      tsit5_step(pr, yk, pk, h[k], Ys, K, ynew + k * pr.d, err + k * pr.d);
    } else if (method == M_ROS23) {
      double k1[DMAX], u2[DMAX], Y1[DMAX], LU[DMAX][DMAX];
      int perm[DMAX];
      if (!ros23_step(pr, yk, pk, h[k], ynew + k * pr.d, err + k * pr.d, k1, u2, Y1, LU, perm)) return 2;
    } else if (method == M_VERN7) {
      double Ys[10][DMAX], K[10][DMAX];
      vern7_step(pr, yk, pk, h[k], Ys, K, ynew + k * pr.d, err + k * pr.d);
    } else {
      double Ys[8][DMAX], U[8][DMAX], LU[DMAX][DMAX];
      int perm[DMAX];
      if (!rodas_step(pr, yk, pk, h[k], Ys, U, ynew + k * pr.d, err + k * pr.d, LU, perm)) return 2;
    }
  }
  return 0;
}

// f and J at given points (used to pin the problem definitions).
int or_rhs(int pid, int64_t n, const double* params, const double* y, const double* w, double* f, double* J) {
  if (dim_of(pid) < 0) return 1;
  Prob pr{pid, dim_of(pid), npar_of(pid), w};
  const int d = pr.d;
  for (int64_t k = 0; k < n; ++k) {
    f_eval(pr, y + k * d, params + k * pr.P, f + k * d);
    if (J) {
      double Jm[DMAX][DMAX];
      jac_y(pr, y + k * d, params + k * pr.P, Jm);
      for (int c = 0; c < d; ++c)
        for (int a = 0; a < d; ++a) J[k * d * d + c * d + a] = Jm[c][a];
    }
  }
  return 0;
}

// The shared-weight gradient of g = r^T J(y, w) u at one point (the weight
// part of the stiff adjoint's Jacobian contraction), for direct tests.
int or_w_contract(int pid, const double* y, const double* w, const double* r, const double* u, double* wbar) {
  if (dim_of(pid) < 0) return 1;
  Prob pr{pid, dim_of(pid), npar_of(pid), w};
  for (int k = 0; k < nshared_of(pid); ++k) wbar[k] = 0.0;
  w_contract(pr, y, r, u, wbar);
  return 0;
}

double or_initial_step(int pid, const double* params, const double* y0, const double* w, double t0, double t1,
                       double rtol, double atol, int order) {
  Prob pr{pid, dim_of(pid), npar_of(pid), w};
  return initial_step(pr, y0, params, t0, t1, rtol, atol, order);
}

}  // extern "C"
