// The Robertson neural right-hand side (paper Appendix A): Robertson with its
// autocatalytic term k2 y2^2 replaced, in both its sink and its source, by a
// shared-weight MLP NN: R^3 -> R (3-16-16-1, tanh hidden, softplus output):
//   y1' = -k1 y1 + k3 y2 y3,  y2' = k1 y1 - k3 y2 y3 - NN(y),  y3' = NN(y),
// theta = (k1, k3) per trajectory, 353 shared weights. A stiff problem, solved
// with Rodas5P or Rosenbrock23, so the network runs in FP64 like the rest of
// the stiff step (weights converted exactly from the FP32 inputs).
//
// The stiff adjoint needs, besides the VJP J^T v + f_theta^T v, the gradient of
// the Jacobian contraction r^T J(y, theta, w) u. Its network part is
// (r3 - r2) grad NN(y) . u: a forward tangent pass along u and a reverse pass
// through both the primal and the tangent values (second derivatives of the
// network with respect to its input and its weights).
//
// The shared-weight gradient is a sum over every lane, stage and step of
// rank-1 products (layer cotangent) x (layer input). Each call stages the
// lane's factors in shared memory and the warp contracts them over its 32
// lanes: lane l owns weights l, l + 32, ... and adds its 32-term sums in lane
// order (deterministic), in FP64, into registers held for the kernel's life.
#pragma once

#include "gs_device.cuh"

namespace gs {

constexpr int NR_H = 16;
constexpr int NR_NW = NR_H * 3 + NR_H + NR_H * NR_H + NR_H + NR_H + 1;  // 353
// Flat weight layout: W1[16][3], b1[16], W2[16][16], b2[16], W3[16], b3.
constexpr int NR_W1 = 0, NR_B1 = 48, NR_W2 = 64, NR_B2 = 320, NR_W3 = 336, NR_B3 = 352;
// Staged row per lane (doubles): a = [layer-3 cotangent | layer-2 cotangents (16)
// | layer-1 cotangents (16)], b = [layer-3 input h2 (16) | layer-2 input h1 (16)
// | layer-1 input (3) | bias multiplier]. Stride 69 (odd) spreads the rows over
// the banks.
constexpr int NR_A0 = 0, NR_A2 = 1, NR_A1 = 17, NR_BH2 = 33, NR_BH1 = 49, NR_BX = 65, NR_BONE = 68;
constexpr int NR_ROW = 69;
constexpr int NR_OWN = (NR_NW + 31) / 32;  // weights per lane
constexpr int NR_STAGE_DOUBLES = 4 * 32 * NR_ROW;  // 4 warps per 128-thread CTA

__device__ __forceinline__ double nr_sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }
__device__ __forceinline__ double nr_softplus(double z) { return fmax(z, 0.0) + log1p(exp(-fabs(z))); }

struct NeuralRobertson {
  static constexpr int D = 3, NP = 2;  // theta = (k1, k3)
  static constexpr bool kWeights = true;

  __device__ __forceinline__ static double* weights() {
    __shared__ double w[NR_NW];
    return w;
  }
  __device__ static void block_setup(const float* shared_w) {
    double* w = weights();
    for (int i = threadIdx.x; i < NR_NW; i += blockDim.x) w[i] = (double)shared_w[i];
  }

  struct Fwd {
    double h1[NR_H], h2[NR_H], z3;
  };
  // Primal pass at x. The compiler barrier keeps the weight loads in place
  // (they are re-read from shared memory at every use, not hoisted).
  __device__ __forceinline__ static void forward(const double (&x)[D], Fwd& F) {
    asm volatile("" ::: "memory");
    const double* w = weights();
#pragma unroll
    for (int i = 0; i < NR_H; ++i)
      F.h1[i] = tanh(fma_(w[NR_W1 + 3 * i + 2], x[2],
                          fma_(w[NR_W1 + 3 * i + 1], x[1], fma_(w[NR_W1 + 3 * i], x[0], w[NR_B1 + i]))));
#pragma unroll
    for (int i = 0; i < NR_H; ++i) {
      double s = w[NR_B2 + i];
#pragma unroll
      for (int j = 0; j < NR_H; ++j) s = fma_(w[NR_W2 + NR_H * i + j], F.h1[j], s);
      F.h2[i] = tanh(s);
    }
    double z = w[NR_B3];
#pragma unroll
    for (int j = 0; j < NR_H; ++j) z = fma_(w[NR_W3 + j], F.h2[j], z);
    F.z3 = z;
  }
  struct Back {
    double g3, g2[NR_H], g1[NR_H];  // cotangents of z3, z2, z1
  };
  // Reverse pass with seed c on NN: the layer cotangents and gx = c grad NN(x).
  __device__ __forceinline__ static void backward(const Fwd& F, double c, Back& B, double (&gx)[D]) {
    asm volatile("" ::: "memory");
    const double* w = weights();
    B.g3 = mul_(c, nr_sigmoid(F.z3));
    double gh1[NR_H];
#pragma unroll
    for (int j = 0; j < NR_H; ++j) gh1[j] = 0.0;
#pragma unroll
    for (int i = 0; i < NR_H; ++i) {
      const double g = mul_(mul_(B.g3, w[NR_W3 + i]), fma_(-F.h2[i], F.h2[i], 1.0));
      B.g2[i] = g;
#pragma unroll
      for (int j = 0; j < NR_H; ++j) gh1[j] = fma_(g, w[NR_W2 + NR_H * i + j], gh1[j]);
    }
#pragma unroll
    for (int j = 0; j < NR_H; ++j) B.g1[j] = mul_(gh1[j], fma_(-F.h1[j], F.h1[j], 1.0));
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < NR_H; ++j) s = fma_(w[NR_W1 + 3 * j + a], B.g1[j], s);
      gx[a] = s;
    }
  }

  __device__ __forceinline__ static void f(const double (&y)[D], const double (&p)[NP], double (&o)[D]) {
    Fwd F;
    forward(y, F);
    const double nn = nr_softplus(F.z3);
    const double rob = fma_(-p[0], y[0], mul_(mul_(p[1], y[1]), y[2]));  // -k1 y1 + k3 y2 y3
    o[0] = rob;
    o[1] = sub_(-rob, nn);
    o[2] = nn;
  }
  // FP32 arguments (the starting-step estimate only): evaluated in FP64.
  __device__ __forceinline__ static void f(const float (&y)[D], const float (&p)[NP], float (&o)[D]) {
    const double yd[D] = {(double)y[0], (double)y[1], (double)y[2]};
    const double pd[NP] = {(double)p[0], (double)p[1]};
    double od[D];
    f(yd, pd, od);
#pragma unroll
    for (int c = 0; c < D; ++c) o[c] = (float)od[c];
  }
  template <class R>
  __device__ __forceinline__ static void jac(const R (&y)[D], const R (&p)[NP], R (&J)[D][D]) {
    Fwd F;
    Back B;
    double g[D];
    forward(y, F);
    backward(F, 1.0, B, g);
    const double k3y2 = mul_(p[1], y[2]), k3y1 = mul_(p[1], y[1]);
    J[0][0] = -p[0]; J[0][1] = k3y2;             J[0][2] = k3y1;
    J[1][0] = sub_(p[0], g[0]); J[1][1] = sub_(-k3y2, g[1]); J[1][2] = sub_(-k3y1, g[2]);
    J[2][0] = g[0];  J[2][1] = g[1];             J[2][2] = g[2];
  }
  // The VJP at y with cotangent v: yb = J^T v, pb += f_theta^T v; the weight
  // cotangent is c dNN/dw with c = v3 - v2 (factors in B, layer inputs in F).
  __device__ __forceinline__ static void vjp_nn(const double (&y)[D], const double (&p)[NP], const double (&v)[D],
                                                double (&yb)[D], double (&pb)[NP], Fwd& F, Back& B) {
    const double q = sub_(v[0], v[1]);
    double g[D];
    forward(y, F);
    backward(F, sub_(v[2], v[1]), B, g);
    yb[0] = fma_(-q, p[0], g[0]);
    yb[1] = fma_(mul_(q, p[1]), y[2], g[1]);
    yb[2] = fma_(mul_(q, p[1]), y[1], g[2]);
    pb[0] = fma_(-q, y[0], pb[0]);
    pb[1] = fma_(mul_(q, y[1]), y[2], pb[1]);
  }
  struct Tan {
    double hd1[NR_H], hd2[NR_H];  // tangents of h1, h2 along u
    double d3, d2[NR_H], d1[NR_H];  // cotangents of the tangent pre-activations zd3, zd2, zd1
  };
  // Gradient of g = r^T J(y) u: gy += dg/dy, pb += dg/dtheta; the weight part
  // (r3 - r2) d/dw (grad NN . u) leaves its primal-layer cotangents in B (with
  // layer inputs F) and its tangent-layer cotangents in T (inputs T.hd*, u).
  __device__ __forceinline__ static void contract_nn(const double (&y)[D], const double (&p)[NP],
                                                     const double (&r)[D], const double (&u)[D], double (&gy)[D],
                                                     double (&pb)[NP], Fwd& F, Back& B, Tan& T) {
    asm volatile("" ::: "memory");
    const double* w = weights();
    // Robertson part: (r1 - r2) (-k1 u1 + k3 (y3 u2 + y2 u3)) (1-based)
    const double q = sub_(r[0], r[1]);
    gy[1] = fma_(mul_(q, p[1]), u[2], gy[1]);
    gy[2] = fma_(mul_(q, p[1]), u[1], gy[2]);
    pb[0] = fma_(-q, u[0], pb[0]);
    pb[1] = fma_(q, fma_(y[2], u[1], mul_(y[1], u[2])), pb[1]);
    // network part: primal and tangent forward passes
    forward(y, F);
    double zd1[NR_H], zd2[NR_H];
#pragma unroll
    for (int i = 0; i < NR_H; ++i) {
      zd1[i] = fma_(w[NR_W1 + 3 * i + 2], u[2], fma_(w[NR_W1 + 3 * i + 1], u[1], mul_(w[NR_W1 + 3 * i], u[0])));
      T.hd1[i] = mul_(fma_(-F.h1[i], F.h1[i], 1.0), zd1[i]);
    }
#pragma unroll
    for (int i = 0; i < NR_H; ++i) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < NR_H; ++j) s = fma_(w[NR_W2 + NR_H * i + j], T.hd1[j], s);
      zd2[i] = s;
      T.hd2[i] = mul_(fma_(-F.h2[i], F.h2[i], 1.0), s);
    }
    double zd3 = 0.0;
#pragma unroll
    for (int j = 0; j < NR_H; ++j) zd3 = fma_(w[NR_W3 + j], T.hd2[j], zd3);
    // reverse through g = sigma(z3) zd3 with seed c
    const double c = sub_(r[2], r[1]);
    const double s3 = nr_sigmoid(F.z3);
    T.d3 = mul_(c, s3);
    B.g3 = mul_(mul_(mul_(c, zd3), s3), sub_(1.0, s3));
    double hd1b[NR_H], h1b[NR_H];
#pragma unroll
    for (int j = 0; j < NR_H; ++j) hd1b[j] = h1b[j] = 0.0;
#pragma unroll
    for (int i = 0; i < NR_H; ++i) {
      const double om = fma_(-F.h2[i], F.h2[i], 1.0);
      const double hd2b = mul_(T.d3, w[NR_W3 + i]);
      const double h2b = fma_(mul_(-2.0, F.h2[i]), mul_(zd2[i], hd2b), mul_(B.g3, w[NR_W3 + i]));
      T.d2[i] = mul_(om, hd2b);
      B.g2[i] = mul_(om, h2b);
#pragma unroll
      for (int j = 0; j < NR_H; ++j) {
        hd1b[j] = fma_(T.d2[i], w[NR_W2 + NR_H * i + j], hd1b[j]);
        h1b[j] = fma_(B.g2[i], w[NR_W2 + NR_H * i + j], h1b[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < NR_H; ++j) {
      const double om = fma_(-F.h1[j], F.h1[j], 1.0);
      T.d1[j] = mul_(om, hd1b[j]);
      B.g1[j] = mul_(om, fma_(mul_(-2.0, F.h1[j]), mul_(zd1[j], hd1b[j]), h1b[j]));
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < NR_H; ++j) s = fma_(w[NR_W1 + 3 * j + a], B.g1[j], s);
      gy[a] = add_(gy[a], s);
    }
  }
};

// Accumulator of the neural Robertson reverse sweep: the per-trajectory
// (k1, k3) gradient (FP64, per lane) and this lane's share of the warp's
// shared-weight gradient (weights lane, lane + 32, ...).
struct NrAcc {
  using Part = double;
  static constexpr int NW = NR_NW;
  PlainAcc<2> th;
  double wacc[NR_OWN];
  double* stage;  // this warp's staging rows (dynamic shared memory)
  __device__ void init(double* stage_base) {
    stage = stage_base + (threadIdx.x >> 5) * 32 * NR_ROW;
#pragma unroll
    for (int o = 0; o < NR_OWN; ++o) wacc[o] = 0.0;
  }
  __device__ void zero() { th.zero(); }
  __device__ __forceinline__ void flush() {}
  __device__ double get(int q) const { return th.get(q); }

  // (a, b) row offsets of flat weight q.
  __device__ __forceinline__ static void decode(int q, int& ao, int& bo) {
    if (q < NR_B1) { ao = NR_A1 + q / 3; bo = NR_BX + q % 3; }
    else if (q < NR_W2) { ao = NR_A1 + (q - NR_B1); bo = NR_BONE; }
    else if (q < NR_B2) { ao = NR_A2 + (q - NR_W2) / NR_H; bo = NR_BH1 + (q - NR_W2) % NR_H; }
    else if (q < NR_W3) { ao = NR_A2 + (q - NR_B2); bo = NR_BONE; }
    else if (q < NR_B3) { ao = NR_A0; bo = NR_BH2 + (q - NR_W3); }
    else { ao = NR_A0; bo = NR_BONE; }
  }
  // Warp-collective: every lane stages one rank-1 set (zeros for lanes without
  // work) and the warp adds the 32 rows' products into the owned weights.
  __device__ __forceinline__ void accumulate(double a0, const double (&a2)[NR_H], const double (&a1)[NR_H],
                                             const double (&bh2)[NR_H], const double (&bh1)[NR_H],
                                             const double (&bx)[3], double bone) {
    const int lane = threadIdx.x & 31;
    double* row = stage + lane * NR_ROW;
    __syncwarp();
    row[NR_A0] = a0;
#pragma unroll
    for (int i = 0; i < NR_H; ++i) {
      row[NR_A2 + i] = a2[i];
      row[NR_A1 + i] = a1[i];
      row[NR_BH2 + i] = bh2[i];
      row[NR_BH1 + i] = bh1[i];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) row[NR_BX + a] = bx[a];
    row[NR_BONE] = bone;
    __syncwarp();
#pragma unroll
    for (int o = 0; o < NR_OWN; ++o) {
      const int q = lane + 32 * o;
      if (q < NR_NW) {
        int ao, bo;
        decode(q, ao, bo);
        double s = 0.0;
        for (int kk = 0; kk < 32; ++kk) s = fma_(stage[kk * NR_ROW + ao], stage[kk * NR_ROW + bo], s);
        wacc[o] = add_(wacc[o], s);
      }
    }
  }

  template <class Pb>
  __device__ __forceinline__ void vjp(const double (&y)[3], const double (&p)[2], const double (&v)[3],
                                      double (&yb)[3]) {
    NeuralRobertson::Fwd F;
    NeuralRobertson::Back B;
    NeuralRobertson::vjp_nn(y, p, v, yb, th.s, F, B);
    accumulate(B.g3, B.g2, B.g1, F.h2, F.h1, y, 1.0);
  }
  template <class Pb>
  __device__ __forceinline__ void jac_contract(const double (&y)[3], const double (&p)[2], const double (&r)[3],
                                               const double (&u)[3], double (&gy)[3]) {
    NeuralRobertson::Fwd F;
    NeuralRobertson::Back B;
    NeuralRobertson::Tan T;
    NeuralRobertson::contract_nn(y, p, r, u, gy, th.s, F, B, T);
    accumulate(B.g3, B.g2, B.g1, F.h2, F.h1, y, 1.0);       // primal-layer terms
    accumulate(T.d3, T.d2, T.d1, T.hd2, T.hd1, u, 0.0);     // tangent-layer terms (no bias)
  }
  // Writes this lane's owned sums into the warp's partial (NR_NW doubles).
  __device__ void finish(void* part_base, size_t warp) {
    double* part = static_cast<double*>(part_base) + warp * NR_NW;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 0; o < NR_OWN; ++o) {
      const int q = lane + 32 * o;
      if (q < NR_NW) part[q] = wacc[o];
    }
  }
};

}  // namespace gs
