// The LV UDE problem: dx/dt = a x - NN(x, y)_1, dy/dt = -d y + NN(x, y)_2 with a
// shared-weight MLP 2-16-16-2 (tanh hidden layers, linear output), FP32.
//
// The record kernel evaluates the network per lane on the FP32 CUDA cores
// (weights in shared memory, broadcast reads); the reverse sweep evaluates and
// differentiates it warp-collectively, its 16 x 16 hidden layer on the tensor
// cores (LvUdeWarp below). The gradient with respect to the
// 354 shared weights is a sum over every lane, stage and step of rank-1
// products, i.e. a dense contraction over the lanes; each warp accumulates it
// with tensor-core MMAs (mma.sync m16n8k8, TF32 inputs split hi + lo so that
// the three products hi*hi + hi*lo + lo*hi carry FP32 accuracy), with the
// lanes as the contraction dimension and the accumulators held in registers
// for the kernel's whole life. Each warp writes its partial sums once; a
// separate kernel adds the partials in warp order (deterministic).
#pragma once

#include "gs_device.cuh"

namespace gs {

constexpr int UDE_H = 16;
constexpr int UDE_NW = UDE_H * 2 + UDE_H + UDE_H * UDE_H + UDE_H + 2 * UDE_H + 2;  // 354
// Flat weight layout: W1[16][2], b1[16], W2[16][16], b2[16], W3[2][16], b3[2].
constexpr int UDE_W1 = 0, UDE_B1 = 32, UDE_W2 = 48, UDE_B2 = 304, UDE_W3 = 320, UDE_B3 = 352;

// tanh(z) = 1 - 2 / (exp(2 z) + 1) with the hardware exp2 and an IEEE
// reciprocal: absolute error ~1e-7 (FP32 level), exact limits +-1.
__device__ __forceinline__ float tanh_f32(float z) {
  const float e = ex2_approx(z * 2.8853900817779268f);  // 2 / ln 2
  return 1.0f - 2.0f * __frcp_rn(e + 1.0f);
}

struct LvUde {
  static constexpr int D = 2, NP = 2;
  static constexpr bool kWeights = true;

  // Shared-memory copy of the 354 weights, one per CTA.
  __device__ __forceinline__ static float* weights() {
    __shared__ float w[UDE_NW];
    return w;
  }
  __device__ static void block_setup(const float* shared_w) {
    float* w = weights();
    for (int i = threadIdx.x; i < UDE_NW; i += blockDim.x) w[i] = shared_w[i];
  }
  // The weights are read from shared memory at every use: the compiler barrier
  // keeps it from hoisting the 354 loads out of the solver loops into
  // registers, which do not hold them (they would spill to local memory).
  __device__ __forceinline__ static void forward(float x, float y, float (&h1)[UDE_H], float (&h2)[UDE_H],
                                                 float (&nn)[2]) {
    asm volatile("" ::: "memory");
    const float* w = weights();
#pragma unroll
    for (int i = 0; i < UDE_H; ++i)
      h1[i] = tanh_f32(fmaf(w[UDE_W1 + 2 * i + 1], y, fmaf(w[UDE_W1 + 2 * i], x, w[UDE_B1 + i])));
#pragma unroll
    for (int i = 0; i < UDE_H; ++i) {
      float s = w[UDE_B2 + i];
#pragma unroll
      for (int j = 0; j < UDE_H; ++j) s = fmaf(w[UDE_W2 + UDE_H * i + j], h1[j], s);
      h2[i] = tanh_f32(s);
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      float s = w[UDE_B3 + o];
#pragma unroll
      for (int j = 0; j < UDE_H; ++j) s = fmaf(w[UDE_W3 + UDE_H * o + j], h2[j], s);
      nn[o] = s;
    }
  }
  __device__ __forceinline__ static void f(const float (&y)[D], const float (&p)[NP], float (&o)[D]) {
    float h1[UDE_H], h2[UDE_H], nn[2];
    forward(y[0], y[1], h1, h2, nn);
    o[0] = fmaf(p[0], y[0], -nn[0]);
    o[1] = fmaf(-p[1], y[1], nn[1]);
  }
};

// ---------------------------------------------------------------------------
// Warp-level TF32 MMA (m16n8k8, row.col, FP32 accumulate).
// Fragment ownership (g = lane / 4, t = lane % 4):
//   A (16x8): a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4)
//   B (8x8):  b0 (t, g), b1 (t+4, g)
//   C (16x8): c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
struct Tf32x2 {  // x = hi + lo, both TF32
  uint32_t hi, lo;
};
__device__ __forceinline__ Tf32x2 split_tf32(float x) {
  Tf32x2 s;
  s.hi = to_tf32(x);
  s.lo = to_tf32(x - __uint_as_float(s.hi));
  return s;
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// c += A B with A, B given as hi/lo splits: hi*hi + hi*lo + lo*hi.
__device__ __forceinline__ void mma_3xtf32(float (&c)[4], const Tf32x2 (&a)[4], const Tf32x2 (&b)[2]) {
  const uint32_t ah[4] = {a[0].hi, a[1].hi, a[2].hi, a[3].hi}, al[4] = {a[0].lo, a[1].lo, a[2].lo, a[3].lo};
  const uint32_t bh[2] = {b[0].hi, b[1].hi}, bl[2] = {b[0].lo, b[1].lo};
  mma_tf32(c, al, bh);
  mma_tf32(c, ah, bl);
  mma_tf32(c, ah, bh);
}

// Per-warp staging of the lanes' factor vectors for the weight-gradient MMAs.
// Row per lane, 72 floats: [gz2 0..15 | h1 16..31 | gz1 32..47 | h2 48..63 |
// x 64, y 65, go0 66, go1 67], with column c of row r stored at
// c ^ ude_sw(r) (rows with bit 2 set swap their 4-column groups pairwise). With
// the stride of 72 the weight-gradient fragment reads (rows t, t + 4, columns
// g) and the hidden-layer fragment reads (rows g, g + 8, columns t, t + 4)
// each hit 32 distinct banks, and so do the per-lane 16-byte row accesses.
constexpr int UDE_ROW = 72;
__device__ __forceinline__ int ude_sw(int row) { return row & 4; }
constexpr int UDE_WARPS_PER_CTA = 4;

__device__ __forceinline__ float* ude_stage() {
  __shared__ __align__(16) float s[UDE_WARPS_PER_CTA][32 * UDE_ROW];
  return s[threadIdx.x >> 5];
}

// ---------------------------------------------------------------------------
// Warp-collective form of the network for the reverse sweep, where every lane
// of a warp evaluates the network together (lanes without work pass zeros).
// The 16 x 16 hidden layer, forward (Z2 = H1 W2^T) and backward
// (GH1 = GZ2 W2), runs on the tensor cores as [32 lanes x 16] x [16 x 16]
// products (mma.sync m16n8k8, 3xTF32: activations split hi + lo per call, W2
// split once per CTA into fragment tables); the 2-wide input and output layers
// and the elementwise work stay per lane. The lanes exchange their vectors
// through the warp's staging rows (the same rows the weight-gradient MMAs read:
// after a VJP they already hold gz2, h1, gz1, h2, x, y, go).
// ---------------------------------------------------------------------------
struct LvUdeWarp : LvUde {
  // B fragments of the two hidden-layer products, per lane, pre-split:
  // [q][kk][nt][lane] = {b0.hi, b0.lo, b1.hi, b1.lo} with q = 0: B[k][n] = W2[n][k]
  // (forward), q = 1: B[k][n] = W2[k][n] (backward); k = 8 kk + t (+4), n = 8 nt + g.
  __device__ __forceinline__ static uint4* frags() {
    __shared__ uint4 f[2 * 2 * 2 * 32];
    return f;
  }
  __device__ static void block_setup(const float* shared_w) {
    LvUde::block_setup(shared_w);
    uint4* f = frags();
    for (int i = threadIdx.x; i < 2 * 2 * 2 * 32; i += blockDim.x) {
      const int lane = i & 31, nt = (i >> 5) & 1, kk = (i >> 6) & 1, q = i >> 7;
      const int g = lane >> 2, t = lane & 3, n = 8 * nt + g, k0 = 8 * kk + t, k1 = k0 + 4;
      const float b0 = q == 0 ? shared_w[UDE_W2 + UDE_H * n + k0] : shared_w[UDE_W2 + UDE_H * k0 + n];
      const float b1 = q == 0 ? shared_w[UDE_W2 + UDE_H * n + k1] : shared_w[UDE_W2 + UDE_H * k1 + n];
      const Tf32x2 s0 = split_tf32(b0), s1 = split_tf32(b1);
      f[i] = make_uint4(s0.hi, s0.lo, s1.hi, s1.lo);
    }
  }
  // c[mt][nt] = rows' [32 x 16] block at column offset `off` times B of product q.
  __device__ __forceinline__ static void hidden_mma(float (&c)[2][2][4], const float* st, int off, int q) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint4* f = frags() + q * 128;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) c[mt][nt][e] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      uint4 bf[2];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) bf[nt] = f[(kk * 2 + nt) * 32 + lane];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const float* r0 = st + (16 * mt + g) * UDE_ROW;
        const float* r1 = r0 + 8 * UDE_ROW;
        const int sw = ude_sw(g), c0 = (off + 8 * kk + t) ^ sw, c1 = (off + 8 * kk + t + 4) ^ sw;
        const Tf32x2 a[4] = {split_tf32(r0[c0]), split_tf32(r1[c0]), split_tf32(r0[c1]), split_tf32(r1[c1])};
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const Tf32x2 b[2] = {{bf[nt].x, bf[nt].y}, {bf[nt].z, bf[nt].w}};
          mma_3xtf32(c[mt][nt], a, b);
        }
      }
    }
  }
  // Forward pass of all lanes: leaves h1 and h2 in the staging rows and
  // returns this lane's network output and h2.
  __device__ __forceinline__ static void forward_warp(float x, float y, float (&h2)[UDE_H], float (&nn)[2]) {
    float* st = ude_stage();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, swl = ude_sw(lane), swg = ude_sw(g);
    float* row = st + lane * UDE_ROW;
    __syncwarp();
    asm volatile("" ::: "memory");
    const float* w = weights();
#pragma unroll
    for (int j = 0; j < UDE_H; j += 4) {
      float h[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        h[u] = tanh_f32(fmaf(w[UDE_W1 + 2 * (j + u) + 1], y, fmaf(w[UDE_W1 + 2 * (j + u)], x, w[UDE_B1 + j + u])));
      *reinterpret_cast<float4*>(row + ((16 + j) ^ swl)) = make_float4(h[0], h[1], h[2], h[3]);
    }
    __syncwarp();
    float c[2][2][4];
    hidden_mma(c, st, 16, 0);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {  // rows g and g + 8 of the tile
          const int r = 16 * mt + g + 8 * hf, col = 8 * nt + 2 * t;
          const float v0 = tanh_f32(c[mt][nt][2 * hf] + w[UDE_B2 + col]);
          const float v1 = tanh_f32(c[mt][nt][2 * hf + 1] + w[UDE_B2 + col + 1]);
          *reinterpret_cast<float2*>(st + r * UDE_ROW + ((48 + col) ^ swg)) = make_float2(v0, v1);
        }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < UDE_H; j += 4) {
      const float4 v = *reinterpret_cast<const float4*>(row + ((48 + j) ^ swl));
      h2[j] = v.x;
      h2[j + 1] = v.y;
      h2[j + 2] = v.z;
      h2[j + 3] = v.w;
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      float s = w[UDE_B3 + o];
#pragma unroll
      for (int j = 0; j < UDE_H; ++j) s = fmaf(w[UDE_W3 + UDE_H * o + j], h2[j], s);
      nn[o] = s;
    }
  }
  __device__ __forceinline__ static void f(const float (&y)[D], const float (&p)[NP], float (&o)[D]) {
    float h2[UDE_H], nn[2];
    forward_warp(y[0], y[1], h2, nn);
    o[0] = fmaf(p[0], y[0], -nn[0]);
    o[1] = fmaf(-p[1], y[1], nn[1]);
  }
  // VJP of all lanes (as LvUde::backprop): yb = J^T v, pb += f_theta^T v, and the
  // staging rows left holding [gz2 | h1 | gz1 | h2 | x, y, go] for the
  // weight-gradient MMAs.
  __device__ __forceinline__ static void backprop_warp(const float (&y)[D], const float (&p)[NP],
                                                       const float (&v)[D], float (&yb)[D], float (&pb)[NP]) {
    float* st = ude_stage();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, swl = ude_sw(lane), swg = ude_sw(g);
    float* row = st + lane * UDE_ROW;
    float h2[UDE_H], nn[2];
    forward_warp(y[0], y[1], h2, nn);
    const float* w = weights();
    const float go0 = -v[0], go1 = v[1];  // f0 = a x - nn0, f1 = -d y + nn1
    *reinterpret_cast<float4*>(row + (64 ^ swl)) = make_float4(y[0], y[1], go0, go1);
#pragma unroll
    for (int j = 0; j < UDE_H; j += 4) {
      float z[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float gh = fmaf(w[UDE_W3 + j + u], go0, w[UDE_W3 + UDE_H + j + u] * go1);
        z[u] = gh * fmaf(-h2[j + u], h2[j + u], 1.0f);
      }
      *reinterpret_cast<float4*>(row + (j ^ swl)) = make_float4(z[0], z[1], z[2], z[3]);
    }
    __syncwarp();
    float c[2][2][4];
    hidden_mma(c, st, 0, 1);  // GH1 = GZ2 W2
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int r = 16 * mt + g + 8 * hf, col = 8 * nt + 2 * t;
          const float2 h1 = *reinterpret_cast<const float2*>(st + r * UDE_ROW + ((16 + col) ^ swg));
          const float z0 = c[mt][nt][2 * hf] * fmaf(-h1.x, h1.x, 1.0f);
          const float z1 = c[mt][nt][2 * hf + 1] * fmaf(-h1.y, h1.y, 1.0f);
          *reinterpret_cast<float2*>(st + r * UDE_ROW + ((32 + col) ^ swg)) = make_float2(z0, z1);
        }
    __syncwarp();
    float gx = 0.0f, gy = 0.0f;
#pragma unroll
    for (int j = 0; j < UDE_H; j += 4) {
      const float4 z = *reinterpret_cast<const float4*>(row + ((32 + j) ^ swl));
      const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        gx = fmaf(w[UDE_W1 + 2 * (j + u)], zz[u], gx);
        gy = fmaf(w[UDE_W1 + 2 * (j + u) + 1], zz[u], gy);
      }
    }
    yb[0] = fmaf(p[0], v[0], gx);
    yb[1] = fmaf(-p[1], v[1], gy);
    pb[0] = fmaf(y[0], v[0], pb[0]);
    pb[1] = fmaf(-y[1], v[1], pb[1]);
  }
};

// ---------------------------------------------------------------------------
// CTA-collective form of the network for the reverse sweep: the CTA's 128
// lanes evaluate it together (lanes without work pass zeros), and the 16 x 16
// hidden layer, forward (Z2 = H1 W2^T) and backward (GH1 = GZ2 W2), is ONE
// [128 lanes x 16] x [16 x 16] product on the fifth-generation tensor cores
// (tcgen05.mma, kind::tf32, M = 128, N = 16, two K = 8 steps; activations and
// weights split hi + lo, the three products hi*hi + lo*hi + hi*lo accumulated
// in FP32 in tensor memory for FP32 accuracy). Each lane writes its row of the
// activation operand to shared memory in the canonical K-major layout (core
// matrices of 8 rows x 16 bytes, no swizzle), one elected thread issues the
// MMAs and commits them to an mbarrier, and each lane reads its own output row
// back from tensor memory (TMEM lane = CTA lane). The weight-gradient
// contraction keeps the warp MMAs of UdeAcc: its 16-row outputs are below the
// tcgen05 minimum of M = 64.
// ---------------------------------------------------------------------------
struct UdeTc {
  // Operand tiles: A hi / lo [128 x 16] (8 KB each); B hi / lo for the forward
  // product (W2 as [n][k]) and the backward one (W2^T), 1 KB each.
  __device__ __forceinline__ static unsigned char* tiles() {
    __shared__ __align__(1024) unsigned char t[2 * 8192 + 4 * 1024];
    return t;
  }
  __device__ __forceinline__ static unsigned long long* mbar() {
    __shared__ __align__(8) unsigned long long m;
    return &m;
  }
  __device__ __forceinline__ static uint32_t* tmem_slot() {
    __shared__ uint32_t t;
    return &t;
  }
  // per-thread parity of the mbarrier phase the next product completes
  __device__ __forceinline__ static unsigned char* phase() {
    __shared__ unsigned char ph[128];
    return ph;
  }
  __device__ __forceinline__ static int* error() {
    __shared__ int e;
    return &e;
  }
  // byte offset of element (row, k) of a [rows x 16] FP32 operand: core matrices
  // of 8 rows x 4 elements, 128 B apart along k (LBO), 512 B apart along rows (SBO)
  __device__ __forceinline__ static int off(int row, int k) {
    return (row >> 3) * 512 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
  }
  __device__ __forceinline__ static uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
  // shared-memory matrix descriptor: start >> 4, LBO 128 B, SBO 512 B, version 1, no swizzle
  __device__ __forceinline__ static uint64_t desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46);
  }
  // instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, N = 16, M = 128
  static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

  // Called by all 128 threads before the sweep (followed by a CTA barrier).
  __device__ static void setup(const float* shared_w) {
    unsigned char* t = tiles();
    for (int i = threadIdx.x; i < 2 * 256; i += blockDim.x) {
      const int q = i >> 8, n = (i >> 4) & 15, k = i & 15;
      const float v = q == 0 ? shared_w[UDE_W2 + UDE_H * n + k] : shared_w[UDE_W2 + UDE_H * k + n];
      const Tf32x2 sp = split_tf32(v);
      *reinterpret_cast<uint32_t*>(t + 16384 + q * 2048 + off(n, k)) = sp.hi;
      *reinterpret_cast<uint32_t*>(t + 16384 + q * 2048 + 1024 + off(n, k)) = sp.lo;
    }
    phase()[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
      *error() = 0;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar())));
      asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if ((threadIdx.x >> 5) == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(saddr(tmem_slot())));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  // Called by all 128 threads after the sweep.
  __device__ static void teardown(int* err_out) {
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if ((threadIdx.x >> 5) == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(*tmem_slot()));
    if (threadIdx.x == 0 && *error() && err_out) atomicExch(err_out, 1);
  }
  // out = in x B_q for this lane's row (in: 16 values), CTA-collective.
  __device__ __forceinline__ static void product(const float (&in)[UDE_H], int q, float (&out)[UDE_H]) {
    unsigned char* t = tiles();
    const int row = threadIdx.x;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const Tf32x2 s0 = split_tf32(in[4 * c]), s1 = split_tf32(in[4 * c + 1]), s2 = split_tf32(in[4 * c + 2]),
                   s3 = split_tf32(in[4 * c + 3]);
      *reinterpret_cast<uint4*>(t + off(row, 4 * c)) = make_uint4(s0.hi, s1.hi, s2.hi, s3.hi);
      *reinterpret_cast<uint4*>(t + 8192 + off(row, 4 * c)) = make_uint4(s0.lo, s1.lo, s2.lo, s3.lo);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot();
    if (threadIdx.x == 0) {
      const uint32_t ah = saddr(t), al = ah + 8192, bh = ah + 16384 + q * 2048, bl = bh + 1024;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {  // K = 16 as two K = 8 steps: the next two core-matrix columns
        const uint32_t o = kk * 256;
        const uint64_t dah = desc(ah + o), dal = desc(al + o), dbh = desc(bh + o), dbl = desc(bl + o);
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(dah), "l"(dbh), "r"(IDESC), "r"(kk));
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(dal), "l"(dbh), "r"(IDESC), "r"(1));
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(dah), "l"(dbl), "r"(IDESC), "r"(1));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(mbar())));
    }
    // wait for the commit (bounded: after ~1 s of polling the product is abandoned
    // and the CTA's error flag set; the host then reports the launch as failed)
    const uint32_t ph = phase()[row];
    uint32_t done = 0;
    for (int spin = 0; spin < (1 << 24) && !done; ++spin) {
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                   : "=r"(done)
                   : "r"(saddr(mbar())), "r"(ph));
    }
    if (!done) *error() = 1;
    phase()[row] = (unsigned char)(ph ^ 1u);
    asm volatile("tcgen05.fence::after_thread_sync;");
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(tmem + ((uint32_t)(row & ~31) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < UDE_H; ++j) out[j] = __uint_as_float(r[j]);
    // (the next product's CTA barrier orders this lane's TMEM read before the
    // next MMA; its operand tiles are free once the commit has arrived)
  }
};

struct LvUdeCta : LvUde {
  static constexpr bool kCta = true;  // the reverse sweep runs its units CTA-collectively
  __device__ static void block_setup(const float* shared_w) {
    LvUde::block_setup(shared_w);
    UdeTc::setup(shared_w);
  }
  __device__ static void block_teardown(int* err) { UdeTc::teardown(err); }
  // Forward pass of all lanes: leaves h1 and h2 in this lane's staging row and
  // returns its network output and h2.
  __device__ __forceinline__ static void forward_cta(float x, float y, float (&h2)[UDE_H], float (&nn)[2]) {
    float* row = ude_stage() + (threadIdx.x & 31) * UDE_ROW;
    const int swl = ude_sw(threadIdx.x & 31);
    asm volatile("" ::: "memory");
    const float* w = weights();
    float h1[UDE_H];
#pragma unroll
    for (int j = 0; j < UDE_H; ++j)
      h1[j] = tanh_f32(fmaf(w[UDE_W1 + 2 * j + 1], y, fmaf(w[UDE_W1 + 2 * j], x, w[UDE_B1 + j])));
#pragma unroll
    for (int j = 0; j < UDE_H; j += 4)
      *reinterpret_cast<float4*>(row + ((16 + j) ^ swl)) = make_float4(h1[j], h1[j + 1], h1[j + 2], h1[j + 3]);
    float z[UDE_H];
    UdeTc::product(h1, 0, z);
#pragma unroll
    for (int j = 0; j < UDE_H; ++j) h2[j] = tanh_f32(z[j] + w[UDE_B2 + j]);
#pragma unroll
    for (int j = 0; j < UDE_H; j += 4)
      *reinterpret_cast<float4*>(row + ((48 + j) ^ swl)) = make_float4(h2[j], h2[j + 1], h2[j + 2], h2[j + 3]);
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      float s = w[UDE_B3 + o];
#pragma unroll
      for (int j = 0; j < UDE_H; ++j) s = fmaf(w[UDE_W3 + UDE_H * o + j], h2[j], s);
      nn[o] = s;
    }
  }
  __device__ __forceinline__ static void f(const float (&y)[D], const float (&p)[NP], float (&o)[D]) {
    float h2[UDE_H], nn[2];
    forward_cta(y[0], y[1], h2, nn);
    o[0] = fmaf(p[0], y[0], -nn[0]);
    o[1] = fmaf(-p[1], y[1], nn[1]);
  }
  // VJP of all lanes (as LvUdeWarp::backprop_warp), leaving this lane's staging
  // row holding [gz2 | h1 | gz1 | h2 | x, y, go] for the weight-gradient MMAs.
  __device__ __forceinline__ static void backprop_cta(const float (&y)[D], const float (&p)[NP], const float (&v)[D],
                                                      float (&yb)[D], float (&pb)[NP]) {
    float* row = ude_stage() + (threadIdx.x & 31) * UDE_ROW;
    const int swl = ude_sw(threadIdx.x & 31);
    float h2[UDE_H], nn[2];
    forward_cta(y[0], y[1], h2, nn);
    const float* w = weights();
    const float go0 = -v[0], go1 = v[1];  // f0 = a x - nn0, f1 = -d y + nn1
    *reinterpret_cast<float4*>(row + (64 ^ swl)) = make_float4(y[0], y[1], go0, go1);
    float gz2[UDE_H];
#pragma unroll
    for (int j = 0; j < UDE_H; ++j) {
      const float gh = fmaf(w[UDE_W3 + j], go0, w[UDE_W3 + UDE_H + j] * go1);
      gz2[j] = gh * fmaf(-h2[j], h2[j], 1.0f);
    }
#pragma unroll
    for (int j = 0; j < UDE_H; j += 4)
      *reinterpret_cast<float4*>(row + (j ^ swl)) = make_float4(gz2[j], gz2[j + 1], gz2[j + 2], gz2[j + 3]);
    float gh1[UDE_H];
    UdeTc::product(gz2, 1, gh1);  // GH1 = GZ2 W2
    float gx = 0.0f, gy = 0.0f;
#pragma unroll
    for (int j = 0; j < UDE_H; j += 4) {
      const float4 hv = *reinterpret_cast<const float4*>(row + ((16 + j) ^ swl));
      const float h1[4] = {hv.x, hv.y, hv.z, hv.w};
      float z[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        z[u] = gh1[j + u] * fmaf(-h1[u], h1[u], 1.0f);
        gx = fmaf(w[UDE_W1 + 2 * (j + u)], z[u], gx);
        gy = fmaf(w[UDE_W1 + 2 * (j + u) + 1], z[u], gy);
      }
      *reinterpret_cast<float4*>(row + ((32 + j) ^ swl)) = make_float4(z[0], z[1], z[2], z[3]);
    }
    yb[0] = fmaf(p[0], v[0], gx);
    yb[1] = fmaf(-p[1], v[1], gy);
    pb[0] = fmaf(y[0], v[0], pb[0]);
    pb[1] = fmaf(-y[1], v[1], pb[1]);
  }
};

// Accumulator of the UDE reverse sweep: the per-trajectory (a, d) gradient
// (compensated FP32, per lane) and the warp's shared-weight gradient in MMA
// accumulator fragments:
//   GA (16 x 24): sum over lanes of gz2 (x) [h1, 1]   -> dW2, db2
//   GB (16 x 8):  sum over lanes of gz1 (x) [x, y, 1]  -> dW1, db1
//   GC (32 x 8):  sum over lanes of [h2, 1] (x) go     -> dW3, db3
struct UdeAcc {
  using Part = float;
  static constexpr int NW = UDE_NW;
  CompensatedAcc<2> th;
  float ga[3][4], gb[4], gc[2][4];
  __device__ void init(double*) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      ga[0][i] = ga[1][i] = ga[2][i] = 0.0f;
      gb[i] = 0.0f;
      gc[0][i] = gc[1][i] = 0.0f;
    }
  }
  __device__ void zero() { th.zero(); }
  __device__ double get(int q) const { return th.get(q); }

  // Warp-collective: every lane of the warp calls it (lanes without work pass
  // v = 0, so their factors contribute exactly zero).
  template <class Pb>
  __device__ __forceinline__ void vjp(const float (&y)[2], const float (&p)[2], const float (&v)[2],
                                      float (&yb)[2]) {
    static_assert(std::is_same<Pb, LvUdeWarp>::value || std::is_same<Pb, LvUdeCta>::value,
                  "the UDE reverse sweep uses a collective form of the network");
    float x[2] = {0.0f, 0.0f};
    if constexpr (std::is_same<Pb, LvUdeCta>::value)
      LvUdeCta::backprop_cta(y, p, v, yb, x);  // leaves the factor rows staged
    else
      LvUdeWarp::backprop_warp(y, p, v, yb, x);
#pragma unroll
    for (int q = 0; q < 2; ++q) th.u[q] = add_(th.u[q], x[q]);
    accumulate();
  }
  __device__ __forceinline__ void flush() { th.flush(); }

  // The weight-gradient MMAs over the warp's staged factor rows.
  __device__ __forceinline__ void accumulate() {
    const float* st = ude_stage();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    __syncwarp();
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {  // contraction over lanes, 8 at a time
      const float* r0 = st + (ks * 8 + t) * UDE_ROW;      // rows with bit 2 clear: columns as stored
      const float* r1 = st + (ks * 8 + t + 4) * UDE_ROW;  // rows with bit 2 set: column c at c ^ 4
      // GA: A[i][k] = gz2_k[i], B[k][j] = (h1_k, 1, 0...)[j]
      {
        const Tf32x2 a[4] = {split_tf32(r0[g]), split_tf32(r0[g + 8]), split_tf32(r1[g ^ 4]),
                             split_tf32(r1[(g + 8) ^ 4])};
#pragma unroll
        for (int nt = 0; nt < 3; ++nt) {
          const int j = nt * 8 + g;
          const float b0 = j < 16 ? r0[16 + j] : (j == 16 ? 1.0f : 0.0f);
          const float b1 = j < 16 ? r1[(16 + j) ^ 4] : (j == 16 ? 1.0f : 0.0f);
          const Tf32x2 b[2] = {split_tf32(b0), split_tf32(b1)};
          mma_3xtf32(ga[nt], a, b);
        }
      }
      // GB: A[i][k] = gz1_k[i], B[k][j] = (x_k, y_k, 1, 0...)[j]
      {
        const Tf32x2 a[4] = {split_tf32(r0[32 + g]), split_tf32(r0[40 + g]), split_tf32(r1[(32 + g) ^ 4]),
                             split_tf32(r1[(40 + g) ^ 4])};
        const float b0 = g < 2 ? r0[64 + g] : (g == 2 ? 1.0f : 0.0f);
        const float b1 = g < 2 ? r1[(64 + g) ^ 4] : (g == 2 ? 1.0f : 0.0f);
        const Tf32x2 b[2] = {split_tf32(b0), split_tf32(b1)};
        mma_3xtf32(gb, a, b);
      }
      // GC: A[i][k] = (h2_k, 1, 0...)[i] over two row tiles, B[k][o] = go_k[o]
      {
        const float b0 = g < 2 ? r0[66 + g] : 0.0f;
        const float b1 = g < 2 ? r1[(66 + g) ^ 4] : 0.0f;
        const Tf32x2 b[2] = {split_tf32(b0), split_tf32(b1)};
        const Tf32x2 a0[4] = {split_tf32(r0[48 + g]), split_tf32(r0[56 + g]), split_tf32(r1[(48 + g) ^ 4]),
                              split_tf32(r1[(56 + g) ^ 4])};
        mma_3xtf32(gc[0], a0, b);
        const float one = (g == 0) ? 1.0f : 0.0f;  // row 16 of GC: the bias db3
        const Tf32x2 a1[4] = {split_tf32(one), split_tf32(0.0f), split_tf32(one), split_tf32(0.0f)};
        mma_3xtf32(gc[1], a1, b);
      }
    }
  }

  // Writes this warp's partial weight gradient (354 floats, the flat layout).
  __device__ void finish(void* part_base, size_t warp) {
    float* part = static_cast<float*>(part_base) + warp * UDE_NW;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // C fragment element (row, col): c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = g + ((e & 2) ? 8 : 0), cc = 2 * t + (e & 1);
#pragma unroll
      for (int nt = 0; nt < 3; ++nt) {  // GA: row r = hidden-2 unit, col j = hidden-1 unit / bias
        const int j = nt * 8 + cc;
        if (j < 16) part[UDE_W2 + UDE_H * r + j] = ga[nt][e];
        else if (j == 16) part[UDE_B2 + r] = ga[nt][e];
      }
      if (cc < 2) part[UDE_W1 + 2 * r + cc] = gb[e];  // GB: dW1[r][cc]
      else if (cc == 2) part[UDE_B1 + r] = gb[e];
      if (cc < 2) part[UDE_W3 + UDE_H * cc + r] = gc[0][e];  // GC tile 0: dW3[o][j] at (j = r, o = cc)
      if (cc < 2 && r == 0) part[UDE_B3 + cc] = gc[1][e];    // GC tile 1 row 16: db3[o]
    }
  }
};

// Adds the per-warp partial weight gradients (nw per warp) in warp order, in
// FP64, and writes the FP32 result.
template <class Part>
__global__ void weight_reduce_kernel(const Part* part, int nw, int nwarps, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nw) return;
  double s = 0.0;
  for (int w = 0; w < nwarps; ++w) s += (double)part[(size_t)w * nw + i];
  out[i] = (float)s;
}

}  // namespace gs
