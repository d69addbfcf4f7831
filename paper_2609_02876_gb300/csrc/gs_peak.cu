// gs_measure_fma_peak: the FMA throughput of the current device's FP64 and
// FP32 pipes, the denominators of the ALU roofline fractions that the
// benchmark reports for the record and reverse kernels.
//
// A grid of full occupancy (8 CTAs of 256 threads per SM) runs CHAINS
// independent fused multiply-add recurrences per thread, x <- x a + b with
// |a| < 1, so that every FMA of a thread has CHAINS - 1 others in flight
// between it and its operand. An FMA counts two flops. The iteration count is
// scaled from a short first launch so that a timed launch takes ~40 ms; the
// figure is the best of five launches timed with CUDA events.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/gs.h"

namespace {

constexpr int CHAINS = 8;
constexpr int TPB = 256;
constexpr int CTAS_PER_SM = 8;

template <class T>
__global__ void __launch_bounds__(TPB) fma_chains(T* out, long long iters, T a, T b) {
  T x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = T(threadIdx.x & 7) + T(c);
#pragma unroll 8
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  if (s == T(-1.25)) out[blockIdx.x] = s;  // never true; keeps the chains live
}

// Packed FP32x2 FMA (one instruction, two IEEE single FMAs).
__global__ void __launch_bounds__(TPB) fma2_chains(float* out, long long iters, float a, float b) {
  float2 x[CHAINS];
  const float2 av = make_float2(a, a), bv = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = make_float2(float(threadIdx.x & 7) + c, float(c) - 3.0f);
#pragma unroll 8
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = __ffma2_rn(x[c], av, bv);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c].x + x[c].y;
  if (s == -1.25f) out[blockIdx.x] = s;
}

// Launches `kind` once with `iters` iterations; returns its device time in ms (< 0 on error).
float timed_launch(int kind, int blocks, long long iters, void* out, cudaEvent_t e0, cudaEvent_t e1) {
  cudaEventRecord(e0, 0);
  if (kind == 0)
    fma_chains<double><<<blocks, TPB>>>(static_cast<double*>(out), iters, 1.0 - 0x1p-20, 0x1p-30);
  else if (kind == 1)
    fma_chains<float><<<blocks, TPB>>>(static_cast<float*>(out), iters, 1.0f - 0x1p-12f, 0x1p-20f);
  else
    fma2_chains<<<blocks, TPB>>>(static_cast<float*>(out), iters, 1.0f - 0x1p-12f, 0x1p-20f);
  cudaEventRecord(e1, 0);
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

}  // namespace

extern "C" gs_status gs_measure_fma_peak(int kind, double* tflops) {
  if (!tflops || kind < 0 || kind > 2) return GS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return GS_ERR_CUDA;
  const int blocks = sms * CTAS_PER_SM;
  void* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * sizeof(double)) != cudaSuccess) return GS_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  gs_status st = GS_OK;
  long long iters = kind == 0 ? 1024 : 16384;
  float ms = timed_launch(kind, blocks, iters, out, e0, e1);  // warm-up and scale
  if (ms <= 0.0f) {
    st = GS_ERR_CUDA;
  } else {
    iters = std::max(1024LL, (long long)(iters * (40.0 / ms)));
    double best = 0.0;
    for (int rep = 0; rep < 5 && st == GS_OK; ++rep) {
      ms = timed_launch(kind, blocks, iters, out, e0, e1);
      if (ms <= 0.0f) {
        st = GS_ERR_CUDA;
        break;
      }
      const double lanes = kind == 2 ? 2.0 : 1.0;  // FMAs per instruction
      const double flops = 2.0 * lanes * CHAINS * (double)iters * blocks * TPB;
      best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    *tflops = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return st;
}
