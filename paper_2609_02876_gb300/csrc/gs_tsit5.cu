// Tsit5 (non-stiff) instantiations of the record and reverse-sweep kernels:
// Lorenz, Van der Pol and the linear test problem, FP64 and FP32-mixed.
#include "gs_kernels.cuh"

// The LV UDE reverse sweep's network: 0 (default) the warp-collective form
// (LvUdeWarp, mma.sync), 1 the CTA-collective form with the hidden layer on
// tcgen05 (LvUdeCta). Both give the same gradients to FP32 rounding (the UDE
// parity tests pass with either); measured at 2^18 trajectories the CTA form's
// reverse sweep takes 45.9 ms against 15.7 ms, because its four warps must meet
// at a CTA barrier and a tensor-memory round trip for each of the ~18
// hidden-layer products of a unit.
#ifndef GS_UDE_CTA
#define GS_UDE_CTA 0
#endif

namespace gs {

bool tsit5_supports(int problem, int precision) {
  if (problem == 5) return precision == 1;  // LV UDE: FP32 network and state, FP64 control
  return (problem == 0 || problem == 1 || problem == 4) && (precision == 0 || precision == 1);
}

cudaError_t launch_tsit5_forward(int problem, int precision, const FwdArgs& a, cudaStream_t s) {
  switch (problem * 2 + precision) {
    case 0: return fwd_dispatch<Tsit5Method, Lorenz, double>(a, s);
    case 1: return fwd_dispatch<Tsit5Method, Lorenz, float>(a, s);
    case 2: return fwd_dispatch<Tsit5Method, VanDerPol, double>(a, s);
    case 3: return fwd_dispatch<Tsit5Method, VanDerPol, float>(a, s);
    case 8: return fwd_dispatch<Tsit5Method, Linear2, double>(a, s);
    case 9: return fwd_dispatch<Tsit5Method, Linear2, float>(a, s);
    case 11: return fwd_dispatch<Tsit5Method, LvUde, float>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tsit5_reverse(int problem, int precision, const RevArgs& a, cudaStream_t s) {
  switch (problem * 2 + precision) {
    case 0: return rev_dispatch<Tsit5Method, Lorenz, double>(a, s);
    case 1: return rev_dispatch<Tsit5Method, Lorenz, float>(a, s);
    case 2: return rev_dispatch<Tsit5Method, VanDerPol, double>(a, s);
    case 3: return rev_dispatch<Tsit5Method, VanDerPol, float>(a, s);
    case 8: return rev_dispatch<Tsit5Method, Linear2, double>(a, s);
    case 9: return rev_dispatch<Tsit5Method, Linear2, float>(a, s);
#if GS_UDE_CTA
    case 11: return rev_dispatch<Tsit5Method, LvUdeCta, float>(a, s);  // CTA-collective network (tcgen05)
#else
    case 11: return rev_dispatch<Tsit5Method, LvUdeWarp, float>(a, s);  // warp-collective network (mma.sync)
#endif
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tsit5_refresh(int problem, int precision, const RevArgs& a, double* arena, double* y_final,
                                 const double* y0, cudaStream_t s) {
  switch (problem * 2 + precision) {
    case 0: return refresh_dispatch<Tsit5Method, Lorenz, double>(a, arena, y_final, y0, s);
    case 1: return refresh_dispatch<Tsit5Method, Lorenz, float>(a, arena, y_final, y0, s);
    case 2: return refresh_dispatch<Tsit5Method, VanDerPol, double>(a, arena, y_final, y0, s);
    case 3: return refresh_dispatch<Tsit5Method, VanDerPol, float>(a, arena, y_final, y0, s);
    case 8: return refresh_dispatch<Tsit5Method, Linear2, double>(a, arena, y_final, y0, s);
    case 9: return refresh_dispatch<Tsit5Method, Linear2, float>(a, arena, y_final, y0, s);
    case 11: return refresh_dispatch<Tsit5Method, LvUde, float>(a, arena, y_final, y0, s);
  }
  return cudaErrorInvalidValue;
}

int ude_max_warps() {
  int dev = 0, sms = 0, threads = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  return (sms > 0 ? sms : 1) * (threads > 0 ? threads : 2048) / 32;
}

}  // namespace gs
