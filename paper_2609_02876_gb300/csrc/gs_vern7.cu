// Verner7 (seventh-order explicit pair) instantiations of the record,
// reverse-sweep and refresh kernels: Lorenz, Van der Pol and the linear test
// problem, FP64.
#include "gs_kernels.cuh"

namespace gs {

bool vern7_supports(int problem, int precision) {
  return (problem == 0 || problem == 1 || problem == 4) && precision == 0;
}

cudaError_t launch_vern7_forward(int problem, int precision, const FwdArgs& a, cudaStream_t s) {
  if (precision != 0) return cudaErrorInvalidValue;
  switch (problem) {
    case 0: return fwd_dispatch<Verner7Method, Lorenz, double>(a, s);
    case 1: return fwd_dispatch<Verner7Method, VanDerPol, double>(a, s);
    case 4: return fwd_dispatch<Verner7Method, Linear2, double>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_vern7_reverse(int problem, int precision, const RevArgs& a, cudaStream_t s) {
  if (precision != 0) return cudaErrorInvalidValue;
  switch (problem) {
    case 0: return rev_dispatch<Verner7Method, Lorenz, double>(a, s);
    case 1: return rev_dispatch<Verner7Method, VanDerPol, double>(a, s);
    case 4: return rev_dispatch<Verner7Method, Linear2, double>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_vern7_refresh(int problem, int precision, const RevArgs& a, double* arena, double* y_final,
                                 const double* y0, cudaStream_t s) {
  if (precision != 0) return cudaErrorInvalidValue;
  switch (problem) {
    case 0: return refresh_dispatch<Verner7Method, Lorenz, double>(a, arena, y_final, y0, s);
    case 1: return refresh_dispatch<Verner7Method, VanDerPol, double>(a, arena, y_final, y0, s);
    case 4: return refresh_dispatch<Verner7Method, Linear2, double>(a, arena, y_final, y0, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gs
