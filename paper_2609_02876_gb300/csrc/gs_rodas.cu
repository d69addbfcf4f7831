// Rodas5P (stiff) instantiations of the record and reverse-sweep kernels:
// Robertson, HIRES, the linear test problem and the neural Robertson, FP64 (the W-matrix LU and its
// solves are FP64 in every precision mode).
#include "gs_kernels.cuh"

namespace gs {

bool rodas_supports(int problem, int precision) {
  return (problem == 2 || problem == 3 || problem == 4 || problem == 6) && precision == 0;
}

cudaError_t launch_rodas_forward(int problem, int precision, const FwdArgs& a, cudaStream_t s) {
  if (precision != 0) return cudaErrorInvalidValue;
  switch (problem) {
    case 2: return fwd_dispatch<Rodas5PMethod, Robertson, double>(a, s);
    case 3: return fwd_dispatch<Rodas5PMethod, Hires, double>(a, s);
    case 4: return fwd_dispatch<Rodas5PMethod, Linear2, double>(a, s);
    case 6: return fwd_dispatch<Rodas5PMethod, NeuralRobertson, double>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_rodas_reverse(int problem, int precision, const RevArgs& a, cudaStream_t s) {
  if (precision != 0) return cudaErrorInvalidValue;
  switch (problem) {
    case 2: return rev_dispatch<Rodas5PMethod, Robertson, double>(a, s);
    case 3: return rev_dispatch<Rodas5PMethod, Hires, double>(a, s);
    case 4: return rev_dispatch<Rodas5PMethod, Linear2, double>(a, s);
    case 6: return rev_dispatch<Rodas5PMethod, NeuralRobertson, double>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_rodas_refresh(int problem, int precision, const RevArgs& a, double* arena, double* y_final,
                                 const double* y0, cudaStream_t s) {
  if (precision != 0) return cudaErrorInvalidValue;
  switch (problem) {
    case 2: return refresh_dispatch<Rodas5PMethod, Robertson, double>(a, arena, y_final, y0, s);
    case 3: return refresh_dispatch<Rodas5PMethod, Hires, double>(a, arena, y_final, y0, s);
    case 4: return refresh_dispatch<Rodas5PMethod, Linear2, double>(a, arena, y_final, y0, s);
    case 6: return refresh_dispatch<Rodas5PMethod, NeuralRobertson, double>(a, arena, y_final, y0, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gs
