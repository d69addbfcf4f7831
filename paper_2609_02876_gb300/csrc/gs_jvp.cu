// Forward-mode (tangent) replay over a recorded mesh: paper Sec. 5, forward
// mode for few inputs. Each trajectory's replay chain y_i = Phi(y_{i-1}; h_i,
// theta) is re-run from y0 over its recorded step sizes (held as data) and
// carries ND tangent directions (yd, pd) alongside: yd_i = dPhi/dy yd_{i-1} +
// dPhi/dtheta pd. The save-time states are the side steps of the record, and
// the built-in loss L = sum_s ||y(t_s)||^2 gets its directional derivative
// dL = sum_s 2 y(t_s) . yd(t_s). A pass changes the same input of every
// trajectory at once, so the number of passes is set by the inputs of one
// trajectory, not by the ensemble size. FP64 only.
//
// Scheduling follows the record kernel: one lane per trajectory, a warp-
// aggregated ticket refill when a trajectory ends, and one convergent tangent
// step per loop iteration for every lane that has a step or a side step to do.
// The record links its segments last to first; a separate index kernel lists
// them in forward order once per record, so that no lane of the compute
// kernel stalls its warp on a chain of dependent loads.
#include "gs_kernels.cuh"

namespace gs {
namespace {

// One thread per trajectory walks its chain from the last segment back to the
// first and writes the indices in forward order. Latency-bound: launched with
// as many resident threads as fit, so the dependent loads of many chains overlap.
__global__ void __launch_bounds__(256) fwd_index_kernel(int64_t n, const long long* head, const int32_t* S,
                                                        const int32_t* status, const double* arena,
                                                        long long arena_cap, int k, int segw,
                                                        unsigned long long* top, long long* fwd_base,
                                                        long long* fwd_seg, long long cap) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long hd = head[t];
    if (status[t] != TRAJ_OK || hd < 0) {
      fwd_base[t] = -1;
      continue;
    }
    const long long nseg = (S[t] + k - 1) / k;
    const long long b = (long long)atomicAdd(top, (unsigned long long)nseg);
    bool ok = (b + nseg <= cap);
    long long seg = hd;
    for (long long q = nseg - 1; q >= 0 && ok; --q) {
      if (seg < 0 || seg >= arena_cap) {
        ok = false;
        break;
      }
      fwd_seg[b + q] = seg;
      seg = __double_as_longlong(arena[seg * segw]);
    }
    fwd_base[t] = (ok && seg < 0) ? b : -1;  // the first segment links to -1
  }
}

enum { J_NONE = 0, J_STEP, J_SIDE, J_DONE, J_FAIL };

struct Tsit5Tangent {
  template <class Pb, int ND>
  __device__ __forceinline__ static bool step(const double (&y)[Pb::D], const double (&yd)[ND][Pb::D],
                                              const double (&p)[Pb::NP], const double (&pd)[ND][Pb::NP], double h,
                                              double (&yn)[Pb::D], double (&ydn)[ND][Pb::D]) {
    tsit5_tangent<Pb, ND>(y, yd, p, pd, h, yn, ydn);
    return true;
  }
};

struct RodasTangent {
  template <class Pb, int ND>
  __device__ __forceinline__ static bool step(const double (&y)[Pb::D], const double (&yd)[ND][Pb::D],
                                              const double (&p)[Pb::NP], const double (&pd)[ND][Pb::NP], double h,
                                              double (&yn)[Pb::D], double (&ydn)[ND][Pb::D]) {
    return rodas_tangent<Pb, ND>(y, yd, p, pd, h, yn, ydn);
  }
};

struct Ros23Tangent {
  template <class Pb, int ND>
  __device__ __forceinline__ static bool step(const double (&y)[Pb::D], const double (&yd)[ND][Pb::D],
                                              const double (&p)[Pb::NP], const double (&pd)[ND][Pb::NP], double h,
                                              double (&yn)[Pb::D], double (&ydn)[ND][Pb::D]) {
    return ros23_tangent<Pb, ND>(y, yd, p, pd, h, yn, ydn);
  }
};

struct Vern7Tangent {
  template <class Pb, int ND>
  __device__ __forceinline__ static bool step(const double (&y)[Pb::D], const double (&yd)[ND][Pb::D],
                                              const double (&p)[Pb::NP], const double (&pd)[ND][Pb::NP], double h,
                                              double (&yn)[Pb::D], double (&ydn)[ND][Pb::D]) {
    vern7_tangent<Pb, ND>(y, yd, p, pd, h, yn, ydn);
    return true;
  }
};

// Outputs of trajectory k: the loss and, per direction, its derivative (into
// loss_dot, or in basis mode into the gradient row of that input).
template <int NP, int ND>
__device__ __forceinline__ void jvp_write(const JvpArgs& a, long long k, double loss, const double (&ldot)[ND]) {
  const long long n = a.n;
  if (a.loss) a.loss[k] = loss;
#pragma unroll
  for (int q = 0; q < ND; ++q) {
    if (a.basis) {
      const int g = a.dir0 + q;
      if (g < NP) {
        if (a.grad_p) a.grad_p[g * n + k] = ldot[q];
      } else if (a.grad_y) {
        a.grad_y[(g - NP) * n + k] = ldot[q];
      }
    } else if (a.loss_dot) {
      a.loss_dot[q * n + k] = ldot[q];
    }
  }
}

template <int D, int NP, int ND>
__device__ __forceinline__ void jvp_fail(const JvpArgs& a, long long k) {
  double nn[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) nn[q] = nan_d();
  jvp_write<NP, ND>(a, k, nan_d(), nn);
  if (!a.basis && a.y_save_dot)
    for (int s = 0; s < a.n_save; ++s)
#pragma unroll
      for (int q = 0; q < ND; ++q)
#pragma unroll
        for (int c = 0; c < D; ++c) a.y_save_dot[(((long long)q * a.n_save + s) * D + c) * a.n + k] = nan_d();
}

// The state and tangents at save time js enter the loss and its derivatives.
template <int D, int ND>
__device__ __forceinline__ void jvp_save(const JvpArgs& a, long long k, int js, const double (&ys)[D],
                                         const double (&yds)[ND][D], double& loss, double (&ldot)[ND]) {
#pragma unroll
  for (int c = 0; c < D; ++c) loss = add_(loss, mul_(ys[c], ys[c]));
#pragma unroll
  for (int q = 0; q < ND; ++q)
#pragma unroll
    for (int c = 0; c < D; ++c) ldot[q] = fma_(add_(ys[c], ys[c]), yds[q][c], ldot[q]);
  if (!a.basis && a.y_save_dot) {
#pragma unroll
    for (int q = 0; q < ND; ++q)
#pragma unroll
      for (int c = 0; c < D; ++c) a.y_save_dot[(((long long)q * a.n_save + js) * D + c) * a.n + k] = yds[q][c];
  }
}

template <class T, class Pb, int ND>
__global__ void __launch_bounds__(TPB_REV) jvp_kernel(const JvpArgs a) {
  constexpr int D = Pb::D, NP = Pb::NP;
  extern __shared__ double smem[];
  const int ns = a.n_save;
  double* s_save = smem;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) s_save[i] = a.save_t[i];
  __syncthreads();

  const long long n = a.n;
  long long k = -1, cur = -1, fb = 0;
  bool drained = false;
  double y[D], yd[ND][D], p[NP], pd[ND][NP], ldot[ND];
  double t = 0.0, tn = 0.0, loss = 0.0;
  int S = 0, nseg = 0, pos = -1, j = 0, m = 0, i = 0, js = 0;

  for (;;) {
    // ---- refill: lanes without a trajectory take the next ticket
    const bool need = (k < 0) && !drained;
    if (__any_sync(FULL_MASK, need)) {
      const long long got = warp_ticket(a.work, need);
      if (need) {
        if (got < n) {
          k = got;
          fb = a.fwd_base[k];
          if (a.status[k] != TRAJ_OK || fb < 0) {
            jvp_fail<D, NP, ND>(a, k);
            k = -1;  // take another ticket next iteration
          } else {
#pragma unroll
            for (int r = 0; r < NP; ++r) p[r] = a.params[r * n + k];
#pragma unroll
            for (int c = 0; c < D; ++c) y[c] = a.y0[c * n + k];
#pragma unroll
            for (int q = 0; q < ND; ++q) {
              const int g = a.dir0 + q;
#pragma unroll
              for (int r = 0; r < NP; ++r)
                pd[q][r] = a.basis ? (g == r ? 1.0 : 0.0)
                                   : (a.params_dot ? a.params_dot[((long long)q * NP + r) * n + k] : 0.0);
#pragma unroll
              for (int c = 0; c < D; ++c)
                yd[q][c] = a.basis ? (g == NP + c ? 1.0 : 0.0)
                                   : (a.y0_dot ? a.y0_dot[((long long)q * D + c) * n + k] : 0.0);
              ldot[q] = 0.0;
            }
            t = a.t0;
            loss = 0.0;
            S = a.S[k];
            nseg = (S + a.k - 1) / a.k;
            pos = -1;
            j = m = 0;
            i = 0;
            js = 0;
          }
        } else {
          drained = true;
        }
      }
    }
    if (!__any_sync(FULL_MASK, k >= 0 || !drained)) break;

    // ---- this lane's next unit
    int mode = J_NONE;
    double uh = 0.0;
    if (k >= 0) {
      for (;;) {
        double hi = 0.0;
        if (i < S) {  // the step out of mesh point i and the next mesh time
          if (j == m) {  // next segment (pos < nseg while i < S; indices checked by the index kernel)
            ++pos;
            cur = a.fwd_seg[fb + pos];
            m = (pos == nseg - 1) ? S - (nseg - 1) * a.k : a.k;
            j = 0;
          }
          hi = a.arena[cur * a.segw + 2 + D + j];
          tn = (i + 1 == S) ? a.t1 : add_(t, hi);
        }
        // saves attached to mesh point i: t_i <= t_s < t_{i+1} (every remaining one at i = S)
        if (js < ns && (i == S || dkey(s_save[js]) < dkey(tn))) {
          if (same_time(s_save[js], t)) {
            jvp_save<D, ND>(a, k, js, y, yd, loss, ldot);
            ++js;
            continue;
          }
          mode = J_SIDE;
          uh = s_save[js] - t;
          break;
        }
        mode = (i == S) ? J_DONE : J_STEP;
        uh = hi;
        break;
      }
    }

    // ---- one tangent step for every lane with a step or a side step. The
    // mode is made opaque to the optimiser, so that steps and side steps share
    // one copy of the unit and the warp runs it once with all its busy lanes.
    __syncwarp();
    asm volatile("" : "+r"(mode));
    if (mode == J_STEP || mode == J_SIDE) {
      double yn[D], ydn[ND][D];
      const bool ok = T::template step<Pb, ND>(y, yd, p, pd, uh, yn, ydn);
      if (!ok) {
        mode = J_FAIL;
      } else if (mode == J_STEP) {
#pragma unroll
        for (int c = 0; c < D; ++c) y[c] = yn[c];
#pragma unroll
        for (int q = 0; q < ND; ++q)
#pragma unroll
          for (int c = 0; c < D; ++c) yd[q][c] = ydn[q][c];
        t = tn;
        ++i;
        ++j;
      } else {
        jvp_save<D, ND>(a, k, js, yn, ydn, loss, ldot);
        ++js;
      }
    }
    if (mode == J_DONE) {
      jvp_write<NP, ND>(a, k, loss, ldot);
      k = -1;
    } else if (mode == J_FAIL) {
      jvp_fail<D, NP, ND>(a, k);
      k = -1;
    }
  }
}

template <class T, class Pb>
cudaError_t jvp_dispatch(const JvpArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)((a.n_save + 1) & ~1) * sizeof(double);
  switch (a.nd) {
    case 1: return persistent_launch(jvp_kernel<T, Pb, 1>, TPB_REV, smem, a.n, s, &a);
    case 2: return persistent_launch(jvp_kernel<T, Pb, 2>, TPB_REV, smem, a.n, s, &a);
    case 3: return persistent_launch(jvp_kernel<T, Pb, 3>, TPB_REV, smem, a.n, s, &a);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fwd_index(int64_t n, const long long* head, const int32_t* S, const int32_t* status,
                             const double* arena, long long arena_cap, int k, int segw, unsigned long long* top,
                             long long* fwd_base, long long* fwd_seg, long long cap, cudaStream_t s) {
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fwd_index_kernel, 256, 0);
  long long blocks = (long long)sm_count() * (bps > 0 ? bps : 1);
  const long long need = (n + 255) / 256;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  fwd_index_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, head, S, status, arena, arena_cap, k, segw, top, fwd_base,
                                                     fwd_seg, cap);
  return cudaGetLastError();
}

bool jvp_supports(int method, int problem) {
  if (method == 1 || method == 4) return problem == 0 || problem == 1 || problem == 4;  // Lorenz, VdP, linear
  if (method == 2 || method == 3) return problem == 2 || problem == 3 || problem == 4;  // Robertson, HIRES, linear
  return false;
}

cudaError_t launch_jvp(int method, int problem, const JvpArgs& a, cudaStream_t s) {
  if (method == 1) {
    switch (problem) {
      case 0: return jvp_dispatch<Tsit5Tangent, Lorenz>(a, s);
      case 1: return jvp_dispatch<Tsit5Tangent, VanDerPol>(a, s);
      case 4: return jvp_dispatch<Tsit5Tangent, Linear2>(a, s);
    }
  } else if (method == 2) {
    switch (problem) {
      case 2: return jvp_dispatch<RodasTangent, Robertson>(a, s);
      case 3: return jvp_dispatch<RodasTangent, Hires>(a, s);
      case 4: return jvp_dispatch<RodasTangent, Linear2>(a, s);
    }
  } else if (method == 3) {
    switch (problem) {
      case 2: return jvp_dispatch<Ros23Tangent, Robertson>(a, s);
      case 3: return jvp_dispatch<Ros23Tangent, Hires>(a, s);
      case 4: return jvp_dispatch<Ros23Tangent, Linear2>(a, s);
    }
  } else if (method == 4) {
    switch (problem) {
      case 0: return jvp_dispatch<Vern7Tangent, Lorenz>(a, s);
      case 1: return jvp_dispatch<Vern7Tangent, VanDerPol>(a, s);
      case 4: return jvp_dispatch<Vern7Tangent, Linear2>(a, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace gs
