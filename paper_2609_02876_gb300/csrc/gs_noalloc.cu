// gs_solve_grad_noalloc: gs_solve_grad without any device allocation.
//
// The record of the ensemble (the accepted-step segments, the per-trajectory
// bookkeeping and the kernels' counters) lives in one file-scope device array
// of GS_NOALLOC_SCRATCH_BYTES that the library declares itself; every GPU that
// loads the library holds it until the process exits. Host code cannot use
// the array's name as a device address, so the address is resolved once per
// device with cudaGetSymbolAddress (on the first call made with that device
// current) and passed to the kernels as a plain pointer.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/gs.h"
#include "gs_internal.h"

using namespace gs;

static __device__ __align__(256) unsigned char g_noalloc_scratch[GS_NOALLOC_SCRATCH_BYTES];

namespace {

struct ScratchCounters {
  unsigned long long work_fwd;
  unsigned long long work_rev;
  unsigned long long arena_top;
  int overflow;
  int any_failed;
};

constexpr int kMaxDevices = 64;
constexpr int kMaxD = 8;
std::mutex g_addr_mu;
unsigned char* g_addr[kMaxDevices] = {nullptr};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch on the current device (resolved once per device).
gs_status scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return GS_ERR_CUDA;
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return GS_OK;
}

}  // namespace

extern "C" gs_status gs_solve_grad_noalloc(int problem_id, int64_t n, const double* params, const double* y0,
                                           const float* shared_w, double t0, double t1, const double* save_t,
                                           int n_save, double rtol, double atol, const gs_options* opt,
                                           gs_stream stream, double* loss_out, double* params_bar, double* y0_bar,
                                           float* shared_w_bar, int32_t* traj_status) {
  (void)shared_w_bar;
  int d = 0, P = 0, stiff = 0, n_shared = 0;
  if (gs_problem_info(problem_id, &d, &P, &stiff, &n_shared) != GS_OK) return GS_ERR_UNKNOWN_PROBLEM;
  if (n < 0 || n > GS_NOALLOC_MAX_TRAJ) return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  if (!params || !y0 || !traj_status) return GS_ERR_INVALID_ARG;
  // Shared-weight problems need the reverse sweep's per-warp weight partials,
  // which live outside the fixed array, and a k = 1 record: not offered here.
  if (n_shared > 0) return GS_ERR_INVALID_ARG;
  if (!std::isfinite(t0) || !std::isfinite(t1) || !(t1 > t0)) return GS_ERR_INVALID_ARG;
  if (n_save < 0 || n_save > MAX_SAVE_HOST || (n_save > 0 && !save_t)) return GS_ERR_INVALID_ARG;
  for (int s = 0; s < n_save; ++s) {
    if (!std::isfinite(save_t[s]) || !(save_t[s] > t0) || save_t[s] > t1) return GS_ERR_INVALID_ARG;
    if (s > 0 && !(save_t[s] > save_t[s - 1])) return GS_ERR_INVALID_ARG;
  }
  if (!std::isfinite(rtol) || !std::isfinite(atol) || rtol < 0 || atol < 0 || (rtol == 0 && atol == 0))
    return GS_ERR_INVALID_ARG;
  gs_options o;
  gs_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != GS_FP64 && o.precision != GS_FP32_MIXED) return GS_ERR_INVALID_ARG;
  if (o.control != GS_CONTROL_FAST) return GS_ERR_INVALID_ARG;  // the default step control only
  const int method = o.method == GS_METHOD_AUTO ? (stiff ? GS_METHOD_RODAS5P : GS_METHOD_TSIT5) : o.method;
  if (method != GS_METHOD_TSIT5 || !tsit5_supports(problem_id, o.precision)) return GS_ERR_INVALID_ARG;
  if (o.ckpt_k < 0 || o.ckpt_k > KMAX_HOST || o.max_steps < 0 || !std::isfinite(o.h0) || o.h0 < 0)
    return GS_ERR_INVALID_ARG;
  if (d > kMaxD) return GS_ERR_INVALID_ARG;

  unsigned char* base = nullptr;
  gs_status st = scratch_address(&base);
  if (st != GS_OK) return st;

  // Carve the scratch: counters | head | S | attempts | status | y(t1) | arena.
  const int k = o.ckpt_k > 0 ? o.ckpt_k : (14 - d > 1 ? 14 - d : 1);
  const int segw = segw_of(d, k);
  const size_t N = (size_t)GS_NOALLOC_MAX_TRAJ;
  size_t off = 0;
  ScratchCounters* ctr = reinterpret_cast<ScratchCounters*>(base + off);
  off = align256(off + sizeof(ScratchCounters));
  long long* head = reinterpret_cast<long long*>(base + off);
  off = align256(off + N * sizeof(long long));
  int32_t* S = reinterpret_cast<int32_t*>(base + off);
  off = align256(off + N * sizeof(int32_t));
  int32_t* natt = reinterpret_cast<int32_t*>(base + off);
  off = align256(off + N * sizeof(int32_t));
  int32_t* status = reinterpret_cast<int32_t*>(base + off);
  off = align256(off + N * sizeof(int32_t));
  double* y_final = reinterpret_cast<double*>(base + off);
  off = align256(off + N * kMaxD * sizeof(double));
  double* arena = reinterpret_cast<double*>(base + off);
  const long long arena_cap = (long long)((GS_NOALLOC_SCRATCH_BYTES - off) / (segw * sizeof(double)));

  cudaStream_t s = (cudaStream_t)stream;
  // The counters must start at zero; everything else is written before it is read.
  if (cudaMemsetAsync(ctr, 0, sizeof(ScratchCounters), s) != cudaSuccess) return GS_ERR_CUDA;

  FwdArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.params = params;
  a.y0 = y0;
  a.shared_w = shared_w;
  a.t0 = t0;
  a.t1 = t1;
  a.rtol = rtol;
  a.atol = atol;
  a.h0 = o.h0;
  a.max_steps = o.max_steps > 0 ? o.max_steps : 1000000;
  a.n_save = n_save;
  if (n_save) std::memcpy(a.save_t, save_t, sizeof(double) * n_save);
  a.step_counts = o.step_counts;
  a.arena = arena;
  a.arena_cap = arena_cap;
  a.arena_top = &ctr->arena_top;
  a.overflow = &ctr->overflow;
  a.any_failed = &ctr->any_failed;
  a.head = head;
  a.S = S;
  a.natt = natt;
  a.status = status;
  a.y_final = y_final;
  a.work = &ctr->work_fwd;
  a.k = k;
  a.segw = segw;
  a.arena_block = 32;  // the fixed array: reserve one flush's worth at a time, wasting at most 31 slots a warp
  if (launch_tsit5_forward(problem_id, o.precision, a, s) != cudaSuccess) return GS_ERR_CUDA;

  RevArgs r;
  std::memset(&r, 0, sizeof(r));
  r.n = n;
  r.params = params;
  r.shared_w = shared_w;
  r.t0 = t0;
  r.t1 = t1;
  r.n_save = n_save;
  if (n_save) std::memcpy(r.save_t, save_t, sizeof(double) * n_save);
  r.loss = loss_out;
  r.params_bar = params_bar;
  r.y0_bar = y0_bar;
  r.status = status;
  r.arena = arena;
  r.arena_cap = arena_cap;
  r.head = head;
  r.S = S;
  r.y_final = y_final;
  r.work = &ctr->work_rev;
  r.k = k;
  r.segw = segw;
  if (launch_tsit5_reverse(problem_id, o.precision, r, s) != cudaSuccess) return GS_ERR_CUDA;

  if (cudaMemcpyAsync(traj_status, status, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GS_ERR_CUDA;
  ScratchCounters hc;
  if (cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
  if (hc.overflow) return GS_ERR_OOM;
  return hc.any_failed ? GS_ERR_TRAJ_FAILED : GS_OK;
}
