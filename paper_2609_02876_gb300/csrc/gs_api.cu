// C-ABI of gradsolve-gb300 (declared in include/gs.h): argument checking, the
// device-resident record, the reusable workspace of gs_solve_grad, and the
// kernel launches. No exception or abort crosses this boundary.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <chrono>
#include <thread>
#include <vector>

#include "../../include/gs.h"
#include "gs_internal.h"

using namespace gs;

namespace {

struct ProblemInfo {
  int d, P, stiff, n_shared;
};

bool problem_info(int pid, ProblemInfo* out) {
  switch (pid) {
    case GS_LORENZ: *out = {3, 3, 0, 0}; return true;
    case GS_VDP: *out = {2, 1, 0, 0}; return true;
    case GS_ROBERTSON: *out = {3, 3, 1, 0}; return true;
    case GS_HIRES: *out = {8, 12, 1, 0}; return true;
    case GS_LINEAR: *out = {2, 4, 0, 0}; return true;
    case GS_LV_UDE: *out = {2, 2, 0, 354}; return true;
    case GS_NEURAL_ROBERTSON: *out = {3, 2, 1, 353}; return true;
  }
  return false;
}


// Expected accepted steps per trajectory at rtol 1e-6, used for the first arena
// size and the choice of the record layout; an underestimate costs one rerun.
int step_guess(int pid) {
  switch (pid) {
    case GS_LORENZ: return 48;
    case GS_VDP: return 100;
    case GS_LV_UDE: return 40;
    case GS_ROBERTSON: return 110;
    case GS_HIRES: return 210;
  }
  return 256;
}
// The same for a tolerance rtol and a method: a method of error order q takes
// ~rtol^(-1/(q+1)) steps (q = 4 for Tsit5 and Rodas5P, 6 for Verner7, 2 for
// Rosenbrock23), Verner7 about 0.65 and Rosenbrock23 about 6 times the steps of
// Tsit5 / Rodas5P at rtol 1e-6.
int step_guess(int pid, double rtol, int method) {
  double base = step_guess(pid), expo = 0.2;
  if (method == GS_METHOD_VERNER7) {
    base *= 0.65;
    expo = 1.0 / 7.0;
  } else if (method == GS_METHOD_ROSENBROCK23) {
    base *= 6.0;
    expo = 1.0 / 3.0;
  }
  const double scale = std::pow(1e-6 / (rtol > 0.0 ? rtol : 1e-6), expo);
  const double g = base * (scale < 1.0 ? 1.0 : scale);
  return (int)std::ceil(g);
}

// Stored-stage records (k = 1): the doubles a step and a side step store (the
// kernels' StageData payloads), and the segment [prev, t, y[d], h, step payload]
// rounded up to a 16-byte multiple. Tsit5: Y_1..Y_5 (a side step also Y_6);
// Verner7: Y_1..Y_8 (a side step also its save state); Rodas5P: U_0..U_7, the
// LU factors, pivot reciprocals and pivots (the stage inputs and the save state
// are rebuilt from them); Rosenbrock23: k1, u2 and the LU of W (Y1 and the save
// state rebuilt).
int stage_step_payload(int method, int d) {
  switch (method) {
    case GS_METHOD_RODAS5P: return 10 * d + d * d;
    case GS_METHOD_ROSENBROCK23: return 4 * d + d * d;
    case GS_METHOD_VERNER7: return 8 * d;
  }
  return 5 * d;  // Tsit5
}
int stage_side_payload(int method, int d) {
  const bool rebuilt = method == GS_METHOD_RODAS5P || method == GS_METHOD_ROSENBROCK23;  // save state rebuilt
  return stage_step_payload(method, d) + (rebuilt ? 0 : d);
}
int stage_segw_of(int method, int d) { return ((3 + d + stage_step_payload(method, d)) + 1) & ~1; }

// Counters that the kernels update; one small device block per record.
struct Counters {
  unsigned long long work_fwd;
  unsigned long long work_rev;
  unsigned long long work_jvp;
  unsigned long long arena_top;
  int overflow;
  int any_failed;
  int tc_error;  // a tensor-core product's completion wait ran out in the reverse sweep
};

}  // namespace

struct gs_record {
  int device = 0;
  int problem = 0, method = GS_METHOD_TSIT5, precision = GS_FP64;
  int d = 0, P = 0, k = 0, segw = 0;
  int arena_block = 32;  // arena slots the record kernel reserves per warp at a time
  int64_t n = 0;
  double t0 = 0, t1 = 0, rtol = 0, atol = 0;
  int n_save = 0;
  double save_t[MAX_SAVE_HOST] = {0};
  // device buffers
  double* arena = nullptr;
  long long arena_cap = 0;
  long long* head = nullptr;
  int32_t* S = nullptr;
  int32_t* natt = nullptr;
  int32_t* status = nullptr;
  double* y_final = nullptr;
  void* wpart = nullptr;  // per-warp shared-weight gradient partials (shared-weight problems)
  // Stored stages (gs_solve_grad's workspace, Tsit5 FP64, k = 1): segments also
  // hold each step's stage data, side_stg (n x n_save x payload) the side steps'.
  int stages = 0;
  double* side_stg = nullptr;
  size_t side_cap = 0;  // doubles
  // chunk staging of a chunked FP32-mixed gs_solve_grad (inputs and outputs of one chunk)
  double* chunk_buf = nullptr;
  size_t chunk_cap = 0;  // doubles
  Counters* ctr = nullptr;
  Counters* ctr_host = nullptr;  // pinned
  int64_t n_cap = 0;             // capacity of the per-trajectory arrays
  long long nseg_total = 0;      // segments the record holds
  mutable size_t bytes = 0;
  // forward-order segment index, built on the first forward-mode call
  mutable long long* fwd_base = nullptr;
  mutable long long* fwd_seg = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // kernel timing (optional)
};

// A solve context: its own reusable record workspace, so that calls on
// different contexts (and streams) run concurrently.
struct gs_context {
  gs_record* ws = nullptr;
  std::mutex mu;
  int device = 0;
};

namespace {

gs_status cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return GS_ERR_OOM;
  return GS_ERR_CUDA;
}

void free_arrays(gs_record* r) {
  cudaFree(r->head);
  cudaFree(r->S);
  cudaFree(r->natt);
  cudaFree(r->status);
  cudaFree(r->y_final);
  r->head = nullptr;
  r->S = r->natt = r->status = nullptr;
  r->y_final = nullptr;
  r->n_cap = 0;
}

constexpr int kMaxDim = 8;  // largest state dimension of the registry

size_t record_bytes(const gs_record* r) {
  return (size_t)r->arena_cap * r->segw * sizeof(double) + r->side_cap * sizeof(double) +
         (size_t)r->n_cap * (sizeof(long long) + 3 * sizeof(int32_t) + kMaxDim * sizeof(double)) +
         sizeof(Counters);
}

// Ensures per-trajectory arrays for n trajectories of dimension d.
gs_status ensure_arrays(gs_record* r, int64_t n, int d) {
  (void)d;
  if (r->n_cap >= n && r->head) return GS_OK;
  free_arrays(r);
  const int64_t m = n > 0 ? n : 1;
  d = kMaxDim;  // y(t1) sized for any problem, so a reused workspace never reallocates for d
  cudaError_t e;
  if ((e = cudaMalloc(&r->head, m * sizeof(long long))) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMalloc(&r->S, m * sizeof(int32_t))) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMalloc(&r->natt, m * sizeof(int32_t))) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMalloc(&r->status, m * sizeof(int32_t))) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMalloc(&r->y_final, m * d * sizeof(double))) != cudaSuccess) return cuda_fail(e);
  r->n_cap = m;
  return GS_OK;
}

gs_status ensure_arena(gs_record* r, long long segs, int segw) {
  if (r->arena && r->arena_cap >= segs && r->segw == segw) return GS_OK;
  cudaFree(r->arena);
  r->arena = nullptr;
  r->arena_cap = 0;
  cudaError_t e = cudaMalloc(&r->arena, (size_t)segs * segw * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e);
  r->arena_cap = segs;
  return GS_OK;
}

gs_status ensure_counters(gs_record* r) {
  if (r->ctr) return GS_OK;
  cudaError_t e = cudaMalloc(&r->ctr, sizeof(Counters));
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMallocHost(&r->ctr_host, sizeof(Counters));
  if (e != cudaSuccess) return cuda_fail(e);
  return GS_OK;
}

gs_status ensure_events(gs_record* r) {
  for (int i = 0; i < 4; ++i)
    if (!r->ev[i] && cudaEventCreate(&r->ev[i]) != cudaSuccess) return GS_ERR_CUDA;
  return GS_OK;
}

void destroy(gs_record* r) {
  if (!r) return;
  for (int i = 0; i < 4; ++i)
    if (r->ev[i]) cudaEventDestroy(r->ev[i]);
  free_arrays(r);
  cudaFree(r->arena);
  cudaFree(r->fwd_base);
  cudaFree(r->fwd_seg);
  cudaFree(r->side_stg);
  cudaFree(r->chunk_buf);
  cudaFree(r->ctr);
  cudaFree(r->wpart);
  cudaFreeHost(r->ctr_host);
  delete r;
}

struct Call {
  int problem;
  ProblemInfo pi;
  int method, precision, k;
  int64_t max_steps;
  double h0;
  int32_t* step_counts;
  float* kernel_ms;
  double timeout_ms;
  int32_t* record_info;
  int control;
  int record_stages;
};

// Kernel launches by method.
cudaError_t launch_forward_m(int method, int problem, int precision, const FwdArgs& a, cudaStream_t s) {
  if (method == GS_METHOD_RODAS5P) return launch_rodas_forward(problem, precision, a, s);
  if (method == GS_METHOD_ROSENBROCK23) return launch_ros23_forward(problem, precision, a, s);
  if (method == GS_METHOD_VERNER7) return launch_vern7_forward(problem, precision, a, s);
  return launch_tsit5_forward(problem, precision, a, s);
}
cudaError_t launch_reverse_m(int method, int problem, int precision, const RevArgs& a, cudaStream_t s) {
  if (method == GS_METHOD_RODAS5P) return launch_rodas_reverse(problem, precision, a, s);
  if (method == GS_METHOD_ROSENBROCK23) return launch_ros23_reverse(problem, precision, a, s);
  if (method == GS_METHOD_VERNER7) return launch_vern7_reverse(problem, precision, a, s);
  return launch_tsit5_reverse(problem, precision, a, s);
}

// Waits for the work queued on s, polling with a deadline when timeout_ms > 0.
gs_status wait_stream(cudaStream_t s, double timeout_ms) {
  if (!(timeout_ms > 0.0)) return cudaStreamSynchronize(s) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
  const auto start = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) return GS_OK;
    if (e != cudaErrorNotReady) return GS_ERR_CUDA;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - start).count();
    if (ms > timeout_ms) return GS_ERR_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

gs_status check_common(int problem_id, int64_t n, const double* params, const double* y0, const float* shared_w,
                       double t0, double t1, const double* save_t, int n_save, double rtol, double atol,
                       const gs_options* opt, Call* c) {
  if (!problem_info(problem_id, &c->pi)) return GS_ERR_UNKNOWN_PROBLEM;
  c->problem = problem_id;
  if (n < 0) return GS_ERR_INVALID_ARG;
  if (n > 0 && (!params || !y0)) return GS_ERR_INVALID_ARG;
  if (c->pi.n_shared > 0 && n > 0 && !shared_w) return GS_ERR_INVALID_ARG;
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
  int method = o.method == GS_METHOD_AUTO ? (c->pi.stiff ? GS_METHOD_RODAS5P : GS_METHOD_TSIT5) : o.method;
  if (method != GS_METHOD_TSIT5 && method != GS_METHOD_RODAS5P && method != GS_METHOD_ROSENBROCK23 &&
      method != GS_METHOD_VERNER7)
    return GS_ERR_INVALID_ARG;
  if (o.ckpt_k < 0 || o.ckpt_k > KMAX_HOST) return GS_ERR_INVALID_ARG;
  if (c->pi.n_shared > 0 && o.ckpt_k > 1) return GS_ERR_INVALID_ARG;  // shared weights: every state stored
  if (o.max_steps < 0 || !std::isfinite(o.h0) || o.h0 < 0) return GS_ERR_INVALID_ARG;
  c->method = method;
  c->precision = o.precision;
  c->k = o.ckpt_k;  // 0: chosen in setup_record from the free device memory
  c->max_steps = o.max_steps > 0 ? o.max_steps : 1000000;
  c->h0 = o.h0;
  c->step_counts = o.step_counts;
  c->kernel_ms = o.kernel_ms;
  if (!std::isfinite(o.timeout_ms) || o.timeout_ms < 0) return GS_ERR_INVALID_ARG;
  c->timeout_ms = o.timeout_ms;
  c->record_info = o.record_info;
  if (o.control != GS_CONTROL_FAST && o.control != GS_CONTROL_FP64) return GS_ERR_INVALID_ARG;
  if (o.control == GS_CONTROL_FP64 && (method != GS_METHOD_TSIT5 || c->pi.n_shared > 0)) return GS_ERR_INVALID_ARG;
  c->control = o.control;
  if (o.record_stages != 0 && o.record_stages != 1) return GS_ERR_INVALID_ARG;
  c->record_stages = o.record_stages;
  if (method == GS_METHOD_TSIT5 && !tsit5_supports(problem_id, o.precision)) return GS_ERR_INVALID_ARG;
  if (method == GS_METHOD_RODAS5P && !rodas_supports(problem_id, o.precision)) return GS_ERR_INVALID_ARG;
  if (method == GS_METHOD_ROSENBROCK23 && !ros23_supports(problem_id, o.precision)) return GS_ERR_INVALID_ARG;
  if (method == GS_METHOD_VERNER7 && !vern7_supports(problem_id, o.precision)) return GS_ERR_INVALID_ARG;
  return GS_OK;
}

// Runs the record kernel into r, growing the arena until it fits.
gs_status run_record(gs_record* r, const Call& c, int64_t n, const double* params, const double* y0,
                     const float* shared_w, double* y_save, cudaStream_t s) {
  FwdArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.params = params;
  a.y0 = y0;
  a.shared_w = shared_w;
  a.t0 = r->t0;
  a.t1 = r->t1;
  a.rtol = r->rtol;
  a.atol = r->atol;
  a.h0 = c.h0;
  a.control = c.control;
  a.max_steps = c.max_steps;
  a.n_save = r->n_save;
  std::memcpy(a.save_t, r->save_t, sizeof(double) * r->n_save);
  a.y_save = y_save;
  a.step_counts = c.step_counts;
  for (int attempt = 0; attempt < 3; ++attempt) {
    a.k = r->k;
    a.segw = r->segw;
    a.arena_block = r->arena_block;
    a.stages = r->stages;
    a.side_stg = r->stages ? r->side_stg : nullptr;
    cudaError_t e = cudaMemsetAsync(r->ctr, 0, sizeof(Counters), s);
    if (e != cudaSuccess) return cuda_fail(e);
    a.arena = r->arena;
    a.arena_cap = r->arena_cap;
    a.arena_top = &r->ctr->arena_top;
    a.overflow = &r->ctr->overflow;
    a.any_failed = &r->ctr->any_failed;
    a.head = r->head;
    a.S = r->S;
    a.natt = r->natt;
    a.status = r->status;
    a.y_final = r->y_final;
    a.work = &r->ctr->work_fwd;
    if (c.kernel_ms) cudaEventRecord(r->ev[0], s);
    e = launch_forward_m(c.method, c.problem, c.precision, a, s);
    if (e != cudaSuccess) return GS_ERR_CUDA;
    if (c.kernel_ms) cudaEventRecord(r->ev[1], s);
    e = cudaMemcpyAsync(r->ctr_host, r->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return GS_ERR_CUDA;
    const gs_status ws = wait_stream(s, c.timeout_ms);
    if (ws != GS_OK) return ws;
    if (!r->ctr_host->overflow) {
      if (c.kernel_ms) cudaEventElapsedTime(&c.kernel_ms[0], r->ev[0], r->ev[1]);
      if (c.record_info) {
        c.record_info[0] = r->k;
        c.record_info[1] = r->stages;
      }
      r->nseg_total = (long long)r->ctr_host->arena_top;
      return GS_OK;
    }
    // The arena was too small: size it to the demand just measured (+1/8) and rerun
    // (as a compact record if the stored-stage one does not fit).
    const long long need = (long long)r->ctr_host->arena_top;
    gs_status st = ensure_arena(r, need + need / 8 + 1024, r->segw);
    if (st == GS_ERR_OOM && r->stages) {
      r->stages = 0;
      r->segw = segw_of(r->d, r->k);
      st = ensure_arena(r, need + need / 8 + 1024, r->segw);
    }
    if (st != GS_OK) return st;
  }
  return GS_ERR_OOM;
}

// Checkpoint interval when the caller leaves it to the library: k = 1 (every
// accepted state stored, nothing recomputed in the reverse sweep) if the
// expected record takes at most half of the free device memory, else a
// 128-byte segment of 14 - d steps (one checkpoint per 14 - d steps).
int auto_ckpt_k(const gs_record* r, int problem, int d, int64_t n) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
  const size_t held = (size_t)r->arena_cap * r->segw * sizeof(double);  // reusable by this record
  const double want = 1.25 * (double)(n > 0 ? n : 1) * step_guess(problem) * segw_of(d, 1) * sizeof(double);
  if (want <= 0.5 * (double)(free_b + held)) return 1;
  return 14 - d > 1 ? 14 - d : 1;
}

// Stored stages when the caller allows them (gs_solve_grad), the method and
// precision support them (Tsit5, Rodas5P, Rosenbrock23 or Verner7, FP64, no
// shared weights, a segment within MAX_STAGE_SEGW doubles), k is automatic, and
// the expected record with its side-step stages takes at most 70% of the free
// device memory (plus what this workspace already holds).
bool choose_stages(const gs_record* r, const Call& c, int64_t n, int n_save, double rtol) {
  if (c.method != GS_METHOD_TSIT5 && c.method != GS_METHOD_RODAS5P && c.method != GS_METHOD_VERNER7 &&
      c.method != GS_METHOD_ROSENBROCK23)
    return false;
  if (c.precision != GS_FP64 || c.pi.n_shared > 0 || c.k > 1) return false;
  if (stage_segw_of(c.method, c.pi.d) > MAX_STAGE_SEGW) return false;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return false;
  const double held = (double)r->arena_cap * r->segw * sizeof(double) + (double)r->side_cap * sizeof(double);
  const double m = (double)(n > 0 ? n : 1);
  const double want =
      m * (1.1 * step_guess(c.problem, rtol, c.method) + 1.0) * stage_segw_of(c.method, c.pi.d) * sizeof(double) +
      m * n_save * (double)stage_side_payload(c.method, c.pi.d) * sizeof(double);
  return want <= 0.7 * ((double)free_b + held);
}

gs_status setup_record(gs_record* r, const Call& c, int64_t n, double t0, double t1, const double* save_t,
                       int n_save, double rtol, double atol, bool allow_stages = false) {
  cudaGetDevice(&r->device);
  r->problem = c.problem;
  r->method = c.method;
  r->precision = c.precision;
  r->d = c.pi.d;
  r->P = c.pi.P;
  r->stages = (allow_stages && choose_stages(r, c, n, n_save, rtol)) ? 1 : 0;
  r->k = r->stages ? 1 : (c.k > 0 ? c.k : (c.pi.n_shared > 0 ? 1 : auto_ckpt_k(r, c.problem, c.pi.d, n)));
  if (c.pi.n_shared > 0 && !r->wpart) {
    const cudaError_t e = cudaMalloc(&r->wpart, (size_t)ude_max_warps() * WPART_BYTES_PER_WARP);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  r->n = n;
  r->t0 = t0;
  r->t1 = t1;
  r->rtol = rtol;
  r->atol = atol;
  r->n_save = n_save;
  if (n_save) std::memcpy(r->save_t, save_t, sizeof(double) * n_save);
  gs_status st = ensure_counters(r);
  if (st != GS_OK) return st;
  if (c.kernel_ms && (st = ensure_events(r)) != GS_OK) return st;
  st = ensure_arrays(r, n, r->d);
  if (st != GS_OK) return st;
  if (r->stages) {
    const size_t need = (size_t)(n > 0 ? n : 1) * (size_t)(n_save > 0 ? n_save : 1) *
                        (size_t)stage_side_payload(c.method, r->d);
    if (r->side_cap < need) {
      cudaFree(r->side_stg);
      r->side_stg = nullptr;
      r->side_cap = 0;
      const cudaError_t e = cudaMalloc(&r->side_stg, need * sizeof(double));
      if (e != cudaSuccess) {
        r->stages = 0;  // fall back to the compact record
        r->k = c.k > 0 ? c.k : auto_ckpt_k(r, c.problem, c.pi.d, n);
      } else {
        r->side_cap = need;
      }
    }
  }
  const int segw = r->stages ? stage_segw_of(c.method, r->d) : segw_of(r->d, r->k);
  if (r->segw != segw) {
    cudaFree(r->arena);
    r->arena = nullptr;
    r->arena_cap = 0;
    r->segw = segw;
  }
  // Expected segments, plus the unused tails of the record kernel's per-warp slot
  // blocks: a warp reserves about an eighth of its expected segments at a time
  // (32 to ARENA_BLOCK_HOST slots), and leaves less than one block unused.
  const long long m = n > 0 ? n : 1;
  const long long per_traj = (step_guess(c.problem, rtol, c.method) + r->k - 1) / r->k + 1;
  const long long warps = std::min<long long>((m + 31) / 32, 4096 * 4);
  long long blk = 32;
  while (blk < ARENA_BLOCK_HOST && 8 * 2 * blk <= m * per_traj / warps) blk *= 2;
  r->arena_block = (int)blk;
  const long long slack = warps * blk;
  const long long want = m * per_traj + slack;
  if (r->arena_cap > 0 && r->arena_cap < want / 4) {  // far too small for this ensemble: start over
    cudaFree(r->arena);
    r->arena = nullptr;
    r->arena_cap = 0;
  }
  if (r->arena_cap == 0) {
    st = ensure_arena(r, want, segw);
    if (st == GS_ERR_OOM && r->stages) {  // the stored-stage record does not fit: compact record
      r->stages = 0;
      r->k = c.k > 0 ? c.k : auto_ckpt_k(r, c.problem, c.pi.d, n);
      r->segw = segw_of(r->d, r->k);
      st = ensure_arena(r, m * ((step_guess(c.problem, rtol, c.method) + r->k - 1) / r->k + 1) + slack, r->segw);
      // (the block size chosen above stays: it depends on the ensemble, not the layout)
    }
    if (st != GS_OK) return st;
  }
  return GS_OK;
}

gs_status launch_reverse(const gs_record* r, const double* params, const float* shared_w,
                         const double* y_save_bar, double* loss, double* params_bar, double* y0_bar,
                         float* shared_w_bar, cudaStream_t s) {
  RevArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = r->n;
  a.params = params;
  a.shared_w = shared_w;
  a.shared_w_bar = shared_w_bar;
  a.t0 = r->t0;
  a.t1 = r->t1;
  a.n_save = r->n_save;
  std::memcpy(a.save_t, r->save_t, sizeof(double) * r->n_save);
  a.y_save_bar = y_save_bar;
  a.loss = loss;
  a.params_bar = params_bar;
  a.y0_bar = y0_bar;
  a.status = r->status;
  a.arena = r->arena;
  a.arena_cap = r->arena_cap;
  a.head = r->head;
  a.S = r->S;
  a.y_final = r->y_final;
  a.wpart = r->wpart;
  a.work = &r->ctr->work_rev;
  a.k = r->k;
  a.segw = r->segw;
  a.stages = r->stages;
  a.side_stg = r->stages ? r->side_stg : nullptr;
  a.tc_error = &r->ctr->tc_error;
  cudaError_t e = cudaMemsetAsync(&r->ctr->work_rev, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  e = launch_reverse_m(r->method, r->problem, r->precision, a, s);
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

// Forward-mode replay launches over directions [g0, g1) of the call, at most
// JVP_MAX_DIR per launch; `a` carries everything but the per-launch fields.
gs_status launch_jvp_range(const gs_record* r, JvpArgs a, int g0, int g1, double* loss_out, cudaStream_t s) {
  const int64_t n = r->n;
  const double* pdot = a.params_dot;
  const double* ydot = a.y0_dot;
  double* ldot = a.loss_dot;
  double* ysd = a.y_save_dot;
  for (int g = g0; g < g1; g += JVP_MAX_DIR) {
    const int nd = (g1 - g) < JVP_MAX_DIR ? (g1 - g) : JVP_MAX_DIR;
    a.dir0 = g;
    a.nd = nd;
    a.loss = (g == g0) ? loss_out : nullptr;
    if (!a.basis) {
      const int64_t q = g - g0;
      a.params_dot = pdot ? pdot + q * r->P * n : nullptr;
      a.y0_dot = ydot ? ydot + q * r->d * n : nullptr;
      a.loss_dot = ldot + q * n;
      a.y_save_dot = ysd ? ysd + q * (int64_t)r->n_save * r->d * n : nullptr;
    }
    cudaError_t e = cudaMemsetAsync(&r->ctr->work_jvp, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return GS_ERR_CUDA;
    e = launch_jvp(r->method, r->problem, a, s);
    if (e != cudaSuccess) return GS_ERR_CUDA;
  }
  return GS_OK;
}

// The record's segments in forward order (built once, on the stream of the
// first forward-mode call).
gs_status ensure_fwd_index(const gs_record* r, cudaStream_t s) {
  if (r->fwd_base) return GS_OK;
  long long* base = nullptr;
  long long* seg = nullptr;
  cudaError_t e = cudaMalloc(&base, (size_t)r->n * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&seg, (size_t)(r->nseg_total > 0 ? r->nseg_total : 1) * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(&r->ctr->work_jvp, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess)
    e = launch_fwd_index(r->n, r->head, r->S, r->status, r->arena, r->arena_cap, r->k, r->segw, &r->ctr->work_jvp,
                         base, seg, r->nseg_total, s);
  if (e != cudaSuccess) {
    cudaFree(base);
    cudaFree(seg);
    return cuda_fail(e);
  }
  r->fwd_base = base;
  r->fwd_seg = seg;
  r->bytes += (size_t)(r->n + (r->nseg_total > 0 ? r->nseg_total : 1)) * sizeof(long long);
  return GS_OK;
}

// The parts of the forward-mode arguments that come from the record.
gs_status jvp_common(const gs_record* r, const double* params, const double* y0, cudaStream_t s, JvpArgs* a) {
  if (!params || !y0) return GS_ERR_INVALID_ARG;
  if (!jvp_supports(r->method, r->problem)) return GS_ERR_INVALID_ARG;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != r->device) return GS_ERR_INVALID_ARG;
  const gs_status st = ensure_fwd_index(r, s);
  if (st != GS_OK) return st;
  std::memset(a, 0, sizeof(*a));
  a->n = r->n;
  a->params = params;
  a->y0 = y0;
  a->t0 = r->t0;
  a->t1 = r->t1;
  a->n_save = r->n_save;
  std::memcpy(a->save_t, r->save_t, sizeof(double) * r->n_save);
  a->status = r->status;
  a->arena = r->arena;
  a->S = r->S;
  a->fwd_base = r->fwd_base;
  a->fwd_seg = r->fwd_seg;
  a->work = &r->ctr->work_jvp;
  a->k = r->k;
  a->segw = r->segw;
  return GS_OK;
}

// Record then reverse into workspace r (the body of gs_solve_grad[_ctx]).
gs_status solve_grad_in(gs_record* r, const Call& c, int64_t n, const double* params, const double* y0,
                        const float* shared_w, double t0, double t1, const double* save_t, int n_save, double rtol,
                        double atol, cudaStream_t s, double* loss_out, double* params_bar, double* y0_bar,
                        float* shared_w_bar, int32_t* traj_status, bool allow_stages) {
  gs_status st = setup_record(r, c, n, t0, t1, save_t, n_save, rtol, atol, allow_stages);
  if (st != GS_OK) return st;
  st = run_record(r, c, n, params, y0, shared_w, nullptr, s);
  if (st != GS_OK) return st;
  if (c.kernel_ms) cudaEventRecord(r->ev[2], s);
  st = launch_reverse(r, params, shared_w, nullptr, loss_out, params_bar, y0_bar, shared_w_bar, s);
  if (st != GS_OK) return st;
  if (c.kernel_ms) cudaEventRecord(r->ev[3], s);
  cudaError_t e = cudaMemcpyAsync(traj_status, r->status, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  e = cudaMemcpyAsync(&r->ctr_host->tc_error, &r->ctr->tc_error, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  st = wait_stream(s, c.timeout_ms);
  if (st != GS_OK) return st;
  if (c.kernel_ms) cudaEventElapsedTime(&c.kernel_ms[1], r->ev[2], r->ev[3]);
  if (r->ctr_host->tc_error) return GS_ERR_CUDA;
  return r->ctr_host->any_failed ? GS_ERR_TRAJ_FAILED : GS_OK;
}

// An FP32-mixed gs_solve_grad of more than two chunks runs chunk by chunk
// (shared-weight problems, step_counts and a wait deadline excepted): the
// compact record of 2^21 Lorenz trajectories takes ~5.5 GB against ~44 GB at
// 2^24, and the reverse sweep's scattered per-lane segment reads run faster
// over the smaller arena (Lorenz 2^24, rtol 1e-6, measured: 48.7 / 43.3 / 40.7
// / 40.4 / 41.4 ms in chunks of 2^18 / 2^19 / 2^20 / 2^21 / 2^22 against 44.0
// ms in one piece). Trajectories are independent, so
// the results equal the one-piece call bit for bit.
//
// The FP64 form, bound by its FP64 pipe, is slower in chunks when the whole
// stored-stage record fits (608 against 603 ms at Lorenz 2^24 in chunks of
// 2^22) and then runs in one piece. An FP64 call whose whole stored-stage
// record would not fit in device memory
// (it then records compactly and its reverse sweep recomputes every stage) but
// a chunk's would, runs in the largest power-of-two chunks (2^18 to 2^23) whose
// stored-stage record fits (gs_solve_grad only; contexts record compactly):
// the reverse sweep then reads the stages instead of recomputing them.
constexpr int64_t MIXED_CHUNK = int64_t(1) << 21;

int64_t solve_chunk(const gs_record* r, const Call& c, int64_t n, int n_save, double rtol, bool allow_stages) {
  if (c.pi.n_shared > 0 || c.step_counts || c.timeout_ms > 0.0) return 0;
  if (c.precision == GS_FP32_MIXED) return n > 2 * MIXED_CHUNK ? MIXED_CHUNK : 0;
  if (!allow_stages || choose_stages(r, c, n, n_save, rtol)) return 0;
  for (int64_t m = int64_t(1) << 23; m >= (int64_t(1) << 18); m >>= 1)
    if (m < n && choose_stages(r, c, m, n_save, rtol)) return m;
  return 0;
}

gs_status solve_grad_chunked(gs_record* r, const Call& c, int64_t n, int64_t ch, const double* params,
                             const double* y0, double t0, double t1, const double* save_t, int n_save, double rtol,
                             double atol, cudaStream_t s, double* loss_out, double* params_bar, double* y0_bar,
                             int32_t* traj_status, bool allow_stages) {
  const int P = c.pi.P, d = c.pi.d;
  const size_t need = (size_t)(2 * (P + d)) * (size_t)ch;  // [P + d][ch] in, [P + d][ch] out
  if (r->chunk_cap < need) {
    cudaFree(r->chunk_buf);
    r->chunk_buf = nullptr;
    r->chunk_cap = 0;
    if (cudaMalloc(&r->chunk_buf, need * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();  // no staging: the one-piece call
      return solve_grad_in(r, c, n, params, y0, nullptr, t0, t1, save_t, n_save, rtol, atol, s, loss_out,
                           params_bar, y0_bar, nullptr, traj_status, allow_stages);
    }
    r->chunk_cap = need;
  }
  double* in_p = r->chunk_buf;             // [P][ch]
  double* in_y = in_p + (size_t)P * ch;    // [d][ch]
  double* out_p = in_y + (size_t)d * ch;   // [P][ch]
  double* out_y = out_p + (size_t)P * ch;  // [d][ch]
  float kms[2] = {0.0f, 0.0f}, sum[2] = {0.0f, 0.0f};
  Call cc = c;
  if (c.kernel_ms) cc.kernel_ms = kms;
  bool failed = false;
  const size_t pitch = (size_t)n * sizeof(double);
  for (int64_t k0 = 0; k0 < n; k0 += ch) {
    const int64_t nc = std::min(ch, n - k0);
    const size_t w = (size_t)nc * sizeof(double);
    if (cudaMemcpy2DAsync(in_p, w, params + k0, pitch, w, P, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpy2DAsync(in_y, w, y0 + k0, pitch, w, d, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return GS_ERR_CUDA;
    const gs_status st = solve_grad_in(r, cc, nc, in_p, in_y, nullptr, t0, t1, save_t, n_save, rtol, atol, s,
                                       loss_out ? loss_out + k0 : nullptr, params_bar ? out_p : nullptr,
                                       y0_bar ? out_y : nullptr, nullptr, traj_status + k0, allow_stages);
    if (st == GS_ERR_TRAJ_FAILED)
      failed = true;
    else if (st != GS_OK)
      return st;
    if (params_bar &&
        cudaMemcpy2DAsync(params_bar + k0, pitch, out_p, w, w, P, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return GS_ERR_CUDA;
    if (y0_bar && cudaMemcpy2DAsync(y0_bar + k0, pitch, out_y, w, w, d, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return GS_ERR_CUDA;
    sum[0] += kms[0];
    sum[1] += kms[1];
  }
  const gs_status ws = wait_stream(s, 0.0);
  if (ws != GS_OK) return ws;
  if (c.kernel_ms) {
    c.kernel_ms[0] = sum[0];
    c.kernel_ms[1] = sum[1];
  }
  return failed ? GS_ERR_TRAJ_FAILED : GS_OK;
}

// gs_solve_grad's reusable record, one per device.
std::mutex g_ws_mu;
std::vector<gs_record*> g_ws;

gs_record* workspace(int dev) {
  if ((int)g_ws.size() <= dev) g_ws.resize(dev + 1, nullptr);
  if (!g_ws[dev]) g_ws[dev] = new (std::nothrow) gs_record();
  return g_ws[dev];
}

// gs_solve_grad_host's device staging, one per device (guarded by g_ws_mu):
// two input and two output chunk slots, a copy stream per direction, a
// compute stream and the events that order them.
struct HostPipe {
  cudaStream_t comp = nullptr, h2d = nullptr, d2h = nullptr;
  cudaEvent_t in_ready[2] = {nullptr, nullptr}, out_ready[2] = {nullptr, nullptr},
              out_free[2] = {nullptr, nullptr};
  double* in[2] = {nullptr, nullptr};   // [P + d][chunk]
  double* out[2] = {nullptr, nullptr};  // [1 + P + d][chunk] doubles, then [chunk] int32 status
  size_t in_bytes = 0, out_bytes = 0;
};
std::vector<HostPipe*> g_pipe;

gs_status host_pipe(int dev, size_t in_bytes, size_t out_bytes, HostPipe** out) {
  if ((int)g_pipe.size() <= dev) g_pipe.resize(dev + 1, nullptr);
  if (!g_pipe[dev]) {
    HostPipe* hp = new (std::nothrow) HostPipe();
    if (!hp) return GS_ERR_OOM;
    if (cudaStreamCreateWithFlags(&hp->comp, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&hp->h2d, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&hp->d2h, cudaStreamNonBlocking) != cudaSuccess)
      return GS_ERR_CUDA;
    for (int i = 0; i < 2; ++i)
      if (cudaEventCreateWithFlags(&hp->in_ready[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&hp->out_ready[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&hp->out_free[i], cudaEventDisableTiming) != cudaSuccess)
        return GS_ERR_CUDA;
    g_pipe[dev] = hp;
  }
  HostPipe* hp = g_pipe[dev];
  if (hp->in_bytes < in_bytes || hp->out_bytes < out_bytes) {
    for (int i = 0; i < 2; ++i) {
      cudaFree(hp->in[i]);
      cudaFree(hp->out[i]);
      hp->in[i] = hp->out[i] = nullptr;
    }
    hp->in_bytes = hp->out_bytes = 0;
    for (int i = 0; i < 2; ++i)
      if (cudaMalloc(&hp->in[i], in_bytes) != cudaSuccess || cudaMalloc(&hp->out[i], out_bytes) != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_OOM;
      }
    hp->in_bytes = in_bytes;
    hp->out_bytes = out_bytes;
  }
  *out = hp;
  return GS_OK;
}

// Rows [rows][n] of a host SoA array, trajectories [k0, k0 + nc), to or from a
// device [rows][nc] block: one strided copy.
cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, int rows,
                      cudaMemcpyKind kind, cudaStream_t s) {
  if (rows <= 0 || width == 0) return cudaSuccess;
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, (size_t)rows, kind, s);
}

}  // namespace

extern "C" {

const char* gs_status_string(gs_status s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_INVALID_ARG: return "invalid argument";
    case GS_ERR_UNKNOWN_PROBLEM: return "unknown problem id";
    case GS_ERR_OOM: return "device out of memory";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_TRAJ_FAILED: return "one or more trajectories failed (see traj_status)";
    case GS_ERR_TIMEOUT: return "timed out waiting for the device";
  }
  return "unknown status";
}

gs_status gs_default_options(gs_options* opt) {
  if (!opt) return GS_ERR_INVALID_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = GS_FP64;
  opt->method = GS_METHOD_AUTO;
  return GS_OK;
}

gs_status gs_problem_info(int problem_id, int* d, int* P, int* stiff, int* n_shared) {
  ProblemInfo pi;
  if (!problem_info(problem_id, &pi)) return GS_ERR_UNKNOWN_PROBLEM;
  if (d) *d = pi.d;
  if (P) *P = pi.P;
  if (stiff) *stiff = pi.stiff;
  if (n_shared) *n_shared = pi.n_shared;
  return GS_OK;
}

gs_status gs_forward_record(int problem_id, int64_t n, const double* params, const double* y0,
                            const float* shared_w, double t0, double t1, const double* save_t, int n_save,
                            double rtol, double atol, const gs_options* opt, gs_stream stream,
                            double* y_save_out, int32_t* traj_status, gs_record** rec_out) {
  if (!rec_out) return GS_ERR_INVALID_ARG;
  *rec_out = nullptr;
  Call c;
  gs_status st = check_common(problem_id, n, params, y0, shared_w, t0, t1, save_t, n_save, rtol, atol, opt, &c);
  if (st != GS_OK) return st;
  if (n > 0 && !traj_status) return GS_ERR_INVALID_ARG;
  c.timeout_ms = 0.0;  // the record handle owns the work: wait for it
  gs_record* r = new (std::nothrow) gs_record();
  if (!r) return GS_ERR_OOM;
  st = setup_record(r, c, n, t0, t1, save_t, n_save, rtol, atol, c.record_stages == 1);
  if (st != GS_OK) { destroy(r); return st; }
  cudaStream_t s = (cudaStream_t)stream;
  if (n > 0) {
    st = run_record(r, c, n, params, y0, shared_w, y_save_out, s);
    if (st != GS_OK) { destroy(r); return st; }
    cudaError_t e = cudaMemcpyAsync(traj_status, r->status, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { destroy(r); return GS_ERR_CUDA; }
  }
  r->bytes = record_bytes(r);
  *rec_out = r;
  return (n > 0 && r->ctr_host->any_failed) ? GS_ERR_TRAJ_FAILED : GS_OK;
}

gs_status gs_reverse(const gs_record* rec, const double* params, const double* y0, const float* shared_w,
                     const double* y_save_bar, double* loss_out, double* params_bar, double* y0_bar,
                     float* shared_w_bar, gs_stream stream) {
  (void)y0;
  if (!rec) return GS_ERR_INVALID_ARG;
  if (rec->n == 0) return GS_OK;
  if (!params) return GS_ERR_INVALID_ARG;
  ProblemInfo pi;
  problem_info(rec->problem, &pi);
  if (pi.n_shared > 0 && !shared_w) return GS_ERR_INVALID_ARG;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != rec->device) return GS_ERR_INVALID_ARG;
  return launch_reverse(rec, params, shared_w, y_save_bar, loss_out, params_bar, y0_bar, shared_w_bar,
                        (cudaStream_t)stream);
}

gs_status gs_replay_jvp(const gs_record* rec, const double* params, const double* y0, int n_dir,
                        const double* params_dot, const double* y0_dot, double* loss_out, double* loss_dot,
                        double* y_save_dot, gs_stream stream) {
  if (!rec) return GS_ERR_INVALID_ARG;
  if (n_dir < 1 || !loss_dot) return GS_ERR_INVALID_ARG;
  if (rec->n == 0) return GS_OK;
  JvpArgs a;
  const gs_status st = jvp_common(rec, params, y0, (cudaStream_t)stream, &a);
  if (st != GS_OK) return st;
  a.params_dot = params_dot;
  a.y0_dot = y0_dot;
  a.loss_dot = loss_dot;
  a.y_save_dot = y_save_dot;
  return launch_jvp_range(rec, a, 0, n_dir, loss_out, (cudaStream_t)stream);
}

gs_status gs_forward_grad(const gs_record* rec, const double* params, const double* y0, double* loss_out,
                          double* params_bar, double* y0_bar, gs_stream stream) {
  if (!rec) return GS_ERR_INVALID_ARG;
  if (!params_bar && !y0_bar) return GS_ERR_INVALID_ARG;
  if (rec->n == 0) return GS_OK;
  JvpArgs a;
  const gs_status st = jvp_common(rec, params, y0, (cudaStream_t)stream, &a);
  if (st != GS_OK) return st;
  a.basis = 1;
  a.grad_p = params_bar;
  a.grad_y = y0_bar;
  const int g0 = params_bar ? 0 : rec->P;
  const int g1 = y0_bar ? rec->P + rec->d : rec->P;
  return launch_jvp_range(rec, a, g0, g1, loss_out, (cudaStream_t)stream);
}

gs_status gs_record_refresh(gs_record* rec, const double* params, const double* y0, const float* shared_w,
                            gs_stream stream) {
  if (!rec) return GS_ERR_INVALID_ARG;
  if (rec->n == 0) return GS_OK;
  if (!params || !y0) return GS_ERR_INVALID_ARG;
  ProblemInfo pi;
  problem_info(rec->problem, &pi);
  if (pi.n_shared > 0 && !shared_w) return GS_ERR_INVALID_ARG;
  if (rec->stages) return GS_ERR_INVALID_ARG;  // its stored stage data would go stale
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != rec->device) return GS_ERR_INVALID_ARG;
  RevArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = rec->n;
  a.params = params;
  a.shared_w = shared_w;
  a.status = rec->status;
  a.arena = rec->arena;
  a.arena_cap = rec->arena_cap;
  a.head = rec->head;
  a.S = rec->S;
  a.k = rec->k;
  a.segw = rec->segw;
  const cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e =
      (rec->method == GS_METHOD_RODAS5P)
          ? launch_rodas_refresh(rec->problem, rec->precision, a, rec->arena, rec->y_final, y0, s)
      : (rec->method == GS_METHOD_ROSENBROCK23)
          ? launch_ros23_refresh(rec->problem, rec->precision, a, rec->arena, rec->y_final, y0, s)
      : (rec->method == GS_METHOD_VERNER7)
          ? launch_vern7_refresh(rec->problem, rec->precision, a, rec->arena, rec->y_final, y0, s)
          : launch_tsit5_refresh(rec->problem, rec->precision, a, rec->arena, rec->y_final, y0, s);
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_solve_grad(int problem_id, int64_t n, const double* params, const double* y0,
                        const float* shared_w, double t0, double t1, const double* save_t, int n_save,
                        double rtol, double atol, const gs_options* opt, gs_stream stream, double* loss_out,
                        double* params_bar, double* y0_bar, float* shared_w_bar, int32_t* traj_status) {
  Call c;
  gs_status st = check_common(problem_id, n, params, y0, shared_w, t0, t1, save_t, n_save, rtol, atol, opt, &c);
  if (st != GS_OK) return st;
  if (n == 0) return GS_OK;
  if (!traj_status) return GS_ERR_INVALID_ARG;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_ws_mu);
  gs_record* r = workspace(dev);
  if (!r) return GS_ERR_OOM;
  if (const int64_t ch = solve_chunk(r, c, n, n_save, rtol, true))
    return solve_grad_chunked(r, c, n, ch, params, y0, t0, t1, save_t, n_save, rtol, atol, (cudaStream_t)stream,
                              loss_out, params_bar, y0_bar, traj_status, true);
  return solve_grad_in(r, c, n, params, y0, shared_w, t0, t1, save_t, n_save, rtol, atol, (cudaStream_t)stream,
                       loss_out, params_bar, y0_bar, shared_w_bar, traj_status, true);
}

gs_status gs_solve_grad_host(int problem_id, int64_t n, const double* params, const double* y0,
                             const float* shared_w, double t0, double t1, const double* save_t, int n_save,
                             double rtol, double atol, const gs_options* opt, int64_t chunk, double* loss_out,
                             double* params_bar, double* y0_bar, float* shared_w_bar, int32_t* traj_status) {
  Call c;
  gs_status st = check_common(problem_id, n, params, y0, shared_w, t0, t1, save_t, n_save, rtol, atol, opt, &c);
  if (st != GS_OK) return st;
  if (chunk < 0 || (opt && opt->step_counts)) return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  if (!traj_status) return GS_ERR_INVALID_ARG;
  const int P = c.pi.P, d = c.pi.d;
  int64_t ch = chunk > 0 ? chunk : ((int64_t)1 << 21);
  if (c.pi.n_shared > 0 || ch > n) ch = n;  // a shared-weight gradient sums the whole ensemble: one chunk
  const int64_t nchunks = (n + ch - 1) / ch;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_ws_mu);
  gs_record* r = workspace(dev);
  if (!r) return GS_ERR_OOM;
  HostPipe* hp = nullptr;
  const size_t in_bytes = (size_t)(P + d) * ch * sizeof(double);
  const size_t out_bytes = (size_t)(1 + P + d) * ch * sizeof(double) + (size_t)ch * sizeof(int32_t);
  if ((st = host_pipe(dev, in_bytes, out_bytes, &hp)) != GS_OK) return st;
  const size_t hp_row = (size_t)n * sizeof(double), hs_row = (size_t)n * sizeof(int32_t);

  auto upload = [&](int64_t ci) -> cudaError_t {
    const int64_t k0 = ci * ch, nc = std::min(ch, n - k0);
    const int slot = (int)(ci & 1);
    double* din = hp->in[slot];
    const size_t w = (size_t)nc * sizeof(double);
    cudaError_t e = copy_rows(din, w, params + k0, hp_row, w, P, cudaMemcpyHostToDevice, hp->h2d);
    if (e == cudaSuccess)
      e = copy_rows(din + (size_t)P * nc, w, y0 + k0, hp_row, w, d, cudaMemcpyHostToDevice, hp->h2d);
    if (e == cudaSuccess) e = cudaEventRecord(hp->in_ready[slot], hp->h2d);
    return e;
  };
  auto download = [&](int64_t ci) -> cudaError_t {
    const int64_t k0 = ci * ch, nc = std::min(ch, n - k0);
    const int slot = (int)(ci & 1);
    const double* dout = hp->out[slot];
    const size_t w = (size_t)nc * sizeof(double);
    cudaError_t e = cudaStreamWaitEvent(hp->d2h, hp->out_ready[slot], 0);
    if (e == cudaSuccess && loss_out)
      e = copy_rows(loss_out + k0, hp_row, dout, w, w, 1, cudaMemcpyDeviceToHost, hp->d2h);
    if (e == cudaSuccess && params_bar)
      e = copy_rows(params_bar + k0, hp_row, dout + nc, w, w, P, cudaMemcpyDeviceToHost, hp->d2h);
    if (e == cudaSuccess && y0_bar)
      e = copy_rows(y0_bar + k0, hp_row, dout + (size_t)(1 + P) * nc, w, w, d, cudaMemcpyDeviceToHost, hp->d2h);
    if (e == cudaSuccess)
      e = copy_rows(traj_status + k0, hs_row, dout + (size_t)(1 + P + d) * nc, (size_t)nc * sizeof(int32_t),
                    (size_t)nc * sizeof(int32_t), 1, cudaMemcpyDeviceToHost, hp->d2h);
    if (e == cudaSuccess) e = cudaEventRecord(hp->out_free[slot], hp->d2h);
    return e;
  };

  gs_status result = GS_OK;
  cudaError_t e = upload(0);
  for (int64_t ci = 0; ci < nchunks && e == cudaSuccess; ++ci) {
    const int64_t nc = std::min(ch, n - ci * ch);
    const int slot = (int)(ci & 1);
    // the next chunk's inputs go to the other slot, whose previous solve has returned
    if (ci + 1 < nchunks && (e = upload(ci + 1)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(hp->comp, hp->in_ready[slot], 0)) != cudaSuccess) break;
    if (ci >= 2 && (e = cudaStreamWaitEvent(hp->comp, hp->out_free[slot], 0)) != cudaSuccess) break;
    double* din = hp->in[slot];
    double* dout = hp->out[slot];
    const gs_status cs = solve_grad_in(r, c, nc, din, din + (size_t)P * nc, shared_w, t0, t1, save_t, n_save, rtol,
                                       atol, hp->comp, dout, dout + nc, dout + (size_t)(1 + P) * nc, shared_w_bar,
                                       reinterpret_cast<int32_t*>(dout + (size_t)(1 + P + d) * nc), true);
    if (cs == GS_ERR_TRAJ_FAILED) {
      result = GS_ERR_TRAJ_FAILED;
    } else if (cs != GS_OK) {
      result = cs;
      break;
    }
    if ((e = cudaEventRecord(hp->out_ready[slot], hp->comp)) != cudaSuccess) break;
    if ((e = download(ci)) != cudaSuccess) break;
  }
  const cudaError_t e1 = cudaStreamSynchronize(hp->h2d);
  const cudaError_t e2 = cudaStreamSynchronize(hp->d2h);
  const cudaError_t e3 = cudaStreamSynchronize(hp->comp);
  if (result != GS_OK && result != GS_ERR_TRAJ_FAILED) return result;
  if (e != cudaSuccess || e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return GS_ERR_CUDA;
  return result;
}

gs_status gs_solve(int problem_id, int64_t n, const double* params, const double* y0, const float* shared_w,
                   double t0, double t1, const double* save_t, int n_save, double rtol, double atol,
                   const gs_options* opt, gs_stream stream, double* y_save_out, double* y_final_out,
                   int32_t* traj_status) {
  Call c;
  gs_status st = check_common(problem_id, n, params, y0, shared_w, t0, t1, save_t, n_save, rtol, atol, opt, &c);
  if (st != GS_OK) return st;
  if (n == 0) return GS_OK;
  if (!traj_status || !y_final_out) return GS_ERR_INVALID_ARG;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_ws_mu);
  gs_record* r = workspace(dev);
  if (!r) return GS_ERR_OOM;
  if ((st = ensure_counters(r)) != GS_OK) return st;
  if (c.kernel_ms && (st = ensure_events(r)) != GS_OK) return st;
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
  a.h0 = c.h0;
  a.control = c.control;
  a.max_steps = c.max_steps;
  a.n_save = n_save;
  if (n_save) std::memcpy(a.save_t, save_t, sizeof(double) * n_save);
  a.y_save = y_save_out;
  a.step_counts = c.step_counts;
  a.k = 0;  // nothing recorded: no arena, no per-trajectory record arrays
  a.segw = 0;
  a.arena_top = &r->ctr->arena_top;
  a.overflow = &r->ctr->overflow;
  a.any_failed = &r->ctr->any_failed;
  a.status = traj_status;
  a.y_final = y_final_out;
  a.work = &r->ctr->work_fwd;
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(r->ctr, 0, sizeof(Counters), s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (c.kernel_ms) cudaEventRecord(r->ev[0], s);
  e = launch_forward_m(c.method, c.problem, c.precision, a, s);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  if (c.kernel_ms) cudaEventRecord(r->ev[1], s);
  e = cudaMemcpyAsync(r->ctr_host, r->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  if ((st = wait_stream(s, c.timeout_ms)) != GS_OK) return st;
  if (c.kernel_ms) cudaEventElapsedTime(&c.kernel_ms[0], r->ev[0], r->ev[1]);
  return r->ctr_host->any_failed ? GS_ERR_TRAJ_FAILED : GS_OK;
}

gs_status gs_context_create(gs_context** ctx) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  *ctx = nullptr;
  gs_context* c = new (std::nothrow) gs_context();
  if (!c) return GS_ERR_OOM;
  c->ws = new (std::nothrow) gs_record();
  if (!c->ws) {
    delete c;
    return GS_ERR_OOM;
  }
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c->ws;
    delete c;
    return GS_ERR_CUDA;
  }
  *ctx = c;
  return GS_OK;
}

gs_status gs_context_destroy(gs_context* ctx) {
  if (!ctx) return GS_OK;
  destroy(ctx->ws);
  delete ctx;
  return GS_OK;
}

gs_status gs_context_bytes(const gs_context* ctx, size_t* bytes) {
  if (!ctx || !bytes) return GS_ERR_INVALID_ARG;
  *bytes = record_bytes(ctx->ws);
  return GS_OK;
}

gs_status gs_solve_grad_ctx(gs_context* ctx, int problem_id, int64_t n, const double* params, const double* y0,
                            const float* shared_w, double t0, double t1, const double* save_t, int n_save,
                            double rtol, double atol, const gs_options* opt, gs_stream stream, double* loss_out,
                            double* params_bar, double* y0_bar, float* shared_w_bar, int32_t* traj_status) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  Call c;
  gs_status st = check_common(problem_id, n, params, y0, shared_w, t0, t1, save_t, n_save, rtol, atol, opt, &c);
  if (st != GS_OK) return st;
  if (n == 0) return GS_OK;
  if (!traj_status) return GS_ERR_INVALID_ARG;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != ctx->device) return GS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(ctx->mu);
  // contexts record compactly: with stored stages the request server's
  // latencies measured worse (0.8 load, 1000 requests: p50 60 / p99 1015 ms
  // against 43 / 865 ms), the stage records of concurrent small launches
  // costing more than their faster reverse sweeps save
  if (const int64_t ch = solve_chunk(ctx->ws, c, n, n_save, rtol, false))
    return solve_grad_chunked(ctx->ws, c, n, ch, params, y0, t0, t1, save_t, n_save, rtol, atol,
                              (cudaStream_t)stream, loss_out, params_bar, y0_bar, traj_status, false);
  return solve_grad_in(ctx->ws, c, n, params, y0, shared_w, t0, t1, save_t, n_save, rtol, atol,
                       (cudaStream_t)stream, loss_out, params_bar, y0_bar, shared_w_bar, traj_status, false);
}

gs_status gs_record_bytes(const gs_record* rec, size_t* bytes) {
  if (!rec || !bytes) return GS_ERR_INVALID_ARG;
  *bytes = rec->bytes;
  return GS_OK;
}

gs_status gs_record_stats(const gs_record* rec, int64_t* n, int64_t* accepted, int64_t* attempted) {
  if (!rec) return GS_ERR_INVALID_ARG;
  if (n) *n = rec->n;
  if (!accepted && !attempted) return GS_OK;
  std::vector<int32_t> S(rec->n), A(rec->n);
  if (rec->n > 0) {
    if (cudaMemcpy(S.data(), rec->S, rec->n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(A.data(), rec->natt, rec->n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return GS_ERR_CUDA;
  }
  int64_t sa = 0, sb = 0;
  for (int64_t i = 0; i < rec->n; ++i) { sa += S[i]; sb += A[i]; }
  if (accepted) *accepted = sa;
  if (attempted) *attempted = sb;
  return GS_OK;
}

gs_status gs_record_export_mesh(const gs_record* rec, int64_t* offsets, double* h) {
  if (!rec || !offsets) return GS_ERR_INVALID_ARG;
  const int64_t n = rec->n;
  std::vector<int32_t> S(n), st(n);
  std::vector<long long> head(n);
  if (n > 0) {
    if (cudaMemcpy(S.data(), rec->S, n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(head.data(), rec->head, n * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(st.data(), rec->status, n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return GS_ERR_CUDA;
  }
  offsets[0] = 0;
  for (int64_t i = 0; i < n; ++i) offsets[i + 1] = offsets[i] + (st[i] == GS_TRAJ_OK ? S[i] : 0);
  if (!h || n == 0) return GS_OK;
  std::vector<double> arena((size_t)rec->arena_cap * rec->segw);
  if (cudaMemcpy(arena.data(), rec->arena, arena.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return GS_ERR_CUDA;
  for (int64_t i = 0; i < n; ++i) {
    if (st[i] != GS_TRAJ_OK) continue;
    // walk segments last to first; the last holds S - (nseg-1) k steps
    const int Sk = S[i];
    int m = Sk - ((Sk - 1) / rec->k) * rec->k;
    long long seg = head[i];
    int64_t end = offsets[i + 1];
    while (seg >= 0) {
      const double* sp = arena.data() + (size_t)seg * rec->segw;
      for (int j = m - 1; j >= 0; --j) h[--end] = sp[2 + rec->d + j];
      long long prev;
      std::memcpy(&prev, sp, sizeof(prev));
      seg = prev;
      m = rec->k;
    }
    if (end != offsets[i]) return GS_ERR_CUDA;  // inconsistent record
  }
  return GS_OK;
}

gs_status gs_record_free(gs_record* rec) {
  destroy(rec);
  return GS_OK;
}

}  // extern "C"
