/*
 * gradsolve-gb300 C-ABI: record-and-replay gradients of ODE ensembles on one GPU.
 *
 * The method (paper Sec. 3.1, "The construction"): every trajectory of an
 * ensemble dy/dt = f(t, y, theta) gets its own adaptive solve (the record, map
 * R) that keeps its accepted step sizes {h_i}; the gradient is the exact
 * reverse-mode derivative of the fixed chain y_i = Phi(y_{i-1}; h_i, theta)
 * (Eq. (replay)) over that frozen mesh, with h held as data.
 *
 * Conventions shared by every entry point:
 *  - Array pointers are DEVICE pointers owned by the caller, laid out
 *    structure-of-arrays with the trajectory index fastest:
 *      params[P][n], y0[d][n], y_save[n_save][d][n], params_bar[P][n],
 *      y0_bar[d][n], loss[n], traj_status[n].
 *    save_t (n_save doubles) is a HOST pointer; its values are copied.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is
 *    enqueued on it; the calls that report per-trajectory failures
 *    (gs_forward_record, gs_solve_grad) synchronise `stream` before returning.
 *  - No exception, abort or device trap crosses this boundary: every failure is
 *    a gs_status return value. Per-trajectory failures are written to
 *    traj_status (GS_TRAJ_*) and the call returns GS_ERR_TRAJ_FAILED; the
 *    gradients of a failed trajectory are NaN.
 *  - Problem ids name the paper's test problems (Appendix A) plus two forms of
 *    this library: GS_LINEAR (dy/dt = A y, A = [[p0, p1], [p2, p3]], a closed-
 *    form test problem) and GS_LV_UDE (Lotka-Volterra with a shared MLP);
 *    GS_NEURAL_ROBERTSON is the paper's Robertson neural right-hand side.
 */
#ifndef GRADSOLVE_GS_H
#define GRADSOLVE_GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gs_record gs_record; /* opaque, device-resident, owned by the library */
typedef void* gs_stream;            /* a cudaStream_t */

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1,     /* a pointer, size, time span, tolerance or option is invalid */
  GS_ERR_UNKNOWN_PROBLEM = 2, /* problem id not in the registry */
  GS_ERR_OOM = 3,             /* device allocation failed */
  GS_ERR_CUDA = 4,            /* a CUDA launch or runtime call failed */
  GS_ERR_TRAJ_FAILED = 5,     /* at least one trajectory's traj_status is not GS_TRAJ_OK */
  GS_ERR_TIMEOUT = 6          /* a bounded wait on device completion ran out */
} gs_status;

/* Per-trajectory status words. */
enum {
  GS_TRAJ_OK = 0,
  GS_TRAJ_MAXSTEPS = 1,     /* attempted steps reached gs_options.max_steps */
  GS_TRAJ_DT_UNDERFLOW = 2, /* |h| < 1e-14 max(1, |t|) */
  GS_TRAJ_NONFINITE = 3,    /* non-finite input, or the error estimate stayed non-finite */
  GS_TRAJ_SINGULAR = 4      /* the Rosenbrock matrix I/(h gamma) - J stayed singular */
};

/* Problem registry (paper Appendix A; GS_LINEAR and GS_LV_UDE are this library's). */
enum {
  GS_LORENZ = 0,
  GS_VDP = 1,
  GS_ROBERTSON = 2,
  GS_HIRES = 3,
  GS_LINEAR = 4,
  GS_LV_UDE = 5,
  /* Robertson with k2 y2^2 replaced by a shared MLP 3-16-16-1 (tanh, softplus
   * output) in its sink and source (paper Appendix A); theta = (k1, k3), 353
   * shared weights (FP32 in shared_w, FP64 in the kernels), stiff, FP64 only,
   * Rodas5P or Rosenbrock23; shared_w_bar is the ensemble sum in FP32. */
  GS_NEURAL_ROBERTSON = 6
};

/* Arithmetic of the stage and adjoint work. GS_FP32_MIXED keeps t and h in
 * FP64; how the error norm and the controller are evaluated is gs_options.control. */
enum { GS_FP64 = 0, GS_FP32_MIXED = 1 };

/* Evaluation of the step-size control (the error norm, the accept test, the
 * controller factor and the starting step of the paper's Sec. 2.1), which only
 * chooses the mesh: the gradient is exact on whatever mesh is recorded.
 *  GS_CONTROL_FAST (default): the forms' cheap evaluation. FP64: each norm
 *    ratio e_c / (atol + rtol max(|y_c|, |ynew_c|)) to FP32 accuracy, squares
 *    summed in FP64; controller factor and starting step in FP32 with the
 *    hardware log2/exp2. FP32-mixed: the whole norm in FP32.
 *  GS_CONTROL_FP64: norm, accept test, controller (0.9 err^(-1/(q+1))
 *    clamped to [0.2, 10]), starting step and the step-size floor test all in
 *    FP64 arithmetic: reciprocals and the controller's root to about 1e-14
 *    and 1e-12 relative (single-precision estimates refined by FP64 Newton
 *    steps), the starting step with IEEE division, square root and pow. The
 *    recorded mesh then follows a plain CPU implementation's to the rounding
 *    of the stage sums. Tsit5 only (no shared-weight problems); other methods
 *    return GS_ERR_INVALID_ARG. */
enum { GS_CONTROL_FAST = 0, GS_CONTROL_FP64 = 1 };

/* One-step methods (paper Sec. 3.2): Tsit5 (Tsitouras 2011) for non-stiff
 * problems, Rodas5P (Steinebach 2023) for stiff ones, the second-order
 * Rosenbrock23 (Shampine & Reichelt 1997, the ode23s formulas) for stiff
 * ones on request, and the seventh-order Verner pair (Sec. 5, higher-order
 * engines; a 10-stage 7(6) table of Verner's structure, FP64, non-stiff
 * problems: Lorenz, Van der Pol, the linear test problem) on request. AUTO
 * picks Tsit5 or Rodas5P by problem. */
enum {
  GS_METHOD_AUTO = 0,
  GS_METHOD_TSIT5 = 1,
  GS_METHOD_RODAS5P = 2,
  GS_METHOD_ROSENBROCK23 = 3,
  GS_METHOD_VERNER7 = 4
};

typedef struct {
  int precision;        /* GS_FP64 or GS_FP32_MIXED */
  int method;           /* GS_METHOD_* */
  int ckpt_k;           /* accepted steps per record segment = state-checkpoint interval,
                           1..32; 0 picks 14 - d (a 128-byte segment) */
  int64_t max_steps;    /* attempted steps per trajectory; 0 = 1000000 */
  double h0;            /* first trial step; 0 = the automatic starting-step algorithm */
  int32_t* step_counts; /* optional DEVICE [2][n] output: accepted, attempted steps */
  float* kernel_ms;     /* optional HOST [2] output of gs_forward_record / gs_solve_grad:
                           device time (ms) of the record kernel and of the reverse kernel
                           (gs_solve_grad only) of this call, from CUDA events on `stream` */
  double timeout_ms;    /* bound on each host wait of gs_solve_grad / gs_solve_grad_ctx;
                           0 = no bound. When it runs out the call returns GS_ERR_TIMEOUT
                           while its work continues on `stream`: synchronise `stream`
                           before using the outputs or calling the library again */
  int32_t* record_info; /* optional HOST [2] output of gs_forward_record / gs_solve_grad /
                           gs_solve_grad_ctx: the record's checkpoint interval k, and 1 if
                           the record also stored every step's stage data (gs_solve_grad
                           chooses that layout in FP64 for Tsit5, Verner7, Rodas5P and
                           Rosenbrock23 when the segment is small enough (not HIRES) and
                           the device memory allows; the reverse sweep then reads the
                           stages instead of recomputing them, with identical results),
                           else 0 */
  int control;          /* GS_CONTROL_FAST or GS_CONTROL_FP64 */
  int record_stages;    /* gs_forward_record only: 1 lets the record also store every step's
                           stage data when gs_solve_grad would (same rule: method, FP64, segment
                           size, free memory), so that gs_reverse recomputes no stage; such a
                           record cannot be refreshed (gs_record_refresh returns
                           GS_ERR_INVALID_ARG). 0 (default): the compact record */
} gs_options;

/* A readable name for a status code (static storage, never NULL). */
const char* gs_status_string(gs_status s);

/* Fills *opt with the defaults (FP64, AUTO method, automatic k and h0). */
gs_status gs_default_options(gs_options* opt);

/* State dimension d, parameter count P, stiffness flag and shared-weight count
 * of a problem (paper Appendix A). */
gs_status gs_problem_info(int problem_id, int* d, int* P, int* stiff, int* n_shared);

/*
 * Record (map R, paper Sec. 3.1): the adaptive solve of every trajectory from
 * t0 to t1 with the weighted RMS error test of Sec. 2.1 (accept iff
 * RMS(e / (atol + rtol max(|y|, |y_new|))) <= 1) and an integral controller.
 * Keeps each trajectory's accepted step sizes plus a state checkpoint every
 * ckpt_k accepted steps in a device-resident record (*rec_out).
 *
 * save_t: n_save strictly increasing HOST times with t0 < save_t[0] and
 * save_t[n_save-1] <= t1 (n_save may be 0, at most 256). Each y(t_s) is one
 * extra step from the last mesh point at or before t_s (paper Sec. 3.4); save
 * times never alter the mesh. y_save_out [n_save][d][n] may be NULL.
 * shared_w: the network weights of GS_LV_UDE (354 floats) or
 * GS_NEURAL_ROBERTSON (353 floats), device, else NULL.
 * traj_status [n] is required. Synchronises `stream`. The record stays valid
 * until gs_record_free and may be replayed any number of times.
 */
gs_status gs_forward_record(int problem_id, int64_t n, const double* params, const double* y0,
                            const float* shared_w, double t0, double t1, const double* save_t, int n_save,
                            double rtol, double atol, const gs_options* opt, gs_stream stream,
                            double* y_save_out, int32_t* traj_status, gs_record** rec_out);

/*
 * Reverse sweep (paper Sec. 3.1-3.2): the discrete adjoint of the replay over
 * the recorded mesh with h held as data. For each trajectory, segments are
 * visited last to first; states inside a segment are recomputed from its
 * checkpoint, stages are recomputed per step, and the stage cotangents are
 * propagated back (for the Rosenbrock methods with one transposed LU solve per
 * stage). (gs_solve_grad's own record may instead hold the stage data, which
 * its reverse sweep reads rather than recomputes; see record_info.)
 *
 * params (and shared_w) must be the values the record's states were computed
 * with: those of gs_forward_record, or those of the last gs_record_refresh.
 * y_save_bar [n_save][d][n] is dL/dy(t_s); NULL selects the built-in loss
 * L = sum_k sum_s ||y_k(t_s)||^2, whose per-trajectory values are written to
 * loss_out [n] if it is not NULL. Outputs params_bar [P][n] and y0_bar [d][n]
 * (either may be NULL); shared_w_bar (the shared-weight problems only) receives the
 * ensemble sum. Enqueued on `stream`, not synchronised.
 */
gs_status gs_reverse(const gs_record* rec, const double* params, const double* y0, const float* shared_w,
                     const double* y_save_bar, double* loss_out, double* params_bar, double* y0_bar,
                     float* shared_w_bar, gs_stream stream);

/*
 * Frozen-mesh reuse (paper Sec. 3.1): re-runs every trajectory's replay chain
 * y_i = Phi(y_{i-1}; h_i, theta) over its recorded mesh with new params [P][n],
 * y0 [d][n] (and shared_w for the shared-weight problems), replacing the record's states. A
 * following gs_reverse with the same params returns the derivative at theta on
 * the mesh R(theta_0) that was recorded, d Psi(theta; sg[R(theta_0)]) / d theta,
 * as a fitting loop that reuses one record needs. The mesh, the save times and
 * the trajectory status words are unchanged; a step whose linear system is
 * singular at the new parameters leaves that trajectory's y(t1) NaN (its
 * gradient is then NaN). Enqueued on `stream`, not synchronised. A record that
 * stores stage data (gs_options.record_stages) is refused with
 * GS_ERR_INVALID_ARG: its stages belong to the recorded parameters.
 */
gs_status gs_record_refresh(gs_record* rec, const double* params, const double* y0, const float* shared_w,
                            gs_stream stream);

/*
 * Forward mode of the replay (paper Sec. 5, forward mode for few inputs): the
 * replay chain y_i = Phi(y_{i-1}; h_i, theta) is re-run from y0 over the
 * record's mesh (h held as data) with tangents carried alongside, giving for
 * each direction (params_dot, y0_dot) the directional derivative of the
 * built-in loss L = sum_s ||y(t_s)||^2 and of the save-time states. One pass
 * moves the same direction index of every trajectory at once.
 *
 * params [P][n], y0 [d][n]: the point of evaluation (any values: the mesh is
 * the record's, the states are recomputed). n_dir >= 1 directions, laid out
 * direction-major: params_dot [n_dir][P][n] and y0_dot [n_dir][d][n] (either
 * may be NULL: a zero tangent). Outputs: loss_dot [n_dir][n] (required),
 * loss_out [n] and y_save_dot [n_dir][n_save][d][n] (either may be NULL).
 * Trajectories whose record is not GS_TRAJ_OK, or whose linear system turns
 * singular, get NaN. Lorenz, Van der Pol and GS_LINEAR (Tsit5, Verner7),
 * Robertson, HIRES and GS_LINEAR (Rodas5P, Rosenbrock23) records;
 * GS_ERR_INVALID_ARG for others.
 * FP64 whatever the record's precision. The first forward-mode call on a
 * record allocates and fills an index of its segments in forward order (8
 * bytes per segment and per trajectory, then included in gs_record_bytes).
 * Enqueued on `stream`, not synchronised.
 */
gs_status gs_replay_jvp(const gs_record* rec, const double* params, const double* y0, int n_dir,
                        const double* params_dot, const double* y0_dot, double* loss_out, double* loss_dot,
                        double* y_save_dot, gs_stream stream);

/*
 * The gradient of the built-in loss by forward mode: gs_replay_jvp along the
 * unit directions of theta (when params_bar [P][n] is not NULL) and of y0
 * (when y0_bar [d][n] is not NULL), P and/or d passes (three directions per
 * kernel launch). Equal to gs_reverse's gradient up to rounding. At least one
 * of params_bar and y0_bar is required; loss_out [n] may be NULL. Enqueued on
 * `stream`, not synchronised.
 */
gs_status gs_forward_grad(const gs_record* rec, const double* params, const double* y0, double* loss_out,
                          double* params_bar, double* y0_bar, gs_stream stream);

/*
 * Record then reverse in one call with the built-in loss (the hot path):
 * loss_out [n], params_bar [P][n], y0_bar [d][n], traj_status [n]. The record
 * lives in a library-owned workspace that is reused by later calls on the same
 * device. Large calls run in chunks through device staging, with a record
 * sized for one chunk (no shared weights, no step_counts, no timeout_ms): an
 * FP32-mixed call of more than 2^22 trajectories in chunks of 2^21; an FP64
 * call whose stored-stage record would not fit in device memory but a chunk's
 * would, in the largest power-of-two chunks (2^18 to 2^23) that fit. Every
 * result equals the one-piece call's bit for bit, kernel_ms sums the chunks'
 * kernel times and record_info describes the last chunk. Synchronises
 * `stream`.
 */
gs_status gs_solve_grad(int problem_id, int64_t n, const double* params, const double* y0,
                        const float* shared_w, double t0, double t1, const double* save_t, int n_save,
                        double rtol, double atol, const gs_options* opt, gs_stream stream, double* loss_out,
                        double* params_bar, double* y0_bar, float* shared_w_bar, int32_t* traj_status);

/*
 * gs_solve_grad from HOST memory, end to end: params [P][n] and y0 [d][n] are
 * read from, and loss_out [n], params_bar [P][n], y0_bar [d][n] and
 * traj_status [n] written to, HOST arrays (page-locked memory lets the copies
 * run asynchronously; pageable memory works, slower). loss_out, params_bar and
 * y0_bar may be NULL (not written); traj_status is required. shared_w and
 * shared_w_bar stay DEVICE pointers (shared-weight problems).
 * The ensemble is solved in chunks of `chunk` trajectories (0: 2^21) on the
 * library's own streams, with the copy of chunk c + 1 to the device and of
 * chunk c - 1 back to the host overlapping the solve of chunk c. Trajectories
 * are independent, so every per-trajectory result equals gs_solve_grad's on
 * the whole ensemble bit for bit. Shared-weight problems run as one chunk
 * (their weight gradient sums the whole ensemble). opt->step_counts must be
 * NULL; opt->kernel_ms and opt->record_info describe the last chunk.
 * Device memory: the gs_solve_grad workspace (sized for one chunk) plus four
 * chunk staging buffers, kept per device for later calls. Synchronous: returns
 * when every output is in host memory; GS_ERR_TRAJ_FAILED as gs_solve_grad.
 */
gs_status gs_solve_grad_host(int problem_id, int64_t n, const double* params, const double* y0,
                             const float* shared_w, double t0, double t1, const double* save_t, int n_save,
                             double rtol, double atol, const gs_options* opt, int64_t chunk, double* loss_out,
                             double* params_bar, double* y0_bar, float* shared_w_bar, int32_t* traj_status);

/*
 * Forward-only solve (paper Sec. 2.1, the adaptive solve of map R without a
 * record): the same accepted mesh, save states and statuses as
 * gs_forward_record, bit for bit, but nothing is stored for a reverse sweep.
 * Arguments as gs_forward_record; y_save_out [n_save][d][n] may be NULL;
 * y_final_out [d][n] (device) receives y(t1) and traj_status [n] (device) the
 * trajectory status, both required when n > 0; y_final_out may be the y0
 * buffer itself (y0 is then replaced by y(t1)). Before its trajectory ends,
 * y_final_out's first row holds the trajectory's starting step. ckpt_k is
 * ignored.
 * Uses only the small counter block of the per-device workspace of
 * gs_solve_grad (no record arena). Synchronises `stream`; returns
 * GS_ERR_TRAJ_FAILED if any trajectory ended with a non-OK status.
 */
gs_status gs_solve(int problem_id, int64_t n, const double* params, const double* y0, const float* shared_w,
                   double t0, double t1, const double* save_t, int n_save, double rtol, double atol,
                   const gs_options* opt, gs_stream stream, double* y_save_out, double* y_final_out,
                   int32_t* traj_status);

/*
 * gs_solve_grad without any device allocation. This entry point has no
 * counterpart in the paper; it exists for callers that cannot call cudaMalloc:
 * for example a process that has handed all free device memory to another
 * framework's caching allocator, or a latency-critical thread that must not
 * pay for, or block on, allocation and the device synchronisation that
 * cudaFree implies. Arguments, layouts and results are those of gs_solve_grad.
 *
 * Scratch: the record lives in one fixed array of GS_NOALLOC_SCRATCH_BYTES
 * (32 MiB) that the library declares as a static device object; every GPU that
 * loads the library holds it until the process exits. Nothing is allocated
 * per call (no cudaMalloc / cudaFree / allocating library routine).
 * Limits: n <= GS_NOALLOC_MAX_TRAJ (16384); a larger n returns
 * GS_ERR_INVALID_ARG before any work. If an ensemble's record does not fit the
 * array (more accepted steps than it holds), the call returns GS_ERR_OOM and
 * its outputs are undefined: split the ensemble.
 * The first call made on a device resolves the array's device address
 * (cudaGetSymbolAddress) for that device; make that first call before any
 * stream capture. Every call shares the one array and overwrites what the
 * previous call left in it: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * Synchronises `stream`. Only Tsit5 problems without shared weights: a
 * shared-weight problem (n_shared > 0, the LV UDE) returns GS_ERR_INVALID_ARG
 * before any work; shared_w and shared_w_bar are not used.
 */
#define GS_NOALLOC_MAX_TRAJ 16384
#define GS_NOALLOC_SCRATCH_BYTES (32u << 20)
gs_status gs_solve_grad_noalloc(int problem_id, int64_t n, const double* params, const double* y0,
                                const float* shared_w, double t0, double t1, const double* save_t, int n_save,
                                double rtol, double atol, const gs_options* opt, gs_stream stream,
                                double* loss_out, double* params_bar, double* y0_bar, float* shared_w_bar,
                                int32_t* traj_status);

/*
 * Solve contexts for concurrent callers (the request server). A context owns
 * its own reusable record workspace on the device that was current when it was
 * created; gs_solve_grad_ctx is gs_solve_grad on that workspace, except that it
 * always records compactly (no stored stages), so calls on different contexts
 * and streams proceed concurrently (calls on one context are serialised by the
 * context). gs_context_bytes reports the device bytes the workspace holds (it
 * grows to the largest ensemble seen).
 */
typedef struct gs_context gs_context;
gs_status gs_context_create(gs_context** ctx);
gs_status gs_context_destroy(gs_context* ctx);
gs_status gs_context_bytes(const gs_context* ctx, size_t* bytes);
gs_status gs_solve_grad_ctx(gs_context* ctx, int problem_id, int64_t n, const double* params, const double* y0,
                            const float* shared_w, double t0, double t1, const double* save_t, int n_save,
                            double rtol, double atol, const gs_options* opt, gs_stream stream, double* loss_out,
                            double* params_bar, double* y0_bar, float* shared_w_bar, int32_t* traj_status);

/* Device bytes held by a record. */
gs_status gs_record_bytes(const gs_record* rec, size_t* bytes);

/* Ensemble size and total accepted / attempted steps of a record. */
gs_status gs_record_stats(const gs_record* rec, int64_t* n, int64_t* accepted, int64_t* attempted);

/* Copies the mesh to HOST arrays: offsets [n+1] (ragged prefix sums of the
 * accepted-step counts) and h [offsets[n]]. Pass h = NULL to get offsets only.
 * Synchronous. Meant for tests and inspection. */
gs_status gs_record_export_mesh(const gs_record* rec, int64_t* offsets, double* h);

/* Releases a record (NULL is accepted). */
gs_status gs_record_free(gs_record* rec);

/*
 * Measured FMA throughput of the current device, in TFLOP/s (an FMA counts
 * two flops): the denominator of the ALU roofline fractions of the record and
 * reverse kernels, whose work is scalar FP64 or FP32 arithmetic per lane (the
 * paper's method has no dense contraction outside the neural right-hand
 * sides). kind 0: FP64 FMA; 1: FP32 FMA; 2: packed FP32x2 FMA (two single
 * FMAs per instruction). A full-occupancy grid of independent FMA chains,
 * best of five ~40 ms launches on the legacy default stream, which the call
 * synchronises. Allocates and frees a small output buffer. Not part of the
 * solve path.
 */
gs_status gs_measure_fma_peak(int kind, double* tflops);

#ifdef __cplusplus
}
#endif

#endif /* GRADSOLVE_GS_H */
