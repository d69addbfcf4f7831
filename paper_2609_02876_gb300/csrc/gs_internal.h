// Internal interface between the C-ABI layer (gs_api.cu) and the kernel
// translation units. Not installed; no torch or Python types.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gs {

constexpr int MAX_SAVE_HOST = 256;
constexpr int KMAX_HOST = 32;  // largest checkpoint interval accepted by the ABI
// Largest stored-stage segment in doubles: the record kernel stages one segment
// per lane in shared memory (128 lanes).
constexpr int MAX_STAGE_SEGW = 72;
// Arena slots the record kernel reserves per warp at a time (FwdArgs::arena_block):
// one atomic per block instead of one per flush; at most arena_block - 1 slots
// per warp stay unused at the end.
constexpr int ARENA_BLOCK_HOST = 256;

// Doubles per compact record segment [prev, t_start, y_start[d], h[k]], rounded
// up to a 16-byte multiple for vector stores. (Rounding up to whole 64-byte
// blocks instead was measured 4% slower for the FP32-mixed Lorenz sweep.)
inline int segw_of(int d, int k) { return ((2 + d + k) + 1) & ~1; }

// Arguments of the record (forward) kernels. Passed by value.
struct FwdArgs {
  int64_t n;
  const double* params;  // [P][n]
  const double* y0;      // [d][n]
  const float* shared_w; // UDE weights or nullptr
  double t0, t1, rtol, atol, h0;
  int64_t max_steps;
  int n_save;
  double* y_save;        // [n_save][d][n] or nullptr
  int32_t* status;       // [n]
  int32_t* step_counts;  // [2][n] or nullptr
  // record
  double* arena;                  // segments of segw doubles
  long long arena_cap;            // segments
  unsigned long long* arena_top;  // segment allocation counter
  int* overflow;                  // set when arena_top passes arena_cap
  long long* head;                // [n] last segment of each trajectory (-1 if none)
  int32_t* S;                     // [n] accepted steps
  int32_t* natt;                  // [n] attempted steps
  double* y_final;                // [d][n] state at t1
  unsigned long long* work;       // trajectory ticket counter
  int* any_failed;                // set when a trajectory ends with a non-OK status
  int k;                          // accepted steps per segment
  int segw;                       // doubles per segment
  int arena_block;                // slots a warp reserves at a time (>= 32; 0 means ARENA_BLOCK_HOST)
  // Stored stages (k = 1, FP64): each segment also holds its step's stage
  // data after h (Tsit5: Y_1..Y_5; Verner7: Y_1..Y_8; Rodas5P: U_0..U_7 and
  // the LU of W with pivot reciprocals and pivots; Rosenbrock23: k1, u2 and the
  // LU of W), and side_stg (n x n_save x payload doubles; layout: side_blocks
  // in gs_kernels.cuh) receives the same for every save-time side step (plus
  // its save state for the explicit methods).
  int stages;
  double* side_stg;
  int control;  // 1: FP64 step control (GS_CONTROL_FP64)
  int h0_pre;   // set by the launcher: 1: y_final[k] holds trajectory k's starting step until k ends;
                // 2: head[k] holds it (as bits) and y_final[., k] the method's carry f(y0)
  double save_t[MAX_SAVE_HOST];
};

// Arguments of the reverse kernels.
struct RevArgs {
  int64_t n;
  const double* params;
  const float* shared_w;
  float* shared_w_bar;
  double t0, t1;
  int n_save;
  const double* y_save_bar;  // [n_save][d][n] or nullptr (built-in loss)
  double* loss;              // [n] or nullptr
  double* params_bar;        // [P][n] or nullptr
  double* y0_bar;            // [d][n] or nullptr
  void* wpart;               // per-warp weight-gradient partials of shared-weight problems
                             // ([warps][354] floats for the LV UDE, [warps][353] doubles for the neural Robertson)
  const int32_t* status;     // [n] recorded status
  const double* arena;
  long long arena_cap;       // segments (bounds every segment index read)
  const long long* head;
  const int32_t* S;
  const double* y_final;
  unsigned long long* work;
  int k, segw;
  int stages;                // the record holds stage inputs (see FwdArgs)
  const double* side_stg;
  int* tc_error;             // set when a tensor-core product's completion wait ran out (or nullptr)
  int t1_pre;                // set by the launcher: y0_bar (and loss) hold lambda (and the loss) after
                             // the save at t1, which the reverse sweep then starts from
  double save_t[MAX_SAVE_HOST];
};

// Arguments of the forward-mode (tangent) replay kernels. Direction q of a
// launch is direction dir0 + q of the call.
struct JvpArgs {
  int64_t n;
  const double* params;      // [P][n]
  const double* y0;          // [d][n]
  const double* params_dot;  // [ND][P][n] of this launch, or nullptr (zero); unused when basis
  const double* y0_dot;      // [ND][d][n] of this launch, or nullptr (zero); unused when basis
  int basis;                 // 1: direction g is the unit vector g of (theta, y0), g = dir0 + q
  int dir0, nd;              // first direction of this launch, directions in it
  double t0, t1;
  int n_save;
  double* loss;              // [n] or nullptr
  double* loss_dot;          // [ND][n] of this launch (not basis), or nullptr
  double* y_save_dot;        // [ND][n_save][d][n] of this launch (not basis), or nullptr
  double* grad_p;            // basis: [P][n] or nullptr
  double* grad_y;            // basis: [d][n] or nullptr
  const int32_t* status;
  const double* arena;
  const int32_t* S;
  const long long* fwd_base;  // [n] first entry of each trajectory in fwd_seg (-1: unusable)
  const long long* fwd_seg;   // segment indices of every trajectory in forward order
  unsigned long long* work;
  int k, segw;
  double save_t[MAX_SAVE_HOST];
};

constexpr int JVP_MAX_DIR = 3;  // tangent directions carried by one launch

// The record's segments in forward order: for every trajectory k with status
// OK, fwd_seg[fwd_base[k] + i] is its i-th segment (fwd_base[k] = -1 if not
// OK or if its chain leaves the arena). `top` is a zeroed counter; cap the
// capacity of fwd_seg.
cudaError_t launch_fwd_index(int64_t n, const long long* head, const int32_t* S, const int32_t* status,
                             const double* arena, long long arena_cap, int k, int segw, unsigned long long* top,
                             long long* fwd_base, long long* fwd_seg, long long cap, cudaStream_t s);

// Forward-mode replay: method GS_METHOD_TSIT5 (1), GS_METHOD_RODAS5P (2), GS_METHOD_ROSENBROCK23 (3) or
// GS_METHOD_VERNER7 (4).
bool jvp_supports(int method, int problem);
cudaError_t launch_jvp(int method, int problem, const JvpArgs& a, cudaStream_t s);

struct LaunchCfg {
  int blocks;
  int threads;
  size_t smem;
};

// Launchers (one per method family). Return cudaSuccess or the launch error.
// problem: GS_* id; precision: 0 FP64, 1 FP32-mixed; saves: write y_save.
cudaError_t launch_tsit5_forward(int problem, int precision, const FwdArgs& a, cudaStream_t s);
cudaError_t launch_tsit5_reverse(int problem, int precision, const RevArgs& a, cudaStream_t s);
bool tsit5_supports(int problem, int precision);
cudaError_t launch_rodas_forward(int problem, int precision, const FwdArgs& a, cudaStream_t s);
cudaError_t launch_rodas_reverse(int problem, int precision, const RevArgs& a, cudaStream_t s);
bool rodas_supports(int problem, int precision);
cudaError_t launch_ros23_forward(int problem, int precision, const FwdArgs& a, cudaStream_t s);
cudaError_t launch_ros23_reverse(int problem, int precision, const RevArgs& a, cudaStream_t s);
bool ros23_supports(int problem, int precision);
cudaError_t launch_ros23_refresh(int problem, int precision, const RevArgs& a, double* arena, double* y_final,
                                 const double* y0, cudaStream_t s);
cudaError_t launch_vern7_forward(int problem, int precision, const FwdArgs& a, cudaStream_t s);
cudaError_t launch_vern7_reverse(int problem, int precision, const RevArgs& a, cudaStream_t s);
bool vern7_supports(int problem, int precision);
cudaError_t launch_vern7_refresh(int problem, int precision, const RevArgs& a, double* arena, double* y_final,
                                 const double* y0, cudaStream_t s);
// Frozen-mesh refresh: re-run each trajectory's state chain over its recorded
// mesh with a.params and y0, rewriting the record's states and y(t1).
cudaError_t launch_tsit5_refresh(int problem, int precision, const RevArgs& a, double* arena, double* y_final,
                                 const double* y0, cudaStream_t s);
cudaError_t launch_rodas_refresh(int problem, int precision, const RevArgs& a, double* arena, double* y_final,
                                 const double* y0, cudaStream_t s);
// Upper bound on the warps of a persistent reverse grid (the number of
// per-warp weight-gradient partials a shared-weight problem can produce).
int ude_max_warps();
constexpr int UDE_NW_HOST = 354;
constexpr int NR_NW_HOST = 353;
// Bytes of one warp's weight-gradient partial, the largest over the shared-weight problems.
constexpr size_t WPART_BYTES_PER_WARP = (UDE_NW_HOST * 4 > NR_NW_HOST * 8) ? UDE_NW_HOST * 4 : NR_NW_HOST * 8;

}  // namespace gs
