// sgml_internal.cuh -- data layout shared by the host side (sgml_api.cu) and the device side
// (sgml_kernels.cu) of libsgml.  Not part of the public ABI.
//
// Memory layout in HBM (one allocation per pool, all problems of the batch back to back):
//   FP64 full-grid pools, N^d doubles per problem at ProblemDesc::off_full:
//     U (solution), F (source), SIG64 (sigma), A64 (per-node a); RESP (accumulated residual of the
//     mixed form, kept as an unevaluated sum hi + lo of two floats: 8 bytes per node)
//   cycle-precision level pools (T = double or float), per problem levels 0..n-1 back to back at
//   ProblemDesc::off_lvl[l], level l holding (2^(n-l)+1)^d nodes (the level-l subset of the single
//   grid stored compactly, row-major [z][y][x]):
//     E, E2 (Jacobi ping-pong of the correction e), B (value of E when last injected from below),
//     R (restricted residual pyramid), SIG (restricted sigma), Q (local step times kappa/(2H^2)),
//     A0 (per-node a, level 0 only).
// Every level array starts on a 256-byte boundary.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sgml {

constexpr int kMaxLevels = 13;  // n <= 12

enum Op : int {
  OP_RESTRICT = 0,
  OP_SWEEP = 1,
  OP_PROLONG = 2,
  OP_INJECT = 3,
  OP_MEAN_ROWS = 4,    // Eq. 10 problems: weighted row sums of u (trapezoid rule)
  OP_MEAN_REDUCE = 5,  // ... their total per problem, in a fixed order -> mean of u
  OP_MEAN_APPLY = 6    // ... u -= mean (Eq. 10's zero-mean solution)
};

// Phase flags
constexpr int kFinalVisit = 1;   // SWEEP: merged last level-0 visit (tooth 0 and the final visit)
constexpr int kFirstOfTooth = 2; // SWEEP: first visit of its tooth
constexpr int kInit = 4;         // PROLONG: first arrival at the target level in this cycle
constexpr int kPair = 8;         // SWEEP: sweeps `sweep` and `sweep + 1` of the visit, fused
constexpr int kTailStart = 16;   // RESTRICT into level n - 3 (3-D mixed form, one problem): one CTA runs
                                 //   this and the following phases up to prev_tooth (exclusive), which
                                 //   touch only the three coarsest levels, in shared memory (coarse tail)

// One step of the cycle's schedule; a grid-wide barrier follows each phase.
struct Phase {
  int op;
  int level;       // level whose nodes the phase writes
  int tooth;       // SWEEP: tooth nu1 of the visit; PROLONG / INJECT: tooth of the visit just ended
  int sweep;       // SWEEP: sweep index inside the visit
  int flags;
  int prev_tooth;  // PROLONG (not kInit): tooth of the last visit at the target level
};

struct ProblemDesc {
  int n;                // N = 2^n + 1 nodes per side at level 0
  int hetero;           // per-node SIG / Q arrays are used
  int a_per_node;       // A64 holds per-node a
  int face_type[6];     // 0 Dirichlet, 1 Neumann (-x,+x,-y,+y,-z,+z)
  double face_value[6]; // Dirichlet value or outward derivative
  double h;
  double a_scalar;
  long long off_full;              // element offset in the FP64 full-grid pools
  long long off_lvl[kMaxLevels];   // element offset of level l in the level pools
  double q_const[kMaxLevels];      // homogeneous problems: delta_tau * kappa / (2 H^2) per level
  double inv_c[kMaxLevels];        // 2 H^2 / kappa per level (the sweep's 1 / c)
  double c0;                       // kappa / (2 h^2) (the level-0 residual's factor)
  float inv_c_f[kMaxLevels];       // FP32 copies of inv_c, q_const, c0 and a_scalar (made on the host:
  float q_const_f[kMaxLevels];     //   a conversion per thread and tile would occupy the FP64 pipe)
  float c0_f, a_scalar_f;
  int project_mean;                // every face Neumann, a >= 0 constant: Eq. 10, zero-mean u
};

// Per-problem running state, written by CTA 0 of the cycle kernel between barriers.
struct ProblemState {
  double fnorm;           // max-norm normaliser of the residual
  double fnorm2;          // L2 normaliser
  double rmax_prev;       // max-norm of the latest residual (sets the next cast scale)
  double scale_used[2];   // scale of the residual cast in cycle c (slot c & 1)
  double inv_scale[2];    // 1 / scale_used (no FP64 division per tile)
  double next_scale;      // cast scale of the next cycle's residual (set by the check)
  float next_scale_f;     // FP32 copies of next_scale and inv_scale
  float inv_scale_f[2];
  double rel, rel_l2;     // latest relative residuals
  double rel_prev;
  int cycles;             // cycles completed since the last reset
  int status;             // sgml_status of the problem
  int grow;               // consecutive cycles with a growing residual
  int hist_len;           // entries of the history row written by the last launch
  double anchor_rel;      // relative residual at the last FP64 anchor (mixed form)
  int anchor_next;        // the next residual is an FP64 anchor (else the FP32-stencil recurrence)
  int last_anchor;        // cycle index of the last anchor in this launch
};

// Norm accumulators and the per-launch stop flag (zeroed by the host before every launch).
struct Accum {
  unsigned long long rmax_bits[2];
  double rsum2[2];
  unsigned long long fmax_bits;
  double fsum2;
  int done;               // the problem stopped in the current launch
  int pad;
};

struct GridSync {
  unsigned long long arrive;  // CTAs arrived at grid barriers so far (round r: r G .. (r + 1) G - 1)
  int error;                  // 1: a barrier timed out
  int active[2];              // any problem still active after the check of cycle c (slot c & 1)
  int pad[3];
};

// Work unit of the tiled phases.  3-D: the kTX x kTY columns starting at (x0, y0) of one level of
// problem b, planes z0 .. z0 + nz - 1 (the CTA marches in z).  2-D: the kTX x kTY nodes at (x0, y0).
// A CTA of kThreads threads covers a tile, two vertically adjacent columns per thread.
// The kernels are compiled once per tile width (namespaces sgml_t32: 32 x 16 tiles, sgml_t64: 64 x 8
// tiles; kTY = 2 * kThreads / kTX); the host picks one per grid (sgml_set_launch, autotuner).
constexpr int kThreads = 256;
struct TileTask {
  int b;
  short x0, y0, z0, nz;
};

struct KernelParams {
  int dim, batch, n_max;
  int mixed;
  const ProblemDesc* probs;
  ProblemState* state;
  Accum* accum;
  const Phase* phases;
  int nphases;
  const TileTask* tasks;         // column-tile pieces of every level
  const int* task_off;           // [kMaxLevels][gridDim.x + 1]: CTA c owns tasks[off[c] .. off[c + 1])
  const TileTask* tasks4;        // the same for the tiles of the four-row sweep (kTX x 4 kThreads / kTX)
  const int* task_off4;
  int quad_levels;               // levels 0 .. quad_levels - 1 sweep with four rows per thread
  const long long* row_prefix;   // [kMaxLevels][batch + 1] cumulative node-row counts per level
  int fresh;                     // lift u and measure f first
  int max_cycles;
  double tol;
  double kappa;                  // stencil constant (consistent or literal)
  double w_edge, w_corner;       // 1/sqrt(2), 1/sqrt(3)
  double omega;                  // delta_tau * D_i of the Jacobi-scaled step
  float w_edge_f, w_corner_f, one_m_omega_f;  // FP32 copies of w_edge, w_corner and 1 - omega
  int n_r;
  int pair_levels;               // levels 0 .. pair_levels - 1 run their sweeps in fused pairs (kPair)
  int tail_cta;                  // CTA that runs the coarse tail (kTailStart)
  GridSync* sync;
  unsigned long long timeout_ns;  // limit of every grid-barrier wait
  int withhold_barrier;          // test aid: CTA 0 withholds its arrival at this barrier (1-based; 0: never)
  double* hist;
  int hist_cap;
  double* rowsum;             // Eq. 10 projection: weighted level-0 row sums of u (row_prefix order)
  double* umean;              // ... and the mean of u per problem
  unsigned long long* diag;   // optional: diagnostic pseudo-residual bits, [batch][diag_cycles][kMaxLevels]
  int diag_cycles;
  unsigned long long* trace;  // optional: globaltimer after each barrier, [cycle][2 + nphases]
  int trace_cycles;
  double *U, *F, *SIG64, *A64;
  float2* RESP;    // accumulated residual of the mixed form, hi + lo float pairs (full grid)
  void *E, *E2, *B, *R, *SIG, *Q;
  void* A0;        // per-node a at level 0 in cycle precision (recurrence operand)
};

// Host-side launchers of the tile-independent kernels (defined once, in the 64-wide kernel unit).
cudaError_t launch_setup_level(int mixed, int dim, const ProblemDesc& P, int level, const double* sig_l,
                               const double* a_l, double kappa, double w_edge, double w_corner,
                               double theta_gain, void* SIG_T, void* Q_T, void* A_T, cudaStream_t s);
cudaError_t launch_restrict64(int dim, const double* src, int Ns, double* dst, int Nt, cudaStream_t s);
cudaError_t launch_residual64(int dim, const ProblemDesc& P, const double* U, const double* F,
                              const double* SIG64, const double* A64, double kappa, double w_edge,
                              double w_corner, double* r, cudaStream_t s);
cudaError_t launch_sigma_gradient(int dim, const ProblemDesc& P, const double* lam, const double* U,
                                  double kappa, double w_edge, double w_corner, double* g, cudaStream_t s);
cudaError_t launch_fill(double* dst, long long n, double v, cudaStream_t s);
// Pure-Neumann sources: v -= trapezoid mean of v (scratch: 257 device doubles; scratch[256] = the
// mean); v += sign * (*d_value).
cudaError_t launch_project_mean(int dim, int n, double* v, double* scratch, cudaStream_t s);
cudaError_t launch_add_scalar(double* v, long long n, const double* d_value, double sign, cudaStream_t s);

}  // namespace sgml

// Launchers of the tiled cycle kernels, one set per tile width.
#define SGML_TILED_LAUNCHERS(NS)                                                                          \
  namespace NS {                                                                                        \
  cudaError_t launch_cycle_kernel(const sgml::KernelParams& p, int precision_mixed, int dim, int blocks,  \
                                  int threads, cudaStream_t s);                                          \
  cudaError_t launch_phase_kernel(const sgml::KernelParams& p, int precision_mixed, int dim, int blocks,  \
                                  int threads, int which, int c, cudaStream_t s);                        \
  int cycle_kernel_occupancy(int precision_mixed, int dim, int threads, int* blocks_per_sm);            \
  size_t cycle_kernel_smem(int precision_mixed);                                                        \
  }
SGML_TILED_LAUNCHERS(sgml_t32)
SGML_TILED_LAUNCHERS(sgml_t64)
