// sgml_api.cu -- host side of libsgml: the C ABI declared in include/sgml.h.
//
// The grid object owns every device buffer (layout in sgml_internal.cuh), the schedule of one
// cycle (Algorithm 3) as a table of phases, and the launch shape of the persistent cooperative
// cycle kernel.  Solves run as one kernel launch each; coefficient pyramids (restricted sigma and a,
// Algorithm 1 applied to coefficients, and the local pseudo-time steps, Sec. 2 and Sec. 3.4) are
// rebuilt by small setup kernels when the coefficients change.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sgml.h"
#include "sgml_internal.cuh"
#include "sgml_schedule.h"
#include "sgml_tasks.h"

using namespace sgml;

static thread_local std::string g_last_error;

static int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define SGML_CUDA(call)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(SGML_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct sgml_grid {
  int dim = 2, batch = 0, mixed = 0, elem = 8;
  cudaStream_t stream = nullptr;
  int device = 0, sms = 0;
  std::vector<ProblemDesc> P;
  std::vector<long long> M0;
  int n_max = 0;
  // device state
  ProblemDesc* d_probs = nullptr;
  ProblemState* d_state = nullptr;
  Accum* d_accum = nullptr;
  GridSync* d_sync = nullptr;
  Phase* d_phases = nullptr;
  int nphases = 0;
  std::vector<Phase> h_phases;  // host copy of the uploaded phase table
  size_t phases_cap = 0;        // capacity of d_phases in entries
  long long* d_rows = nullptr;
  TileTask* d_tasks = nullptr;
  int* d_task_off = nullptr;
  TileTask* d_tasks4 = nullptr;  // tiles of the four-row sweep
  int* d_task_off4 = nullptr;
  double* d_hist = nullptr;
  int hist_cap = 0;
  double *U = nullptr, *F = nullptr, *SIG64 = nullptr, *A64 = nullptr;
  double* pyr64 = nullptr;     // FP64 scratch of the coefficient pyramid (levels >= 1), kept between builds
  long long pyr64_cap = 0;     // its size in doubles
  float2* RESP = nullptr;  // mixed form: accumulated residual as hi + lo float pairs
  void* A0 = nullptr;
  void *E = nullptr, *E2 = nullptr, *B = nullptr, *R = nullptr, *SIG = nullptr, *Q = nullptr;
  long long full_total = 0, lvl_total = 0;
  // parameters
  int n_r = 2;
  double theta = 0.7;
  int stencil = SGML_STENCIL_CONSISTENT;
  int max_cycles = 200;
  int threads = kThreads, ctas_per_sm = 0, blocks = 0, z_waves = 1;
  int tile_x = 64;  // 32 (32 x 16 tiles) or 64 (64 x 8 tiles)
  int slab_z = 32;  // slab height of the slab cut of large 3-D levels (0: contiguous runs only)
  int pair_levels = 0;  // levels whose sweeps run in fused pairs (3-D mixed form only; off by default)
  int quad_levels = 0;  // levels whose sweeps run four rows per thread (3-D mixed form only; off by default)
  bool coarse_tail = true;  // 3-D mixed form, one problem: one CTA runs the three coarsest levels' phases
  int tail_cta = 0;         // ... the last CTA without tiles on the levels around the tail (its SM's
                            //     instruction cache then holds the tail's code, not the next phases')
  int mode = 0;  // 0: one persistent cooperative launch per call, 1: one launch per phase
  unsigned long long timeout_ns = 2000000000ull;  // limit of every grid-barrier wait (2 s)
  int withhold_barrier = 0;  // test aid: CTA 0 withholds its arrival at this barrier (0: never)
  bool dirty_coeffs = true, dirty_desc = true, dirty_phases = true, dirty_tiles = true, fresh = true;
  long long launches = 0;
  ProblemState* h_state = nullptr;  // pinned
  double* d_rowsum = nullptr;             // pure-Neumann projection: level-0 row sums of u
  double* d_umean = nullptr;              // ... mean of u per problem
  double* d_fmean = nullptr;              // ... source projection scratch (257 doubles per problem)
  std::vector<double> f_shift;            // mean already subtracted from each problem's F
  std::vector<char> f_checked;            // F's projection matches the current boundary conditions
  unsigned long long* d_diag = nullptr;   // diagnostic pseudo-residuals (sgml_set_diagnostics)
  int diag_cycles = 0;
  double* d_scratch = nullptr;            // staging of host arrays for sgml_residual / sgml_sigma_gradient
  long long scratch_cap = 0;              // ... its size in doubles (grown once, then reused)
  unsigned long long* d_trace = nullptr;  // per-phase timestamps (sgml_set_trace)
  int trace_cycles = 0;
  int trace_last_cycles = 0;
};

// Tiled kernels of the grid's tile width.
static cudaError_t launch_cycle(sgml_grid* g, const KernelParams& p) {
  return g->tile_x == 32 ? sgml_t32::launch_cycle_kernel(p, g->mixed, g->dim, g->blocks, kThreads, g->stream)
                         : sgml_t64::launch_cycle_kernel(p, g->mixed, g->dim, g->blocks, kThreads, g->stream);
}
static cudaError_t launch_phase(sgml_grid* g, const KernelParams& p, int which, int c) {
  return g->tile_x == 32 ? sgml_t32::launch_phase_kernel(p, g->mixed, g->dim, g->blocks, kThreads, which, c, g->stream)
                         : sgml_t64::launch_phase_kernel(p, g->mixed, g->dim, g->blocks, kThreads, which, c, g->stream);
}
static int occupancy(sgml_grid* g, int* bps) {
  return g->tile_x == 32 ? sgml_t32::cycle_kernel_occupancy(g->mixed, g->dim, kThreads, bps)
                         : sgml_t64::cycle_kernel_occupancy(g->mixed, g->dim, kThreads, bps);
}

// ------------------------------------------------------------------------------------------------
// Constants of the radial stencil (Eq. 5)
// ------------------------------------------------------------------------------------------------
static double w_edge() { return 1.0 / std::sqrt(2.0); }
static double w_corner() { return 1.0 / std::sqrt(3.0); }

// sum_o w_o over the 8 / 26 neighbours
static double weight_sum(int dim) {
  return dim == 3 ? 6.0 + 12.0 * w_edge() + 8.0 * w_corner() : 4.0 + 4.0 * w_edge();
}

// sum_o w_o o_1^2
static double weight_moment(int dim) {
  return dim == 3 ? 2.0 + 8.0 * w_edge() + 8.0 * w_corner() : 2.0 + 4.0 * w_edge();
}

static double kappa_of(int dim, int stencil) {
  if (stencil == SGML_STENCIL_LITERAL) return dim == 3 ? 3.0 / 13.0 : 0.5;
  return 2.0 / weight_moment(dim);
}

// delta_tau * D_i of the Jacobi-scaled step for theta = 1: kappa_consistent * S / 2.
static double jacobi_gain(int dim) { return (2.0 / weight_moment(dim)) * weight_sum(dim) / 2.0; }

static long long side(int n, int l) { return (1LL << (n - l)) + 1; }
static long long nodes(int dim, int n, int l) {
  long long N = side(n, l);
  return dim == 3 ? N * N * N : N * N;
}
static long long round_up(long long x, long long a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------------------------------------------
// Schedule of one cycle (Algorithm 3): build_phases in sgml_schedule.h.
// ------------------------------------------------------------------------------------------------
// Coarse tail (see kTailStart): 3-D mixed form, one problem of at least four levels, persistent
// launch, no diagnostics, and no fused pairs or four-row tiles on the tail levels.
static int effective_pair_levels(const sgml_grid* g);
static int effective_quad_levels(const sgml_grid* g);
static bool uses_tail(const sgml_grid* g) {
  const int lt = g->n_max - 3;
  return g->coarse_tail && g->dim == 3 && g->mixed && g->batch == 1 && g->n_max >= 4 && !g->d_diag && g->mode == 0 &&
         effective_pair_levels(g) <= lt && effective_quad_levels(g) <= lt;
}

// Eq. 10 problems: every face Neumann and a >= 0 constant (a < 0 everywhere is well posed as is).
static bool projects_mean(const sgml_grid* g, const ProblemDesc& P) {
  for (int k = 0; k < 2 * g->dim; ++k)
    if (P.face_type[k] != SGML_NEUMANN) return false;
  return !P.a_per_node && P.a_scalar >= 0.0;
}

static bool any_projects_mean(const sgml_grid* g) {
  for (const ProblemDesc& P : g->P)
    if (projects_mean(g, P)) return true;
  return false;
}

// Fused pairs and four-row tiles: 3-D mixed form only, and not while diagnostics are recorded
// (only the single-sweep kernels compute the pseudo-residual).
static int effective_pair_levels(const sgml_grid* g) {
  return (g->dim == 3 && g->mixed && !g->d_diag) ? g->pair_levels : 0;
}
static int effective_quad_levels(const sgml_grid* g) {
  return (g->dim == 3 && g->mixed && !g->d_diag) ? g->quad_levels : 0;
}

static int upload_phases(sgml_grid* g) {
  std::vector<Phase> ph = build_phases(g->n_max, g->n_r, effective_pair_levels(g), any_projects_mean(g), uses_tail(g));
  const bool same = g->d_phases && ph.size() == g->h_phases.size() &&
                    std::memcmp(ph.data(), g->h_phases.data(), sizeof(Phase) * ph.size()) == 0;
  if (!same) {  // (re)upload only a changed table, reallocating only when it grew
    if (ph.size() > g->phases_cap) {
      if (g->d_phases) SGML_CUDA(cudaFree(g->d_phases));
      g->d_phases = nullptr;
      g->phases_cap = 0;
      SGML_CUDA(cudaMalloc(&g->d_phases, sizeof(Phase) * std::max<size_t>(ph.size(), 1)));
      g->phases_cap = ph.size();
    }
    SGML_CUDA(cudaMemcpyAsync(g->d_phases, ph.data(), sizeof(Phase) * ph.size(), cudaMemcpyHostToDevice, g->stream));
    SGML_CUDA(cudaStreamSynchronize(g->stream));
    g->h_phases = ph;
  }
  g->nphases = (int)ph.size();
  g->dirty_phases = false;
  return SGML_OK;
}

// Work tables: column tiles of every level (3-D: z cut into chunks so that each level has about
// z_waves tiles per CTA) and the prefix of node rows per level.
static int upload_tiles(sgml_grid* g) {
  int bps = 0;
  if (occupancy(g, &bps) != 0 || bps < 1)
    return fail(SGML_ERR_CUDA, "occupancy query failed for the cycle kernel");
  if (g->ctas_per_sm > 0) bps = std::min(bps, g->ctas_per_sm);
  g->blocks = g->sms * bps;
  std::vector<long long> rp((size_t)kMaxLevels * (g->batch + 1), 0);
  std::vector<int> nb(g->batch), dir_hi(g->batch);
  for (int b = 0; b < g->batch; ++b) {
    nb[b] = g->P[b].n;
    dir_hi[b] = (g->P[b].face_type[1] == SGML_DIRICHLET ? 1 : 0) | (g->P[b].face_type[3] == SGML_DIRICHLET ? 2 : 0);
  }
  for (int l = 0; l < kMaxLevels; ++l)
    for (int b = 0; b < g->batch; ++b) {
      const int n = g->P[b].n;
      const long long N = side(n, std::min(l, n - 1));
      const long long rows = (l <= n - 1) ? (g->dim == 3 ? N * N : N) : 0;
      rp[(size_t)l * (g->batch + 1) + b + 1] = rp[(size_t)l * (g->batch + 1) + b] + rows;
    }
  // z_waves equal pieces per CTA: piece j goes to CTA j mod G (z_waves = 1: one contiguous share each)
  // (the slab cut deals its pieces to the CTAs itself: z_waves does not apply)
  const int G = g->blocks, W = g->slab_z > 0 ? 1 : g->z_waves, Gp = G * W;
  auto partition = [&](int tx, int ty, std::vector<TileTask>& tasks, std::vector<int>& toff) {
    std::vector<TileTask> pieces((size_t)partition_bound(g->dim, nb.data(), g->batch, Gp, tx, ty, g->slab_z));
    std::vector<int> poff((size_t)kMaxLevels * (Gp + 1));
    pieces.resize(build_partition(g->dim, nb.data(), dir_hi.data(), g->batch, Gp, tx, ty, pieces.data(),
                                  poff.data(), g->slab_z));
    tasks.clear();
    tasks.reserve(pieces.size());
    toff.assign((size_t)kMaxLevels * (G + 1), 0);
    for (int l = 0; l < kMaxLevels; ++l) {
      const int* po = poff.data() + (size_t)l * (Gp + 1);
      int* o = toff.data() + (size_t)l * (G + 1);
      for (int c = 0; c < G; ++c) {
        o[c] = (int)tasks.size();
        for (int w = 0; w < W; ++w) {
          const int j = c + w * G;
          for (int t = po[j]; t < po[j + 1]; ++t) tasks.push_back(pieces[t]);
        }
      }
      o[G] = (int)tasks.size();
    }
  };
  std::vector<TileTask> tasks, tasks4;
  std::vector<int> toff, toff4;
  partition(g->tile_x, 2 * kThreads / g->tile_x, tasks, toff);
  g->tail_cta = pick_tail_cta(toff, G, g->n_max);
  if (effective_quad_levels(g) > 0) partition(g->tile_x, 4 * kThreads / g->tile_x, tasks4, toff4);
  if (g->d_rows) SGML_CUDA(cudaFree(g->d_rows));
  if (g->d_tasks) SGML_CUDA(cudaFree(g->d_tasks));
  if (g->d_task_off) SGML_CUDA(cudaFree(g->d_task_off));
  if (g->d_tasks4) SGML_CUDA(cudaFree(g->d_tasks4));
  if (g->d_task_off4) SGML_CUDA(cudaFree(g->d_task_off4));
  g->d_rows = nullptr;
  g->d_tasks = nullptr;
  g->d_task_off = nullptr;
  g->d_tasks4 = nullptr;
  g->d_task_off4 = nullptr;
  SGML_CUDA(cudaMalloc(&g->d_rows, sizeof(long long) * rp.size()));
  SGML_CUDA(cudaMalloc(&g->d_tasks, sizeof(TileTask) * std::max<size_t>(tasks.size(), 1)));
  SGML_CUDA(cudaMalloc(&g->d_task_off, sizeof(int) * toff.size()));
  SGML_CUDA(cudaMemcpyAsync(g->d_rows, rp.data(), sizeof(long long) * rp.size(), cudaMemcpyHostToDevice, g->stream));
  SGML_CUDA(cudaMemcpyAsync(g->d_tasks, tasks.data(), sizeof(TileTask) * tasks.size(), cudaMemcpyHostToDevice, g->stream));
  SGML_CUDA(cudaMemcpyAsync(g->d_task_off, toff.data(), sizeof(int) * toff.size(), cudaMemcpyHostToDevice, g->stream));
  if (!tasks4.empty()) {
    SGML_CUDA(cudaMalloc(&g->d_tasks4, sizeof(TileTask) * tasks4.size()));
    SGML_CUDA(cudaMalloc(&g->d_task_off4, sizeof(int) * toff4.size()));
    SGML_CUDA(cudaMemcpyAsync(g->d_tasks4, tasks4.data(), sizeof(TileTask) * tasks4.size(), cudaMemcpyHostToDevice,
                              g->stream));
    SGML_CUDA(cudaMemcpyAsync(g->d_task_off4, toff4.data(), sizeof(int) * toff4.size(), cudaMemcpyHostToDevice,
                              g->stream));
  }
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  g->dirty_tiles = false;
  return SGML_OK;
}

static int ensure_hetero_pools(sgml_grid* g, bool need_a) {
  if (!g->SIG64) {
    SGML_CUDA(cudaMalloc(&g->SIG64, sizeof(double) * g->full_total));
    SGML_CUDA(cudaMalloc(&g->SIG, (size_t)g->elem * g->lvl_total));
    SGML_CUDA(cudaMalloc(&g->Q, (size_t)g->elem * g->lvl_total));
    SGML_CUDA(cudaMemsetAsync(g->SIG, 0, (size_t)g->elem * g->lvl_total, g->stream));
    SGML_CUDA(cudaMemsetAsync(g->Q, 0, (size_t)g->elem * g->lvl_total, g->stream));
  }
  if (need_a && !g->A64) {
    SGML_CUDA(cudaMalloc(&g->A64, sizeof(double) * g->full_total));
    SGML_CUDA(cudaMemsetAsync(g->A64, 0, sizeof(double) * g->full_total, g->stream));
    SGML_CUDA(cudaMalloc(&g->A0, (size_t)g->elem * g->lvl_total));
    SGML_CUDA(cudaMemsetAsync(g->A0, 0, (size_t)g->elem * g->lvl_total, g->stream));
  }
  return SGML_OK;
}

// FP32 copies of the per-level constants (the kernels of the mixed form read them directly).
static void fill_float_copies(ProblemDesc& P) {
  for (int l = 0; l < kMaxLevels; ++l) P.inv_c_f[l] = (float)P.inv_c[l], P.q_const_f[l] = (float)P.q_const[l];
  P.c0_f = (float)P.c0;
  P.a_scalar_f = (float)P.a_scalar;
}

// Coefficient pyramid: restricted sigma / a and the local steps of every level (setup, excluded
// from the solve).  Homogeneous problems get one constant per level computed here.
static int build_coeffs(sgml_grid* g) {
  const double kap = kappa_of(g->dim, g->stencil);
  const double tg = g->theta * jacobi_gain(g->dim);
  // FP64 scratch for the restricted sigma / a of every heterogeneous problem's levels >= 1, allocated
  // once (re-setting coefficients, e.g. every step of an end-to-end loop, then costs no allocation)
  long long need = 0;
  for (const ProblemDesc& P : g->P)
    if (P.hetero)
      for (int l = 1; l <= P.n - 1; ++l) need += nodes(g->dim, P.n, l) * (P.a_per_node ? 2 : 1);
  if (need > g->pyr64_cap) {
    if (g->pyr64) SGML_CUDA(cudaFree(g->pyr64));
    g->pyr64 = nullptr;
    g->pyr64_cap = 0;
    SGML_CUDA(cudaMalloc(&g->pyr64, sizeof(double) * need));
    g->pyr64_cap = need;
  }
  double* next = g->pyr64;
  for (int b = 0; b < g->batch; ++b) {
    ProblemDesc& P = g->P[b];
    for (int l = 0; l < kMaxLevels; ++l) P.q_const[l] = 0.0, P.inv_c[l] = 0.0;
    P.c0 = kap / (2.0 * P.h * P.h);
    for (int l = 0; l <= P.n - 1; ++l) {
      const double H = P.h * (double)(1LL << l);
      P.inv_c[l] = 2.0 * H * H / kap;
      const double c = kap / (2.0 * H * H);
      const double D = c * 2.0 * weight_sum(g->dim) - P.a_scalar;
      P.q_const[l] = tg / D * c;
    }
    fill_float_copies(P);
    if (!P.hetero) continue;
    // level pyramid of sigma (and a) in FP64 temporaries
    std::vector<double*> sig(P.n, nullptr), av(P.n, nullptr);
    sig[0] = g->SIG64 + P.off_full;
    av[0] = P.a_per_node ? g->A64 + P.off_full : nullptr;
    for (int l = 1; l <= P.n - 1; ++l) {
      const long long M = nodes(g->dim, P.n, l);
      sig[l] = next;
      next += M;
      SGML_CUDA(launch_restrict64(g->dim, sig[l - 1], (int)side(P.n, l - 1), sig[l], (int)side(P.n, l), g->stream));
      g->launches++;
      if (P.a_per_node) {
        av[l] = next;
        next += M;
        SGML_CUDA(launch_restrict64(g->dim, av[l - 1], (int)side(P.n, l - 1), av[l], (int)side(P.n, l), g->stream));
        g->launches++;
      }
    }
    for (int l = 0; l <= P.n - 1; ++l) {
      SGML_CUDA(launch_setup_level(g->mixed, g->dim, P, l, sig[l], av[l], kap, w_edge(), w_corner(), tg, g->SIG, g->Q,
                                   (l == 0 && P.a_per_node) ? g->A0 : nullptr, g->stream));
      g->launches++;
    }
  }
  g->dirty_coeffs = false;
  g->dirty_desc = true;
  return SGML_OK;
}

static int upload_desc(sgml_grid* g) {
  for (ProblemDesc& P : g->P) P.project_mean = projects_mean(g, P) ? 1 : 0;
  SGML_CUDA(cudaMemcpyAsync(g->d_probs, g->P.data(), sizeof(ProblemDesc) * g->batch, cudaMemcpyHostToDevice, g->stream));
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  g->dirty_desc = false;
  return SGML_OK;
}

// Eq. 10 problems solve L u = f - <f>: the mean of F is subtracted (and added back if the problem
// later stops being one); their faces must carry zero derivatives.
static int project_sources(sgml_grid* g) {
  const bool any = any_projects_mean(g);
  if (any && !g->d_rowsum) {
    long long rows = 0;
    for (const ProblemDesc& P : g->P) rows += g->dim == 3 ? (long long)side(P.n, 0) * side(P.n, 0) : side(P.n, 0);
    SGML_CUDA(cudaMalloc(&g->d_rowsum, sizeof(double) * rows));
    SGML_CUDA(cudaMalloc(&g->d_umean, sizeof(double) * g->batch));
    SGML_CUDA(cudaMalloc(&g->d_fmean, sizeof(double) * 257 * g->batch));
  }
  for (int b = 0; b < g->batch; ++b) {
    if (g->f_checked[b]) continue;
    ProblemDesc& P = g->P[b];
    const bool pn = projects_mean(g, P);
    if (pn)
      for (int k = 0; k < 2 * g->dim; ++k)
        if (P.face_value[k] != 0.0)
          return fail(SGML_ERR_ARG, "an all-Neumann problem with a >= 0 needs zero normal derivatives (Eq. 10)");
    double* F = g->F + P.off_full;
    double* scr = g->d_fmean + (size_t)257 * b;
    if (pn) {
      SGML_CUDA(launch_project_mean(g->dim, P.n, F, scr, g->stream));
      double m = 0.0;
      SGML_CUDA(cudaMemcpyAsync(&m, scr + 256, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
      SGML_CUDA(cudaStreamSynchronize(g->stream));
      g->f_shift[b] += m;
      g->launches += 3;
    } else if (g->f_shift[b] != 0.0) {
      SGML_CUDA(cudaMemcpyAsync(scr + 256, &g->f_shift[b], sizeof(double), cudaMemcpyHostToDevice, g->stream));
      SGML_CUDA(launch_add_scalar(F, nodes(g->dim, P.n, 0), scr + 256, 1.0, g->stream));
      SGML_CUDA(cudaStreamSynchronize(g->stream));
      g->f_shift[b] = 0.0;
      g->launches += 1;
    }
    g->f_checked[b] = 1;
  }
  return SGML_OK;
}

static int prepare(sgml_grid* g) {
  int st;
  if (g->dirty_coeffs && (st = build_coeffs(g)) != SGML_OK) return st;
  if ((st = project_sources(g)) != SGML_OK) return st;
  if (g->dirty_desc && (st = upload_desc(g)) != SGML_OK) return st;
  if (g->dirty_phases && (st = upload_phases(g)) != SGML_OK) return st;
  if (g->dirty_tiles && (st = upload_tiles(g)) != SGML_OK) return st;
  return SGML_OK;
}

static int ensure_hist(sgml_grid* g, int cap) {
  if (cap <= g->hist_cap) return SGML_OK;
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  if (g->d_hist) SGML_CUDA(cudaFree(g->d_hist));
  g->hist_cap = std::max(cap, 256);
  SGML_CUDA(cudaMalloc(&g->d_hist, sizeof(double) * (size_t)g->hist_cap * g->batch));
  SGML_CUDA(cudaMemsetAsync(g->d_hist, 0, sizeof(double) * (size_t)g->hist_cap * g->batch, g->stream));
  return SGML_OK;
}

// One launch of the persistent cycle kernel: up to max_cycles cycles per problem, stopping a
// problem when its relative residual reaches tol (tol < 0: never).
static int launch(sgml_grid* g, int max_cycles, double tol) {
  int st;
  if ((st = prepare(g)) != SGML_OK) return st;
  if ((st = ensure_hist(g, max_cycles + 1)) != SGML_OK) return st;
  const bool fresh = g->fresh;
  SGML_CUDA(cudaMemsetAsync(g->d_accum, 0, sizeof(Accum) * g->batch, g->stream));
  SGML_CUDA(cudaMemsetAsync(g->d_sync, 0, sizeof(GridSync), g->stream));
  if (fresh) SGML_CUDA(cudaMemsetAsync(g->d_state, 0, sizeof(ProblemState) * g->batch, g->stream));
  KernelParams p;
  std::memset(&p, 0, sizeof(p));
  p.dim = g->dim;
  p.batch = g->batch;
  p.n_max = g->n_max;
  p.mixed = g->mixed;
  p.probs = g->d_probs;
  p.state = g->d_state;
  p.accum = g->d_accum;
  p.phases = g->d_phases;
  p.nphases = g->nphases;
  p.tasks = g->d_tasks;
  p.task_off = g->d_task_off;
  p.tasks4 = g->d_tasks4;
  p.task_off4 = g->d_task_off4;
  p.quad_levels = g->d_tasks4 ? effective_quad_levels(g) : 0;
  p.row_prefix = g->d_rows;
  p.fresh = fresh ? 1 : 0;
  p.max_cycles = max_cycles;
  p.tol = tol;
  p.kappa = kappa_of(g->dim, g->stencil);
  p.w_edge = w_edge();
  p.w_corner = w_corner();
  p.omega = g->theta * jacobi_gain(g->dim);
  p.w_edge_f = (float)p.w_edge;
  p.w_corner_f = (float)p.w_corner;
  p.one_m_omega_f = (float)(1.0 - p.omega);
  p.n_r = g->n_r;
  p.pair_levels = effective_pair_levels(g);
  p.tail_cta = g->tail_cta;
  p.sync = g->d_sync;
  p.timeout_ns = g->timeout_ns;
  p.withhold_barrier = g->withhold_barrier;
  p.hist = g->d_hist;
  p.hist_cap = g->hist_cap;
  p.trace = g->d_trace;
  p.trace_cycles = g->d_trace ? g->trace_cycles : 0;
  p.rowsum = g->d_rowsum;
  p.umean = g->d_umean;
  p.diag = g->d_diag;
  p.diag_cycles = g->d_diag ? g->diag_cycles : 0;
  if (g->d_diag)
    SGML_CUDA(cudaMemsetAsync(g->d_diag, 0, sizeof(unsigned long long) * (size_t)g->batch * g->diag_cycles * kMaxLevels,
                              g->stream));
  if (g->d_trace) {
    SGML_CUDA(cudaMemsetAsync(g->d_trace, 0, sizeof(unsigned long long) * (size_t)g->trace_cycles * (g->nphases + 3), g->stream));
    g->trace_last_cycles = std::min(g->trace_cycles, max_cycles + 1);
  }
  p.U = g->U;
  p.F = g->F;
  p.SIG64 = g->SIG64;
  p.A64 = g->A64;
  p.RESP = g->RESP;
  p.A0 = g->A0;
  p.E = g->E;
  p.E2 = g->E2;
  p.B = g->B;
  p.R = g->R;
  p.SIG = g->SIG;
  p.Q = g->Q;
  if (g->mode == 0) {
    SGML_CUDA(launch_cycle(g, p));
    g->launches++;
  } else {
    // one launch per phase: the same device code, kernel boundaries instead of grid barriers
    auto one = [&](int which, int c) -> cudaError_t {
      g->launches++;
      return launch_phase(g, p, which, c);
    };
    if (fresh) SGML_CUDA(one(-3, 0));
    for (int c = 0;; ++c) {
      SGML_CUDA(one(-2, c));
      SGML_CUDA(one(-1, c));
      if (c >= max_cycles) break;
      if (tol >= 0.0) {
        GridSync s;
        SGML_CUDA(cudaMemcpyAsync(&s, g->d_sync, sizeof(GridSync), cudaMemcpyDeviceToHost, g->stream));
        SGML_CUDA(cudaStreamSynchronize(g->stream));
        if (!s.active[c & 1]) break;
      }
      for (int q = 0; q < g->nphases; ++q) SGML_CUDA(one(q, c));
    }
  }
  g->fresh = false;
  return SGML_OK;
}

static int sync_and_check(sgml_grid* g) {
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  GridSync s;
  SGML_CUDA(cudaMemcpy(&s, g->d_sync, sizeof(GridSync), cudaMemcpyDeviceToHost));
  if (s.error) return fail(SGML_ERR_BARRIER_TIMEOUT, "a grid barrier of the cycle kernel timed out");
  SGML_CUDA(cudaMemcpy(g->h_state, g->d_state, sizeof(ProblemState) * g->batch, cudaMemcpyDeviceToHost));
  return SGML_OK;
}

static bool valid(sgml_grid* g) { return g != nullptr && g->batch > 0; }

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------
extern "C" {

int sgml_create_grid(int dim, int batch, const int* n_levels, int precision, void* cuda_stream, sgml_grid_t* out) {
  if (!out) return fail(SGML_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (dim != 2 && dim != 3) return fail(SGML_ERR_ARG, "dim must be 2 or 3");
  if (batch < 1 || batch > 65536 || !n_levels) return fail(SGML_ERR_ARG, "batch must be in 1..65536 with n_levels given");
  if (precision != SGML_FP64 && precision != SGML_MIXED) return fail(SGML_ERR_ARG, "precision must be SGML_FP64 or SGML_MIXED");
  const int nmax_allowed = dim == 3 ? 10 : 12;
  for (int b = 0; b < batch; ++b)
    if (n_levels[b] < 1 || n_levels[b] > nmax_allowed)
      return fail(SGML_ERR_ARG, "n_levels[b] out of range (1..12 in 2-D, 1..10 in 3-D)");
  sgml_grid* g = new sgml_grid();
  g->dim = dim;
  g->batch = batch;
  g->mixed = precision == SGML_MIXED;
  g->slab_z = g->mixed ? 32 : 0;  // the FP64 form is FP64-pipe bound: the slab cut's halo planes cost more than it saves
  g->elem = g->mixed ? 4 : 8;
  g->stream = (cudaStream_t)cuda_stream;
  g->P.resize(batch);
  g->f_shift.assign(batch, 0.0);
  g->f_checked.assign(batch, 0);
  long long full = 0, lvl = 0;
  for (int b = 0; b < batch; ++b) {
    ProblemDesc& P = g->P[b];
    std::memset(&P, 0, sizeof(P));
    P.n = n_levels[b];
    P.h = 1.0 / (double)((1LL << P.n));
    P.off_full = full;
    full += round_up(nodes(dim, P.n, 0), 32);
    for (int l = 0; l <= P.n - 1; ++l) {
      P.off_lvl[l] = lvl;
      lvl += round_up(nodes(dim, P.n, l), 64);
    }
    g->n_max = std::max(g->n_max, P.n);
  }
  g->full_total = full;
  g->lvl_total = lvl;
  auto cleanup = [&](int code, const std::string& m) {
    sgml_destroy(g);
    return fail(code, m);
  };
  cudaError_t e;
#define ALLOC(ptr, bytes)                                                      \
  if ((e = cudaMalloc((void**)&(ptr), (bytes))) != cudaSuccess) return cleanup(SGML_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e)); \
  if ((e = cudaMemsetAsync((ptr), 0, (bytes), g->stream)) != cudaSuccess) return cleanup(SGML_ERR_CUDA, cudaGetErrorString(e));
  if ((e = cudaGetDevice(&g->device)) != cudaSuccess) return cleanup(SGML_ERR_CUDA, cudaGetErrorString(e));
  if ((e = cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device)) != cudaSuccess)
    return cleanup(SGML_ERR_CUDA, cudaGetErrorString(e));
  ALLOC(g->U, sizeof(double) * full);
  ALLOC(g->F, sizeof(double) * full);
  if (g->mixed) {
    ALLOC(g->RESP, sizeof(float2) * full);
  }
  ALLOC(g->E, (size_t)g->elem * lvl);
  ALLOC(g->E2, (size_t)g->elem * lvl);
  ALLOC(g->B, (size_t)g->elem * lvl);
  ALLOC(g->R, (size_t)g->elem * lvl);
  ALLOC(g->d_probs, sizeof(ProblemDesc) * batch);
  ALLOC(g->d_state, sizeof(ProblemState) * batch);
  ALLOC(g->d_accum, sizeof(Accum) * batch);
  ALLOC(g->d_sync, sizeof(GridSync));
#undef ALLOC
  if ((e = cudaMallocHost(&g->h_state, sizeof(ProblemState) * batch)) != cudaSuccess)
    return cleanup(SGML_ERR_CUDA, cudaGetErrorString(e));
  std::memset(g->h_state, 0, sizeof(ProblemState) * batch);
  if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cleanup(SGML_ERR_CUDA, cudaGetErrorString(e));
  *out = g;
  return SGML_OK;
}

int sgml_set_params(sgml_grid_t g, int n_r, double theta, int schedule, int stencil, int dt_mode, int max_cycles) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (n_r < 1 || n_r > 64) return fail(SGML_ERR_ARG, "n_r must be in 1..64");
  if (!(theta > 0.0 && theta <= 2.0)) return fail(SGML_ERR_ARG, "theta must be in (0, 2]");
  if (schedule != 0) return fail(SGML_ERR_ARG, "only schedule 0 (zig-zag reading of Algorithm 3) is implemented");
  if (stencil != SGML_STENCIL_CONSISTENT && stencil != SGML_STENCIL_LITERAL) return fail(SGML_ERR_ARG, "bad stencil");
  if (dt_mode != 0) return fail(SGML_ERR_ARG, "only dt_mode 0 (Jacobi-scaled local step) is implemented");
  if (max_cycles < 0) return fail(SGML_ERR_ARG, "max_cycles must be >= 0");
  if (n_r != g->n_r) g->dirty_phases = true;
  if (theta != g->theta || stencil != g->stencil) g->dirty_coeffs = true;
  g->n_r = n_r;
  g->theta = theta;
  g->stencil = stencil;
  g->max_cycles = max_cycles;
  g->fresh = true;
  return SGML_OK;
}

int sgml_set_coeffs(sgml_grid_t g, int problem, const double* sigma, const double* a, double a_scalar) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (problem < -1 || problem >= g->batch) return fail(SGML_ERR_ARG, "problem out of range");
  if (!(a_scalar <= 1.0)) return fail(SGML_ERR_ARG, "a_scalar must be <= 1");
  int st;
  if ((sigma || a) && (st = ensure_hetero_pools(g, a != nullptr)) != SGML_OK) return st;
  long long src = 0;
  for (int b = (problem < 0 ? 0 : problem); b < (problem < 0 ? g->batch : problem + 1); ++b) {
    ProblemDesc& P = g->P[b];
    const long long M = nodes(g->dim, P.n, 0);
    P.hetero = (sigma || a) ? 1 : 0;
    P.a_per_node = a ? 1 : 0;
    P.a_scalar = a ? 0.0 : a_scalar;
    g->f_checked[b] = 0;
    if (sigma) SGML_CUDA(cudaMemcpyAsync(g->SIG64 + P.off_full, sigma + src, sizeof(double) * M, cudaMemcpyDefault, g->stream));
    else if (a) {
      SGML_CUDA(launch_fill(g->SIG64 + P.off_full, M, 1.0, g->stream));
      g->launches++;
    }
    if (a) SGML_CUDA(cudaMemcpyAsync(g->A64 + P.off_full, a + src, sizeof(double) * M, cudaMemcpyDefault, g->stream));
    src += M;
  }
  g->dirty_coeffs = true;
  g->dirty_desc = true;
  g->dirty_phases = true;  // the Eq. 10 projection phases depend on a
  g->fresh = true;
  return SGML_OK;
}

int sgml_set_source(sgml_grid_t g, int problem, const double* f) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (problem < -1 || problem >= g->batch || !f) return fail(SGML_ERR_ARG, "problem out of range or f NULL");
  long long src = 0;
  for (int b = (problem < 0 ? 0 : problem); b < (problem < 0 ? g->batch : problem + 1); ++b) {
    const long long M = nodes(g->dim, g->P[b].n, 0);
    SGML_CUDA(cudaMemcpyAsync(g->F + g->P[b].off_full, f + src, sizeof(double) * M, cudaMemcpyDefault, g->stream));
    src += M;
    g->f_shift[b] = 0.0;
    g->f_checked[b] = 0;
  }
  g->fresh = true;
  return SGML_OK;
}

int sgml_set_bc(sgml_grid_t g, int problem, const int* face_type, const double* face_value) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (problem < -1 || problem >= g->batch || !face_type) return fail(SGML_ERR_ARG, "problem out of range or face_type NULL");
  const int nf = 2 * g->dim;
  for (int k = 0; k < nf; ++k)
    if (face_type[k] != SGML_DIRICHLET && face_type[k] != SGML_NEUMANN) return fail(SGML_ERR_ARG, "bad face type");
  for (int b = (problem < 0 ? 0 : problem); b < (problem < 0 ? g->batch : problem + 1); ++b) {
    ProblemDesc& P = g->P[b];
    for (int k = 0; k < 6; ++k) {
      P.face_type[k] = k < nf ? face_type[k] : SGML_DIRICHLET;
      P.face_value[k] = (k < nf && face_value) ? face_value[k] : 0.0;
    }
    g->f_checked[b] = 0;
    // Nodes that become fixed must hold a zero correction and a zero residual (the sweeps and the
    // residual never write fixed nodes, and the stencils and restrictions of their neighbours read
    // them): clear the problem's level arrays.
    long long lvl = 0;
    for (int l = 0; l <= P.n - 1; ++l) lvl += round_up(nodes(g->dim, P.n, l), 64);
    const size_t off = (size_t)g->elem * P.off_lvl[0], bytes = (size_t)g->elem * lvl;
    for (void* a : {g->E, g->E2, g->B, g->R})
      SGML_CUDA(cudaMemsetAsync((char*)a + off, 0, bytes, g->stream));
  }
  g->dirty_desc = true;
  g->dirty_tiles = true;
  g->dirty_phases = true;  // the pure-Neumann projection phases
  g->fresh = true;
  return SGML_OK;
}

int sgml_run_cycle(sgml_grid_t g, int ncycles) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (ncycles < 0) return fail(SGML_ERR_ARG, "ncycles must be >= 0");
  return launch(g, ncycles, -1.0);
}

int sgml_solve_to_tol(sgml_grid_t g, double rtol, int* cycles_out, double* rel_res_out) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (!(rtol >= 0.0)) return fail(SGML_ERR_ARG, "rtol must be >= 0");
  g->fresh = true;
  int st = launch(g, g->max_cycles, rtol);
  if (st != SGML_OK) return st;
  if ((st = sync_and_check(g)) != SGML_OK) return st;
  int worst = SGML_OK;
  for (int b = 0; b < g->batch; ++b) {
    if (cycles_out) cycles_out[b] = g->h_state[b].cycles;
    if (rel_res_out) rel_res_out[b] = g->h_state[b].rel;
    if (g->h_state[b].status < worst) worst = g->h_state[b].status;
  }
  if (worst != SGML_OK) {
    char buf[128];
    std::snprintf(buf, sizeof(buf), "solve ended with status %d for at least one problem", worst);
    g_last_error = buf;
  }
  return worst;
}

int sgml_residual_norm(sgml_grid_t g, int norm, double* rel_out) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if ((norm != SGML_NORM_MAX && norm != SGML_NORM_L2) || !rel_out) return fail(SGML_ERR_ARG, "bad norm or rel_out NULL");
  int st = launch(g, 0, -1.0);
  if (st != SGML_OK) return st;
  if ((st = sync_and_check(g)) != SGML_OK) return st;
  for (int b = 0; b < g->batch; ++b) rel_out[b] = norm == SGML_NORM_MAX ? g->h_state[b].rel : g->h_state[b].rel_l2;
  return SGML_OK;
}

int sgml_get_solution(sgml_grid_t g, int problem, double* u) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (problem < 0 || problem >= g->batch || !u) return fail(SGML_ERR_ARG, "problem out of range or u NULL");
  const ProblemDesc& P = g->P[problem];
  SGML_CUDA(cudaMemcpyAsync(u, g->U + P.off_full, sizeof(double) * nodes(g->dim, P.n, 0), cudaMemcpyDefault, g->stream));
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  return SGML_OK;
}

int sgml_get_stats(sgml_grid_t g, int problem, int* cycles, double* rel_max, int* status) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (problem < 0 || problem >= g->batch) return fail(SGML_ERR_ARG, "problem out of range");
  int st = sync_and_check(g);
  if (st != SGML_OK) return st;
  if (cycles) *cycles = g->h_state[problem].cycles;
  if (rel_max) *rel_max = g->h_state[problem].rel;
  if (status) *status = g->h_state[problem].status;
  return SGML_OK;
}

int sgml_get_history(sgml_grid_t g, int problem, double* hist, int cap, int* count) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (problem < 0 || problem >= g->batch || !hist || cap < 0) return fail(SGML_ERR_ARG, "bad arguments");
  int st = sync_and_check(g);
  if (st != SGML_OK) return st;
  // the row holds the relative residual before each cycle of the last launch and after its last
  int n = std::min(std::min(cap, g->hist_cap), g->h_state[problem].hist_len);
  std::vector<double> row(g->hist_cap);
  SGML_CUDA(cudaMemcpy(row.data(), g->d_hist + (size_t)problem * g->hist_cap, sizeof(double) * g->hist_cap, cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) hist[i] = row[i];
  if (count) *count = n;
  return SGML_OK;
}

// Device memory the kernels can read directly: a device (or managed) pointer of the grid's device.
static bool device_resident(const sgml_grid* g, const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == g->device);
}

// Grid-owned staging area of at least `count` doubles (allocated once per size increase).
static int ensure_scratch(sgml_grid* g, long long count) {
  if (count <= g->scratch_cap) return SGML_OK;
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  if (g->d_scratch) SGML_CUDA(cudaFree(g->d_scratch));
  g->d_scratch = nullptr;
  g->scratch_cap = 0;
  SGML_CUDA(cudaMalloc(&g->d_scratch, sizeof(double) * count));
  g->scratch_cap = count;
  return SGML_OK;
}

// Node arrays of the per-problem FP64 kernels: device arrays are used in place, host arrays are
// staged through the grid's scratch (slot k of M doubles).
struct Staged {
  const double* in[2] = {nullptr, nullptr};
  double* out = nullptr;
  bool copy_out = false;
};

static int stage(sgml_grid* g, long long M, const double* a, const double* b, double* out, Staged& st) {
  const double* src[2] = {a, b};
  int need = 0;
  bool dev[3];
  for (int k = 0; k < 2; ++k) dev[k] = src[k] ? device_resident(g, src[k]) : true;
  dev[2] = device_resident(g, out);
  for (int k = 0; k < 3; ++k) need += dev[k] ? 0 : 1;
  int st_ = ensure_scratch(g, need * M);
  if (st_ != SGML_OK) return st_;
  int slot = 0;
  for (int k = 0; k < 2; ++k) {
    if (!src[k] || dev[k]) {
      st.in[k] = src[k];
      continue;
    }
    double* d = g->d_scratch + (long long)(slot++) * M;
    SGML_CUDA(cudaMemcpyAsync(d, src[k], sizeof(double) * M, cudaMemcpyDefault, g->stream));
    st.in[k] = d;
  }
  st.out = dev[2] ? out : g->d_scratch + (long long)(slot++) * M;
  st.copy_out = !dev[2];
  return SGML_OK;
}

int sgml_residual(sgml_grid_t g, int problem, const double* u, double* r) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (problem < 0 || problem >= g->batch || !u || !r) return fail(SGML_ERR_ARG, "bad arguments");
  int st;
  if ((st = project_sources(g)) != SGML_OK) return st;
  if (g->dirty_desc && (st = upload_desc(g)) != SGML_OK) return st;
  if (r == u) return fail(SGML_ERR_ARG, "r must not alias u");
  const ProblemDesc& P = g->P[problem];
  const long long M = nodes(g->dim, P.n, 0);
  Staged sg;
  if ((st = stage(g, M, u, nullptr, r, sg)) != SGML_OK) return st;
  SGML_CUDA(launch_residual64(g->dim, P, sg.in[0], g->F + P.off_full, g->SIG64 ? g->SIG64 + P.off_full : nullptr,
                              g->A64 ? g->A64 + P.off_full : nullptr, kappa_of(g->dim, g->stencil), w_edge(),
                              w_corner(), sg.out, g->stream));
  g->launches++;
  if (sg.copy_out) SGML_CUDA(cudaMemcpyAsync(r, sg.out, sizeof(double) * M, cudaMemcpyDefault, g->stream));
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  return SGML_OK;
}

int sgml_sigma_gradient(sgml_grid_t g, int problem, const double* lambda, const double* u, double* grad) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (problem < 0 || problem >= g->batch || !lambda || !u || !grad) return fail(SGML_ERR_ARG, "bad arguments");
  const ProblemDesc& P = g->P[problem];
  for (int k = 0; k < 2 * g->dim; ++k)
    if (P.face_type[k] != SGML_DIRICHLET) return fail(SGML_ERR_ARG, "the sigma gradient needs all faces Dirichlet");
  const long long M = nodes(g->dim, P.n, 0);
  if (grad == lambda || grad == u) return fail(SGML_ERR_ARG, "grad must not alias lambda or u");
  Staged sg;
  int st;
  if ((st = stage(g, M, lambda, u, grad, sg)) != SGML_OK) return st;
  SGML_CUDA(launch_sigma_gradient(g->dim, P, sg.in[0], sg.in[1], kappa_of(g->dim, g->stencil), w_edge(), w_corner(),
                                  sg.out, g->stream));
  g->launches++;
  if (sg.copy_out) SGML_CUDA(cudaMemcpyAsync(grad, sg.out, sizeof(double) * M, cudaMemcpyDefault, g->stream));
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  return SGML_OK;
}

int sgml_set_launch(sgml_grid_t g, int ctas_per_sm, int z_waves, int mode, int tile_x, int slab_z) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (ctas_per_sm < 0 || z_waves < 1 || z_waves > 64 || (mode != 0 && mode != 1) || (tile_x != 32 && tile_x != 64) ||
      slab_z < 0 || slab_z > 4096)
    return fail(SGML_ERR_ARG, "ctas_per_sm >= 0, z_waves in 1..64, mode 0 or 1, tile_x 32 or 64, slab_z in 0..4096");
  g->ctas_per_sm = ctas_per_sm;
  g->z_waves = z_waves;
  g->mode = mode;
  g->tile_x = tile_x;
  g->slab_z = slab_z;
  g->dirty_tiles = true;
  g->dirty_phases = true;  // the coarse tail runs in the persistent launch only
  return SGML_OK;
}

int sgml_set_coarse_tail(sgml_grid_t g, int on) {
  if (!valid(g) || (on != 0 && on != 1)) return fail(SGML_ERR_ARG, "invalid grid, or on not 0 / 1");
  g->coarse_tail = on != 0;
  g->dirty_phases = true;
  return SGML_OK;
}

int sgml_set_barrier_test(sgml_grid_t g, double wait_limit_s, int withhold_barrier) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (!(wait_limit_s >= 1e-4 && wait_limit_s <= 60.0) || withhold_barrier < 0)
    return fail(SGML_ERR_ARG, "wait_limit_s must be in [1e-4, 60] and withhold_barrier >= 0");
  g->timeout_ns = (unsigned long long)(wait_limit_s * 1e9);
  g->withhold_barrier = withhold_barrier;
  return SGML_OK;
}

int sgml_set_fusion(sgml_grid_t g, int pair_levels) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (pair_levels < 0 || pair_levels > kMaxLevels) return fail(SGML_ERR_ARG, "pair_levels must be in 0..13");
  g->pair_levels = pair_levels;
  g->dirty_phases = true;
  return SGML_OK;
}

int sgml_set_quad(sgml_grid_t g, int quad_levels) {
  if (!valid(g)) return fail(SGML_ERR_ARG, "invalid grid");
  if (quad_levels < 0 || quad_levels > kMaxLevels) return fail(SGML_ERR_ARG, "quad_levels must be in 0..13");
  g->quad_levels = quad_levels;
  g->dirty_tiles = true;
  g->dirty_phases = true;  // the coarse tail needs single sweeps on its levels
  return SGML_OK;
}

int sgml_get_phases(sgml_grid_t g, int* out, int cap, int* count) {
  if (!valid(g) || !count || (cap > 0 && !out)) return fail(SGML_ERR_ARG, "invalid grid or output");
  const std::vector<Phase> ph = build_phases(g->n_max, g->n_r, effective_pair_levels(g), any_projects_mean(g));
  *count = (int)ph.size();
  for (int q = 0; q < (int)ph.size() && q < cap; ++q) {
    out[4 * q + 0] = ph[q].op;
    out[4 * q + 1] = ph[q].level;
    out[4 * q + 2] = ph[q].sweep;
    out[4 * q + 3] = ph[q].op == OP_SWEEP ? ((ph[q].flags & kPair) ? 2 : 1) : 0;
  }
  return SGML_OK;
}

int sgml_set_trace(sgml_grid_t g, int cycles) {
  if (!valid(g) || cycles < 0 || cycles > 100000) return fail(SGML_ERR_ARG, "invalid grid or cycles");
  int st;
  if ((st = prepare(g)) != SGML_OK) return st;
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  if (g->d_trace) SGML_CUDA(cudaFree(g->d_trace));
  g->d_trace = nullptr;
  g->trace_cycles = cycles;
  if (cycles > 0) SGML_CUDA(cudaMalloc(&g->d_trace, sizeof(unsigned long long) * (size_t)cycles * (g->nphases + 3)));
  return SGML_OK;
}

int sgml_get_trace(sgml_grid_t g, double* us, int cap, int* nphases, int* ncycles) {
  if (!valid(g) || !us || !nphases || !ncycles) return fail(SGML_ERR_ARG, "bad arguments");
  if (g->mode != 0 || !g->d_trace) return fail(SGML_ERR_ARG, "tracing is off (sgml_set_trace) or the grid is in phase mode");
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  const int w = g->nphases + 3;
  std::vector<unsigned long long> t((size_t)g->trace_cycles * w);
  SGML_CUDA(cudaMemcpy(t.data(), g->d_trace, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost));
  // durations: slot k of cycle c is stamp(k) - stamp(k - 1); slot 0 of cycle c spans from the
  // previous cycle's last stamp (or is 0 for the first cycle)
  int n = 0;
  for (int c = 0; c < g->trace_last_cycles && (n + 1) * w <= cap; ++c) {
    if (t[(size_t)c * w] == 0) break;
    for (int k = 0; k < w; ++k) {
      const unsigned long long a = t[(size_t)c * w + k];
      const unsigned long long prev = k > 0 ? t[(size_t)c * w + k - 1] : 0;
      us[(size_t)n * w + k] = (a && prev && a >= prev) ? (double)(a - prev) * 1e-3 : 0.0;
    }
    ++n;
  }
  *nphases = w;
  *ncycles = n;
  return SGML_OK;
}

int sgml_set_diagnostics(sgml_grid_t g, int cycles) {
  if (!valid(g) || cycles < 0 || cycles > 100000) return fail(SGML_ERR_ARG, "invalid grid or cycles");
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  if (g->d_diag) SGML_CUDA(cudaFree(g->d_diag));
  g->d_diag = nullptr;
  g->diag_cycles = cycles;
  if (cycles > 0) {
    const size_t bytes = sizeof(unsigned long long) * (size_t)g->batch * cycles * kMaxLevels;
    SGML_CUDA(cudaMalloc(&g->d_diag, bytes));
    SGML_CUDA(cudaMemsetAsync(g->d_diag, 0, bytes, g->stream));
  }
  g->dirty_phases = true;  // pairs are not built while diagnostics are on
  g->dirty_tiles = true;
  return SGML_OK;
}

int sgml_get_diagnostics(sgml_grid_t g, int problem, double* out, int cap, int* cycles_out) {
  if (!valid(g) || problem < 0 || problem >= g->batch || !out || !cycles_out)
    return fail(SGML_ERR_ARG, "invalid grid, problem or output");
  if (!g->d_diag) return fail(SGML_ERR_ARG, "diagnostics are off (sgml_set_diagnostics)");
  SGML_CUDA(cudaStreamSynchronize(g->stream));
  std::vector<unsigned long long> bits((size_t)g->diag_cycles * kMaxLevels);
  SGML_CUDA(cudaMemcpy(bits.data(), g->d_diag + (size_t)problem * g->diag_cycles * kMaxLevels,
                       sizeof(unsigned long long) * bits.size(), cudaMemcpyDeviceToHost));
  const int n = std::min(g->diag_cycles, cap / kMaxLevels);
  for (int k = 0; k < n * kMaxLevels; ++k) {
    unsigned long long b = bits[k];
    double v;
    std::memcpy(&v, &b, sizeof(v));
    out[k] = v;
  }
  *cycles_out = n;
  return SGML_OK;
}

int sgml_get_launch_info(sgml_grid_t g, int* ctas, int* threads_per_cta, int* smem_bytes) {
  if (!valid(g) || !ctas || !threads_per_cta || !smem_bytes) return fail(SGML_ERR_ARG, "invalid grid or NULL output");
  int st;
  if ((st = prepare(g)) != SGML_OK) return st;
  *ctas = g->blocks;
  *threads_per_cta = kThreads;
  *smem_bytes = (int)(g->tile_x == 32 ? sgml_t32::cycle_kernel_smem(g->mixed) : sgml_t64::cycle_kernel_smem(g->mixed));
  return SGML_OK;
}

int sgml_launch_count(sgml_grid_t g, long long* count) {
  if (!valid(g) || !count) return fail(SGML_ERR_ARG, "invalid grid or count NULL");
  *count = g->launches;
  return SGML_OK;
}

int sgml_destroy(sgml_grid_t g) {
  if (!g) return SGML_OK;
  cudaStreamSynchronize(g->stream);
  void* ptrs[] = {g->U, g->F, g->SIG64, g->A64, g->pyr64, g->RESP, g->A0, g->E, g->E2, g->B, g->R, g->SIG, g->Q,
                  g->d_probs, g->d_state, g->d_accum, g->d_sync, g->d_phases, g->d_rows, g->d_tasks,
                  g->d_task_off, g->d_tasks4, g->d_task_off4, g->d_hist, g->d_trace, g->d_diag,
                  g->d_rowsum, g->d_umean, g->d_fmean, g->d_scratch};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (g->h_state) cudaFreeHost(g->h_state);
  delete g;
  return SGML_OK;
}

const char* sgml_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
