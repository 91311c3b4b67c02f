// sgml_noalloc.cu -- sgml_solve_noalloc: a solve that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they want a solve: frameworks whose
// memory pool owns the whole device and forbids allocations made behind its back, embedded or
// real-time hosts whose device-memory budget is fixed at start-up (and which cannot afford the
// implicit synchronisation of cudaMalloc / cudaFree inside a control loop), and services that must
// not fail for lack of memory once they are running.  This entry point serves them: the caller
// passes device pointers for the inputs and the output, and every intermediate array (the level
// pyramid, the residual accumulator, the schedule tables, the per-problem state and the barrier
// words) lives in one file-scope `__device__` array of kNoAllocBytes bytes.  Every GPU that loads
// the library holds that array until the process exits.
//
// The paper has no counterpart: this is a packaging of the same cycle kernel (Algorithms 1-3) for
// callers without an allocator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "sgml.h"
#include "sgml_internal.cuh"
#include "sgml_tasks.h"

using namespace sgml;

namespace {

constexpr size_t kNoAllocBytes = 24u << 20;  // 24 MiB of scratch per device
constexpr int kMaxDevices = 64;
constexpr int kMaxTasks = 8192;
constexpr int kMaxPhases = 256;
constexpr int kMaxToff = kMaxLevels * 1025;  // up to 1024 CTAs

__device__ __align__(256) unsigned char g_scratch[kNoAllocBytes];

thread_local std::string t_error;
std::mutex g_table_mutex;

int fail(int code, const char* msg) {
  t_error = msg;
  return code;
}

// Device address of g_scratch on each device, looked up once with that device current.  Read and
// written only with g_table_mutex held.
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

int scratch_address(unsigned char** out) {  // caller holds g_table_mutex
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(SGML_ERR_CUDA, "no current device");
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr) return fail(SGML_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
    g_scratch_addr[dev] = (unsigned char*)ptr;
  }
  *out = g_scratch_addr[dev];
  return SGML_OK;
}

double w_edge() { return 1.0 / std::sqrt(2.0); }
double w_corner() { return 1.0 / std::sqrt(3.0); }
double weight_sum(int dim) { return dim == 3 ? 6.0 + 12.0 * w_edge() + 8.0 * w_corner() : 4.0 + 4.0 * w_edge(); }
double weight_moment(int dim) { return dim == 3 ? 2.0 + 8.0 * w_edge() + 8.0 * w_corner() : 2.0 + 4.0 * w_edge(); }
double kappa(int dim) { return 2.0 / weight_moment(dim); }
long long side(int n, int l) { return (1LL << (n - l)) + 1; }
long long nodes(int dim, int n, int l) {
  const long long N = side(n, l);
  return dim == 3 ? N * N * N : N * N;
}
size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// The kernel dereferences f, sigma and u directly: each must be device (or managed) memory that the
// current device can address.  A host pointer, or memory of another GPU, is refused instead of
// becoming a stray device access.
bool on_current_device(const void* ptr, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unregistered host pointer
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Bump layout inside the scratch array.
struct Bump {
  size_t used = 0;
  size_t take(size_t bytes) {
    const size_t at = used;
    used = align256(used + bytes);
    return at;
  }
};

}  // namespace

extern "C" int sgml_solve_noalloc(int dim, int n, int precision, const double* f, const double* sigma,
                                  double a_scalar, const int* face_type, const double* face_value, double rtol,
                                  int max_cycles, double* u, int* cycles_out, double* rel_out, void* cuda_stream) {
  if (dim != 2 && dim != 3) return fail(SGML_ERR_ARG, "dim must be 2 or 3");
  if (n < 1 || n > (dim == 3 ? 10 : 12)) return fail(SGML_ERR_ARG, "n out of range");
  if (precision != SGML_FP64 && precision != SGML_MIXED) return fail(SGML_ERR_ARG, "bad precision");
  if (!f || !u || !face_type) return fail(SGML_ERR_ARG, "f, u and face_type are required");
  if (!(a_scalar <= 0.0) || !(rtol >= 0.0) || max_cycles < 0 || max_cycles > 100000) return fail(SGML_ERR_ARG, "bad a_scalar, rtol or max_cycles");
  for (int k = 0; k < 2 * dim; ++k)
    if (face_type[k] != SGML_DIRICHLET && face_type[k] != SGML_NEUMANN) return fail(SGML_ERR_ARG, "bad face type");
  const bool mixed = precision == SGML_MIXED;
  const int elem = mixed ? 4 : 8;
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  // ---- layout ----------------------------------------------------------------------------
  ProblemDesc P;
  std::memset(&P, 0, sizeof(P));
  P.n = n;
  P.h = 1.0 / (double)(1LL << n);
  P.hetero = sigma ? 1 : 0;
  P.a_scalar = a_scalar;
  for (int k = 0; k < 6; ++k) {
    P.face_type[k] = k < 2 * dim ? face_type[k] : SGML_DIRICHLET;
    P.face_value[k] = (k < 2 * dim && face_value) ? face_value[k] : 0.0;
  }
  {
    bool all_neumann = true;
    for (int k = 0; k < 2 * dim; ++k) all_neumann = all_neumann && P.face_type[k] == SGML_NEUMANN;
    if (all_neumann && a_scalar >= 0.0)
      return fail(SGML_ERR_ARG, "all-Neumann problems with a >= 0 need the mean projection of the grid API");
  }
  long long lvl = 0;
  for (int l = 0; l <= n - 1; ++l) {
    P.off_lvl[l] = lvl;
    lvl += (nodes(dim, n, l) + 63) / 64 * 64;
  }
  const long long M0 = nodes(dim, n, 0);
  Bump bump;
  const size_t o_desc = bump.take(sizeof(ProblemDesc));
  const size_t o_state = bump.take(sizeof(ProblemState));
  const size_t o_accum = bump.take(sizeof(Accum));
  const size_t o_sync = bump.take(sizeof(GridSync));
  const size_t o_phases = bump.take(sizeof(Phase) * kMaxPhases);
  const size_t o_tasks = bump.take(sizeof(TileTask) * kMaxTasks);
  const size_t o_toff = bump.take(sizeof(int) * kMaxToff);
  const size_t o_rows = bump.take(sizeof(long long) * kMaxLevels * 2);
  const size_t o_hist = bump.take(sizeof(double) * (max_cycles + 1));
  const size_t lvl_bytes = (size_t)elem * lvl;
  const size_t o_E = bump.take(lvl_bytes), o_E2 = bump.take(lvl_bytes), o_B = bump.take(lvl_bytes);
  const size_t o_R = bump.take(lvl_bytes);
  const size_t o_SIG = sigma ? bump.take(lvl_bytes) : 0, o_Q = sigma ? bump.take(lvl_bytes) : 0;
  const size_t o_RES = mixed ? bump.take(sizeof(float2) * M0) : 0;
  size_t o_tmp[kMaxLevels] = {0};
  if (sigma)
    for (int l = 1; l <= n - 1; ++l) o_tmp[l] = bump.take(sizeof(double) * nodes(dim, n, l));
  if (bump.used > kNoAllocBytes)
    return fail(SGML_ERR_ARG, "problem too large for the no-alloc scratch (24 MiB: e.g. 65^3 or 513^2 in either precision)");

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(SGML_ERR_CUDA, "no current device");
  if (!on_current_device(f, dev) || !on_current_device(u, dev) || (sigma && !on_current_device(sigma, dev)))
    return fail(SGML_ERR_ARG, "f, sigma and u must be device memory of the current device");

  // the scratch address table and the static partition tables below are shared by all host threads
  std::lock_guard<std::mutex> lock(g_table_mutex);
  unsigned char* base = nullptr;
  int st = scratch_address(&base);
  if (st != SGML_OK) return st;

  // ---- host-side tables (stack memory) ------------------------------------------------------
  int bps = 0;
  if (sgml_t64::cycle_kernel_occupancy(mixed ? 1 : 0, dim, kThreads, &bps) != 0 || bps < 1)
    return fail(SGML_ERR_CUDA, "occupancy query failed");
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(SGML_ERR_CUDA, "multiprocessor count query failed");
  const int blocks = sms * bps;

  long long rows[kMaxLevels * 2];
  for (int l = 0; l < kMaxLevels; ++l) {
    rows[2 * l] = 0;
    const long long N = side(n, std::min(l, n - 1));
    rows[2 * l + 1] = l <= n - 1 ? (dim == 3 ? N * N : N) : 0;
  }
  // partition tables in static host storage (no allocation); the mutex taken above serialises
  // their use
  static TileTask tasks[kMaxTasks];
  static int toff[kMaxToff];
  constexpr int kTX = 64, kTY = 2 * kThreads / 64;  // the 64 x 8 tile kernels
  if (blocks > 1024 || partition_bound(dim, &n, 1, blocks, kTX, kTY) > kMaxTasks)
    return fail(SGML_ERR_ARG, "problem too large for the no-alloc task table");
  const int dir_hi = (P.face_type[1] == SGML_DIRICHLET ? 1 : 0) | (P.face_type[3] == SGML_DIRICHLET ? 2 : 0);
  const int nt = build_partition(dim, &n, &dir_hi, 1, blocks, kTX, kTY, tasks, toff);
  const size_t toff_bytes = sizeof(int) * (size_t)kMaxLevels * (blocks + 1);

  // schedule of one cycle (Algorithm 3, zig-zag reading, n_r = 2)
  const int n_r = 2;
  Phase phases[kMaxPhases];
  int np = 0;
  for (int l = 1; l <= n - 1; ++l) phases[np++] = Phase{OP_RESTRICT, l, l - 1, 0, 0, 0};
  struct Visit {
    int level, tooth, first, final_visit;
  };
  Visit vs[3 * kMaxLevels + 1];
  int nv = 0;
  for (int nu1 = n - 1; nu1 >= 1; --nu1) {
    vs[nv++] = {nu1, nu1, 1, 0};
    vs[nv++] = {nu1 - 1, nu1, 0, 0};
    vs[nv++] = {nu1, nu1, 0, 0};
  }
  vs[nv++] = {0, 0, 1, 1};
  for (int q = 0; q < nv; ++q) {
    const Visit& v = vs[q];
    if (q > 0) {
      const Visit& w = vs[q - 1];
      if (v.level == w.level - 1) phases[np++] = Phase{OP_PROLONG, v.level, w.tooth, 0, v.tooth == w.tooth ? kInit : 0, v.level + 1};
      else if (v.level == w.level + 1) phases[np++] = Phase{OP_INJECT, v.level, w.tooth, 0, 0, 0};
    }
    const int k = (int)std::min<long long>(n_r, 1LL << std::min(n - v.tooth, 30));
    const int kk = v.final_visit ? 3 * k : k;
    for (int s = 0; s < kk; ++s)
      phases[np++] = Phase{OP_SWEEP, v.level, v.tooth, s, (v.final_visit ? kFinalVisit : 0) | (v.first ? kFirstOfTooth : 0), 0};
  }

  const double theta = 0.7;
  const double kap = kappa(dim);
  const double tg = theta * (kappa(dim) * weight_sum(dim) / 2.0);
  P.c0 = kap / (2.0 * P.h * P.h);
  for (int l = 0; l <= n - 1; ++l) {
    const double H = P.h * (double)(1LL << l);
    const double c = kap / (2.0 * H * H);
    P.q_const[l] = tg / (c * 2.0 * weight_sum(dim) - a_scalar) * c;
    P.inv_c[l] = 2.0 * H * H / kap;
  }
  for (int l = 0; l < kMaxLevels; ++l) P.inv_c_f[l] = (float)P.inv_c[l], P.q_const_f[l] = (float)P.q_const[l];
  P.c0_f = (float)P.c0;
  P.a_scalar_f = (float)P.a_scalar;

  // ---- uploads and clears (stream-ordered, no allocation) ---------------------------------
#define NA_CUDA(call)                                                     \
  do {                                                                    \
    if ((call) != cudaSuccess) return fail(SGML_ERR_CUDA, #call " failed"); \
  } while (0)
  NA_CUDA(cudaMemcpyAsync(base + o_desc, &P, sizeof(P), cudaMemcpyHostToDevice, stream));
  NA_CUDA(cudaMemcpyAsync(base + o_phases, phases, sizeof(Phase) * np, cudaMemcpyHostToDevice, stream));
  NA_CUDA(cudaMemcpyAsync(base + o_tasks, tasks, sizeof(TileTask) * nt, cudaMemcpyHostToDevice, stream));
  NA_CUDA(cudaMemcpyAsync(base + o_toff, toff, toff_bytes, cudaMemcpyHostToDevice, stream));
  NA_CUDA(cudaMemcpyAsync(base + o_rows, rows, sizeof(rows), cudaMemcpyHostToDevice, stream));
  // the scratch keeps the previous call's contents: clear everything that must start at zero
  NA_CUDA(cudaMemsetAsync(base + o_state, 0, sizeof(ProblemState), stream));
  NA_CUDA(cudaMemsetAsync(base + o_accum, 0, sizeof(Accum), stream));
  NA_CUDA(cudaMemsetAsync(base + o_sync, 0, sizeof(GridSync), stream));
  NA_CUDA(cudaMemsetAsync(base + o_E, 0, lvl_bytes, stream));
  NA_CUDA(cudaMemsetAsync(base + o_E2, 0, lvl_bytes, stream));
  NA_CUDA(cudaMemsetAsync(base + o_B, 0, lvl_bytes, stream));
  NA_CUDA(cudaMemsetAsync(base + o_R, 0, lvl_bytes, stream));

  // coefficient pyramid (restricted sigma and local steps) for a heterogeneous problem
  if (sigma) {
    const double* sig_l[kMaxLevels] = {nullptr};
    sig_l[0] = sigma;
    for (int l = 1; l <= n - 1; ++l) {
      sig_l[l] = (const double*)(base + o_tmp[l]);
      NA_CUDA(launch_restrict64(dim, sig_l[l - 1], (int)side(n, l - 1), (double*)(base + o_tmp[l]), (int)side(n, l), stream));
    }
    for (int l = 0; l <= n - 1; ++l)
      NA_CUDA(launch_setup_level(mixed ? 1 : 0, dim, P, l, sig_l[l], nullptr, kap, w_edge(), w_corner(), tg,
                                 base + o_SIG, base + o_Q, nullptr, stream));
  }

  KernelParams p;
  std::memset(&p, 0, sizeof(p));
  p.dim = dim;
  p.batch = 1;
  p.n_max = n;
  p.mixed = mixed ? 1 : 0;
  p.probs = (const ProblemDesc*)(base + o_desc);
  p.state = (ProblemState*)(base + o_state);
  p.accum = (Accum*)(base + o_accum);
  p.phases = (const Phase*)(base + o_phases);
  p.nphases = np;
  p.tasks = (const TileTask*)(base + o_tasks);
  p.task_off = (const int*)(base + o_toff);
  p.row_prefix = (const long long*)(base + o_rows);
  p.fresh = 1;
  p.max_cycles = max_cycles;
  p.tol = rtol;
  p.kappa = kap;
  p.w_edge = w_edge();
  p.w_corner = w_corner();
  p.omega = tg;
  p.w_edge_f = (float)p.w_edge;
  p.w_corner_f = (float)p.w_corner;
  p.one_m_omega_f = (float)(1.0 - p.omega);
  p.n_r = n_r;
  p.sync = (GridSync*)(base + o_sync);
  p.timeout_ns = 2000000000ull;
  p.hist = (double*)(base + o_hist);
  p.hist_cap = max_cycles + 1;
  p.U = u;
  p.F = const_cast<double*>(f);
  p.SIG64 = const_cast<double*>(sigma);
  p.A64 = nullptr;
  p.RESP = mixed ? (float2*)(base + o_RES) : nullptr;
  p.E = base + o_E;
  p.E2 = base + o_E2;
  p.B = base + o_B;
  p.R = base + o_R;
  p.SIG = sigma ? base + o_SIG : nullptr;
  p.Q = sigma ? base + o_Q : nullptr;
  p.A0 = nullptr;
  NA_CUDA(sgml_t64::launch_cycle_kernel(p, mixed ? 1 : 0, dim, blocks, kThreads, stream));

  ProblemState S;
  GridSync G;
  NA_CUDA(cudaMemcpyAsync(&S, base + o_state, sizeof(S), cudaMemcpyDeviceToHost, stream));
  NA_CUDA(cudaMemcpyAsync(&G, base + o_sync, sizeof(G), cudaMemcpyDeviceToHost, stream));
  NA_CUDA(cudaStreamSynchronize(stream));
#undef NA_CUDA
  if (G.error) return fail(SGML_ERR_BARRIER_TIMEOUT, "a grid barrier of the cycle kernel timed out");
  if (cycles_out) *cycles_out = S.cycles;
  if (rel_out) *rel_out = S.rel;
  if (S.status != SGML_OK) return fail(S.status, "the solve did not converge");
  return SGML_OK;
}

extern "C" const char* sgml_noalloc_last_error(void) { return t_error.c_str(); }
