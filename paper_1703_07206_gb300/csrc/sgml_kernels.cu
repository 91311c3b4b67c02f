// sgml_kernels.cu -- device code of libsgml (sm_103a).
//
// One persistent cooperative kernel runs whole solves: the FP64 outer step (residual of the
// accumulated solution, Sec. 2 last paragraphs; max/L2 norms, Sec. 3.1), then the schedule of the
// single cycle (Algorithm 3) as phases -- restriction passes (Algorithm 1, Eqs. 3-4), Jacobi sweeps
// of the pseudo-time equation (Eq. 2) with the radial stencil (Eq. 5) at stride 2^nu, and the
// interpolation of a visit's change to the finer levels (Algorithm 2, I_lambda) -- separated by a
// bounded grid-wide barrier, so no level pays a kernel launch.
//
// Deferred interpolation: each level keeps its compact copy E_l of the correction on the level-l
// subset.  Moving one level finer, the change of the level just visited (E_{l+1} - B_{l+1}) is
// interpolated with the tensor-product hat functions and added to E_l; moving one level coarser,
// E_{l+1} = B_{l+1} = E_l restricted to the coarser subset (injection).  Since relaxation at level l
// reads only level-l nodes and multilinear interpolation is nested, this gives the values of
// interpolating every visit's change to the whole single grid right after the visit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sgml_internal.cuh"

#ifndef SGML_TILE_X
#define SGML_TILE_X 64
#endif
#ifndef SGML_KNS
#define SGML_KNS sgml_t64
#endif

namespace SGML_KNS {
using namespace sgml;
constexpr int kTX = SGML_TILE_X, kTY = 2 * (kThreads / kTX);

// ---------------------------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ int refl(int i, int N) { return i < 0 ? -i : (i > N - 1 ? 2 * (N - 1) - i : i); }
// The image index, clamped into the level (cells past the image of the far edge: never used).
__device__ __forceinline__ int refl_clamp(int i, int N) {
  i = refl(i, N);
  return i < 0 ? 0 : (i > N - 1 ? N - 1 : i);
}

__device__ __forceinline__ int level_side(int n, int l) { return (1 << (n - l)) + 1; }

template <int DIM>
__device__ __forceinline__ long long level_nodes(int N) {
  return DIM == 3 ? (long long)N * N * N : (long long)N * N;
}

template <int DIM>
__device__ __forceinline__ void decode(long long local, int N, int& i, int& j, int& k) {
  int l = (int)local;
  i = l % N;
  l /= N;
  if (DIM == 3) {
    j = l % N;
    k = l / N;
  } else {
    j = l;
    k = 0;
  }
}

template <int DIM>
__device__ __forceinline__ int lin(int i, int j, int k, int N) {
  return DIM == 3 ? (k * N + j) * N + i : j * N + i;
}

// Node on a Dirichlet face (compact coordinates of a level with N nodes per side).
template <int DIM>
__device__ __forceinline__ bool is_fixed(const ProblemDesc& P, int N, int i, int j, int k) {
  if ((i == 0 && P.face_type[0] == 0) || (i == N - 1 && P.face_type[1] == 0)) return true;
  if ((j == 0 && P.face_type[2] == 0) || (j == N - 1 && P.face_type[3] == 0)) return true;
  if (DIM == 3 && ((k == 0 && P.face_type[4] == 0) || (k == N - 1 && P.face_type[5] == 0))) return true;
  return false;
}

template <int DIM>
__device__ __forceinline__ double dirichlet_value(const ProblemDesc& P, int N, int i, int j, int k) {
  if (i == 0 && P.face_type[0] == 0) return P.face_value[0];
  if (i == N - 1 && P.face_type[1] == 0) return P.face_value[1];
  if (j == 0 && P.face_type[2] == 0) return P.face_value[2];
  if (j == N - 1 && P.face_type[3] == 0) return P.face_value[3];
  if (DIM == 3) {
    if (k == 0 && P.face_type[4] == 0) return P.face_value[4];
    if (k == N - 1 && P.face_type[5] == 0) return P.face_value[5];
  }
  return 0.0;
}

__device__ __forceinline__ double nan_max(double a, double b) {
  if (a != a) return a;
  if (b != b) return b;
  return a > b ? a : b;
}

// Diagnostic pseudo-residual (Sec. 3.1): the largest |delta L_l e - r_l| met by the sweeps of a
// level, recorded per problem, cycle and level when the grid asks for it.  At a node it is
// |e_new - e| / dtau; the CTA's maximum, in the units of the unscaled residual, is merged into
// diag[(b * diag_cycles + c) * kMaxLevels + l] (non-negative doubles order like their bits).
// Diagnostic pseudo-residual of one node, |e_new - e| / dtau = |e_new - e| c / q: kept per thread as
// max |e_new - e| / q in the cycle precision and scaled by c = 1 / inv_c once (in the FP32 form a
// reciprocal per node instead of an FP64 division, which would double the sweep's time).
template <typename T>
__device__ __forceinline__ T diag_term(T de, T q) {
  if constexpr (sizeof(T) == 4) return fabsf(de) * __frcp_rn(q);
  else return fabs(de) / q;
}

// Problem 0's pseudo-residuals of the current cycle, per level, folded in shared memory and committed
// to global memory once per cycle (diag_commit): a global atomic per tile on one address per level
// serialised hundreds of CTAs, and the recording cost more than the solve.
__shared__ unsigned long long s_diag0[kMaxLevels];

// A tile's pseudo-residual: each thread holds max |e_new - e| / q over its nodes in the cycle
// precision; the warps reduce that (no FP64 work per thread) and one lane per warp scales it by
// 1 / (inv_c s), which commutes with the maximum.
template <typename T>
__device__ void diag_flush(const KernelParams& p, int b, int c, int l, T mx, T inv_c) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  double m = 0.0;
  if (lane == 0) m = (double)mx / (double)inv_c / p.state[b].scale_used[c & 1];
  if (b == 0) {  // (positive doubles order like their bit patterns)
    if (lane == 0 && m > 0.0) atomicMax(&s_diag0[l], (unsigned long long)__double_as_longlong(m));
    return;
  }
  __shared__ double s_dmx[32];
  if (lane == 0) s_dmx[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, s_dmx[w]);
    if (c < p.diag_cycles && mm > 0.0) {
      unsigned long long* slot = &p.diag[((long long)b * p.diag_cycles + c) * kMaxLevels + l];
      const unsigned long long bits = (unsigned long long)__double_as_longlong(mm);
      if (bits > *(volatile unsigned long long*)slot) atomicMax(slot, bits);
    }
  }
  __syncthreads();
}

// Commit problem 0's folded pseudo-residuals of cycle c (every CTA, after the cycle's last phase).
__device__ void diag_commit(const KernelParams& p, int c) {
  __syncthreads();
  if (threadIdx.x < kMaxLevels) {
    const unsigned long long v = s_diag0[threadIdx.x];
    s_diag0[threadIdx.x] = 0ull;
    if (v != 0ull && c < p.diag_cycles) atomicMax(&p.diag[(long long)c * kMaxLevels + threadIdx.x], v);
  }
  __syncthreads();
}

// Explicitly rounded arithmetic for the stencil sums and updates: the compiler may otherwise
// contract a * b + c into an FMA in one copy of inlined or unrolled code and not in another, which
// would make a node's value depend on which tile, z-piece or loop iteration computed it.  With
// these, results are identical bit for bit whatever the launch shape and work partition.
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}


__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// ---------------------------------------------------------------------------------------------
// Bounded grid barrier.  Every wait has a time limit; on expiry the barrier records the error and
// every CTA returns from the kernel at its next barrier, so a fault in the schedule can never hang
// the GPU.  Requires all CTAs to be co-resident (cooperative launch).
// ---------------------------------------------------------------------------------------------
// Test aid (KernelParams::withhold_barrier = k >= 1): CTA 0 withholds its arrival at the k-th
// barrier of the launch, so that every CTA's bounded wait runs out and the launch ends with the
// timeout status -- the error path is exercised without any fault.
__shared__ int s_barriers;  // barriers this CTA has passed in the launch (counted only for the test aid)

__device__ bool grid_sync(GridSync* gs, unsigned long long timeout_ns, int withhold_barrier) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned long long G = gridDim.x;
    unsigned long long old;
    bool arrive = true;
    if (withhold_barrier > 0 && blockIdx.x == 0) arrive = ++s_barriers != withhold_barrier;
    if (arrive) {
      // arrival: release (the CTA's writes, ordered before by the CTA barrier, become visible) and, for
      // the last CTA to arrive, acquire (the others' writes are visible to it)
      asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], 1;" : "=l"(old) : "l"(&gs->arrive) : "memory");
    } else {
      asm volatile("ld.relaxed.gpu.u64 %0, [%1];" : "=l"(old) : "l"(&gs->arrive) : "memory");
      old = old / G * G;  // this round's target is never reached: the wait below runs out
    }
    const unsigned long long target = (old / G + 1) * G;  // every CTA of this round has arrived
    if (old + 1 < target || !arrive) {  // the last CTA to arrive knows it from the returned value
      const unsigned long long t0 = globaltimer();
      unsigned spins = 0;
      for (;;) {
        unsigned long long seen;
        // relaxed polling: an acquire per poll would invalidate L1 each time, under the feet of the
        // SM's other CTA (measured: the 2-D batch, which reads problem descriptors through L1,
        // took 43 % longer); one acquire load follows once every CTA has arrived
        asm volatile("ld.relaxed.gpu.u64 %0, [%1];" : "=l"(seen) : "l"(&gs->arrive) : "memory");
        if (seen >= target) {
          asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(seen) : "l"(&gs->arrive) : "memory");
          break;
        }
        if ((++spins & 31u) == 0u) {
          if (ld_volatile(&gs->error)) {  // another CTA gave up: stop too
            ok = 0;
            break;
          }
          if (globaltimer() - t0 > timeout_ns) {
            atomicExch(&gs->error, 1);
            ok = 0;
            break;
          }
        }
      }
    }
    // No error load on success: only a timed-out CTA sets the flag, and it leaves the kernel, so
    // every other CTA meets the flag while it spins at the next barrier (one load round trip less
    // per barrier).  The acquire of the last arrival, or the acquire load after the polling, then the
    // CTA barrier below, orders the CTA's later reads after the other CTAs' writes; no separate fence
    // (measured: 8-14 % less per barrier than release + relaxed polling + fence.acq_rel).
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------------------------
// Work distribution.  Tiled phases take column tiles (TileTask) of one level, CTA c handling tasks
// c, c + G, ...; row phases take node rows (fixed y, z) of one level, one row per warp.
// ---------------------------------------------------------------------------------------------
// Per-CTA copies of the launch-constant tables, loaded once at kernel start: the first
// kPhaseCache phases of the schedule, this CTA's task range of every level and its first
// kTaskCache tasks per level.  A phase then starts without a chain of dependent global loads
// (the coarse levels' phases are short enough for those latencies to matter).
constexpr int kPhaseCache = 128, kTaskCache = 2;
__shared__ Phase s_phase[kPhaseCache];
__shared__ int s_toff[kMaxLevels][2];
__shared__ TileTask s_task[kMaxLevels][kTaskCache];

// Also cached: problem 0's descriptor, the number of node rows of every level (row phases), and,
// once per cycle, the problems' stop flags (written by the convergence check between two barriers):
// every phase reads them, and after a grid barrier each would be an L2 round trip.
constexpr int kDoneCache = 256;
__shared__ ProblemDesc s_prob0;
__shared__ long long s_rows[kMaxLevels];
__shared__ unsigned char s_done[kDoneCache];

__device__ __forceinline__ const ProblemDesc& prob_at(const KernelParams& p, int b) {
  return b == 0 ? s_prob0 : p.probs[b];
}

__device__ __forceinline__ bool done_at(const KernelParams& p, int b) {
  return b < kDoneCache ? s_done[b] != 0 : p.accum[b].done != 0;
}

// Problem 0's cast scales for the current cycle (set by the check), cached with the stop flags.
struct Scales {
  double next, inv[2];
  float next_f, inv_f[2];
};
__shared__ Scales s_scales0;

__device__ void load_done(const KernelParams& p) {
  for (int b = threadIdx.x; b < p.batch && b < kDoneCache; b += blockDim.x)
    s_done[b] = (unsigned char)(ld_volatile(&p.accum[b].done) != 0);
  if (threadIdx.x == 0) {
    const volatile ProblemState& S = p.state[0];
    s_scales0.next = S.next_scale;
    s_scales0.inv[0] = S.inv_scale[0];
    s_scales0.inv[1] = S.inv_scale[1];
    s_scales0.next_f = S.next_scale_f;
    s_scales0.inv_f[0] = S.inv_scale_f[0];
    s_scales0.inv_f[1] = S.inv_scale_f[1];
  }
  __syncthreads();
}

// A launch constant in the arithmetic type V: the double, or the FP32 copy the host or the check
// made of it.  (A conversion per thread and tile occupies GB300's FP64 pipe for ~1 us a phase.)
template <typename V>
__device__ __forceinline__ V cv(double d, float f) {
  if constexpr (sizeof(V) == 4) return f;
  else return (V)d;
}

// 1 / s of cycle c's residual cast (slot c & 1), double and float.
__device__ __forceinline__ double inv_scale_at(const KernelParams& p, int b, int slot) {
  return b == 0 ? s_scales0.inv[slot] : p.state[b].inv_scale[slot];
}
__device__ __forceinline__ float inv_scale_f_at(const KernelParams& p, int b, int slot) {
  return b == 0 ? s_scales0.inv_f[slot] : p.state[b].inv_scale_f[slot];
}

__device__ void load_tables(const KernelParams& p) {
  if (threadIdx.x == 0) s_prob0 = p.probs[0];
  if (threadIdx.x == 0) s_barriers = 0;
  if (threadIdx.x < kMaxLevels) s_diag0[threadIdx.x] = 0ull;
  if (threadIdx.x < kMaxLevels) s_rows[threadIdx.x] = p.row_prefix[(long long)threadIdx.x * (p.batch + 1) + p.batch];
  for (int i = threadIdx.x; i < p.nphases && i < kPhaseCache; i += blockDim.x) s_phase[i] = p.phases[i];
  if (threadIdx.x < kMaxLevels) {
    const int l = threadIdx.x;
    const int* o = p.task_off + (long long)l * (gridDim.x + 1) + blockIdx.x;
    const int t0 = o[0], t1 = o[1];
    s_toff[l][0] = t0;
    s_toff[l][1] = t1;
    for (int j = 0; j < kTaskCache && t0 + j < t1; ++j) s_task[l][j] = p.tasks[t0 + j];
  }
  __syncthreads();
}

__device__ __forceinline__ Phase phase_at(const KernelParams& p, int q) {
  return q < kPhaseCache ? s_phase[q] : p.phases[q];
}

__device__ __forceinline__ TileTask task_at(const KernelParams& p, int l, int t) {
  const int j = t - s_toff[l][0];
  return j < kTaskCache ? s_task[l][j] : p.tasks[t];
}

template <class Body>
__device__ __forceinline__ void for_tasks(const KernelParams& p, int l, Body&& body) {
  const int t0 = s_toff[l][0], t1 = s_toff[l][1];
  for (int t = t0; t < t1; ++t) body(task_at(p, l, t));
}

// Rows of level l of all problems; body(b, N, y, z) runs on one warp (lanes cover x).
template <int DIM, class Body>
__device__ __forceinline__ void for_rows(const KernelParams& p, int l, Body&& body) {
  const long long* rp = p.row_prefix + (long long)l * (p.batch + 1);
  const long long total = s_rows[l];
  const int warps = blockDim.x >> 5;
  int b = 0;
  for (long long r = (long long)blockIdx.x * warps + (threadIdx.x >> 5); r < total; r += (long long)gridDim.x * warps) {
    if (p.batch > 1)
      while (rp[b + 1] <= r) ++b;
    const ProblemDesc& P = prob_at(p, b);
    const int N = level_side(P.n, l);
    const int local = (int)(r - rp[b]);
    body(b, P, N, DIM == 3 ? local % N : local, DIM == 3 ? local / N : 0);
  }
}

// Number of sweeps of a visit of tooth nu1 for a problem with n levels (Algorithm 3).
__device__ __forceinline__ int visit_sweeps(int n_r, int n, int tooth, bool final_visit) {
  const int e = n - tooth;
  const int cap = e >= 30 ? (1 << 30) : (1 << e);
  const int k = n_r < cap ? n_r : cap;
  return final_visit ? 3 * k : k;
}

// Levels whose sweeps run two at a time (fused pairs, 3-D mixed form): sweep s reads E or E2 by the
// parity of its pair index s / 2 there, of s elsewhere; a visit of k sweeps ends in E2 if it flipped
// the buffers an odd number of times.
__device__ __forceinline__ bool paired_level(const KernelParams& p, int l) { return l < p.pair_levels; }
__device__ __forceinline__ int sweep_parity(const KernelParams& p, int l, int sweep) {
  return (paired_level(p, l) ? sweep >> 1 : sweep) & 1;
}
__device__ __forceinline__ int visit_flips(const KernelParams& p, int l, int k) {
  return paired_level(p, l) ? (k + 1) >> 1 : k;
}

// Halo of a kTX x kTY tile: (kTX + 2) x (kTY + 2) cells, at most kCells per thread.  Thread
// (tx, ty) = (tid % 32, tid / 32) owns the columns (x0 + tx, y0 + 2 ty + r), r = 0, 1.
constexpr int kHX = kTX + 2, kHY = kTY + 2, kHalo = kHX * kHY;
constexpr int kCells = (kHalo + kThreads - 1) / kThreads;
static_assert(kTY == 2 * (kThreads / kTX), "two rows per thread");

struct HaloCells {
  int off[kCells];        // y * N + x of the cell (images applied), -1 if the thread has no such cell
  double ghost[kCells];   // Neumann image offset 2 k h g of the cell (x, y directions)
};

__device__ __forceinline__ HaloCells halo_cells(const ProblemDesc& P, int N, int x0, int y0, bool flux) {
  HaloCells hc;
#pragma unroll
  for (int s = 0; s < kCells; ++s) {
    const int k = threadIdx.x + s * kThreads;
    hc.off[s] = -1;
    hc.ghost[s] = 0.0;
    if (k < kHalo) {
      int gx = x0 - 1 + k % kHX, gy = y0 - 1 + k / kHX;
      // cells past the image of the far edge (a tile overhanging a small level) are never read by
      // a node of the level: no copy is issued for them (their shared-memory slots keep stale
      // values, used only by threads that own no node)
      if (gx > N || gy > N) continue;
      double g = 0.0;
      if (flux) {
        if (gx < 0 && P.face_type[0] == 1) g += 2.0 * P.h * P.face_value[0];
        if (gx > N - 1 && P.face_type[1] == 1) g += 2.0 * P.h * P.face_value[1];
        if (gy < 0 && P.face_type[2] == 1) g += 2.0 * P.h * P.face_value[2];
        if (gy > N - 1 && P.face_type[3] == 1) g += 2.0 * P.h * P.face_value[3];
      }
      gx = refl(gx, N);
      gy = refl(gy, N);
      gx = gx < 0 ? 0 : (gx > N - 1 ? N - 1 : gx);
      gy = gy < 0 ? 0 : (gy > N - 1 ? N - 1 : gy);
      hc.off[s] = gy * N + gx;
      hc.ghost[s] = g;
    }
  }
  return hc;
}

// 2-D tiles, whose set-up is paid per tile (no z-march to spread it over): a tile whose halo lies
// inside the level needs no images, clamps or face tests -- each halo offset is one multiply-add.
__device__ __forceinline__ bool tile_interior(int N, int x0, int y0) {
  return x0 >= 1 && y0 >= 1 && x0 + kTX <= N - 1 && y0 + kTY <= N - 1;
}

__device__ __forceinline__ HaloCells halo_cells_2d(const ProblemDesc& P, int N, int x0, int y0, bool interior) {
  if (!interior) return halo_cells(P, N, x0, y0, false);
  HaloCells hc;
#pragma unroll
  for (int s = 0; s < kCells; ++s) {
    const int k = threadIdx.x + s * kThreads;
    hc.off[s] = k < kHalo ? (y0 - 1 + k / kHX) * N + (x0 - 1 + k % kHX) : -1;
    hc.ghost[s] = 0.0;
  }
  return hc;
}

__device__ __forceinline__ double z_ghost(const ProblemDesc& P, int z, int N) {
  if (z < 0 && P.face_type[4] == 1) return 2.0 * P.h * P.face_value[4];
  if (z > N - 1 && P.face_type[5] == 1) return 2.0 * P.h * P.face_value[5];
  return 0.0;
}

// The two columns a thread owns in a tile: in-level flags, 2-D offsets, and whether an x / y face
// fixes them (Dirichlet); z faces are checked per plane.
struct Columns {
  int off[2];
  bool in[2];
  bool fixed_xy[2];
  bool dz0, dz1;  // -z / +z faces are Dirichlet
};

__device__ __forceinline__ Columns own_columns(const ProblemDesc& P, int N, int x0, int y0) {
  Columns cl;
  const int x = x0 + (int)(threadIdx.x % kTX);
  const bool fx = (x == 0 && P.face_type[0] == 0) || (x == N - 1 && P.face_type[1] == 0);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int y = y0 + 2 * (int)(threadIdx.x / kTX) + r;
    cl.in[r] = x < N && y < N;
    cl.off[r] = y * N + x;
    cl.fixed_xy[r] = fx || (y == 0 && P.face_type[2] == 0) || (y == N - 1 && P.face_type[3] == 0);
  }
  cl.dz0 = P.face_type[4] == 0;
  cl.dz1 = P.face_type[5] == 0;
  return cl;
}

__device__ __forceinline__ Columns own_columns_2d(const ProblemDesc& P, int N, int x0, int y0, bool interior) {
  if (!interior) return own_columns(P, N, x0, y0);
  Columns cl;
  const int x = x0 + (int)(threadIdx.x % kTX), y = y0 + 2 * (int)(threadIdx.x / kTX);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    cl.in[r] = true;
    cl.off[r] = (y + r) * N + x;
    cl.fixed_xy[r] = false;
  }
  cl.dz0 = cl.dz1 = false;
  return cl;
}

__device__ __forceinline__ bool z_fixed(const Columns& cl, int z, int N) {
  return (z == 0 && cl.dz0) || (z == N - 1 && cl.dz1);
}
__device__ __forceinline__ bool z_fixed(bool dz0, bool dz1, int z, int N) {
  return (z == 0 && dz0) || (z == N - 1 && dz1);
}

// Block reduction of (max, sum) and one atomic per block into the accumulators.
__device__ void block_flush(double mx, double s2, unsigned long long* mx_dst, double* s2_dst) {
  __shared__ double smx[32], ss2[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = nan_max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    smx[warp] = mx;
    ss2[warp] = s2;
  }
  __syncthreads();
  if (warp == 0) {
    mx = lane < nwarps ? smx[lane] : 0.0;
    s2 = lane < nwarps ? ss2[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = nan_max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      atomicMax(mx_dst, (unsigned long long)__double_as_longlong(mx));
      atomicAdd(s2_dst, s2);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async): the tiled phases keep several planes (3-D) or
// tiles (2-D) in flight per CTA so that HBM latency is hidden behind the stencil arithmetic.
// ---------------------------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_t(T* smem, const T* gmem) {
  cp_async<sizeof(T)>(smem, gmem);
}

// Pipeline depths (stages of shared memory per CTA).
#ifndef SGML_SWEEP_STAGES
#define SGML_SWEEP_STAGES 4
#endif
#ifndef SGML_OUTER_STAGES
#define SGML_OUTER_STAGES 5
#endif
#ifndef SGML_MIN_CTAS
#define SGML_MIN_CTAS 2
#endif
constexpr int kSweepStages = SGML_SWEEP_STAGES;  // loads issued kSweepStages - 2 planes ahead
constexpr int kOuterStages = SGML_OUTER_STAGES;  // loads issued kOuterStages - 3 planes ahead (three resident)
// A z-piece of at most kSweepStages - 1 planes issues all its planes before its first step, whose wait
// leaves kSweepStages - 3 copy groups pending: plane 0 is then complete only while the piece has more
// planes than that, which its three-plane minimum guarantees for four or five stages (not six).
static_assert(kSweepStages >= 4 && kSweepStages <= 5, "sweep pipelines are written for 4 or 5 stages");

template <typename T>
struct SweepStage {
  T e[kHalo];            // correction e on the halo tile
  T s[kHalo];            // sigma on the halo tile (heterogeneous problems)
  T r[2 * kThreads];     // restricted residual at the tile's nodes
  T q[2 * kThreads];     // local step factor at the tile's nodes
  double u[2 * kThreads];  // FP64 solution (last sweep of a cycle)
};

// Stage of the residual phases: halo tiles of the operand (u in FP64, or e in the cycle precision)
// and of sigma, the right-hand side at the tile's nodes (f, or the previous residual), and a
// per-node Helmholtz coefficient.
template <typename V>
struct ResStage {
  V u[kHalo];
  V s[kHalo];
  double f[2 * kThreads];
  V a[2 * kThreads];
};

template <typename T>
constexpr size_t sweep_smem_bytes() {
  return sizeof(SweepStage<T>) * kSweepStages;
}
constexpr size_t outer_smem_bytes() { return sizeof(ResStage<double>) * kOuterStages; }
// ProlongStage<T> (defined with the interpolation phase): (kTX/2+1)(kTY/2+1) coarse cells x 2 plus
// 2 x 2 x kThreads fine values; 6 stages in FP32 (loads four coarse planes ahead), 4 in FP64.
template <typename T>
__host__ __device__ constexpr int prolong_stages() { return sizeof(T) == 4 ? 6 : 4; }
template <typename T>
constexpr size_t prolong_smem_bytes() {
  return prolong_stages<T>() * (sizeof(T) * 2 * (kTX / 2 + 1) * (kTY / 2 + 1) + sizeof(T) * 4 * kThreads);
}


// ---------------------------------------------------------------------------------------------
// Lift: u = Dirichlet values on fixed nodes, 0 on unknowns; ||f|| over the unknowns.  One node row
// per warp; each warp folds its rows' norms and flushes them when its problem changes.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void warp_flush(double mx, double s2, unsigned long long* mx_dst, double* s2_dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = nan_max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(mx_dst, (unsigned long long)__double_as_longlong(mx));
    atomicAdd(s2_dst, s2);
  }
}

template <typename T, int DIM>
__device__ void phase_lift(const KernelParams& p) {
  const int lane = threadIdx.x & 31;
  int cur = -1;
  double mx = 0.0, s2 = 0.0;
  for_rows<DIM>(p, 0, [&](int b, const ProblemDesc& P, int N, int y, int z) {
    if (b != cur) {
      if (cur >= 0) warp_flush(mx, s2, &p.accum[cur].fmax_bits, &p.accum[cur].fsum2);
      cur = b;
      mx = s2 = 0.0;
    }
    const long long row = P.off_full + ((long long)z * N + y) * N;
    for (int x = lane; x < N; x += 32) {
      if (is_fixed<DIM>(P, N, x, y, z)) {
        p.U[row + x] = dirichlet_value<DIM>(P, N, x, y, z);
      } else {
        p.U[row + x] = 0.0;
        const double f = p.F[row + x];
        mx = nan_max(mx, fabs(f));
        s2 += f * f;
      }
    }
  });
  if (cur >= 0) warp_flush(mx, s2, &p.accum[cur].fmax_bits, &p.accum[cur].fsum2);
}

// Scale of the residual cast of cycle c (mixed form): 1 / (max-norm of the previous residual).
__device__ __forceinline__ double cast_scale(const KernelParams& p, int b, int c) {
  if (!p.mixed) return 1.0;
  double ref = (c == 0 && p.fresh) ? __longlong_as_double((long long)p.accum[b].fmax_bits)
                                   : p.state[b].rmax_prev;
  return (ref > 0.0 && ref < 1e300) ? 1.0 / ref : 1.0;
}

// The cast scale of cycle c's residual: computed here for the first cycle of a fresh launch, else
// the value the previous cycle's check stored (no FP64 division per tile).
__device__ __forceinline__ double outer_scale(const KernelParams& p, int b, int c) {
  if (c == 0 && p.fresh) return cast_scale(p, b, c);
  return b == 0 ? s_scales0.next : p.state[b].next_scale;
}
__device__ __forceinline__ float outer_scale_f(const KernelParams& p, int b, int c) {
  if (c == 0 && p.fresh) return (float)cast_scale(p, b, c);
  return b == 0 ? s_scales0.next_f : p.state[b].next_scale_f;
}

// ---------------------------------------------------------------------------------------------
// Residual phases.  Anchor (FP64, Sec. 2's recurrence restarted from the accumulated solution):
// r = f - delta L_0 u.  Recurrence (mixed form, the paper's r_i = r_{i-1} - delta L(e_{i-1})):
// r = r_prev - delta L_0 e / s with e the previous cycle's correction in FP32 (scale s), the
// stencil applied in FP32 and r kept as an unevaluated sum hi + lo of two floats, updated with
// error-free transformations (Knuth's two-sum) on the FP32 pipe: about 48 significant bits, far
// more than the FP32 stencil term that is subtracted, and no FP64 instruction per node.  Both evaluate Eq. 5 as
// sigma-weighted differences (v_o - v_c) grouped in face, edge and corner classes, write the cast
// level-0 source of the next cycle and the max / L2 norms; Neumann images carry 2 k h g in the
// anchor (the correction e satisfies homogeneous conditions).  3-D tiles march in z keeping
// kOuterStages - 3 planes in flight (three resident for the stencil); 2-D tiles are pipelined across
// the CTA's tasks.
// ---------------------------------------------------------------------------------------------
template <typename V>
struct ResSrc {
  const V* u;          // operand, packed N^d array of the problem
  const V* s;          // sigma (heterogeneous problems)
  const double* rhs;   // anchor: f; recurrence: the hi/lo float pairs of r_prev, moved as 8-byte words
  const V* a;          // per-node a, or null for a_scalar
  double a_scalar;
  double opscale;      // r = rhs - opscale * (delta L v)
  float opscale32;     // the same, rounded to FP32 (recurrence)
  bool images;         // Neumann images carry the prescribed derivative (anchor only)
};

// Does the tile need Neumann image offsets (non-zero prescribed derivative on a face it touches)?
__device__ __forceinline__ bool tile_has_flux(const ProblemDesc& P, int N, int x0, int y0, int dim) {
  bool f = false;
  if (P.face_type[0] == 1 && P.face_value[0] != 0.0 && x0 == 0) f = true;
  if (P.face_type[1] == 1 && P.face_value[1] != 0.0 && x0 + kTX >= N - 1) f = true;
  if (P.face_type[2] == 1 && P.face_value[2] != 0.0 && y0 == 0) f = true;
  if (P.face_type[3] == 1 && P.face_value[3] != 0.0 && y0 + kTY >= N - 1) f = true;
  if (dim == 3 && ((P.face_type[4] == 1 && P.face_value[4] != 0.0) || (P.face_type[5] == 1 && P.face_value[5] != 0.0)))
    f = true;
  return f;
}

// Add one plane's contribution to the class sums of the thread's two nodes: the 4 x 3 block of
// cells around the two columns, dz = the plane's offset (-1, 0, +1).
template <typename V, bool HET>
__device__ __forceinline__ void res_plane(const ResStage<V>& S, int b0, int dz, const V uc[2], const V sc[2],
                                          V cls[2][3]) {
  V a[4][3], s[4][3];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      a[i][j] = S.u[b0 + i * kHX + j];
      if (HET) s[i][j] = S.s[b0 + i * kHX + j];
    }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int dy = i - 1, dx = j - 1;
        if (dx == 0 && dy == 0 && dz == 0) continue;
        const int nz = (dx != 0) + (dy != 0) + (dz != 0);
        const V du = a[r + i][j] - uc[r];
        if (HET) cls[r][nz - 1] = fma(sc[r] + s[r + i][j], du, cls[r][nz - 1]);
        else cls[r][nz - 1] += du;
      }
}

// Finish one node: r = rhs - opscale * (c0 * sum + a * v_c); store the cast source (and, in the
// mixed form, r as a hi/lo float pair); fold |r| and r^2 into the thread's norms (accumulated in
// V: FP64 for the anchor, FP32 for the recurrence, whose norms only steer the schedule).
__device__ __forceinline__ float nan_maxf(float a, float b) {
  if (a != a) return a;
  if (b != b) return b;
  return a > b ? a : b;
}

// Knuth's two-sum: s + e == a + b exactly (round-to-nearest, no contraction into FMA).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ float2 word_as_pair(double w) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(w);
  return make_float2(__uint_as_float((unsigned)(bits & 0xffffffffull)), __uint_as_float((unsigned)(bits >> 32)));
}

template <typename T, typename V>
__device__ __forceinline__ void res_finish(const ResSrc<V>& src, V c0v, V sum, V uc, V a, double rhs, double scale,
                                           float scale32, T* R0, float2* RES, long long idx, V& mx, V& s2) {
  if constexpr (sizeof(V) == 8) {
    const double r = __fma_rn(-src.opscale, __fma_rn((double)c0v, (double)sum, __dmul_rn((double)a, (double)uc)), rhs);
    mx = nan_max(mx, fabs(r));
    s2 = fma(r, r, s2);
    if (RES) {
      const float hi = (float)r;
      RES[idx] = make_float2(hi, (float)(r - (double)hi));
    }
    R0[idx] = (T)(r * scale);
  } else {
    const float d = __fmul_rn(__fmaf_rn(c0v, sum, __fmul_rn(a, uc)), src.opscale32);
    const float2 prev = word_as_pair(rhs);
    float hs, he, h, l;
    two_sum(prev.x, -d, hs, he);
    two_sum(hs, __fadd_rn(prev.y, he), h, l);
    RES[idx] = make_float2(h, l);
    R0[idx] = (T)(h * scale32);
    mx = nan_maxf(mx, fabsf(h));
    s2 = fmaf(h, h, s2);
  }
}

// A fresh solve whose lift is zero -- every Dirichlet value and every prescribed flux zero, and not an
// Eq. 10 problem (whose residuals follow the mean projection) -- starts from u = 0, so its first
// residual is r = f - delta L 0 = f exactly at every unknown: the anchor's values, bits included
// (the stencil terms are exact zeros), without reading u and sigma or spending FP64 instructions
// on the stencil.
template <int DIM>
__device__ __forceinline__ bool zero_lift(const ProblemDesc& P) {
  if (P.project_mean) return false;
#pragma unroll
  for (int k = 0; k < 2 * DIM; ++k)
    if (P.face_value[k] != 0.0) return false;
  return true;
}

// The anchor's bookkeeping of one unknown whose residual is r = f: norms and the float pair.
__device__ __forceinline__ void res_of_source(double f, float2* RES, long long idx, double& mx, double& s2) {
  mx = nan_max(mx, fabs(f));
  s2 = fma(f, f, s2);
  if (RES) {
    const float hi = (float)f;
    RES[idx] = make_float2(hi, (float)(f - (double)hi));
  }
}

template <typename T>
__device__ void residual3_zero(const KernelParams& p, const TileTask& tk, int c) {
  const ProblemDesc& P = prob_at(p, tk.b);
  const int N = level_side(P.n, 0);
  const Columns cl = own_columns(P, N, tk.x0, tk.y0);
  const double scale = outer_scale(p, tk.b, c);
  T* R0 = (T*)p.R + P.off_lvl[0];
  float2* RES = p.RESP ? p.RESP + P.off_full : nullptr;
  const double* F = p.F + P.off_full;
  const long long NN = (long long)N * N;
  double mx = 0.0, s2 = 0.0;
#pragma unroll 4
  for (int z = tk.z0; z < tk.z0 + tk.nz; ++z) {
    if (z_fixed(cl, z, N)) continue;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (!cl.in[r] || cl.fixed_xy[r]) continue;
      const long long idx = (long long)z * NN + cl.off[r];
      const double f = F[idx];
      res_of_source(f, RES, idx, mx, s2);
      R0[idx] = (T)(f * scale);
    }
  }
  block_flush(mx, s2, &p.accum[tk.b].rmax_bits[c & 1], &p.accum[tk.b].rsum2[c & 1]);
}

template <typename T, typename V, bool HET>
__device__ void residual3(const KernelParams& p, const TileTask& tk, int c, ResStage<V>* st, const ResSrc<V>& src) {
  constexpr int D = kOuterStages;
  const ProblemDesc& P = prob_at(p, tk.b);
  const int N = level_side(P.n, 0);
  const int tid = threadIdx.x;
  const Columns cl = own_columns(P, N, tk.x0, tk.y0);
  const double scale = outer_scale(p, tk.b, c);
  const float scale32 = outer_scale_f(p, tk.b, c);
  T* R0 = (T*)p.R + P.off_lvl[0];
  float2* RES = p.RESP ? p.RESP + P.off_full : nullptr;
  const bool flux = src.images && tile_has_flux(P, N, tk.x0, tk.y0, 3);
  const HaloCells hc = halo_cells(P, N, tk.x0, tk.y0, flux);
  const V c0v = cv<V>(P.c0 * (HET ? 1.0 : 2.0), P.c0_f * (HET ? 1.0f : 2.0f));
  const V a_s = cv<V>(src.a_scalar, P.a_scalar_f);
  const V w_e = cv<V>(p.w_edge, p.w_edge_f), w_c = cv<V>(p.w_corner, p.w_corner_f);
  const int b0 = (2 * (tid / kTX)) * kHX + (tid % kTX);  // top-left of the thread's 4 x 3 block
  const int nplanes = tk.nz + 2;
  const long long NN = (long long)N * N;
  V mx = (V)0, s2 = (V)0;
  auto issue = [&](int k) {
    if (k < nplanes) {
      ResStage<V>& S = st[k % D];
      const int zz = tk.z0 - 1 + k;
      const long long base = (long long)refl(zz, N) * NN;
      const V* u = src.u + base;
#pragma unroll
      for (int s = 0; s < kCells; ++s)
        if (hc.off[s] >= 0) {
          cp_async_t(&S.u[tid + s * kThreads], u + hc.off[s]);
          if (HET) cp_async_t(&S.s[tid + s * kThreads], src.s + base + hc.off[s]);
        }
      if (k >= 1 && k <= tk.nz) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
          if (cl.in[r]) {
            cp_async_t(&S.f[tid + r * kThreads], src.rhs + base + cl.off[r]);
            if (src.a) cp_async_t(&S.a[tid + r * kThreads], src.a + base + cl.off[r]);
          }
      }
    }
    cp_async_commit();
  };
  for (int k = 0; k < D - 3; ++k) issue(k);
  for (int k = 0; k < nplanes; ++k) {
    cp_async_wait<D - 4>();
    __syncthreads();
    issue(k + D - 3);
    if (flux) {  // Neumann images: u_image = u_mirror + 2 k h g, added once to the arrived plane
      ResStage<V>& S = st[k % D];
      const double gz = z_ghost(P, tk.z0 - 1 + k, N);
#pragma unroll
      for (int s = 0; s < kCells; ++s)
        if (hc.off[s] >= 0) S.u[tid + s * kThreads] += (V)(hc.ghost[s] + gz);
      __syncthreads();
    }
    if (k >= 2) {
      const int z = tk.z0 + k - 2;
      const ResStage<V>& S1 = st[(k - 1) % D];
      V uc[2], sc[2], cls[2][3];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        uc[r] = S1.u[b0 + (r + 1) * kHX + 1];
        sc[r] = HET ? S1.s[b0 + (r + 1) * kHX + 1] : (V)1;
        cls[r][0] = cls[r][1] = cls[r][2] = (V)0;
      }
      res_plane<V, HET>(st[(k - 2) % D], b0, -1, uc, sc, cls);
      res_plane<V, HET>(S1, b0, 0, uc, sc, cls);
      res_plane<V, HET>(st[k % D], b0, 1, uc, sc, cls);
      const bool zf = z_fixed(cl, z, N);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (!cl.in[r] || cl.fixed_xy[r] || zf) continue;
        const V sum = rn_fma(w_c, cls[r][2], rn_fma(w_e, cls[r][1], cls[r][0]));
        const V a = src.a ? S1.a[tid + r * kThreads] : a_s;
        res_finish<T, V>(src, c0v, sum, uc[r], a, S1.f[tid + r * kThreads], scale, scale32, R0, RES,
                         (long long)z * NN + cl.off[r], mx, s2);
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  block_flush((double)mx, (double)s2, &p.accum[tk.b].rmax_bits[c & 1], &p.accum[tk.b].rsum2[c & 1]);
}

// The FP32 recurrence with each plane's 4 x 3 block read from shared memory once: the block stays
// in registers for the next plane step, where it is the lower neighbour plane.  The node at plane
// m accumulates its class sums in the order dz = -1, 0 (step m), +1 (step m + 1) -- the order and
// arithmetic of residual3, so results are identical to it bit for bit, with a third of its
// shared-memory loads.
template <typename V, bool HET>
__device__ __forceinline__ void res_part(const V a[4][3], const V s[4][3], int dz, const V uc[2], const V sc[2],
                                         V cls[2][3]) {
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int dy = i - 1, dx = j - 1;
        if (dx == 0 && dy == 0 && dz == 0) continue;
        const int nz = (dx != 0) + (dy != 0) + (dz != 0);
        const V du = a[r + i][j] - uc[r];
        if (HET) cls[r][nz - 1] = fma(sc[r] + s[r + i][j], du, cls[r][nz - 1]);
        else cls[r][nz - 1] += du;
      }
}

template <typename T, bool HET>
__device__ void residual3r(const KernelParams& p, const TileTask& tk, int c, ResStage<T>* st, const ResSrc<T>& src) {
  using V = T;
  constexpr int D = kOuterStages;
  const ProblemDesc& P = prob_at(p, tk.b);
  const int N = level_side(P.n, 0);
  const int tid = threadIdx.x;
  const Columns cl = own_columns(P, N, tk.x0, tk.y0);
  const double scale = outer_scale(p, tk.b, c);
  const float scale32 = outer_scale_f(p, tk.b, c);
  T* R0 = (T*)p.R + P.off_lvl[0];
  float2* RES = p.RESP + P.off_full;
  const HaloCells hc = halo_cells(P, N, tk.x0, tk.y0, false);
  const V c0v = cv<V>(P.c0 * (HET ? 1.0 : 2.0), P.c0_f * (HET ? 1.0f : 2.0f));
  const V a_s = cv<V>(src.a_scalar, P.a_scalar_f);
  const V w_e = cv<V>(p.w_edge, p.w_edge_f), w_c = cv<V>(p.w_corner, p.w_corner_f);
  const int b0 = (2 * (tid / kTX)) * kHX + (tid % kTX);
  const int nplanes = tk.nz + 2;
  const long long NN = (long long)N * N;
  V mx = (V)0, s2 = (V)0;
  auto issue = [&](int k) {
    if (k < nplanes) {
      ResStage<V>& S = st[k % D];
      const long long base = (long long)refl(tk.z0 - 1 + k, N) * NN;
#pragma unroll
      for (int q = 0; q < kCells; ++q)
        if (hc.off[q] >= 0) {
          cp_async_t(&S.u[tid + q * kThreads], src.u + base + hc.off[q]);
          if (HET) cp_async_t(&S.s[tid + q * kThreads], src.s + base + hc.off[q]);
        }
      if (k >= 1 && k <= tk.nz) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
          if (cl.in[r]) {
            cp_async_t(&S.f[tid + r * kThreads], src.rhs + base + cl.off[r]);
            if (src.a) cp_async_t(&S.a[tid + r * kThreads], src.a + base + cl.off[r]);
          }
      }
    }
    cp_async_commit();
  };
  for (int k = 0; k < D - 3; ++k) issue(k);
  V pu[4][3], ps[4][3], puc[2], psc[2], pcls[2][3];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) pu[i][j] = ps[i][j] = (V)0;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    puc[r] = psc[r] = (V)0;
    pcls[r][0] = pcls[r][1] = pcls[r][2] = (V)0;
  }
  for (int k = 0; k < nplanes; ++k) {
    cp_async_wait<D - 4>();
    __syncthreads();
    issue(k + D - 3);
    const ResStage<V>& S = st[k % D];
    V a[4][3], sg[4][3], uc[2], sc[2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        a[i][j] = S.u[b0 + i * kHX + j];
        sg[i][j] = HET ? S.s[b0 + i * kHX + j] : (V)0;
      }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      uc[r] = a[r + 1][1];
      sc[r] = HET ? sg[r + 1][1] : (V)1;
    }
    if (k >= 2) {  // the nodes of plane k - 1 receive this plane (dz = +1) and are finished
      res_part<V, HET>(a, sg, 1, puc, psc, pcls);
      const int z = tk.z0 + k - 2;
      const bool zf = z_fixed(cl, z, N);
      const ResStage<V>& S1 = st[(k - 1) % D];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (!cl.in[r] || cl.fixed_xy[r] || zf) continue;
        const V sum = rn_fma(w_c, pcls[r][2], rn_fma(w_e, pcls[r][1], pcls[r][0]));
        const V av = src.a ? S1.a[tid + r * kThreads] : a_s;
        res_finish<T, V>(src, c0v, sum, puc[r], av, S1.f[tid + r * kThreads], scale, scale32, R0, RES,
                         (long long)z * NN + cl.off[r], mx, s2);
      }
    }
    V cls[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r) cls[r][0] = cls[r][1] = cls[r][2] = (V)0;
    if (k >= 1) res_part<V, HET>(pu, ps, -1, uc, sc, cls);
    res_part<V, HET>(a, sg, 0, uc, sc, cls);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        pu[i][j] = a[i][j];
        ps[i][j] = sg[i][j];
      }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      puc[r] = uc[r];
      psc[r] = sc[r];
      pcls[r][0] = cls[r][0];
      pcls[r][1] = cls[r][1];
      pcls[r][2] = cls[r][2];
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  block_flush((double)mx, (double)s2, &p.accum[tk.b].rmax_bits[c & 1], &p.accum[tk.b].rsum2[c & 1]);
}

// Residual sources of problem b in cycle c: the anchor (FP64 solution) or the recurrence (FP32
// correction of the previous cycle).
template <typename T>
__device__ __forceinline__ bool use_anchor(const KernelParams& p, int b, int c) {
  // Eq. 10 problems: every residual from the projected u (the FP32 recurrence does not follow the
  // projection's constant shift)
  return !p.mixed || c == 0 || p.state[b].anchor_next || prob_at(p, b).project_mean;
}

__device__ __forceinline__ ResSrc<double> anchor_src(const KernelParams& p, const ProblemDesc& P) {
  ResSrc<double> s;
  s.u = p.U + P.off_full;
  s.s = P.hetero ? p.SIG64 + P.off_full : nullptr;
  s.rhs = p.F + P.off_full;
  s.a = P.a_per_node ? p.A64 + P.off_full : nullptr;
  s.a_scalar = P.a_scalar;
  s.opscale = 1.0;
  s.opscale32 = 1.0f;
  s.images = true;
  return s;
}

template <typename T>
__device__ __forceinline__ ResSrc<T> recur_src(const KernelParams& p, const ProblemDesc& P, int b, int c) {
  ResSrc<T> s;
  // the cycle's last level-0 sweep wrote E2 after an even number of flips before it, E otherwise
  const int flips = visit_flips(p, 0, visit_sweeps(p.n_r, P.n, 0, true));
  s.u = (((flips - 1) & 1) ? (const T*)p.E : (const T*)p.E2) + P.off_lvl[0];
  s.s = P.hetero ? (const T*)p.SIG + P.off_lvl[0] : nullptr;
  s.rhs = reinterpret_cast<const double*>(p.RESP + P.off_full);
  s.a = P.a_per_node ? (const T*)p.A0 + P.off_lvl[0] : nullptr;
  s.a_scalar = P.a_scalar;
  s.opscale = inv_scale_at(p, b, (c - 1) & 1);
  s.opscale32 = inv_scale_f_at(p, b, (c - 1) & 1);
  s.images = false;
  return s;
}

// 2-D: one halo tile per task, the CTA's tasks pipelined kOuterStages - 2 deep, in one pass: each
// task's problem takes the FP64 anchor or (mixed form) the FP32 recurrence.  The stage slots are
// sized for the anchor's FP64 layout, so both kinds of tile share the pipeline (two passes over all
// tiles, one per kind, cost a pipeline wait and a CTA barrier per skipped tile).
// The loads of a 2-D residual tile: the operand and sigma on the halo, the right-hand side and a at
// the tile's nodes (pointers already offset to the problem's arrays; P is read only on the level's
// edges).
template <typename V>
__device__ __forceinline__ void res2_issue(const KernelParams& p, const TileTask& tk, int N, ResStage<V>& S,
                                           const V* u, const V* sg, const double* rhs, const V* a) {
  const int tid = threadIdx.x;
  HaloCells hc;
  Columns cl;
  if (tile_interior(N, tk.x0, tk.y0)) {
    hc = halo_cells_2d(s_prob0, N, tk.x0, tk.y0, true);  // the descriptor is not read
    cl = own_columns_2d(s_prob0, N, tk.x0, tk.y0, true);
  } else {
    const ProblemDesc& P = prob_at(p, tk.b);
    hc = halo_cells(P, N, tk.x0, tk.y0, false);
    cl = own_columns(P, N, tk.x0, tk.y0);
  }
#pragma unroll
  for (int s = 0; s < kCells; ++s)
    if (hc.off[s] >= 0) {
      cp_async_t(&S.u[tid + s * kThreads], u + hc.off[s]);
      if (sg) cp_async_t(&S.s[tid + s * kThreads], sg + hc.off[s]);
    }
#pragma unroll
  for (int r = 0; r < 2; ++r)
    if (cl.in[r]) {
      cp_async_t(&S.f[tid + r * kThreads], rhs + cl.off[r]);
      if (a) cp_async_t(&S.a[tid + r * kThreads], a + cl.off[r]);
    }
}

template <typename T, typename V>
__device__ __forceinline__ void res2_compute(const KernelParams& p, const ProblemDesc& P, const TileTask& tk, int c,
                                             ResStage<V>& S, const ResSrc<V>& src, V& mx, V& s2) {
  const int tid = threadIdx.x;
  const int b0 = (2 * (tid / kTX)) * kHX + (tid % kTX);
  const int N = level_side(P.n, 0);
  if (src.images && tile_has_flux(P, N, tk.x0, tk.y0, 2)) {
    const HaloCells hc = halo_cells(P, N, tk.x0, tk.y0, true);
#pragma unroll
    for (int s = 0; s < kCells; ++s)
      if (hc.off[s] >= 0) S.u[tid + s * kThreads] += (V)hc.ghost[s];
    __syncthreads();
  }
  const Columns cl = own_columns_2d(P, N, tk.x0, tk.y0, tile_interior(N, tk.x0, tk.y0));
  V uc[2], sc[2], cls[2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    uc[r] = S.u[b0 + (r + 1) * kHX + 1];
    sc[r] = src.s ? S.s[b0 + (r + 1) * kHX + 1] : (V)1;
    cls[r][0] = cls[r][1] = cls[r][2] = (V)0;
  }
  if (src.s) res_plane<V, true>(S, b0, 0, uc, sc, cls);
  else res_plane<V, false>(S, b0, 0, uc, sc, cls);
  const V c0v = cv<V>(P.c0 * (src.s ? 1.0 : 2.0), P.c0_f * (src.s ? 1.0f : 2.0f));
  const double scale = outer_scale(p, tk.b, c);
  const float scale32 = outer_scale_f(p, tk.b, c);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (!cl.in[r] || cl.fixed_xy[r]) continue;
    const V sum = rn_fma(cv<V>(p.w_edge, p.w_edge_f), cls[r][1], cls[r][0]);
    const V a = src.a ? S.a[tid + r * kThreads] : cv<V>(src.a_scalar, P.a_scalar_f);
    res_finish<T, V>(src, c0v, sum, uc[r], a, S.f[tid + r * kThreads], scale, scale32, (T*)p.R + P.off_lvl[0],
                     p.RESP ? p.RESP + P.off_full : nullptr, cl.off[r], mx, s2);
  }
}

// 2-D tile of a fresh zero-lift problem's first residual (r = f, see residual3_zero).
template <typename T>
__device__ __forceinline__ void res2_zero(const KernelParams& p, const ProblemDesc& P, const TileTask& tk, int c,
                                          double& mx, double& s2) {
  const int N = level_side(P.n, 0);
  const Columns cl = own_columns_2d(P, N, tk.x0, tk.y0, tile_interior(N, tk.x0, tk.y0));
  const double scale = outer_scale(p, tk.b, c);
  T* R0 = (T*)p.R + P.off_lvl[0];
  float2* RES = p.RESP ? p.RESP + P.off_full : nullptr;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (!cl.in[r] || cl.fixed_xy[r]) continue;
    const double f = p.F[P.off_full + cl.off[r]];
    res_of_source(f, RES, cl.off[r], mx, s2);
    R0[cl.off[r]] = (T)(f * scale);
  }
}

template <typename T>
__device__ void residual2(const KernelParams& p, int c, unsigned char* smem) {
  constexpr int D = kOuterStages;
  constexpr size_t kSlot = sizeof(ResStage<double>);
  static_assert(sizeof(ResStage<T>) <= kSlot && kSlot % 16 == 0, "residual stage slots");
  const int t0 = s_toff[0][0], J = s_toff[0][1] - s_toff[0][0];  // level 0
  auto task = [&](int j) -> const TileTask& { return p.tasks[t0 + j]; };
  auto slot = [&](int j) { return smem + (size_t)(j % D) * kSlot; };
  // The loads keep the sources of the last problem they met (a CTA's tasks run problem by problem).
  int ib = -1, ikind = 0;  // ikind: 0 none (problem done), 1 FP64 anchor, 2 FP32 recurrence
  int iN = 0;
  const void *iu = nullptr, *isg = nullptr, *ia = nullptr;
  const double* irhs = nullptr;
  auto issue = [&](int j) {
    if (j < J) {
      const TileTask tk = task(j);  // by value: the cp.async statements clobber memory
      if (tk.b != ib) {
        ib = tk.b;
        const ProblemDesc& P = prob_at(p, ib);
        iN = level_side(P.n, 0);
        ikind = done_at(p, ib) ? 0 : (c == 0 && p.fresh && zero_lift<2>(P) ? 3 : (use_anchor<T>(p, ib, c) ? 1 : 2));
        if (ikind == 1) {
          const ResSrc<double> src = anchor_src(p, P);
          iu = src.u, isg = src.s, irhs = src.rhs, ia = src.a;
        } else if (ikind == 2) {
          if constexpr (sizeof(T) == 4) {
            const ResSrc<T> src = recur_src<T>(p, P, ib, c);
            iu = src.u, isg = src.s, irhs = src.rhs, ia = src.a;
          }
        }
      }
      if (ikind == 1) {
        res2_issue<double>(p, tk, iN, *(ResStage<double>*)slot(j), (const double*)iu, (const double*)isg, irhs,
                           (const double*)ia);
      } else if (ikind == 2) {
        if constexpr (sizeof(T) == 4)
          res2_issue<T>(p, tk, iN, *(ResStage<T>*)slot(j), (const T*)iu, (const T*)isg, irhs, (const T*)ia);
      }
    }
    cp_async_commit();
  };
  // The norms of a problem's tiles are summed per thread and flushed (one block reduction and two
  // atomics) when the CTA moves to another problem: a CTA's tasks run problem by problem, and a
  // flush per tile costs a CTA barrier and FP64 reductions per 512 nodes.
  int ab = -1;          // problem whose norms are being summed (-1: none)
  int akind = 0;        // ... through the FP64 anchor (1) or r = f (3): double sums; the recurrence (2): V = T
  double dmx = 0.0, ds2 = 0.0;
  T fmx = (T)0, fs2 = (T)0;
  auto flush = [&]() {  // uniform over the CTA (block_flush holds CTA barriers)
    if (ab < 0) return;
    if (akind != 2) block_flush(dmx, ds2, &p.accum[ab].rmax_bits[c & 1], &p.accum[ab].rsum2[c & 1]);
    else block_flush((double)fmx, (double)fs2, &p.accum[ab].rmax_bits[c & 1], &p.accum[ab].rsum2[c & 1]);
    dmx = ds2 = 0.0;
    fmx = fs2 = (T)0;
    ab = -1;
  };
  for (int j = 0; j < D - 2; ++j) issue(j);
  for (int j = 0; j < J; ++j) {
    cp_async_wait<D - 3>();
    __syncthreads();
    issue(j + D - 2);
    const TileTask tk = task(j);
    if (done_at(p, tk.b)) continue;  // uniform over the CTA
    if (tk.b != ab) {
      flush();
      ab = tk.b;
      akind = c == 0 && p.fresh && zero_lift<2>(prob_at(p, ab)) ? 3 : (use_anchor<T>(p, tk.b, c) ? 1 : 2);
    }
    const ProblemDesc& P = prob_at(p, tk.b);
    if (akind == 3) {
      res2_zero<T>(p, P, tk, c, dmx, ds2);
    } else if (akind == 1) {
      res2_compute<T, double>(p, P, tk, c, *(ResStage<double>*)slot(j), anchor_src(p, P), dmx, ds2);
    } else if constexpr (sizeof(T) == 4) {
      res2_compute<T, T>(p, P, tk, c, *(ResStage<T>*)slot(j), recur_src<T>(p, P, tk.b, c), fmx, fs2);
    }
  }
  flush();
  cp_async_wait<0>();
  __syncthreads();
}

template <typename T, int DIM>
__device__ void phase_outer(const KernelParams& p, int c, unsigned char* smem) {
  if (DIM == 2) {
    residual2<T>(p, c, smem);
    return;
  }
  for_tasks(p, 0, [&](const TileTask& tk) {
    if (done_at(p, tk.b)) return;
    const ProblemDesc& P = prob_at(p, tk.b);
    if (c == 0 && p.fresh && zero_lift<3>(P)) {
      residual3_zero<T>(p, tk, c);
    } else if (use_anchor<T>(p, tk.b, c)) {
      const ResSrc<double> src = anchor_src(p, P);
      if (P.hetero) residual3<T, double, true>(p, tk, c, (ResStage<double>*)smem, src);
      else residual3<T, double, false>(p, tk, c, (ResStage<double>*)smem, src);
    } else {
      const ResSrc<T> src = recur_src<T>(p, P, tk.b, c);
      if constexpr (sizeof(T) == 4) {
        if (P.hetero) residual3r<T, true>(p, tk, c, (ResStage<T>*)smem, src);
        else residual3r<T, false>(p, tk, c, (ResStage<T>*)smem, src);
      } else {
        if (P.hetero) residual3<T, T, true>(p, tk, c, (ResStage<T>*)smem, src);
        else residual3<T, T, false>(p, tk, c, (ResStage<T>*)smem, src);
      }
    }
  });
}

// Convergence check after the outer step of cycle c (CTA 0 only): relative residuals, stop
// decisions, history, next cast scale.  Writes sync->active[c & 1].
template <typename T, int DIM>
__device__ void phase_check(const KernelParams& p, int c) {
  int any = 0;
  for (int b = threadIdx.x; b < p.batch; b += blockDim.x) {
    ProblemState& S = p.state[b];
    Accum& A = p.accum[b];
    if (A.done) continue;
    const double rmax = __longlong_as_double((long long)A.rmax_bits[c & 1]);
    const double rs2 = A.rsum2[c & 1];
    if (c == 0 && p.fresh) {
      const double fmax = __longlong_as_double((long long)A.fmax_bits);
      S.fnorm = fmax > 0.0 ? fmax : rmax;
      S.fnorm2 = fmax > 0.0 ? sqrt(A.fsum2) : sqrt(rs2);
      S.rel_prev = 1e300;
      S.grow = 0;
    }
    S.scale_used[c & 1] = cast_scale(p, b, c);
    S.inv_scale[c & 1] = 1.0 / S.scale_used[c & 1];
    S.inv_scale_f[c & 1] = (float)S.inv_scale[c & 1];
    // (a NaN norm must stay NaN: it ends the solve with SGML_ERR_NONFINITE below, not as converged)
    const double rel = S.fnorm > 0.0 ? rmax / S.fnorm : (S.fnorm == 0.0 ? 0.0 : S.fnorm + rmax);
    const double rel2 = S.fnorm2 > 0.0 ? sqrt(rs2) / S.fnorm2 : (S.fnorm2 == 0.0 ? 0.0 : S.fnorm2 + rs2);
    S.rel = rel;
    S.rel_l2 = rel2;
    if (c < p.hist_cap) p.hist[(long long)b * p.hist_cap + c] = rel;
    S.hist_len = c + 1;
    if (c > 0) S.cycles += 1;
    const bool anchored = !p.mixed || c == 0 || S.anchor_next;
    S.grow = (rel > S.rel_prev) ? S.grow + 1 : 0;
    S.rel_prev = rel;
    S.rmax_prev = rmax;
    S.next_scale = cast_scale(p, b, c + 1);
    S.next_scale_f = (float)S.next_scale;
    if (anchored) {
      S.anchor_rel = rel;
      S.last_anchor = c;
    }
    int st = 0, stop = 0;
    if (!(rel <= 1e300)) {
      st = -6;  // SGML_ERR_NONFINITE
      stop = 1;
    } else if (anchored && rel <= p.tol) {
      stop = 1;
    } else if (S.grow >= 3 && rel > 1.0) {
      st = -4;  // SGML_ERR_DIVERGED
      stop = 1;
    } else if (c >= p.max_cycles) {
      st = p.tol >= 0.0 ? -3 : 0;  // SGML_ERR_NOT_CONVERGED for a solve; fine for run_cycle
      stop = 1;
    }
    // Mixed form: the next residual is the FP64 anchor once the residual fell 1e4-fold since the last
    // anchor or 64 cycles passed, when the tolerance may have been reached, and after the launch's
    // last cycle.  The recurrence's error is that of the FP32 stencil applied to each correction,
    // ~1e-7 of the residual it removes (measured at 257^3: the recurrence residual within 1.3e-7 of
    // the exact FP64 residual of the same iterate), so after a 1e4-fold fall it is still ~1e-3 of
    // the current residual; convergence is accepted on anchored residuals only.
    S.anchor_next = !p.mixed || rel <= 1e-4 * S.anchor_rel || rel <= p.tol || c + 1 >= p.max_cycles ||
                    c + 1 - S.last_anchor >= 64;
    S.status = st;
    A.done = stop;
    A.rmax_bits[(c + 1) & 1] = 0ull;
    A.rsum2[(c + 1) & 1] = 0.0;
    if (!stop) any = 1;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) p.sync->active[c & 1] = any;
}

// ---------------------------------------------------------------------------------------------
// Jacobi sweep of the pseudo-time equation at level l (Eq. 2, explicit Euler, local step):
//   e_new = e + dtau (delta L_l e - r_l)
//         = (1 - omega) e_i + q_i (sigma_i CS(e) + CS(sigma e) - r_i / c),  c = kappa / (2 H^2),
// with CS(v) = sum_o w_o v_{i+o} over the level-l neighbours, q_i = dtau_i c and
// omega = dtau_i D_i (constant for the Jacobi-scaled step).  3-D: each plane's in-plane face and
// corner sums of the thread's two nodes come from one 4 x 3 block of shared memory and are combined
// across three planes held in registers (faces = F(z) + v(z-1) + v(z+1), edges = C(z) + F(z-1) +
// F(z+1), corners = C(z-1) + C(z+1)); plane loads run kSweepStages - 2 planes ahead with cp.async.
// The last sweep of a cycle adds its result, unscaled, to the FP64 solution (and keeps it as the
// recurrence operand in the mixed form).
// ---------------------------------------------------------------------------------------------
template <typename T>
struct PlaneSums {
  T v, F, C;     // e at the own column, in-plane face sum, in-plane corner sum
  T sv, sF, sC;  // the same for sigma * e
};

struct SweepCtl {
  bool active, zero_in, last;
  int N;
  long long off;
};

__device__ __forceinline__ SweepCtl sweep_ctl(const KernelParams& p, const Phase& ph, int b) {
  SweepCtl s;
  const ProblemDesc& P = prob_at(p, b);
  const bool final_visit = (ph.flags & kFinalVisit) != 0;
  const int k_b = visit_sweeps(p.n_r, P.n, ph.tooth, final_visit);
  const int span = (ph.flags & kPair) ? 2 : 1;  // sweeps this phase performs
  s.active = !done_at(p, b) && ph.tooth <= P.n - 1 && ph.sweep + span - 1 < k_b;
  s.zero_in = ph.sweep == 0 && (ph.flags & kFirstOfTooth) && ph.tooth == P.n - 1;
  s.last = final_visit && ph.sweep + span - 1 == k_b - 1;
  s.N = level_side(P.n, ph.level);
  s.off = P.off_lvl[ph.level];
  return s;
}

// In-plane sums of the thread's two nodes from the 4 x 3 block at b0.
template <typename T, bool HET>
__device__ __forceinline__ void plane_sums2(const SweepStage<T>& S, int b0, bool zero, PlaneSums<T> ps[2]) {
  if (zero) {
#pragma unroll
    for (int r = 0; r < 2; ++r) ps[r].v = ps[r].F = ps[r].C = ps[r].sv = ps[r].sF = ps[r].sC = (T)0;
    return;
  }
  T a[4][3], se[4][3];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      a[i][j] = S.e[b0 + i * kHX + j];
      if (HET) se[i][j] = rn_mul(S.s[b0 + i * kHX + j], a[i][j]);
    }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    ps[r].v = a[r + 1][1];
    ps[r].F = (a[r + 1][0] + a[r + 1][2]) + (a[r][1] + a[r + 2][1]);
    ps[r].C = (a[r][0] + a[r][2]) + (a[r + 2][0] + a[r + 2][2]);
    if (HET) {
      ps[r].sv = se[r + 1][1];
      ps[r].sF = (se[r + 1][0] + se[r + 1][2]) + (se[r][1] + se[r + 2][1]);
      ps[r].sC = (se[r][0] + se[r][2]) + (se[r + 2][0] + se[r + 2][2]);
    } else {
      ps[r].sv = ps[r].sF = ps[r].sC = (T)0;
    }
  }
}

// Per-task constants of the update: 1 - omega, 1 / c = 2 H^2 / kappa, and q for a homogeneous problem
// (precomputed per level on the host: an FP64 division per tile costs the FP64 pipe ~1 us per phase).
template <typename T>
struct SweepConst {
  T one_m_omega, inv_c, q_const, w_e, w_c;
};

template <typename T>
__device__ __forceinline__ SweepConst<T> sweep_const(const KernelParams& p, const ProblemDesc& P, int l) {
  SweepConst<T> k;
  k.one_m_omega = cv<T>(1.0 - p.omega, p.one_m_omega_f);
  k.inv_c = cv<T>(P.inv_c[l], P.inv_c_f[l]);
  k.q_const = cv<T>(P.q_const[l], P.q_const_f[l]);
  k.w_e = cv<T>(p.w_edge, p.w_edge_f);
  k.w_c = cv<T>(p.w_corner, p.w_corner_f);
  return k;
}

template <typename T, bool HET>
__device__ __forceinline__ T sweep_update(const SweepConst<T>& k, const SweepStage<T>& S, int slot, int cc, T CSe,
                                          T CSse, T e_c) {
  const T r_i = S.r[slot];
  if (HET) return rn_fma(S.q[slot], rn_fma(-r_i, k.inv_c, rn_fma(S.s[cc], CSe, CSse)), rn_mul(k.one_m_omega, e_c));
  return rn_fma(k.q_const, rn_fma(-r_i, k.inv_c, rn_mul((T)2, CSe)), rn_mul(k.one_m_omega, e_c));
}

template <typename T, bool HET, bool LAST, bool DIAG = false>
__device__ void sweep3(const KernelParams& p, const Phase& ph, int c, const TileTask& tk, SweepStage<T>* st,
                       const SweepCtl& sc) {
  constexpr int D = kSweepStages;
  const ProblemDesc& P = prob_at(p, tk.b);
  const int N = sc.N;
  const int tid = threadIdx.x;
  const Columns cl = own_columns(P, N, tk.x0, tk.y0);
  const bool odd = sweep_parity(p, ph.level, ph.sweep) != 0;
  const T* src = odd ? (const T*)p.E2 + sc.off : (const T*)p.E + sc.off;
  T* dst = odd ? (T*)p.E + sc.off : (T*)p.E2 + sc.off;
  const T* R = (const T*)p.R + sc.off;
  const T* SG = HET ? (const T*)p.SIG + sc.off : nullptr;
  const T* Q = HET ? (const T*)p.Q + sc.off : nullptr;
  double* Ug = p.U + P.off_full;
  const HaloCells hc = halo_cells(P, N, tk.x0, tk.y0, false);
  const SweepConst<T> kc = sweep_const<T>(p, P, ph.level);
  const int b0 = (2 * (tid / kTX)) * kHX + (tid % kTX);
  const double inv_scale = LAST ? inv_scale_at(p, tk.b, c & 1) : 0.0;
  const bool keep = !LAST || p.mixed;
  const bool zero_in = sc.zero_in;
  const int nplanes = tk.nz + 2;
  const long long NN = (long long)N * N;
  auto issue = [&](int k) {
    if (k < nplanes) {
      SweepStage<T>& S = st[k % D];
      const int zz = tk.z0 - 1 + k;
      const unsigned base = (unsigned)refl(zz, N) * (unsigned)NN;
#pragma unroll
      for (int s = 0; s < kCells; ++s)
        if (hc.off[s] >= 0) {
          const unsigned o = base + (unsigned)hc.off[s];
          if (!zero_in) cp_async_t(&S.e[tid + s * kThreads], src + o);
          if (HET) cp_async_t(&S.s[tid + s * kThreads], SG + o);
        }
      if (k >= 1 && k <= tk.nz) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
          if (cl.in[r]) {
            const unsigned o = base + (unsigned)cl.off[r];
            cp_async_t(&S.r[tid + r * kThreads], R + o);
            if (HET) cp_async_t(&S.q[tid + r * kThreads], Q + o);
            if (LAST) cp_async_t(&S.u[tid + r * kThreads], Ug + o);
          }
      }
    }
    cp_async_commit();
  };
  // A piece of one plane (the coarse levels' usual share) fetches its three planes in one round trip.
  const int pre = nplanes <= D - 1 ? nplanes : D - 2;
  for (int k = 0; k < pre; ++k) issue(k);
  T dmx = (T)0;  // diagnostic pseudo-residual of the thread's nodes, times inv_c (DIAG)
  // One plane step: wait for plane k, start plane k + D - 2, form its in-plane sums into `nw`,
  // update the nodes of plane k - 1 from (m, o, nw).  The z loop is unrolled by three so that the
  // three-plane window rotates by renaming instead of moving registers.
  auto step = [&](int k, const PlaneSums<T>* m, const PlaneSums<T>* o, PlaneSums<T>* nw) {
    cp_async_wait<D - 3>();
    __syncthreads();
    if (k + D - 2 >= pre) issue(k + D - 2);
    else cp_async_commit();
    plane_sums2<T, HET>(st[k % D], b0, zero_in, nw);
    if (k >= 2) {
      const int z = tk.z0 + k - 2;
      const bool zf = z_fixed(cl, z, N);
      const SweepStage<T>& S = st[(k - 1) % D];
      const unsigned zoff = (unsigned)z * (unsigned)NN;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (!cl.in[r] || cl.fixed_xy[r] || zf) continue;
        const T CSe = rn_fma(kc.w_c, m[r].C + nw[r].C,
                             rn_fma(kc.w_e, (o[r].C + m[r].F) + nw[r].F, (o[r].F + m[r].v) + nw[r].v));
        const T CSse = HET ? rn_fma(kc.w_c, m[r].sC + nw[r].sC,
                                    rn_fma(kc.w_e, (o[r].sC + m[r].sF) + nw[r].sF, (o[r].sF + m[r].sv) + nw[r].sv))
                           : (T)0;
        const int slot = tid + r * kThreads;
        const T e_new = sweep_update<T, HET>(kc, S, slot, b0 + (r + 1) * kHX + 1, CSe, CSse, o[r].v);
        if (DIAG) dmx = fmax(dmx, diag_term(e_new - o[r].v, HET ? S.q[slot] : kc.q_const));
        const unsigned idx = zoff + (unsigned)cl.off[r];
        if (LAST) Ug[idx] = __fma_rn((double)e_new, inv_scale, S.u[slot]);
        if (keep) dst[idx] = e_new;
      }
    }
  };
  PlaneSums<T> A[2], B[2], C[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) A[r] = B[r] = C[r] = PlaneSums<T>{};
  for (int k = 0; k < nplanes; k += 3) {
    step(k, A, B, C);
    if (k + 1 < nplanes) step(k + 1, B, C, A);
    if (k + 2 < nplanes) step(k + 2, C, A, B);
  }
  cp_async_wait<0>();
  __syncthreads();
  if (DIAG) diag_flush<T>(p, tk.b, c, ph.level, dmx, kc.inv_c);
}

// ---------------------------------------------------------------------------------------------
// Level sweep of the FP64 form (3-D).  On a GPU with a narrow FP64 pipe the FP64 sweep is bound by
// its FP64 instruction count, not by HBM, so its arithmetic is arranged to need fewer of them (25
// per node for a heterogeneous problem instead of 36) -- the same Jacobi update (Eq. 2 with the
// radial stencil of Eq. 5), summed in another order:
//   - sigma * e is formed once per halo cell (in place of sigma in shared memory, after each
//     thread has kept sigma at its own two nodes), not once per use by the 2 x 3 threads around it;
//   - a thread's two nodes share the horizontal pair sums of its 4 x 3 block (face sums
//     F = A(r + 1) + (v(r) + v(r + 2)), corner sums C = A(r) + A(r + 2), A(r) = v(r, x-1) + v(r, x+1));
//   - the z sums are rolled as in the four-row sweep: with t = v + w_e F + w_c C and m = F + w_e C
//     of a plane, CS at plane z is (m_z + t_{z-1}) + t_{z+1} (two registers per node and array
//     instead of three planes of sums).
// Explicitly rounded throughout, so every node's value is independent of the tile and launch shape.
// ---------------------------------------------------------------------------------------------
template <bool HET, bool LAST>
__device__ void sweep3_f64(const KernelParams& p, const Phase& ph, int c, const TileTask& tk, SweepStage<double>* st,
                           const SweepCtl& sc) {
  using T = double;
  constexpr int D = kSweepStages;
  const ProblemDesc& P = prob_at(p, tk.b);
  const int N = sc.N;
  const int tid = threadIdx.x;
  const Columns cl = own_columns(P, N, tk.x0, tk.y0);
  const bool odd = sweep_parity(p, ph.level, ph.sweep) != 0;
  const T* src = odd ? (const T*)p.E2 + sc.off : (const T*)p.E + sc.off;
  T* dst = odd ? (T*)p.E + sc.off : (T*)p.E2 + sc.off;
  const T* R = (const T*)p.R + sc.off;
  const T* SG = HET ? (const T*)p.SIG + sc.off : nullptr;
  const T* Q = HET ? (const T*)p.Q + sc.off : nullptr;
  double* Ug = p.U + P.off_full;
  const HaloCells hc = halo_cells(P, N, tk.x0, tk.y0, false);
  const SweepConst<T> kc = sweep_const<T>(p, P, ph.level);
  const int b0 = (2 * (tid / kTX)) * kHX + (tid % kTX);
  const double inv_scale = LAST ? inv_scale_at(p, tk.b, c & 1) : 0.0;
  const bool zero_in = sc.zero_in;
  const int nplanes = tk.nz + 2;
  const unsigned NN = (unsigned)N * (unsigned)N;
  auto issue = [&](int k) {
    if (k < nplanes) {
      SweepStage<T>& S = st[k % D];
      const unsigned base = (unsigned)refl(tk.z0 - 1 + k, N) * NN;
#pragma unroll
      for (int q = 0; q < kCells; ++q)
        if (hc.off[q] >= 0) {
          const unsigned o = base + (unsigned)hc.off[q];
          if (!zero_in) cp_async_t(&S.e[tid + q * kThreads], src + o);
          if (HET) cp_async_t(&S.s[tid + q * kThreads], SG + o);
        }
      if (k >= 1 && k <= tk.nz) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
          if (cl.in[r]) {
            const unsigned o = base + (unsigned)cl.off[r];
            cp_async_t(&S.r[tid + r * kThreads], R + o);
            if (HET) cp_async_t(&S.q[tid + r * kThreads], Q + o);
            if (LAST) cp_async_t(&S.u[tid + r * kThreads], Ug + o);
          }
      }
    }
    cp_async_commit();
  };
  const int pre = nplanes <= D - 1 ? nplanes : D - 2;
  for (int k = 0; k < pre; ++k) issue(k);
  // rolled z sums (Se = m_{z} + t_{z-1} awaiting t_{z+1}, Te = t_z) of e and sigma e, and e and sigma
  // at the thread's two nodes one plane behind
  T Se[2], Te[2], Ss[2], Ts[2], vp[2], sp[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) Se[r] = Te[r] = Ss[r] = Ts[r] = vp[r] = sp[r] = (T)0;
  for (int k = 0; k < nplanes; ++k) {
    cp_async_wait<D - 3>();
    __syncthreads();
    if (k + D - 2 >= pre) issue(k + D - 2);
    else cp_async_commit();
    SweepStage<T>& S = st[k % D];
    T t[2], m[2], ts[2], ms[2], v[2], sv[2];
    if (zero_in) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        t[r] = m[r] = ts[r] = ms[r] = v[r] = (T)0;
        sv[r] = HET ? S.s[b0 + (r + 1) * kHX + 1] : (T)0;
      }
    } else {
      if (HET) {  // sigma at the own nodes, then sigma * e in place of sigma on the plane's halo tile
#pragma unroll
        for (int r = 0; r < 2; ++r) sv[r] = S.s[b0 + (r + 1) * kHX + 1];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kCells; ++q)
          if (hc.off[q] >= 0) S.s[tid + q * kThreads] = rn_mul(S.s[tid + q * kThreads], S.e[tid + q * kThreads]);
        __syncthreads();
      }
      T a[4][3], se[4][3];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          a[i][j] = S.e[b0 + i * kHX + j];
          if (HET) se[i][j] = S.s[b0 + i * kHX + j];
        }
      T A[4], As[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        A[i] = rn_add(a[i][0], a[i][2]);
        if (HET) As[i] = rn_add(se[i][0], se[i][2]);
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const T F = rn_add(A[r + 1], rn_add(a[r][1], a[r + 2][1]));
        const T C = rn_add(A[r], A[r + 2]);
        v[r] = a[r + 1][1];
        t[r] = rn_fma(kc.w_c, C, rn_fma(kc.w_e, F, v[r]));
        m[r] = rn_fma(kc.w_e, C, F);
        if (HET) {
          const T sF = rn_add(As[r + 1], rn_add(se[r][1], se[r + 2][1]));
          const T sC = rn_add(As[r], As[r + 2]);
          ts[r] = rn_fma(kc.w_c, sC, rn_fma(kc.w_e, sF, se[r + 1][1]));
          ms[r] = rn_fma(kc.w_e, sC, sF);
        } else {
          ts[r] = ms[r] = sv[r] = (T)0;
        }
      }
    }
    if (k >= 2) {  // the nodes of plane k - 1 receive this plane (dz = +1) and are updated
      const int z = tk.z0 + k - 2;
      const bool zf = z_fixed(cl, z, N);
      const SweepStage<T>& S1 = st[(k - 1) % D];
      const unsigned zoff = (unsigned)z * NN;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (!cl.in[r] || cl.fixed_xy[r] || zf) continue;
        const int slot = tid + r * kThreads;
        const T CSe = rn_add(Se[r], t[r]);
        const T r_i = S1.r[slot];
        T e_new;
        if (HET) {
          const T CSse = rn_add(Ss[r], ts[r]);
          e_new = rn_fma(S1.q[slot], rn_fma(-r_i, kc.inv_c, rn_fma(sp[r], CSe, CSse)), rn_mul(kc.one_m_omega, vp[r]));
        } else {
          e_new = rn_fma(kc.q_const, rn_fma(-r_i, kc.inv_c, rn_mul((T)2, CSe)), rn_mul(kc.one_m_omega, vp[r]));
        }
        const unsigned idx = zoff + (unsigned)cl.off[r];
        if (LAST) Ug[idx] = __fma_rn(e_new, inv_scale, S1.u[slot]);
        else dst[idx] = e_new;
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      Se[r] = rn_add(m[r], Te[r]);
      Te[r] = t[r];
      if (HET) {
        Ss[r] = rn_add(ms[r], Ts[r]);
        Ts[r] = ts[r];
      }
      vp[r] = v[r];
      sp[r] = sv[r];
    }
  }
  cp_async_wait<0>();
  __syncthreads();
}

// 2-D: one halo tile per task, the CTA's tasks pipelined kSweepStages - 2 deep, in one pass: whether
// this is a problem's last sweep of the cycle (adding e / s into the FP64 solution) is decided per
// tile (two passes, one per kind, cost a pipeline wait and a CTA barrier per skipped tile).
template <typename T, bool DIAG = false>
__device__ void sweep2(const KernelParams& p, const Phase& ph, int c, SweepStage<T>* st) {
  constexpr int D = kSweepStages;
  const int l = ph.level;
  const int t0 = s_toff[l][0], J = s_toff[l][1] - s_toff[l][0];
  const int tid = threadIdx.x;
  const int b0 = (2 * (tid / kTX)) * kHX + (tid % kTX);
  const bool odd = sweep_parity(p, l, ph.sweep) != 0;
  const T* Esrc = odd ? (const T*)p.E2 : (const T*)p.E;
  T* Edst = odd ? (T*)p.E : (T*)p.E2;
  auto task = [&](int j) -> const TileTask& { return p.tasks[t0 + j]; };
  // The control of a tile (SweepCtl, sigma per node or not) is its problem's; a CTA's tasks run
  // problem by problem, so the loads and the update each keep the control of the last problem
  // they met instead of re-deriving it per tile.
  int ib = -1;
  SweepCtl isc{};
  bool ihet = false;
  auto issue = [&](int j) {
    if (j < J) {
      const TileTask tk = task(j);  // by value: the cp.async statements clobber memory
      if (tk.b != ib) {
        ib = tk.b;
        isc = sweep_ctl(p, ph, ib);
        ihet = prob_at(p, ib).hetero != 0;
      }
      if (isc.active) {
        const int N = isc.N;
        const bool interior = tile_interior(N, tk.x0, tk.y0);
        HaloCells hc;
        Columns cl;
        if (interior) {
          hc = halo_cells_2d(s_prob0, N, tk.x0, tk.y0, true);  // the descriptor is not read
          cl = own_columns_2d(s_prob0, N, tk.x0, tk.y0, true);
        } else {
          const ProblemDesc& P = prob_at(p, tk.b);
          hc = halo_cells(P, N, tk.x0, tk.y0, false);
          cl = own_columns(P, N, tk.x0, tk.y0);
        }
        SweepStage<T>& S = st[j % D];
        const T* src = Esrc + isc.off;
#pragma unroll
        for (int s = 0; s < kCells; ++s)
          if (hc.off[s] >= 0) {
            if (!isc.zero_in) cp_async_t(&S.e[tid + s * kThreads], src + hc.off[s]);
            if (ihet) cp_async_t(&S.s[tid + s * kThreads], (const T*)p.SIG + isc.off + hc.off[s]);
          }
#pragma unroll
        for (int r = 0; r < 2; ++r)
          if (cl.in[r]) {
            cp_async_t(&S.r[tid + r * kThreads], (const T*)p.R + isc.off + cl.off[r]);
            if (ihet) cp_async_t(&S.q[tid + r * kThreads], (const T*)p.Q + isc.off + cl.off[r]);
            if (isc.last) cp_async_t(&S.u[tid + r * kThreads], p.U + prob_at(p, tk.b).off_full + cl.off[r]);
          }
      }
    }
    cp_async_commit();
  };
  int cb = -1;
  SweepCtl csc{};
  bool chet = false;
  SweepConst<T> kc{};
  for (int j = 0; j < D - 2; ++j) issue(j);
  for (int j = 0; j < J; ++j) {
    cp_async_wait<D - 3>();
    __syncthreads();
    issue(j + D - 2);
    const TileTask tk = task(j);
    if (tk.b != cb) {
      cb = tk.b;
      csc = sweep_ctl(p, ph, cb);
      const ProblemDesc& P = prob_at(p, cb);
      chet = P.hetero != 0;
      kc = sweep_const<T>(p, P, l);
    }
    if (!csc.active) continue;
    T dmx = (T)0;  // pseudo-residual times inv_c (DIAG)
    const int N = csc.N;
    const Columns cl = tile_interior(N, tk.x0, tk.y0) ? own_columns_2d(s_prob0, N, tk.x0, tk.y0, true)
                                                      : own_columns(prob_at(p, tk.b), N, tk.x0, tk.y0);
    const SweepStage<T>& S = st[j % D];
    PlaneSums<T> ps[2];
    if (chet) plane_sums2<T, true>(S, b0, csc.zero_in, ps);
    else plane_sums2<T, false>(S, b0, csc.zero_in, ps);
    T* dst = Edst + csc.off;
    const bool last = csc.last;
    const double inv_scale = last ? inv_scale_at(p, tk.b, c & 1) : 0.0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (!cl.in[r] || cl.fixed_xy[r]) continue;
      const T CSe = rn_fma(kc.w_e, ps[r].C, ps[r].F);
      const int slot = tid + r * kThreads, cc = b0 + (r + 1) * kHX + 1;
      const T e_new = chet ? sweep_update<T, true>(kc, S, slot, cc, CSe, rn_fma(kc.w_e, ps[r].sC, ps[r].sF), ps[r].v)
                           : sweep_update<T, false>(kc, S, slot, cc, CSe, (T)0, ps[r].v);
      if (DIAG) dmx = fmax(dmx, diag_term(e_new - ps[r].v, chet ? S.q[slot] : kc.q_const));
      if (last) p.U[prob_at(p, tk.b).off_full + cl.off[r]] = __fma_rn((double)e_new, inv_scale, S.u[slot]);
      if (!last || p.mixed) dst[cl.off[r]] = e_new;
    }
    if (DIAG) diag_flush<T>(p, tk.b, c, l, dmx, kc.inv_c);
  }
  cp_async_wait<0>();
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// Two consecutive Jacobi sweeps of a visit in one z-march (3-D, FP32 cycle).  The second sweep at
// a node needs the first sweep's result on its 3 x 3 x 3 neighbourhood, so the first sweep is
// evaluated on the tile widened by one cell on every side ((kTX + 2) x (kTY + 2) cells; the ring is
// evaluated by both neighbouring tiles with the same arithmetic) from inputs widened by two.  Its
// planes pass through one shared-memory plane buffer one plane behind the loads, and the second
// sweep runs one plane further behind, so each input plane crosses HBM once for both sweeps and the
// intermediate correction never leaves the SM.  The z sums of both sweeps are rolled: with
// t = v + w_e F + w_c C (a plane's part in the sums of the planes above and below) and
// m = F + w_e C (its part in its own), CS(e) at plane z is (m_z + t_{z-1}) + t_{z+1}.  Mirror
// images in x and y are loaded mirrored and the in-plane sums are symmetric, so a ring cell outside
// the domain holds exactly the first sweep at its mirror node.
// ---------------------------------------------------------------------------------------------
constexpr int kPX = kTX + 4, kPY = kTY + 4, kPHalo = kPX * kPY;   // inputs: the tile + 2 cells
constexpr int kPCells = (kPHalo + kThreads - 1) / kThreads;
constexpr int kEX = kTX + 2, kEY = kTY + 2, kERegion = kEX * kEY;  // first sweep: the tile + 1 cell
constexpr int kECells = (kERegion + kThreads - 1) / kThreads;
constexpr int kUnits = (kEY / 2) * kEX;  // first-sweep work units: two vertically adjacent cells
constexpr int kUnitSlots = (kUnits + kThreads - 1) / kThreads;
constexpr int kPairStages = 5;  // planes k - 2 .. k resident, loads two planes ahead
static_assert(kEY % 2 == 0, "two-cell units");

template <typename T>
struct PairStage {
  T e[kPHalo];             // correction e on the widened input tile
  T s[kPHalo];             // sigma on the same cells
  T r[kERegion];           // restricted residual on the first sweep's cells
  T q[kERegion];           // local step factor on the same cells
  double u[2 * kThreads];  // FP64 solution at the tile's nodes (last sweep of a cycle)
};

template <typename T>
constexpr size_t pair_smem_bytes() {
  return sizeof(PairStage<T>) * kPairStages + sizeof(T) * kERegion;
}

struct PairCells {
  int in_off[kPCells];  // y * N + x of the thread's input cells (images applied, clamped), -1: none
  int e_off[kECells];   // the same for the thread's first-sweep cells
};

__device__ __forceinline__ PairCells pair_cells(int N, int x0, int y0) {
  PairCells pc;
#pragma unroll
  for (int s = 0; s < kPCells; ++s) {
    const int k = threadIdx.x + s * kThreads;
    pc.in_off[s] = k < kPHalo ? refl_clamp(y0 - 2 + k / kPX, N) * N + refl_clamp(x0 - 2 + k % kPX, N) : -1;
  }
#pragma unroll
  for (int s = 0; s < kECells; ++s) {
    const int k = threadIdx.x + s * kThreads;
    pc.e_off[s] = k < kERegion ? refl_clamp(y0 - 1 + k / kEX, N) * N + refl_clamp(x0 - 1 + k % kEX, N) : -1;
  }
  return pc;
}

// The thread's first-sweep units: unit u = tid + j kThreads covers the cells (ex, 2 pu) and
// (ex, 2 pu + 1) of the widened tile, pu = u / kEX, ex = u % kEX.
struct PairUnits {
  int b1[kUnitSlots];    // top-left of the unit's 4 x 3 input block, -1: no unit
  int eidx[kUnitSlots];  // first-sweep index of the unit's upper cell
  unsigned fixed;        // bit 2 j + r: cell r of unit j mirrors onto a Dirichlet x / y face node
};

__device__ __forceinline__ PairUnits pair_units(const ProblemDesc& P, int N, int x0, int y0) {
  PairUnits pu;
  pu.fixed = 0u;
#pragma unroll
  for (int j = 0; j < kUnitSlots; ++j) {
    const int u = threadIdx.x + j * kThreads;
    pu.b1[j] = pu.eidx[j] = -1;
    if (u >= kUnits) continue;
    const int py = u / kEX, ex = u % kEX;
    pu.b1[j] = 2 * py * kPX + ex;
    pu.eidx[j] = 2 * py * kEX + ex;
    const int rx = refl_clamp(x0 - 1 + ex, N);
    const bool fx = (rx == 0 && P.face_type[0] == 0) || (rx == N - 1 && P.face_type[1] == 0);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int ry = refl_clamp(y0 - 1 + 2 * py + r, N);
      if (fx || (ry == 0 && P.face_type[2] == 0) || (ry == N - 1 && P.face_type[3] == 0)) pu.fixed |= 1u << (2 * j + r);
    }
  }
  return pu;
}

// In-plane sums of the two cells of a 4 x 3 block (pitch W) of e and sigma * e: v, F, C per cell
// and the same for sigma e, plus sigma at the two centres.
template <typename T, bool HET, int W>
__device__ __forceinline__ void block_sums(const T* e, int be, const T* sg, int bs, T v[2], T F[2], T C[2], T sv[2],
                                           T sF[2], T sC[2], T sc[2]) {
  T a[4][3], se[4][3];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      a[i][j] = e[be + i * W + j];
      if (HET) se[i][j] = rn_mul(sg[bs + i * kPX + j], a[i][j]);
    }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    v[r] = a[r + 1][1];
    F[r] = (a[r + 1][0] + a[r + 1][2]) + (a[r][1] + a[r + 2][1]);
    C[r] = (a[r][0] + a[r][2]) + (a[r + 2][0] + a[r + 2][2]);
    if (HET) {
      sv[r] = se[r + 1][1];
      sF[r] = (se[r + 1][0] + se[r + 1][2]) + (se[r][1] + se[r + 2][1]);
      sC[r] = (se[r][0] + se[r][2]) + (se[r + 2][0] + se[r + 2][2]);
      sc[r] = sg[bs + (r + 1) * kPX + 1];
    } else {
      sv[r] = sF[r] = sC[r] = sc[r] = (T)0;
    }
  }
}

template <typename T, bool HET, bool LAST>
__device__ void sweep3_pair(const KernelParams& p, const Phase& ph, int c, const TileTask& tk, PairStage<T>* st,
                            T* ebuf, const SweepCtl& sc) {
  constexpr int D = kPairStages;
  const ProblemDesc& P = prob_at(p, tk.b);
  const int N = sc.N;
  const int tid = threadIdx.x;
  const Columns cl = own_columns(P, N, tk.x0, tk.y0);
  const bool odd = sweep_parity(p, ph.level, ph.sweep) != 0;
  const T* src = odd ? (const T*)p.E2 + sc.off : (const T*)p.E + sc.off;
  T* dst = odd ? (T*)p.E + sc.off : (T*)p.E2 + sc.off;
  const T* R = (const T*)p.R + sc.off;
  const T* SG = HET ? (const T*)p.SIG + sc.off : nullptr;
  const T* Q = HET ? (const T*)p.Q + sc.off : nullptr;
  double* Ug = p.U + P.off_full;
  const PairCells pc = pair_cells(N, tk.x0, tk.y0);
  const PairUnits pu = pair_units(P, N, tk.x0, tk.y0);
  const SweepConst<T> kc = sweep_const<T>(p, P, ph.level);
  const double inv_scale = LAST ? inv_scale_at(p, tk.b, c & 1) : 0.0;
  const bool zero_in = sc.zero_in;
  const int nplanes = tk.nz + 4;
  const unsigned NN = (unsigned)N * (unsigned)N;
  // second sweep: the thread's two tile nodes (tx, ty2 + r)
  const int tx = tid % kTX, ty2 = 2 * (tid / kTX);
  const int b2 = ty2 * kEX + tx;             // their 4 x 3 block in the plane buffer
  const int b2s = (ty2 + 1) * kPX + tx + 1;  // the same cells in the input tile (sigma)
  const int e2 = (ty2 + 1) * kEX + tx + 1;   // first-sweep index of the upper node (r, q)
  auto issue = [&](int k) {
    if (k < nplanes) {
      PairStage<T>& S = st[k % D];
      const unsigned base = (unsigned)refl(tk.z0 - 2 + k, N) * NN;
#pragma unroll
      for (int q = 0; q < kPCells; ++q)
        if (pc.in_off[q] >= 0) {
          const unsigned o = base + (unsigned)pc.in_off[q];
          if (zero_in) S.e[tid + q * kThreads] = (T)0;
          else cp_async_t(&S.e[tid + q * kThreads], src + o);
          if (HET) cp_async_t(&S.s[tid + q * kThreads], SG + o);
        }
      if (k >= 1 && k <= tk.nz + 2) {  // planes the first sweep evaluates
#pragma unroll
        for (int q = 0; q < kECells; ++q)
          if (pc.e_off[q] >= 0) {
            const unsigned o = base + (unsigned)pc.e_off[q];
            cp_async_t(&S.r[tid + q * kThreads], R + o);
            if (HET) cp_async_t(&S.q[tid + q * kThreads], Q + o);
          }
      }
      if (LAST && k >= 2 && k <= tk.nz + 1) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
          if (cl.in[r]) cp_async_t(&S.u[tid + r * kThreads], Ug + base + (unsigned)cl.off[r]);
      }
    }
    cp_async_commit();
  };
  for (int k = 0; k < D - 3; ++k) issue(k);
  // rolled z sums: first sweep per unit and cell, second sweep per tile node
  T S1e[kUnitSlots][2], T1e[kUnitSlots][2], S1s[kUnitSlots][2], T1s[kUnitSlots][2], v1[kUnitSlots][2], s1[kUnitSlots][2];
  T S2e[2], T2e[2], S2s[2], T2s[2], v2[2], s2[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
#pragma unroll
    for (int j = 0; j < kUnitSlots; ++j) S1e[j][r] = T1e[j][r] = S1s[j][r] = T1s[j][r] = v1[j][r] = s1[j][r] = (T)0;
    S2e[r] = T2e[r] = S2s[r] = T2s[r] = v2[r] = s2[r] = (T)0;
  }
  for (int k = 0; k < nplanes; ++k) {
    cp_async_wait<D - 4>();
    __syncthreads();
    issue(k + D - 3);
    const PairStage<T>& S0 = st[k % D];            // input plane k (z0 - 2 + k)
    const PairStage<T>& S1 = st[(k + D - 1) % D];  // input plane k - 1
    // first sweep: sums of plane k; completes the first sweep at plane k - 1
    const bool zf1 = z_fixed(cl, tk.z0 - 3 + k, N);
#pragma unroll
    for (int j = 0; j < kUnitSlots; ++j) {
      if (pu.b1[j] < 0) continue;
      T v[2], F[2], C[2], sv[2], sF[2], sC[2], sgc[2];
      block_sums<T, HET, kPX>(S0.e, pu.b1[j], S0.s, pu.b1[j], v, F, C, sv, sF, sC, sgc);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const T t = rn_fma(kc.w_c, C[r], rn_fma(kc.w_e, F[r], v[r]));
        const T m = rn_fma(kc.w_e, C[r], F[r]);
        const T ts = HET ? rn_fma(kc.w_c, sC[r], rn_fma(kc.w_e, sF[r], sv[r])) : (T)0;
        const T ms = HET ? rn_fma(kc.w_e, sC[r], sF[r]) : (T)0;
        if (k >= 2) {
          const int ei = pu.eidx[j] + r * kEX;
          const T CSe = rn_add(S1e[j][r], t);
          T en;
          if (zf1 || ((pu.fixed >> (2 * j + r)) & 1u)) {
            en = v1[j][r];
          } else if (HET) {
            const T CSse = rn_add(S1s[j][r], ts);
            en = rn_fma(S1.q[ei], rn_fma(-S1.r[ei], kc.inv_c, rn_fma(s1[j][r], CSe, CSse)),
                        rn_mul(kc.one_m_omega, v1[j][r]));
          } else {
            en = rn_fma(kc.q_const, rn_fma(-S1.r[ei], kc.inv_c, rn_mul((T)2, CSe)), rn_mul(kc.one_m_omega, v1[j][r]));
          }
          ebuf[ei] = en;
        }
        S1e[j][r] = rn_add(m, T1e[j][r]);
        T1e[j][r] = t;
        if (HET) {
          S1s[j][r] = rn_add(ms, T1s[j][r]);
          T1s[j][r] = ts;
        }
        v1[j][r] = v[r];
        s1[j][r] = sgc[r];
      }
    }
    __syncthreads();  // the plane buffer holds the first sweep at plane k - 1
    if (k >= 2) {
      // second sweep: sums of the buffer around the tile nodes; completes plane k - 2
      T v[2], F[2], C[2], sv[2], sF[2], sC[2], sgc[2];
      block_sums<T, HET, kEX>(ebuf, b2, S1.s, b2s, v, F, C, sv, sF, sC, sgc);
      const int z2 = tk.z0 - 4 + k;
      const bool zf2 = k < 4 || z_fixed(cl, z2, N);
      const PairStage<T>& S2 = st[(k + D - 2) % D];  // input plane k - 2 (= z2)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const T t = rn_fma(kc.w_c, C[r], rn_fma(kc.w_e, F[r], v[r]));
        const T m = rn_fma(kc.w_e, C[r], F[r]);
        const T ts = HET ? rn_fma(kc.w_c, sC[r], rn_fma(kc.w_e, sF[r], sv[r])) : (T)0;
        const T ms = HET ? rn_fma(kc.w_e, sC[r], sF[r]) : (T)0;
        if (!zf2 && cl.in[r] && !cl.fixed_xy[r]) {
          const int ei = e2 + r * kEX;
          const T CSe = rn_add(S2e[r], t);
          T en;
          if (HET) {
            const T CSse = rn_add(S2s[r], ts);
            en = rn_fma(S2.q[ei], rn_fma(-S2.r[ei], kc.inv_c, rn_fma(s2[r], CSe, CSse)), rn_mul(kc.one_m_omega, v2[r]));
          } else {
            en = rn_fma(kc.q_const, rn_fma(-S2.r[ei], kc.inv_c, rn_mul((T)2, CSe)), rn_mul(kc.one_m_omega, v2[r]));
          }
          const unsigned idx = (unsigned)z2 * NN + (unsigned)cl.off[r];
          if (LAST) Ug[idx] = __fma_rn((double)en, inv_scale, S2.u[tid + r * kThreads]);
          dst[idx] = en;
        }
        S2e[r] = rn_add(m, T2e[r]);
        T2e[r] = t;
        if (HET) {
          S2s[r] = rn_add(ms, T2s[r]);
          T2s[r] = ts;
        }
        v2[r] = v[r];
        s2[r] = sgc[r];
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// Level-0 sweep with four rows per thread (3-D, FP32 cycle): tiles of kTX x kTY4 columns
// (64 x 16 or 32 x 32) from a partition of their own.  Each thread forms the in-plane sums of four
// vertically adjacent nodes from one 6 x 3 block of shared memory (4.5 loads per node and array
// instead of 6), and the z sums are rolled: with t = v + w_e F + w_c C (a plane's part in the sums
// of the planes above and below) and m = F + w_e C (its part in its own), CS(e) at plane z is
// (m_z + t_{z-1}) + t_{z+1}, two registers per node and array.  The per-plane pipeline overhead
// is spread over twice the nodes of the two-row sweep, and the wider halo tile costs 16 % instead
// of 29 %.
// ---------------------------------------------------------------------------------------------
constexpr int kTY4 = 4 * kThreads / kTX, kHY4 = kTY4 + 2, kHalo4 = kHX * kHY4;
constexpr int kCells4 = (kHalo4 + kThreads - 1) / kThreads;

template <typename T>
struct QuadStage {
  T e[kHalo4];
  T s[kHalo4];
  T r[4 * kThreads];
  T q[4 * kThreads];
};  // (the last sweep's FP64 solution is prefetched into registers one plane ahead)

template <typename T>
constexpr size_t quad_smem_bytes() {
  return sizeof(QuadStage<T>) * kSweepStages;
}

struct Columns4 {
  int off[4];
  bool in[4];
  bool fixed_xy[4];
  bool dz0, dz1;
};

__device__ __forceinline__ Columns4 own_columns4(const ProblemDesc& P, int N, int x0, int y0) {
  Columns4 cl;
  const int x = x0 + (int)(threadIdx.x % kTX);
  const bool fx = (x == 0 && P.face_type[0] == 0) || (x == N - 1 && P.face_type[1] == 0);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int y = y0 + 4 * (int)(threadIdx.x / kTX) + r;
    cl.in[r] = x < N && y < N;
    cl.off[r] = y * N + x;
    cl.fixed_xy[r] = fx || (y == 0 && P.face_type[2] == 0) || (y == N - 1 && P.face_type[3] == 0);
  }
  cl.dz0 = P.face_type[4] == 0;
  cl.dz1 = P.face_type[5] == 0;
  return cl;
}

__device__ __forceinline__ void halo_cells4(int N, int x0, int y0, int off[kCells4]) {
#pragma unroll
  for (int s = 0; s < kCells4; ++s) {
    const int k = threadIdx.x + s * kThreads;
    off[s] = k < kHalo4 ? refl_clamp(y0 - 1 + k / kHX, N) * N + refl_clamp(x0 - 1 + k % kHX, N) : -1;
  }
}

template <class Body>
__device__ __forceinline__ void for_tasks4(const KernelParams& p, int l, Body&& body) {
  const int* o = p.task_off4 + (long long)l * (gridDim.x + 1) + blockIdx.x;
  const int t0 = o[0], t1 = o[1];
  for (int t = t0; t < t1; ++t) body(p.tasks4[t]);
}

template <typename T, bool HET, bool LAST>
__device__ void sweep3q(const KernelParams& p, const Phase& ph, int c, const TileTask& tk, QuadStage<T>* st,
                        const SweepCtl& sc) {
  constexpr int D = kSweepStages;
  const ProblemDesc& P = prob_at(p, tk.b);
  const int N = sc.N;
  const int tid = threadIdx.x;
  const Columns4 cl = own_columns4(P, N, tk.x0, tk.y0);
  const bool odd = sweep_parity(p, ph.level, ph.sweep) != 0;
  const T* src = odd ? (const T*)p.E2 + sc.off : (const T*)p.E + sc.off;
  T* dst = odd ? (T*)p.E + sc.off : (T*)p.E2 + sc.off;
  const T* R = (const T*)p.R + sc.off;
  const T* SG = HET ? (const T*)p.SIG + sc.off : nullptr;
  const T* Q = HET ? (const T*)p.Q + sc.off : nullptr;
  double* Ug = p.U + P.off_full;
  int hoff[kCells4];
  halo_cells4(N, tk.x0, tk.y0, hoff);
  const SweepConst<T> kc = sweep_const<T>(p, P, ph.level);
  const int b0 = (4 * (tid / kTX)) * kHX + (tid % kTX);  // top-left of the thread's 6 x 3 block
  const double inv_scale = LAST ? inv_scale_at(p, tk.b, c & 1) : 0.0;
  const bool keep = !LAST || p.mixed;
  const bool zero_in = sc.zero_in;
  const int nplanes = tk.nz + 2;
  const unsigned NN = (unsigned)N * (unsigned)N;
  auto issue = [&](int k) {
    if (k < nplanes) {
      QuadStage<T>& S = st[k % D];
      const unsigned base = (unsigned)refl(tk.z0 - 1 + k, N) * NN;
#pragma unroll
      for (int s = 0; s < kCells4; ++s)
        if (hoff[s] >= 0) {
          const unsigned o = base + (unsigned)hoff[s];
          if (!zero_in) cp_async_t(&S.e[tid + s * kThreads], src + o);
          if (HET) cp_async_t(&S.s[tid + s * kThreads], SG + o);
        }
      if (k >= 1 && k <= tk.nz) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (cl.in[r]) {
            const unsigned o = base + (unsigned)cl.off[r];
            cp_async_t(&S.r[tid + r * kThreads], R + o);
            if (HET) cp_async_t(&S.q[tid + r * kThreads], Q + o);
          }
      }
    }
    cp_async_commit();
  };
  for (int k = 0; k < D - 2; ++k) issue(k);
  // rolled z sums of the thread's four nodes, and their e and sigma one plane behind
  T Se[4], Te[4], Ss[4], Ts[4], vp[4], sp[4];
  double u_old[4], u_new[4];  // last sweep: FP64 solution of the planes being updated / arriving
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    Se[r] = Te[r] = Ss[r] = Ts[r] = vp[r] = sp[r] = (T)0;
    u_old[r] = u_new[r] = 0.0;
  }
  for (int k = 0; k < nplanes; ++k) {
    cp_async_wait<D - 3>();
    __syncthreads();
    issue(k + D - 2);
    if (LAST && k >= 1 && k <= tk.nz) {  // solution of plane k, used when it is updated next step
      const unsigned zo = (unsigned)(tk.z0 - 1 + k) * NN;
#pragma unroll
      for (int r = 0; r < 4; ++r) u_new[r] = cl.in[r] ? Ug[zo + (unsigned)cl.off[r]] : 0.0;
    }
    const QuadStage<T>& S = st[k % D];
    T t[4], m[4], ts[4], ms[4], v[4], sv[4];
    if (zero_in) {
#pragma unroll
      for (int r = 0; r < 4; ++r) t[r] = m[r] = ts[r] = ms[r] = v[r] = (T)0;
#pragma unroll
      for (int r = 0; r < 4; ++r) sv[r] = HET ? S.s[b0 + (r + 1) * kHX + 1] : (T)0;
    } else {
      T a[6][3], se[6][3];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          a[i][j] = S.e[b0 + i * kHX + j];
          if (HET) se[i][j] = rn_mul(S.s[b0 + i * kHX + j], a[i][j]);
        }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const T F = (a[r + 1][0] + a[r + 1][2]) + (a[r][1] + a[r + 2][1]);
        const T C = (a[r][0] + a[r][2]) + (a[r + 2][0] + a[r + 2][2]);
        v[r] = a[r + 1][1];
        t[r] = rn_fma(kc.w_c, C, rn_fma(kc.w_e, F, v[r]));
        m[r] = rn_fma(kc.w_e, C, F);
        if (HET) {
          const T sF = (se[r + 1][0] + se[r + 1][2]) + (se[r][1] + se[r + 2][1]);
          const T sC = (se[r][0] + se[r][2]) + (se[r + 2][0] + se[r + 2][2]);
          ts[r] = rn_fma(kc.w_c, sC, rn_fma(kc.w_e, sF, se[r + 1][1]));
          ms[r] = rn_fma(kc.w_e, sC, sF);
          sv[r] = S.s[b0 + (r + 1) * kHX + 1];
        } else {
          ts[r] = ms[r] = sv[r] = (T)0;
        }
      }
    }
    if (k >= 2) {
      const int z = tk.z0 + k - 2;
      const bool zf = z_fixed(cl.dz0, cl.dz1, z, N);
      const QuadStage<T>& S1 = st[(k - 1) % D];
      const unsigned zoff = (unsigned)z * NN;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (!cl.in[r] || cl.fixed_xy[r] || zf) continue;
        const int slot = tid + r * kThreads;
        const T CSe = rn_add(Se[r], t[r]);
        const T r_i = S1.r[slot];
        T e_new;
        if (HET) {
          const T CSse = rn_add(Ss[r], ts[r]);
          e_new = rn_fma(S1.q[slot], rn_fma(-r_i, kc.inv_c, rn_fma(sp[r], CSe, CSse)), rn_mul(kc.one_m_omega, vp[r]));
        } else {
          e_new = rn_fma(kc.q_const, rn_fma(-r_i, kc.inv_c, rn_mul((T)2, CSe)), rn_mul(kc.one_m_omega, vp[r]));
        }
        const unsigned idx = zoff + (unsigned)cl.off[r];
        if (LAST) Ug[idx] = __fma_rn((double)e_new, inv_scale, u_old[r]);
        if (keep) dst[idx] = e_new;
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (LAST) u_old[r] = u_new[r];
      Se[r] = rn_add(m[r], Te[r]);
      Te[r] = t[r];
      if (HET) {
        Ss[r] = rn_add(ms[r], Ts[r]);
        Ts[r] = ts[r];
      }
      vp[r] = v[r];
      sp[r] = sv[r];
    }
  }
  cp_async_wait<0>();
  __syncthreads();
}

// Dynamic shared memory of the cycle kernel: the largest phase (fused pairs and four-row sweeps:
// FP32 only).
template <typename T>
constexpr size_t phase_smem_bytes() {
  constexpr size_t a = sweep_smem_bytes<T>() > outer_smem_bytes() ? sweep_smem_bytes<T>() : outer_smem_bytes();
  constexpr size_t b = a > prolong_smem_bytes<T>() ? a : prolong_smem_bytes<T>() + 64;
  constexpr size_t c = (sizeof(T) == 4 && pair_smem_bytes<T>() > b) ? pair_smem_bytes<T>() : b;
  return (sizeof(T) == 4 && quad_smem_bytes<T>() > c) ? quad_smem_bytes<T>() : c;
}

template <typename T, int DIM>
__device__ void phase_sweep(const KernelParams& p, const Phase& ph, int c, unsigned char* smem) {
  SweepStage<T>* st = (SweepStage<T>*)smem;
  if (DIM == 2) {
    if (p.diag) sweep2<T, true>(p, ph, c, st);
    else sweep2<T>(p, ph, c, st);
    return;
  }
  if constexpr (sizeof(T) == 4) {
    if (!(ph.flags & kPair) && ph.level < p.quad_levels && !p.diag) {
      QuadStage<T>* qst = (QuadStage<T>*)smem;
      for_tasks4(p, ph.level, [&](const TileTask& tk) {
        const SweepCtl sc = sweep_ctl(p, ph, tk.b);
        if (!sc.active) return;
        const bool het = prob_at(p, tk.b).hetero != 0;
        if (sc.last) {
          if (het) sweep3q<T, true, true>(p, ph, c, tk, qst, sc);
          else sweep3q<T, false, true>(p, ph, c, tk, qst, sc);
        } else {
          if (het) sweep3q<T, true, false>(p, ph, c, tk, qst, sc);
          else sweep3q<T, false, false>(p, ph, c, tk, qst, sc);
        }
      });
      return;
    }
  }
  for_tasks(p, ph.level, [&](const TileTask& tk) {
    const SweepCtl sc = sweep_ctl(p, ph, tk.b);
    if (!sc.active) return;
    const bool het = prob_at(p, tk.b).hetero != 0;
    if constexpr (sizeof(T) == 4) {
      if (ph.flags & kPair) {
        PairStage<T>* pst = (PairStage<T>*)smem;
        T* ebuf = (T*)(smem + sizeof(PairStage<T>) * kPairStages);
        if (sc.last) {
          if (het) sweep3_pair<T, true, true>(p, ph, c, tk, pst, ebuf, sc);
          else sweep3_pair<T, false, true>(p, ph, c, tk, pst, ebuf, sc);
        } else {
          if (het) sweep3_pair<T, true, false>(p, ph, c, tk, pst, ebuf, sc);
          else sweep3_pair<T, false, false>(p, ph, c, tk, pst, ebuf, sc);
        }
        return;
      }
    }
    if constexpr (sizeof(T) == 8) {
      if (!p.diag) {  // the FP64 form's sweep with fewer FP64 instructions per node
        if (sc.last) {
          if (het) sweep3_f64<true, true>(p, ph, c, tk, st, sc);
          else sweep3_f64<false, true>(p, ph, c, tk, st, sc);
        } else {
          if (het) sweep3_f64<true, false>(p, ph, c, tk, st, sc);
          else sweep3_f64<false, false>(p, ph, c, tk, st, sc);
        }
        return;
      }
    }
    if (p.diag) {
      if (sc.last) {
        if (het) sweep3<T, true, true, true>(p, ph, c, tk, st, sc);
        else sweep3<T, false, true, true>(p, ph, c, tk, st, sc);
      } else {
        if (het) sweep3<T, true, false, true>(p, ph, c, tk, st, sc);
        else sweep3<T, false, false, true>(p, ph, c, tk, st, sc);
      }
      return;
    }
    if (sc.last) {
      if (het) sweep3<T, true, true>(p, ph, c, tk, st, sc);
      else sweep3<T, false, true>(p, ph, c, tk, st, sc);
    } else {
      if (het) sweep3<T, true, false>(p, ph, c, tk, st, sc);
      else sweep3<T, false, false>(p, ph, c, tk, st, sc);
    }
  });
}

// ---------------------------------------------------------------------------------------------
// Row phases: restriction, interpolation to the next finer level, injection to the next coarser.
// ---------------------------------------------------------------------------------------------

// One line of the restriction stencil, 1/4 f(x - 1) + 1/2 f(x) + 1/4 f(x + 1), explicitly rounded so
// that its value never depends on how the compiler contracts the expression.
template <typename T>
__device__ __forceinline__ T restrict_line(T a, T b, T c) {
  return rn_fma((T)0.25, c, rn_fma((T)0.5, b, rn_mul((T)0.25, a)));
}

// Row phases issue the loads of several x positions per lane before storing (a row of a large level
// would otherwise take one load round trip per 32 nodes).
constexpr int kRestrictBatch = 2, kInjectBatch = 4;

// Restriction pass: level l-1 -> level l (Eqs. 3-4 at distance 2^(l-1) h), even images.
template <typename T, int DIM>
__device__ void phase_restrict(const KernelParams& p, int l) {
  T* R = (T*)p.R;
  const int lane = threadIdx.x & 31;
  for_rows<DIM>(p, l, [&](int b, const ProblemDesc& P, int N, int y, int z) {
    if (l > P.n - 1 || done_at(p, b)) return;
    const int Ns = level_side(P.n, l - 1);
    const T* src = R + P.off_lvl[l - 1];
    T* dst = R + P.off_lvl[l] + ((long long)z * N + y) * N;
    long long rows[3][3];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
        rows[dz][dy] = ((long long)(DIM == 3 ? refl(2 * z + dz - 1, Ns) : 0) * Ns + refl(2 * y + dy - 1, Ns)) * Ns;
    // kRestrictBatch x positions per lane are formed before any is stored (source and destination
    // share one array, so the compiler would not move the next position's loads above a store)
    for (int xb = lane; xb < N; xb += 32 * kRestrictBatch) {
      T acc[kRestrictBatch];
#pragma unroll
      for (int u = 0; u < kRestrictBatch; ++u) {
        const int x = xb + 32 * u;
        acc[u] = (T)0;
        if (x >= N) continue;
        const int xm = refl(2 * x - 1, Ns), x0 = 2 * x, xp = refl(2 * x + 1, Ns);
#pragma unroll
        for (int dz = 0; dz < (DIM == 3 ? 3 : 1); ++dz) {
          T accz = (T)0;
#pragma unroll
          for (int dy = 0; dy < 3; ++dy) {
            const T* row = src + rows[DIM == 3 ? dz : 0][dy];
            accz = rn_fma(dy == 1 ? (T)0.5 : (T)0.25, restrict_line(row[xm], row[x0], row[xp]), accz);
          }
          acc[u] = DIM == 3 ? rn_fma(dz == 1 ? (T)0.5 : (T)0.25, accz, acc[u]) : rn_add(acc[u], accz);
        }
      }
#pragma unroll
      for (int u = 0; u < kRestrictBatch; ++u)
        if (xb + 32 * u < N) dst[xb + 32 * u] = acc[u];
    }
  });
}

// The same restriction for a 3-D level l as a z-march over the level-l tiles of the work partition:
// the level-(l-1) planes 2z - 1, 2z, 2z + 1 of the tile's footprint ((2 kTX + 1) x (2 kTY + 1) cells,
// images applied) are staged in shared memory once per tile -- an odd plane serves two level-l planes
// -- and every node forms its in-plane 3 x 3 sums from shared memory, in the operation order of
// phase_restrict (bit-identical results).  A row phase re-reads the shared rows and planes of the
// finer level through L2 (2.25x); here each footprint cell is fetched once per tile.  Nodes of tiles
// the partition leaves out (all on a Dirichlet face) are not written: their values reach only
// Dirichlet nodes of the coarser levels, which no stencil reads.
constexpr int kRX = 2 * kTX + 1, kRY = 2 * kTY + 1, kRCells = kRX * kRY;
constexpr int kRSlots = (kRCells + kThreads - 1) / kThreads;
constexpr int kRestrictStages = 4;  // loads issued two fine planes ahead

template <typename T>
struct RestrictStage {
  T v[kRSlots * kThreads];  // one fine plane of the footprint, row-major (row = kRX cells)
};
static_assert(sizeof(RestrictStage<float>) * kRestrictStages <= phase_smem_bytes<float>(), "shared memory");
static_assert(sizeof(RestrictStage<double>) * kRestrictStages <= phase_smem_bytes<double>(), "shared memory");

// Kept out of line with plain arguments, so that its registers do not enter the allocation of the
// persistent kernel's other phases.
template <typename T>
__device__ __noinline__ void restrict3(const T* __restrict__ src, T* __restrict__ dst, int N, int x0, int y0, int z0,
                                       int nz, RestrictStage<T>* st) {
  constexpr int D = kRestrictStages;
  const int Ns = 2 * N - 1;
  const long long NNs = (long long)Ns * Ns, NN = (long long)N * N;
  const int tid = threadIdx.x, tx = tid % kTX, ty = tid / kTX;
  const int X0 = 2 * x0 - 1, Y0 = 2 * y0 - 1;
  const int nfine = 2 * nz + 1;  // fine planes 2 z0 - 1 .. 2 (z0 + nz - 1) + 1
  // footprint cell c of the thread: fine (X, Y) = (X0 + c % kRX, Y0 + c / kRX), images applied;
  // cells past the image of the far edge serve no node of the level and are not fetched (-1)
  int coff[kRSlots];
#pragma unroll
  for (int s = 0; s < kRSlots; ++s) {
    const int c = tid + s * kThreads;
    const int X = X0 + c % kRX, Y = Y0 + c / kRX;
    coff[s] = (c < kRCells && X <= Ns && Y <= Ns) ? refl(Y, Ns) * Ns + refl(X, Ns) : -1;
  }
  auto issue = [&](int k) {
    if (k < nfine) {
      const T* plane = src + (long long)refl(2 * z0 - 1 + k, Ns) * NNs;
      T* v = st[k % D].v;
#pragma unroll
      for (int s = 0; s < kRSlots; ++s)
        if (coff[s] >= 0) cp_async_t(&v[tid + s * kThreads], plane + coff[s]);
    }
    cp_async_commit();
  };
  const int x = x0 + tx;
  bool in[2];
  int off[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int y = y0 + 2 * ty + r;
    in[r] = x < N && y < N;
    off[r] = y * N + x;
  }
  for (int k = 0; k < D - 2; ++k) issue(k);
  T acc[2] = {(T)0, (T)0};
  for (int k = 0; k < nfine; ++k) {
    cp_async_wait<D - 3>();
    __syncthreads();
    issue(k + D - 2);
    const T* v = st[k % D].v;
    T q[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      T accz = (T)0;
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        const T* row = v + (2 * (2 * ty + r) + dy) * kRX + 2 * tx;
        accz = rn_fma(dy == 1 ? (T)0.5 : (T)0.25, restrict_line(row[0], row[1], row[2]), accz);
      }
      q[r] = accz;
    }
    // fine plane k is plane dz = k - 2 j of the level-l plane z0 + j
    if (k & 1) {
#pragma unroll
      for (int r = 0; r < 2; ++r) acc[r] = rn_fma((T)0.5, q[r], acc[r]);
    } else {
      if (k >= 2) {
        const long long zoff = (long long)(z0 + k / 2 - 1) * NN;
#pragma unroll
        for (int r = 0; r < 2; ++r)
          if (in[r]) dst[zoff + off[r]] = rn_fma((T)0.25, q[r], acc[r]);
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) acc[r] = rn_fma((T)0.25, q[r], (T)0);
    }
  }
  cp_async_wait<0>();
  __syncthreads();
}

// Restriction passes of 3-D problems into levels 1 .. kTiledRestrictLevels run as tile z-marches;
// coarser levels (a few thousand nodes or fewer per problem) keep the row phase.
#ifndef SGML_TILED_RESTRICT_LEVELS
#define SGML_TILED_RESTRICT_LEVELS 2
#endif
constexpr int kTiledRestrictLevels = SGML_TILED_RESTRICT_LEVELS;

template <typename T, int DIM>
__device__ void phase_restrict_any(const KernelParams& p, int l, unsigned char* smem) {
  if (DIM == 3 && l <= kTiledRestrictLevels) {
    for_tasks(p, l, [&](const TileTask& tk) {
      if (done_at(p, tk.b)) return;
      const ProblemDesc& P = prob_at(p, tk.b);
      restrict3<T>((const T*)p.R + P.off_lvl[l - 1], (T*)p.R + P.off_lvl[l], level_side(P.n, l), tk.x0, tk.y0,
                   tk.z0, tk.nz, (RestrictStage<T>*)smem);
    });
    return;
  }
  phase_restrict<T, DIM>(p, l);
}

// Buffer holding the result of a visit of tooth `tooth` at a level (E if the visit flipped the
// ping-pong buffers an even number of times, E2 otherwise).
template <typename T>
__device__ __forceinline__ T* visit_result(const KernelParams& p, const ProblemDesc& P, int tooth, int l) {
  const int k = visit_sweeps(p.n_r, P.n, tooth, false);
  return ((visit_flips(p, l, k) & 1) ? (T*)p.E2 : (T*)p.E) + P.off_lvl[l];
}

// Moving one level finer: E_l (+)= I(E_{l+1} - B_{l+1}) on every level-l node (hat-function
// interpolation between consecutive levels, Algorithm 2's I_lambda).  3-D: tiles march over coarse
// planes; each stage holds one coarse plane of the tile's footprint (17 x 9 coarse nodes, the
// change formed once per coarse node) and the previous values of the two fine planes it completes
// (2 cz - 1 from coarse planes cz - 1 and cz, 2 cz from cz alone).
constexpr int kCX = kTX / 2 + 1, kCY = kTY / 2 + 1, kCoarse = kCX * kCY;
static_assert(kCoarse <= kThreads, "one coarse cell per thread");

template <typename T>
struct ProlongStage {
  T d[kCoarse];            // coarse values, then the change (value - B)
  T b[kCoarse];            // B at the coarse nodes
  T base[2][2 * kThreads];  // previous fine values of planes 2 cz - 1 and 2 cz at the tile's nodes
};

static_assert(sizeof(ProlongStage<float>) * prolong_stages<float>() <= phase_smem_bytes<float>(), "shared memory");
static_assert(sizeof(ProlongStage<double>) * prolong_stages<double>() <= phase_smem_bytes<double>(), "shared memory");

// (a + b) / 2, explicitly rounded.
template <typename T>
__device__ __forceinline__ T half_sum(T a, T b) {
  return rn_mul((T)0.5, rn_add(a, b));
}

template <typename T>
__device__ void prolong3(const KernelParams& p, const Phase& ph, const TileTask& tk, ProlongStage<T>* st) {
  constexpr int D = prolong_stages<T>();
  const int l = ph.level;
  const bool init = (ph.flags & kInit) != 0;
  const ProblemDesc& P = prob_at(p, tk.b);
  const int N = level_side(P.n, l), Nc = level_side(P.n, l + 1);
  const long long NN = (long long)N * N, NNc = (long long)Nc * Nc;
  const T* src = visit_result<T>(p, P, ph.tooth, l + 1);
  const T* Bc = (const T*)p.B + P.off_lvl[l + 1];
  const T* base = init ? nullptr : visit_result<T>(p, P, ph.prev_tooth, l);
  T* El = (T*)p.E + P.off_lvl[l];
  const int tid = threadIdx.x, tx = tid % kTX, ty = tid / kTX;
  const Columns cl = own_columns(P, N, tk.x0, tk.y0);
  const int cx0 = tk.x0 >> 1, cy0 = tk.y0 >> 1;
  // coarse footprint cells this thread loads (at most one: kCoarse <= kThreads); cells past the
  // level's far edge (a tile overhanging a small level) are read by no node and not loaded
  const int cell_x = tid % kCX, cell_y = tid / kCX;
  const bool has_cell = tid < kCoarse && cx0 + cell_x <= Nc - 1 && cy0 + cell_y <= Nc - 1;
  const int coff = min(cy0 + cell_y, Nc - 1) * Nc + min(cx0 + cell_x, Nc - 1);
  // interpolation weights of the thread's column (x) and its two rows (y even, y odd)
  const int x = tk.x0 + tx;
  const int lx0 = tx >> 1, lx1 = lx0 + (x & 1);
  const int zc_first = tk.z0 >> 1;                       // coarse plane of the first fine plane
  const int zc_last = (tk.z0 + tk.nz - 1 + 1) >> 1;      // coarse plane of the last fine plane's upper corner
  const int nplanes = zc_last - zc_first + 1;
  auto fine_in = [&](int z) { return z >= tk.z0 && z < tk.z0 + tk.nz; };
  auto issue = [&](int k) {
    if (k < nplanes) {
      ProlongStage<T>& S = st[k % D];
      const int cz = zc_first + k;
      if (has_cell) {
        cp_async_t(&S.d[tid], src + cz * NNc + coff);
        if (!init) cp_async_t(&S.b[tid], Bc + cz * NNc + coff);
      }
      if (!init) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int z = 2 * cz - 1 + j;
          if (fine_in(z)) {
#pragma unroll
            for (int r = 0; r < 2; ++r)
              if (cl.in[r]) cp_async_t(&S.base[j][tid + r * kThreads], base + z * NN + cl.off[r]);
          }
        }
      }
    }
    cp_async_commit();
  };
  // interpolated change at the thread's two nodes from one coarse plane (the change of a coarse node,
  // value - B, is formed by every thread that reads it: no barrier between forming and reading)
  auto delta = [&](const ProlongStage<T>& S, int i) { return init ? S.d[i] : rn_add(S.d[i], -S.b[i]); };
  auto plane_val = [&](const ProlongStage<T>& S, T out[2]) {
    const T a0 = delta(S, ty * kCX + lx0), a1 = delta(S, ty * kCX + lx1);
    const T b0 = delta(S, (ty + 1) * kCX + lx0), b1 = delta(S, (ty + 1) * kCX + lx1);
    const T ra = (x & 1) ? half_sum(a0, a1) : a0;
    const T rb = (x & 1) ? half_sum(b0, b1) : b0;
    out[0] = ra;                // y even: the coarse row itself
    out[1] = half_sum(ra, rb);  // y odd: halfway between two coarse rows
  };
  for (int k = 0; k < D - 2; ++k) issue(k);
  T prev[2] = {(T)0, (T)0};
  for (int k = 0; k < nplanes; ++k) {
    cp_async_wait<D - 3>();
    __syncthreads();
    issue(k + D - 2);
    const ProlongStage<T>& S = st[k % D];
    T cur[2];
    plane_val(S, cur);
    const int cz = zc_first + k;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int z = 2 * cz - 1 + j;  // odd fine plane (between cz - 1 and cz), then the even one (at cz)
      if (!fine_in(z) || (j == 0 && k == 0)) continue;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (!cl.in[r]) continue;
        const T v = j == 0 ? half_sum(prev[r], cur[r]) : cur[r];
        const T b = init ? (T)0 : S.base[j][tid + r * kThreads];
        El[z * NN + cl.off[r]] = rn_add(b, v);
      }
    }
    prev[0] = cur[0];
    prev[1] = cur[1];
  }
  cp_async_wait<0>();
  __syncthreads();
}

template <typename T, int DIM>
__device__ void phase_prolong_rows(const KernelParams& p, const Phase& ph) {
  const int l = ph.level;
  const bool init = (ph.flags & kInit) != 0;
  const int lane = threadIdx.x & 31;
  for_rows<DIM>(p, l, [&](int b, const ProblemDesc& P, int N, int y, int z) {
    if (ph.tooth > P.n - 1 || done_at(p, b)) return;
    const int Nc = level_side(P.n, l + 1);
    const T* src = visit_result<T>(p, P, ph.tooth, l + 1);
    const T* Bc = (const T*)p.B + P.off_lvl[l + 1];
    const T* base = init ? nullptr : visit_result<T>(p, P, ph.prev_tooth, l);
    T* El = (T*)p.E + P.off_lvl[l];
    const long long row = ((long long)z * N + y) * N;
    // coarse rows contributing to this fine row, with weights
    const int y0 = y >> 1, z0 = z >> 1;
    const int ny = (y & 1) ? 2 : 1, nz = (DIM == 3 && (z & 1)) ? 2 : 1;
    const T wyz = (ny == 2 ? (T)0.5 : (T)1) * (nz == 2 ? (T)0.5 : (T)1);
    for (int x = lane; x < N; x += 32) {
      const int x0 = x >> 1;
      const bool odd = x & 1;
      T val = (T)0;
      for (int cz = 0; cz < nz; ++cz)
        for (int cy = 0; cy < ny; ++cy) {
          const long long cr = ((long long)(DIM == 3 ? z0 + cz : 0) * Nc + (y0 + cy)) * Nc;
          T d = src[cr + x0] - (init ? (T)0 : Bc[cr + x0]);
          if (odd) d = (T)0.5 * (d + (src[cr + x0 + 1] - (init ? (T)0 : Bc[cr + x0 + 1])));
          val += d;
        }
      val *= wyz;
      El[row + x] = (init ? (T)0 : base[row + x]) + val;
    }
  });
}

template <typename T, int DIM>
__device__ void phase_prolong(const KernelParams& p, const Phase& ph, unsigned char* smem) {
  if (DIM == 3) {
    for_tasks(p, ph.level, [&](const TileTask& tk) {
      if (ph.tooth > prob_at(p, tk.b).n - 1 || done_at(p, tk.b)) return;
      prolong3<T>(p, ph, tk, (ProlongStage<T>*)smem);
    });
    return;
  }
  phase_prolong_rows<T, DIM>(p, ph);
}

// Moving one level coarser: E_l = B_l = (result at level l-1) on the level-l subset.
template <typename T, int DIM>
__device__ void phase_inject(const KernelParams& p, const Phase& ph) {
  const int l = ph.level;
  const int lane = threadIdx.x & 31;
  for_rows<DIM>(p, l, [&](int b, const ProblemDesc& P, int N, int y, int z) {
    if (ph.tooth > P.n - 1 || l > P.n - 1 || done_at(p, b)) return;
    const int Nf = level_side(P.n, l - 1);
    const T* src = visit_result<T>(p, P, ph.tooth, l - 1) + ((long long)(2 * z) * Nf + 2 * y) * Nf;
    const long long row = ((long long)z * N + y) * N;
    T* E = (T*)p.E + P.off_lvl[l] + row;
    T* B = (T*)p.B + P.off_lvl[l] + row;
    for (int xb = lane; xb < N; xb += 32 * kInjectBatch) {
      T v[kInjectBatch];
#pragma unroll
      for (int u = 0; u < kInjectBatch; ++u) v[u] = xb + 32 * u < N ? src[2 * (xb + 32 * u)] : (T)0;
#pragma unroll
      for (int u = 0; u < kInjectBatch; ++u)
        if (xb + 32 * u < N) {
          E[xb + 32 * u] = v[u];
          B[xb + 32 * u] = v[u];
        }
    }
  });
}

// ---------------------------------------------------------------------------------------------
// Pure-Neumann problems with a >= 0 (Sec. 3.2, Eq. 10): after the cycle's last sweep the constant mode is
// projected out of u, u -= <u> with <u> the trapezoid-rule mean -- for a = 0 it spans the
// operator's null space, for a > 0 the pseudo-time iteration would let it grow.  Deterministic:
// weighted row sums by warps (a fixed shuffle tree), one CTA per problem adds them in a fixed
// order, then every node is shifted.
// ---------------------------------------------------------------------------------------------
template <int DIM>
__device__ void phase_mean_rows(const KernelParams& p) {
  const int lane = threadIdx.x & 31;
  for_rows<DIM>(p, 0, [&](int b, const ProblemDesc& P, int N, int y, int z) {
    if (!P.project_mean || done_at(p, b)) return;
    const double* u = p.U + P.off_full + ((long long)z * N + y) * N;
    double s = 0.0;
    for (int x = lane; x < N; x += 32) s += (x == 0 || x == N - 1) ? 0.5 * u[x] : u[x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const double wy = (y == 0 || y == N - 1) ? 0.5 : 1.0;
      const double wz = DIM == 3 ? ((z == 0 || z == N - 1) ? 0.5 : 1.0) : 1.0;
      p.rowsum[p.row_prefix[b] + (DIM == 3 ? (long long)z * N + y : y)] = s * wy * wz;
    }
  });
}

// (the partial sums live in the dynamic shared memory: static shared memory is kept small so that two
// CTAs per SM fit the 196 KB shared-memory carveout and leave L1 its 60 KB)
__device__ void phase_mean_reduce(const KernelParams& p, int dim, unsigned char* smem) {
  double* s_part = (double*)smem;
  for (int b = blockIdx.x; b < p.batch; b += gridDim.x) {
    const ProblemDesc& P = prob_at(p, b);
    if (!P.project_mean || done_at(p, b)) continue;
    const long long r0 = p.row_prefix[b], rows = p.row_prefix[b + 1] - r0;
    const long long chunk = (rows + kThreads - 1) / kThreads;
    double s = 0.0;
    for (long long r = threadIdx.x * chunk; r < (threadIdx.x + 1) * chunk && r < rows; ++r) s += p.rowsum[r0 + r];
    s_part[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) s_part[threadIdx.x] += s_part[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double cells = dim == 3 ? (double)(1LL << (3 * P.n)) : (double)(1LL << (2 * P.n));  // sum of the weights
      p.umean[b] = s_part[0] / cells;
    }
    __syncthreads();
  }
}

template <int DIM>
__device__ void phase_mean_apply(const KernelParams& p) {
  const int lane = threadIdx.x & 31;
  for_rows<DIM>(p, 0, [&](int b, const ProblemDesc& P, int N, int y, int z) {
    if (!P.project_mean || done_at(p, b)) return;
    double* u = p.U + P.off_full + ((long long)z * N + y) * N;
    const double m = p.umean[b];
    for (int x = lane; x < N; x += 32) u[x] -= m;
  });
}

// ---------------------------------------------------------------------------------------------
// Coarse tail (3-D mixed form, one problem): the phases of a cycle that touch only the three
// coarsest levels (9^3, 5^3 and 3^3 nodes: the restriction passes into them, the visits of teeth
// n - 1 and n - 2 and the start of tooth n - 3) are about a quarter of a cycle's phases, and on the
// whole grid each costs a grid barrier and an L2 round trip for a few hundred nodes.  CTA 0 runs
// them instead with all their arrays in shared memory and CTA barriers between them, while the
// other CTAs wait at one grid barrier.  Every operation is the grid phase's own arithmetic in the
// same order (restriction: phase_restrict; sweep: sweep3's plane sums and update; interpolation:
// prolong3; injection: phase_inject), so results are bit-identical.  In: the restricted residual of
// level n - 4 (17^3), sigma and the step factor of the tail levels; out: E, E2, B and R of the tail
// levels.  Kept out of line with plain arguments, so that the persistent kernel's other phases keep
// their register allocation.
// ---------------------------------------------------------------------------------------------
constexpr int kTailLevels = 3;
// nodes of tail level j (9^3, 5^3, 3^3) and its offset in shared memory (E, E2, B, R, S, Q per level)
__host__ __device__ constexpr int tail_nodes(int j) { return j == 0 ? 729 : (j == 1 ? 125 : 27); }
__host__ __device__ constexpr int tail_off(int j) { return j == 0 ? 0 : (j == 1 ? 6 * 729 : 6 * 729 + 6 * 125); }
constexpr int kTailRf = 6 * (729 + 125 + 27);                           // staged residual of level n - 4
constexpr int kTailFloats = kTailRf + 17 * 17 * 17;
static_assert(sizeof(float) * kTailFloats <= phase_smem_bytes<float>(), "shared memory");
enum TailArr { kTE = 0, kTE2 = 1, kTB = 2, kTR = 3, kTS = 4, kTQ = 5 };

struct TailPlane {
  float v, F, C, sv, sF, sC;
};

// The tail's operations on one level of N nodes per side (9, 5 or 3), one node per thread and pass;
// each is the grid phase's arithmetic in the same order.  One instance per operation (the tail's code
// is fetched cold once per cycle: fewer instances, fewer misses).  Node i of a level decodes with a
// float reciprocal, exact here: (i + 1/2) / N lies at least 1/(2N) from an integer and i < 2^13.
__device__ __forceinline__ void tail_decode(int i, int N, float inv_n, int& x, int& y, int& z) {
  const int q = __float2int_rz(((float)i + 0.5f) * inv_n);
  z = __float2int_rz(((float)q + 0.5f) * inv_n);
  x = i - q * N;
  y = q - z * N;
}

__device__ __forceinline__ void tail_restrict(int N, const float* src, float* dst) {
  const int Ns = 2 * N - 1, M = N * N * N;
  const float inv_n = 1.0f / (float)N;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int x, y, z;
    tail_decode(i, N, inv_n, x, y, z);
    const int xm = refl(2 * x - 1, Ns), x0 = 2 * x, xp = refl(2 * x + 1, Ns);
    float acc = 0.0f;
#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
      float accz = 0.0f;
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        const float* row = src + (refl(2 * z + dz - 1, Ns) * Ns + refl(2 * y + dy - 1, Ns)) * Ns;
        accz = rn_fma(dy == 1 ? 0.5f : 0.25f, restrict_line(row[xm], row[x0], row[xp]), accz);
      }
      acc = rn_fma(dz == 1 ? 0.5f : 0.25f, accz, acc);
    }
    dst[i] = acc;
  }
}

__device__ __forceinline__ void tail_sweep(int N, const ProblemDesc& P, const float* src, float* dst, const float* S,
                                           const float* Qv, const float* Rl, bool het, bool zero_in, float inv_c,
                                           float q_const, float one_m_omega, float w_e, float w_c) {
  const int M = N * N * N;
  const float inv_n = 1.0f / (float)N;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int x, y, z;
    tail_decode(i, N, inv_n, x, y, z);
    if (is_fixed<3>(P, N, x, y, z)) continue;
    const int xs[3] = {refl(x - 1, N), x, refl(x + 1, N)};
    const int ys[3] = {refl(y - 1, N), y, refl(y + 1, N)};
    TailPlane pl[3];  // planes z - 1, z, z + 1: sweep3's in-plane sums
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int zz = refl(z - 1 + k, N);
      float a[3][3], se[3][3];
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          const int idx = (zz * N + ys[ii]) * N + xs[jj];
          a[ii][jj] = zero_in ? 0.0f : src[idx];
          se[ii][jj] = het ? rn_mul(S[idx], a[ii][jj]) : 0.0f;
        }
      pl[k].v = a[1][1];
      pl[k].F = (a[1][0] + a[1][2]) + (a[0][1] + a[2][1]);
      pl[k].C = (a[0][0] + a[0][2]) + (a[2][0] + a[2][2]);
      pl[k].sv = se[1][1];
      pl[k].sF = (se[1][0] + se[1][2]) + (se[0][1] + se[2][1]);
      pl[k].sC = (se[0][0] + se[0][2]) + (se[2][0] + se[2][2]);
    }
    const TailPlane &m = pl[0], &o = pl[1], &nw = pl[2];
    const float CSe = rn_fma(w_c, m.C + nw.C, rn_fma(w_e, (o.C + m.F) + nw.F, (o.F + m.v) + nw.v));
    if (het) {
      const float CSse = rn_fma(w_c, m.sC + nw.sC, rn_fma(w_e, (o.sC + m.sF) + nw.sF, (o.sF + m.sv) + nw.sv));
      dst[i] = rn_fma(Qv[i], rn_fma(-Rl[i], inv_c, rn_fma(S[i], CSe, CSse)), rn_mul(one_m_omega, o.v));
    } else {
      dst[i] = rn_fma(q_const, rn_fma(-Rl[i], inv_c, rn_mul(2.0f, CSe)), rn_mul(one_m_omega, o.v));
    }
  }
}

__device__ __forceinline__ void tail_prolong(int N, const float* src, const float* Bc, const float* base, float* El,
                                             bool init) {
  const int Nc = (N + 1) / 2, M = N * N * N;
  const float inv_n = 1.0f / (float)N;
  auto delta = [&](int cx, int cy, int cz) {
    const int c = (cz * Nc + cy) * Nc + cx;
    return init ? src[c] : rn_add(src[c], -Bc[c]);
  };
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int x, y, z;
    tail_decode(i, N, inv_n, x, y, z);
    const int cx = x >> 1, cy = y >> 1;
    auto plane = [&](int cz) {  // prolong3's in-plane interpolation from coarse plane cz
      const float a0 = delta(cx, cy, cz), a1 = delta(cx + (x & 1), cy, cz);
      const float ra = (x & 1) ? half_sum(a0, a1) : a0;
      if (!(y & 1)) return ra;
      const float b0 = delta(cx, cy + 1, cz), b1 = delta(cx + (x & 1), cy + 1, cz);
      const float rb = (x & 1) ? half_sum(b0, b1) : b0;
      return half_sum(ra, rb);
    };
    const float v = (z & 1) ? half_sum(plane(z >> 1), plane((z >> 1) + 1)) : plane(z >> 1);
    El[i] = rn_add(init ? 0.0f : base[i], v);
  }
}

__device__ __forceinline__ void tail_inject(int N, const float* src, float* El, float* Bl) {
  const int Nf = 2 * N - 1, M = N * N * N;
  const float inv_n = 1.0f / (float)N;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int x, y, z;
    tail_decode(i, N, inv_n, x, y, z);
    const float v = src[((2 * z) * Nf + 2 * y) * Nf + 2 * x];
    El[i] = v;
    Bl[i] = v;
  }
}

__device__ __noinline__ void coarse_tail(const Phase* phases, int q0, int q1, float* E, float* E2, float* Bg,
                                         float* R, const float* SIG, const float* Q, float one_m_omega, float w_e,
                                         float w_c, int n_r, unsigned long long* stamps) {
  extern __shared__ __align__(16) unsigned char tail_smem[];  // the kernel's dynamic shared memory
  float* sm = reinterpret_cast<float*>(tail_smem);
  const ProblemDesc& P = s_prob0;
  const int n = P.n, lt = n - kTailLevels;
  const bool het = P.hetero != 0;
  const int tid = threadIdx.x, nt = blockDim.x;
  auto arr = [&](int l, int which) { return sm + tail_off(l - lt) + which * tail_nodes(l - lt); };
  auto result = [&](int tooth, int l) {  // buffer holding the visit result of tooth `tooth` at level l
    return arr(l, (visit_sweeps(n_r, n, tooth, false) & 1) ? kTE2 : kTE);
  };
  // in (asynchronous copies, one wait): sigma and q of the tail levels, R of level lt - 1; E, E2
  // zeroed meanwhile (fixed nodes stay 0)
  for (int j = 0; j < kTailLevels; ++j) {
    const int l = lt + j, M = tail_nodes(j);
    if (het)
      for (int i = tid; i < M; i += nt) {
        cp_async_t(&arr(l, kTS)[i], &SIG[P.off_lvl[l] + i]);
        cp_async_t(&arr(l, kTQ)[i], &Q[P.off_lvl[l] + i]);
      }
  }
  for (int i = tid; i < 17 * 17 * 17; i += nt) cp_async_t(&sm[kTailRf + i], &R[P.off_lvl[lt - 1] + i]);
  cp_async_commit();
  for (int j = 0; j < kTailLevels; ++j)
    for (int i = tid; i < 2 * tail_nodes(j); i += nt) arr(lt + j, kTE)[i] = 0.0f;
  cp_async_wait<0>();
  __syncthreads();
  for (int q = q0; q < q1; ++q) {
    const Phase ph = q < kPhaseCache ? s_phase[q] : phases[q];
    const int l = ph.level, N = level_side(n, l);
    if (ph.op == OP_RESTRICT) {
      tail_restrict(N, l == lt ? sm + kTailRf : arr(l - 1, kTR), arr(l, kTR));
    } else if (ph.op == OP_SWEEP) {
      const bool odd = (ph.sweep & 1) != 0;
      const bool zero_in = ph.sweep == 0 && (ph.flags & kFirstOfTooth) && ph.tooth == n - 1;
      tail_sweep(N, P, arr(l, odd ? kTE2 : kTE), arr(l, odd ? kTE : kTE2), arr(l, kTS), arr(l, kTQ), arr(l, kTR), het,
                 zero_in, P.inv_c_f[l], P.q_const_f[l], one_m_omega, w_e, w_c);
    } else if (ph.op == OP_PROLONG) {
      const bool init = (ph.flags & kInit) != 0;
      tail_prolong(N, result(ph.tooth, l + 1), arr(l + 1, kTB), init ? nullptr : result(ph.prev_tooth, l), arr(l, kTE),
                   init);
    } else {  // OP_INJECT
      tail_inject(N, result(ph.tooth, l - 1), arr(l, kTE), arr(l, kTB));
    }
    __syncthreads();
    if (stamps && tid == 0) stamps[3 + q] = globaltimer();
  }
  // out: the tail levels' E, E2, B and R (read by the phases after the tail and by the next cycle)
  for (int j = 0; j < kTailLevels; ++j) {
    const int l = lt + j, M = tail_nodes(j);
    const long long o = P.off_lvl[l];
    for (int i = tid; i < M; i += nt) {
      E[o + i] = arr(l, kTE)[i];
      E2[o + i] = arr(l, kTE2)[i];
      Bg[o + i] = arr(l, kTB)[i];
      R[o + i] = arr(l, kTR)[i];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// The persistent cycle kernel
// ---------------------------------------------------------------------------------------------
template <typename T, int DIM>
__device__ __forceinline__ void run_phase(const KernelParams& p, const Phase& ph, int c, unsigned char* sm) {
  switch (ph.op) {
    case OP_RESTRICT: phase_restrict_any<T, DIM>(p, ph.level, sm); break;
    case OP_SWEEP: phase_sweep<T, DIM>(p, ph, c, sm); break;
    case OP_PROLONG: phase_prolong<T, DIM>(p, ph, sm); break;
    case OP_INJECT: phase_inject<T, DIM>(p, ph); break;
    case OP_MEAN_ROWS: phase_mean_rows<DIM>(p); break;
    case OP_MEAN_REDUCE: phase_mean_reduce(p, DIM, sm); break;
    default: phase_mean_apply<DIM>(p); break;
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads, SGML_MIN_CTAS) cycle_kernel(const KernelParams p) {
  extern __shared__ __align__(16) unsigned char sm[];
  load_tables(p);
  load_done(p);
  if (p.fresh) {
    phase_lift<T, DIM>(p);
    if (!grid_sync(p.sync, p.timeout_ns, p.withhold_barrier)) return;
  }
  // Optional trace: CTA 0 stamps the global timer after every barrier of the first cycles.
  auto stamp = [&](int c, int slot) {
    if (p.trace && blockIdx.x == 0 && threadIdx.x == 0 && c < p.trace_cycles)
      p.trace[(long long)c * (p.nphases + 3) + slot] = globaltimer();
  };
  for (int c = 0;; ++c) {
    stamp(c, 0);
    phase_outer<T, DIM>(p, c, sm);
    if (!grid_sync(p.sync, p.timeout_ns, p.withhold_barrier)) return;
    stamp(c, 1);
    if (blockIdx.x == 0) phase_check<T, DIM>(p, c);
    if (!grid_sync(p.sync, p.timeout_ns, p.withhold_barrier)) return;
    stamp(c, 2);
    if (!ld_volatile(&p.sync->active[c & 1])) break;
    load_done(p);
    for (int q = 0; q < p.nphases; ++q) {
      const Phase ph = phase_at(p, q);
      if (DIM == 3 && sizeof(T) == 4 && (ph.flags & kTailStart)) {
        // coarse tail: one CTA runs phases q .. ph.prev_tooth - 1 in shared memory, one grid barrier
        if ((int)blockIdx.x == p.tail_cta)
          coarse_tail(p.phases, q, ph.prev_tooth, (float*)p.E, (float*)p.E2, (float*)p.B, (float*)p.R,
                      (const float*)p.SIG, (const float*)p.Q, p.one_m_omega_f, p.w_edge_f, p.w_corner_f, p.n_r,
                      (p.trace && c < p.trace_cycles) ? p.trace + (long long)c * (p.nphases + 3) : nullptr);
        q = ph.prev_tooth - 1;
        if (!grid_sync(p.sync, p.timeout_ns, p.withhold_barrier)) return;
        stamp(c, 3 + q);
        continue;
      }
      run_phase<T, DIM>(p, ph, c, sm);
      if (!grid_sync(p.sync, p.timeout_ns, p.withhold_barrier)) return;
      stamp(c, 3 + q);
    }
    if (p.diag) diag_commit(p, c);
  }
}

// One phase per launch (profiling / graph-capture mode).  which: -3 lift, -2 outer step,
// -1 convergence check (launch with one CTA), >= 0 index into the phase table.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads, SGML_MIN_CTAS) phase_kernel(const KernelParams p, int which, int c) {
  extern __shared__ __align__(16) unsigned char sm[];
  load_tables(p);
  load_done(p);
  if (which == -3) {
    phase_lift<T, DIM>(p);
  } else if (which == -2) {
    phase_outer<T, DIM>(p, c, sm);
  } else if (which == -1) {
    if (blockIdx.x == 0) phase_check<T, DIM>(p, c);
  } else {
    const Phase ph = phase_at(p, which);
    run_phase<T, DIM>(p, ph, c, sm);
    if (p.diag) diag_commit(p, c);
  }
}

// ---------------------------------------------------------------------------------------------
// FP64 residual at one level-0 unknown: r = f - delta L_0 u (Eq. 5 + a u), Neumann images carry
// the prescribed outward derivative.  The link terms are formed as sigma-weighted differences
// (u_o - u_i), grouped into face, edge and corner classes.
// ---------------------------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ double residual_at(const ProblemDesc& P, int N, int i, int j, int k,
                                              const double* __restrict__ U, const double* __restrict__ F,
                                              const double* __restrict__ SIG, const double* __restrict__ A,
                                              double kappa, double w_edge, double w_corner) {
  const int c = lin<DIM>(i, j, k, N);
  const double uc = U[c];
  const double sc = P.hetero ? SIG[c] : 1.0;
  double cls[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz) {
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (dx == 0 && dy == 0 && dz == 0) continue;
        const int nz = (dx != 0) + (dy != 0) + (dz != 0);
        double ghost = 0.0;
        int ii = i + dx, jj = j + dy, kk = k + dz;
        if (ii < 0) { ghost += 2.0 * P.h * P.face_value[0]; ii = 1; }
        if (ii > N - 1) { ghost += 2.0 * P.h * P.face_value[1]; ii = N - 2; }
        if (jj < 0) { ghost += 2.0 * P.h * P.face_value[2]; jj = 1; }
        if (jj > N - 1) { ghost += 2.0 * P.h * P.face_value[3]; jj = N - 2; }
        if (DIM == 3) {
          if (kk < 0) { ghost += 2.0 * P.h * P.face_value[4]; kk = 1; }
          if (kk > N - 1) { ghost += 2.0 * P.h * P.face_value[5]; kk = N - 2; }
        }
        const int o = lin<DIM>(ii, jj, kk, N);
        const double du = (U[o] + ghost) - uc;
        const double t = P.hetero ? (sc + SIG[o]) * du : 2.0 * du;
        cls[nz - 1] += t;
      }
    }
  }
  const double sum = cls[0] + w_edge * cls[1] + (DIM == 3 ? w_corner * cls[2] : 0.0);
  const double a = P.a_per_node ? A[c] : P.a_scalar;
  const double Lu = kappa / (2.0 * P.h * P.h) * sum + a * uc;
  return F[c] - Lu;
}

template <typename T, int DIM>
static void* phase_fn() {
  return (void*)phase_kernel<T, DIM>;
}

template <typename T, int DIM>
static void* cycle_fn() {
  return (void*)cycle_kernel<T, DIM>;
}

static size_t smem_for(int mixed) { return mixed ? phase_smem_bytes<float>() : phase_smem_bytes<double>(); }

static void* pick(int mixed, int dim, bool cycle) {
  if (cycle) {
    if (mixed) return dim == 3 ? cycle_fn<float, 3>() : cycle_fn<float, 2>();
    return dim == 3 ? cycle_fn<double, 3>() : cycle_fn<double, 2>();
  }
  if (mixed) return dim == 3 ? phase_fn<float, 3>() : phase_fn<float, 2>();
  return dim == 3 ? phase_fn<double, 3>() : phase_fn<double, 2>();
}

// Opt the kernel into its dynamic shared memory (above the 48 KB default); idempotent.
static cudaError_t prepare_fn(void* fn, int mixed) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_for(mixed));
}

cudaError_t launch_phase_kernel(const KernelParams& p, int mixed, int dim, int blocks, int threads, int which, int c,
                                cudaStream_t s) {
  (void)threads;
  void* fn = pick(mixed, dim, false);
  cudaError_t e = prepare_fn(fn, mixed);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&p, (void*)&which, (void*)&c};
  return cudaLaunchKernel(fn, dim3(which == -1 ? 1 : blocks), dim3(kThreads), args, smem_for(mixed), s);
}

cudaError_t launch_cycle_kernel(const KernelParams& p, int mixed, int dim, int blocks, int threads, cudaStream_t s) {
  (void)threads;
  void* fn = pick(mixed, dim, true);
  cudaError_t e = prepare_fn(fn, mixed);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&p};
  return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(kThreads), args, smem_for(mixed), s);
}

size_t cycle_kernel_smem(int mixed) { return smem_for(mixed); }

int cycle_kernel_occupancy(int mixed, int dim, int threads, int* blocks_per_sm) {
  (void)threads;
  void* fn = pick(mixed, dim, true);
  if (prepare_fn(fn, mixed) != cudaSuccess) return 1;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kThreads, smem_for(mixed));
}

// ---------------------------------------------------------------------------------------------
// Setup kernels (coefficient pyramid), residual and adjoint gradient: plain FP64 node kernels.
// ---------------------------------------------------------------------------------------------

// One restriction pass of a coefficient field (FP64, even images on every face).
template <int DIM>
__global__ void restrict64_kernel(const double* __restrict__ src, int Ns, double* __restrict__ dst, int Nt) {
  const long long M = level_nodes<DIM>(Nt);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < M; t += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decode<DIM>(t, Nt, i, j, k);
    double acc = 0.0;
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const double w = (dx ? 0.25 : 0.5) * (dy ? 0.25 : 0.5) * (DIM == 3 ? (dz ? 0.25 : 0.5) : 1.0);
          acc += w * src[lin<DIM>(refl(2 * i + dx, Ns), refl(2 * j + dy, Ns), DIM == 3 ? refl(2 * k + dz, Ns) : 0, Ns)];
        }
    dst[t] = acc;
  }
}

// Level-l coefficients in cycle precision: SIG = sigma_l, Q = dtau_l * kappa / (2 H^2) with the
// Jacobi-scaled step dtau = theta * gain / D_i, D_i = kappa/(2H^2) sum_o w_o (sigma_i + sigma_o) - a_i.
template <typename T, int DIM>
__global__ void setup_level_kernel(ProblemDesc P, int l, const double* __restrict__ sig, const double* __restrict__ a,
                                   double kappa, double w_edge, double w_corner, double theta_gain,
                                   T* __restrict__ SIG, T* __restrict__ Q, T* __restrict__ AT) {
  const int N = level_side(P.n, l);
  const long long M = level_nodes<DIM>(N);
  const double H = P.h * (double)(1 << l);
  const double cH = kappa / (2.0 * H * H);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < M; t += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decode<DIM>(t, N, i, j, k);
    const double sc = sig ? sig[t] : 1.0;
    double cls[3] = {0.0, 0.0, 0.0};
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (dx == 0 && dy == 0 && dz == 0) continue;
          const int nz = (dx != 0) + (dy != 0) + (dz != 0);
          const double so = sig ? sig[lin<DIM>(refl(i + dx, N), refl(j + dy, N), DIM == 3 ? refl(k + dz, N) : 0, N)] : 1.0;
          cls[nz - 1] += sc + so;
        }
    const double sum = cls[0] + w_edge * cls[1] + (DIM == 3 ? w_corner * cls[2] : 0.0);
    const double av = a ? a[t] : P.a_scalar;
    const double D = cH * sum - av;
    SIG[t] = (T)sc;
    Q[t] = (T)(theta_gain / D * cH);
    if (AT) AT[t] = (T)av;
  }
}

template <int DIM>
__global__ void residual64_kernel(ProblemDesc P, const double* __restrict__ U, const double* __restrict__ F,
                                  const double* __restrict__ SIG, const double* __restrict__ A, double kappa,
                                  double w_edge, double w_corner, double* __restrict__ r) {
  const int N = level_side(P.n, 0);
  const long long M = level_nodes<DIM>(N);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < M; t += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decode<DIM>(t, N, i, j, k);
    r[t] = is_fixed<DIM>(P, N, i, j, k) ? 0.0 : residual_at<DIM>(P, N, i, j, k, U, F, SIG, A, kappa, w_edge, w_corner);
  }
}

template <int DIM>
__global__ void sigma_gradient_kernel(ProblemDesc P, const double* __restrict__ lam, const double* __restrict__ U,
                                      double kappa, double w_edge, double w_corner, double* __restrict__ g) {
  const int N = level_side(P.n, 0);
  const long long M = level_nodes<DIM>(N);
  const double c0 = kappa / (2.0 * P.h * P.h);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < M; t += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decode<DIM>(t, N, i, j, k);
    const double lc = lam[t], uc = U[t];
    double cls[3] = {0.0, 0.0, 0.0};
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (dx == 0 && dy == 0 && dz == 0) continue;
          const int ii = i + dx, jj = j + dy, kk = k + dz;
          if (ii < 0 || ii > N - 1 || jj < 0 || jj > N - 1) continue;
          if (DIM == 3 && (kk < 0 || kk > N - 1)) continue;
          const int nz = (dx != 0) + (dy != 0) + (dz != 0);
          const int o = lin<DIM>(ii, jj, kk, N);
          cls[nz - 1] += (lam[o] - lc) * (U[o] - uc);
        }
    g[t] = c0 * (cls[0] + w_edge * cls[1] + (DIM == 3 ? w_corner * cls[2] : 0.0));
  }
}

__global__ void fill_kernel(double* dst, long long n, double v) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    dst[t] = v;
}

}  // namespace SGML_KNS

#ifdef SGML_DEFINE_COMMON
namespace sgml {
using namespace SGML_KNS;
static int grid_for(long long M) {
  long long b = (M + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

cudaError_t launch_restrict64(int dim, const double* src, int Ns, double* dst, int Nt, cudaStream_t s) {
  const long long M = dim == 3 ? (long long)Nt * Nt * Nt : (long long)Nt * Nt;
  if (dim == 3) restrict64_kernel<3><<<grid_for(M), 256, 0, s>>>(src, Ns, dst, Nt);
  else restrict64_kernel<2><<<grid_for(M), 256, 0, s>>>(src, Ns, dst, Nt);
  return cudaGetLastError();
}

cudaError_t launch_setup_level(int mixed, int dim, const ProblemDesc& P, int l, const double* sig, const double* a,
                               double kappa, double w_edge, double w_corner, double theta_gain, void* SIG_T,
                               void* Q_T, void* A_T, cudaStream_t s) {
  const int N = (1 << (P.n - l)) + 1;
  const long long M = dim == 3 ? (long long)N * N * N : (long long)N * N;
  const long long off = P.off_lvl[l];
  if (mixed) {
    float* S = (float*)SIG_T + off;
    float* Q = (float*)Q_T + off;
    float* AT = A_T ? (float*)A_T + off : nullptr;
    if (dim == 3) setup_level_kernel<float, 3><<<grid_for(M), 256, 0, s>>>(P, l, sig, a, kappa, w_edge, w_corner, theta_gain, S, Q, AT);
    else setup_level_kernel<float, 2><<<grid_for(M), 256, 0, s>>>(P, l, sig, a, kappa, w_edge, w_corner, theta_gain, S, Q, AT);
  } else {
    double* S = (double*)SIG_T + off;
    double* Q = (double*)Q_T + off;
    double* AT = A_T ? (double*)A_T + off : nullptr;
    if (dim == 3) setup_level_kernel<double, 3><<<grid_for(M), 256, 0, s>>>(P, l, sig, a, kappa, w_edge, w_corner, theta_gain, S, Q, AT);
    else setup_level_kernel<double, 2><<<grid_for(M), 256, 0, s>>>(P, l, sig, a, kappa, w_edge, w_corner, theta_gain, S, Q, AT);
  }
  return cudaGetLastError();
}

cudaError_t launch_residual64(int dim, const ProblemDesc& P, const double* U, const double* F, const double* SIG64,
                              const double* A64, double kappa, double w_edge, double w_corner, double* r,
                              cudaStream_t s) {
  const int N = (1 << P.n) + 1;
  const long long M = dim == 3 ? (long long)N * N * N : (long long)N * N;
  if (dim == 3) residual64_kernel<3><<<grid_for(M), 256, 0, s>>>(P, U, F, SIG64, A64, kappa, w_edge, w_corner, r);
  else residual64_kernel<2><<<grid_for(M), 256, 0, s>>>(P, U, F, SIG64, A64, kappa, w_edge, w_corner, r);
  return cudaGetLastError();
}

cudaError_t launch_sigma_gradient(int dim, const ProblemDesc& P, const double* lam, const double* U, double kappa,
                                  double w_edge, double w_corner, double* g, cudaStream_t s) {
  const int N = (1 << P.n) + 1;
  const long long M = dim == 3 ? (long long)N * N * N : (long long)N * N;
  if (dim == 3) sigma_gradient_kernel<3><<<grid_for(M), 256, 0, s>>>(P, lam, U, kappa, w_edge, w_corner, g);
  else sigma_gradient_kernel<2><<<grid_for(M), 256, 0, s>>>(P, lam, U, kappa, w_edge, w_corner, g);
  return cudaGetLastError();
}

// Trapezoid-rule mean of one problem's full-grid array (pure-Neumann source projection), in a
// fixed order: per-block sums of contiguous ranges, then one block adds them.
__global__ void mean_partial_kernel(int dim, int N, const double* __restrict__ v, double* __restrict__ part) {
  __shared__ double s_part[256];
  const long long M = dim == 3 ? (long long)N * N * N : (long long)N * N;
  const long long chunk = (M + gridDim.x - 1) / gridDim.x;
  const long long i0 = (long long)blockIdx.x * chunk, i1 = i0 + chunk < M ? i0 + chunk : M;
  double s = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const int x = (int)(i % N), y = (int)((i / N) % N), z = dim == 3 ? (int)(i / ((long long)N * N)) : 0;
    double w = (x == 0 || x == N - 1) ? 0.5 : 1.0;
    if (y == 0 || y == N - 1) w *= 0.5;
    if (dim == 3 && (z == 0 || z == N - 1)) w *= 0.5;
    s += w * v[i];
  }
  s_part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s_part[threadIdx.x] += s_part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s_part[0];
}

__global__ void mean_finish_kernel(int parts, double cells, const double* __restrict__ part, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < parts; ++k) s += part[k];
    *out = s / cells;
  }
}

__global__ void add_scalar_kernel(double* v, long long n, const double* __restrict__ d, double sign) {
  const double a = sign * *d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[i] += a;
}

cudaError_t launch_project_mean(int dim, int n, double* v, double* scratch, cudaStream_t s) {
  // scratch: 257 doubles; scratch[256] receives the mean, which is then subtracted from v.
  const int N = (1 << n) + 1;
  const long long M = dim == 3 ? (long long)N * N * N : (long long)N * N;
  const int parts = 256;
  mean_partial_kernel<<<parts, 256, 0, s>>>(dim, N, v, scratch);
  mean_finish_kernel<<<1, 32, 0, s>>>(parts, dim == 3 ? (double)(1LL << (3 * n)) : (double)(1LL << (2 * n)), scratch,
                                       scratch + 256);
  add_scalar_kernel<<<grid_for(M), 256, 0, s>>>(v, M, scratch + 256, -1.0);
  return cudaGetLastError();
}

cudaError_t launch_add_scalar(double* v, long long n, const double* d_value, double sign, cudaStream_t s) {
  add_scalar_kernel<<<grid_for(n), 256, 0, s>>>(v, n, d_value, sign);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* dst, long long n, double v, cudaStream_t s) {
  fill_kernel<<<grid_for(n), 256, 0, s>>>(dst, n, v);
  return cudaGetLastError();
}

}  // namespace sgml
#endif
