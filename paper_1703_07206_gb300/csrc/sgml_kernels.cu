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

namespace sgml {

// ---------------------------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ int refl(int i, int N) { return i < 0 ? -i : (i > N - 1 ? 2 * (N - 1) - i : i); }

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

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// ---------------------------------------------------------------------------------------------
// Bounded grid barrier.  Every wait has a time limit; on expiry the barrier records the error and
// every CTA returns from the kernel at its next barrier, so a fault in the schedule can never hang
// the GPU.  Requires all CTAs to be co-resident (cooperative launch).
// ---------------------------------------------------------------------------------------------
__device__ bool grid_sync(GridSync* gs, unsigned long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned int g = ld_acquire(&gs->gen);
    __threadfence();
    unsigned int prev = atomicAdd(&gs->count, 1u);
    if (prev == gridDim.x - 1) {
      atomicExch(&gs->count, 0u);
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    } else {
      unsigned long long t0 = globaltimer();
      while (ld_acquire(&gs->gen) == g) {
        if (ld_volatile(&gs->error)) {
          ok = 0;
          break;
        }
        if (globaltimer() - t0 > timeout_ns) {
          atomicExch(&gs->error, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (ld_volatile(&gs->error)) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
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

// ---------------------------------------------------------------------------------------------
// Tile iteration: level-l nodes of all problems are cut into tiles of `tile` nodes (tiles never
// straddle problems); CTA c takes tiles c, c + G, ...  Uniform across the CTA.
// ---------------------------------------------------------------------------------------------
template <class Body>
__device__ __forceinline__ void for_tiles(const KernelParams& p, int l, Body&& body) {
  const long long* tp = p.tile_prefix + (long long)l * (p.batch + 1);
  const long long total = tp[p.batch];
  int b = 0;
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    while (tp[b + 1] <= t) ++b;
    body(b, (t - tp[b]) * p.tile + threadIdx.x);
  }
}

// ---------------------------------------------------------------------------------------------
// Phases
// ---------------------------------------------------------------------------------------------

// Lift the Dirichlet values into u (0 on unknowns) and accumulate ||f|| over the unknowns.
template <typename T, int DIM>
__device__ void phase_lift(const KernelParams& p) {
  int cur = -1;
  double mx = 0.0, s2 = 0.0;
  for_tiles(p, 0, [&](int b, long long local) {
    if (b != cur) {
      if (cur >= 0) block_flush(mx, s2, &p.accum[cur].fmax_bits, &p.accum[cur].fsum2);
      cur = b;
      mx = s2 = 0.0;
    }
    const ProblemDesc& P = p.probs[b];
    const int N = level_side(P.n, 0);
    if (local >= level_nodes<DIM>(N)) return;
    int i, j, k;
    decode<DIM>(local, N, i, j, k);
    const long long g = P.off_full + local;
    if (is_fixed<DIM>(P, N, i, j, k)) {
      p.U[g] = dirichlet_value<DIM>(P, N, i, j, k);
    } else {
      p.U[g] = 0.0;
      const double f = p.F[g];
      mx = nan_max(mx, fabs(f));
      s2 += f * f;
    }
  });
  if (cur >= 0) block_flush(mx, s2, &p.accum[cur].fmax_bits, &p.accum[cur].fsum2);
}

// Scale of the residual cast of cycle c (mixed form): 1 / (max-norm of the previous residual).
__device__ __forceinline__ double cast_scale(const KernelParams& p, int b, int c) {
  if (!p.mixed) return 1.0;
  double ref = (c == 0 && p.fresh) ? __longlong_as_double((long long)p.accum[b].fmax_bits)
                                   : p.state[b].rmax_prev;
  return (ref > 0.0 && ref < 1e300) ? 1.0 / ref : 1.0;
}

// Outer step (FP64): r = f - delta L_0 u, its norms, and the cast (scaled) level-0 source of the
// cycle.  The correction of the previous cycle was already added to u by its last sweep.
template <typename T, int DIM>
__device__ void phase_outer(const KernelParams& p, int c) {
  T* R = (T*)p.R;
  int cur = -1;
  double mx = 0.0, s2 = 0.0, scale = 1.0;
  bool active = false;
  for_tiles(p, 0, [&](int b, long long local) {
    if (b != cur) {
      if (cur >= 0) block_flush(mx, s2, &p.accum[cur].rmax_bits[c & 1], &p.accum[cur].rsum2[c & 1]);
      cur = b;
      mx = s2 = 0.0;
      active = !p.accum[b].done;
      scale = cast_scale(p, b, c);
    }
    if (!active) return;
    const ProblemDesc& P = p.probs[b];
    const int N = level_side(P.n, 0);
    if (local >= level_nodes<DIM>(N)) return;
    int i, j, k;
    decode<DIM>(local, N, i, j, k);
    T* R0 = R + P.off_lvl[0];
    if (is_fixed<DIM>(P, N, i, j, k)) {
      R0[local] = (T)0;
      return;
    }
    const double r = residual_at<DIM>(P, N, i, j, k, p.U + P.off_full, p.F + P.off_full,
                                      p.SIG64 ? p.SIG64 + P.off_full : nullptr,
                                      p.A64 ? p.A64 + P.off_full : nullptr, p.kappa, p.w_edge, p.w_corner);
    R0[local] = (T)(r * scale);
    mx = nan_max(mx, fabs(r));
    s2 += r * r;
  });
  if (cur >= 0) block_flush(mx, s2, &p.accum[cur].rmax_bits[c & 1], &p.accum[cur].rsum2[c & 1]);
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
    const double rel = S.fnorm > 0.0 ? rmax / S.fnorm : 0.0;
    const double rel2 = S.fnorm2 > 0.0 ? sqrt(rs2) / S.fnorm2 : 0.0;
    S.rel = rel;
    S.rel_l2 = rel2;
    if (c < p.hist_cap) p.hist[(long long)b * p.hist_cap + c] = rel;
    S.hist_len = c + 1;
    if (c > 0) S.cycles += 1;
    S.grow = (rel > S.rel_prev) ? S.grow + 1 : 0;
    S.rel_prev = rel;
    S.rmax_prev = rmax;
    int st = 0, stop = 0;
    if (!(rel <= 1e300)) {
      st = -6;  // SGML_ERR_NONFINITE
      stop = 1;
    } else if (rel <= p.tol) {
      stop = 1;
    } else if (S.grow >= 3 && rel > 1.0) {
      st = -4;  // SGML_ERR_DIVERGED
      stop = 1;
    } else if (c >= p.max_cycles) {
      st = p.tol >= 0.0 ? -3 : 0;  // SGML_ERR_NOT_CONVERGED for a solve; fine for run_cycle
      stop = 1;
    }
    S.status = st;
    A.done = stop;
    A.rmax_bits[(c + 1) & 1] = 0ull;
    A.rsum2[(c + 1) & 1] = 0.0;
    if (!stop) any = 1;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) p.sync->active[c & 1] = any;
}

// Number of sweeps of a visit of tooth nu1 for a problem with n levels (Algorithm 3).
__device__ __forceinline__ int visit_sweeps(int n_r, int n, int tooth, bool final_visit) {
  const int e = n - tooth;
  const int cap = e >= 30 ? (1 << 30) : (1 << e);
  const int k = n_r < cap ? n_r : cap;
  return final_visit ? 3 * k : k;
}

// Restriction pass: level l-1 -> level l (Eqs. 3-4 at distance 2^(l-1) h), even images.
template <typename T, int DIM>
__device__ void phase_restrict(const KernelParams& p, int l) {
  T* R = (T*)p.R;
  for_tiles(p, l, [&](int b, long long local) {
    const ProblemDesc& P = p.probs[b];
    if (l > P.n - 1 || p.accum[b].done) return;
    const int Nt = level_side(P.n, l), Ns = level_side(P.n, l - 1);
    if (local >= level_nodes<DIM>(Nt)) return;
    int i, j, k;
    decode<DIM>(local, Nt, i, j, k);
    const T* src = R + P.off_lvl[l - 1];
    T acc = (T)0;
#pragma unroll
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz) {
      const int kk = DIM == 3 ? refl(2 * k + dz, Ns) : 0;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int jj = refl(2 * j + dy, Ns);
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int ii = refl(2 * i + dx, Ns);
          const T w = (T)((dx ? 0.25 : 0.5) * (dy ? 0.25 : 0.5) * (DIM == 3 ? (dz ? 0.25 : 0.5) : 1.0));
          acc += w * src[lin<DIM>(ii, jj, kk, Ns)];
        }
      }
    }
    R[P.off_lvl[l] + local] = acc;
  });
}

// One Jacobi sweep of the pseudo-time equation at level l (Eq. 2, explicit Euler, local step):
//   e_new = e + dtau (delta L_l e - r_l)
//         = (1 - omega) e_i + q_i (sigma_i CS(e) + CS(sigma e) - r_i / c),  c = kappa / (2 H^2),
// with CS(v) = sum_o w_o v_{i+o} over the level-l neighbours, q_i = dtau_i c and
// omega = dtau_i D_i (constant for the Jacobi-scaled step).  The last sweep of a cycle adds its
// result, unscaled, to the FP64 solution instead of storing it.
template <typename T, int DIM>
__device__ void phase_sweep(const KernelParams& p, const Phase& ph, int c) {
  T* E = (T*)p.E;
  T* E2 = (T*)p.E2;
  const T* R = (const T*)p.R;
  const T* SG = (const T*)p.SIG;
  const T* Q = (const T*)p.Q;
  const int l = ph.level;
  const bool final_visit = (ph.flags & kFinalVisit) != 0;
  const T one_m_omega = (T)(1.0 - p.omega);
  const T w_e = (T)p.w_edge, w_c = (T)p.w_corner;
  for_tiles(p, l, [&](int b, long long local) {
    const ProblemDesc& P = p.probs[b];
    if (ph.tooth > P.n - 1 || p.accum[b].done) return;
    const int k_b = visit_sweeps(p.n_r, P.n, ph.tooth, final_visit);
    if (ph.sweep >= k_b) return;
    const int N = level_side(P.n, l);
    if (local >= level_nodes<DIM>(N)) return;
    int i, j, k;
    decode<DIM>(local, N, i, j, k);
    const bool zero_in = ph.sweep == 0 && (ph.flags & kFirstOfTooth) && ph.tooth == P.n - 1;
    const bool last = final_visit && ph.sweep == k_b - 1;
    const long long off = P.off_lvl[l];
    const T* src = (ph.sweep & 1) ? E2 + off : E + off;
    T* dst = (ph.sweep & 1) ? E + off : E2 + off;
    if (is_fixed<DIM>(P, N, i, j, k)) {
      if (!last) dst[local] = (T)0;
      return;
    }
    const double H = P.h * (double)(1 << l);
    const T inv_c = (T)(2.0 * H * H / p.kappa);
    T e_c = (T)0, cs_e[3] = {(T)0, (T)0, (T)0}, cs_se[3] = {(T)0, (T)0, (T)0};
    const T* sg = SG + off;
    if (!zero_in) {
      e_c = src[local];
#pragma unroll
      for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz) {
        const int kk = DIM == 3 ? refl(k + dz, N) : 0;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          const int jj = refl(j + dy, N);
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0 && dz == 0) continue;
            const int nz = (dx != 0) + (dy != 0) + (dz != 0);
            const int o = lin<DIM>(refl(i + dx, N), jj, kk, N);
            const T ev = src[o];
            cs_e[nz - 1] += ev;
            if (P.hetero) cs_se[nz - 1] += sg[o] * ev;
          }
        }
      }
    }
    const T CSe = cs_e[0] + w_e * cs_e[1] + (DIM == 3 ? w_c * cs_e[2] : (T)0);
    const T r_i = R[off + local];
    T e_new;
    if (P.hetero) {
      const T CSse = cs_se[0] + w_e * cs_se[1] + (DIM == 3 ? w_c * cs_se[2] : (T)0);
      e_new = one_m_omega * e_c + Q[off + local] * (sg[local] * CSe + CSse - r_i * inv_c);
    } else {
      e_new = one_m_omega * e_c + (T)P.q_const[l] * ((T)2 * CSe - r_i * inv_c);
    }
    if (last) {
      p.U[P.off_full + local] += (double)e_new / p.state[b].scale_used[c & 1];
    } else {
      dst[local] = e_new;
    }
  });
}

// Buffer holding the result of a visit of tooth `tooth` at a level (E if the visit did an even
// number of sweeps, E2 otherwise).
template <typename T>
__device__ __forceinline__ T* visit_result(const KernelParams& p, const ProblemDesc& P, int tooth, int l) {
  const int k = visit_sweeps(p.n_r, P.n, tooth, false);
  return ((k & 1) ? (T*)p.E2 : (T*)p.E) + P.off_lvl[l];
}

// Moving one level finer: E_l (+)= I(E_{l+1} - B_{l+1}) on every level-l node (hat-function
// interpolation, Algorithm 2's I_lambda, between consecutive levels).
template <typename T, int DIM>
__device__ void phase_prolong(const KernelParams& p, const Phase& ph) {
  const int l = ph.level;
  const bool init = (ph.flags & kInit) != 0;
  const T* B = (const T*)p.B;
  for_tiles(p, l, [&](int b, long long local) {
    const ProblemDesc& P = p.probs[b];
    if (ph.tooth > P.n - 1 || p.accum[b].done) return;
    const int N = level_side(P.n, l), Nc = level_side(P.n, l + 1);
    if (local >= level_nodes<DIM>(N)) return;
    int i, j, k;
    decode<DIM>(local, N, i, j, k);
    T* El = (T*)p.E + P.off_lvl[l];
    if (is_fixed<DIM>(P, N, i, j, k)) {
      El[local] = (T)0;
      return;
    }
    const T* src = visit_result<T>(p, P, ph.tooth, l + 1);
    const T* Bc = B + P.off_lvl[l + 1];
    const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
    const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (DIM == 3 && (k & 1)) ? 2 : 1;
    const T half = (T)0.5;
    T val = (T)0;
    for (int cz = 0; cz < nk; ++cz)
      for (int cy = 0; cy < nj; ++cy)
        for (int cx = 0; cx < ni; ++cx) {
          const int o = lin<DIM>(i0 + cx, j0 + cy, DIM == 3 ? k0 + cz : 0, Nc);
          const T w = (ni == 2 ? half : (T)1) * (nj == 2 ? half : (T)1) * (nk == 2 ? half : (T)1);
          const T d = init ? src[o] : src[o] - Bc[o];
          val += w * d;
        }
    const T base = init ? (T)0 : visit_result<T>(p, P, ph.prev_tooth, l)[local];
    El[local] = base + val;
  });
}

// Moving one level coarser: E_{l} = B_{l} = (result at level l-1) on the level-l subset.
template <typename T, int DIM>
__device__ void phase_inject(const KernelParams& p, const Phase& ph) {
  const int l = ph.level;
  for_tiles(p, l, [&](int b, long long local) {
    const ProblemDesc& P = p.probs[b];
    if (ph.tooth > P.n - 1 || l > P.n - 1 || p.accum[b].done) return;
    const int N = level_side(P.n, l), Nf = level_side(P.n, l - 1);
    if (local >= level_nodes<DIM>(N)) return;
    int i, j, k;
    decode<DIM>(local, N, i, j, k);
    const T* src = visit_result<T>(p, P, ph.tooth, l - 1);
    const T v = src[lin<DIM>(2 * i, 2 * j, 2 * k, Nf)];
    ((T*)p.E)[P.off_lvl[l] + local] = v;
    ((T*)p.B)[P.off_lvl[l] + local] = v;
  });
}

// ---------------------------------------------------------------------------------------------
// The persistent cycle kernel
// ---------------------------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(1024) cycle_kernel(const KernelParams p) {
  if (p.fresh) {
    phase_lift<T, DIM>(p);
    if (!grid_sync(p.sync, p.timeout_ns)) return;
  }
  for (int c = 0;; ++c) {
    phase_outer<T, DIM>(p, c);
    if (!grid_sync(p.sync, p.timeout_ns)) return;
    if (blockIdx.x == 0) phase_check<T, DIM>(p, c);
    if (!grid_sync(p.sync, p.timeout_ns)) return;
    if (!ld_volatile(&p.sync->active[c & 1])) break;
    for (int q = 0; q < p.nphases; ++q) {
      const Phase ph = p.phases[q];
      switch (ph.op) {
        case OP_RESTRICT: phase_restrict<T, DIM>(p, ph.level); break;
        case OP_SWEEP: phase_sweep<T, DIM>(p, ph, c); break;
        case OP_PROLONG: phase_prolong<T, DIM>(p, ph); break;
        default: phase_inject<T, DIM>(p, ph); break;
      }
      if (!grid_sync(p.sync, p.timeout_ns)) return;
    }
  }
}

template <typename T, int DIM>
static void* cycle_fn() {
  return (void*)cycle_kernel<T, DIM>;
}

static void* pick_cycle(int mixed, int dim) {
  if (mixed) return dim == 3 ? cycle_fn<float, 3>() : cycle_fn<float, 2>();
  return dim == 3 ? cycle_fn<double, 3>() : cycle_fn<double, 2>();
}

cudaError_t launch_cycle_kernel(const KernelParams& p, int mixed, int dim, int blocks, int threads,
                                cudaStream_t s) {
  void* args[] = {(void*)&p};
  return cudaLaunchCooperativeKernel(pick_cycle(mixed, dim), dim3(blocks), dim3(threads), args, 0, s);
}

int cycle_kernel_occupancy(int mixed, int dim, int threads, int* blocks_per_sm) {
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, pick_cycle(mixed, dim), threads, 0);
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
                                   T* __restrict__ SIG, T* __restrict__ Q) {
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
                               void* Q_T, cudaStream_t s) {
  const int N = (1 << (P.n - l)) + 1;
  const long long M = dim == 3 ? (long long)N * N * N : (long long)N * N;
  const long long off = P.off_lvl[l];
  if (mixed) {
    float* S = (float*)SIG_T + off;
    float* Q = (float*)Q_T + off;
    if (dim == 3) setup_level_kernel<float, 3><<<grid_for(M), 256, 0, s>>>(P, l, sig, a, kappa, w_edge, w_corner, theta_gain, S, Q);
    else setup_level_kernel<float, 2><<<grid_for(M), 256, 0, s>>>(P, l, sig, a, kappa, w_edge, w_corner, theta_gain, S, Q);
  } else {
    double* S = (double*)SIG_T + off;
    double* Q = (double*)Q_T + off;
    if (dim == 3) setup_level_kernel<double, 3><<<grid_for(M), 256, 0, s>>>(P, l, sig, a, kappa, w_edge, w_corner, theta_gain, S, Q);
    else setup_level_kernel<double, 2><<<grid_for(M), 256, 0, s>>>(P, l, sig, a, kappa, w_edge, w_corner, theta_gain, S, Q);
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

cudaError_t launch_fill(double* dst, long long n, double v, cudaStream_t s) {
  fill_kernel<<<grid_for(n), 256, 0, s>>>(dst, n, v);
  return cudaGetLastError();
}

}  // namespace sgml
