// sgml_post.cu -- post-processing of the vortex application (Sec. 3.3): the velocity v = curl psi
// of a solved stream vector potential (Eq. 14) and streamlines of v; and the grid motion of the
// grid-deformation application (Sec. 3.2, Eq. 11).
//
// The paper leaves curl and streamlines to its visualisation tool.  Readings: second-order central differences at
// interior nodes, second-order one-sided differences (-3 f0 + 4 f1 - f2) / (2h) on the faces;
// streamlines by the classical fourth-order Runge-Kutta method with a fixed step, the velocity
// interpolated trilinearly between nodes, a path ending when a stage point or its next position
// leaves the unit cube.  Grid motion: read as in the header (forward Euler over nsteps equal steps
// of pseudo-time, central differences with Neumann images, multilinear interpolation, trapezoid
// integral of f, coordinates clamped to the unit square / cube).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "sgml.h"

namespace {

thread_local std::string g_post_error;

int post_fail(int code, const std::string& msg) {
  g_post_error = msg;
  return code;
}

// d f / d x_axis at node (i, j, k) of an N^3 array (axis 0: x, 1: y, 2: z).
__device__ __forceinline__ double deriv(const double* __restrict__ f, int N, double inv2h, int i, int j, int k,
                                        int axis) {
  const long long sx = 1, sy = N, sz = (long long)N * N;
  const long long c = (long long)k * sz + (long long)j * sy + i;
  const int m = axis == 0 ? i : (axis == 1 ? j : k);
  const long long s = axis == 0 ? sx : (axis == 1 ? sy : sz);
  if (m == 0) return (-3.0 * f[c] + 4.0 * f[c + s] - f[c + 2 * s]) * inv2h;
  if (m == N - 1) return (3.0 * f[c] - 4.0 * f[c - s] + f[c - 2 * s]) * inv2h;
  return (f[c + s] - f[c - s]) * inv2h;
}

// Nodes on the faces of the cube (2 N^2 + 4 (N - 1)(N - 2) of them), one thread each: one-sided
// differences where a neighbour is missing.  Face index t: the planes z = 0 and z = N - 1 first,
// then, plane by plane, the ring of each inner plane.
__global__ void curl_faces_kernel(int N, double inv2h, const double* __restrict__ psi, double* __restrict__ v) {
  const long long NN = (long long)N * N, ring = 4LL * (N - 1), total = 2 * NN + (long long)(N - 2) * ring;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= total) return;
  int i, j, k;
  if (t < 2 * NN) {
    k = t < NN ? 0 : N - 1;
    const long long r = t % NN;
    j = (int)(r / N);
    i = (int)(r % N);
  } else {
    const long long r = t - 2 * NN;
    k = 1 + (int)(r / ring);
    const int q = (int)(r % ring);  // ring position: y = 0 row, y = N - 1 row, then x = 0 / x = N - 1 columns
    if (q < N) {
      j = 0, i = q;
    } else if (q < 2 * N) {
      j = N - 1, i = q - N;
    } else {
      const int m = q - 2 * N;  // 0 .. 2 (N - 2) - 1
      j = 1 + m / 2;
      i = (m & 1) ? N - 1 : 0;
    }
  }
  const long long M = NN * N;
  const double* px = psi;
  const double* py = psi + M;
  const double* pz = psi + 2 * M;
  const long long c = ((long long)k * N + j) * N + i;
  v[c] = deriv(pz, N, inv2h, i, j, k, 1) - deriv(py, N, inv2h, i, j, k, 2);
  v[M + c] = deriv(px, N, inv2h, i, j, k, 2) - deriv(pz, N, inv2h, i, j, k, 0);
  v[2 * M + c] = deriv(py, N, inv2h, i, j, k, 0) - deriv(px, N, inv2h, i, j, k, 1);
}

// Inner nodes (1 <= i, j, k <= N - 2): one thread per (x, y) column of a z-chunk, a block of 32 x 8
// columns; the thread walks its chunk in z keeping psi_x and psi_y of planes k - 1, k, k + 1 in
// registers (their z derivatives), while the x and y derivatives read the neighbouring columns,
// which the block's other threads load in the same plane step (L1 hits).  GB300's FP64 pipe bounds
// this kernel, so a node takes 12 FP64 instructions: each component is the difference of two
// central differences, scaled once, ((f_a(+) - f_a(-)) - (f_b(+) - f_b(-))) / 2h; the faces are a
// kernel of their own, so no warp carries their one-sided arithmetic.
constexpr int kCurlBX = 32, kCurlBY = 8;

__global__ void __launch_bounds__(kCurlBX * kCurlBY) curl_kernel(int N, int zlen, double inv2h,
                                                                 const double* __restrict__ psi,
                                                                 double* __restrict__ v) {
  const int i = 1 + blockIdx.x * kCurlBX + threadIdx.x, j = 1 + blockIdx.y * kCurlBY + threadIdx.y;
  const int k0 = 1 + blockIdx.z * zlen, k1 = min(N - 1, k0 + zlen);
  if (i >= N - 1 || j >= N - 1 || k0 >= k1) return;
  const long long M = (long long)N * N * N, NN = (long long)N * N;
  const double* px = psi;
  const double* py = psi + M;
  const double* pz = psi + 2 * M;
  const long long col = (long long)j * N + i;
  double xm = px[(k0 - 1) * NN + col], x0 = px[k0 * NN + col];  // psi_x, psi_y at planes k - 1, k
  double ym = py[(k0 - 1) * NN + col], y0 = py[k0 * NN + col];
  for (int k = k0; k < k1; ++k) {
    const long long c = k * NN + col;
    const double xp = px[c + NN], yp = py[c + NN];
    v[c] = ((pz[c + N] - pz[c - N]) - (yp - ym)) * inv2h;
    v[M + c] = ((xp - xm) - (pz[c + 1] - pz[c - 1])) * inv2h;
    v[2 * M + c] = ((py[c + 1] - py[c - 1]) - (px[c + N] - px[c - N])) * inv2h;
    xm = x0, x0 = xp, ym = y0, y0 = yp;
  }
}

__device__ __forceinline__ bool inside(const double x[3]) {
  return x[0] >= 0.0 && x[0] <= 1.0 && x[1] >= 0.0 && x[1] <= 1.0 && x[2] >= 0.0 && x[2] <= 1.0;
}

__device__ void interp(const double* __restrict__ v, int N, const double x[3], double out[3]) {
  const long long M = (long long)N * N * N;
  const double s = (double)(N - 1);
  int i0[3];
  double t[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double g = x[a] * s;
    int i = (int)floor(g);
    i = i < 0 ? 0 : (i > N - 2 ? N - 2 : i);
    i0[a] = i;
    t[a] = g - (double)i;
  }
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    const double* f = v + comp * M;
    double acc = 0.0;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);
          acc += w * f[((long long)(i0[2] + dz) * N + (i0[1] + dy)) * N + (i0[0] + dx)];
        }
    out[comp] = acc;
  }
}

// One thread per seed: streamlines are independent.
__global__ void streamline_kernel(int N, const double* __restrict__ v, const double* __restrict__ seeds, int nseeds,
                                  double dt, int nsteps, double* __restrict__ paths, int* __restrict__ lengths) {
  const int sd = blockIdx.x * blockDim.x + threadIdx.x;
  if (sd >= nseeds) return;
  double x[3] = {seeds[3 * sd], seeds[3 * sd + 1], seeds[3 * sd + 2]};
  double* out = paths + (long long)sd * (nsteps + 1) * 3;
  int len = 0;
  if (inside(x)) {
    out[0] = x[0], out[1] = x[1], out[2] = x[2];
    len = 1;
    for (int st = 0; st < nsteps; ++st) {
      double k1[3], k2[3], k3[3], k4[3], y[3], xn[3];
      interp(v, N, x, k1);
#pragma unroll
      for (int a = 0; a < 3; ++a) y[a] = x[a] + 0.5 * dt * k1[a];
      if (!inside(y)) break;
      interp(v, N, y, k2);
#pragma unroll
      for (int a = 0; a < 3; ++a) y[a] = x[a] + 0.5 * dt * k2[a];
      if (!inside(y)) break;
      interp(v, N, y, k3);
#pragma unroll
      for (int a = 0; a < 3; ++a) y[a] = x[a] + dt * k3[a];
      if (!inside(y)) break;
      interp(v, N, y, k4);
#pragma unroll
      for (int a = 0; a < 3; ++a) xn[a] = x[a] + dt / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
      if (!inside(xn)) break;
#pragma unroll
      for (int a = 0; a < 3; ++a) x[a] = xn[a], out[3 * len + a] = xn[a];
      ++len;
    }
  }
  lengths[sd] = len;
}

// ---- Grid motion of the grid-deformation application (Sec. 3.2, Eq. 11) ----------------------
// Trapezoid-rule integral over the unit square / cube and minimum of the node field f: per-block
// partials (grid-stride over the nodes, warp shuffles, one shared slot per warp), folded in a
// fixed order by one block.
constexpr int kRedThreads = 256;

__device__ __forceinline__ void block_fold(double& s, double& m, double* sh_s, double* sh_m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh_s[w] = s, sh_m[w] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    s = sh_s[0], m = sh_m[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) s += sh_s[k], m = fmin(m, sh_m[k]);
  }
}

__global__ void __launch_bounds__(kRedThreads) integral_partial_kernel(int dim, int N, long long M,
                                                                       const double* __restrict__ f,
                                                                       double* __restrict__ part) {
  __shared__ double sh_s[kRedThreads / 32], sh_m[kRedThreads / 32];
  const double h = 1.0 / (double)(N - 1);
  double s = 0.0, m = INFINITY;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    long long r = i;
    double w = 1.0;
    for (int a = 0; a < dim; ++a) {
      const int c = (int)(r % N);
      r /= N;
      w *= (c == 0 || c == N - 1) ? 0.5 * h : h;
    }
    const double v = f[i];
    s += w * v;
    m = fmin(m, v);
  }
  block_fold(s, m, sh_s, sh_m);
  if (threadIdx.x == 0) part[2 * blockIdx.x] = s, part[2 * blockIdx.x + 1] = m;
}

__global__ void __launch_bounds__(kRedThreads) integral_finish_kernel(int nparts, const double* __restrict__ part,
                                                                      double* __restrict__ out) {
  __shared__ double sh_s[kRedThreads / 32], sh_m[kRedThreads / 32];
  double s = 0.0, m = INFINITY;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) s += part[2 * k], m = fmin(m, part[2 * k + 1]);
  block_fold(s, m, sh_s, sh_m);
  if (threadIdx.x == 0) out[0] = s, out[1] = m;
}

// d u / d x_a at node c by central differences with the Neumann images u(-1) = u(1), u(N) = u(N-2).
template <int DIM>
__device__ __forceinline__ double neumann_deriv(const double* __restrict__ u, int N, double two_h, const int c[DIM],
                                                int a) {
  long long stride = 1, base = 0;
  for (int b = DIM - 1; b >= 0; --b) base = base * N + c[b];
  for (int b = 0; b < a; ++b) stride *= N;
  const int up = c[a] + 1 > N - 1 ? N - 2 : c[a] + 1;
  const int dn = c[a] - 1 < 0 ? 1 : c[a] - 1;
  return (__ldg(u + base + (long long)(up - c[a]) * stride) - __ldg(u + base + (long long)(dn - c[a]) * stride)) /
         two_h;
}

// One thread per node: nsteps forward-Euler steps of dx/dt = -grad u / (t f + F), grad u and f
// interpolated multilinearly from the node values of the cell holding the moving node (the node
// values of grad u formed on the fly from u), every coordinate clamped to [0, 1].
template <int DIM>
__global__ void __launch_bounds__(256) grid_motion_kernel(int N, long long M, const double* __restrict__ u,
                                                          const double* __restrict__ f, double F, double t0,
                                                          double dt, int nsteps, double* __restrict__ x) {
  const double h = 1.0 / (double)(N - 1);
  const double two_h = 2.0 * h;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    double p[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) p[a] = fmin(fmax(x[a * M + i], 0.0), 1.0);
    for (int k = 0; k < nsteps; ++k) {
      const double t = t0 + (double)k * dt;
      int i0[DIM];
      double w[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const double g = p[a] * (double)(N - 1);
        int c = (int)floor(g);
        c = c < 0 ? 0 : (c > N - 2 ? N - 2 : c);
        i0[a] = c;
        w[a] = g - (double)c;
      }
      double fi = 0.0, gi[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) gi[a] = 0.0;
#pragma unroll
      for (int corner = 0; corner < (1 << DIM); ++corner) {
        int c[DIM];
        double wt = 1.0;
        long long idx = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const int up = (corner >> a) & 1;
          c[a] = i0[a] + up;
          wt *= up ? w[a] : 1.0 - w[a];
        }
#pragma unroll
        for (int a = DIM - 1; a >= 0; --a) idx = idx * N + c[a];
        fi += wt * __ldg(f + idx);
#pragma unroll
        for (int a = 0; a < DIM; ++a) gi[a] += wt * neumann_deriv<DIM>(u, N, two_h, c, a);
      }
      const double den = t * fi + F;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const double v = -gi[a] / den;
        p[a] = fmin(fmax(p[a] + dt * v, 0.0), 1.0);
      }
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a * M + i] = p[a];
  }
}

bool device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int sgml_curl(int n, const double* psi, double* v, void* cuda_stream) {
  if (n < 1 || n > 10) return post_fail(SGML_ERR_ARG, "n must be in 1..10");
  if (!psi || !v || psi == v) return post_fail(SGML_ERR_ARG, "psi and v must be distinct non-NULL arrays");
  if (!device_pointer(psi) || !device_pointer(v)) return post_fail(SGML_ERR_ARG, "psi and v must be device arrays");
  const int N = (1 << n) + 1;
  const double h = 1.0 / (double)(N - 1);
  // inner nodes in z-chunks: enough blocks for several waves of the GPU, chunks as long as that allows
  const int Ni = N - 2;  // inner nodes per side (N >= 3)
  const int bx = (Ni + kCurlBX - 1) / kCurlBX, by = (Ni + kCurlBY - 1) / kCurlBY;
  const int chunks = std::min(Ni, std::max(1, (4096 + bx * by - 1) / (bx * by)));
  const int zlen = (Ni + chunks - 1) / chunks;
  const dim3 grid((unsigned)bx, (unsigned)by, (unsigned)((Ni + zlen - 1) / zlen));
  const double inv2h = 1.0 / (2.0 * h);
  curl_kernel<<<grid, dim3(kCurlBX, kCurlBY), 0, (cudaStream_t)cuda_stream>>>(N, zlen, inv2h, psi, v);
  const long long faces = 2LL * N * N + 4LL * (N - 1) * (N - 2);
  curl_faces_kernel<<<(unsigned)((faces + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(N, inv2h, psi, v);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SGML_OK : post_fail(SGML_ERR_CUDA, cudaGetErrorString(e));
}

int sgml_streamlines(int n, const double* v, const double* seeds, int nseeds, double dt, int nsteps, double* paths,
                     int* lengths, void* cuda_stream) {
  if (n < 1 || n > 10) return post_fail(SGML_ERR_ARG, "n must be in 1..10");
  if (nseeds < 0 || nsteps < 0 || !(dt > 0.0)) return post_fail(SGML_ERR_ARG, "nseeds, nsteps >= 0 and dt > 0");
  if (nseeds == 0) return SGML_OK;
  if (!v || !seeds || !paths || !lengths) return post_fail(SGML_ERR_ARG, "NULL array");
  if (!device_pointer(v) || !device_pointer(seeds) || !device_pointer(paths) || !device_pointer(lengths))
    return post_fail(SGML_ERR_ARG, "v, seeds, paths and lengths must be device arrays");
  const int N = (1 << n) + 1;
  streamline_kernel<<<(nseeds + 127) / 128, 128, 0, (cudaStream_t)cuda_stream>>>(N, v, seeds, nseeds, dt, nsteps,
                                                                                 paths, lengths);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SGML_OK : post_fail(SGML_ERR_CUDA, cudaGetErrorString(e));
}

int sgml_grid_motion(int dim, int n, const double* u, const double* f, double t0, double t1, int nsteps, double* x,
                     void* cuda_stream) {
  if (dim != 2 && dim != 3) return post_fail(SGML_ERR_ARG, "dim must be 2 or 3");
  if (n < 1 || n > (dim == 2 ? 14 : 10)) return post_fail(SGML_ERR_ARG, "n must be in 1..14 (2-D) or 1..10 (3-D)");
  if (!(t0 >= 0.0) || !(t1 >= t0) || nsteps < 0) return post_fail(SGML_ERR_ARG, "need 0 <= t0 <= t1 and nsteps >= 0");
  if (!u || !f || !x) return post_fail(SGML_ERR_ARG, "NULL array");
  if ((const void*)x == (const void*)u || (const void*)x == (const void*)f)
    return post_fail(SGML_ERR_ARG, "x must not alias u or f");
  if (!device_pointer(u) || !device_pointer(f) || !device_pointer(x))
    return post_fail(SGML_ERR_ARG, "u, f and x must be device arrays");
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  const int N = (1 << n) + 1;
  long long M = 1;
  for (int a = 0; a < dim; ++a) M *= N;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (M + kRedThreads - 1) / kRedThreads;
  const int parts = (int)(want < 4LL * sms ? want : 4LL * sms);
  double* scratch = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&scratch, sizeof(double) * (2 * (size_t)parts + 2), s);
  if (e != cudaSuccess) return post_fail(SGML_ERR_CUDA, cudaGetErrorString(e));
  integral_partial_kernel<<<parts, kRedThreads, 0, s>>>(dim, N, M, f, scratch);
  integral_finish_kernel<<<1, kRedThreads, 0, s>>>(parts, scratch, scratch + 2 * parts);
  double Fm[2] = {0.0, 0.0};
  e = cudaMemcpyAsync(Fm, scratch + 2 * parts, sizeof(Fm), cudaMemcpyDeviceToHost, s);
  const cudaError_t e_sync = e == cudaSuccess ? cudaStreamSynchronize(s) : e;
  cudaFreeAsync(scratch, s);
  if (e_sync != cudaSuccess) return post_fail(SGML_ERR_CUDA, cudaGetErrorString(e_sync));
  const double F = Fm[0], fmin_v = Fm[1];
  // t f + F >= min(F, F + t1 min f) for an interpolated f inside the domain
  if (!(F > 0.0) || !(F + t1 * fmin_v > 0.0))
    return post_fail(SGML_ERR_ARG, "the velocity denominator t f + int f must stay positive (int f = " +
                                       std::to_string(F) + ", min f = " + std::to_string(fmin_v) + ")");
  const double dt = nsteps > 0 ? (t1 - t0) / (double)nsteps : 0.0;
  const long long blocks = (M + 255) / 256;
  if (dim == 2)
    grid_motion_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(N, M, u, f, F, t0, dt, nsteps, x);
  else
    grid_motion_kernel<3><<<(unsigned)blocks, 256, 0, s>>>(N, M, u, f, F, t0, dt, nsteps, x);
  e = cudaGetLastError();
  return e == cudaSuccess ? SGML_OK : post_fail(SGML_ERR_CUDA, cudaGetErrorString(e));
}

const char* sgml_post_last_error(void) { return g_post_error.c_str(); }

}  // extern "C"
