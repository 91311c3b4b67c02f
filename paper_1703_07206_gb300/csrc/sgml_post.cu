// sgml_post.cu -- post-processing of the vortex application (Sec. 3.3): the velocity v = curl psi
// of a solved stream vector potential (Eq. 14) and streamlines of v.
//
// The paper leaves both to its visualisation tool.  Readings: second-order central differences at
// interior nodes, second-order one-sided differences (-3 f0 + 4 f1 - f2) / (2h) on the faces;
// streamlines by the classical fourth-order Runge-Kutta method with a fixed step, the velocity
// interpolated trilinearly between nodes, a path ending when a stage point or its next position
// leaves the unit cube.
#include <cuda_runtime.h>

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

__global__ void curl_kernel(int N, double inv2h, const double* __restrict__ psi, double* __restrict__ v) {
  const long long M = (long long)N * N * N;
  const double* px = psi;
  const double* py = psi + M;
  const double* pz = psi + 2 * M;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < M; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % N), j = (int)((c / N) % N), k = (int)(c / ((long long)N * N));
    v[c] = deriv(pz, N, inv2h, i, j, k, 1) - deriv(py, N, inv2h, i, j, k, 2);
    v[M + c] = deriv(px, N, inv2h, i, j, k, 2) - deriv(pz, N, inv2h, i, j, k, 0);
    v[2 * M + c] = deriv(py, N, inv2h, i, j, k, 0) - deriv(px, N, inv2h, i, j, k, 1);
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
  const long long M = (long long)N * N * N;
  const double h = 1.0 / (double)(N - 1);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (M + 255) / 256;
  const int blocks = (int)(want < 8LL * sms ? want : 8LL * sms);
  curl_kernel<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(N, 1.0 / (2.0 * h), psi, v);
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

const char* sgml_post_last_error(void) { return g_post_error.c_str(); }

}  // extern "C"
