// Shared helpers of the FDA Burton-Miller library: complex arithmetic for double2/float2,
// CUDA error plumbing, a thread-local last-error string, and device buffers owned by handles.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include <math.h>
#include <string>
#include <vector>

#include "../../include/fdbem.h"

#define FDA_PI 3.14159265358979323846

namespace fda {

void set_error(const char* fmt, ...);
const char* last_error();

// --- error plumbing: every host function returns an int status; nothing throws across the ABI ---
#define FDA_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      fda::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));   \
      return e_ == cudaErrorMemoryAllocation ? FDA_E_OOM : FDA_E_CUDA;                      \
    }                                                                                       \
  } while (0)

#define FDA_TRY(expr)      \
  do {                     \
    int rc_ = (expr);      \
    if (rc_ != FDA_OK) return rc_; \
  } while (0)

#define FDA_LAUNCH_CHECK() FDA_CUDA(cudaGetLastError())

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// --- device buffer owned by a handle (freed with the handle) ---
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  int alloc(size_t count) {
    release();
    if (count == 0) return FDA_OK;
    cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      set_error("cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
      return FDA_E_OOM;
    }
    n = count;
    return FDA_OK;
  }
  int zero(cudaStream_t s = 0) {
    if (p && n) FDA_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    return FDA_OK;
  }
  int upload(const T* h, size_t count) {
    FDA_TRY(alloc(count));
    if (count) FDA_CUDA(cudaMemcpy(p, h, count * sizeof(T), cudaMemcpyHostToDevice));
    return FDA_OK;
  }
  int upload(const std::vector<T>& v) { return upload(v.data(), v.size()); }
  int download(std::vector<T>& v) const {
    v.resize(n);
    if (n) FDA_CUDA(cudaMemcpy(v.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost));
    return FDA_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
  ~DBuf() { release(); }
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
};

}  // namespace fda

// --- complex arithmetic (interleaved re, im) ---
template <typename R> struct cpx_t;
template <> struct cpx_t<double> { typedef double2 type; };
template <> struct cpx_t<float> { typedef float2 type; };

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cjmul(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cjmul(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc += a * b
__host__ __device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
__host__ __device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
// acc += conj(a) * b
__host__ __device__ __forceinline__ void cjfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
__host__ __device__ __forceinline__ void cjfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 conjc(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 conjc(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ double2 to_d(double2 a) { return a; }
__device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
template <typename C> __device__ __forceinline__ C from_d(double2 a);
template <> __device__ __forceinline__ double2 from_d<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

__device__ __forceinline__ void atomic_cadd(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}
__device__ __forceinline__ void atomic_cadd(float2* p, float2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_csum(double2 v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}
__device__ __forceinline__ float2 warp_csum(float2 v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}

// Helmholtz kernel pieces (Eq. fundsol and the layer operators). r = x - y.
// Returns G and fills dG/dn_y, dG/dn_x, d2G/dn_x dn_y as requested.
struct KernVals {
  double2 G, Dy, Dx, H;
};

__device__ __forceinline__ KernVals helmholtz4(const double* x, const double* nx, const double* y, const double* ny,
                                               double k) {
  double r0 = x[0] - y[0], r1 = x[1] - y[1], r2 = x[2] - y[2];
  double R2 = r0 * r0 + r1 * r1 + r2 * r2;
  double R = sqrt(R2);
  double iR = 1.0 / R;
  double sn, cs;
  sincos(k * R, &sn, &cs);
  double g = iR * (0.25 / FDA_PI);
  double2 G = make_double2(g * cs, g * sn);
  double rnx = (r0 * nx[0] + r1 * nx[1] + r2 * nx[2]) * iR;
  double rny = (r0 * ny[0] + r1 * ny[1] + r2 * ny[2]) * iR;
  double nxny = nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2];
  KernVals o;
  o.G = G;
  // dG/dn_y = G (1/R - ik) rny
  o.Dy = cscale(cmul(G, make_double2(iR, -k)), rny);
  // dG/dn_x = G (ik - 1/R) rnx
  o.Dx = cscale(cmul(G, make_double2(-iR, k)), rnx);
  // d2G = G/R^2 [ nxny (1 - ikR) - rnx rny (3 - 3ikR - k^2R^2) ]
  double kR = k * R;
  double2 t = make_double2(nxny - rnx * rny * (3.0 - kR * kR), -nxny * kR + rnx * rny * 3.0 * kR);
  o.H = cscale(cmul(G, t), iR * iR);
  return o;
}
