// bm_rhs_plane_wave_noalloc: the plane-wave right-hand side without any device allocation.
//
// bm_rhs_plane_wave copies the incident directions into a buffer it allocates with cudaMalloc on every
// call. Some callers cannot allocate device memory when they need a right-hand side: code running inside
// a memory pool or allocator callback, codes that forbid allocation after start-up (real-time or
// certified runs), or code that has handed the whole device to another allocator. This variant keeps the
// directions in a fixed file-scope device array instead.
//
// Contract (see include/fdbem.h):
//  - at most FDA_RHS_NOALLOC_MAX directions per call; larger requests fail with FDA_E_INVALID_ARG;
//  - the array lives in every GPU that loads the library until the process exits;
//  - the first call on a device looks up the array's device address for that device (set-up); make that
//    first call before any stream capture;
//  - every call shares the one array, which keeps the previous call's directions: calls that overlap on
//    the GPU (different streams, no ordering between them) race on it.
#include <mutex>

#include "internal.cuh"

#define FDA_RHS_NOALLOC_MAX 1024
#define FDA_RHS_NOALLOC_DEVICES 64

// Fixed scratch: nrhs x 3 directions (doubles). Every call overwrites the entries it uses, so nothing in
// it has to start at zero.
static __device__ __align__(256) double g_rhs_dirs[3 * FDA_RHS_NOALLOC_MAX];

static double* g_rhs_dirs_addr[FDA_RHS_NOALLOC_DEVICES] = {nullptr};
static std::mutex g_rhs_mu;

// Device address of g_rhs_dirs on the current device (looked up once per device, with it current).
static int rhs_scratch_address(double** out) {
  int dev = 0;
  FDA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= FDA_RHS_NOALLOC_DEVICES) {
    fda::set_error("device %d beyond the %d devices bm_rhs_plane_wave_noalloc supports", dev, FDA_RHS_NOALLOC_DEVICES);
    return FDA_E_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_rhs_mu);
  if (!g_rhs_dirs_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_dirs);
    if (e != cudaSuccess || !p) {
      fda::set_error("cudaGetSymbolAddress(g_rhs_dirs) failed: %s", cudaGetErrorString(e));
      return FDA_E_CUDA;
    }
    g_rhs_dirs_addr[dev] = (double*)p;
  }
  *out = g_rhs_dirs_addr[dev];
  return FDA_OK;
}

// b = u_inc + alpha du_inc/dn_x, u_inc = exp(i k d.x), d normalised here (same arithmetic as
// bm_rhs_plane_wave, which normalises on the host before copying).
static __global__ void k_plane_wave_fixed(const double* x, const double* n, int64_t N, const double* dirs,
                                          int nrhs, double k, double2 alpha, double2* b) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N * nrhs) return;
  int r = (int)(q / N);
  int64_t i = q - (int64_t)r * N;
  double d0 = dirs[3 * r], d1 = dirs[3 * r + 1], d2 = dirs[3 * r + 2];
  double l = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  d0 /= l;
  d1 /= l;
  d2 /= l;
  double ph = k * (d0 * x[3 * i] + d1 * x[3 * i + 1] + d2 * x[3 * i + 2]);
  double sn, cs;
  sincos(ph, &sn, &cs);
  double2 u = make_double2(cs, sn);
  double dn = d0 * n[3 * i] + d1 * n[3 * i + 1] + d2 * n[3 * i + 2];
  double2 dudn = cmul(make_double2(0, k * dn), u);
  b[q] = cadd(u, cmul(alpha, dudn));
}

extern "C" int bm_rhs_plane_wave_noalloc(const bm_problem_t* prob, const double* dirs, int nrhs, void* b_dev,
                                         void* stream) {
  if (!prob || !dirs || !b_dev) {
    fda::set_error("NULL argument");
    return FDA_E_INVALID_ARG;
  }
  if (nrhs < 1 || nrhs > FDA_RHS_NOALLOC_MAX) {
    fda::set_error("bm_rhs_plane_wave_noalloc takes 1..%d directions (got %d); use bm_rhs_plane_wave for more",
                   FDA_RHS_NOALLOC_MAX, nrhs);
    return FDA_E_INVALID_ARG;
  }
  for (int r = 0; r < nrhs; ++r) {
    double l = dirs[3 * r] * dirs[3 * r] + dirs[3 * r + 1] * dirs[3 * r + 1] + dirs[3 * r + 2] * dirs[3 * r + 2];
    if (!(l > 0) || !std::isfinite(l)) {
      fda::set_error("direction %d has zero or non-finite length", r);
      return FDA_E_INVALID_ARG;
    }
  }
  double* scratch = nullptr;
  FDA_TRY(rhs_scratch_address(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  FDA_CUDA(cudaMemcpyAsync(scratch, dirs, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, s));
  k_plane_wave_fixed<<<fda::cdiv(prob->N * nrhs, 256), 256, 0, s>>>(prob->x.p, prob->n.p, prob->N, scratch, nrhs,
                                                                    prob->k, prob->alpha, (double2*)b_dev);
  FDA_LAUNCH_CHECK();
  FDA_CUDA(cudaStreamSynchronize(s));
  return FDA_OK;
}
