// bm_rhs_plane_wave_noalloc: the plane-wave right-hand side without any device allocation.
//
// bm_rhs_plane_wave copies the incident directions into a buffer it allocates with cudaMalloc on every
// call. Some callers may issue CUDA calls but must not allocate device memory when they need a
// right-hand side: codes that forbid allocation after start-up (real-time or certified runs, where
// every byte is reserved up front), or code that has handed the rest of the device to another allocator
// and may not take memory behind its back. This variant keeps the directions in a fixed file-scope
// device array instead.
//
// Contract (declared in include/fdbem.h):
//  - at most FDA_RHS_NOALLOC_MAX directions per call; larger requests fail with FDA_E_INVALID_ARG;
//  - the array lives in every GPU that loads the library until the process exits;
//  - set-up: the first call in a CUDA context of a device looks up the array's device address there
//    (cudaGetSymbolAddress, with that device current) and keeps it for that context; make that first
//    call before any stream capture begins. A context created later on the same device (for example
//    after cudaDeviceReset) is recognised by its context id and gets its own look-up;
//  - every call shares the one array, which keeps the previous call's directions: calls that overlap on
//    the GPU (different streams, no ordering between them) race on it;
//  - the call waits for its stream before it returns.
#include <cuda.h>

#include <mutex>

#include "internal.cuh"

#define FDA_RHS_NOALLOC_MAX 1024
#define FDA_RHS_NOALLOC_DEVICES 64

// Fixed scratch: nrhs x 3 directions (doubles). Every call overwrites the entries it uses, so nothing in
// it has to start at zero.
static __device__ __align__(256) double g_rhs_dirs[3 * FDA_RHS_NOALLOC_MAX];

namespace {

// Per device: the context the address was looked up in (its driver-assigned id, never reused within a
// process) and the address.
struct ScratchAddr {
  unsigned long long ctx_id = 0;
  bool valid = false;
  double* addr = nullptr;
};
ScratchAddr g_rhs_addr[FDA_RHS_NOALLOC_DEVICES];
std::mutex g_rhs_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// id of the current context, resolved through the runtime's driver entry points (no link to libcuda)
int current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
      fda::set_error("driver entry points cuCtxGetCurrent / cuCtxGetId are not available");
      return FDA_E_CUDA;
    }
    get_current = (CtxGetCurrentFn)f1;
    get_id = (CtxGetIdFn)f2;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS) {
    fda::set_error("no current CUDA context");
    return FDA_E_CUDA;
  }
  return FDA_OK;
}

// Device address of g_rhs_dirs in the current context: looked up once per context of each device, with
// that device current.
int rhs_scratch_address(double** out) {
  int dev = 0;
  FDA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= FDA_RHS_NOALLOC_DEVICES) {
    fda::set_error("device %d beyond the %d devices bm_rhs_plane_wave_noalloc supports", dev, FDA_RHS_NOALLOC_DEVICES);
    return FDA_E_INVALID_ARG;
  }
  // the context id before the look-up; a thread with no current context yet gets one from the runtime
  // during the look-up, and the id is read again after it
  unsigned long long id = 0;
  const bool have_ctx = current_context_id(&id) == FDA_OK;
  std::lock_guard<std::mutex> lock(g_rhs_mu);
  ScratchAddr& e = g_rhs_addr[dev];
  if (!have_ctx || !e.valid || e.ctx_id != id) {
    void* p = nullptr;
    cudaError_t rc = cudaGetSymbolAddress(&p, g_rhs_dirs);
    if (rc != cudaSuccess || !p) {
      fda::set_error("cudaGetSymbolAddress(g_rhs_dirs) failed: %s", cudaGetErrorString(rc));
      return FDA_E_CUDA;
    }
    FDA_TRY(current_context_id(&id));
    e.addr = (double*)p;
    e.ctx_id = id;
    e.valid = true;
  }
  *out = e.addr;
  return FDA_OK;
}

// b = u_inc + alpha du_inc/dn_x, u_inc = exp(i k d.x), d normalised here (same arithmetic as
// bm_rhs_plane_wave, which normalises on the host before copying).
__global__ void k_plane_wave_fixed(const double* x, const double* n, int64_t N, const double* dirs, int nrhs,
                                   double k, double2 alpha, double2* b) {
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

}  // namespace

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
  FDA_TRY(fda::problem_device_current(prob));
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
