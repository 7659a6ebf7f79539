// Internal handle layouts and cross-file helpers of the FDA Burton-Miller library.
#pragma once
#include "common.cuh"

#define FDA_MAXLEV 22

struct bm_net_s;
struct bm_precond_s;

struct bm_problem_s {
  int64_t ne = 0, N = 0, nn = 0;
  double k = 0;
  double2 alpha = {0, 0};
  int particles = 0;         // 1: points with normals (no elements): the particle summation of Sec. 5.1
  int device = 0;            // the CUDA device that holds the problem's arrays (current at creation)
  fda::DBuf<double> nodes;   // nn x 3
  fda::DBuf<int32_t> elems;  // ne x 6
  fda::DBuf<double> x, n, w; // N x 3, N x 3 (paper normal, into the body), N
};

struct fda_tree_s {
  bm_problem_s* prob = nullptr;
  int leaf_max = 0;
  int64_t N = 0, nbox = 0, ndir = 0, nm2l = 0;
  int nlev = 0;
  double corner[3] = {0, 0, 0}, side = 1.0;
  int32_t hf[FDA_MAXLEV] = {0}, T[FDA_MAXLEV] = {0}, nw[FDA_MAXLEV] = {0};
  // device
  fda::DBuf<int64_t> perm;      // tree position -> DOF
  fda::DBuf<uint64_t> keys;
  fda::DBuf<int32_t> lev, ix, iy, iz, nch, leaf;
  fda::DBuf<int64_t> par, cbeg, pb, pe;
  fda::DBuf<int64_t> direct;    // ndir x 2
  fda::DBuf<int64_t> m2l_box;   // nm2l x 2
  fda::DBuf<int32_t> m2l_info;  // nm2l x 6
  // host mirrors (export + host-side scheduling of the plan)
  std::vector<int64_t> h_perm, h_par, h_cbeg, h_pb, h_pe, h_direct, h_m2l_box;
  std::vector<uint64_t> h_keys;
  std::vector<int32_t> h_lev, h_ix, h_iy, h_iz, h_nch, h_leaf, h_m2l_info;
  std::vector<int32_t> h_level_hf, h_level_T, h_level_n;
};

namespace fda {

// FDA_E_INVALID_ARG unless the problem's device is the current one (kernels read its arrays there)
inline int problem_device_current(const bm_problem_s* P) {
  int dev = -1;
  FDA_CUDA(cudaGetDevice(&dev));
  if (dev != P->device) {
    set_error("the problem lives on device %d but device %d is current", P->device, dev);
    return FDA_E_INVALID_ARG;
  }
  return FDA_OK;
}

// exclusive prefix sum of n int64 values (in may alias out)
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total_host, cudaStream_t s);
// stable LSD radix sort of (key, value) pairs on the low `bits` bits of the keys
int radix_sort_pairs(uint64_t* keys, int64_t* vals, int64_t n, int bits, cudaStream_t s);

// integer wedge rule shared by the list builder (see fdbem.h)
__host__ __device__ __forceinline__ int32_t wedge_of(int n, int32_t dx, int32_t dy, int32_t dz) {
  int64_t d[3] = {dx, dy, dz};
  int64_t ad[3] = {d[0] < 0 ? -d[0] : d[0], d[1] < 0 ? -d[1] : d[1], d[2] < 0 ? -d[2] : d[2]};
  int a = 0;
  if (ad[1] > ad[a]) a = 1;
  if (ad[2] > ad[a]) a = 2;
  int64_t m = ad[a];
  int face = 2 * a + (d[a] > 0 ? 0 : 1);
  int o1 = (a == 0) ? 1 : 0, o2 = (a == 2) ? 1 : 2;
  int64_t c1 = ((int64_t)n * (d[o1] + m)) / (2 * m);
  int64_t c2 = ((int64_t)n * (d[o2] + m)) / (2 * m);
  if (c1 > n - 1) c1 = n - 1;
  if (c2 > n - 1) c2 = n - 1;
  return (int32_t)(face * (int64_t)n * n + c1 * n + c2);
}

}  // namespace fda
