// Octree and interaction lists on the GPU (Sec. 3.1.1), integer rules:
//   quantised 63-bit Morton keys -> stable radix sort -> level-synchronous split of boxes
//   holding more than N_p points -> near/interaction lists by a dual recursion over near
//   pairs from (root, root), with directional wedges for the high-frequency levels.
// All decisions are integer (the FP64 quantisation uses explicitly rounded operations), so
// the result is bit-identical to any other implementation of the same rules.
#include "internal.cuh"

#include <algorithm>

namespace fda {

// ------------------------------------------------------------------ scan
static __global__ void k_scan_chunks(const int64_t* in, int64_t* out, int64_t* sums, int64_t n) {
  __shared__ int64_t sh[1024];
  int64_t base = (int64_t)blockIdx.x * 1024;
  int t = threadIdx.x;
  int64_t v = (base + t < n) ? in[base + t] : 0;
  sh[t] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t a = (t >= o) ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += a;
    __syncthreads();
  }
  if (base + t < n) out[base + t] = sh[t] - v;  // exclusive
  if (t == 1023) sums[blockIdx.x] = sh[1023];
}

static __global__ void k_scan_sums(int64_t* sums, int64_t nb, int64_t* total) {
  __shared__ int64_t sh[1024];
  __shared__ int64_t carry;
  int t = threadIdx.x;
  if (t == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += 1024) {
    int64_t v = (base + t < nb) ? sums[base + t] : 0;
    sh[t] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int64_t a = (t >= o) ? sh[t - o] : 0;
      __syncthreads();
      sh[t] += a;
      __syncthreads();
    }
    if (base + t < nb) sums[base + t] = carry + sh[t] - v;
    __syncthreads();
    if (t == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (t == 0) *total = carry;
}

static __global__ void k_scan_add(int64_t* out, const int64_t* sums, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  if (i < n) out[i] += sums[blockIdx.x];
}

int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total_host, cudaStream_t s) {
  if (n <= 0) {
    if (total_host) *total_host = 0;
    return FDA_OK;
  }
  int64_t nb = (n + 1023) / 1024;
  DBuf<int64_t> sums, tot;
  FDA_TRY(sums.alloc(nb));
  FDA_TRY(tot.alloc(1));
  k_scan_chunks<<<(unsigned)nb, 1024, 0, s>>>(in, out, sums.p, n);
  k_scan_sums<<<1, 1024, 0, s>>>(sums.p, nb, tot.p);
  k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(out, sums.p, n);
  FDA_LAUNCH_CHECK();
  if (total_host) {
    FDA_CUDA(cudaMemcpyAsync(total_host, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
  } else {
    FDA_CUDA(cudaStreamSynchronize(s));
  }
  return FDA_OK;
}

// ------------------------------------------------------------------ stable LSD radix sort (8-bit digits)
static __global__ void k_radix_hist(const uint64_t* keys, int64_t n, int shift, int64_t* hist, int64_t nblk) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

static __global__ void k_radix_scatter(const uint64_t* kin, const int64_t* vin, uint64_t* kout, int64_t* vout,
                                       int64_t n, int shift, const int64_t* off, int64_t nblk) {
  __shared__ int wcnt[8][256];
  int t = threadIdx.x, w = t >> 5, lane = t & 31;
  for (int q = t; q < 8 * 256; q += 256) (&wcnt[0][0])[q] = 0;
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * 256 + t;
  bool valid = i < n;
  unsigned d = valid ? (unsigned)((kin[i] >> shift) & 255u) : 256u + lane;  // invalid lanes never match digits
  unsigned peers = __match_any_sync(0xffffffffu, d);
  int rank = __popc(peers & ((1u << lane) - 1u));
  if (valid && rank == 0) wcnt[w][d] = __popc(peers);
  __syncthreads();
  if (valid) {
    int before = 0;
    for (int q = 0; q < w; ++q) before += wcnt[q][d];
    int64_t pos = off[(int64_t)d * nblk + blockIdx.x] + before + rank;
    kout[pos] = kin[i];
    vout[pos] = vin[i];
  }
}

int radix_sort_pairs(uint64_t* keys, int64_t* vals, int64_t n, int bits, cudaStream_t s) {
  if (n <= 1) return FDA_OK;
  int64_t nblk = (n + 255) / 256;
  DBuf<uint64_t> k2;
  DBuf<int64_t> v2, hist;
  FDA_TRY(k2.alloc(n));
  FDA_TRY(v2.alloc(n));
  FDA_TRY(hist.alloc(256 * nblk));
  uint64_t *ka = keys, *kb = k2.p;
  int64_t *va = vals, *vb = v2.p;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    k_radix_hist<<<(unsigned)nblk, 256, 0, s>>>(ka, n, shift, hist.p, nblk);
    FDA_LAUNCH_CHECK();
    FDA_TRY(exclusive_scan_i64(hist.p, hist.p, 256 * nblk, nullptr, s));
    k_radix_scatter<<<(unsigned)nblk, 256, 0, s>>>(ka, va, kb, vb, n, shift, hist.p, nblk);
    FDA_LAUNCH_CHECK();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    FDA_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    FDA_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  }
  FDA_CUDA(cudaStreamSynchronize(s));
  return FDA_OK;
}

// ------------------------------------------------------------------ bounding box + Morton keys
static __global__ void k_bbox_partial(const double* x, int64_t N, double* part) {
  __shared__ double lo[3][256], hi[3][256];
  int t = threadIdx.x;
  double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = (int64_t)blockIdx.x * 256 + t; i < N; i += (int64_t)gridDim.x * 256)
    for (int d = 0; d < 3; ++d) {
      double v = x[3 * i + d];
      l[d] = fmin(l[d], v);
      h[d] = fmax(h[d], v);
    }
  for (int d = 0; d < 3; ++d) {
    lo[d][t] = l[d];
    hi[d][t] = h[d];
  }
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o)
      for (int d = 0; d < 3; ++d) {
        lo[d][t] = fmin(lo[d][t], lo[d][t + o]);
        hi[d][t] = fmax(hi[d][t], hi[d][t + o]);
      }
    __syncthreads();
  }
  if (t == 0)
    for (int d = 0; d < 3; ++d) {
      part[6 * blockIdx.x + d] = lo[d][0];
      part[6 * blockIdx.x + 3 + d] = hi[d][0];
    }
}

__device__ __forceinline__ uint64_t spread3(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

// q = floor((x - corner) / side * 2^21), every operation explicitly rounded (no contraction)
static __global__ void k_morton(const double* x, int64_t N, double c0, double c1, double c2, double side,
                                uint64_t* keys, int64_t* idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double cc[3] = {c0, c1, c2};
  uint64_t q[3];
  for (int d = 0; d < 3; ++d) {
    double t = __dsub_rn(x[3 * i + d], cc[d]);
    double u = __ddiv_rn(t, side);
    double v = __dmul_rn(u, 2097152.0);
    double f = floor(v);
    int64_t qi = (int64_t)f;
    qi = qi < 0 ? 0 : (qi > 2097151 ? 2097151 : qi);
    q[d] = (uint64_t)qi;
  }
  keys[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
  idx[i] = i;
}

// ------------------------------------------------------------------ octree split
__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* a, int64_t lo, int64_t hi, uint64_t v) {
  while (lo < hi) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

struct BoxArrays {
  int32_t *lev, *ix, *iy, *iz, *nch, *leaf;
  int64_t *par, *cbeg, *pb, *pe;
};

static __global__ void k_split_count(BoxArrays B, const uint64_t* keys, int64_t lb, int64_t le, int l, int leaf_max,
                                     int64_t* bounds, int64_t* nchild) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t b = lb + q;
  if (b >= le) return;
  int64_t p0 = B.pb[b], p1 = B.pe[b];
  int64_t cnt = 0;
  if (p1 - p0 > leaf_max && l < 21) {
    uint64_t prefix = (spread3((uint64_t)B.ix[b]) << 2) | (spread3((uint64_t)B.iy[b]) << 1) | spread3((uint64_t)B.iz[b]);
    int sh = 3 * (20 - l);
    int64_t prev = p0;
    for (int o = 0; o < 8; ++o) {
      uint64_t lo = ((prefix << 3) | (uint64_t)o) << sh;
      int64_t s = (o == 0) ? p0 : lower_bound_u64(keys, p0, p1, lo);
      bounds[9 * q + o] = s;
      if (o > 0 && s > prev) ++cnt;
      prev = s;
    }
    bounds[9 * q + 8] = p1;
    if (p1 > prev) ++cnt;
  }
  nchild[q] = cnt;
}

static __global__ void k_split_write(BoxArrays B, int64_t lb, int64_t le, int l, int leaf_max,
                                     const int64_t* bounds, const int64_t* off, int64_t child_base) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t b = lb + q;
  if (b >= le) return;
  if (!(B.pe[b] - B.pb[b] > leaf_max && l < 21)) return;  // same rule as k_split_count
  int64_t c = child_base + off[q];
  int n = 0;
  for (int o = 0; o < 8; ++o) {
    int64_t s0 = bounds[9 * q + o], s1 = bounds[9 * q + o + 1];
    if (s1 <= s0) continue;
    int64_t ci = c + n;
    B.lev[ci] = l + 1;
    B.ix[ci] = 2 * B.ix[b] + ((o >> 2) & 1);
    B.iy[ci] = 2 * B.iy[b] + ((o >> 1) & 1);
    B.iz[ci] = 2 * B.iz[b] + (o & 1);
    B.nch[ci] = 0;
    B.leaf[ci] = 1;
    B.par[ci] = b;
    B.cbeg[ci] = -1;
    B.pb[ci] = s0;
    B.pe[ci] = s1;
    ++n;
  }
  B.nch[b] = n;
  B.leaf[b] = 0;
  B.cbeg[b] = c;
}

// ------------------------------------------------------------------ lists
struct LevelRules {
  int32_t hf[FDA_MAXLEV], T[FDA_MAXLEV], n[FDA_MAXLEV];
};

static __global__ void k_pairs_count(BoxArrays B, const int64_t* cur, int64_t ncur, int l, LevelRules R,
                                     int64_t* ndir, int64_t* nnext, int64_t* nm2l) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= ncur) return;
  int64_t P = cur[2 * u], Q = cur[2 * u + 1];
  int64_t d = 0, nx = 0, nm = 0;
  if (B.leaf[P] || B.leaf[Q]) {
    d = 1;
  } else {
    int Tn = R.T[l + 1];
    for (int64_t c = B.cbeg[P]; c < B.cbeg[P] + B.nch[P]; ++c)
      for (int64_t e = B.cbeg[Q]; e < B.cbeg[Q] + B.nch[Q]; ++e) {
        int32_t dx = B.ix[e] - B.ix[c], dy = B.iy[e] - B.iy[c], dz = B.iz[e] - B.iz[c];
        int32_t m = max(abs(dx), max(abs(dy), abs(dz)));
        if (m <= Tn + 1)
          ++nx;
        else
          ++nm;
      }
  }
  ndir[u] = d;
  nnext[u] = nx;
  nm2l[u] = nm;
}

static __global__ void k_pairs_write(BoxArrays B, const int64_t* cur, int64_t ncur, int l, LevelRules R,
                                     const int64_t* odir, const int64_t* onext, const int64_t* om2l, int64_t dir_base,
                                     int64_t m2l_base, int64_t* direct, int64_t* next, int64_t* m2l_box,
                                     int32_t* m2l_info) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= ncur) return;
  int64_t P = cur[2 * u], Q = cur[2 * u + 1];
  if (B.leaf[P] || B.leaf[Q]) {
    int64_t o = dir_base + odir[u];
    direct[2 * o] = P;
    direct[2 * o + 1] = Q;
    return;
  }
  int64_t on = onext[u], om = m2l_base + om2l[u];
  int L = l + 1;
  int Tn = R.T[L];
  for (int64_t c = B.cbeg[P]; c < B.cbeg[P] + B.nch[P]; ++c)
    for (int64_t e = B.cbeg[Q]; e < B.cbeg[Q] + B.nch[Q]; ++e) {
      int32_t dx = B.ix[e] - B.ix[c], dy = B.iy[e] - B.iy[c], dz = B.iz[e] - B.iz[c];
      int32_t m = max(abs(dx), max(abs(dy), abs(dz)));
      if (m <= Tn + 1) {
        next[2 * on] = c;
        next[2 * on + 1] = e;
        ++on;
      } else {
        m2l_box[2 * om] = c;
        m2l_box[2 * om + 1] = e;
        int32_t* inf = m2l_info + 6 * om;
        inf[0] = L;
        inf[1] = dx;
        inf[2] = dy;
        inf[3] = dz;
        if (R.hf[L]) {
          inf[4] = wedge_of(R.n[L], -dx, -dy, -dz);  // source's outgoing wedge (source -> target)
          inf[5] = wedge_of(R.n[L], dx, dy, dz);     // target's incoming wedge (target -> source)
        } else {
          inf[4] = 0;
          inf[5] = 0;
        }
        ++om;
      }
    }
}

static __global__ void k_pair_keys(const int64_t* pairs, int64_t n, int64_t stride, uint64_t* keys, int64_t* idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = (uint64_t)(pairs[2 * i] * stride + pairs[2 * i + 1]);
  idx[i] = i;
}

template <typename T, int W>
static __global__ void k_gather_rows(const T* in, const int64_t* idx, int64_t n, T* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t s = idx[i];
#pragma unroll
  for (int q = 0; q < W; ++q) out[W * i + q] = in[W * s + q];
}

template <typename T>
static int grow(DBuf<T>& b, size_t need, size_t used) {
  if (need <= b.n) return FDA_OK;
  size_t cap = std::max(need, 2 * b.n + 1024);
  T* np = nullptr;
  cudaError_t e = cudaMalloc((void**)&np, cap * sizeof(T));
  if (e != cudaSuccess) {
    set_error("cudaMalloc(%zu): %s", cap * sizeof(T), cudaGetErrorString(e));
    return FDA_E_OOM;
  }
  if (used) FDA_CUDA(cudaMemcpy(np, b.p, used * sizeof(T), cudaMemcpyDeviceToDevice));
  b.release();
  b.p = np;
  b.n = cap;
  return FDA_OK;
}

}  // namespace fda

using namespace fda;

static int box_grow(fda_tree_s* T, size_t need, size_t used) {
  FDA_TRY(grow(T->lev, need, used));
  FDA_TRY(grow(T->ix, need, used));
  FDA_TRY(grow(T->iy, need, used));
  FDA_TRY(grow(T->iz, need, used));
  FDA_TRY(grow(T->nch, need, used));
  FDA_TRY(grow(T->leaf, need, used));
  FDA_TRY(grow(T->par, need, used));
  FDA_TRY(grow(T->cbeg, need, used));
  FDA_TRY(grow(T->pb, need, used));
  FDA_TRY(grow(T->pe, need, used));
  return FDA_OK;
}

static BoxArrays box_arrays(fda_tree_s* T) {
  BoxArrays B;
  B.lev = T->lev.p;
  B.ix = T->ix.p;
  B.iy = T->iy.p;
  B.iz = T->iz.p;
  B.nch = T->nch.p;
  B.leaf = T->leaf.p;
  B.par = T->par.p;
  B.cbeg = T->cbeg.p;
  B.pb = T->pb.p;
  B.pe = T->pe.p;
  return B;
}

int fda_tree_build_impl(bm_problem_s* P, int leaf_max, fda_tree_s* T) {
  cudaStream_t s = 0;
  const int64_t N = P->N;
  T->prob = P;
  T->leaf_max = leaf_max;
  T->N = N;
  // 1. bounding box (exact min/max), root cube on the host with the same FP64 operations as any
  //    other implementation of the rules: centre = (lo+hi)/2, side = extent * (1 + 2^-20)
  int nbb = (int)std::min<int64_t>(1024, (N + 255) / 256);
  DBuf<double> part;
  FDA_TRY(part.alloc(6 * nbb));
  k_bbox_partial<<<nbb, 256, 0, s>>>(P->x.p, N, part.p);
  FDA_LAUNCH_CHECK();
  std::vector<double> hp;
  FDA_TRY(part.download(hp));
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int b = 0; b < nbb; ++b)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], hp[6 * b + d]);
      hi[d] = std::max(hi[d], hp[6 * b + 3 + d]);
    }
  double ext = 0.0;
  for (int d = 0; d < 3; ++d) ext = std::max(ext, hi[d] - lo[d]);
  volatile double one_plus = 1.0 + 9.5367431640625e-07;
  double side = ext * one_plus;
  if (!(side > 0.0)) side = 1.0;
  T->side = side;
  for (int d = 0; d < 3; ++d) {
    volatile double c = 0.5 * (lo[d] + hi[d]);
    volatile double hs = 0.5 * side;
    T->corner[d] = c - hs;
  }
  // 2. Morton keys + stable sort (ties by DOF index)
  FDA_TRY(T->keys.alloc(N));
  FDA_TRY(T->perm.alloc(N));
  k_morton<<<cdiv(N, 256), 256, 0, s>>>(P->x.p, N, T->corner[0], T->corner[1], T->corner[2], side, T->keys.p,
                                        T->perm.p);
  FDA_LAUNCH_CHECK();
  FDA_TRY(radix_sort_pairs(T->keys.p, T->perm.p, N, 63, s));
  // 3. level-synchronous split
  size_t cap = std::max<size_t>(1024, (size_t)(4 * N / std::max(1, leaf_max) + 64));
  FDA_TRY(box_grow(T, cap, 0));
  {
    int32_t zero = 0, one = 1;
    int64_t m1 = -1, z64 = 0, n64 = N;
    FDA_CUDA(cudaMemcpy(T->lev.p, &zero, 4, cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(T->ix.p, &zero, 4, cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(T->iy.p, &zero, 4, cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(T->iz.p, &zero, 4, cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(T->nch.p, &zero, 4, cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(T->leaf.p, &one, 4, cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(T->par.p, &m1, 8, cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(T->cbeg.p, &m1, 8, cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(T->pb.p, &z64, 8, cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(T->pe.p, &n64, 8, cudaMemcpyHostToDevice));
  }
  int64_t nbox = 1, lb = 0, le = 1;
  int l = 0;
  std::vector<int64_t> level_begin(1, 0);
  while (l < 21) {
    int64_t nl = le - lb;
    DBuf<int64_t> bounds, nchild;
    FDA_TRY(bounds.alloc(9 * nl));
    FDA_TRY(nchild.alloc(nl));
    k_split_count<<<cdiv(nl, 128), 128, 0, s>>>(box_arrays(T), T->keys.p, lb, le, l, leaf_max, bounds.p, nchild.p);
    FDA_LAUNCH_CHECK();
    int64_t total = 0;
    FDA_TRY(exclusive_scan_i64(nchild.p, nchild.p, nl, &total, s));
    if (total == 0) break;
    FDA_TRY(box_grow(T, nbox + total, nbox));
    k_split_write<<<cdiv(nl, 128), 128, 0, s>>>(box_arrays(T), lb, le, l, leaf_max, bounds.p, nchild.p, le);
    FDA_LAUNCH_CHECK();
    nbox += total;
    lb = le;
    le = nbox;
    ++l;
    level_begin.push_back(lb);
  }
  T->nbox = nbox;
  T->nlev = l + 1;
  if (T->nlev > FDA_MAXLEV) {
    set_error("tree depth %d exceeds %d", T->nlev, FDA_MAXLEV);
    return FDA_E_INVALID_ARG;
  }
  // 4. per-level regime rules (host FP64, same operations as any implementation of the rules)
  const double k = P->k;
  int Lhf = -1;
  LevelRules R;
  for (int q = 0; q < FDA_MAXLEV; ++q) R.hf[q] = R.T[q] = 0, R.n[q] = 1;
  for (int q = 0; q < T->nlev; ++q) {
    volatile double w = ldexp(side, -q);
    volatile double kw = k * w;
    R.hf[q] = (kw >= 2.0 * FDA_PI) ? 1 : 0;
    volatile double t = kw / FDA_PI;
    R.T[q] = R.hf[q] ? (int32_t)floor(t) : 0;
    if (R.hf[q]) Lhf = q;
  }
  for (int q = 0; q < T->nlev; ++q) R.n[q] = R.hf[q] ? (1 << (Lhf - q)) : 1;
  for (int q = 0; q < FDA_MAXLEV; ++q) {
    T->hf[q] = R.hf[q];
    T->T[q] = R.T[q];
    T->nw[q] = R.n[q];
  }
  // 5. dual recursion over near pairs
  DBuf<int64_t> cur, nxt;
  FDA_TRY(cur.alloc(2));
  {
    int64_t rr[2] = {0, 0};
    FDA_CUDA(cudaMemcpy(cur.p, rr, 16, cudaMemcpyHostToDevice));
  }
  int64_t ncur = 1, ndir = 0, nm = 0;
  DBuf<int64_t> direct, m2lb;
  DBuf<int32_t> m2li;
  for (int q = 0; q < T->nlev && ncur > 0; ++q) {
    DBuf<int64_t> cd, cn, cm;
    FDA_TRY(cd.alloc(ncur));
    FDA_TRY(cn.alloc(ncur));
    FDA_TRY(cm.alloc(ncur));
    k_pairs_count<<<cdiv(ncur, 128), 128, 0, s>>>(box_arrays(T), cur.p, ncur, q, R, cd.p, cn.p, cm.p);
    FDA_LAUNCH_CHECK();
    int64_t td = 0, tn = 0, tm = 0;
    FDA_TRY(exclusive_scan_i64(cd.p, cd.p, ncur, &td, s));
    FDA_TRY(exclusive_scan_i64(cn.p, cn.p, ncur, &tn, s));
    FDA_TRY(exclusive_scan_i64(cm.p, cm.p, ncur, &tm, s));
    FDA_TRY(grow(direct, 2 * (ndir + td), 2 * ndir));
    FDA_TRY(grow(m2lb, 2 * (nm + tm), 2 * nm));
    FDA_TRY(grow(m2li, 6 * (nm + tm), 6 * nm));
    FDA_TRY(nxt.alloc(2 * std::max<int64_t>(tn, 1)));
    k_pairs_write<<<cdiv(ncur, 128), 128, 0, s>>>(box_arrays(T), cur.p, ncur, q, R, cd.p, cn.p, cm.p, ndir, nm,
                                                   direct.p, nxt.p, m2lb.p, m2li.p);
    FDA_LAUNCH_CHECK();
    FDA_CUDA(cudaStreamSynchronize(s));
    ndir += td;
    nm += tm;
    std::swap(cur.p, nxt.p);
    std::swap(cur.n, nxt.n);
    ncur = tn;
  }
  // 6. canonical order by (target, source)
  const int64_t stride = nbox + 1;
  T->ndir = ndir;
  T->nm2l = nm;
  FDA_TRY(T->direct.alloc(2 * std::max<int64_t>(ndir, 1)));
  FDA_TRY(T->m2l_box.alloc(2 * std::max<int64_t>(nm, 1)));
  FDA_TRY(T->m2l_info.alloc(6 * std::max<int64_t>(nm, 1)));
  int keybits = 1;
  while (keybits < 63 && ((uint64_t)1 << keybits) <= (uint64_t)(stride * stride)) ++keybits;
  if (ndir > 0) {
    DBuf<uint64_t> kk;
    DBuf<int64_t> id;
    FDA_TRY(kk.alloc(ndir));
    FDA_TRY(id.alloc(ndir));
    k_pair_keys<<<cdiv(ndir, 256), 256, 0, s>>>(direct.p, ndir, stride, kk.p, id.p);
    FDA_LAUNCH_CHECK();
    FDA_TRY(radix_sort_pairs(kk.p, id.p, ndir, keybits, s));
    k_gather_rows<int64_t, 2><<<cdiv(ndir, 256), 256, 0, s>>>(direct.p, id.p, ndir, T->direct.p);
    FDA_LAUNCH_CHECK();
  }
  if (nm > 0) {
    DBuf<uint64_t> kk;
    DBuf<int64_t> id;
    FDA_TRY(kk.alloc(nm));
    FDA_TRY(id.alloc(nm));
    k_pair_keys<<<cdiv(nm, 256), 256, 0, s>>>(m2lb.p, nm, stride, kk.p, id.p);
    FDA_LAUNCH_CHECK();
    FDA_TRY(radix_sort_pairs(kk.p, id.p, nm, keybits, s));
    k_gather_rows<int64_t, 2><<<cdiv(nm, 256), 256, 0, s>>>(m2lb.p, id.p, nm, T->m2l_box.p);
    k_gather_rows<int32_t, 6><<<cdiv(nm, 256), 256, 0, s>>>(m2li.p, id.p, nm, T->m2l_info.p);
    FDA_LAUNCH_CHECK();
  }
  FDA_CUDA(cudaDeviceSynchronize());
  // 7. host mirrors
  auto dl = [&](auto& dbuf, auto& vec, size_t n) -> int {
    vec.resize(n);
    if (n) FDA_CUDA(cudaMemcpy(vec.data(), dbuf.p, n * sizeof(vec[0]), cudaMemcpyDeviceToHost));
    return FDA_OK;
  };
  FDA_TRY(dl(T->perm, T->h_perm, N));
  FDA_TRY(dl(T->keys, T->h_keys, N));
  FDA_TRY(dl(T->lev, T->h_lev, nbox));
  FDA_TRY(dl(T->ix, T->h_ix, nbox));
  FDA_TRY(dl(T->iy, T->h_iy, nbox));
  FDA_TRY(dl(T->iz, T->h_iz, nbox));
  FDA_TRY(dl(T->nch, T->h_nch, nbox));
  FDA_TRY(dl(T->leaf, T->h_leaf, nbox));
  FDA_TRY(dl(T->par, T->h_par, nbox));
  FDA_TRY(dl(T->cbeg, T->h_cbeg, nbox));
  FDA_TRY(dl(T->pb, T->h_pb, nbox));
  FDA_TRY(dl(T->pe, T->h_pe, nbox));
  FDA_TRY(dl(T->direct, T->h_direct, 2 * ndir));
  FDA_TRY(dl(T->m2l_box, T->h_m2l_box, 2 * nm));
  FDA_TRY(dl(T->m2l_info, T->h_m2l_info, 6 * nm));
  T->h_level_hf.assign(T->hf, T->hf + T->nlev);
  T->h_level_T.assign(T->T, T->T + T->nlev);
  T->h_level_n.assign(T->nw, T->nw + T->nlev);
  return FDA_OK;
}
