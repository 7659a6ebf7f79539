// Learned leaf-block preconditioner for flexible GMRES.
//
// For every leaf box L of the tree, y_L = A_LL^-1 r_L with A_LL = (1/2) I + (near-field self block of L),
// inverted once in FP64 (Gauss-Jordan, one CTA per leaf) and stored in FP32. A small network, shared by all
// points, reads per point the residual and the block solution normalised by the leaf's complex mean
// residual s_L (features u = r/s_L, v = y/s_L and the leaf mean of v: 6 reals), and outputs two complex
// weights, z_i = w1_i r_i + w2_i y_i. Architecture 6 -> H -> H -> 4 with tanh hidden layers; the last
// layer starts at zero with bias (1, 0, 0, 0), i.e. the identity preconditioner.
// Training minimises sum over pairs of |z - e|^2 / |e|^2 on residual/correction pairs (r, e = x* - x)
// harvested from GMRES solves; hand-written forward, backward (shared-memory gradient accumulation) and
// Adam kernels, FP32.
#include "plan.cuh"

#define NET_IN 6
#define NET_OUT 4
#define NET_HMAX 64

struct bm_net_s {
  int H = 32;
  int nparam = 0;
  fda::DBuf<float> w, g, m, v;  // parameters, gradient, Adam moments
  int64_t step = 0;
};

struct bm_precond_s {
  fda_plan_s* plan = nullptr;
  int64_t nleaf = 0;
  fda::DBuf<int64_t> leaf_pb, leaf_pe, inv_off;  // per leaf: point range (tree order), inverse offset
  fda::DBuf<float2> inv;                          // nr x nr column-major per leaf
  fda::DBuf<int32_t> pt_leaf;                     // tree point -> leaf index (-1 if none)
  fda::DBuf<float2> rt, yt, zt, et;               // tree-order work vectors (N each)
  fda::DBuf<float2> seg;                          // per leaf: s_L, mean(v)
  fda::DBuf<float> loss_acc;
};

namespace fda {

int gmres_solve(fda_plan_s* P, const double2* b, double2* x, int nrhs, const bm_gmres_opts_t* o,
                bm_gmres_stats_t* st, cudaStream_t s, bm_precond_s* pc, bm_net_s* net);

// offsets of the parameter blocks: W1 (H x 6), b1 (H), W2 (H x H), b2 (H), W3 (4 x H), b3 (4)
struct NetLayout {
  int H, W1, b1, W2, b2, W3, b3, n;
  __host__ __device__ NetLayout(int h) : H(h) {
    W1 = 0;
    b1 = W1 + h * NET_IN;
    W2 = b1 + h;
    b2 = W2 + h * h;
    W3 = b2 + h;
    b3 = W3 + NET_OUT * h;
    n = b3 + NET_OUT;
  }
};

// ------------------------------------------------------------------ block-Jacobi inverses
static __global__ void k_leaf_inverse(const int64_t* leaf_pb, const int64_t* leaf_pe, const int64_t* blk_off,
                                      const double2* near, const int64_t* inv_off, float2* inv) {
  extern __shared__ unsigned char smem_raw[];
  const int64_t L = blockIdx.x;
  const int n = (int)(leaf_pe[L] - leaf_pb[L]);
  double2* M = (double2*)smem_raw;  // n x 2n, row-major
  const int W = 2 * n;
  const double2* B = near + blk_off[L];  // self block, column-major n x n
  for (int q = threadIdx.x; q < n * W; q += blockDim.x) {
    int i = q / W, j = q - i * W;
    double2 v = make_double2(0, 0);
    if (j < n) {
      v = B[(int64_t)j * n + i];
      if (i == j) v.x += 0.5;
    } else if (j - n == i) {
      v = make_double2(1, 0);
    }
    M[q] = v;
  }
  __syncthreads();
  __shared__ int piv;
  for (int c = 0; c < n; ++c) {
    if (threadIdx.x == 0) {
      int p = c;
      double best = cabs2(M[c * W + c]);
      for (int r = c + 1; r < n; ++r) {
        double a = cabs2(M[r * W + c]);
        if (a > best) best = a, p = r;
      }
      piv = p;
    }
    __syncthreads();
    if (piv != c)
      for (int j = threadIdx.x; j < W; j += blockDim.x) {
        double2 t = M[c * W + j];
        M[c * W + j] = M[piv * W + j];
        M[piv * W + j] = t;
      }
    __syncthreads();
    double2 d = M[c * W + c];
    double dd = cabs2(d);
    double2 inv_d = make_double2(d.x / dd, -d.y / dd);
    __syncthreads();
    for (int j = threadIdx.x; j < W; j += blockDim.x) M[c * W + j] = cmul(M[c * W + j], inv_d);
    __syncthreads();
    for (int q = threadIdx.x; q < n * W; q += blockDim.x) {
      int r = q / W, j = q - r * W;
      if (r == c) continue;
      double2 f = M[r * W + c];
      if (j == c) continue;
      M[q] = csub(M[q], cmul(f, M[c * W + j]));
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (r != c) M[r * W + c] = make_double2(0, 0);
    __syncthreads();
  }
  float2* out = inv + inv_off[L];
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
    int i = q % n, j = q / n;  // column-major
    double2 v = M[i * W + n + j];
    out[q] = make_float2((float)v.x, (float)v.y);
  }
}

// y_L = inv_L r_L (tree order)
static __global__ void k_leaf_apply(const int64_t* leaf_pb, const int64_t* leaf_pe, const int64_t* inv_off,
                                    const float2* inv, const float2* r, float2* y) {
  const int64_t L = blockIdx.x;
  const int64_t p0 = leaf_pb[L];
  const int n = (int)(leaf_pe[L] - p0);
  __shared__ float2 rs[256];
  for (int q = threadIdx.x; q < n; q += blockDim.x) rs[q] = r[p0 + q];
  __syncthreads();
  const float2* Mi = inv + inv_off[L];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float2 a = make_float2(0, 0);
    for (int j = 0; j < n; ++j) cfma(a, Mi[(int64_t)j * n + i], rs[j]);
    y[p0 + i] = a;
  }
}

// per-leaf statistics: s_L = mean r (falls back to the RMS of r when the mean is tiny), mean(y)/s_L
static __global__ void k_seg_stats(const int64_t* leaf_pb, const int64_t* leaf_pe, const float2* r, const float2* y,
                                   float2* seg) {
  const int64_t L = blockIdx.x;
  const int64_t p0 = leaf_pb[L];
  const int n = (int)(leaf_pe[L] - p0);
  float2 sr = make_float2(0, 0), sy = make_float2(0, 0);
  float ss = 0;
  for (int q = threadIdx.x; q < n; q += 32) {
    sr = cadd(sr, r[p0 + q]);
    sy = cadd(sy, y[p0 + q]);
    ss += cabs2(r[p0 + q]);
  }
  sr = warp_csum(sr);
  sy = warp_csum(sy);
  ss = warp_sum(ss);
  if (threadIdx.x == 0) {
    float2 mr = make_float2(sr.x / n, sr.y / n);
    float rms = sqrtf(ss / n);
    float am = sqrtf(cabs2(mr));
    float2 s = (am > 1e-3f * rms && am > 0) ? mr : make_float2(rms > 0 ? rms : 1.0f, 0.0f);
    float den = cabs2(s);
    float2 is = make_float2(s.x / den, -s.y / den);
    float2 my = make_float2(sy.x / n, sy.y / n);
    seg[2 * L] = s;
    seg[2 * L + 1] = cmul(my, is);
  }
}

// forward of one point; fills hidden activations when requested
__device__ __forceinline__ void net_forward(const float* w, const NetLayout& Ly, const float* f, float* h1, float* h2,
                                            float* o) {
  const int H = Ly.H;
  for (int j = 0; j < H; ++j) {
    float a = w[Ly.b1 + j];
#pragma unroll
    for (int q = 0; q < NET_IN; ++q) a = fmaf(w[Ly.W1 + j * NET_IN + q], f[q], a);
    h1[j] = tanhf(a);
  }
  for (int j = 0; j < H; ++j) {
    float a = w[Ly.b2 + j];
    for (int q = 0; q < H; ++q) a = fmaf(w[Ly.W2 + j * H + q], h1[q], a);
    h2[j] = tanhf(a);
  }
  for (int j = 0; j < NET_OUT; ++j) {
    float a = w[Ly.b3 + j];
    for (int q = 0; q < H; ++q) a = fmaf(w[Ly.W3 + j * H + q], h2[q], a);
    o[j] = a;
  }
}

__device__ __forceinline__ void point_features(const float2 r, const float2 y, const float2 s, const float2 mv,
                                               float* f) {
  float den = cabs2(s);
  float2 is = make_float2(s.x / den, -s.y / den);
  float2 u = cmul(r, is), v = cmul(y, is);
  f[0] = u.x;
  f[1] = u.y;
  f[2] = v.x;
  f[3] = v.y;
  f[4] = mv.x;
  f[5] = mv.y;
}

// z = w1 r + w2 y
static __global__ void k_net_apply(const float* w, int H, int64_t N, const int32_t* pt_leaf, const float2* seg,
                                   const float2* r, const float2* y, float2* z) {
  extern __shared__ float sw[];
  NetLayout Ly(H);
  for (int q = threadIdx.x; q < Ly.n; q += blockDim.x) sw[q] = w[q];
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int L = pt_leaf[i];
  if (L < 0) {
    z[i] = r[i];
    return;
  }
  float f[NET_IN], h1[NET_HMAX], h2[NET_HMAX], o[NET_OUT];
  point_features(r[i], y[i], seg[2 * L], seg[2 * L + 1], f);
  net_forward(sw, Ly, f, h1, h2, o);
  float2 a = cmul(make_float2(o[0], o[1]), r[i]);
  cfma(a, make_float2(o[2], o[3]), y[i]);
  z[i] = a;
}

// loss and gradient: sum over points of |z - e|^2 * inv_E (per pair weight); gradient accumulated in shared
// memory, then added to the global gradient
static __global__ void k_net_grad(const float* w, int H, int64_t N, const int32_t* pt_leaf, const float2* seg,
                                  const float2* r, const float2* y, const float2* e, float invE, float* grad,
                                  float* loss) {
  extern __shared__ float sm[];
  NetLayout Ly(H);
  float* sw = sm;
  float* sg = sm + Ly.n;
  for (int q = threadIdx.x; q < Ly.n; q += blockDim.x) {
    sw[q] = w[q];
    sg[q] = 0;
  }
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float lsum = 0;
  if (i < N && pt_leaf[i] >= 0) {
    int L = pt_leaf[i];
    float f[NET_IN], h1[NET_HMAX], h2[NET_HMAX], o[NET_OUT];
    float2 ri = r[i], yi = y[i];
    point_features(ri, yi, seg[2 * L], seg[2 * L + 1], f);
    net_forward(sw, Ly, f, h1, h2, o);
    float2 zi = cmul(make_float2(o[0], o[1]), ri);
    cfma(zi, make_float2(o[2], o[3]), yi);
    float2 d = csub(zi, e[i]);
    lsum = cabs2(d) * invE;
    // dL/dz = 2 invE (z - e) as a real pair; dz/do0 = r, dz/do1 = i r, dz/do2 = y, dz/do3 = i y
    float gx = 2.f * invE * d.x, gy = 2.f * invE * d.y;
    float go[NET_OUT] = {gx * ri.x + gy * ri.y, -gx * ri.y + gy * ri.x, gx * yi.x + gy * yi.y,
                         -gx * yi.y + gy * yi.x};
    float dh2[NET_HMAX], dh1[NET_HMAX];
    for (int j = 0; j < NET_OUT; ++j) {
      atomicAdd(&sg[Ly.b3 + j], go[j]);
      for (int q = 0; q < H; ++q) atomicAdd(&sg[Ly.W3 + j * H + q], go[j] * h2[q]);
    }
    for (int q = 0; q < H; ++q) {
      float a = 0;
      for (int j = 0; j < NET_OUT; ++j) a = fmaf(sw[Ly.W3 + j * H + q], go[j], a);
      dh2[q] = a * (1.f - h2[q] * h2[q]);
    }
    for (int j = 0; j < H; ++j) {
      atomicAdd(&sg[Ly.b2 + j], dh2[j]);
      for (int q = 0; q < H; ++q) atomicAdd(&sg[Ly.W2 + j * H + q], dh2[j] * h1[q]);
    }
    for (int q = 0; q < H; ++q) {
      float a = 0;
      for (int j = 0; j < H; ++j) a = fmaf(sw[Ly.W2 + j * H + q], dh2[j], a);
      dh1[q] = a * (1.f - h1[q] * h1[q]);
    }
    for (int j = 0; j < H; ++j) {
      atomicAdd(&sg[Ly.b1 + j], dh1[j]);
      for (int q = 0; q < NET_IN; ++q) atomicAdd(&sg[Ly.W1 + j * NET_IN + q], dh1[j] * f[q]);
    }
  }
  lsum = warp_sum(lsum);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, lsum);
  __syncthreads();
  for (int q = threadIdx.x; q < Ly.n; q += blockDim.x)
    if (sg[q] != 0.f) atomicAdd(&grad[q], sg[q]);
}

static __global__ void k_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                              float eps, float c1, float c2) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  float gq = g[q];
  m[q] = b1 * m[q] + (1 - b1) * gq;
  v[q] = b2 * v[q] + (1 - b2) * gq * gq;
  w[q] -= lr * (m[q] / c1) / (sqrtf(v[q] / c2) + eps);
}

static __global__ void k_to_tree32(const double2* x, const int64_t* perm, int64_t N, float2* xt) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < N) xt[t] = make_float2((float)x[perm[t]].x, (float)x[perm[t]].y);
}
static __global__ void k_from_tree32(const float2* zt, const int64_t* perm, int64_t N, double2* z) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < N) z[perm[t]] = make_double2(zt[t].x, zt[t].y);
}
static __global__ void k_sumsq(const double2* e, int64_t N, float* out) {
  double a = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    a += cabs2(e[i]);
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, (float)a);
}

// z = M(r) for a user-order FP64 vector r (used inside flexible GMRES)
int precond_apply(bm_precond_s* Pc, bm_net_s* net, const double2* r, double2* z, cudaStream_t s) {
  fda_tree_s* T = Pc->plan->tree;
  const int64_t N = T->N;
  k_to_tree32<<<cdiv(N, 256), 256, 0, s>>>(r, T->perm.p, N, Pc->rt.p);
  k_leaf_apply<<<(unsigned)Pc->nleaf, 64, 0, s>>>(Pc->leaf_pb.p, Pc->leaf_pe.p, Pc->inv_off.p, Pc->inv.p, Pc->rt.p,
                                                  Pc->yt.p);
  k_seg_stats<<<(unsigned)Pc->nleaf, 32, 0, s>>>(Pc->leaf_pb.p, Pc->leaf_pe.p, Pc->rt.p, Pc->yt.p, Pc->seg.p);
  NetLayout Ly(net->H);
  k_net_apply<<<cdiv(N, 128), 128, sizeof(float) * Ly.n, s>>>(net->w.p, net->H, N, Pc->pt_leaf.p, Pc->seg.p,
                                                              Pc->rt.p, Pc->yt.p, Pc->zt.p);
  k_from_tree32<<<cdiv(N, 256), 256, 0, s>>>(Pc->zt.p, T->perm.p, N, z);
  FDA_LAUNCH_CHECK();
  return FDA_OK;
}

}  // namespace fda

using namespace fda;

extern "C" {

int bm_net_create(int hidden, uint64_t seed, bm_net_t** out) {
  if (!out || hidden < 1 || hidden > NET_HMAX) {
    set_error("hidden width must lie in [1, %d]", NET_HMAX);
    return FDA_E_INVALID_ARG;
  }
  bm_net_s* n = new (std::nothrow) bm_net_s();
  if (!n) return FDA_E_OOM;
  n->H = hidden;
  NetLayout Ly(hidden);
  n->nparam = Ly.n;
  std::vector<float> w(Ly.n, 0.f);
  uint64_t st = seed ? seed : 0x9e3779b97f4a7c15ull;
  auto rnd = [&]() {  // splitmix64 -> uniform(-1, 1)
    st += 0x9e3779b97f4a7c15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
  };
  for (int q = 0; q < hidden * NET_IN; ++q) w[Ly.W1 + q] = rnd() * sqrtf(3.0f / NET_IN);
  for (int q = 0; q < hidden * hidden; ++q) w[Ly.W2 + q] = rnd() * sqrtf(3.0f / hidden);
  w[Ly.b3 + 0] = 1.0f;  // identity preconditioner at start: z = r
  int rc = n->w.upload(w);
  if (rc == FDA_OK) rc = n->g.alloc(Ly.n);
  if (rc == FDA_OK) rc = n->m.alloc(Ly.n);
  if (rc == FDA_OK) rc = n->v.alloc(Ly.n);
  if (rc == FDA_OK) rc = n->m.zero();
  if (rc == FDA_OK) rc = n->v.zero();
  if (rc != FDA_OK) {
    delete n;
    return rc;
  }
  FDA_CUDA(cudaDeviceSynchronize());
  *out = n;
  return FDA_OK;
}

int bm_net_params(bm_net_t* net, float* get_host, const float* set_host, int* nparam) {
  if (!net) {
    set_error("net is NULL");
    return FDA_E_INVALID_ARG;
  }
  if (nparam) *nparam = net->nparam;
  if (set_host) FDA_CUDA(cudaMemcpy(net->w.p, set_host, sizeof(float) * net->nparam, cudaMemcpyHostToDevice));
  if (get_host) FDA_CUDA(cudaMemcpy(get_host, net->w.p, sizeof(float) * net->nparam, cudaMemcpyDeviceToHost));
  return FDA_OK;
}

void bm_net_destroy(bm_net_t* net) { delete net; }

int bm_precond_create(fda_plan_t* plan, bm_precond_t** out) {
  if (!plan || !out) {
    set_error("NULL argument");
    return FDA_E_INVALID_ARG;
  }
  *out = nullptr;
  if (plan->prob->particles || plan->cfg.op != 0) {
    set_error("the leaf-block preconditioner needs the boundary-element operator A (op = 0)");
    return FDA_E_STATE;
  }
  if (plan->cfg.drop_fp64) {
    set_error("the leaf-block preconditioner inverts the FP64 near-field blocks, which a drop_fp64 plan released");
    return FDA_E_STATE;
  }
  fda_tree_s* T = plan->tree;
  bm_precond_s* Pc = new (std::nothrow) bm_precond_s();
  if (!Pc) return FDA_E_OOM;
  Pc->plan = plan;
  // leaves that own a self block (every leaf of the near-field lists), their block offsets
  std::vector<int64_t> tleaf, tptr, src, boff;
  FDA_TRY(plan->near_tleaf.download(tleaf));
  FDA_TRY(plan->near_tptr.download(tptr));
  FDA_TRY(plan->near_src.download(src));
  FDA_TRY(plan->near_off.download(boff));
  std::vector<int64_t> lpb, lpe, selfoff, ioff;
  std::vector<int32_t> ptl(T->N, -1);
  int64_t itot = 0;
  int maxn = 0;
  for (size_t u = 0; u < tleaf.size(); ++u) {
    int64_t L = tleaf[u];
    int64_t so = -1;
    for (int64_t q = tptr[u]; q < tptr[u + 1]; ++q)
      if (src[q] == L) so = boff[q];
    int n = (int)(T->h_pe[L] - T->h_pb[L]);
    if (so < 0 || n > 64) continue;  // leaves without a self block (or oversized) keep z = r
    int32_t idx = (int32_t)lpb.size();
    lpb.push_back(T->h_pb[L]);
    lpe.push_back(T->h_pe[L]);
    selfoff.push_back(so);
    ioff.push_back(itot);
    itot += (int64_t)n * n;
    maxn = std::max(maxn, n);
    for (int64_t t = T->h_pb[L]; t < T->h_pe[L]; ++t) ptl[t] = idx;
  }
  Pc->nleaf = (int64_t)lpb.size();
  DBuf<int64_t> dself;
  int rc = FDA_OK;
  rc = Pc->leaf_pb.upload(lpb);
  if (rc == FDA_OK) rc = Pc->leaf_pe.upload(lpe);
  if (rc == FDA_OK) rc = Pc->inv_off.upload(ioff);
  if (rc == FDA_OK) rc = dself.upload(selfoff);
  if (rc == FDA_OK) rc = Pc->pt_leaf.upload(ptl);
  if (rc == FDA_OK) rc = Pc->inv.alloc(std::max<int64_t>(itot, 1));
  if (rc == FDA_OK) rc = Pc->rt.alloc(T->N);
  if (rc == FDA_OK) rc = Pc->yt.alloc(T->N);
  if (rc == FDA_OK) rc = Pc->zt.alloc(T->N);
  if (rc == FDA_OK) rc = Pc->et.alloc(T->N);
  if (rc == FDA_OK) rc = Pc->seg.alloc(2 * std::max<int64_t>(Pc->nleaf, 1));
  if (rc == FDA_OK) rc = Pc->loss_acc.alloc(2);
  if (rc != FDA_OK) {
    delete Pc;
    return rc;
  }
  if (Pc->nleaf > 0) {
    size_t sm = sizeof(double2) * (size_t)maxn * 2 * maxn;
    FDA_CUDA(cudaFuncSetAttribute(k_leaf_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(sm, 1)));
    k_leaf_inverse<<<(unsigned)Pc->nleaf, 256, sm>>>(Pc->leaf_pb.p, Pc->leaf_pe.p, dself.p, plan->op64.near.p,
                                                     Pc->inv_off.p, Pc->inv.p);
    FDA_LAUNCH_CHECK();
  }
  FDA_CUDA(cudaDeviceSynchronize());
  *out = Pc;
  return FDA_OK;
}

void bm_precond_destroy(bm_precond_t* p) { delete p; }

static __global__ void k_pair(const double2* b, const double2* ax, const double2* xs, const double2* x, int64_t N,
                              double2* r, double2* e) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  r[i] = csub(b[i], ax[i]);
  e[i] = csub(xs[i], x[i]);
}

int bm_residual_pair(fda_plan_t* plan, const void* b, const void* xstar, const void* x, void* r, void* e,
                     void* stream) {
  if (!plan || !b || !xstar || !x || !r || !e) {
    set_error("NULL argument");
    return FDA_E_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = plan->tree->N;
  FDA_TRY(plan_matvec(plan, FDA_PREC_FP64, x, r, 1, FDA_CPLX128, s, false));  // r = A x
  k_pair<<<cdiv(N, 256), 256, 0, s>>>((const double2*)b, (const double2*)r, (const double2*)xstar,
                                      (const double2*)x, N, (double2*)r, (double2*)e);
  FDA_LAUNCH_CHECK();
  FDA_CUDA(cudaStreamSynchronize(s));
  return FDA_OK;
}

int bm_fgmres_solve(fda_plan_t* plan, bm_precond_t* precond, bm_net_t* net, const void* b, void* x, int nrhs,
                    const bm_gmres_opts_t* opts, bm_gmres_stats_t* stats, void* stream) {
  if (!plan || !precond || !net || !b || !x || !opts || nrhs < 1) {
    set_error("NULL argument or nrhs < 1");
    return FDA_E_INVALID_ARG;
  }
  if (precond->plan != plan) {
    set_error("preconditioner belongs to another plan");
    return FDA_E_INVALID_ARG;
  }
  if (!(opts->tol > 0) || opts->restart < 1 || opts->max_iter < 1) {
    set_error("bad GMRES options");
    return FDA_E_INVALID_ARG;
  }
  return gmres_solve(plan, (const double2*)b, (double2*)x, nrhs, opts, stats, (cudaStream_t)stream, precond, net);
}

int bm_precond_apply(bm_precond_t* Pc, bm_net_t* net, const void* r, void* z, void* stream) {
  if (!Pc || !net || !r || !z) {
    set_error("NULL argument");
    return FDA_E_INVALID_ARG;
  }
  FDA_TRY(precond_apply(Pc, net, (const double2*)r, (double2*)z, (cudaStream_t)stream));
  FDA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return FDA_OK;
}

int bm_precond_train_step(bm_precond_t* Pc, bm_net_t* net, const void* r, const void* e, int npairs, double lr,
                          double* loss, float* grad_host, void* stream) {
  if (!Pc || !net || !r || !e || npairs < 1) {
    set_error("NULL argument or npairs < 1");
    return FDA_E_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  fda_tree_s* T = Pc->plan->tree;
  const int64_t N = T->N;
  NetLayout Ly(net->H);
  FDA_CUDA(cudaMemsetAsync(net->g.p, 0, sizeof(float) * Ly.n, s));
  FDA_CUDA(cudaMemsetAsync(Pc->loss_acc.p, 0, sizeof(float) * 2, s));
  for (int q = 0; q < npairs; ++q) {
    const double2* rq = (const double2*)r + (int64_t)q * N;
    const double2* eq = (const double2*)e + (int64_t)q * N;
    k_to_tree32<<<cdiv(N, 256), 256, 0, s>>>(rq, T->perm.p, N, Pc->rt.p);
    k_to_tree32<<<cdiv(N, 256), 256, 0, s>>>(eq, T->perm.p, N, Pc->et.p);
    k_leaf_apply<<<(unsigned)Pc->nleaf, 64, 0, s>>>(Pc->leaf_pb.p, Pc->leaf_pe.p, Pc->inv_off.p, Pc->inv.p,
                                                    Pc->rt.p, Pc->yt.p);
    k_seg_stats<<<(unsigned)Pc->nleaf, 32, 0, s>>>(Pc->leaf_pb.p, Pc->leaf_pe.p, Pc->rt.p, Pc->yt.p, Pc->seg.p);
    FDA_CUDA(cudaMemsetAsync(Pc->loss_acc.p + 1, 0, sizeof(float), s));
    k_sumsq<<<256, 256, 0, s>>>(eq, N, Pc->loss_acc.p + 1);
    float E = 0;
    FDA_CUDA(cudaMemcpyAsync(&E, Pc->loss_acc.p + 1, sizeof(float), cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    float invE = E > 0 ? 1.0f / (E * npairs) : 0.f;
    k_net_grad<<<cdiv(N, 128), 128, sizeof(float) * 2 * Ly.n, s>>>(net->w.p, net->H, N, Pc->pt_leaf.p, Pc->seg.p,
                                                                    Pc->rt.p, Pc->yt.p, Pc->et.p, invE, net->g.p,
                                                                    Pc->loss_acc.p);
    FDA_LAUNCH_CHECK();
  }
  float lh = 0;
  FDA_CUDA(cudaMemcpyAsync(&lh, Pc->loss_acc.p, sizeof(float), cudaMemcpyDeviceToHost, s));
  if (grad_host) FDA_CUDA(cudaMemcpyAsync(grad_host, net->g.p, sizeof(float) * Ly.n, cudaMemcpyDeviceToHost, s));
  if (lr > 0) {
    net->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
    k_adam<<<cdiv(Ly.n, 256), 256, 0, s>>>(net->w.p, net->g.p, net->m.p, net->v.p, Ly.n, (float)lr, b1, b2, 1e-8f,
                                          c1, c2);
    FDA_LAUNCH_CHECK();
  }
  FDA_CUDA(cudaStreamSynchronize(s));
  if (loss) *loss = lh;
  return FDA_OK;
}

}  // extern "C"
