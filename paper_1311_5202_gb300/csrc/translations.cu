// Plan builder: translation operators of the FDA for the Burton-Miller kernels and the near field.
//
// Per level l carrying representations (Sec. 3.1.2):
//   candidates (LF: cube surfaces, KIFMM style; HF: spheres around the box for the equivalent points and a
//   cone of far check points for the canonical wedge (1,0,0), rotated to the other wedges),
//   equivalent points b = columns and check points a = rows selected by pivoted QR of W G(X, Y),
//   R = W G(a, b) = U Sigma V^H truncated at sigma_i >= eps sigma_1 (Eq. svdr, invr), s = rank.
// Compressed operators (Eq. cmps..cmpt), with the Burton-Miller modifications of Sec. 3.2:
//   S~ = Sigma^-1 U^H [W dG/dn_y(a, y_j)] diag(w_j)           (Eq. evas2mh: dipole check potentials)
//   M~ = Sigma_l^-1 U_l^H [W G(a_l, b_{l+1})] V_{l+1},  L~ = M~^T (Eq. cmpl)
//   K~ = V^T G(b_target, b_source) V                          (incoming check points = outgoing equivalents)
//   T~ = [(G + alpha dG/dn_x)(x_i, a) W] conj(U) Sigma^-1       (Eq. eval2t)
//   low rank: K~ = U^ V^ by rank-revealing QR when the rank is below s/2 (Eq. lrdk).
// Near field: direct blocks K_H(x_i, y_j) w_j over the near leaf pairs and the correction matrix
// C_ij = wbar_ij - [j != i] K_H(x_i, y_j) w_j of Eq. kcorrection, both in tree order.
#include "plan.cuh"

#include <algorithm>
#include <array>
#include <chrono>
#include <map>
#include <tuple>
#include <unordered_map>

namespace fda {

struct QRJob {
  double2* A;
  int m, n, lda, kmax;
  double tol;
  int* perm;
  int* rank;
  double2* rdiag;
  double2* tau;
  double* cn;
};
struct QFormJob {
  const double2* A;
  int m, lda, r;
  const double2* tau;
  double2* Q;
  int ldq;
};
struct SVDJob {
  double2* A;
  int m, n, lda;
  double2* V;
  int ldv;
  int* sweeps;
};
int pivoted_qr_batched(const std::vector<QRJob>& jobs, cudaStream_t s);
int form_q_batched(const std::vector<QFormJob>& jobs, cudaStream_t s);
int jacobi_svd_batched(const std::vector<SVDJob>& jobs, cudaStream_t s);
int gaussian_fill(double2* out, int64_t n, uint64_t seed);

// ------------------------------------------------------------------ candidate point sets (host)
static void cube_surface(int p, double scale, std::vector<double>& out) {
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j)
      for (int k = 0; k < p; ++k) {
        if (i != 0 && i != p - 1 && j != 0 && j != p - 1 && k != 0 && k != p - 1) continue;
        out.push_back(scale * (-1.0 + 2.0 * i / (p - 1)));
        out.push_back(scale * (-1.0 + 2.0 * j / (p - 1)));
        out.push_back(scale * (-1.0 + 2.0 * k / (p - 1)));
      }
}

static void fib_sphere(int n, double r, std::vector<double>& out) {
  for (int j = 0; j < n; ++j) {
    double z = 1.0 - 2.0 * (j + 0.5) / n;
    double ph = (j + 0.5) * FDA_PI * (3.0 - sqrt(5.0));
    double s = sqrt(std::max(0.0, 1.0 - z * z));
    out.push_back(r * s * cos(ph));
    out.push_back(r * s * sin(ph));
    out.push_back(r * z);
  }
}

// unit directions in the cap of half-angle th around +x
static void fib_cap_x(int n, double th, std::vector<double>& out) {
  for (int j = 0; j < n; ++j) {
    double c = 1.0 - (1.0 - cos(th)) * (j + 0.5) / n;
    double ph = (j + 0.5) * FDA_PI * (3.0 - sqrt(5.0));
    double s = sqrt(std::max(0.0, 1.0 - c * c));
    out.push_back(c);
    out.push_back(s * cos(ph));
    out.push_back(s * sin(ph));
  }
}

static void wedge_center(int n, int wid, double* d) {
  int face = wid / (n * n), cell = wid % (n * n);
  int a = face / 2, sg = face % 2;
  int c1 = cell / n, c2 = cell % n;
  int o1 = (a == 0) ? 1 : 0, o2 = (a == 2) ? 1 : 2;
  d[a] = sg == 0 ? 1.0 : -1.0;
  d[o1] = -1.0 + (2.0 * c1 + 1.0) / n;
  d[o2] = -1.0 + (2.0 * c2 + 1.0) / n;
  double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int q = 0; q < 3; ++q) d[q] /= l;
}

// rotation taking e_x to d (Rodrigues); pi about e_z for d = -e_x
static void rot_x_to(const double* d, double* R) {
  double c = d[0];
  if (c > 1 - 1e-15) {
    double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    memcpy(R, I, sizeof(I));
    return;
  }
  if (c < -1 + 1e-15) {
    double Z[9] = {-1, 0, 0, 0, -1, 0, 0, 0, 1};
    memcpy(R, Z, sizeof(Z));
    return;
  }
  double ax[3] = {0, -d[2], d[1]};  // e_x x d
  double sn = sqrt(ax[1] * ax[1] + ax[2] * ax[2]);
  for (int q = 0; q < 3; ++q) ax[q] /= sn;
  double K[9] = {0, -ax[2], ax[1], ax[2], 0, -ax[0], -ax[1], ax[0], 0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int q = 0; q < 3; ++q) s += K[3 * i + q] * K[3 * q + j];
      K2[3 * i + j] = s;
    }
  for (int q = 0; q < 9; ++q) R[q] = (q % 4 == 0 ? 1.0 : 0.0) + sn * K[q] + (1 - c) * K2[q];
}

static double cell_half_angle(int n) {
  double best = 0;
  for (int wid = 0; wid < n * n; ++wid) {
    double c[3];
    wedge_center(n, wid, c);
    int c1 = wid / n, c2 = wid % n;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        double q[3] = {1.0, -1.0 + 2.0 * (c1 + a) / n, -1.0 + 2.0 * (c2 + b) / n};
        double l = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        double d = (q[0] * c[0] + q[1] * c[1] + q[2] * c[2]) / l;
        best = std::max(best, acos(std::min(1.0, d)));
      }
  }
  return best;
}

// parent-level wedge z -> child-level wedge (nested face cells; 0 when the child level is LF)
static int child_wedge(const LevelOps& Lp, const LevelOps& Lc, int z) {
  if (!Lc.hf) return 0;
  int n = Lp.n, nc = Lc.n;
  int face = z / (n * n), cell = z % (n * n);
  int c1 = cell / n, c2 = cell % n;
  return face * nc * nc + (c1 / 2) * nc + (c2 / 2);
}

// ------------------------------------------------------------------ kernel-matrix generators
struct PtSet {
  const double* p;  // canonical points (count x 3)
  const double* rot;  // 9 or nullptr
  double c[3];      // centre shift
};

__device__ __forceinline__ void pt_get(const PtSet& S, int i, double* out) {
  const double* q = S.p + 3 * i;
  if (S.rot) {
    const double* R = S.rot;
    out[0] = R[0] * q[0] + R[1] * q[1] + R[2] * q[2] + S.c[0];
    out[1] = R[3] * q[0] + R[4] * q[1] + R[5] * q[2] + S.c[1];
    out[2] = R[6] * q[0] + R[7] * q[1] + R[8] * q[2] + S.c[2];
  } else {
    out[0] = q[0] + S.c[0];
    out[1] = q[1] + S.c[1];
    out[2] = q[2] + S.c[2];
  }
}

__device__ __forceinline__ double2 greens(const double* x, const double* y, double k) {
  double r0 = x[0] - y[0], r1 = x[1] - y[1], r2 = x[2] - y[2];
  double R = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
  double sn, cs;
  sincos(k * R, &sn, &cs);
  double g = 0.25 / FDA_PI / R;
  return make_double2(g * cs, g * sn);
}

// out[i + j m] = W_i G(X_i, Y_j) for one batch item per blockIdx.y
struct GJob {
  PtSet X, Y;
  const double* W;
  int m, n;
  double2* out;
  int ld;
};
static __global__ void k_gen_G(const GJob* jobs, double k) {
  const GJob J = jobs[blockIdx.y];
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)J.m * J.n;
       q += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(q % J.m), j = (int)(q / J.m);
    double x[3], y[3];
    pt_get(J.X, i, x);
    pt_get(J.Y, j, y);
    double2 g = greens(x, y, k);
    if (J.W) g = cscale(g, J.W[i]);
    J.out[i + (int64_t)j * J.ld] = g;
  }
}

static int gen_G(const std::vector<GJob>& jobs, double k) {
  if (jobs.empty()) return FDA_OK;
  DBuf<GJob> dj;
  FDA_TRY(dj.upload(jobs));
  for (size_t b0 = 0; b0 < jobs.size(); b0 += 65535) {
    unsigned nb = (unsigned)std::min<size_t>(65535, jobs.size() - b0);
    k_gen_G<<<dim3(64, nb), 256>>>(dj.p + b0, k);
    FDA_LAUNCH_CHECK();
  }
  return FDA_OK;
}

// E_up (S2M) : out[i + j sc] = W_i dG/dn_y(c + R a_i, y_j) w_j, zero for j >= nC (pad to ncol)
// E_dn (L2T) : out[j + i nrow] = (G + alpha dG/dn_x)(x_j, c + R a_i) W_i, zero rows j >= nC
struct LeafJob {
  PtSet A;      // check points around the leaf centre (rotated for the wedge)
  const double* W;
  int sc;
  int64_t pbeg;  // first tree position of the leaf
  int nC;
  double2* out;
};
static __global__ void k_gen_leaf(const LeafJob* jobs, const double* xt, const double* nt, const double* wt,
                                  double k, double2 alpha, int ncol, int mode, int particles, int op, double2 gamma) {
  const LeafJob J = jobs[blockIdx.y];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < J.sc * ncol; q += gridDim.x * blockDim.x) {
    int i = q % J.sc, j = q / J.sc;
    double2 v = make_double2(0, 0);
    if (j < J.nC) {
      double a[3];
      pt_get(J.A, i, a);
      int64_t p = J.pbeg + j;
      const double* y = xt + 3 * p;
      const double* ny = nt + 3 * p;
      if (mode == 0) {
        // dG/dn_y(a, y) with r = a - y; particle sums: (G + alpha dG/dn_y)(a, y) (Eq. sum)
        double dummy[3] = {0, 0, 0};
        KernVals K = helmholtz4(a, dummy, y, ny, k);
        // operator B: monopole sources (S + alpha M); A + gamma B (Robin data): dipole + gamma monopole
        const double2 src = op == 2 ? cadd(K.Dy, cmul(gamma, K.G)) : (op ? K.G : K.Dy);
        v = particles ? cscale(cadd(K.G, cmul(alpha, K.Dy)), J.W[i] * wt[p]) : cscale(src, J.W[i] * wt[p]);
        J.out[i + (int64_t)j * J.sc] = v;
      } else {
        // (G + alpha dG/dn_x)(x, a) with r = x - a; particle sums: G(x, a)
        double dummy[3] = {0, 0, 0};
        KernVals K = helmholtz4(y, ny, a, dummy, k);
        v = particles ? cscale(K.G, J.W[i]) : cscale(cadd(K.G, cmul(alpha, K.Dx)), J.W[i]);
        J.out[j + (int64_t)i * ncol] = v;
      }
    } else {
      if (mode == 0)
        J.out[i + (int64_t)j * J.sc] = v;
      else
        J.out[j + (int64_t)i * ncol] = v;
    }
  }
}

// compact [ld x ncols] blocks to [rows x cols] (column-major) at the given offsets
struct CopyJob {
  const double2* src;
  int ld, rows, cols;
  double2* dst;
};
static __global__ void k_compact(const CopyJob* jobs) {
  const CopyJob J = jobs[blockIdx.y];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < J.rows * J.cols; q += gridDim.x * blockDim.x) {
    int i = q % J.rows, j = q / J.rows;
    J.dst[q] = J.src[i + (int64_t)j * J.ld];
  }
}

static __global__ void k_conj_copy(const double2* a, double2* b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = conjc(a[i]);
}

// V^ (r x s) from the pivoted-QR output: V^[:, perm[j]] = R[:, j], R upper trapezoidal
static __global__ void k_build_vhat(const double2* A, int lda, const double2* rdiag, const int* perm, int r, int s,
                                    double2* vh) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < r * s; q += gridDim.x * blockDim.x) {
    int i = q % r, j = q / r;
    double2 v = make_double2(0, 0);
    if (j == i)
      v = rdiag[i];
    else if (j > i)
      v = A[i + (int64_t)j * lda];
    vh[i + (int64_t)perm[j] * r] = v;
  }
}

// near blocks: one CTA per block, entries column-major (rows = target points)
struct NearJob {
  int64_t tb, te, sb, se;  // target / source tree-position ranges
  int64_t off;
};
static __global__ void k_gen_near(const NearJob* jobs, const double* xt, const double* nt, const double* wt, double k,
                                  double2 alpha, double2* out, int particles, int op, double2 gamma) {
  const NearJob J = jobs[blockIdx.x];
  int64_t nr = J.te - J.tb, nc = J.se - J.sb;
  for (int64_t q = threadIdx.x; q < nr * nc; q += blockDim.x) {
    int64_t i = J.tb + q % nr, j = J.sb + q / nr;
    double2 v = make_double2(0, 0);
    if (i != j) {
      KernVals K = helmholtz4(xt + 3 * i, nt + 3 * i, xt + 3 * j, nt + 3 * j, k);
      const double2 ka = cadd(K.Dy, cmul(alpha, K.H)), kb = cadd(K.G, cmul(alpha, K.Dx));
      v = particles ? cscale(cadd(K.G, cmul(alpha, K.Dy)), wt[j])
                    : cscale(op == 2 ? cadd(ka, cmul(gamma, kb)) : (op ? kb : ka), wt[j]);
    }
    out[J.off + q] = v;
  }
}

static __global__ void k_permute_geom(const double* x, const double* n, const double* w, const int64_t* perm,
                                      int64_t N, double* xt, double* nt, double* wt, int64_t* iperm) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  int64_t i = perm[t];
  for (int d = 0; d < 3; ++d) {
    xt[3 * t + d] = x[3 * i + d];
    nt[3 * t + d] = n[3 * i + d];
  }
  wt[t] = w[i];
  iperm[i] = t;
}

// corrections to tree order
static __global__ void k_corr_counts(const int64_t* perm, const int64_t* di_ptr, int64_t N, int64_t* cnt) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  int64_t i = perm[t];
  cnt[t] = 6 * (di_ptr[i + 1] - di_ptr[i]);
}
static __global__ void k_corr_scatter(const int64_t* perm, const int64_t* iperm, const int64_t* di_ptr,
                                      const int32_t* di_cols, const double2* corr, const int64_t* rowptr, int64_t N,
                                      int32_t* col, double2* val) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  int64_t i = perm[t];
  int64_t o = rowptr[t];
  for (int64_t p = di_ptr[i]; p < di_ptr[i + 1]; ++p) {
    int64_t e = di_cols[p];
    for (int g = 0; g < 6; ++g) {
      col[o] = (int32_t)iperm[6 * e + g];
      val[o] = corr[6 * p + g];
      ++o;
    }
  }
}

// Fold correction entries whose column lies in the row's direct blocks into those blocks; flag the rest.
static __global__ void k_merge_corr(const int64_t* cptr, const int32_t* ccol, const double2* cval,
                                    const int32_t* row_leaf, const int64_t* tleaf, const int64_t* tptr,
                                    const int64_t* srcbox, const int64_t* boff, const int64_t* pb, const int64_t* pe,
                                    int64_t N, double2* near, int64_t* keep_cnt, int8_t* keep) {
  int64_t ti = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ti >= N) return;
  int u = row_leaf[ti];
  int64_t kept = 0;
  for (int64_t p = cptr[ti]; p < cptr[ti + 1]; ++p) {
    int64_t j = ccol[p];
    bool done = false;
    if (u >= 0) {
      int64_t L = tleaf[u], tb = pb[L], nr = pe[L] - tb;
      for (int64_t q = tptr[u]; q < tptr[u + 1]; ++q) {
        int64_t Q = srcbox[q], sb = pb[Q], se = pe[Q];
        if (j >= sb && j < se) {
          int64_t idx = boff[q] + (j - sb) * nr + (ti - tb);
          near[idx] = cadd(near[idx], cval[p]);
          done = true;
          break;
        }
      }
    }
    keep[p] = done ? 0 : 1;
    kept += done ? 0 : 1;
  }
  keep_cnt[ti] = kept;
}

static __global__ void k_compact_corr(const int64_t* cptr, const int32_t* ccol, const double2* cval,
                                      const int8_t* keep, const int64_t* nptr, int64_t N, int32_t* ncol,
                                      double2* nval) {
  int64_t ti = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ti >= N) return;
  int64_t o = nptr[ti];
  for (int64_t p = cptr[ti]; p < cptr[ti + 1]; ++p)
    if (keep[p]) {
      ncol[o] = ccol[p];
      nval[o] = cval[p];
      ++o;
    }
}

template <typename A, typename B>
static __global__ void k_convert(const A* a, B* b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = from_d<B>(to_d(a[i]));
}

template <typename C>
static int to_fp32(const DBuf<double2>& a, DBuf<C>& b) {
  FDA_TRY(b.alloc(a.n));
  if (a.n) {
    k_convert<double2, C><<<cdiv(a.n, 256), 256>>>(a.p, b.p, (int64_t)a.n);
    FDA_LAUNCH_CHECK();
  }
  return FDA_OK;
}

// Tensor maps of the TMA-fed V^ kernel: for every level whose V^ stage has swapped-kernel units, the level's
// outgoing coefficient vectors of the first right-hand side (boxes consecutive in the tree, nw vectors of s
// complex values each) as a 2-D FP32 tensor of 2 s columns. A level whose map cannot be encoded keeps the
// other V^ kernels.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static int build_vtm_maps(fda_plan_s* P) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f)
      return FDA_OK;  // no tensor maps: the TMA-fed kernel stays unused
    encode = (EncodeTiledFn)f;
  }
  for (int l = 0; l < FDA_MAXLEV; ++l) {
    P->vtm_ok[l] = false;
    const LevelOps& L = P->lev[l];
    if (P->h_vsw_units[l].empty() || !L.used || L.s <= 0 || (L.s & 1)) continue;
    const int64_t b0 = L.box_begin, b1 = L.box_end;
    if (b1 <= b0 || P->h_slot[b0] < 0) continue;
    const int64_t base = P->h_slot[b0];
    const int64_t nvec = (b1 - b0) * L.nw;
    if (nvec >= ((int64_t)1 << 31)) continue;
    void* addr = P->cout32.p + base;
    if ((reinterpret_cast<uintptr_t>(addr) & 15) != 0) continue;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * L.s), (cuuint64_t)nvec};
    const cuuint64_t strides[1] = {(cuuint64_t)(8 * L.s)};
    const cuuint32_t box[2] = {32, 1};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(&P->vtm_map[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, addr, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
      P->vtm_ok[l] = true;
      P->vtm_base[l] = base;
    }
  }
  return FDA_OK;
}

static double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------------ plan build
int plan_build(fda_tree_s* T, const fda_config_t* cfg, fda_plan_s* P) {
  bm_problem_s* pr = T->prob;
  const double k = pr->k, eps = cfg->eps;
  const double2 alpha = pr->alpha;
  P->tree = T;
  P->prob = pr;
  P->cfg = *cfg;
  P->near_csep = cfg->near_split;  // 0, 1 or 2 (checked at the entry point)
  P->near_form = cfg->near_form;
  if (P->cfg.nrhs_max < 1) P->cfg.nrhs_max = 1;
  FDA_TRY(upload_geometry_constants());
  const int64_t N = T->N, nbox = T->nbox;
  double t0 = now_ms();

  // tree-order geometry
  DBuf<double> xt, nt, wt;
  FDA_TRY(xt.alloc(3 * N));
  FDA_TRY(nt.alloc(3 * N));
  FDA_TRY(wt.alloc(N));
  FDA_TRY(P->iperm.alloc(N));
  k_permute_geom<<<cdiv(N, 256), 256>>>(pr->x.p, pr->n.p, pr->w.p, T->perm.p, N, xt.p, nt.p, wt.p, P->iperm.p);
  FDA_LAUNCH_CHECK();

  // levels carrying representations
  int lmin = FDA_MAXLEV, lmax = T->nlev - 1;
  for (int64_t q = 0; q < T->nm2l; ++q) lmin = std::min(lmin, T->h_m2l_info[6 * q]);
  const bool far = T->nm2l > 0;
  if (!far) lmin = lmax + 1;
  P->lmin = lmin;
  P->lmax = lmax;
  std::vector<int64_t> lb(T->nlev + 1, nbox);
  for (int64_t b = nbox - 1; b >= 0; --b) lb[T->h_lev[b]] = b;
  for (int l = T->nlev - 1; l >= 0; --l)
    if (lb[l] == nbox) lb[l] = lb[l + 1];
  std::vector<double> cen(3 * nbox);
  for (int64_t b = 0; b < nbox; ++b) {
    double w = ldexp(T->side, -T->h_lev[b]);
    cen[3 * b] = T->corner[0] + w * (T->h_ix[b] + 0.5);
    cen[3 * b + 1] = T->corner[1] + w * (T->h_iy[b] + 0.5);
    cen[3 * b + 2] = T->corner[2] + w * (T->h_iz[b] + 0.5);
  }

  // ---- 1. point selection and SVD per level
  struct Cand {
    std::vector<double> Y, X, W;
    DBuf<double> dY, dX, dW;
    DBuf<double2> A, A2, R, V;
    DBuf<int> perm, perm2, rank;
    DBuf<double2> rd, tau, rd2, tau2;
    DBuf<double> cn, cn2;
    DBuf<int> sweeps;
  };
  std::vector<Cand> cand(FDA_MAXLEV);
  std::vector<int> qlev;
  const double lam = 2 * FDA_PI / k;
  if (far) {
    for (int l = lmin; l <= lmax; ++l) {
      LevelOps& L = P->lev[l];
      Cand& C = cand[l];
      L.used = true;
      L.hf = T->hf[l] != 0;
      L.n = T->nw[l];
      L.nw = L.hf ? 6 * L.n * L.n : 1;
      L.w = ldexp(T->side, -l);
      L.box_begin = lb[l];
      L.box_end = lb[l + 1];
      double h = 0.5 * L.w;
      int p_ext = std::max(0, (int)ceil(2.0 * k * L.w / FDA_PI));  // resolve oscillation across the box
      int pe = std::max(eps < 5e-6 ? 10 : 8, std::min(16, 6 + p_ext));
      if (!L.hf) {
        cube_surface(pe, 1.05 * h, C.Y);
        cube_surface(std::max(5, pe - 3), 0.6 * h, C.Y);
        cube_surface(pe + 2, 2.95 * h, C.X);
        C.W.assign(C.X.size() / 3, 1.0);
      } else {
        double rad = 1.05 * sqrt(3.0) * h;
        int ne = (int)(2.0 * (k * rad + 8) * (k * rad + 8));
        fib_sphere(ne, rad, C.Y);
        fib_sphere(std::max(50, ne / 3), 0.6 * rad, C.Y);
        int Tl = T->T[l];
        double th = cell_half_angle(L.n) + asin(sqrt(3.0) / (2.0 * (Tl + 2))) + 0.05;
        th = std::min(th, FDA_PI);
        double rmin = 0.98 * (Tl + 1.5) * L.w;
        int nd = (int)(2.0 * (1 - cos(th)) / 2.0 * (k * rad + 8) * (k * rad + 8)) + 40;
        std::vector<double> dirs;
        fib_cap_x(nd, th, dirs);
        const double radii[7] = {1, 1.3, 1.8, 2.6, 4, 8, 20};
        for (double rr : radii)
          for (int j = 0; j < nd; ++j) {
            for (int d = 0; d < 3; ++d) C.X.push_back(rr * rmin * dirs[3 * j + d]);
            C.W.push_back(rr * rmin / L.w);
          }
        L.rot.resize(9 * L.nw);
        for (int z = 0; z < L.nw; ++z) {
          double d[3];
          wedge_center(L.n, z, d);
          rot_x_to(d, &L.rot[9 * z]);
        }
      }
      if (!L.hf) {
        L.rot = {1, 0, 0, 0, 1, 0, 0, 0, 1};
      }
      (void)lam;
      int m = (int)(C.X.size() / 3), n = (int)(C.Y.size() / 3);
      FDA_TRY(C.dY.upload(C.Y));
      FDA_TRY(C.dX.upload(C.X));
      FDA_TRY(C.dW.upload(C.W));
      FDA_TRY(C.A.alloc((size_t)m * n));
      FDA_TRY(C.perm.alloc(n));
      FDA_TRY(C.rank.alloc(2));
      FDA_TRY(C.rd.alloc(n));
      FDA_TRY(C.tau.alloc(n));
      FDA_TRY(C.cn.alloc(n));
      GJob g;
      g.X = {C.dX.p, nullptr, {0, 0, 0}};
      g.Y = {C.dY.p, nullptr, {0, 0, 0}};
      g.W = C.dW.p;
      g.m = m;
      g.n = n;
      g.out = C.A.p;
      g.ld = m;
      FDA_TRY(gen_G({g}, k));
      qlev.push_back(l);
    }
    // Equivalent points: a randomized interpolative decomposition of the candidate matrix A = W G(X, Y).
    // A Gaussian sketch S = Omega A (ell x n, ell << m) keeps A's column space, and the column-pivoted QR of
    // S to tolerance 0.1 eps selects the columns; a sketch whose rank comes within 8 of ell is redrawn with
    // twice the rows (up to m), so that the selection never saturates the sketch.
    std::vector<int> ell(qlev.size()), done(qlev.size(), 0);
    for (size_t q = 0; q < qlev.size(); ++q) {
      const Cand& C = cand[qlev[q]];
      const int m = (int)(C.X.size() / 3), n = (int)(C.Y.size() / 3);
      ell[q] = std::min(std::min(m, n), 256);
    }
    std::vector<DBuf<double2>> Om(qlev.size()), Sk(qlev.size());
    for (int round = 0; round < 8; ++round) {
      std::vector<QRJob> qj;
      std::vector<size_t> which;
      for (size_t q = 0; q < qlev.size(); ++q) {
        if (done[q]) continue;
        Cand& C = cand[qlev[q]];
        const int m = (int)(C.X.size() / 3), n = (int)(C.Y.size() / 3), e = ell[q];
        FDA_TRY(Om[q].alloc((size_t)e * m));
        FDA_TRY(Sk[q].alloc((size_t)e * n));
        FDA_TRY(gaussian_fill(Om[q].p, (int64_t)e * m, 0x5EEDull + 7919ull * (uint64_t)qlev[q] + 104729ull * round));
        DBuf<const double2*> da, db;
        DBuf<double2*> dc;
        const double2* ha[1] = {Om[q].p};
        const double2* hb[1] = {C.A.p};
        double2* hc[1] = {Sk[q].p};
        FDA_TRY(da.upload(ha, 1));
        FDA_TRY(db.upload(hb, 1));
        FDA_TRY(dc.upload(hc, 1));
        FDA_TRY(zgemm_batched('N', 'N', e, n, m, make_double2(1, 0), da.p, e, db.p, m, make_double2(0, 0), dc.p, e, 1,
                              0));
        FDA_CUDA(cudaDeviceSynchronize());
        QRJob qq;
        qq.A = Sk[q].p;
        qq.m = e;
        qq.n = n;
        qq.lda = e;
        qq.kmax = std::min(e, n);
        qq.tol = 0.1 * eps;
        qq.perm = C.perm.p;
        qq.rank = C.rank.p;
        qq.rdiag = C.rd.p;
        qq.tau = C.tau.p;
        qq.cn = C.cn.p;
        qj.push_back(qq);
        which.push_back(q);
      }
      if (qj.empty()) break;
      FDA_TRY(pivoted_qr_batched(qj, 0));
      for (size_t u = 0; u < which.size(); ++u) {
        const size_t q = which[u];
        Cand& C = cand[qlev[q]];
        const int m = (int)(C.X.size() / 3), n = (int)(C.Y.size() / 3);
        int rk = 0;
        FDA_CUDA(cudaMemcpy(&rk, C.rank.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (rk < ell[q] - 8 || ell[q] >= std::min(m, n)) {
          done[q] = 1;
        } else {
          ell[q] = std::min(std::min(m, n), 2 * ell[q]);
        }
      }
    }
    for (size_t q = 0; q < qlev.size(); ++q) {
      Om[q].release();
      Sk[q].release();
    }
    // selected equivalent points -> row selection on (W G(X, b))^H
    std::vector<QRJob> qjobs2;
    for (int l : qlev) {
      LevelOps& L = P->lev[l];
      Cand& C = cand[l];
      int rk = 0;
      FDA_CUDA(cudaMemcpy(&rk, C.rank.p, sizeof(int), cudaMemcpyDeviceToHost));
      std::vector<int> pm;
      FDA_TRY(C.perm.download(pm));
      L.se = rk;
      L.b.resize(3 * rk);
      for (int j = 0; j < rk; ++j)
        for (int d = 0; d < 3; ++d) L.b[3 * j + d] = C.Y[3 * pm[j] + d];
      FDA_TRY(L.d_b.upload(L.b));
      int m = (int)(C.X.size() / 3);
      // A2 = (W G(X, b))^H  : rk x m  -> generate G(b, X) W (rows b) then conj
      FDA_TRY(C.A2.alloc((size_t)rk * m));
      GJob g;
      g.X = {L.d_b.p, nullptr, {0, 0, 0}};
      g.Y = {C.dX.p, nullptr, {0, 0, 0}};
      g.W = nullptr;
      g.m = rk;
      g.n = m;
      g.out = C.A2.p;
      g.ld = rk;
      FDA_TRY(gen_G({g}, k));
      // scale column j by W_j and conjugate: (W G(X,b))^H [j-th col] = conj(W_j G(b, X_j))
      {
        std::vector<double2> dummy;
        (void)dummy;
      }
      FDA_TRY(C.perm2.alloc(m));
      FDA_TRY(C.rd2.alloc(m));
      FDA_TRY(C.tau2.alloc(m));
      FDA_TRY(C.cn2.alloc(m));
      QRJob q;
      q.A = C.A2.p;
      q.m = rk;
      q.n = m;
      q.lda = rk;
      q.kmax = std::min(rk, m);
      q.tol = 0.1 * eps;
      q.perm = C.perm2.p;
      q.rank = C.rank.p + 1;
      q.rdiag = C.rd2.p;
      q.tau = C.tau2.p;
      q.cn = C.cn2.p;
      qjobs2.push_back(q);
    }
    // weights on the columns of the transposed problem: multiply column j by W_j (conjugation does not
    // change pivoting or norms)
    for (size_t q = 0; q < qlev.size(); ++q) {
      Cand& C = cand[qlev[q]];
      int rk = qjobs2[q].m, m = qjobs2[q].n;
      std::vector<double2> h((size_t)rk * m);
      FDA_CUDA(cudaMemcpy(h.data(), C.A2.p, h.size() * sizeof(double2), cudaMemcpyDeviceToHost));
      for (int j = 0; j < m; ++j)
        for (int i = 0; i < rk; ++i) h[i + (size_t)j * rk] = cscale(h[i + (size_t)j * rk], C.W[j]);
      FDA_CUDA(cudaMemcpy(C.A2.p, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice));
    }
    FDA_TRY(pivoted_qr_batched(qjobs2, 0));
    // R = W_a G(a, b) and its SVD
    std::vector<SVDJob> sjobs;
    for (size_t q = 0; q < qlev.size(); ++q) {
      int l = qlev[q];
      LevelOps& L = P->lev[l];
      Cand& C = cand[l];
      int rk2 = 0;
      FDA_CUDA(cudaMemcpy(&rk2, C.rank.p + 1, sizeof(int), cudaMemcpyDeviceToHost));
      std::vector<int> pm;
      FDA_TRY(C.perm2.download(pm));
      L.sc = rk2;
      L.a.resize(3 * rk2);
      L.Wa.resize(rk2);
      for (int i = 0; i < rk2; ++i) {
        for (int d = 0; d < 3; ++d) L.a[3 * i + d] = C.X[3 * pm[i] + d];
        L.Wa[i] = C.W[pm[i]];
      }
      FDA_TRY(L.d_a.upload(L.a));
      FDA_TRY(L.d_Wa.upload(L.Wa));
      FDA_TRY(L.d_rot.upload(L.rot));
      FDA_TRY(C.R.alloc((size_t)L.sc * L.se));
      FDA_TRY(C.V.alloc((size_t)L.se * L.se));
      FDA_TRY(C.sweeps.alloc(1));
      GJob g;
      g.X = {L.d_a.p, nullptr, {0, 0, 0}};
      g.Y = {L.d_b.p, nullptr, {0, 0, 0}};
      g.W = L.d_Wa.p;
      g.m = L.sc;
      g.n = L.se;
      g.out = C.R.p;
      g.ld = L.sc;
      FDA_TRY(gen_G({g}, k));
      SVDJob sj;
      sj.A = C.R.p;
      sj.m = L.sc;
      sj.n = L.se;
      sj.lda = L.sc;
      sj.V = C.V.p;
      sj.ldv = L.se;
      sj.sweeps = C.sweeps.p;
      sjobs.push_back(sj);
    }
    const double t_svd0 = now_ms();
    FDA_TRY(jacobi_svd_batched(sjobs, 0));
    P->setup_ms[1] = now_ms() - t_svd0;
    for (size_t q = 0; q < qlev.size(); ++q) {
      int l = qlev[q];
      LevelOps& L = P->lev[l];
      Cand& C = cand[l];
      std::vector<double2> hR, hV;
      FDA_TRY(C.R.download(hR));
      FDA_TRY(C.V.download(hV));
      std::vector<double> sg(L.se);
      for (int j = 0; j < L.se; ++j) {
        double s2 = 0;
        for (int i = 0; i < L.sc; ++i) s2 += cabs2(hR[i + (size_t)j * L.sc]);
        sg[j] = sqrt(s2);
      }
      std::vector<int> ord(L.se);
      for (int j = 0; j < L.se; ++j) ord[j] = j;
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sg[a] > sg[b]; });
      double s1 = sg[ord[0]];
      int s = 0;
      while (s < L.se && s < L.sc && sg[ord[s]] >= eps * s1) ++s;
      // an even rank keeps every coefficient vector 16-byte aligned (two complex FP32 values per vector
      // atomic in the tensor-core epilogue); the extra singular vector only adds accuracy
      if ((s & 1) && s < L.se && s < L.sc) ++s;
      L.s = s;
      L.sigma.resize(s);
      std::vector<double2> Ph((size_t)L.sc * s), Pch((size_t)L.sc * s), Vh((size_t)L.se * s);
      for (int c = 0; c < s; ++c) {
        int j = ord[c];
        double sj = sg[j];
        L.sigma[c] = sj;
        for (int i = 0; i < L.sc; ++i) {
          double2 u = cscale(hR[i + (size_t)j * L.sc], 1.0 / sj);  // u_c
          Ph[i + (size_t)c * L.sc] = cscale(u, 1.0 / sj);            // U Sigma^-1
          Pch[i + (size_t)c * L.sc] = conjc(Ph[i + (size_t)c * L.sc]);
        }
        for (int i = 0; i < L.se; ++i) Vh[i + (size_t)c * L.se] = hV[i + (size_t)j * L.se];
      }
      FDA_TRY(L.P.upload(Ph));
      FDA_TRY(L.Pc.upload(Pch));
      FDA_TRY(L.V.upload(Vh));
    }
  }
  double t1 = now_ms();
  P->setup_ms[0] = t1 - t0 - P->setup_ms[1];

  // ---- 2. coefficient slots
  P->h_slot.assign(nbox, -1);
  int64_t off = 0;
  if (far)
    for (int64_t b = lb[lmin]; b < nbox; ++b) {
      const LevelOps& L = P->lev[T->h_lev[b]];
      P->h_slot[b] = off;
      off += (int64_t)L.nw * L.s;
    }
  P->n_coef = off;
  FDA_TRY(P->slot.upload(P->h_slot));

  // ---- 3. leaf operators S~ and T~
  std::vector<int64_t> s_off, t_off;
  int64_t s_tot = 0, t_tot = 0;
  if (far) {
    for (int64_t b = lb[lmin]; b < nbox; ++b)
      if (T->h_leaf[b]) P->h_leaves.push_back(b);
    s_off.resize(P->h_leaves.size());
    t_off.resize(P->h_leaves.size());
    for (size_t q = 0; q < P->h_leaves.size(); ++q) {
      int64_t b = P->h_leaves[q];
      const LevelOps& L = P->lev[T->h_lev[b]];
      int64_t nC = T->h_pe[b] - T->h_pb[b];
      s_off[q] = s_tot;
      t_off[q] = t_tot;
      s_tot += (int64_t)L.nw * L.s * nC;
      t_tot += (int64_t)L.nw * L.s * nC;
      P->bytes_s2m_l2t += 2.0 * L.nw * L.s * nC * 16.0;
    }
  }
  FDA_TRY(P->leaves.upload(P->h_leaves));
  FDA_TRY(P->leaf_s_off.upload(s_off));
  FDA_TRY(P->leaf_t_off.upload(t_off));
  FDA_TRY(P->op64.S.alloc(std::max<int64_t>(s_tot, 1)));
  FDA_TRY(P->op64.T.alloc(std::max<int64_t>(t_tot, 1)));
  if (far) {
    // batches per level and wedge
    for (int l = lmin; l <= lmax; ++l) {
      LevelOps& L = P->lev[l];
      std::vector<size_t> items;
      int ncol = 1;
      for (size_t q = 0; q < P->h_leaves.size(); ++q)
        if (T->h_lev[P->h_leaves[q]] == l) {
          items.push_back(q);
          ncol = std::max<int>(ncol, (int)(T->h_pe[P->h_leaves[q]] - T->h_pb[P->h_leaves[q]]));
        }
      if (items.empty()) continue;
      const int64_t BATCH = 2048;
      DBuf<double2> E, Out;
      FDA_TRY(E.alloc((size_t)BATCH * L.sc * ncol));
      FDA_TRY(Out.alloc((size_t)BATCH * L.s * ncol));
      for (int mode = 0; mode < 2; ++mode)
        for (size_t i0 = 0; i0 < items.size() * L.nw; i0 += BATCH) {
          size_t nb = std::min<size_t>(BATCH, items.size() * L.nw - i0);
          std::vector<LeafJob> lj(nb);
          std::vector<const double2*> Ap(nb), Bp(nb);
          std::vector<double2*> Cp(nb);
          std::vector<CopyJob> cj(nb);
          for (size_t u = 0; u < nb; ++u) {
            size_t it = (i0 + u) / L.nw;
            int z = (int)((i0 + u) % L.nw);
            int64_t b = P->h_leaves[items[it]];
            LeafJob& J = lj[u];
            J.A.p = L.d_a.p;
            J.A.rot = L.d_rot.p + 9 * z;
            for (int d = 0; d < 3; ++d) J.A.c[d] = cen[3 * b + d];
            J.W = L.d_Wa.p;
            J.sc = L.sc;
            J.pbeg = T->h_pb[b];
            J.nC = (int)(T->h_pe[b] - T->h_pb[b]);
            J.out = E.p + u * (size_t)L.sc * ncol;
            Cp[u] = Out.p + u * (size_t)L.s * ncol;
            if (mode == 0) {
              Ap[u] = L.P.p;   // op C
              Bp[u] = J.out;   // sc x ncol
            } else {
              Ap[u] = J.out;   // ncol x sc
              Bp[u] = L.Pc.p;  // sc x s
            }
            int64_t nC = J.nC;
            if (mode == 0)
              cj[u] = {Cp[u], L.s, L.s, (int)nC, P->op64.S.p + s_off[items[it]] + (int64_t)z * L.s * nC};
            else
              cj[u] = {Cp[u], ncol, (int)nC, L.s, P->op64.T.p + t_off[items[it]] + (int64_t)z * L.s * nC};
          }
          DBuf<LeafJob> dlj;
          FDA_TRY(dlj.upload(lj));
          k_gen_leaf<<<dim3(16, (unsigned)nb), 256>>>(dlj.p, xt.p, nt.p, wt.p, k, alpha, ncol, mode,
                                                      pr->particles, P->cfg.op,
                                                      make_double2(P->cfg.gamma_re, P->cfg.gamma_im));
          FDA_LAUNCH_CHECK();
          DBuf<const double2*> dA, dB;
          DBuf<double2*> dC;
          FDA_TRY(dA.upload(Ap));
          FDA_TRY(dB.upload(Bp));
          FDA_TRY(dC.upload(Cp));
          if (mode == 0)
            FDA_TRY(zgemm_batched('C', 'N', L.s, ncol, L.sc, make_double2(1, 0), dA.p, L.sc, dB.p, L.sc,
                                  make_double2(0, 0), dC.p, L.s, nb, 0));
          else
            FDA_TRY(zgemm_batched('N', 'N', ncol, L.s, L.sc, make_double2(1, 0), dA.p, ncol, dB.p, L.sc,
                                  make_double2(0, 0), dC.p, ncol, nb, 0));
          DBuf<CopyJob> dcj;
          FDA_TRY(dcj.upload(cj));
          k_compact<<<dim3(8, (unsigned)nb), 256>>>(dcj.p);
          FDA_LAUNCH_CHECK();
          FDA_CUDA(cudaDeviceSynchronize());
        }
    }
  }
  double t2 = now_ms();
  P->setup_ms[2] = t2 - t1;

  // ---- 4. M~ per (level, octant, wedge)
  int64_t m_tot = 0;
  for (int l = lmin; l < lmax; ++l) {
    P->m_off[l] = m_tot;
    m_tot += 8LL * P->lev[l].nw * P->lev[l].s * P->lev[l + 1].s;
  }
  FDA_TRY(P->op64.M.alloc(std::max<int64_t>(m_tot, 1)));
  for (int l = lmin; l < lmax && far; ++l) {
    LevelOps& L = P->lev[l];
    LevelOps& Lc = P->lev[l + 1];
    for (int64_t b = L.box_begin; b < L.box_end; ++b)
      if (!T->h_leaf[b]) P->h_parents[l].push_back(b);
    FDA_TRY(P->parents[l].upload(P->h_parents[l]));
    int nitem = 8 * L.nw;
    const int BATCH = 256;
    DBuf<double2> G, S1;
    FDA_TRY(G.alloc((size_t)BATCH * L.sc * Lc.se));
    FDA_TRY(S1.alloc((size_t)BATCH * L.s * Lc.se));
    for (int i0 = 0; i0 < nitem; i0 += BATCH) {
      int nb = std::min(BATCH, nitem - i0);
      std::vector<GJob> gj(nb);
      std::vector<const double2*> A1(nb), B1(nb), A2(nb), B2(nb);
      std::vector<double2*> C1(nb), C2(nb);
      for (int u = 0; u < nb; ++u) {
        int o = (i0 + u) / L.nw, z = (i0 + u) % L.nw;
        int zc = child_wedge(L, Lc, z);
        double dl[3] = {(((o >> 2) & 1) - 0.5) * 0.5 * L.w, (((o >> 1) & 1) - 0.5) * 0.5 * L.w,
                        ((o & 1) - 0.5) * 0.5 * L.w};
        GJob& g = gj[u];
        g.X = {L.d_a.p, L.d_rot.p + 9 * z, {0, 0, 0}};
        g.Y = {Lc.d_b.p, Lc.d_rot.p + 9 * zc, {dl[0], dl[1], dl[2]}};
        g.W = L.d_Wa.p;
        g.m = L.sc;
        g.n = Lc.se;
        g.out = G.p + (size_t)u * L.sc * Lc.se;
        g.ld = L.sc;
        A1[u] = L.P.p;
        B1[u] = g.out;
        C1[u] = S1.p + (size_t)u * L.s * Lc.se;
        A2[u] = C1[u];
        B2[u] = Lc.V.p;
        C2[u] = P->op64.M.p + P->m_off[l] + (int64_t)(o * L.nw + z) * L.s * Lc.s;
      }
      FDA_TRY(gen_G(gj, k));
      DBuf<const double2*> dA1, dB1, dA2, dB2;
      DBuf<double2*> dC1, dC2;
      FDA_TRY(dA1.upload(A1));
      FDA_TRY(dB1.upload(B1));
      FDA_TRY(dC1.upload(C1));
      FDA_TRY(dA2.upload(A2));
      FDA_TRY(dB2.upload(B2));
      FDA_TRY(dC2.upload(C2));
      FDA_TRY(zgemm_batched('C', 'N', L.s, Lc.se, L.sc, make_double2(1, 0), dA1.p, L.sc, dB1.p, L.sc,
                            make_double2(0, 0), dC1.p, L.s, nb, 0));
      FDA_TRY(zgemm_batched('N', 'N', L.s, Lc.s, Lc.se, make_double2(1, 0), dA2.p, L.s, dB2.p, Lc.se,
                            make_double2(0, 0), dC2.p, L.s, nb, 0));
      FDA_CUDA(cudaDeviceSynchronize());
    }
    // algorithmic flops: M2M + L2L, every parent box x wedge x child
    for (int64_t b : P->h_parents[l]) P->flops_m2m += 2.0 * 8.0 * L.nw * T->h_nch[b] * (double)L.s * Lc.s;
  }
  double t3 = now_ms();
  P->setup_ms[3] = t3 - t2;

  // ---- 5. K~ per (level, offset); M2L schedule
  struct OffInfo {
    int32_t dx, dy, dz, wo, wi;
    int64_t count;
    int64_t k_off;   // dense K~ offset, or -1
    int64_t u_off, v_off;  // low-rank U^, V^ offsets
    int rank;
  };
  std::vector<std::vector<OffInfo>> offs(FDA_MAXLEV);
  std::vector<int32_t> pair_off(T->nm2l);
  for (int l = 0; l < FDA_MAXLEV; ++l) {
    std::map<std::tuple<int, int, int>, int> idx;
    for (int64_t q = 0; q < T->nm2l; ++q) {
      const int32_t* inf = &T->h_m2l_info[6 * q];
      if (inf[0] != l) continue;
      auto key = std::make_tuple(inf[1], inf[2], inf[3]);
      auto it = idx.find(key);
      int id;
      if (it == idx.end()) {
        id = (int)offs[l].size();
        idx[key] = id;
        offs[l].push_back({inf[1], inf[2], inf[3], inf[4], inf[5], 0, -1, -1, -1, 0});
      } else {
        id = it->second;
      }
      offs[l][id].count++;
      pair_off[q] = id;
      P->m2l_pairs[l]++;
    }
    P->m2l_offsets[l] = (int64_t)offs[l].size();
  }
  int64_t k_tot = 0;
  for (int l = lmin; l <= lmax && far; ++l)
    for (auto& o : offs[l]) {
      o.k_off = k_tot;
      k_tot += (int64_t)P->lev[l].s * P->lev[l].s;
    }
  FDA_TRY(P->op64.K.alloc(std::max<int64_t>(k_tot, 1)));
  for (int l = lmin; l <= lmax && far; ++l) {
    LevelOps& L = P->lev[l];
    int no = (int)offs[l].size();
    if (!no) continue;
    const int BATCH = 128;
    DBuf<double2> G, T1;
    FDA_TRY(G.alloc((size_t)BATCH * L.se * L.se));
    FDA_TRY(T1.alloc((size_t)BATCH * L.se * L.s));
    for (int i0 = 0; i0 < no; i0 += BATCH) {
      int nb = std::min(BATCH, no - i0);
      std::vector<GJob> gj(nb);
      std::vector<const double2*> A1(nb), B1(nb), A2(nb), B2(nb);
      std::vector<double2*> C1(nb), C2(nb);
      for (int u = 0; u < nb; ++u) {
        const OffInfo& o = offs[l][i0 + u];
        GJob& g = gj[u];
        g.X = {L.d_b.p, L.d_rot.p + 9 * (L.hf ? o.wi : 0), {0, 0, 0}};
        g.Y = {L.d_b.p, L.d_rot.p + 9 * (L.hf ? o.wo : 0), {o.dx * L.w, o.dy * L.w, o.dz * L.w}};
        g.W = nullptr;
        g.m = L.se;
        g.n = L.se;
        g.out = G.p + (size_t)u * L.se * L.se;
        g.ld = L.se;
        A1[u] = g.out;
        B1[u] = L.V.p;
        C1[u] = T1.p + (size_t)u * L.se * L.s;
        A2[u] = L.V.p;
        B2[u] = C1[u];
        C2[u] = P->op64.K.p + o.k_off;
      }
      FDA_TRY(gen_G(gj, k));
      DBuf<const double2*> dA1, dB1, dA2, dB2;
      DBuf<double2*> dC1, dC2;
      FDA_TRY(dA1.upload(A1));
      FDA_TRY(dB1.upload(B1));
      FDA_TRY(dC1.upload(C1));
      FDA_TRY(dA2.upload(A2));
      FDA_TRY(dB2.upload(B2));
      FDA_TRY(dC2.upload(C2));
      FDA_TRY(zgemm_batched('N', 'N', L.se, L.s, L.se, make_double2(1, 0), dA1.p, L.se, dB1.p, L.se,
                            make_double2(0, 0), dC1.p, L.se, nb, 0));
      FDA_TRY(zgemm_batched('T', 'N', L.s, L.s, L.se, make_double2(1, 0), dA2.p, L.se, dB2.p, L.se,
                            make_double2(0, 0), dC2.p, L.s, nb, 0));
      FDA_CUDA(cudaDeviceSynchronize());
    }
  }
  double t4 = now_ms();
  P->setup_ms[4] = t4 - t3;

  // ---- 6. low-rank factors of K~ (Sec. 4.2)
  int64_t lr_tot = 0;
  if (cfg->lowrank && far) {
    for (int l = lmin; l <= lmax; ++l) {
      LevelOps& L = P->lev[l];
      int no = (int)offs[l].size();
      if (!no || L.s < 4) continue;
      const int BATCH = 512;
      int kmax = (L.s + 1) / 2;
      DBuf<double2> W, rd, tau;
      DBuf<int> perm, rank;
      DBuf<double> cn;
      FDA_TRY(W.alloc((size_t)BATCH * L.s * L.s));
      FDA_TRY(rd.alloc((size_t)BATCH * kmax));
      FDA_TRY(tau.alloc((size_t)BATCH * kmax));
      FDA_TRY(perm.alloc((size_t)BATCH * L.s));
      FDA_TRY(rank.alloc(BATCH));
      FDA_TRY(cn.alloc((size_t)BATCH * L.s));
      for (int i0 = 0; i0 < no; i0 += BATCH) {
        int nb = std::min(BATCH, no - i0);
        std::vector<QRJob> qj(nb);
        for (int u = 0; u < nb; ++u) {
          FDA_CUDA(cudaMemcpy(W.p + (size_t)u * L.s * L.s, P->op64.K.p + offs[l][i0 + u].k_off,
                              sizeof(double2) * L.s * L.s, cudaMemcpyDeviceToDevice));
          QRJob& q = qj[u];
          q.A = W.p + (size_t)u * L.s * L.s;
          q.m = L.s;
          q.n = L.s;
          q.lda = L.s;
          q.kmax = kmax;
          q.tol = 0.5 * eps;
          q.perm = perm.p + (size_t)u * L.s;
          q.rank = rank.p + u;
          q.rdiag = rd.p + (size_t)u * kmax;
          q.tau = tau.p + (size_t)u * kmax;
          q.cn = cn.p + (size_t)u * L.s;
        }
        FDA_TRY(pivoted_qr_batched(qj, 0));
        std::vector<int> rk(nb);
        FDA_CUDA(cudaMemcpy(rk.data(), rank.p, sizeof(int) * nb, cudaMemcpyDeviceToHost));
        // allocate low-rank storage (grow pool)
        std::vector<QFormJob> fj;
        std::vector<std::pair<int, int>> which;
        int64_t need = 0;
        for (int u = 0; u < nb; ++u)
          if (2 * rk[u] < L.s) need += 2LL * rk[u] * L.s;
        if (need) {
          DBuf<double2>& pool = P->op64.lr;
          size_t newn = lr_tot + need;
          if (newn > pool.n) {
            double2* np = nullptr;
            size_t cap = std::max(newn, 2 * pool.n);
            if (cudaMalloc((void**)&np, cap * sizeof(double2)) != cudaSuccess) {
              set_error("low-rank pool allocation failed");
              return FDA_E_OOM;
            }
            if (lr_tot) FDA_CUDA(cudaMemcpy(np, pool.p, lr_tot * sizeof(double2), cudaMemcpyDeviceToDevice));
            pool.release();
            pool.p = np;
            pool.n = cap;
          }
        }
        for (int u = 0; u < nb; ++u) {
          OffInfo& o = offs[l][i0 + u];
          if (!(2 * rk[u] < L.s) || rk[u] < 1) continue;
          o.rank = rk[u];
          o.u_off = lr_tot;
          o.v_off = lr_tot + (int64_t)rk[u] * L.s;
          lr_tot += 2LL * rk[u] * L.s;
          QFormJob f;
          f.A = W.p + (size_t)u * L.s * L.s;
          f.m = L.s;
          f.lda = L.s;
          f.r = rk[u];
          f.tau = tau.p + (size_t)u * kmax;
          f.Q = P->op64.lr.p + o.u_off;
          f.ldq = L.s;
          fj.push_back(f);
          k_build_vhat<<<32, 256>>>(W.p + (size_t)u * L.s * L.s, L.s, rd.p + (size_t)u * kmax,
                                    perm.p + (size_t)u * L.s, rk[u], L.s, P->op64.lr.p + o.v_off);
          FDA_LAUNCH_CHECK();
          P->m2l_lowrank[l]++;
        }
        FDA_TRY(form_q_batched(fj, 0));
      }
    }
  }
  // the low-rank pool grew by doubling: trim it to the factors it holds
  if (P->op64.lr.n > (size_t)std::max<int64_t>(lr_tot, 1)) {
    DBuf<double2> lr;
    FDA_TRY(lr.alloc(std::max<int64_t>(lr_tot, 1)));
    if (lr_tot) FDA_CUDA(cudaMemcpy(lr.p, P->op64.lr.p, sizeof(double2) * lr_tot, cudaMemcpyDeviceToDevice));
    std::swap(P->op64.lr.p, lr.p);
    std::swap(P->op64.lr.n, lr.n);
  }
  // keep the dense K~ only for the offsets without a low-rank form: the products read U^ and V^ for the others
  {
    int64_t keep = 0;
    std::vector<CopyJob> cj;
    for (int l = lmin; l <= lmax && far; ++l)
      for (auto& o : offs[l]) {
        if (o.rank > 0) continue;
        const int sl = P->lev[l].s;
        cj.push_back({P->op64.K.p + o.k_off, sl, sl, sl, nullptr});
        o.k_off = keep;
        keep += (int64_t)sl * sl;
      }
    for (int l = lmin; l <= lmax && far; ++l)
      for (auto& o : offs[l])
        if (o.rank > 0) o.k_off = -1;
    DBuf<double2> Kd;
    FDA_TRY(Kd.alloc(std::max<int64_t>(keep, 1)));
    {
      int64_t o2 = 0;
      for (auto& j : cj) {
        j.dst = Kd.p + o2;
        o2 += (int64_t)j.rows * j.cols;
      }
    }
    if (!cj.empty()) {
      DBuf<CopyJob> dcj;
      FDA_TRY(dcj.upload(cj));
      for (size_t b0 = 0; b0 < cj.size(); b0 += 65535) {
        k_compact<<<dim3(16, (unsigned)std::min<size_t>(65535, cj.size() - b0)), 256>>>(dcj.p + b0);
        FDA_LAUNCH_CHECK();
      }
      FDA_CUDA(cudaDeviceSynchronize());
    }
    std::swap(P->op64.K.p, Kd.p);
    std::swap(P->op64.K.n, Kd.n);
  }
  double t5 = now_ms();
  P->setup_ms[5] = t5 - t4;

  // M2L pairs grouped by (level, offset) and units
  {
    std::vector<int64_t> order(T->nm2l);
    for (int64_t q = 0; q < T->nm2l; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
      int la = T->h_m2l_info[6 * a], lb2 = T->h_m2l_info[6 * b];
      if (la != lb2) return la < lb2;
      return pair_off[a] < pair_off[b];
    });
    std::vector<int64_t> ps(T->nm2l), pt(T->nm2l), pm(T->nm2l, -1);
    int64_t mid = 0;
    for (int64_t u = 0; u < T->nm2l; ++u) {
      int64_t q = order[u];
      const int32_t* inf = &T->h_m2l_info[6 * q];
      int l = inf[0];
      const LevelOps& L = P->lev[l];
      int64_t tb = T->h_m2l_box[2 * q], sb = T->h_m2l_box[2 * q + 1];
      ps[u] = P->h_slot[sb] + (int64_t)(L.hf ? inf[4] : 0) * L.s;
      pt[u] = P->h_slot[tb] + (int64_t)(L.hf ? inf[5] : 0) * L.s;
      const OffInfo& o = offs[l][pair_off[q]];
      if (o.rank > 0) {
        pm[u] = mid;
        mid += (o.rank + 1) & ~1;  // even stride: every intermediate vector starts 16-byte aligned
      }
      double fl = o.rank > 0 ? 16.0 * o.rank * L.s : 8.0 * L.s * L.s;
      P->flops_m2l += fl;
      P->m2l_flops_lev[l] += fl;
    }
    for (int l = 0; l < FDA_MAXLEV; ++l)
      for (const OffInfo& o : offs[l])
        P->m2l_op_bytes_lev[l] += 16.0 * (o.rank > 0 ? 2.0 * o.rank * P->lev[l].s : (double)P->lev[l].s * P->lev[l].s);
    P->n_pairs = T->nm2l;
    P->n_mid = mid;
    FDA_TRY(P->pair_src.upload(ps));
    FDA_TRY(P->pair_tgt.upload(pt));
    FDA_TRY(P->pair_mid.upload(pm));
    // FMA units: row tile per (level, stage) minimising the padded rows (plus a per-tile gather cost); the
    // low-rank V^ stage has as many rows as the rank, often below 20
    for (int l = 0; l < FDA_MAXLEV; ++l) {
      P->fma_tm[l][0] = P->fma_tm[l][1] = 64;
      if (offs[l].empty() || !P->lev[l].used) continue;
      double best = 1e300;
      for (int tm : {16, 32, 64}) {
        double c = 0;
        for (const OffInfo& o : offs[l]) {
          const int M = o.rank > 0 ? o.rank : P->lev[l].s;
          c += (double)o.count * ((M + tm - 1) / tm) * (tm + 16);
        }
        if (c < best) best = c, P->fma_tm[l][0] = tm;
      }
    }
    int64_t u = 0;
    while (u < T->nm2l) {
      int64_t q = order[u];
      int l = T->h_m2l_info[6 * q];
      int id = pair_off[q];
      int64_t v = u;
      while (v < T->nm2l && T->h_m2l_info[6 * order[v]] == l && pair_off[order[v]] == id) ++v;
      const OffInfo& o = offs[l][id];
      const LevelOps& L = P->lev[l];
      const int TM0 = P->fma_tm[l][0], TM1 = P->fma_tm[l][1];
      const int CP = std::max(64, 2048 / TM0);  // pairs per unit: fills the stage-0 column tile at nrhs = 1
      for (int64_t p0 = u; p0 < v; p0 += CP) {
        int pc = (int)std::min<int64_t>(CP, v - p0);
        // tensor-core units: up to 256 output rows each
        if (o.rank > 0) {
          for (int m0 = 0; m0 < o.rank; m0 += 256) {
            P->h_tc_units[l][0].push_back({o.v_off, o.rank, L.s, p0, pc, m0, 1, 0});
            P->tc_max_rows[l][0] = std::max(P->tc_max_rows[l][0], std::min(256, o.rank - m0));
          }
          for (int m0 = 0; m0 < L.s; m0 += 256) {
            P->h_tc_units[l][1].push_back({o.u_off, L.s, o.rank, p0, pc, m0, 2, 0});
            P->tc_max_rows[l][1] = std::max(P->tc_max_rows[l][1], std::min(256, L.s - m0));
          }
        } else {
          for (int m0 = 0; m0 < L.s; m0 += 256) {
            P->h_tc_units[l][0].push_back({o.k_off, L.s, L.s, p0, pc, m0, 0, 0});
            P->tc_max_rows[l][0] = std::max(P->tc_max_rows[l][0], std::min(256, L.s - m0));
          }
        }
        if (o.rank > 0) {
          for (int m0 = 0; m0 < o.rank; m0 += TM0)
            P->h_units[l][0].push_back({o.v_off, o.rank, L.s, p0, pc, m0, 1, 0});
          for (int m0 = 0; m0 < L.s; m0 += TM1)
            P->h_units[l][1].push_back({o.u_off, L.s, o.rank, p0, pc, m0, 2, 0});
        } else {
          for (int m0 = 0; m0 < L.s; m0 += TM0) P->h_units[l][0].push_back({o.k_off, L.s, L.s, p0, pc, m0, 0, 0});
        }
      }
      u = v;
    }
    for (int l = 0; l < FDA_MAXLEV; ++l)
      for (int st = 0; st < 2; ++st) {
        FDA_TRY(P->units[l][st].upload(P->h_units[l][st]));
        FDA_TRY(P->tc_units[l][st].upload(P->h_tc_units[l][st]));
      }
    // tensor-core (TF32) form: every operator pre-expanded into its shared-memory image, units of up to
    // 128 pairs that cover all output rows
    if ((P->cfg.m2l_tensor == 1 || P->cfg.m2l_tensor == 3) && P->cfg.precision == FDA_PREC_FP32) {
      std::vector<TcImgJob> jobs;
      int64_t img_tot = 0;
      const int split = P->cfg.m2l_tensor == 3 ? 1 : 0;  // 3xTF32: each image followed by its remainders
      auto add_img = [&](const double2* src, int M, int K, int64_t ld, int trans) {
        int64_t off = img_tot;
        jobs.push_back({src, M, K, off, ld, trans, split});
        img_tot += tc3_image_floats(M, K) * (split ? 2 : 1);
        return off;
      };
      std::vector<std::vector<std::array<int64_t, 3>>> img_of(FDA_MAXLEV);  // (k, v, u) image offsets
      for (int l = lmin; l <= lmax && far; ++l) {
        img_of[l].resize(offs[l].size());
        const int sl = P->lev[l].s;
        for (size_t i = 0; i < offs[l].size(); ++i) {
          const OffInfo& o = offs[l][i];
          auto add = [&](const double2* src, int M, int K) { return add_img(src, M, K, M, 0); };
          if (o.rank > 0) {
            img_of[l][i] = {-1, add(P->op64.lr.p + o.v_off, o.rank, sl), add(P->op64.lr.p + o.u_off, sl, o.rank)};
          } else {
            img_of[l][i] = {add(P->op64.K.p + o.k_off, sl, sl), -1, -1};
          }
        }
      }
      // M2M and L2L as grouped products on the same kernel: one group per (level, octant, parent wedge) with
      // operator M~(o, z) (child wedge -> parent wedge, Eq. cmpm) and its plain transpose (parent wedge ->
      // child wedge, Eq. cmpl), and one "pair" per parent that has a child in octant o
      std::vector<int64_t> mms, mmt, lls, llt;
      for (int l = lmin; l < lmax && far; ++l) {
        const LevelOps& L = P->lev[l];
        const LevelOps& Lc = P->lev[l + 1];
        if (P->h_parents[l].empty() || (2 * L.s + 127) / 128 > 4 || (2 * Lc.s + 127) / 128 > 4) continue;
        std::vector<std::vector<std::pair<int64_t, int64_t>>> byo(8);  // (parent, child)
        for (int64_t pb : P->h_parents[l])
          for (int c = 0; c < T->h_nch[pb]; ++c) {
            const int64_t cb = T->h_cbeg[pb] + c;
            const int o = ((T->h_ix[cb] & 1) << 2) | ((T->h_iy[cb] & 1) << 1) | (T->h_iz[cb] & 1);
            byo[o].push_back({pb, cb});
          }
        for (int o = 0; o < 8; ++o) {
          if (byo[o].empty()) continue;
          for (int z = 0; z < L.nw; ++z) {
            const double2* Mz = P->op64.M.p + P->m_off[l] + (int64_t)(o * L.nw + z) * L.s * Lc.s;
            const int zc = child_wedge(L, Lc, z);
            const int64_t im = add_img(Mz, L.s, Lc.s, L.s, 0);
            const int64_t il = add_img(Mz, Lc.s, L.s, L.s, 1);
            const int64_t p0 = (int64_t)mms.size();
            for (const auto& pc : byo[o]) {
              const int64_t child = P->h_slot[pc.second] + (int64_t)zc * Lc.s;
              const int64_t parent = P->h_slot[pc.first] + (int64_t)z * L.s;
              mms.push_back(child);
              mmt.push_back(parent);
              lls.push_back(parent);
              llt.push_back(child);
            }
            const int64_t np = (int64_t)byo[o].size();
            for (int64_t c0 = 0; c0 < np; c0 += 128) {
              const int pc = (int)std::min<int64_t>(128, np - c0);
              P->h_mm_units[l].push_back({im, L.s, Lc.s, p0 + c0, pc, 0, 0, 0});
              P->h_ll_units[l].push_back({il, Lc.s, L.s, p0 + c0, pc, 0, 0, 0});
            }
          }
        }
        P->mm_mt[l] = (2 * L.s + 127) / 128;
        P->ll_mt[l] = (2 * Lc.s + 127) / 128;
      }
      FDA_TRY(P->mm_src.upload(mms));
      FDA_TRY(P->mm_tgt.upload(mmt));
      FDA_TRY(P->ll_src.upload(lls));
      FDA_TRY(P->ll_tgt.upload(llt));
      for (int l = 0; l < FDA_MAXLEV; ++l) {
        FDA_TRY(P->mm_units[l].upload(P->h_mm_units[l]));
        FDA_TRY(P->ll_units[l].upload(P->h_ll_units[l]));
      }
      FDA_TRY(P->tc_img.alloc(std::max<int64_t>(img_tot, 1)));
      FDA_TRY(tc3_build_images(jobs, P->tc_img.p));
      const int CP3 = 128;
      int64_t u3 = 0;
      while (u3 < T->nm2l) {
        int64_t q = order[u3];
        int l = T->h_m2l_info[6 * q];
        int id = pair_off[q];
        int64_t v = u3;
        while (v < T->nm2l && T->h_m2l_info[6 * order[v]] == l && pair_off[order[v]] == id) ++v;
        const OffInfo& o = offs[l][id];
        const int sl = P->lev[l].s;
        if (o.rank > 0 && 2 * o.rank <= 64 && (sl & 1) == 0 && (2 * sl + 127) / 128 <= 4) {
          for (int64_t p0 = u3; p0 < v; p0 += 512) {
            const int pc = (int)std::min<int64_t>(512, v - p0);
            P->h_ws_units[l].push_back({img_of[l][id][2], sl, o.rank, p0, pc, 0, 2, 0});
            P->ws_mt[l] = std::max(P->ws_mt[l], (2 * sl + 127) / 128);
          }
        }
        for (int64_t p0 = u3; p0 < v; p0 += CP3) {
          int pc = (int)std::min<int64_t>(CP3, v - p0);
          if (o.rank > 0) {
            P->h_tc3_units[l][0].push_back({img_of[l][id][1], o.rank, sl, p0, pc, 0, 1, 0});
            P->h_tc3_units[l][1].push_back({img_of[l][id][2], sl, o.rank, p0, pc, 0, 2, 0});
            P->tc3_mt[l][0] = std::max(P->tc3_mt[l][0], (2 * o.rank + 127) / 128);
            P->tc3_mt[l][1] = std::max(P->tc3_mt[l][1], (2 * sl + 127) / 128);
            P->tc3_maxk[l][0] = std::max(P->tc3_maxk[l][0], sl);
            P->tc3_maxk[l][1] = std::max(P->tc3_maxk[l][1], o.rank);
          } else {
            P->h_tc3_units[l][0].push_back({img_of[l][id][0], sl, sl, p0, pc, 0, 0, 0});
            P->tc3_mt[l][0] = std::max(P->tc3_mt[l][0], (2 * sl + 127) / 128);
            P->tc3_maxk[l][0] = std::max(P->tc3_maxk[l][0], sl);
          }
        }
        u3 = v;
      }
      // short-K units (K fits two 32-wide real chunks) first: they run as a separate single-stage launch
      for (int l = 0; l < FDA_MAXLEV; ++l)
        for (int st = 0; st < 2; ++st) {
          auto& v = P->h_tc3_units[l][st];
          auto mid_it = std::stable_partition(v.begin(), v.end(), [](const GemmUnit& u) { return 2 * u.K <= 64; });
          P->tc3_split[l][st] = (int64_t)(mid_it - v.begin());
          FDA_TRY(P->tc3_units[l][st].upload(v));
        }
      // the same stage-0 units for the swapped V^ kernel (mode 1, by TMEM class of round16(2 r)) and the dense
      // ones beside it (mode 0)
      for (int l = 0; l < FDA_MAXLEV; ++l) {
        auto cls = [](const GemmUnit& u) {
          const int nm = ((2 * u.M + 15) / 16) * 16;
          return nm <= 32 ? 0 : nm <= 64 ? 1 : nm <= 128 ? 2 : 3;
        };
        std::vector<GemmUnit> byc[4];
        for (const GemmUnit& u : P->h_tc3_units[l][0]) {
          if (u.mode == 1 && 2 * u.M <= 256) {
            byc[cls(u)].push_back(u);
          } else {
            P->h_dn_units[l].push_back(u);
            P->dn_mt[l] = std::max(P->dn_mt[l], (2 * u.M + 127) / 128);
            P->dn_maxk[l] = std::max(P->dn_maxk[l], u.K);
          }
        }
        for (int c = 0; c < 4; ++c) {
          P->vsw_cls[l][c] = (int64_t)P->h_vsw_units[l].size();
          P->h_vsw_units[l].insert(P->h_vsw_units[l].end(), byc[c].begin(), byc[c].end());
        }
        P->vsw_cls[l][4] = (int64_t)P->h_vsw_units[l].size();
        FDA_TRY(P->vsw_units[l].upload(P->h_vsw_units[l]));
        FDA_TRY(P->dn_units[l].upload(P->h_dn_units[l]));
        FDA_TRY(P->ws_units[l].upload(P->h_ws_units[l]));
      }
    }
  }

  // ---- 7. near field: corrections (Eq. kcorrection) and direct blocks
  {
    DBuf<int64_t> di_ptr;
    DBuf<int32_t> di_cols;
    DBuf<double2> corr;
    double ms = 0;
    if (pr->particles) {
      // particle sums: plain kernel values everywhere, no locally corrected weights
      FDA_TRY(di_ptr.alloc(N + 1));
      FDA_TRY(di_ptr.zero());
      FDA_TRY(di_cols.alloc(1));
      FDA_TRY(corr.alloc(6));
      P->diag_c = make_double2(0.0, 0.0);
    } else {
      const double2 gamma = make_double2(P->cfg.gamma_re, P->cfg.gamma_im);
      FDA_TRY(near_corrections(pr, di_ptr, di_cols, corr, &ms, P->cfg.op, gamma));
      // operator A: 1/2 I + Dbar + alpha Hbar; operator B (radiation data): Sbar + alpha Mbar - alpha/2 I;
      // Robin data: A + gamma B, diagonal 1/2 - gamma alpha/2
      const double2 half_alpha = make_double2(-0.5 * pr->alpha.x, -0.5 * pr->alpha.y);
      P->diag_c = P->cfg.op == 2 ? cadd(make_double2(0.5, 0.0), cmul(gamma, half_alpha))
                                 : (P->cfg.op ? half_alpha : make_double2(0.5, 0.0));
    }
    P->setup_ms[6] = ms;
    DBuf<int64_t> cnt;
    FDA_TRY(cnt.alloc(N));
    k_corr_counts<<<cdiv(N, 256), 256>>>(T->perm.p, di_ptr.p, N, cnt.p);
    FDA_LAUNCH_CHECK();
    FDA_TRY(P->corr_ptr.alloc(N + 1));
    int64_t tot = 0;
    FDA_TRY(exclusive_scan_i64(cnt.p, P->corr_ptr.p, N, &tot, 0));
    FDA_CUDA(cudaMemcpy(P->corr_ptr.p + N, &tot, sizeof(int64_t), cudaMemcpyHostToDevice));
    P->corr_entries = tot;
    FDA_TRY(P->corr_col.alloc(std::max<int64_t>(tot, 1)));
    FDA_TRY(P->op64.corr.alloc(std::max<int64_t>(tot, 1)));
    k_corr_scatter<<<cdiv(N, 256), 256>>>(T->perm.p, P->iperm.p, di_ptr.p, di_cols.p, corr.p, P->corr_ptr.p, N,
                                          P->corr_col.p, P->op64.corr.p);
    FDA_LAUNCH_CHECK();
    FDA_CUDA(cudaDeviceSynchronize());
  }
  double t6 = now_ms();
  {
    // expand direct pairs to leaf targets; group by target leaf
    std::vector<std::pair<int64_t, int64_t>> blocks;
    for (int64_t q = 0; q < T->ndir; ++q) {
      int64_t Pb = T->h_direct[2 * q], Qb = T->h_direct[2 * q + 1];
      if (T->h_leaf[Pb]) {
        blocks.push_back({Pb, Qb});
      } else {
        std::vector<int64_t> st{Pb};
        while (!st.empty()) {
          int64_t b = st.back();
          st.pop_back();
          if (T->h_leaf[b])
            blocks.push_back({b, Qb});
          else
            for (int c = T->h_nch[b] - 1; c >= 0; --c) st.push_back(T->h_cbeg[b] + c);
        }
      }
    }
    std::sort(blocks.begin(), blocks.end());
    // Each target leaf's blocks form one column-major matrix whose first entry is 4-entry aligned (32 B in
    // FP32), so the streaming kernel can fetch it with bulk copies; the gaps are zero.
    std::vector<int64_t> tleaf, tptr, src, boff, coff, nbase, xbase;
    std::vector<int32_t> ncolv, xcol;
    std::vector<NearJob> jobs;
    int64_t eoff = 0, ccur = 0, entries = 0;
    int max_nr = 0;
    for (size_t q = 0; q < blocks.size(); ++q) {
      int64_t L = blocks[q].first, Q = blocks[q].second;
      if (q == 0 || L != blocks[q - 1].first) {
        if (q > 0) ncolv.push_back((int32_t)ccur);
        eoff = (eoff + 3) & ~(int64_t)3;
        tleaf.push_back(L);
        tptr.push_back((int64_t)q);
        nbase.push_back(eoff);
        xbase.push_back((int64_t)xcol.size());
        ccur = 0;
        max_nr = std::max(max_nr, (int)(T->h_pe[L] - T->h_pb[L]));
      }
      src.push_back(Q);
      boff.push_back(eoff);
      coff.push_back(ccur);
      for (int64_t j = T->h_pb[Q]; j < T->h_pe[Q]; ++j) xcol.push_back((int32_t)j);
      ccur += T->h_pe[Q] - T->h_pb[Q];
      jobs.push_back({T->h_pb[L], T->h_pe[L], T->h_pb[Q], T->h_pe[Q], eoff});
      int64_t ne = (T->h_pe[L] - T->h_pb[L]) * (T->h_pe[Q] - T->h_pb[Q]);
      eoff += ne;
      entries += ne;
    }
    if (!blocks.empty()) ncolv.push_back((int32_t)ccur);
    tptr.push_back((int64_t)blocks.size());
    xbase.push_back((int64_t)xcol.size());
    const int64_t alloc_entries = ((eoff + 3) & ~(int64_t)3) + 4;
    P->n_near_tleaf = (int64_t)tleaf.size();
    P->n_blocks = (int64_t)blocks.size();
    P->near_entries = entries;
    P->near_max_nr = max_nr;
    // balanced partition of the target leaves over the streaming kernel's persistent CTAs
    {
      int dev = 0, nsm = 1;
      FDA_CUDA(cudaGetDevice(&dev));
      FDA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      const int64_t nt = (int64_t)tleaf.size();
      std::vector<int64_t> cost(nt + 1, 0);
      for (int64_t u = 0; u < nt; ++u) {
        int64_t nr = T->h_pe[tleaf[u]] - T->h_pb[tleaf[u]];
        cost[u + 1] = cost[u] + nr * ncolv[u] + 64 * nr + 256;  // entries + per-row and per-leaf overheads
      }
      auto partition = [&](int per_sm, int* grid_out, DBuf<int32_t>& dpart) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(per_sm * (int64_t)nsm, nt));
        std::vector<int32_t> part(grid + 1, 0);
        int64_t u = 0;
        for (int b = 1; b < grid; ++b) {
          int64_t target = cost[nt] * b / grid;
          while (u < nt && cost[u + 1] <= target) ++u;
          part[b] = (int32_t)u;
        }
        part[grid] = (int32_t)nt;
        *grid_out = grid;
        return dpart.upload(part);
      };
      // three CTAs per SM alone; two or one when the far field runs beside it on the side stream
      FDA_TRY(partition(3, &P->near_grid, P->near_part));
      FDA_TRY(partition(2, &P->near_grid_ov[0], P->near_part_ov[0]));
      FDA_TRY(partition(1, &P->near_grid_ov[1], P->near_part_ov[1]));
    }
    FDA_TRY(P->near_tleaf.upload(tleaf));
    FDA_TRY(P->near_tptr.upload(tptr));
    FDA_TRY(P->near_src.upload(src));
    FDA_TRY(P->near_off.upload(boff));
    FDA_TRY(P->near_coff.upload(coff));
    FDA_TRY(P->near_nbase.upload(nbase));
    FDA_TRY(P->near_ncol.upload(ncolv));
    FDA_TRY(P->near_xbase.upload(xbase));
    FDA_TRY(P->near_xcol.upload(xcol));
    {
      std::vector<NsMeta> meta(tleaf.size());
      for (size_t u = 0; u < tleaf.size(); ++u) {
        meta[u].tb = T->h_pb[tleaf[u]];
        meta[u].xb = xbase[u];
        meta[u].nb = nbase[u];
        meta[u].nr = (int32_t)(T->h_pe[tleaf[u]] - T->h_pb[tleaf[u]]);
        meta[u].ncol = ncolv[u];
      }
      FDA_TRY(P->near_meta.upload(meta));
    }
    FDA_TRY(P->op64.near.alloc(alloc_entries));
    FDA_TRY(P->op64.near.zero());
    DBuf<NearJob> dj;
    FDA_TRY(dj.upload(jobs));
    for (size_t b0 = 0; b0 < jobs.size(); b0 += 65535) {
      unsigned nb = (unsigned)std::min<size_t>(65535, jobs.size() - b0);
      k_gen_near<<<nb, 256>>>(dj.p + b0, xt.p, nt.p, wt.p, k, alpha, P->op64.near.p, pr->particles,
                              P->cfg.op, make_double2(P->cfg.gamma_re, P->cfg.gamma_im));
      FDA_LAUNCH_CHECK();
    }
    FDA_CUDA(cudaDeviceSynchronize());
    // fold the corrections that fall inside a row's direct blocks into the blocks
    std::vector<int32_t> row_leaf(N, -1);
    for (size_t u = 0; u < tleaf.size(); ++u)
      for (int64_t ti = T->h_pb[tleaf[u]]; ti < T->h_pe[tleaf[u]]; ++ti) row_leaf[ti] = (int32_t)u;
    DBuf<int32_t> d_row_leaf;
    FDA_TRY(d_row_leaf.upload(row_leaf));
    DBuf<int64_t> keep_cnt, nptr;
    DBuf<int8_t> keep;
    FDA_TRY(keep_cnt.alloc(N));
    FDA_TRY(keep.alloc(std::max<int64_t>(P->corr_entries, 1)));
    k_merge_corr<<<cdiv(N, 128), 128>>>(P->corr_ptr.p, P->corr_col.p, P->op64.corr.p, d_row_leaf.p, P->near_tleaf.p,
                                        P->near_tptr.p, P->near_src.p, P->near_off.p, T->pb.p, T->pe.p, N,
                                        P->op64.near.p, keep_cnt.p, keep.p);
    FDA_LAUNCH_CHECK();
    FDA_TRY(nptr.alloc(N + 1));
    int64_t kept = 0;
    FDA_TRY(exclusive_scan_i64(keep_cnt.p, nptr.p, N, &kept, 0));
    FDA_CUDA(cudaMemcpy(nptr.p + N, &kept, sizeof(int64_t), cudaMemcpyHostToDevice));
    DBuf<int32_t> ncol;
    DBuf<double2> nval;
    FDA_TRY(ncol.alloc(std::max<int64_t>(kept, 1)));
    FDA_TRY(nval.alloc(std::max<int64_t>(kept, 1)));
    k_compact_corr<<<cdiv(N, 128), 128>>>(P->corr_ptr.p, P->corr_col.p, P->op64.corr.p, keep.p, nptr.p, N, ncol.p,
                                          nval.p);
    FDA_LAUNCH_CHECK();
    FDA_CUDA(cudaDeviceSynchronize());
    P->corr_merged = P->corr_entries - kept;
    P->corr_entries = kept;
    std::swap(P->corr_ptr.p, nptr.p);
    std::swap(P->corr_ptr.n, nptr.n);
    std::swap(P->corr_col.p, ncol.p);
    std::swap(P->corr_col.n, ncol.n);
    std::swap(P->op64.corr.p, nval.p);
    std::swap(P->op64.corr.n, nval.n);
  }
  double t7 = now_ms();
  P->setup_ms[7] = t7 - t6;

  // ---- 8. FP32 operator copies and workspaces
  const int nr = P->cfg.nrhs_max;
  FDA_TRY(P->tc_err.alloc(1));
  FDA_TRY(P->tc_err.zero());
  if (!P->cfg.drop_fp64) {
    FDA_TRY(P->xt64.alloc((size_t)N * nr));
    FDA_TRY(P->yt64.alloc((size_t)N * nr));
    FDA_TRY(P->cout64.alloc((size_t)std::max<int64_t>(P->n_coef, 1) * nr));
    FDA_TRY(P->cin64.alloc((size_t)std::max<int64_t>(P->n_coef, 1) * nr));
    FDA_TRY(P->mid64.alloc((size_t)std::max<int64_t>(P->n_mid, 1) * nr));
  }
  if (P->cfg.precision == FDA_PREC_FP32) {
    FDA_TRY(to_fp32(P->op64.S, P->op32.S));
    FDA_TRY(to_fp32(P->op64.T, P->op32.T));
    FDA_TRY(to_fp32(P->op64.M, P->op32.M));
    FDA_TRY(to_fp32(P->op64.K, P->op32.K));
    FDA_TRY(to_fp32(P->op64.near, P->op32.near));
    FDA_TRY(to_fp32(P->op64.corr, P->op32.corr));
    if (P->op64.lr.n) FDA_TRY(to_fp32(P->op64.lr, P->op32.lr));
    FDA_TRY(P->xt32.alloc((size_t)N * nr));
    FDA_TRY(P->xdup32.alloc((size_t)N));
    FDA_TRY(P->yt32.alloc((size_t)N * nr));
    FDA_TRY(P->cout32.alloc((size_t)std::max<int64_t>(P->n_coef, 1) * nr));
    FDA_TRY(P->cin32.alloc((size_t)std::max<int64_t>(P->n_coef, 1) * nr));
    FDA_TRY(P->mid32.alloc((size_t)std::max<int64_t>(P->n_mid, 1) * nr));
    FDA_TRY(build_vtm_maps(P));
    {  // the far field is the longer branch of a two-stream product: its CTAs go first when slots free up
      int lo = 0, hi = 0;
      FDA_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      FDA_CUDA(cudaStreamCreateWithPriority(&P->side, cudaStreamNonBlocking, hi));
      for (int i = 0; i < 4; ++i) {
        FDA_CUDA(cudaStreamCreateWithPriority(&P->lvs[i], cudaStreamNonBlocking, hi));
        FDA_CUDA(cudaEventCreateWithFlags(&P->ev_lvj[i], cudaEventDisableTiming));
      }
      for (int l = 0; l < FDA_MAXLEV; ++l) FDA_CUDA(cudaEventCreateWithFlags(&P->ev_lev[l], cudaEventDisableTiming));
    }
    FDA_CUDA(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
    FDA_CUDA(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
    if (P->cfg.drop_fp64) {  // FP32-only plan: the FP64 masters go once their copies exist
      FDA_CUDA(cudaDeviceSynchronize());
      P->op64.S.release();
      P->op64.T.release();
      P->op64.M.release();
      P->op64.K.release();
      P->op64.near.release();
      P->op64.corr.release();
      P->op64.lr.release();
    }
  }
  {
    std::vector<int> ls(FDA_MAXLEV, 0), lnw(FDA_MAXLEV, 1);
    for (int l = 0; l < FDA_MAXLEV; ++l) ls[l] = P->lev[l].s, lnw[l] = P->lev[l].nw;
    FDA_TRY(P->lev_s.upload(ls));
    FDA_TRY(P->lev_nw.upload(lnw));
    for (int64_t b : P->h_leaves) P->max_leaf = std::max<int>(P->max_leaf, (int)(T->h_pe[b] - T->h_pb[b]));
  }
  FDA_CUDA(cudaDeviceSynchronize());
  return FDA_OK;
}

}  // namespace fda
