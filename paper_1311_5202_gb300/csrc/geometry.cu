// Geometry and near-field corrections of the locally corrected Nystrom method (Sec. 2.2).
//
//  k_nystrom       : Nystrom points, paper normals (into the body) and weights of the 6-point rule.
//  local regions   : D_i = elements whose distance to x_i is <= 2x their longest vertex chord
//                    (distance = min over the element's 6 nodes and 6 Nystrom points), found by
//                    hashing element centroids into a uniform grid of cell size >= every element's reach.
//  k_corrections   : one warp per (x_i, element in D_i): moments of dG/dn_y and d2G/dn_x dn_y (or, for the
//                    radiation right-hand side, of G and dG/dn_x) against
//                    the basis xi1^p xi2^q (p+q <= 2) (Eq. local correction), the 6x6 solve, and the
//                    correction C_ij = wbar_ij - [j != i] K_H(x_i, y_j) w_j of Eq. kcorrection.
//                    Element carrying x_i: polar coordinates about x_i; the hypersingular moment is the
//                    Hadamard finite part for a spherical exclusion, with the rho^-2 and rho^-1 terms
//                    of the Laurent expansion subtracted and integrated in closed form.
//                    Other elements: depth-first subdivision into 4 until the nearest sample point is
//                    >= 2.5 x the sub-triangle diameter, then a collapsed 8x8 Gauss-Legendre rule.
#include "internal.cuh"

namespace fda {

// ------------------------------------------------------------------ constants
__constant__ double c_gxi[6][2];
__constant__ double c_gw[6];
__constant__ double c_phiinv[6][6];  // solves sum_j phi_n(xi_j) w_j = I_n  ->  w = PhiInv I
__constant__ double c_gl8x[8], c_gl8w[8];
__constant__ double c_gl12x[12], c_gl12w[12];
__constant__ double c_gl14x[14], c_gl14w[14];

// published 6-point (degree 4) rule on the reference triangle, two barycentric orbits
static const double kA1 = 0.44594849091596488632, kB1 = 0.10810301816807022736;
static const double kA2 = 0.09157621350977074346, kB2 = 0.81684757298045851308;
static const double kW1 = 0.22338158967801146570, kW2 = 0.10995174365532186764;

static void gauss_legendre_host(int n, double* x, double* w) {
  // Newton on P_n, nodes mapped to [0,1]
  for (int i = 0; i < n; ++i) {
    double z = cos(FDA_PI * (i + 0.75) / (n + 0.5)), dp = 0;
    for (int it = 0; it < 200; ++it) {
      double p0 = 1, p1 = 0;
      for (int j = 1; j <= n; ++j) {
        double p2 = p1;
        p1 = p0;
        p0 = ((2 * j - 1) * z * p1 - (j - 1) * p2) / j;
      }
      dp = n * (z * p0 - p1) / (z * z - 1);
      double dz = p0 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1 - z);
    w[i] = 1.0 / ((1 - z * z) * dp * dp);
  }
}

int upload_geometry_constants() {
  static bool done = false;
  if (done) return FDA_OK;
  const double b1 = kB1, b2 = kB2;
  double gxi[6][2] = {{kA1, kA1}, {b1, kA1}, {kA1, b1}, {kA2, kA2}, {b2, kA2}, {kA2, b2}};
  double gw[6] = {0.5 * kW1, 0.5 * kW1, 0.5 * kW1, 0.5 * kW2, 0.5 * kW2, 0.5 * kW2};
  // inverse of M[n][j] = phi_n(xi_j), phi = {1, s, t, s^2, s t, t^2}, by Gauss-Jordan
  double M[6][12];
  for (int j = 0; j < 6; ++j) {
    double s = gxi[j][0], t = gxi[j][1];
    double ph[6] = {1, s, t, s * s, s * t, t * t};
    for (int n = 0; n < 6; ++n) M[n][j] = ph[n];
  }
  for (int n = 0; n < 6; ++n)
    for (int j = 0; j < 6; ++j) M[n][6 + j] = (n == j);
  for (int c = 0; c < 6; ++c) {
    int p = c;
    for (int r = c + 1; r < 6; ++r)
      if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
    for (int q = 0; q < 12; ++q) std::swap(M[c][q], M[p][q]);
    double d = M[c][c];
    for (int q = 0; q < 12; ++q) M[c][q] /= d;
    for (int r = 0; r < 6; ++r)
      if (r != c) {
        double f = M[r][c];
        for (int q = 0; q < 12; ++q) M[r][q] -= f * M[c][q];
      }
  }
  double inv[6][6];
  for (int n = 0; n < 6; ++n)
    for (int j = 0; j < 6; ++j) inv[n][j] = M[n][6 + j];
  double x8[8], w8[8], x12[12], w12[12], x14[14], w14[14];
  gauss_legendre_host(8, x8, w8);
  gauss_legendre_host(12, x12, w12);
  gauss_legendre_host(14, x14, w14);
  FDA_CUDA(cudaMemcpyToSymbol(c_gxi, gxi, sizeof(gxi)));
  FDA_CUDA(cudaMemcpyToSymbol(c_gw, gw, sizeof(gw)));
  FDA_CUDA(cudaMemcpyToSymbol(c_phiinv, inv, sizeof(inv)));
  FDA_CUDA(cudaMemcpyToSymbol(c_gl8x, x8, sizeof(x8)));
  FDA_CUDA(cudaMemcpyToSymbol(c_gl8w, w8, sizeof(w8)));
  FDA_CUDA(cudaMemcpyToSymbol(c_gl12x, x12, sizeof(x12)));
  FDA_CUDA(cudaMemcpyToSymbol(c_gl12w, w12, sizeof(w12)));
  FDA_CUDA(cudaMemcpyToSymbol(c_gl14x, x14, sizeof(x14)));
  FDA_CUDA(cudaMemcpyToSymbol(c_gl14w, w14, sizeof(w14)));
  done = true;
  return FDA_OK;
}

// ------------------------------------------------------------------ quadratic triangle
struct Tri6 {
  double P[6][3];
  double h11[3], h12[3], h22[3];  // constant second derivatives
};

__device__ __forceinline__ void tri_load(Tri6& E, const double* nodes, const int32_t* el) {
  for (int a = 0; a < 6; ++a) {
    int64_t v = el[a];
    E.P[a][0] = nodes[3 * v];
    E.P[a][1] = nodes[3 * v + 1];
    E.P[a][2] = nodes[3 * v + 2];
  }
  for (int d = 0; d < 3; ++d) {
    // N0 = L0(2L0-1), N1 = s(2s-1), N2 = t(2t-1), N3 = 4 L0 s, N4 = 4 s t, N5 = 4 t L0
    E.h11[d] = 4 * E.P[0][d] + 4 * E.P[1][d] - 8 * E.P[3][d];
    E.h22[d] = 4 * E.P[0][d] + 4 * E.P[2][d] - 8 * E.P[5][d];
    E.h12[d] = 4 * E.P[0][d] - 4 * E.P[3][d] + 4 * E.P[4][d] - 4 * E.P[5][d];
  }
}

// position y, tangents ys = dy/dxi1, yt = dy/dxi2
__device__ __forceinline__ void tri_map(const Tri6& E, double s, double t, double* y, double* ys, double* yt) {
  double L = 1.0 - s - t;
  double N[6] = {L * (2 * L - 1), s * (2 * s - 1), t * (2 * t - 1), 4 * L * s, 4 * s * t, 4 * t * L};
  double Ns[6] = {1 - 4 * L, 4 * s - 1, 0, 4 * (L - s), 4 * t, -4 * t};
  double Nt[6] = {1 - 4 * L, 0, 4 * t - 1, -4 * s, 4 * s, 4 * (L - t)};
  for (int d = 0; d < 3; ++d) {
    double a = 0, b = 0, c = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      a = fma(N[q], E.P[q][d], a);
      b = fma(Ns[q], E.P[q][d], b);
      c = fma(Nt[q], E.P[q][d], c);
    }
    y[d] = a;
    ys[d] = b;
    yt[d] = c;
  }
}

// point, paper normal (-(ys x yt)/J) and Jacobian J
__device__ __forceinline__ void tri_point(const Tri6& E, double s, double t, double* y, double* n, double& J) {
  double ys[3], yt[3];
  tri_map(E, s, t, y, ys, yt);
  double c0 = ys[1] * yt[2] - ys[2] * yt[1];
  double c1 = ys[2] * yt[0] - ys[0] * yt[2];
  double c2 = ys[0] * yt[1] - ys[1] * yt[0];
  J = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  double iJ = -1.0 / J;
  n[0] = c0 * iJ;
  n[1] = c1 * iJ;
  n[2] = c2 * iJ;
}

__device__ __forceinline__ void basis6(double s, double t, double* p) {
  p[0] = 1;
  p[1] = s;
  p[2] = t;
  p[3] = s * s;
  p[4] = s * t;
  p[5] = t * t;
}

// ------------------------------------------------------------------ a1: Nystrom points
// The Nystrom points feed the integer tree rules, so they are evaluated in the plain order of the
// definition y = sum_k N_k(xi) P_k, n = -(y_s x y_t)/|y_s x y_t|, w = w_g |y_s x y_t|, every operation
// explicitly rounded (no contraction): any other implementation of the same formulas in that order gets
// the same bits.
__device__ __forceinline__ double rm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ra(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rs(double a, double b) { return __dsub_rn(a, b); }

static __global__ void k_nystrom(const double* nodes, const int32_t* elems, int64_t ne, double* x, double* n,
                                 double* w) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * ne) return;
  int64_t e = i / 6;
  int g = (int)(i - 6 * e);
  const int32_t* el = elems + 6 * e;
  const double s = c_gxi[g][0], t = c_gxi[g][1];
  const double L = rs(rs(1.0, s), t);
  const double N[6] = {rm(L, rs(rm(2.0, L), 1.0)), rm(s, rs(rm(2.0, s), 1.0)), rm(t, rs(rm(2.0, t), 1.0)),
                       rm(rm(4.0, L), s),        rm(rm(4.0, s), t),        rm(rm(4.0, t), L)};
  const double A[6] = {-rs(rm(4.0, L), 1.0), rs(rm(4.0, s), 1.0), 0.0, rm(4.0, rs(L, s)), rm(4.0, t), -rm(4.0, t)};
  const double B[6] = {-rs(rm(4.0, L), 1.0), 0.0, rs(rm(4.0, t), 1.0), -rm(4.0, s), rm(4.0, s), rm(4.0, rs(L, t))};
  double y[3], ys[3], yt[3];
  for (int d = 0; d < 3; ++d) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int q = 0; q < 6; ++q) {
      double p = nodes[3 * (int64_t)el[q] + d];
      a = ra(a, rm(N[q], p));
      b = ra(b, rm(A[q], p));
      c = ra(c, rm(B[q], p));
    }
    y[d] = a;
    ys[d] = b;
    yt[d] = c;
  }
  double c0 = rs(rm(ys[1], yt[2]), rm(ys[2], yt[1]));
  double c1 = rs(rm(ys[2], yt[0]), rm(ys[0], yt[2]));
  double c2 = rs(rm(ys[0], yt[1]), rm(ys[1], yt[0]));
  double J = __dsqrt_rn(ra(ra(rm(c0, c0), rm(c1, c1)), rm(c2, c2)));
  for (int d = 0; d < 3; ++d) x[3 * i + d] = y[d];
  n[3 * i + 0] = __ddiv_rn(-c0, J);
  n[3 * i + 1] = __ddiv_rn(-c1, J);
  n[3 * i + 2] = __ddiv_rn(-c2, J);
  w[i] = rm(c_gw[g], J);
}

int nystrom_points(bm_problem_s* P) {
  FDA_TRY(upload_geometry_constants());
  FDA_TRY(P->x.alloc(3 * P->N));
  FDA_TRY(P->n.alloc(3 * P->N));
  FDA_TRY(P->w.alloc(P->N));
  k_nystrom<<<cdiv(P->N, 128), 128>>>(P->nodes.p, P->elems.p, P->ne, P->x.p, P->n.p, P->w.p);
  FDA_LAUNCH_CHECK();
  FDA_CUDA(cudaDeviceSynchronize());
  return FDA_OK;
}

// ------------------------------------------------------------------ local regions by grid hashing
// per element: longest vertex chord, 12 sample points (6 nodes + 6 Nystrom points), centroid, reach
static __global__ void k_elem_info(const double* nodes, const int32_t* elems, int64_t ne, double* info /*ne x 5*/) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  Tri6 E;
  tri_load(E, nodes, elems + 6 * e);
  auto d3 = [](const double* a, const double* b) {
    double u = a[0] - b[0], v = a[1] - b[1], w = a[2] - b[2];
    return sqrt(u * u + v * v + w * w);
  };
  double side = fmax(d3(E.P[0], E.P[1]), fmax(d3(E.P[1], E.P[2]), d3(E.P[2], E.P[0])));
  double c[3];
  for (int d = 0; d < 3; ++d) c[d] = (E.P[0][d] + E.P[1][d] + E.P[2][d]) / 3.0;
  double r = 0;
  for (int a = 0; a < 6; ++a) r = fmax(r, d3(E.P[a], c));
  for (int g = 0; g < 6; ++g) {
    double y[3], n[3], J;
    tri_point(E, c_gxi[g][0], c_gxi[g][1], y, n, J);
    r = fmax(r, d3(y, c));
  }
  info[5 * e + 0] = c[0];
  info[5 * e + 1] = c[1];
  info[5 * e + 2] = c[2];
  info[5 * e + 3] = side;
  info[5 * e + 4] = 2.0 * side + r;  // reach: any point within 2*side of a sample is within this of c
}

struct GridSpec {
  double lo[3], h;
  int64_t dim[3];
};

__device__ __forceinline__ int64_t grid_cell(const GridSpec& G, const double* p, int64_t* ijk) {
  for (int d = 0; d < 3; ++d) {
    int64_t q = (int64_t)floor((p[d] - G.lo[d]) / G.h);
    q = q < 0 ? 0 : (q >= G.dim[d] ? G.dim[d] - 1 : q);
    ijk[d] = q;
  }
  return (ijk[0] * G.dim[1] + ijk[1]) * G.dim[2] + ijk[2];
}

static __global__ void k_elem_cells(const double* info, int64_t ne, GridSpec G, uint64_t* key, int64_t* idx) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int64_t ijk[3];
  key[e] = (uint64_t)grid_cell(G, info + 5 * e, ijk);
  idx[e] = e;
}

static __global__ void k_cell_ranges(const uint64_t* key, int64_t ne, int64_t* cstart, int64_t* cend) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  if (i == 0 || key[i] != key[i - 1]) cstart[key[i]] = i;
  if (i == ne - 1 || key[i] != key[i + 1]) cend[key[i]] = i + 1;
}

__device__ __forceinline__ bool in_local_region(const double* nodes, const int32_t* el, const double* xs_e,
                                                double side, const double* x) {
  double dmin = 1e300;
  for (int a = 0; a < 6; ++a) {
    int64_t v = el[a];
    double u0 = x[0] - nodes[3 * v], u1 = x[1] - nodes[3 * v + 1], u2 = x[2] - nodes[3 * v + 2];
    dmin = fmin(dmin, sqrt(u0 * u0 + u1 * u1 + u2 * u2));
  }
  for (int g = 0; g < 6; ++g) {
    double u0 = x[0] - xs_e[3 * g], u1 = x[1] - xs_e[3 * g + 1], u2 = x[2] - xs_e[3 * g + 2];
    dmin = fmin(dmin, sqrt(u0 * u0 + u1 * u1 + u2 * u2));
  }
  return dmin <= 2.0 * side;
}

#define DI_MAX 512
template <bool FILL>
static __global__ void k_local_regions(const double* nodes, const int32_t* elems, const double* xs,
                                       const double* info, GridSpec G, const int64_t* cstart, const int64_t* cend,
                                       const int64_t* esorted, int64_t N, int64_t* cnt, const int64_t* rowptr,
                                       int32_t* cols, int* overflow) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* x = xs + 3 * i;
  int64_t ijk[3];
  grid_cell(G, x, ijk);
  int64_t c = 0;
  int64_t base = FILL ? rowptr[i] : 0;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) {
        int64_t a = ijk[0] + dx, b = ijk[1] + dy, q = ijk[2] + dz;
        if (a < 0 || b < 0 || q < 0 || a >= G.dim[0] || b >= G.dim[1] || q >= G.dim[2]) continue;
        int64_t cell = (a * G.dim[1] + b) * G.dim[2] + q;
        for (int64_t p = cstart[cell]; p < cend[cell]; ++p) {
          int64_t e = esorted[p];
          if (in_local_region(nodes, elems + 6 * e, xs + 18 * e, info[5 * e + 3], x)) {
            if (FILL) {
              // insertion in ascending element order
              int64_t pos = base + c;
              while (pos > base && cols[pos - 1] > (int32_t)e) {
                cols[pos] = cols[pos - 1];
                --pos;
              }
              cols[pos] = (int32_t)e;
            }
            ++c;
          }
        }
      }
  if (!FILL) {
    cnt[i] = c;
    if (c > DI_MAX) atomicExch(overflow, 1);
  }
}

int local_regions(bm_problem_s* P, DBuf<int64_t>& rowptr, DBuf<int32_t>& cols) {
  const int64_t ne = P->ne, N = P->N;
  DBuf<double> info;
  FDA_TRY(info.alloc(5 * ne));
  k_elem_info<<<cdiv(ne, 128), 128>>>(P->nodes.p, P->elems.p, ne, info.p);
  FDA_LAUNCH_CHECK();
  std::vector<double> hi;
  FDA_TRY(info.download(hi));
  GridSpec G;
  double lo[3] = {1e300, 1e300, 1e300}, up[3] = {-1e300, -1e300, -1e300}, reach = 0;
  for (int64_t e = 0; e < ne; ++e) {
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], hi[5 * e + d] - hi[5 * e + 4]);
      up[d] = std::max(up[d], hi[5 * e + d] + hi[5 * e + 4]);
    }
    reach = std::max(reach, hi[5 * e + 4]);
  }
  G.h = reach * 1.0000001;
  for (;;) {
    int64_t tot = 1;
    for (int d = 0; d < 3; ++d) {
      G.lo[d] = lo[d];
      G.dim[d] = (int64_t)ceil((up[d] - lo[d]) / G.h) + 1;
      tot *= G.dim[d];
    }
    if (tot <= (int64_t)1 << 26) break;
    G.h *= 1.5;
  }
  int64_t ncell = G.dim[0] * G.dim[1] * G.dim[2];
  DBuf<uint64_t> ekey;
  DBuf<int64_t> eidx, cstart, cend;
  FDA_TRY(ekey.alloc(ne));
  FDA_TRY(eidx.alloc(ne));
  FDA_TRY(cstart.alloc(ncell));
  FDA_TRY(cend.alloc(ncell));
  FDA_TRY(cstart.zero());
  FDA_TRY(cend.zero());
  k_elem_cells<<<cdiv(ne, 256), 256>>>(info.p, ne, G, ekey.p, eidx.p);
  FDA_LAUNCH_CHECK();
  int bits = 1;
  while (bits < 63 && ((uint64_t)1 << bits) <= (uint64_t)ncell) ++bits;
  FDA_TRY(radix_sort_pairs(ekey.p, eidx.p, ne, bits, 0));
  k_cell_ranges<<<cdiv(ne, 256), 256>>>(ekey.p, ne, cstart.p, cend.p);
  FDA_LAUNCH_CHECK();
  DBuf<int64_t> cnt;
  DBuf<int> ovf;
  FDA_TRY(cnt.alloc(N));
  FDA_TRY(ovf.alloc(1));
  FDA_TRY(ovf.zero());
  k_local_regions<false><<<cdiv(N, 128), 128>>>(P->nodes.p, P->elems.p, P->x.p, info.p, G, cstart.p, cend.p,
                                                 eidx.p, N, cnt.p, nullptr, nullptr, ovf.p);
  FDA_LAUNCH_CHECK();
  int hov = 0;
  FDA_CUDA(cudaMemcpy(&hov, ovf.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (hov) {
    set_error("a local region holds more than %d elements (mesh far from uniform?)", DI_MAX);
    return FDA_E_INVALID_ARG;
  }
  FDA_TRY(rowptr.alloc(N + 1));
  int64_t total = 0;
  FDA_TRY(exclusive_scan_i64(cnt.p, rowptr.p, N, &total, 0));
  FDA_CUDA(cudaMemcpy(rowptr.p + N, &total, sizeof(int64_t), cudaMemcpyHostToDevice));
  FDA_TRY(cols.alloc(std::max<int64_t>(total, 1)));
  k_local_regions<true><<<cdiv(N, 128), 128>>>(P->nodes.p, P->elems.p, P->x.p, info.p, G, cstart.p, cend.p,
                                                eidx.p, N, nullptr, rowptr.p, cols.p, nullptr);
  FDA_LAUNCH_CHECK();
  FDA_CUDA(cudaDeviceSynchronize());
  return FDA_OK;
}

// ------------------------------------------------------------------ a5: moments and corrections
// Accumulators of one lane: 6 moments of dG/dn_y and 6 of d2G/dn_x dn_y.
struct Mom {
  double2 D[6], H[6];
};

__device__ __forceinline__ void mom_zero(Mom& m) {
#pragma unroll
  for (int q = 0; q < 6; ++q) m.D[q] = m.H[q] = make_double2(0, 0);
}

// Self element: x = y(xi0). One lane per angular node; the radial integral runs in the lane.
// op 0: moments of dG/dn_y and d2G/dn_x dn_y (finite part); op 1: moments of G and dG/dn_x (both bounded in
// polar coordinates, no finite-part terms), the kernels of the radiation right-hand side (S + alpha M) q.
__device__ void moments_self_warp(const Tri6& E, int g, double k, Mom& acc, int op) {
  const int lane = threadIdx.x & 31;
  const double s0 = c_gxi[g][0], t0 = c_gxi[g][1];
  double x[3], xs[3], xt[3];
  tri_map(E, s0, t0, x, xs, xt);
  double N0[3] = {xs[1] * xt[2] - xs[2] * xt[1], xs[2] * xt[0] - xs[0] * xt[2], xs[0] * xt[1] - xs[1] * xt[0]};
  double J0 = sqrt(N0[0] * N0[0] + N0[1] * N0[1] + N0[2] * N0[2]);
  double nx[3] = {-N0[0] / J0, -N0[1] / J0, -N0[2] / J0};
  // dJ/dxi_a = N0 . dN/dxi_a / J0,  dN/dxi1 = h11 x yt + ys x h12,  dN/dxi2 = h12 x yt + ys x h22
  auto cr = [](const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
  };
  double u1[3], u2[3], v1[3], v2[3];
  cr(E.h11, xt, u1);
  cr(xs, E.h12, u2);
  cr(E.h12, xt, v1);
  cr(xs, E.h22, v2);
  double dJs = 0, dJt = 0;
  for (int d = 0; d < 3; ++d) {
    dJs += N0[d] * (u1[d] + u2[d]);
    dJt += N0[d] * (v1[d] + v2[d]);
  }
  dJs /= J0;
  dJt /= J0;
  double phi0[6];
  basis6(s0, t0, phi0);
  // angular break points per edge, relative to the foot of the perpendicular from xi0
  const double V[3][2] = {{0, 0}, {1, 0}, {0, 1}};
  double bp[3][24];
  int nbp[3];
  double dperp[3], thn[3];
  int total = 0;
  int nsub_off[3];
  for (int ed = 0; ed < 3; ++ed) {
    double px = V[ed][0] - s0, py = V[ed][1] - t0;
    double qx = V[(ed + 1) % 3][0] - s0, qy = V[(ed + 1) % 3][1] - t0;
    double ex = qx - px, ey = qy - py, el = sqrt(ex * ex + ey * ey);
    ex /= el;
    ey /= el;
    double pr = -(px * ex + py * ey);
    double fx = px + pr * ex, fy = py + pr * ey;  // foot of the perpendicular (relative to xi0)
    double dp = sqrt(fx * fx + fy * fy);
    dperp[ed] = dp;
    thn[ed] = atan2(fy, fx);
    double cf = fx / dp, sf = fy / dp;
    double aP = atan2(-px * sf + py * cf, px * cf + py * sf);
    double aQ = atan2(-qx * sf + qy * cf, qx * cf + qy * sf);
    int n = 0;
    bp[ed][n++] = aP;
    // grade towards the poles of 1/cos at -pi/2 and +pi/2: each piece no longer than its distance
    if (aP < 0) {
      double dl = 0.5 * FDA_PI + aP;
      double lim = fmin(0.0, aQ);
      for (double q = 2 * dl; -0.5 * FDA_PI + q < lim && n < 11; q *= 2) bp[ed][n++] = -0.5 * FDA_PI + q;
      if (aQ > 0) bp[ed][n++] = 0.0;
    }
    if (aQ > 0) {
      double du = 0.5 * FDA_PI - aQ;
      double lim = fmax(0.0, aP);
      double tmp[11];
      int m = 0;
      for (double q = 2 * du; 0.5 * FDA_PI - q > lim && m < 11; q *= 2) tmp[m++] = 0.5 * FDA_PI - q;
      for (int r = m - 1; r >= 0; --r) bp[ed][n++] = tmp[r];
    }
    bp[ed][n++] = aQ;
    nbp[ed] = n;
    nsub_off[ed] = total;
    total += (n - 1) * 12;
  }
  for (int node = lane; node < total; node += 32) {
    int ed = (node >= nsub_off[2]) ? 2 : (node >= nsub_off[1] ? 1 : 0);
    int loc = node - nsub_off[ed];
    int iv = loc / 12, gq = loc - 12 * iv;
    double pa = bp[ed][iv], pb = bp[ed][iv + 1];
    if (!(pb > pa)) continue;
    double ph = pa + (pb - pa) * c_gl12x[gq];
    double wth = (pb - pa) * c_gl12w[gq];
    double th = thn[ed] + ph;
    double e1, e2;
    sincos(th, &e2, &e1);
    double rhohat = dperp[ed] / cos(ph);
    double A[3], B[3];
    for (int d = 0; d < 3; ++d) {
      A[d] = xs[d] * e1 + xt[d] * e2;
      B[d] = 0.5 * (E.h11[d] * e1 * e1 + 2.0 * E.h12[d] * e1 * e2 + E.h22[d] * e2 * e2);
    }
    double A2 = A[0] * A[0] + A[1] * A[1] + A[2] * A[2];
    double An = sqrt(A2);
    double AB = A[0] * B[0] + A[1] * B[1] + A[2] * B[2];
    double J1 = dJs * e1 + dJt * e2;
    double dphi[6] = {0, e1, e2, 2 * s0 * e1, t0 * e1 + s0 * e2, 2 * t0 * e2};
    double c3 = 0.25 / FDA_PI / (A2 * An);
    double Fm2[6], Fm1[6];
    for (int q = 0; q < 6; ++q) {
      Fm2[q] = op ? 0.0 : phi0[q] * J0 * c3;
      Fm1[q] = op ? 0.0 : (J1 * phi0[q] + J0 * dphi[q] - 3.0 * J0 * phi0[q] * AB / A2) * c3;
    }
    // radial integral of the regular part
    double2 rD[6], rH[6];
    for (int q = 0; q < 6; ++q) rD[q] = rH[q] = make_double2(0, 0);
    for (int b = 0; b < 14; ++b) {
      double rho = rhohat * c_gl14x[b], wr = rhohat * c_gl14w[b];
      double ss = s0 + rho * e1, tt = t0 + rho * e2;
      double y[3], ny[3], J;
      tri_point(E, ss, tt, y, ny, J);
      KernVals K = helmholtz4(x, nx, y, ny, k);
      double ph6[6];
      basis6(ss, tt, ph6);
      double f = wr * J * rho;
      double ir = 1.0 / rho;
      const double2 k1 = op ? K.G : K.Dy, k2 = op ? K.Dx : K.H;
      for (int q = 0; q < 6; ++q) {
        rD[q] = cadd(rD[q], cscale(k1, f * ph6[q]));
        double2 h = cscale(k2, f * ph6[q]);
        h.x -= wr * (Fm2[q] * ir * ir + Fm1[q] * ir);
        rH[q] = cadd(rH[q], h);
      }
    }
    // closed-form finite-part terms: F_{-1} ln(rhohat/beta) - F_{-2} (gamma/beta^2 + 1/rhohat)
    double beta = 1.0 / An, gob2 = -AB / A2;  // gamma/beta^2 = -(A.B)/|A|^2
    double lg = log(rhohat / beta);
    for (int q = 0; q < 6; ++q) {
      acc.D[q] = cadd(acc.D[q], cscale(rD[q], wth));
      double2 h = cscale(rH[q], wth);
      h.x += wth * (Fm1[q] * lg - Fm2[q] * (gob2 + 1.0 / rhohat));
      acc.H[q] = cadd(acc.H[q], h);
    }
  }
}

// Nearby element: depth-first subdivision, the warp walks one shared stack.
#define SUB_STACK 64
__device__ void moments_near_warp(const Tri6& E, const double* x, const double* nx, double k, Mom& acc,
                                  double (*stk)[6], int op) {
  const int lane = threadIdx.x & 31;
  int sp = 0;
  if (lane == 0) {
    stk[0][0] = 0;
    stk[0][1] = 0;
    stk[0][2] = 1;
    stk[0][3] = 0;
    stk[0][4] = 0;
    stk[0][5] = 1;
  }
  sp = 1;
  __syncwarp();
  int depth_guard = 0;
  while (sp > 0) {
    --sp;
    double T0s = stk[sp][0], T0t = stk[sp][1], T1s = stk[sp][2], T1t = stk[sp][3], T2s = stk[sp][4],
           T2t = stk[sp][5];
    __syncwarp();
    // sample points: 3 vertices, 3 mid-edges, centroid (lanes 0..6)
    double dist = 1e300, vx[3] = {0, 0, 0};
    if (lane < 7) {
      double ss, tt;
      if (lane < 3) {
        ss = lane == 0 ? T0s : (lane == 1 ? T1s : T2s);
        tt = lane == 0 ? T0t : (lane == 1 ? T1t : T2t);
      } else if (lane == 3) {
        ss = 0.5 * (T0s + T1s), tt = 0.5 * (T0t + T1t);
      } else if (lane == 4) {
        ss = 0.5 * (T1s + T2s), tt = 0.5 * (T1t + T2t);
      } else if (lane == 5) {
        ss = 0.5 * (T2s + T0s), tt = 0.5 * (T2t + T0t);
      } else {
        ss = (T0s + T1s + T2s) / 3.0, tt = (T0t + T1t + T2t) / 3.0;
      }
      double ys[3], yt[3];
      tri_map(E, ss, tt, vx, ys, yt);
      double u0 = x[0] - vx[0], u1 = x[1] - vx[1], u2 = x[2] - vx[2];
      dist = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
    }
    for (int o = 16; o > 0; o >>= 1) dist = fmin(dist, __shfl_xor_sync(0xffffffffu, dist, o));
    // diameter from the three mapped vertices
    double p0[3], p1[3], p2[3];
    for (int d = 0; d < 3; ++d) {
      p0[d] = __shfl_sync(0xffffffffu, vx[d], 0);
      p1[d] = __shfl_sync(0xffffffffu, vx[d], 1);
      p2[d] = __shfl_sync(0xffffffffu, vx[d], 2);
    }
    auto d3 = [](const double* a, const double* b) {
      double u = a[0] - b[0], v = a[1] - b[1], w = a[2] - b[2];
      return sqrt(u * u + v * v + w * w);
    };
    double diam = fmax(d3(p0, p1), fmax(d3(p1, p2), d3(p2, p0)));
    bool leaf = (dist >= 2.5 * diam) || (sp + 4 > SUB_STACK) || (depth_guard > 20000);
    ++depth_guard;
    if (leaf) {
      double es = T1s - T0s, et = T1t - T0t, fs = T2s - T0s, ft = T2t - T0t;
      double jac = fabs(es * ft - et * fs);
      for (int q = lane; q < 64; q += 32) {
        int a = q >> 3, b = q & 7;
        double u = c_gl8x[a], v = c_gl8x[b] * (1.0 - c_gl8x[a]);
        double wq = c_gl8w[a] * c_gl8w[b] * (1.0 - c_gl8x[a]) * jac;
        double ss = T0s + u * es + v * fs, tt = T0t + u * et + v * ft;
        double y[3], ny[3], J;
        tri_point(E, ss, tt, y, ny, J);
        KernVals K = helmholtz4(x, nx, y, ny, k);
        double ph6[6];
        basis6(ss, tt, ph6);
        double f = wq * J;
        const double2 k1 = op ? K.G : K.Dy, k2 = op ? K.Dx : K.H;
        for (int r = 0; r < 6; ++r) {
          acc.D[r] = cadd(acc.D[r], cscale(k1, f * ph6[r]));
          acc.H[r] = cadd(acc.H[r], cscale(k2, f * ph6[r]));
        }
      }
    } else {
      double m01s = 0.5 * (T0s + T1s), m01t = 0.5 * (T0t + T1t);
      double m12s = 0.5 * (T1s + T2s), m12t = 0.5 * (T1t + T2t);
      double m20s = 0.5 * (T2s + T0s), m20t = 0.5 * (T2t + T0t);
      if (lane == 0) {
        double C[4][6] = {{T0s, T0t, m01s, m01t, m20s, m20t},
                          {m01s, m01t, T1s, T1t, m12s, m12t},
                          {m20s, m20t, m12s, m12t, T2s, T2t},
                          {m01s, m01t, m12s, m12t, m20s, m20t}};
        for (int c = 0; c < 4; ++c)
          for (int q = 0; q < 6; ++q) stk[sp + c][q] = C[c][q];
      }
      sp += 4;
    }
    __syncwarp();
  }
}

// One warp per (row i, element e in D_i). Output: 6 correction values per work item.
static __global__ void k_corrections(const double* nodes, const int32_t* elems, const double* xs, const double* ns,
                                     const double* ws, double k, double2 alpha, const int64_t* rowptr,
                                     const int32_t* dcols, int64_t N, int64_t nitems, const int64_t* item_row,
                                     double2* corr /* nitems x 6 */, int op) {
  __shared__ double stk_all[4][SUB_STACK][6];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t it = (int64_t)blockIdx.x * 4 + wib;
  if (it >= nitems) return;
  int64_t i = item_row[it];
  int64_t e = dcols[it];
  Tri6 E;
  tri_load(E, nodes, elems + 6 * e);
  const double* x = xs + 3 * i;
  const double* nx = ns + 3 * i;
  Mom m;
  mom_zero(m);
  if (i / 6 == e)
    moments_self_warp(E, (int)(i - 6 * e), k, m, op);
  else
    moments_near_warp(E, x, nx, k, m, stk_all[wib], op);
  for (int q = 0; q < 6; ++q) {
    m.D[q] = warp_csum(m.D[q]);
    m.H[q] = warp_csum(m.H[q]);
  }
  if (lane < 6) {
    int j = lane;
    double2 wd = make_double2(0, 0), wh = make_double2(0, 0);
    for (int q = 0; q < 6; ++q) {
      wd = cadd(wd, cscale(m.D[q], c_phiinv[j][q]));
      wh = cadd(wh, cscale(m.H[q], c_phiinv[j][q]));
    }
    double2 wbar = cadd(wd, cmul(alpha, wh));
    int64_t col = 6 * e + j;
    if (col != i) {
      KernVals K = helmholtz4(x, nx, xs + 3 * col, ns + 3 * col, k);
      double2 kh = op ? cadd(K.G, cmul(alpha, K.Dx)) : cadd(K.Dy, cmul(alpha, K.H));
      wbar = csub(wbar, cscale(kh, ws[col]));
    }
    corr[6 * it + j] = wbar;
  }
}

static __global__ void k_item_rows(const int64_t* rowptr, int64_t N, int64_t* item_row) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) item_row[p] = i;
}

static __global__ void k_axpy_c(double2* y, const double2* x, double2 a, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = cadd(y[i], cmul(a, x[i]));
}

// Corrections in user DOF order: CSR with one entry per (row, element in D_i, local point j). op = 2 (Robin
// data): the corrections of operator A plus gamma times those of operator B (same local regions).
int near_corrections(bm_problem_s* P, DBuf<int64_t>& di_ptr, DBuf<int32_t>& di_cols, DBuf<double2>& corr,
                     double* ms, int op, double2 gamma) {
  if (op == 2) {
    DBuf<int64_t> p2;
    DBuf<int32_t> c2;
    DBuf<double2> corr_b;
    double ms_a = 0, ms_b = 0;
    FDA_TRY(near_corrections(P, di_ptr, di_cols, corr, &ms_a, 0, gamma));
    FDA_TRY(near_corrections(P, p2, c2, corr_b, &ms_b, 1, gamma));
    k_axpy_c<<<cdiv((int64_t)corr.n, 256), 256>>>(corr.p, corr_b.p, gamma, (int64_t)corr.n);
    FDA_LAUNCH_CHECK();
    FDA_CUDA(cudaDeviceSynchronize());
    if (ms) *ms = ms_a + ms_b;
    return FDA_OK;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  FDA_TRY(upload_geometry_constants());
  FDA_TRY(local_regions(P, di_ptr, di_cols));
  int64_t nitems = 0;
  FDA_CUDA(cudaMemcpy(&nitems, di_ptr.p + P->N, sizeof(int64_t), cudaMemcpyDeviceToHost));
  DBuf<int64_t> item_row;
  FDA_TRY(item_row.alloc(std::max<int64_t>(nitems, 1)));
  k_item_rows<<<cdiv(P->N, 256), 256>>>(di_ptr.p, P->N, item_row.p);
  FDA_LAUNCH_CHECK();
  FDA_TRY(corr.alloc(6 * std::max<int64_t>(nitems, 1)));
  const int64_t chunk = 1 << 20;
  for (int64_t s0 = 0; s0 < nitems; s0 += chunk) {
    int64_t n = std::min(chunk, nitems - s0);
    k_corrections<<<cdiv(n, 4), 128>>>(P->nodes.p, P->elems.p, P->x.p, P->n.p, P->w.p, P->k, P->alpha,
                                       di_ptr.p, di_cols.p + s0, P->N, n, item_row.p + s0, corr.p + 6 * s0, op);
    FDA_LAUNCH_CHECK();
  }
  FDA_CUDA(cudaDeviceSynchronize());
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float t = 0;
  cudaEventElapsedTime(&t, e0, e1);
  if (ms) *ms = t;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return FDA_OK;
}

}  // namespace fda
