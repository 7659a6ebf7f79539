/*
 * ORACLE — test infrastructure only. Plain, slow, FP64 CPU reference for the
 * Burton-Miller Nystrom system of Cao, Wen, Xiao & Liu (fast directional BEM).
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may load
 * this library. It shares no code with the GPU path.
 *
 * What it computes (each piece cites the passage it follows):
 *   - Nystrom points of curved 6-node triangles: the 6-point Gauss rule of the
 *     regular-element quadrature, N = 6 N_e (Sec. 2.2).
 *   - Kernels G = e^{ikr}/(4 pi r) (Eq. fundsol) and its normal derivatives
 *     dG/dn_y, dG/dn_x, d2G/dn_x dn_y of the layer operators (Eq. operator).
 *   - Local region D_i: elements within 2x their largest side of x_i (Sec. 2.2).
 *   - Locally corrected weights: the 6x6 moment system with basis xi1^p xi2^q,
 *     p+q<=2 (Eq. local correction). Moments over the element carrying x_i are
 *     weakly singular (dG/dn_y) or hypersingular (d2G/dn_x dn_y, Hadamard
 *     finite part, Sec. 2.1); they use polar coordinates around x_i with the
 *     finite-part formula for a spherical exclusion neighbourhood (Guiggiani's
 *     direct method). Nearly singular moments use recursive subdivision (Sec. 2.2).
 *   - Particle summation of Sec. 5.1 (Eq. sum) by direct summation.
 *   - Rows of any combination of the four layer operators with their own corrected weights, such as the
 *     radiation right-hand side (S + alpha M - alpha/2 I) q of Eq. bm.
 *   - Corrected sum K_bar (Eq. kcorrection) and the rigid-scatter operator
 *     A = c I + beta_D Dbar + beta_H Hbar (Eq. bm with q = 0, Eq. hmat),
 *     row by row, O(N) per row.
 *   - Octree and interaction lists of Sec. 3.1.1 under integer rules:
 *     quantised Morton keys, split while count > N_p, near field
 *     (LF: adjacent; HF: dist <= c_d k w^2 with c_d = 1/pi), interaction field
 *     I^C = N^P \ N^C by a dual recursion, and directional wedges
 *     (cells of a grid on the faces of the cube [-1,1]^3).
 *
 * Normal convention: the paper's n points out of the fluid domain, i.e. into
 * the scatterer (this is what makes Eq. IE the exterior representation and
 * u = 1/(1-ik) the pulsating-sphere answer of Sec. 5.2). Elements are given
 * counter-clockwise seen from outside, so n = -(dy/dxi1 x dy/dxi2)/J.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double PI_ = 3.14159265358979323846;

/* ---------------- 6-point degree-4 Gauss rule on the reference triangle ---------------- */
/* Symmetric rule (Dunavant, degree 4): two orbits of barycentric points. */
static const double QA1 = 0.44594849091596488632, QB1 = 0.10810301816807022736;
static const double QA2 = 0.09157621350977074346, QB2 = 0.81684757298045851308;
static const double QW1 = 0.22338158967801146570, QW2 = 0.10995174365532186764;
/* Point order j = 0..5 (xi1, xi2); DOF index = 6 * element + j. */
static const double GXI[6][2] = {
    {QA1, QA1}, {QB1, QA1}, {QA1, QB1}, {QA2, QA2}, {QB2, QA2}, {QA2, QB2}};
static const double GWT[6] = {0.5 * QW1, 0.5 * QW1, 0.5 * QW1, 0.5 * QW2, 0.5 * QW2, 0.5 * QW2};

/* ---------------- quadrature controls (settable from tests) ---------------- */
static int q_ntheta = 16;     /* Gauss-Legendre points per angular sub-interval, singular element */
static int q_nrho = 20;       /* Gauss-Legendre points along each ray, singular element */
static double q_eta = 3.0;    /* subdivision stops when dist >= eta * diam */
static int q_nsub = 10;       /* collapsed-square Gauss-Legendre order per sub-triangle */
static int q_maxdepth = 14;   /* subdivision depth limit */
static int q_debug = 0;       /* bit 0: drop F_{-1}; bit 1: drop the gamma term; bit 2: flip normals */

void orc_set_quadrature(int ntheta, int nrho, double eta, int nsub, int maxdepth) {
  if (ntheta > 0) q_ntheta = ntheta;
  if (nrho > 0) q_nrho = nrho;
  if (eta > 0) q_eta = eta;
  if (nsub > 0) q_nsub = nsub;
  if (maxdepth > 0) q_maxdepth = maxdepth;
}
void orc_set_debug(int flags) { q_debug = flags; }

/* Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_n. */
#define GL_MAX 64
static void gauss_legendre01(int n, double* x, double* w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(PI_ * (i + 0.75) / (n + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      pp = n * (z * p0 - p1) / (z * z - 1.0);
      double dz = p0 / pp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double wi = 2.0 / ((1.0 - z * z) * pp * pp);
    x[i] = 0.5 * (1.0 - z);
    x[n - 1 - i] = 0.5 * (1.0 + z);
    w[i] = 0.5 * wi;
    w[n - 1 - i] = 0.5 * wi;
  }
}

int orc_gauss_legendre01(int n, double* x, double* w) {
  if (n < 1 || n > GL_MAX) return -1;
  gauss_legendre01(n, x, w);
  return 0;
}

void orc_nystrom_rule(double* xi /*6x2*/, double* w /*6*/) {
  for (int j = 0; j < 6; ++j) {
    xi[2 * j] = GXI[j][0];
    xi[2 * j + 1] = GXI[j][1];
    w[j] = GWT[j];
  }
}

/* ---------------- element geometry ---------------- */
typedef struct {
  double P[6][3];
  double y11[3], y12[3], y22[3]; /* constant second derivatives of the quadratic map */
} elem_t;

static const double D11[6] = {4, 4, 0, -8, 0, 0};
static const double D22[6] = {4, 0, 4, 0, 0, -8};
static const double D12[6] = {4, 0, 0, -4, 4, -4};

static void elem_load(elem_t* E, const double* nodes, const int32_t* el) {
  for (int a = 0; a < 6; ++a)
    for (int d = 0; d < 3; ++d) E->P[a][d] = nodes[3 * (int64_t)el[a] + d];
  for (int d = 0; d < 3; ++d) {
    E->y11[d] = E->y12[d] = E->y22[d] = 0.0;
    for (int a = 0; a < 6; ++a) {
      E->y11[d] += D11[a] * E->P[a][d];
      E->y12[d] += D12[a] * E->P[a][d];
      E->y22[d] += D22[a] * E->P[a][d];
    }
  }
}

/* position and tangents of the 6-node map at (s, t) = (xi1, xi2) */
static void elem_eval(const elem_t* E, double s, double t, double y[3], double y1[3], double y2[3]) {
  double L0 = 1.0 - s - t;
  double N[6] = {L0 * (2 * L0 - 1), s * (2 * s - 1), t * (2 * t - 1), 4 * L0 * s, 4 * s * t, 4 * t * L0};
  double A[6] = {-(4 * L0 - 1), 4 * s - 1, 0.0, 4 * (L0 - s), 4 * t, -4 * t};
  double B[6] = {-(4 * L0 - 1), 0.0, 4 * t - 1, -4 * s, 4 * s, 4 * (L0 - t)};
  for (int d = 0; d < 3; ++d) {
    double a = 0, b = 0, c = 0;
    for (int q = 0; q < 6; ++q) {
      a += N[q] * E->P[q][d];
      b += A[q] * E->P[q][d];
      c += B[q] * E->P[q][d];
    }
    y[d] = a;
    y1[d] = b;
    y2[d] = c;
  }
}

static inline void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static inline double dist3(const double a[3], const double b[3]) {
  double d[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
  return norm3(d);
}

/* point, paper normal (into the body) and area Jacobian at (s, t) */
static void elem_point(const elem_t* E, double s, double t, double y[3], double n[3], double* J) {
  double y1[3], y2[3], c[3];
  elem_eval(E, s, t, y, y1, y2);
  cross3(y1, y2, c);
  double j = norm3(c);
  double sg = (q_debug & 4) ? 1.0 : -1.0;
  for (int d = 0; d < 3; ++d) n[d] = sg * c[d] / j;
  *J = j;
}

/* ---------------- kernels (Eq. fundsol and the layer operators) ---------------- */
/* r = x - y. Returns G, dG/dn_y, dG/dn_x, d2G/dn_x dn_y. */
static void kern4(const double x[3], const double nx[3], const double y[3], const double ny[3], double k,
                  cplx out[4]) {
  double r[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
  double R = norm3(r);
  double rnx = dot3(r, nx) / R, rny = dot3(r, ny) / R, nxny = dot3(nx, ny);
  cplx G = cexp(I * k * R) / (4.0 * PI_ * R);
  out[0] = G;
  out[1] = G * (1.0 / R - I * k) * rny;
  out[2] = G * (I * k - 1.0 / R) * rnx;
  out[3] = G / (R * R) * (nxny * (1.0 - I * k * R) - rnx * rny * (3.0 - 3.0 * I * k * R - k * k * R * R));
}

int orc_kernel_eval(int64_t m, const double* x, const double* nx, const double* y, const double* ny, double k,
                    double* out /* m x 4 complex */) {
  for (int64_t i = 0; i < m; ++i) {
    cplx o[4];
    kern4(x + 3 * i, nx + 3 * i, y + 3 * i, ny + 3 * i, k, o);
    for (int q = 0; q < 4; ++q) {
      out[8 * i + 2 * q] = creal(o[q]);
      out[8 * i + 2 * q + 1] = cimag(o[q]);
    }
  }
  return 0;
}

/* ---------------- particle summation (Sec. 5.1, Eq. sum) ----------------
 * p_i = sum_{j != i} [G(x_i, y_j) + alpha dG/dn_y(x_i, y_j)] q_j at the listed rows, by direct summation
 * (the "straightforward summation" the paper measures the FDA against). Points are both targets and
 * sources; normals are those of the sources. */
int orc_particle_rows(const double* x, const double* n, int64_t N, double k, double alpha_re, double alpha_im,
                      const double* q /* N complex */, const int64_t* rows, int64_t nrows, double* out) {
  const cplx alpha = alpha_re + I * alpha_im;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = rows[r];
    cplx acc = 0;
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue;
      cplx kv[4];
      kern4(x + 3 * i, n + 3 * i, x + 3 * j, n + 3 * j, k, kv);
      acc += (kv[0] + alpha * kv[1]) * (q[2 * j] + I * q[2 * j + 1]);
    }
    out[2 * r] = creal(acc);
    out[2 * r + 1] = cimag(acc);
  }
  return 0;
}

/* The same sum at arbitrary target points t (not sources): p(t) = sum_j [G + alpha dG/dn_y](t, y_j) q_j. */
int orc_particle_field(const double* x, const double* n, int64_t N, double k, double alpha_re, double alpha_im,
                       const double* q, const double* t, int64_t nt, double* out) {
  const cplx alpha = alpha_re + I * alpha_im;
  const double zero[3] = {0, 0, 0};
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nt; ++r) {
    cplx acc = 0;
    for (int64_t j = 0; j < N; ++j) {
      cplx kv[4];
      kern4(t + 3 * r, zero, x + 3 * j, n + 3 * j, k, kv);
      acc += (kv[0] + alpha * kv[1]) * (q[2 * j] + I * q[2 * j + 1]);
    }
    out[2 * r] = creal(acc);
    out[2 * r + 1] = cimag(acc);
  }
  return 0;
}

/* ---------------- polynomial basis of the local correction ---------------- */
static inline void basis(double s, double t, double phi[6]) {
  phi[0] = 1.0;
  phi[1] = s;
  phi[2] = t;
  phi[3] = s * s;
  phi[4] = s * t;
  phi[5] = t * t;
}
static inline void basis_dir(double s, double t, double e1, double e2, double dphi[6]) {
  dphi[0] = 0.0;
  dphi[1] = e1;
  dphi[2] = e2;
  dphi[3] = 2 * s * e1;
  dphi[4] = t * e1 + s * e2;
  dphi[5] = 2 * t * e2;
}

/* Phi[n][j] = phi_n(xi_j); PhiInv solves sum_j Phi[n][j] w_j = I_n. */
static double PhiInv[6][6];
static int phi_ready = 0;
static void phi_init(void) {
  if (phi_ready) return;
  double M[6][12];
  for (int n = 0; n < 6; ++n) {
    for (int j = 0; j < 6; ++j) {
      double p[6];
      basis(GXI[j][0], GXI[j][1], p);
      M[n][j] = p[n];
      M[n][6 + j] = (n == j) ? 1.0 : 0.0;
    }
  }
  for (int c = 0; c < 6; ++c) { /* Gauss-Jordan with partial pivoting */
    int piv = c;
    for (int r = c + 1; r < 6; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    for (int q = 0; q < 12; ++q) {
      double tmp = M[c][q];
      M[c][q] = M[piv][q];
      M[piv][q] = tmp;
    }
    double d = M[c][c];
    for (int q = 0; q < 12; ++q) M[c][q] /= d;
    for (int r = 0; r < 6; ++r)
      if (r != c) {
        double f = M[r][c];
        for (int q = 0; q < 12; ++q) M[r][q] -= f * M[c][q];
      }
  }
  for (int n = 0; n < 6; ++n)
    for (int j = 0; j < 6; ++j) PhiInv[n][j] = M[n][6 + j];
  phi_ready = 1;
}

void orc_phi_matrix(double* phi /*6x6, [n][j]*/, double* phiinv /*6x6*/) {
  phi_init();
  for (int n = 0; n < 6; ++n)
    for (int j = 0; j < 6; ++j) {
      double p[6];
      basis(GXI[j][0], GXI[j][1], p);
      phi[6 * n + j] = p[n];
      phiinv[6 * n + j] = PhiInv[n][j];
    }
}

/* ---------------- moments over the element carrying x_i (singular) ---------------- */
/* ID[n] = int dG/dn_y phi_n dS (weakly singular on a smooth surface: bounded in polar coordinates).
 * IH[n] = finite part of int d2G/dn_x dn_y phi_n dS. In polar coordinates (rho, theta) about
 * xi0 the integrand F = K phi J rho has the expansion F_{-2}/rho^2 + F_{-1}/rho + O(1); the
 * finite part for a spherical exclusion neighbourhood is
 *   sum over sectors of int dtheta { int_0^rhohat (F - F_{-2}/rho^2 - F_{-1}/rho) drho
 *        + F_{-1} ln(rhohat/beta) - F_{-2} (gamma/beta^2 + 1/rhohat) },
 * with y(xi0 + rho e) - x = rho A + rho^2 B, beta = 1/|A|, gamma = -(A.B)/|A|^4.
 * Only the Laplace part (n_x.n_y)/(4 pi R^3) of d2G/dn_x dn_y reaches order rho^-2 or rho^-1:
 *   F_{-2} = phi0 J0 / (4 pi |A|^3),
 *   F_{-1} = (J1 phi0 + J0 phi1 - 3 J0 phi0 (A.B)/|A|^2) / (4 pi |A|^3),
 * J1, phi1 the directional derivatives of J and phi along e at xi0. */
static void moments_self4(const elem_t* E, int g, double k, cplx IG[6], cplx ID[6], cplx IM[6], cplx IH[6]) {
  double gx[GL_MAX], gw[GL_MAX], rx[GL_MAX], rw[GL_MAX];
  gauss_legendre01(q_ntheta, gx, gw);
  gauss_legendre01(q_nrho, rx, rw);
  double s0 = GXI[g][0], t0 = GXI[g][1];
  double x[3], x1[3], x2[3], N0[3], nx[3];
  elem_eval(E, s0, t0, x, x1, x2);
  cross3(x1, x2, N0);
  double J0 = norm3(N0);
  double sg = (q_debug & 4) ? 1.0 : -1.0;
  for (int d = 0; d < 3; ++d) nx[d] = sg * N0[d] / J0;
  /* gradient of J at xi0: dJ/dxi_a = N0 . dN/dxi_a / J0 */
  double dN1[3], dN2[3], ta[3], tb[3];
  cross3(E->y11, x2, ta);
  cross3(x1, E->y12, tb);
  for (int d = 0; d < 3; ++d) dN1[d] = ta[d] + tb[d];
  cross3(E->y12, x2, ta);
  cross3(x1, E->y22, tb);
  for (int d = 0; d < 3; ++d) dN2[d] = ta[d] + tb[d];
  double gJ1 = dot3(N0, dN1) / J0, gJ2 = dot3(N0, dN2) / J0;
  double phi0[6];
  basis(s0, t0, phi0);
  for (int n = 0; n < 6; ++n) IG[n] = ID[n] = IM[n] = IH[n] = 0.0;
  const double V[3][2] = {{0, 0}, {1, 0}, {0, 1}};
  for (int ed = 0; ed < 3; ++ed) {
    const double* Pv = V[ed];
    const double* Qv = V[(ed + 1) % 3];
    double ux = Qv[0] - Pv[0], uy = Qv[1] - Pv[1], ul = sqrt(ux * ux + uy * uy);
    ux /= ul;
    uy /= ul;
    double pr = (s0 - Pv[0]) * ux + (t0 - Pv[1]) * uy;
    double fx = Pv[0] + pr * ux - s0, fy = Pv[1] + pr * uy - t0;
    double dperp = sqrt(fx * fx + fy * fy), thn = atan2(fy, fx);
    /* angles relative to the foot of the perpendicular, in (-pi/2, pi/2); rhohat = dperp / cos(phi) */
    double phP = atan2(-(Pv[0] - s0) * fy / dperp + (Pv[1] - t0) * fx / dperp,
                       ((Pv[0] - s0) * fx + (Pv[1] - t0) * fy) / dperp);
    double phQ = atan2(-(Qv[0] - s0) * fy / dperp + (Qv[1] - t0) * fx / dperp,
                       ((Qv[0] - s0) * fx + (Qv[1] - t0) * fy) / dperp);
    /* break points: the foot (if inside the edge) and a geometric grading towards the poles of
       1/cos(phi) at +-pi/2, so every sub-interval is no longer than its distance to the pole */
    double bp[128];
    int nb = 0;
    bp[nb++] = phP;
    if (phP < 0.0) {
      double dl = 0.5 * PI_ + phP; /* distance of the lower end to -pi/2 */
      for (double q = 2 * dl; -0.5 * PI_ + q < fmin(0.0, phQ) && nb < 60; q *= 2) bp[nb++] = -0.5 * PI_ + q;
      if (phQ > 0.0) bp[nb++] = 0.0;
    }
    if (phQ > 0.0) {
      double du = 0.5 * PI_ - phQ;
      double tmp[64];
      int nt = 0;
      for (double q = 2 * du; 0.5 * PI_ - q > fmax(0.0, phP) && nt < 60; q *= 2) tmp[nt++] = 0.5 * PI_ - q;
      for (int q = nt - 1; q >= 0; --q) bp[nb++] = tmp[q];
    }
    bp[nb++] = phQ;
    for (int iv = 0; iv + 1 < nb; ++iv) {
      double pa = bp[iv], pb = bp[iv + 1];
      if (!(pb > pa)) continue;
      for (int a = 0; a < q_ntheta; ++a) {
        double ph = pa + (pb - pa) * gx[a], wth = (pb - pa) * gw[a];
        double th = thn + ph;
        double e1 = cos(th), e2 = sin(th);
        double rhohat = dperp / cos(ph);
        double A[3], B[3];
        for (int d = 0; d < 3; ++d) {
          A[d] = x1[d] * e1 + x2[d] * e2;
          B[d] = 0.5 * (E->y11[d] * e1 * e1 + 2 * E->y12[d] * e1 * e2 + E->y22[d] * e2 * e2);
        }
        double An = norm3(A), AB = dot3(A, B);
        double J1 = gJ1 * e1 + gJ2 * e2;
        double phi1[6];
        basis_dir(s0, t0, e1, e2, phi1);
        double Fm2[6], Fm1[6];
        double c3 = 1.0 / (4 * PI_ * An * An * An);
        for (int n = 0; n < 6; ++n) {
          Fm2[n] = phi0[n] * J0 * c3;
          Fm1[n] = (J1 * phi0[n] + J0 * phi1[n] - 3.0 * J0 * phi0[n] * AB / (An * An)) * c3;
          if (q_debug & 1) Fm1[n] = 0.0;
        }
        double beta = 1.0 / An, gamma = -AB / (An * An * An * An);
        if (q_debug & 2) gamma = 0.0;
        for (int b = 0; b < q_nrho; ++b) {
          double rho = rhohat * rx[b], wr = rhohat * rw[b];
          double y[3], ny[3], J;
          elem_point(E, s0 + rho * e1, t0 + rho * e2, y, ny, &J);
          cplx kk[4];
          kern4(x, nx, y, ny, k, kk);
          double phi[6];
          basis(s0 + rho * e1, t0 + rho * e2, phi);
          for (int n = 0; n < 6; ++n) {
            /* G ~ 1/rho and dG/dn_x ~ (r.n_x)/rho^3 ~ 1/rho: bounded once multiplied by rho */
            IG[n] += wth * wr * kk[0] * phi[n] * J * rho;
            ID[n] += wth * wr * kk[1] * phi[n] * J * rho;
            IM[n] += wth * wr * kk[2] * phi[n] * J * rho;
            IH[n] += wth * wr * (kk[3] * phi[n] * J * rho - Fm2[n] / (rho * rho) - Fm1[n] / rho);
          }
        }
        for (int n = 0; n < 6; ++n)
          IH[n] += wth * (Fm1[n] * log(rhohat / beta) - Fm2[n] * (gamma / (beta * beta) + 1.0 / rhohat));
      }
    }
  }
}

static void moments_self(const elem_t* E, int g, double k, cplx ID[6], cplx IH[6]) {
  cplx IG[6], IM[6];
  moments_self4(E, g, k, IG, ID, IM, IH);
}

/* ---------------- moments over a nearby element (nearly singular): recursive subdivision ---------------- */
static void moments_sub_rec(const elem_t* E, const double x[3], const double nx[3], double k, const double T[3][2],
                            int depth, const double* qx, const double* qw, cplx I4[4][6]) {
  double pts[7][2] = {
      {T[0][0], T[0][1]},
      {T[1][0], T[1][1]},
      {T[2][0], T[2][1]},
      {0.5 * (T[0][0] + T[1][0]), 0.5 * (T[0][1] + T[1][1])},
      {0.5 * (T[1][0] + T[2][0]), 0.5 * (T[1][1] + T[2][1])},
      {0.5 * (T[2][0] + T[0][0]), 0.5 * (T[2][1] + T[0][1])},
      {(T[0][0] + T[1][0] + T[2][0]) / 3.0, (T[0][1] + T[1][1] + T[2][1]) / 3.0}};
  double P[7][3], ya[3], yb[3];
  for (int q = 0; q < 7; ++q) elem_eval(E, pts[q][0], pts[q][1], P[q], ya, yb);
  double diam = fmax(dist3(P[0], P[1]), fmax(dist3(P[1], P[2]), dist3(P[2], P[0])));
  double dmin = 1e300;
  for (int q = 0; q < 7; ++q) dmin = fmin(dmin, dist3(x, P[q]));
  if (dmin >= q_eta * diam || depth >= q_maxdepth) {
    double ex = T[1][0] - T[0][0], ey = T[1][1] - T[0][1];
    double fx = T[2][0] - T[0][0], fy = T[2][1] - T[0][1];
    double jac = fabs(ex * fy - ey * fx);
    for (int a = 0; a < q_nsub; ++a)
      for (int b = 0; b < q_nsub; ++b) {
        double u = qx[a], v = qx[b] * (1.0 - qx[a]);
        double w = qw[a] * qw[b] * (1.0 - qx[a]) * jac;
        double s = T[0][0] + u * ex + v * fx, t = T[0][1] + u * ey + v * fy;
        double y[3], ny[3], J;
        elem_point(E, s, t, y, ny, &J);
        cplx kk[4];
        kern4(x, nx, y, ny, k, kk);
        double phi[6];
        basis(s, t, phi);
        for (int n = 0; n < 6; ++n)
          for (int q = 0; q < 4; ++q) I4[q][n] += w * kk[q] * phi[n] * J;
      }
    return;
  }
  double m01[2] = {pts[3][0], pts[3][1]}, m12[2] = {pts[4][0], pts[4][1]}, m20[2] = {pts[5][0], pts[5][1]};
  double C[4][3][2] = {
      {{T[0][0], T[0][1]}, {m01[0], m01[1]}, {m20[0], m20[1]}},
      {{m01[0], m01[1]}, {T[1][0], T[1][1]}, {m12[0], m12[1]}},
      {{m20[0], m20[1]}, {m12[0], m12[1]}, {T[2][0], T[2][1]}},
      {{m01[0], m01[1]}, {m12[0], m12[1]}, {m20[0], m20[1]}}};
  for (int c = 0; c < 4; ++c) moments_sub_rec(E, x, nx, k, (const double(*)[2])C[c], depth + 1, qx, qw, I4);
}

/* moments of G, dG/dn_y, dG/dn_x, d2G/dn_x dn_y (I4[0..3]) over a nearby element */
static void moments_near4(const elem_t* E, const double x[3], const double nx[3], double k, cplx I4[4][6]) {
  double qx[GL_MAX], qw[GL_MAX];
  gauss_legendre01(q_nsub, qx, qw);
  for (int q = 0; q < 4; ++q)
    for (int n = 0; n < 6; ++n) I4[q][n] = 0.0;
  const double T[3][2] = {{0, 0}, {1, 0}, {0, 1}};
  moments_sub_rec(E, x, nx, k, T, 0, qx, qw, I4);
}

static void moments_near(const elem_t* E, const double x[3], const double nx[3], double k, cplx ID[6], cplx IH[6]) {
  cplx I4[4][6];
  moments_near4(E, x, nx, k, I4);
  for (int n = 0; n < 6; ++n) {
    ID[n] = I4[1][n];
    IH[n] = I4[3][n];
  }
}

/* Moments of element e for target x (x = Nystrom point g of e when self_g >= 0). */
int orc_moments(const double* nodes, const int32_t* elems, int64_t e, int self_g, const double* x, const double* nx,
                double k, double* out /* 2 x 6 complex: ID then IH */) {
  elem_t E;
  elem_load(&E, nodes, elems + 6 * e);
  cplx ID[6], IH[6];
  if (self_g >= 0)
    moments_self(&E, self_g, k, ID, IH);
  else
    moments_near(&E, x, nx, k, ID, IH);
  for (int n = 0; n < 6; ++n) {
    out[2 * n] = creal(ID[n]);
    out[2 * n + 1] = cimag(ID[n]);
    out[12 + 2 * n] = creal(IH[n]);
    out[12 + 2 * n + 1] = cimag(IH[n]);
  }
  return 0;
}

/* ---------------- Nystrom points ---------------- */
int orc_geometry(const double* nodes, int64_t nn, const int32_t* elems, int64_t ne, double* xs, double* ns,
                 double* ws) {
  (void)nn;
  for (int64_t e = 0; e < ne; ++e) {
    elem_t E;
    elem_load(&E, nodes, elems + 6 * e);
    for (int j = 0; j < 6; ++j) {
      double J;
      int64_t i = 6 * e + j;
      elem_point(&E, GXI[j][0], GXI[j][1], xs + 3 * i, ns + 3 * i, &J);
      ws[i] = GWT[j] * J;
    }
  }
  return 0;
}

/* ---------------- local region D_i ---------------- */
/* D_i: elements whose distance to x_i is <= 2x their largest side. Distance = min over the element's
 * 6 nodes and 6 Nystrom points; largest side = longest of the three vertex chords. */
static int in_local_region(const elem_t* E, const double* xsE /* 6x3 Nystrom points of E */, const double x[3]) {
  double side = fmax(dist3(E->P[0], E->P[1]), fmax(dist3(E->P[1], E->P[2]), dist3(E->P[2], E->P[0])));
  double d = 1e300;
  for (int a = 0; a < 6; ++a) d = fmin(d, dist3(x, E->P[a]));
  for (int a = 0; a < 6; ++a) d = fmin(d, dist3(x, xsE + 3 * a));
  return d <= 2.0 * side;
}

typedef struct {
  const double* nodes;
  const int32_t* elems;
  int64_t ne;
  double* xs;
  double* ns;
  double* ws;
} mesh_t;

static int mesh_init(mesh_t* M, const double* nodes, int64_t nn, const int32_t* elems, int64_t ne) {
  M->nodes = nodes;
  M->elems = elems;
  M->ne = ne;
  int64_t N = 6 * ne;
  M->xs = (double*)malloc(sizeof(double) * 3 * N);
  M->ns = (double*)malloc(sizeof(double) * 3 * N);
  M->ws = (double*)malloc(sizeof(double) * N);
  if (!M->xs || !M->ns || !M->ws) return -1;
  orc_geometry(nodes, nn, elems, ne, M->xs, M->ns, M->ws);
  return 0;
}
static void mesh_free(mesh_t* M) {
  free(M->xs);
  free(M->ns);
  free(M->ws);
}

/* local-region elements of point i, appended to list (returns count, -1 on overflow) */
static int64_t local_region(const mesh_t* M, int64_t i, int32_t* list, int64_t cap) {
  int64_t c = 0;
  const double* x = M->xs + 3 * i;
  for (int64_t e = 0; e < M->ne; ++e) {
    elem_t E;
    elem_load(&E, M->nodes, M->elems + 6 * e);
    if (in_local_region(&E, M->xs + 18 * e, x)) {
      if (c >= cap) return -1;
      list[c++] = (int32_t)e;
    }
  }
  return c;
}

int orc_local_region(const double* nodes, int64_t nn, const int32_t* elems, int64_t ne, const int64_t* rows,
                     int64_t nrows, int64_t cap, int64_t* counts, int32_t* lists) {
  mesh_t M;
  if (mesh_init(&M, nodes, nn, elems, ne)) return -2;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t c = local_region(&M, rows[r], lists + r * cap, cap);
    counts[r] = c;
    if (c < 0) err = -1;
  }
  mesh_free(&M);
  return err;
}

/* corrected weights of row i for both kernels: wD, wH are (count x 6) */
static int64_t row_corrections(const mesh_t* M, int64_t i, double k, int32_t* list, int64_t cap, cplx* wD,
                               cplx* wH) {
  phi_init();
  int64_t c = local_region(M, i, list, cap);
  if (c < 0) return c;
  int64_t ei = i / 6;
  int gi = (int)(i % 6);
  const double* x = M->xs + 3 * i;
  const double* nx = M->ns + 3 * i;
  for (int64_t q = 0; q < c; ++q) {
    elem_t E;
    elem_load(&E, M->nodes, M->elems + 6 * (int64_t)list[q]);
    cplx ID[6], IH[6];
    if (list[q] == ei)
      moments_self(&E, gi, k, ID, IH);
    else
      moments_near(&E, x, nx, k, ID, IH);
    for (int j = 0; j < 6; ++j) {
      cplx a = 0, b = 0;
      for (int n = 0; n < 6; ++n) {
        a += PhiInv[j][n] * ID[n];
        b += PhiInv[j][n] * IH[n];
      }
      wD[6 * q + j] = a;
      wH[6 * q + j] = b;
    }
  }
  return c;
}

int orc_correction_weights(const double* nodes, int64_t nn, const int32_t* elems, int64_t ne, double k,
                           const int64_t* rows, int64_t nrows, int64_t cap, int64_t* counts, int32_t* lists,
                           double* wD /* nrows x cap x 6 complex */, double* wH) {
  mesh_t M;
  if (mesh_init(&M, nodes, nn, elems, ne)) return -2;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    cplx* a = (cplx*)(wD + 2 * 6 * cap * r);
    cplx* b = (cplx*)(wH + 2 * 6 * cap * r);
    int64_t c = row_corrections(&M, rows[r], k, lists + r * cap, cap, a, b);
    counts[r] = c;
    if (c < 0) err = -1;
  }
  mesh_free(&M);
  return err;
}

/* ---------------- rows of A = c I + beta_D Dbar + beta_H Hbar (Eq. kcorrection, Eq. bm) ---------------- */
#define DI_CAP 4096
static int row_apply(const mesh_t* M, int64_t i, double k, double c, cplx bD, cplx bH, const cplx* xv, cplx* out,
                     cplx* dense_row) {
  int32_t list[DI_CAP];
  cplx* wD = (cplx*)malloc(sizeof(cplx) * 6 * DI_CAP);
  cplx* wH = (cplx*)malloc(sizeof(cplx) * 6 * DI_CAP);
  if (!wD || !wH) {
    free(wD);
    free(wH);
    return -2;
  }
  int64_t nl = row_corrections(M, i, k, list, DI_CAP, wD, wH);
  if (nl < 0) {
    free(wD);
    free(wH);
    return -1;
  }
  int64_t N = 6 * M->ne;
  char* inD = (char*)calloc((size_t)M->ne, 1);
  for (int64_t q = 0; q < nl; ++q) inD[list[q]] = 1;
  const double* x = M->xs + 3 * i;
  const double* nx = M->ns + 3 * i;
  cplx acc = c * (xv ? xv[i] : 0.0);
  if (dense_row) {
    for (int64_t j = 0; j < N; ++j) dense_row[j] = 0.0;
    dense_row[i] += c;
  }
  for (int64_t e = 0; e < M->ne; ++e) {
    if (inD[e]) continue;
    for (int a = 0; a < 6; ++a) {
      int64_t j = 6 * e + a;
      cplx kk[4];
      kern4(x, nx, M->xs + 3 * j, M->ns + 3 * j, k, kk);
      cplx v = (bD * kk[1] + bH * kk[3]) * M->ws[j];
      if (xv) acc += v * xv[j];
      if (dense_row) dense_row[j] += v;
    }
  }
  for (int64_t q = 0; q < nl; ++q)
    for (int a = 0; a < 6; ++a) {
      int64_t j = 6 * (int64_t)list[q] + a;
      cplx v = bD * wD[6 * q + a] + bH * wH[6 * q + a];
      if (xv) acc += v * xv[j];
      if (dense_row) dense_row[j] += v;
    }
  free(inD);
  free(wD);
  free(wH);
  if (out) *out = acc;
  return 0;
}

/* ---------------- rows of c I + bS Sbar + bD Dbar + bM Mbar + bH Hbar (all four layer operators) ----------------
 * The corrected weights of every kernel come from its own moments (Eq. local correction); the radiation
 * right-hand side of Eq. bm is (Sbar + alpha Mbar - alpha/2 I) q. */
static int row_apply4(const mesh_t* M, int64_t i, double k, cplx c, const cplx b[4], const cplx* xv, cplx* out) {
  phi_init();
  int32_t* list = (int32_t*)malloc(sizeof(int32_t) * DI_CAP);
  cplx* wb = (cplx*)malloc(sizeof(cplx) * 6 * DI_CAP);
  if (!list || !wb) {
    free(list);
    free(wb);
    return -2;
  }
  int64_t nl = local_region(M, i, list, DI_CAP);
  if (nl < 0) {
    free(list);
    free(wb);
    return -1;
  }
  const int64_t ei = i / 6;
  const int gi = (int)(i % 6);
  const double* x = M->xs + 3 * i;
  const double* nx = M->ns + 3 * i;
  for (int64_t q = 0; q < nl; ++q) {
    elem_t E;
    elem_load(&E, M->nodes, M->elems + 6 * (int64_t)list[q]);
    cplx I4[4][6];
    if (list[q] == ei)
      moments_self4(&E, gi, k, I4[0], I4[1], I4[2], I4[3]);
    else
      moments_near4(&E, x, nx, k, I4);
    for (int j = 0; j < 6; ++j) {
      cplx a = 0;
      for (int n = 0; n < 6; ++n) a += PhiInv[j][n] * (b[0] * I4[0][n] + b[1] * I4[1][n] + b[2] * I4[2][n] + b[3] * I4[3][n]);
      wb[6 * q + j] = a;
    }
  }
  char* inD = (char*)calloc((size_t)M->ne, 1);
  for (int64_t q = 0; q < nl; ++q) inD[list[q]] = 1;
  cplx acc = c * xv[i];
  for (int64_t e = 0; e < M->ne; ++e) {
    if (inD[e]) continue;
    for (int a = 0; a < 6; ++a) {
      int64_t j = 6 * e + a;
      cplx kk[4];
      kern4(x, nx, M->xs + 3 * j, M->ns + 3 * j, k, kk);
      acc += (b[0] * kk[0] + b[1] * kk[1] + b[2] * kk[2] + b[3] * kk[3]) * M->ws[j] * xv[j];
    }
  }
  for (int64_t q = 0; q < nl; ++q)
    for (int a = 0; a < 6; ++a) acc += wb[6 * q + a] * xv[6 * (int64_t)list[q] + a];
  free(inD);
  free(list);
  free(wb);
  *out = acc;
  return 0;
}

int orc_rows4(const double* nodes, int64_t nn, const int32_t* elems, int64_t ne, double k, double c_re, double c_im,
              const double* b /* 4 complex: S, D, M, H */, const double* xv, const int64_t* rows, int64_t nrows,
              double* y) {
  mesh_t M;
  if (mesh_init(&M, nodes, nn, elems, ne)) return -2;
  const cplx c = c_re + I * c_im;
  cplx bb[4];
  for (int q = 0; q < 4; ++q) bb[q] = b[2 * q] + I * b[2 * q + 1];
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    cplx o = 0;
    if (row_apply4(&M, rows[r], k, c, bb, (const cplx*)xv, &o)) err = -1;
    y[2 * r] = creal(o);
    y[2 * r + 1] = cimag(o);
  }
  mesh_free(&M);
  return err;
}

int orc_matvec_rows(const double* nodes, int64_t nn, const int32_t* elems, int64_t ne, double k, double c,
                    double bD_re, double bD_im, double bH_re, double bH_im, const double* xv /* N complex */,
                    const int64_t* rows, int64_t nrows, double* y /* nrows complex */) {
  mesh_t M;
  if (mesh_init(&M, nodes, nn, elems, ne)) return -2;
  cplx bD = bD_re + I * bD_im, bH = bH_re + I * bH_im;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    cplx o;
    if (row_apply(&M, rows[r], k, c, bD, bH, (const cplx*)xv, &o, NULL)) err = -1;
    y[2 * r] = creal(o);
    y[2 * r + 1] = cimag(o);
  }
  mesh_free(&M);
  return err;
}

int orc_dense_matrix(const double* nodes, int64_t nn, const int32_t* elems, int64_t ne, double k, double c,
                     double bD_re, double bD_im, double bH_re, double bH_im, double* A /* N x N complex */) {
  mesh_t M;
  if (mesh_init(&M, nodes, nn, elems, ne)) return -2;
  cplx bD = bD_re + I * bD_im, bH = bH_re + I * bH_im;
  int64_t N = 6 * ne;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < N; ++i) {
    if (row_apply(&M, i, k, c, bD, bH, NULL, NULL, (cplx*)(A + 2 * N * i))) err = -1;
  }
  mesh_free(&M);
  return err;
}

/* ================================================================================================ */
/* Octree and interaction lists (Sec. 3.1.1) under integer rules                                    */
/* ================================================================================================ */
#define QBITS 21

typedef struct {
  int64_t N;
  int leaf_max;
  double k;
  double corner[3], side;
  int64_t* perm;
  uint64_t* keys;
  int64_t nbox, cap;
  int32_t *lev, *bx, *by, *bz, *nch, *leaf;
  int64_t *par, *cbeg, *pb, *pe;
  int nlev;
  int32_t lev_hf[QBITS + 2], lev_T[QBITS + 2], lev_n[QBITS + 2];
  int64_t ndir, capd;
  int64_t *dt, *ds;
  int64_t nm, capm;
  int64_t *mt, *ms;
  int32_t *ml, *mdx, *mdy, *mdz, *mwo, *mwi;
} otree_t;

typedef struct {
  uint64_t key;
  int64_t idx;
} kv_t;
static int kv_cmp(const void* a, const void* b) {
  const kv_t* x = (const kv_t*)a;
  const kv_t* y = (const kv_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static uint64_t spread3(uint64_t v) {
  uint64_t r = 0;
  for (int b = 0; b < QBITS; ++b) r |= ((v >> b) & 1ull) << (3 * b);
  return r;
}

static void box_push(otree_t* T, int l, int32_t x, int32_t y, int32_t z, int64_t parent, int64_t b, int64_t e) {
  if (T->nbox == T->cap) {
    T->cap = T->cap ? 2 * T->cap : 1024;
#define GROW(p, t) p = (t*)realloc(p, sizeof(t) * T->cap)
    GROW(T->lev, int32_t);
    GROW(T->bx, int32_t);
    GROW(T->by, int32_t);
    GROW(T->bz, int32_t);
    GROW(T->nch, int32_t);
    GROW(T->leaf, int32_t);
    GROW(T->par, int64_t);
    GROW(T->cbeg, int64_t);
    GROW(T->pb, int64_t);
    GROW(T->pe, int64_t);
#undef GROW
  }
  int64_t i = T->nbox++;
  T->lev[i] = l;
  T->bx[i] = x;
  T->by[i] = y;
  T->bz[i] = z;
  T->nch[i] = 0;
  T->leaf[i] = 1;
  T->par[i] = parent;
  T->cbeg[i] = -1;
  T->pb[i] = b;
  T->pe[i] = e;
}

/* wedge index of integer direction d at a level with n cells per face edge (Sec. 3.1.1, directional
 * wedges): face = axis of largest |d_i| (lowest axis on ties) and its sign; cell along each remaining
 * axis j (increasing order) = min(n-1, floor(n (d_j + m) / (2m))), m = |d_face|. */
static int32_t wedge_of(int n, int32_t dx, int32_t dy, int32_t dz) {
  int64_t d[3] = {dx, dy, dz};
  int64_t ad[3] = {llabs(d[0]), llabs(d[1]), llabs(d[2])};
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

int32_t orc_wedge_of(int n, int32_t dx, int32_t dy, int32_t dz) { return wedge_of(n, dx, dy, dz); }

static void dir_push(otree_t* T, int64_t t, int64_t s) {
  if (T->ndir == T->capd) {
    T->capd = T->capd ? 2 * T->capd : 4096;
    T->dt = (int64_t*)realloc(T->dt, sizeof(int64_t) * T->capd);
    T->ds = (int64_t*)realloc(T->ds, sizeof(int64_t) * T->capd);
  }
  T->dt[T->ndir] = t;
  T->ds[T->ndir] = s;
  T->ndir++;
}
static void m2l_push(otree_t* T, int l, int64_t t, int64_t s, int32_t dx, int32_t dy, int32_t dz) {
  if (T->nm == T->capm) {
    T->capm = T->capm ? 2 * T->capm : 4096;
#define GROW(p, ty) p = (ty*)realloc(p, sizeof(ty) * T->capm)
    GROW(T->mt, int64_t);
    GROW(T->ms, int64_t);
    GROW(T->ml, int32_t);
    GROW(T->mdx, int32_t);
    GROW(T->mdy, int32_t);
    GROW(T->mdz, int32_t);
    GROW(T->mwo, int32_t);
    GROW(T->mwi, int32_t);
#undef GROW
  }
  int64_t i = T->nm++;
  T->mt[i] = t;
  T->ms[i] = s;
  T->ml[i] = l;
  T->mdx[i] = dx;
  T->mdy[i] = dy;
  T->mdz[i] = dz;
  if (T->lev_hf[l]) {
    int n = T->lev_n[l];
    T->mwo[i] = wedge_of(n, -dx, -dy, -dz); /* source's outgoing wedge: direction source -> target */
    T->mwi[i] = wedge_of(n, dx, dy, dz);    /* target's incoming wedge: direction target -> source */
  } else {
    T->mwo[i] = 0;
    T->mwi[i] = 0;
  }
}

typedef struct {
  int64_t a, b;
} pair_t;
static int pair_cmp(const void* x, const void* y) {
  const pair_t* p = (const pair_t*)x;
  const pair_t* q = (const pair_t*)y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  return p->b < q->b ? -1 : (p->b > q->b);
}

void* orc_tree_build(const double* pts, int64_t N, int leaf_max, double k) {
  otree_t* T = (otree_t*)calloc(1, sizeof(otree_t));
  T->N = N;
  T->leaf_max = leaf_max;
  T->k = k;
  /* root cube: bounding-box centre, side = largest extent * (1 + 2^-20) */
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin(lo[d], pts[3 * i + d]);
      hi[d] = fmax(hi[d], pts[3 * i + d]);
    }
  double ext = 0.0;
  for (int d = 0; d < 3; ++d) ext = fmax(ext, hi[d] - lo[d]);
  double side = ext * (1.0 + 9.5367431640625e-07);
  if (!(side > 0.0)) side = 1.0;
  T->side = side;
  for (int d = 0; d < 3; ++d) T->corner[d] = 0.5 * (lo[d] + hi[d]) - 0.5 * side;
  /* quantise to 21-bit integer coordinates and sort Morton keys (ties by input index) */
  kv_t* kv = (kv_t*)malloc(sizeof(kv_t) * (N > 0 ? N : 1));
  for (int64_t i = 0; i < N; ++i) {
    uint64_t q[3];
    for (int d = 0; d < 3; ++d) {
      double t = pts[3 * i + d] - T->corner[d];
      double u = t / side;
      double v = u * 2097152.0;
      double f = floor(v);
      int64_t qi = (int64_t)f;
      if (qi < 0) qi = 0;
      if (qi > (1 << QBITS) - 1) qi = (1 << QBITS) - 1;
      q[d] = (uint64_t)qi;
    }
    kv[i].key = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    kv[i].idx = i;
  }
  qsort(kv, (size_t)N, sizeof(kv_t), kv_cmp);
  T->perm = (int64_t*)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
  T->keys = (uint64_t*)malloc(sizeof(uint64_t) * (N > 0 ? N : 1));
  for (int64_t i = 0; i < N; ++i) {
    T->perm[i] = kv[i].idx;
    T->keys[i] = kv[i].key;
  }
  free(kv);
  /* level-by-level split of boxes holding more than leaf_max points */
  box_push(T, 0, 0, 0, 0, -1, 0, N);
  int64_t lb = 0, le = 1;
  int l = 0;
  while (l < QBITS) {
    int64_t before = T->nbox;
    for (int64_t b = lb; b < le; ++b) {
      if (T->pe[b] - T->pb[b] <= leaf_max) continue;
      int sh = 3 * (QBITS - 1 - l);
      int64_t p = T->pb[b];
      T->cbeg[b] = T->nbox;
      T->leaf[b] = 0;
      while (p < T->pe[b]) {
        int oct = (int)((T->keys[p] >> sh) & 7ull);
        int64_t q = p;
        while (q < T->pe[b] && (int)((T->keys[q] >> sh) & 7ull) == oct) ++q;
        box_push(T, l + 1, 2 * T->bx[b] + ((oct >> 2) & 1), 2 * T->by[b] + ((oct >> 1) & 1),
                 2 * T->bz[b] + (oct & 1), b, p, q);
        T->nch[b]++;
        p = q;
      }
    }
    if (T->nbox == before) break;
    lb = le;
    le = T->nbox;
    ++l;
  }
  T->nlev = l + 1;
  /* per-level regime and near-field threshold: HF iff k w >= 2 pi; T = floor(k w / pi) in HF, 0 in LF */
  int Lhf = -1;
  for (int q = 0; q < T->nlev; ++q) {
    double w = ldexp(side, -q);
    double kw = k * w;
    T->lev_hf[q] = (kw >= 2.0 * PI_) ? 1 : 0;
    T->lev_T[q] = T->lev_hf[q] ? (int32_t)floor(kw / PI_) : 0;
    if (T->lev_hf[q]) Lhf = q;
  }
  for (int q = 0; q < T->nlev; ++q) T->lev_n[q] = T->lev_hf[q] ? (1 << (Lhf - q)) : 1;
  /* dual recursion over near pairs, starting from (root, root) */
  pair_t* cur = (pair_t*)malloc(sizeof(pair_t));
  int64_t ncur = 1;
  cur[0].a = 0;
  cur[0].b = 0;
  for (int q = 0; q < T->nlev && ncur > 0; ++q) {
    int64_t capn = 1024, nn = 0;
    pair_t* nxt = (pair_t*)malloc(sizeof(pair_t) * capn);
    for (int64_t u = 0; u < ncur; ++u) {
      int64_t P = cur[u].a, Q = cur[u].b;
      if (T->leaf[P] || T->leaf[Q]) {
        dir_push(T, P, Q);
        continue;
      }
      for (int64_t c = T->cbeg[P]; c < T->cbeg[P] + T->nch[P]; ++c)
        for (int64_t d = T->cbeg[Q]; d < T->cbeg[Q] + T->nch[Q]; ++d) {
          int32_t dx = T->bx[d] - T->bx[c], dy = T->by[d] - T->by[c], dz = T->bz[d] - T->bz[c];
          int32_t m = abs(dx);
          if (abs(dy) > m) m = abs(dy);
          if (abs(dz) > m) m = abs(dz);
          if (m <= T->lev_T[q + 1] + 1) {
            if (nn == capn) {
              capn *= 2;
              nxt = (pair_t*)realloc(nxt, sizeof(pair_t) * capn);
            }
            nxt[nn].a = c;
            nxt[nn].b = d;
            nn++;
          } else {
            m2l_push(T, q + 1, c, d, dx, dy, dz);
          }
        }
    }
    free(cur);
    cur = nxt;
    ncur = nn;
  }
  free(cur);
  /* canonical order: by (target, source) */
  {
    pair_t* p = (pair_t*)malloc(sizeof(pair_t) * (T->ndir ? T->ndir : 1));
    for (int64_t i = 0; i < T->ndir; ++i) {
      p[i].a = T->dt[i];
      p[i].b = T->ds[i];
    }
    qsort(p, (size_t)T->ndir, sizeof(pair_t), pair_cmp);
    for (int64_t i = 0; i < T->ndir; ++i) {
      T->dt[i] = p[i].a;
      T->ds[i] = p[i].b;
    }
    free(p);
  }
  {
    int64_t n = T->nm;
    pair_t* p = (pair_t*)malloc(sizeof(pair_t) * (n ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
      p[i].a = T->mt[i] * (int64_t)(T->nbox + 1) + T->ms[i];
      p[i].b = i;
    }
    qsort(p, (size_t)n, sizeof(pair_t), pair_cmp);
    int64_t *mt = (int64_t*)malloc(8 * (n ? n : 1)), *ms = (int64_t*)malloc(8 * (n ? n : 1));
    int32_t* tmp[6];
    int32_t* src[6] = {T->ml, T->mdx, T->mdy, T->mdz, T->mwo, T->mwi};
    for (int f = 0; f < 6; ++f) tmp[f] = (int32_t*)malloc(4 * (n ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
      int64_t o = p[i].b;
      mt[i] = T->mt[o];
      ms[i] = T->ms[o];
      for (int f = 0; f < 6; ++f) tmp[f][i] = src[f][o];
    }
    for (int64_t i = 0; i < n; ++i) {
      T->mt[i] = mt[i];
      T->ms[i] = ms[i];
      for (int f = 0; f < 6; ++f) src[f][i] = tmp[f][i];
    }
    free(mt);
    free(ms);
    for (int f = 0; f < 6; ++f) free(tmp[f]);
    free(p);
  }
  return T;
}

void orc_tree_sizes(void* h, int64_t* out) {
  otree_t* T = (otree_t*)h;
  out[0] = T->nbox;
  out[1] = T->nlev;
  out[2] = T->ndir;
  out[3] = T->nm;
}

void orc_tree_export(void* h, double* geom /*4*/, int64_t* perm, uint64_t* keys, int32_t* box_i32 /*nbox x 6*/,
                     int64_t* box_i64 /*nbox x 4*/, int32_t* lev_i32 /*nlev x 3*/, int64_t* direct /*ndir x 2*/,
                     int64_t* m2l_i64 /*nm x 2*/, int32_t* m2l_i32 /*nm x 6*/) {
  otree_t* T = (otree_t*)h;
  for (int d = 0; d < 3; ++d) geom[d] = T->corner[d];
  geom[3] = T->side;
  memcpy(perm, T->perm, sizeof(int64_t) * T->N);
  memcpy(keys, T->keys, sizeof(uint64_t) * T->N);
  for (int64_t b = 0; b < T->nbox; ++b) {
    box_i32[6 * b + 0] = T->lev[b];
    box_i32[6 * b + 1] = T->bx[b];
    box_i32[6 * b + 2] = T->by[b];
    box_i32[6 * b + 3] = T->bz[b];
    box_i32[6 * b + 4] = T->nch[b];
    box_i32[6 * b + 5] = T->leaf[b];
    box_i64[4 * b + 0] = T->par[b];
    box_i64[4 * b + 1] = T->cbeg[b];
    box_i64[4 * b + 2] = T->pb[b];
    box_i64[4 * b + 3] = T->pe[b];
  }
  for (int q = 0; q < T->nlev; ++q) {
    lev_i32[3 * q + 0] = T->lev_hf[q];
    lev_i32[3 * q + 1] = T->lev_T[q];
    lev_i32[3 * q + 2] = T->lev_n[q];
  }
  for (int64_t i = 0; i < T->ndir; ++i) {
    direct[2 * i] = T->dt[i];
    direct[2 * i + 1] = T->ds[i];
  }
  for (int64_t i = 0; i < T->nm; ++i) {
    m2l_i64[2 * i] = T->mt[i];
    m2l_i64[2 * i + 1] = T->ms[i];
    m2l_i32[6 * i + 0] = T->ml[i];
    m2l_i32[6 * i + 1] = T->mdx[i];
    m2l_i32[6 * i + 2] = T->mdy[i];
    m2l_i32[6 * i + 3] = T->mdz[i];
    m2l_i32[6 * i + 4] = T->mwo[i];
    m2l_i32[6 * i + 5] = T->mwi[i];
  }
}

void orc_tree_free(void* h) {
  otree_t* T = (otree_t*)h;
  if (!T) return;
  free(T->perm);
  free(T->keys);
  free(T->lev);
  free(T->bx);
  free(T->by);
  free(T->bz);
  free(T->nch);
  free(T->leaf);
  free(T->par);
  free(T->cbeg);
  free(T->pb);
  free(T->pe);
  free(T->dt);
  free(T->ds);
  free(T->mt);
  free(T->ms);
  free(T->ml);
  free(T->mdx);
  free(T->mdy);
  free(T->mdz);
  free(T->mwo);
  free(T->mwi);
  free(T);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
