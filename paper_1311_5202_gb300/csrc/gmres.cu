// GMRES on A x = b (Eq. Axb; the paper solves with GMRES, tolerance = eps, Sec. 5.2).
// Restarted GMRES(m); Arnoldi in FP64 on the GPU with classical Gram-Schmidt applied twice (two passes of
// block dot products + update per step; numerically on par with modified Gram-Schmidt); the tiny Hessenberg
// least-squares problem (Givens rotations) on the host. Iterative refinement: outer FP64 residual
// r = b - A64 x, inner GMRES with the plan's FP32 operator on A d = r, x += d.
#include "plan.cuh"

#include <chrono>
#include <complex>

namespace fda {

typedef std::complex<double> zc;

int precond_apply(bm_precond_s* Pc, bm_net_s* net, const double2* r, double2* z, cudaStream_t s);

#define GM_NB 256
// partial[q * nb + blk] = sum_i conj(V_q[i]) w[i]
static __global__ void k_multidot(const double2* V, int64_t ldv, int nv, const double2* w, int64_t N,
                                  double2* partial, int nb) {
  __shared__ double2 sh[GM_NB / 32];
  const int q = blockIdx.y;
  const double2* v = V + (int64_t)q * ldv;
  double2 acc = make_double2(0, 0);
  for (int64_t i = (int64_t)blockIdx.x * GM_NB + threadIdx.x; i < N; i += (int64_t)nb * GM_NB) cjfma(acc, v[i], w[i]);
  acc = warp_csum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0, 0);
    for (int u = 0; u < GM_NB / 32; ++u) s = cadd(s, sh[u]);
    partial[(int64_t)q * nb + blockIdx.x] = s;
  }
}

static __global__ void k_reduce_partials(const double2* partial, int nb, int nv, double2* h, double2* hacc) {
  int q = blockIdx.x;
  __shared__ double2 sh[256];
  double2 s = make_double2(0, 0);
  for (int u = threadIdx.x; u < nb; u += 256) s = cadd(s, partial[(int64_t)q * nb + u]);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    h[q] = sh[0];
    if (hacc) hacc[q] = cadd(hacc[q], sh[0]);
  }
}

// w -= sum_q h_q V_q
static __global__ void k_update(const double2* V, int64_t ldv, int nv, const double2* h, double2* w, int64_t N) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double2 a = w[i];
  for (int q = 0; q < nv; ++q) {
    double2 hq = h[q];
    cfma(a, make_double2(-hq.x, -hq.y), V[(int64_t)q * ldv + i]);
  }
  w[i] = a;
}

static __global__ void k_scale_copy(const double2* w, double2* v, const double* nrm, int64_t N) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = 1.0 / *nrm;
  v[i] = cscale(w[i], s);
}

static __global__ void k_axpby(double2* y, const double2* x, double a, double b, int64_t N) {
  // y = a x + b y (real a, b)
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  y[i] = make_double2(a * x[i].x + b * y[i].x, a * x[i].y + b * y[i].y);
}

static __global__ void k_add_combo(double2* x, const double2* V, int64_t ldv, const double2* y, int k, int64_t N) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double2 a = x[i];
  for (int q = 0; q < k; ++q) cfma(a, y[q], V[(int64_t)q * ldv + i]);
  x[i] = a;
}

static __global__ void k_norm_partial(const double2* w, int64_t N, double* partial, int nb) {
  __shared__ double sh[GM_NB / 32];
  double acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * GM_NB + threadIdx.x; i < N; i += (int64_t)nb * GM_NB) acc += cabs2(w[i]);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int u = 0; u < GM_NB / 32; ++u) s += sh[u];
    partial[blockIdx.x] = s;
  }
}
static __global__ void k_norm_final(const double* partial, int nb, double* out) {
  __shared__ double sh[256];
  double s = 0;
  for (int u = threadIdx.x; u < nb; u += 256) s += partial[u];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(sh[0]);
}

struct GmCtx {
  fda_plan_s* P;
  bm_precond_s* pc = nullptr;  // flexible GMRES right preconditioner (optional)
  bm_net_s* net = nullptr;
  cudaStream_t s;
  int64_t N;
  int nb;
  DBuf<double2> partial, h, hacc;
  DBuf<double> npart, nrm;
  double ms_matvec = 0;
  int matvecs = 0;
};

static int dev_norm(GmCtx& C, const double2* w, double* host) {
  k_norm_partial<<<C.nb, GM_NB, 0, C.s>>>(w, C.N, C.npart.p, C.nb);
  k_norm_final<<<1, 256, 0, C.s>>>(C.npart.p, C.nb, C.nrm.p);
  FDA_LAUNCH_CHECK();
  if (host) {
    FDA_CUDA(cudaMemcpyAsync(host, C.nrm.p, sizeof(double), cudaMemcpyDeviceToHost, C.s));
    FDA_CUDA(cudaStreamSynchronize(C.s));
  }
  return FDA_OK;
}

static int apply_A(GmCtx& C, int prec, const double2* x, double2* y) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, C.s);
  int rc = plan_matvec(C.P, prec, x, y, 1, FDA_CPLX128, C.s, false);
  cudaEventRecord(b, C.s);
  cudaEventSynchronize(b);
  float t = 0;
  cudaEventElapsedTime(&t, a, b);
  C.ms_matvec += t;
  C.matvecs++;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

// GMRES(m) on one column: x (in/out), b. Returns FDA_OK when ||b - A x|| <= tol ||b|| (operator `prec`).
static int gmres_core(GmCtx& C, int prec, const double2* b, double2* x, double tol, int m, int maxit, int* iters,
                      double* relres, bool x0_zero) {
  const int64_t N = C.N;
  fda_plan_s* P = C.P;
  if (P->gm_V.n < (size_t)(m + 1) * N) FDA_TRY(P->gm_V.alloc((size_t)(m + 1) * N));
  if (P->gm_w.n < (size_t)N) FDA_TRY(P->gm_w.alloc(N));
  if (P->gm_r.n < (size_t)N) FDA_TRY(P->gm_r.alloc(N));
  const bool flex = C.pc != nullptr;
  if (flex && P->gm_x.n < (size_t)m * N) FDA_TRY(P->gm_x.alloc((size_t)m * N));
  double2* Z = flex ? P->gm_x.p : nullptr;  // z_j = M(v_j)
  double2* V = P->gm_V.p;
  double2* w = P->gm_w.p;
  double2* r = P->gm_r.p;
  double bn = 0;
  FDA_TRY(dev_norm(C, b, &bn));
  if (!std::isfinite(bn)) {
    set_error("right-hand side holds NaN or Inf");
    return FDA_E_NAN;
  }
  if (x0_zero) FDA_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * N, C.s));
  if (bn == 0) {
    FDA_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * N, C.s));
    *relres = 0;
    return FDA_OK;
  }
  int it = 0;
  double best = 1e300, prev_cycle = 1e300;
  std::vector<zc> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1);
  std::vector<double2> hh(m + 1), hy(m);
  while (true) {
    // r = b - A x
    if (x0_zero && it == 0) {
      FDA_CUDA(cudaMemcpyAsync(r, b, sizeof(double2) * N, cudaMemcpyDeviceToDevice, C.s));
    } else {
      FDA_TRY(apply_A(C, prec, x, r));
      k_axpby<<<cdiv(N, 256), 256, 0, C.s>>>(r, b, 1.0, -1.0, N);
      FDA_LAUNCH_CHECK();
    }
    double beta = 0;
    FDA_TRY(dev_norm(C, r, &beta));
    if (!std::isfinite(beta)) {
      set_error("GMRES residual became NaN or Inf");
      *relres = beta;
      return FDA_E_NAN;
    }
    *relres = beta / bn;
    if (beta / bn <= tol) {
      *iters = it;
      return FDA_OK;
    }
    if (it >= maxit) {
      *iters = it;
      set_error("GMRES reached %d iterations at relative residual %.3e", it, beta / bn);
      return FDA_E_NOT_CONVERGED;
    }
    if (!(beta < 0.999999 * prev_cycle)) {
      *iters = it;
      set_error("GMRES stagnated over a restart cycle (relative residual %.3e)", beta / bn);
      return FDA_E_BREAKDOWN;
    }
    prev_cycle = beta;
    FDA_CUDA(cudaMemcpyAsync(C.nrm.p, &beta, sizeof(double), cudaMemcpyHostToDevice, C.s));
    k_scale_copy<<<cdiv(N, 256), 256, 0, C.s>>>(r, V, C.nrm.p, N);
    FDA_LAUNCH_CHECK();
    std::fill(H.begin(), H.end(), zc(0));
    std::fill(g.begin(), g.end(), zc(0));
    g[0] = beta;
    int j = 0;
    for (; j < m && it < maxit; ++j) {
      if (flex) {
        FDA_TRY(precond_apply(C.pc, C.net, V + (int64_t)j * N, Z + (int64_t)j * N, C.s));
        FDA_TRY(apply_A(C, prec, Z + (int64_t)j * N, w));
      } else {
        FDA_TRY(apply_A(C, prec, V + (int64_t)j * N, w));
      }
      ++it;
      FDA_CUDA(cudaMemsetAsync(C.hacc.p, 0, sizeof(double2) * (j + 1), C.s));
      for (int pass = 0; pass < 2; ++pass) {
        k_multidot<<<dim3(C.nb, j + 1), GM_NB, 0, C.s>>>(V, N, j + 1, w, N, C.partial.p, C.nb);
        k_reduce_partials<<<j + 1, 256, 0, C.s>>>(C.partial.p, C.nb, j + 1, C.h.p, C.hacc.p);
        k_update<<<cdiv(N, 256), 256, 0, C.s>>>(V, N, j + 1, C.h.p, w, N);
        FDA_LAUNCH_CHECK();
      }
      double hn = 0;
      FDA_TRY(dev_norm(C, w, nullptr));
      FDA_CUDA(cudaMemcpyAsync(hh.data(), C.hacc.p, sizeof(double2) * (j + 1), cudaMemcpyDeviceToHost, C.s));
      FDA_CUDA(cudaMemcpyAsync(&hn, C.nrm.p, sizeof(double), cudaMemcpyDeviceToHost, C.s));
      FDA_CUDA(cudaStreamSynchronize(C.s));
      if (!std::isfinite(hn)) {
        set_error("Arnoldi vector became NaN or Inf");
        return FDA_E_NAN;
      }
      for (int q = 0; q <= j; ++q) H[q + (size_t)j * (m + 1)] = zc(hh[q].x, hh[q].y);
      H[j + 1 + (size_t)j * (m + 1)] = hn;
      if (hn > 0) {
        k_scale_copy<<<cdiv(N, 256), 256, 0, C.s>>>(w, V + (int64_t)(j + 1) * N, C.nrm.p, N);
        FDA_LAUNCH_CHECK();
      }
      // Givens: G = [[conj c, conj s], [-s, c]]
      for (int q = 0; q < j; ++q) {
        zc a = H[q + (size_t)j * (m + 1)], bb = H[q + 1 + (size_t)j * (m + 1)];
        H[q + (size_t)j * (m + 1)] = std::conj(cs[q]) * a + std::conj(sn[q]) * bb;
        H[q + 1 + (size_t)j * (m + 1)] = -sn[q] * a + cs[q] * bb;
      }
      zc a = H[j + (size_t)j * (m + 1)], bb = H[j + 1 + (size_t)j * (m + 1)];
      double den = std::sqrt(std::norm(a) + std::norm(bb));
      cs[j] = den > 0 ? a / den : zc(1);
      sn[j] = den > 0 ? bb / den : zc(0);
      H[j + (size_t)j * (m + 1)] = den;
      H[j + 1 + (size_t)j * (m + 1)] = 0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = std::conj(cs[j]) * g[j];
      double est = std::abs(g[j + 1]) / bn;
      best = std::min(best, est);
      if (est <= tol || hn == 0) {
        ++j;
        break;
      }
    }
    // y = H^-1 g (upper triangular j x j), x += V y
    int kk = j;
    std::vector<zc> y(kk);
    for (int q = kk - 1; q >= 0; --q) {
      zc sacc = g[q];
      for (int u = q + 1; u < kk; ++u) sacc -= H[q + (size_t)u * (m + 1)] * y[u];
      y[q] = sacc / H[q + (size_t)q * (m + 1)];
    }
    for (int q = 0; q < kk; ++q) hy[q] = make_double2(y[q].real(), y[q].imag());
    FDA_CUDA(cudaMemcpyAsync(C.h.p, hy.data(), sizeof(double2) * kk, cudaMemcpyHostToDevice, C.s));
    k_add_combo<<<cdiv(N, 256), 256, 0, C.s>>>(x, flex ? Z : V, N, C.h.p, kk, N);
    FDA_LAUNCH_CHECK();
    x0_zero = false;
  }
}

// ------------------------------------------------------------------ lockstep block form (nrhs > 1)
// Every column keeps its own Krylov space, Hessenberg matrix and Givens rotations; all columns advance
// together so that each step applies the operator once to the block [v_j^(0) .. v_j^(nc-1)] (N x nc,
// column-major, the layout fda_matvec takes). V is stored block by block: V[(j nc + c) N + i].
// partial[((c (q1) + q) nb + blk] = sum_i conj(V_q^(c)[i]) w^(c)[i]
static __global__ void k_multidot_blk(const double2* V, int nc, int q1, const double2* W, int64_t N, double2* partial,
                                      int nb) {
  __shared__ double2 sh[GM_NB / 32];
  const int q = blockIdx.y, c = blockIdx.z;
  const double2* v = V + ((int64_t)q * nc + c) * N;
  const double2* w = W + (int64_t)c * N;
  double2 acc = make_double2(0, 0);
  for (int64_t i = (int64_t)blockIdx.x * GM_NB + threadIdx.x; i < N; i += (int64_t)nb * GM_NB) cjfma(acc, v[i], w[i]);
  acc = warp_csum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 sum = make_double2(0, 0);
    for (int u = 0; u < GM_NB / 32; ++u) sum = cadd(sum, sh[u]);
    partial[((int64_t)c * q1 + q) * nb + blockIdx.x] = sum;
  }
}

// h[c q1 + q] = sum of partials, hacc += h
static __global__ void k_reduce_blk(const double2* partial, int nb, double2* h, double2* hacc) {
  const int64_t cq = blockIdx.x;
  __shared__ double2 sh[256];
  double2 sum = make_double2(0, 0);
  for (int u = threadIdx.x; u < nb; u += 256) sum = cadd(sum, partial[cq * nb + u]);
  sh[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    h[cq] = sh[0];
    hacc[cq] = cadd(hacc[cq], sh[0]);
  }
}

// w^(c) -= sum_q h[c q1 + q] V_q^(c)
static __global__ void k_update_blk(const double2* V, int nc, int q1, const double2* h, double2* W, int64_t N) {
  const int c = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double2 a = W[(int64_t)c * N + i];
  for (int q = 0; q < q1; ++q) {
    const double2 hq = h[(int64_t)c * q1 + q];
    cfma(a, make_double2(-hq.x, -hq.y), V[((int64_t)q * nc + c) * N + i]);
  }
  W[(int64_t)c * N + i] = a;
}

// out[c] = ||W^(c)||
static __global__ void k_norm_blk(const double2* W, int64_t N, double* out) {
  const int c = blockIdx.x;
  __shared__ double sh[1024 / 32];
  double acc = 0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) acc += cabs2(W[(int64_t)c * N + i]);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0;
    for (int u = 0; u < (int)(blockDim.x >> 5); ++u) sum += sh[u];
    out[c] = sqrt(sum);
  }
}

// dst^(c) = src^(c) * scale[c] (scale 0 for finished columns)
static __global__ void k_scale_blk(const double2* src, double2* dst, const double* scale, int64_t N) {
  const int c = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  dst[(int64_t)c * N + i] = cscale(src[(int64_t)c * N + i], scale[c]);
}

// x^(c) += sum_q y[c m + q] V_q^(c), q < k[c]
static __global__ void k_add_combo_blk(double2* X, const double2* V, int nc, const double2* y, int m, const int* kk,
                                       int64_t N) {
  const int c = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double2 a = X[(int64_t)c * N + i];
  for (int q = 0; q < kk[c]; ++q) cfma(a, y[(int64_t)c * m + q], V[((int64_t)q * nc + c) * N + i]);
  X[(int64_t)c * N + i] = a;
}

// r^(c) = b^(c) - r^(c)
static __global__ void k_resid_blk(double2* R, const double2* B, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  R[i] = make_double2(B[i].x - R[i].x, B[i].y - R[i].y);
}

struct BlkWork {
  DBuf<double2> V, W, R, partial, h, hacc, y;
  DBuf<double> nrm, scale;
  DBuf<int> kk;
};

static int blk_norms(GmCtx& C, const double2* W, int nc, BlkWork& B, std::vector<double>& out) {
  k_norm_blk<<<nc, 1024, 0, C.s>>>(W, C.N, B.nrm.p);
  FDA_LAUNCH_CHECK();
  out.resize(nc);
  FDA_CUDA(cudaMemcpyAsync(out.data(), B.nrm.p, sizeof(double) * nc, cudaMemcpyDeviceToHost, C.s));
  FDA_CUDA(cudaStreamSynchronize(C.s));
  return FDA_OK;
}

static int apply_A_blk(GmCtx& C, int prec, const double2* x, double2* y, int nc) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, C.s);
  int rc = plan_matvec(C.P, prec, x, y, nc, FDA_CPLX128, C.s, false);
  cudaEventRecord(b, C.s);
  cudaEventSynchronize(b);
  float t = 0;
  cudaEventElapsedTime(&t, a, b);
  C.ms_matvec += t;
  C.matvecs++;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

// Lockstep GMRES(m) on nc columns: X (in/out, N x nc), Bv (N x nc). Column c is finished when
// ||b - A x|| <= tol ||b|| (operator `prec`); iters counts block steps (one matvec on the block each).
static int gmres_block(GmCtx& C, int prec, const double2* Bv, double2* X, int nc, double tol, int m, int maxit,
                       int* iters, std::vector<double>& relres, bool x0_zero, BlkWork& B) {
  const int64_t N = C.N;
  const int64_t NB = N * nc;
  auto ensure = [](auto& buf, size_t count) { return buf.n < count ? buf.alloc(count) : (int)FDA_OK; };
  FDA_TRY(ensure(B.V, (size_t)(m + 1) * NB));
  FDA_TRY(ensure(B.W, (size_t)NB));
  FDA_TRY(ensure(B.R, (size_t)NB));
  FDA_TRY(ensure(B.partial, (size_t)C.nb * (m + 1) * nc));
  FDA_TRY(ensure(B.h, (size_t)(m + 1) * nc));
  FDA_TRY(ensure(B.hacc, (size_t)(m + 1) * nc));
  FDA_TRY(ensure(B.y, (size_t)m * nc));
  FDA_TRY(ensure(B.nrm, (size_t)nc));
  FDA_TRY(ensure(B.scale, (size_t)nc));
  FDA_TRY(ensure(B.kk, (size_t)nc));
  std::vector<double> bn, beta(nc), hn;
  FDA_TRY(blk_norms(C, Bv, nc, B, bn));
  relres.assign(nc, 0.0);
  for (int c = 0; c < nc; ++c)
    if (!std::isfinite(bn[c])) {
      set_error("right-hand side %d holds NaN or Inf", c);
      return FDA_E_NAN;
    }
  if (x0_zero) FDA_CUDA(cudaMemsetAsync(X, 0, sizeof(double2) * NB, C.s));
  const size_t ldh = (size_t)m + 1;
  std::vector<zc> H((size_t)nc * ldh * m), cs((size_t)nc * m), sn((size_t)nc * m), g((size_t)nc * ldh);
  std::vector<double2> hh((size_t)nc * (m + 1)), hy((size_t)nc * m);
  std::vector<int> kk(nc), live(nc);
  std::vector<double> prev_cycle(nc, 1e300), sc(nc);
  int it = 0;
  while (true) {
    // R = B - A X
    if (x0_zero && it == 0) {
      FDA_CUDA(cudaMemcpyAsync(B.R.p, Bv, sizeof(double2) * NB, cudaMemcpyDeviceToDevice, C.s));
    } else {
      FDA_TRY(apply_A_blk(C, prec, X, B.R.p, nc));
      k_resid_blk<<<cdiv(NB, 256), 256, 0, C.s>>>(B.R.p, Bv, NB);
      FDA_LAUNCH_CHECK();
    }
    FDA_TRY(blk_norms(C, B.R.p, nc, B, beta));
    int nlive = 0;
    bool stagnated = false;
    for (int c = 0; c < nc; ++c) {
      if (!std::isfinite(beta[c])) {
        set_error("GMRES residual of column %d became NaN or Inf", c);
        return FDA_E_NAN;
      }
      relres[c] = bn[c] > 0 ? beta[c] / bn[c] : 0.0;
      live[c] = bn[c] > 0 && relres[c] > tol;
      if (live[c] && !(beta[c] < 0.999999 * prev_cycle[c])) stagnated = true;
      prev_cycle[c] = beta[c];
      nlive += live[c];
      sc[c] = live[c] ? 1.0 / beta[c] : 0.0;
    }
    if (nlive == 0) {
      *iters = it;
      return FDA_OK;
    }
    if (it >= maxit) {
      *iters = it;
      set_error("block GMRES reached %d steps with %d columns above tolerance", it, nlive);
      return FDA_E_NOT_CONVERGED;
    }
    if (stagnated) {
      *iters = it;
      set_error("block GMRES stagnated over a restart cycle");
      return FDA_E_BREAKDOWN;
    }
    FDA_CUDA(cudaMemcpyAsync(B.scale.p, sc.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, C.s));
    k_scale_blk<<<dim3(cdiv(N, 256), nc), 256, 0, C.s>>>(B.R.p, B.V.p, B.scale.p, N);
    FDA_LAUNCH_CHECK();
    std::fill(H.begin(), H.end(), zc(0));
    std::fill(g.begin(), g.end(), zc(0));
    for (int c = 0; c < nc; ++c) {
      g[(size_t)c * ldh] = live[c] ? beta[c] : 0.0;
      kk[c] = 0;
    }
    std::vector<int> act = live;  // columns still iterating in this cycle
    int j = 0;
    for (; j < m && it < maxit; ++j) {
      FDA_TRY(apply_A_blk(C, prec, B.V.p + (int64_t)j * NB, B.W.p, nc));
      ++it;
      FDA_CUDA(cudaMemsetAsync(B.hacc.p, 0, sizeof(double2) * (j + 1) * nc, C.s));
      for (int pass = 0; pass < 2; ++pass) {
        k_multidot_blk<<<dim3(C.nb, j + 1, nc), GM_NB, 0, C.s>>>(B.V.p, nc, j + 1, B.W.p, N, B.partial.p, C.nb);
        k_reduce_blk<<<(j + 1) * nc, 256, 0, C.s>>>(B.partial.p, C.nb, B.h.p, B.hacc.p);
        k_update_blk<<<dim3(cdiv(N, 256), nc), 256, 0, C.s>>>(B.V.p, nc, j + 1, B.h.p, B.W.p, N);
        FDA_LAUNCH_CHECK();
      }
      FDA_CUDA(cudaMemcpyAsync(hh.data(), B.hacc.p, sizeof(double2) * (j + 1) * nc, cudaMemcpyDeviceToHost, C.s));
      FDA_TRY(blk_norms(C, B.W.p, nc, B, hn));
      int nact = 0;
      for (int c = 0; c < nc; ++c) {
        if (!act[c]) {
          sc[c] = 0.0;
          continue;
        }
        if (!std::isfinite(hn[c])) {
          set_error("Arnoldi vector of column %d became NaN or Inf", c);
          return FDA_E_NAN;
        }
        zc* Hc = &H[(size_t)c * ldh * m];
        zc* csc = &cs[(size_t)c * m];
        zc* snc = &sn[(size_t)c * m];
        zc* gc = &g[(size_t)c * ldh];
        for (int q = 0; q <= j; ++q) Hc[q + (size_t)j * ldh] = zc(hh[(size_t)c * (j + 1) + q].x, hh[(size_t)c * (j + 1) + q].y);
        Hc[j + 1 + (size_t)j * ldh] = hn[c];
        for (int q = 0; q < j; ++q) {
          zc a = Hc[q + (size_t)j * ldh], bb = Hc[q + 1 + (size_t)j * ldh];
          Hc[q + (size_t)j * ldh] = std::conj(csc[q]) * a + std::conj(snc[q]) * bb;
          Hc[q + 1 + (size_t)j * ldh] = -snc[q] * a + csc[q] * bb;
        }
        zc a = Hc[j + (size_t)j * ldh], bb = Hc[j + 1 + (size_t)j * ldh];
        double den = std::sqrt(std::norm(a) + std::norm(bb));
        csc[j] = den > 0 ? a / den : zc(1);
        snc[j] = den > 0 ? bb / den : zc(0);
        Hc[j + (size_t)j * ldh] = den;
        Hc[j + 1 + (size_t)j * ldh] = 0;
        gc[j + 1] = -snc[j] * gc[j];
        gc[j] = std::conj(csc[j]) * gc[j];
        kk[c] = j + 1;
        const double est = std::abs(gc[j + 1]) / bn[c];
        if (est <= tol || hn[c] == 0) {
          act[c] = 0;  // finished in this cycle: its Krylov basis stops here
          sc[c] = 0.0;
        } else {
          sc[c] = 1.0 / hn[c];
          ++nact;
        }
      }
      if (nact == 0) {
        ++j;
        break;
      }
      FDA_CUDA(cudaMemcpyAsync(B.scale.p, sc.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, C.s));
      k_scale_blk<<<dim3(cdiv(N, 256), nc), 256, 0, C.s>>>(B.W.p, B.V.p + (int64_t)(j + 1) * NB, B.scale.p, N);
      FDA_LAUNCH_CHECK();
    }
    // y = H^-1 g per column, X += V y
    for (int c = 0; c < nc; ++c) {
      const zc* Hc = &H[(size_t)c * ldh * m];
      const zc* gc = &g[(size_t)c * ldh];
      std::vector<zc> y(kk[c]);
      for (int q = kk[c] - 1; q >= 0; --q) {
        zc sacc = gc[q];
        for (int u = q + 1; u < kk[c]; ++u) sacc -= Hc[q + (size_t)u * ldh] * y[u];
        y[q] = sacc / Hc[q + (size_t)q * ldh];
      }
      for (int q = 0; q < m; ++q)
        hy[(size_t)c * m + q] = q < kk[c] ? make_double2(y[q].real(), y[q].imag()) : make_double2(0, 0);
    }
    FDA_CUDA(cudaMemcpyAsync(B.y.p, hy.data(), sizeof(double2) * m * nc, cudaMemcpyHostToDevice, C.s));
    FDA_CUDA(cudaMemcpyAsync(B.kk.p, kk.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, C.s));
    k_add_combo_blk<<<dim3(cdiv(N, 256), nc), 256, 0, C.s>>>(X, B.V.p, nc, B.y.p, m, B.kk.p, N);
    FDA_LAUNCH_CHECK();
    x0_zero = false;
  }
}

// Block solve of nc columns: plain lockstep GMRES, or FP64 refinement around the lockstep FP32 solve.
static int gmres_solve_block(GmCtx& C, const double2* b, double2* x, int nc, const bm_gmres_opts_t* o, int m, int mi,
                             int* total_it, int* outer, double* worst) {
  fda_plan_s* P = C.P;
  BlkWork B;
  std::vector<double> rel;
  int it = 0;
  // refinement: outer residual with the FP64 operator or the 3xTF32 FP32 product; the inner solve needs only a
  // few digits and runs single-pass TF32 translations (on plans without 3xTF32 images the plain FP32 product)
  int oprec = o->refine_residual ? FDA_PREC_FP32 : FDA_PREC_FP64;  // refine_residual = 2 ends on FP64
  const int iprec = FDA_PREC_TF32;
  if (!o->refine) {
    const int aprec = P->cfg.drop_fp64 ? FDA_PREC_FP32 : FDA_PREC_FP64;  // FP32-only plans: FP32 operator
    int rc = gmres_block(C, aprec, b, x, nc, o->tol, m, o->max_iter, &it, rel, !o->x0_given, B);
    *total_it += it;
    for (double r : rel) *worst = std::max(*worst, r);
    return rc;
  }
  if (P->cfg.precision != FDA_PREC_FP32) {
    set_error("refine = 1 needs a plan built with FDA_PREC_FP32");
    return FDA_E_STATE;
  }
  const int64_t NB = C.N * nc;
  DBuf<double2> Rb, Z;
  FDA_TRY(Rb.alloc(NB));
  FDA_TRY(Z.alloc(NB));
  std::vector<double> bn, rn;
  FDA_TRY(B.nrm.alloc(nc));
  FDA_TRY(blk_norms(C, b, nc, B, bn));
  if (!o->x0_given) FDA_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * NB, C.s));
  double prev = 1e300;
  int rc = FDA_E_NOT_CONVERGED;
  std::vector<double> sc(nc);
  for (int k = 0; k < 50; ++k) {
    if (k == 0 && !o->x0_given) {
      FDA_CUDA(cudaMemcpyAsync(Rb.p, b, sizeof(double2) * NB, cudaMemcpyDeviceToDevice, C.s));
    } else {
      FDA_TRY(apply_A_blk(C, oprec, x, Rb.p, nc));
      k_resid_blk<<<cdiv(NB, 256), 256, 0, C.s>>>(Rb.p, b, NB);
      FDA_LAUNCH_CHECK();
    }
    FDA_TRY(blk_norms(C, Rb.p, nc, B, rn));
    double wr = 0, worst_abs = 0;
    for (int c = 0; c < nc; ++c) {
      if (!std::isfinite(rn[c])) {
        set_error("refinement residual of column %d holds NaN or Inf", c);
        return FDA_E_NAN;
      }
      const double r = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
      wr = std::max(wr, r);
      worst_abs = std::max(worst_abs, r);
      sc[c] = r <= o->tol ? 0.0 : 1.0;  // finished columns get a zero inner right-hand side
    }
    *worst = wr;
    if (wr <= o->tol) {
      if (o->refine_residual == 2 && oprec != FDA_PREC_FP64) {  // confirm with the FP64 residual
        oprec = FDA_PREC_FP64;
        prev = 1e300;
        continue;
      }
      rc = FDA_OK;
      break;
    }
    if (*total_it >= o->max_iter) {
      set_error("iterative refinement reached %d iterations at relative residual %.3e", *total_it, wr);
      break;
    }
    if (!(worst_abs < 0.9 * prev)) {
      set_error("iterative refinement stagnated at %.3e", wr);
      rc = FDA_E_BREAKDOWN;
      break;
    }
    prev = worst_abs;
    ++*outer;
    {
      DBuf<double> dsc;
      FDA_TRY(dsc.upload(sc));
      k_scale_blk<<<dim3(cdiv(C.N, 256), nc), 256, 0, C.s>>>(Rb.p, Rb.p, dsc.p, C.N);
      FDA_LAUNCH_CHECK();
      FDA_CUDA(cudaStreamSynchronize(C.s));
    }
    const double itol = o->inner_tol > 0 ? o->inner_tol : 1e-4;
    int iit = 0;
    int irc = gmres_block(C, iprec, Rb.p, Z.p, nc, std::max(itol, o->tol / std::max(wr, 1e-300)), mi,
                          o->max_iter - *total_it, &iit, rel, true, B);
    *total_it += iit;
    if (irc != FDA_OK && irc != FDA_E_NOT_CONVERGED && irc != FDA_E_BREAKDOWN) {
      rc = irc;
      break;
    }
    k_axpby<<<cdiv(NB, 256), 256, 0, C.s>>>(x, Z.p, 1.0, 1.0, NB);
    FDA_LAUNCH_CHECK();
  }
  return rc;
}

int gmres_solve(fda_plan_s* P, const double2* b, double2* x, int nrhs, const bm_gmres_opts_t* o,
                bm_gmres_stats_t* st, cudaStream_t s, bm_precond_s* pc, bm_net_s* net) {
  auto t0 = std::chrono::steady_clock::now();
  GmCtx C;
  C.P = P;
  C.pc = pc;
  C.net = net;
  C.s = s;
  C.N = P->tree->N;
  C.nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (C.N + GM_NB - 1) / GM_NB));
  int m = std::max(1, std::min(512, o->restart));
  int mi = std::max(1, std::min(512, o->inner_restart > 0 ? o->inner_restart : o->restart));
  if (o->refine_residual < 0 || o->refine_residual > 2) {
    set_error("refine_residual must be 0, 1 or 2");
    return FDA_E_INVALID_ARG;
  }
  if (o->refine && o->refine_residual && (P->cfg.precision != FDA_PREC_FP32 || P->cfg.m2l_tensor != 3)) {
    set_error("refine_residual = 1 or 2 needs a plan built with FDA_PREC_FP32 and m2l_tensor = 3 (3xTF32 images)");
    return FDA_E_STATE;
  }
  if (P->cfg.drop_fp64 && o->refine && o->refine_residual != 1) {
    set_error("the plan released its FP64 operators (drop_fp64): solve with refine = 0, or refine_residual = 1");
    return FDA_E_STATE;
  }
  const int oprec0 = o->refine_residual ? FDA_PREC_FP32 : FDA_PREC_FP64;
  const int iprec = FDA_PREC_TF32;  // see gmres_solve_block
  FDA_TRY(C.partial.alloc((size_t)C.nb * (std::max(m, mi) + 1)));
  FDA_TRY(C.h.alloc(std::max(m, mi) + 1));
  FDA_TRY(C.hacc.alloc(std::max(m, mi) + 1));
  FDA_TRY(C.npart.alloc(C.nb));
  FDA_TRY(C.nrm.alloc(1));
  int total_it = 0, outer = 0, rc = FDA_OK;
  double worst = 0;
  if (nrhs > 1 && !pc) {
    rc = gmres_solve_block(C, b, x, nrhs, o, m, mi, &total_it, &outer, &worst);
    FDA_CUDA(cudaStreamSynchronize(s));
    if (st) {
      st->iterations = total_it;
      st->outer_iterations = outer;
      st->rel_residual = worst;
      st->ms_matvec = C.ms_matvec;
      st->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      st->status = rc;
    }
    return rc;
  }
  for (int c = 0; c < nrhs; ++c) {
    const double2* bc = b + (int64_t)c * C.N;
    double2* xc = x + (int64_t)c * C.N;
    double rel = 0;
    int it = 0;
    if (!o->refine) {
      rc = gmres_core(C, P->cfg.drop_fp64 ? FDA_PREC_FP32 : FDA_PREC_FP64, bc, xc, o->tol, m, o->max_iter, &it,
                      &rel, !o->x0_given);
      total_it += it;
    } else {
      if (P->cfg.precision != FDA_PREC_FP32) {
        set_error("refine = 1 needs a plan built with FDA_PREC_FP32");
        return FDA_E_STATE;
      }
      if (P->gm_z.n < (size_t)C.N) FDA_TRY(P->gm_z.alloc(C.N));
      if (P->gm_b.n < (size_t)C.N) FDA_TRY(P->gm_b.alloc(C.N));
      double bn = 0;
      FDA_TRY(dev_norm(C, bc, &bn));
      if (!o->x0_given) FDA_CUDA(cudaMemsetAsync(xc, 0, sizeof(double2) * C.N, s));
      double prev = 1e300;
      int oprec = oprec0;  // refine_residual = 2 switches to FP64 for the final check
      rc = FDA_E_NOT_CONVERGED;
      for (int k = 0; k < 50; ++k) {
        // outer residual with the FP64 operator (or the 3xTF32 FP32 product)
        if (k == 0 && !o->x0_given) {
          FDA_CUDA(cudaMemcpyAsync(P->gm_b.p, bc, sizeof(double2) * C.N, cudaMemcpyDeviceToDevice, s));
        } else {
          FDA_TRY(apply_A(C, oprec, xc, P->gm_b.p));
          k_axpby<<<cdiv(C.N, 256), 256, 0, s>>>(P->gm_b.p, bc, 1.0, -1.0, C.N);
          FDA_LAUNCH_CHECK();
        }
        double rn = 0;
        FDA_TRY(dev_norm(C, P->gm_b.p, &rn));
        rel = rn / bn;
        if (!std::isfinite(rn)) {
          set_error("refinement residual holds NaN or Inf (right-hand side or operator)");
          rc = FDA_E_NAN;
          break;
        }
        if (rel <= o->tol) {
          if (o->refine_residual == 2 && oprec != FDA_PREC_FP64) {  // confirm with the FP64 residual
            oprec = FDA_PREC_FP64;
            prev = 1e300;
            continue;
          }
          rc = FDA_OK;
          break;
        }
        if (total_it >= o->max_iter) {
          set_error("iterative refinement reached %d iterations at relative residual %.3e", total_it, rel);
          break;
        }
        if (!(rn < 0.9 * prev)) {
          set_error("iterative refinement stagnated at %.3e", rel);
          rc = FDA_E_BREAKDOWN;
          break;
        }
        prev = rn;
        ++outer;
        double itol = o->inner_tol > 0 ? o->inner_tol : 1e-4;
        int iit = 0;
        double irel = 0;
        int irc = gmres_core(C, iprec, P->gm_b.p, P->gm_z.p, std::max(itol, o->tol / std::max(rel, 1e-300)),
                             mi, o->max_iter - total_it, &iit, &irel, true);
        total_it += iit;
        if (irc != FDA_OK && irc != FDA_E_NOT_CONVERGED && irc != FDA_E_BREAKDOWN) {
          rc = irc;
          break;
        }
        k_axpby<<<cdiv(C.N, 256), 256, 0, s>>>(xc, P->gm_z.p, 1.0, 1.0, C.N);
        FDA_LAUNCH_CHECK();
      }
    }
    worst = std::max(worst, rel);
    if (rc != FDA_OK) break;
  }
  FDA_CUDA(cudaStreamSynchronize(s));
  if (rc == FDA_OK && P->tc_err.p) {  // a bounded device wait that gave up invalidates the solve
    int flag = 0;
    FDA_CUDA(cudaMemcpy(&flag, P->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
      set_error("a bounded device wait gave up during the solve");
      rc = FDA_E_TIMEOUT;
    }
  }
  if (st) {
    st->iterations = total_it;
    st->outer_iterations = outer;
    st->rel_residual = worst;
    st->ms_matvec = C.ms_matvec;
    st->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    st->status = rc;
  }
  return rc;
}

}  // namespace fda
