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
  FDA_TRY(C.partial.alloc((size_t)C.nb * (std::max(m, mi) + 1)));
  FDA_TRY(C.h.alloc(std::max(m, mi) + 1));
  FDA_TRY(C.hacc.alloc(std::max(m, mi) + 1));
  FDA_TRY(C.npart.alloc(C.nb));
  FDA_TRY(C.nrm.alloc(1));
  int total_it = 0, outer = 0, rc = FDA_OK;
  double worst = 0;
  for (int c = 0; c < nrhs; ++c) {
    const double2* bc = b + (int64_t)c * C.N;
    double2* xc = x + (int64_t)c * C.N;
    double rel = 0;
    int it = 0;
    if (!o->refine) {
      rc = gmres_core(C, FDA_PREC_FP64, bc, xc, o->tol, m, o->max_iter, &it, &rel, !o->x0_given);
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
      rc = FDA_E_NOT_CONVERGED;
      for (int k = 0; k < 50; ++k) {
        // outer residual with the FP64 operator
        if (k == 0 && !o->x0_given) {
          FDA_CUDA(cudaMemcpyAsync(P->gm_b.p, bc, sizeof(double2) * C.N, cudaMemcpyDeviceToDevice, s));
        } else {
          FDA_TRY(apply_A(C, FDA_PREC_FP64, xc, P->gm_b.p));
          k_axpby<<<cdiv(C.N, 256), 256, 0, s>>>(P->gm_b.p, bc, 1.0, -1.0, C.N);
          FDA_LAUNCH_CHECK();
        }
        double rn = 0;
        FDA_TRY(dev_norm(C, P->gm_b.p, &rn));
        rel = rn / bn;
        if (!std::isfinite(rn)) {
          rc = FDA_E_NAN;
          break;
        }
        if (rel <= o->tol) {
          rc = FDA_OK;
          break;
        }
        if (total_it >= o->max_iter) break;
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
        int irc = gmres_core(C, FDA_PREC_FP32, P->gm_b.p, P->gm_z.p, std::max(itol, o->tol / std::max(rel, 1e-300)),
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
