// Dense FP64 complex linear algebra for the translation precompute (Sec. 4.1, 4.2):
//   - batched GEMM C = alpha op(A) op(B) + beta C (column-major, op in {N, T, C});
//   - column-pivoted Householder QR with rank truncation at |R_kk| < tol |R_00| (one CTA per matrix):
//     selects equivalent/check points and gives low-rank factors K~ = U^ V^ ;
//   - one-sided Jacobi SVD (one CTA per matrix), for R = U Sigma V^H of Eq. svdr.
#include "internal.cuh"

namespace fda {

// ------------------------------------------------------------------ batched ZGEMM
template <int OPA, int OPB>
static __global__ void k_zgemm_batched(int M, int N, int K, double2 alpha, const double2* const* Ap, int lda,
                                       const double2* const* Bp, int ldb, double2 beta, double2* const* Cp,
                                       int ldc) {
  __shared__ double2 As[16][33];
  __shared__ double2 Bs[16][33];
  const double2* A = Ap[blockIdx.z];
  const double2* B = Bp[blockIdx.z];
  double2* C = Cp[blockIdx.z];
  int t = threadIdx.x, tx = t & 31, ty = t >> 5;
  int m0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  double2 acc[4];
  for (int j = 0; j < 4; ++j) acc[j] = make_double2(0, 0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int q = t; q < 512; q += 256) {
      int mm = q & 31, kk = q >> 5;
      int gm = m0 + mm, gk = k0 + kk;
      double2 v = make_double2(0, 0);
      if (gm < M && gk < K) {
        if (OPA == 0)
          v = A[gm + (int64_t)gk * lda];
        else {
          v = A[gk + (int64_t)gm * lda];
          if (OPA == 2) v.y = -v.y;
        }
      }
      As[kk][mm] = v;
      int nn = q & 31;
      int gn = n0 + nn;
      double2 w = make_double2(0, 0);
      if (gn < N && gk < K) {
        if (OPB == 0)
          w = B[gk + (int64_t)gn * ldb];
        else {
          w = B[gn + (int64_t)gk * ldb];
          if (OPB == 2) w.y = -w.y;
        }
      }
      Bs[kk][nn] = w;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      double2 a = As[kk][tx];
      for (int j = 0; j < 4; ++j) cfma(acc[j], a, Bs[kk][ty + 8 * j]);
    }
    __syncthreads();
  }
  int gm = m0 + tx;
  if (gm >= M) return;
  for (int j = 0; j < 4; ++j) {
    int gn = n0 + ty + 8 * j;
    if (gn >= N) continue;
    double2* c = C + gm + (int64_t)gn * ldc;
    double2 r = cmul(alpha, acc[j]);
    if (beta.x != 0 || beta.y != 0) r = cadd(r, cmul(beta, *c));
    *c = r;
  }
}

int zgemm_batched(char opa, char opb, int M, int N, int K, double2 alpha, const double2* const* A, int lda,
                  const double2* const* B, int ldb, double2 beta, double2* const* C, int ldc, int64_t batch,
                  cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return FDA_OK;
  int oa = opa == 'N' ? 0 : (opa == 'T' ? 1 : 2);
  int ob = opb == 'N' ? 0 : (opb == 'T' ? 1 : 2);
  for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
    int64_t nb = std::min<int64_t>(65535, batch - b0);
    dim3 g(cdiv(M, 32), cdiv(N, 32), (unsigned)nb);
#define ZG(a, b) \
  if (oa == a && ob == b) k_zgemm_batched<a, b><<<g, 256, 0, s>>>(M, N, K, alpha, A + b0, lda, B + b0, ldb, beta, C + b0, ldc)
    ZG(0, 0);
    ZG(0, 1);
    ZG(0, 2);
    ZG(1, 0);
    ZG(1, 1);
    ZG(1, 2);
    ZG(2, 0);
    ZG(2, 1);
    ZG(2, 2);
#undef ZG
    FDA_LAUNCH_CHECK();
  }
  return FDA_OK;
}

// ------------------------------------------------------------------ block reductions
template <int NT>
__device__ __forceinline__ void block_argmax(double v, int idx, double* sv, int* si, double& outv, int& outi) {
  int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    double v2 = __shfl_down_sync(0xffffffffu, v, o);
    int i2 = __shfl_down_sync(0xffffffffu, idx, o);
    if (v2 > v || (v2 == v && i2 < idx)) v = v2, idx = i2;
  }
  if (lane == 0) sv[w] = v, si[w] = idx;
  __syncthreads();
  if (t == 0) {
    double bv = sv[0];
    int bi = si[0];
    for (int q = 1; q < NT / 32; ++q)
      if (sv[q] > bv || (sv[q] == bv && si[q] < bi)) bv = sv[q], bi = si[q];
    sv[0] = bv;
    si[0] = bi;
  }
  __syncthreads();
  outv = sv[0];
  outi = si[0];
  __syncthreads();
}

// ------------------------------------------------------------------ pivoted QR
// A (m x n, lda) is overwritten by the Householder vectors (column k holds v_k in rows k..m-1) and the
// strictly upper part of R. rdiag/tau (kmax) hold R_kk and the reflector scales, perm (n) the column order.
// Stops at the first k with max trailing column norm < tol * |R_00| (or k = min(m, n, kmax)).
struct QRJob {
  double2* A;
  int m, n, lda, kmax;
  double tol;
  int* perm;
  int* rank;
  double2* rdiag;
  double2* tau;
  double* cn;  // n scratch
};

#define QR_NT 512
static __global__ void __launch_bounds__(QR_NT) k_pivqr(const QRJob* jobs) {
  const QRJob J = jobs[blockIdx.x];
  __shared__ double sv[QR_NT / 32];
  __shared__ int si[QR_NT / 32];
  __shared__ double2 s_alpha, s_tau;
  __shared__ int s_stop;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = QR_NT / 32;
  const int m = J.m, n = J.n, kmax = min(J.kmax, min(m, n));
  double2* A = J.A;
  for (int j = t; j < n; j += QR_NT) {
    J.perm[j] = j;
    double s = 0;
    for (int i = 0; i < m; ++i) s += cabs2(A[i + (int64_t)j * J.lda]);
    J.cn[j] = s;
  }
  __syncthreads();
  double r00 = 0;
  int k = 0;
  for (; k < kmax; ++k) {
    double bv = -1;
    int bi = k;
    for (int j = k + t; j < n; j += QR_NT)
      if (J.cn[j] > bv) bv = J.cn[j], bi = j;
    double mv;
    int mi;
    block_argmax<QR_NT>(bv, bi, sv, si, mv, mi);
    double nrm = sqrt(fmax(mv, 0.0));
    if (k == 0) r00 = nrm;
    if (nrm == 0.0 || (k > 0 && nrm < J.tol * r00)) break;
    // swap columns k and mi
    if (mi != k) {
      for (int i = t; i < m; i += QR_NT) {
        double2 a = A[i + (int64_t)k * J.lda];
        A[i + (int64_t)k * J.lda] = A[i + (int64_t)mi * J.lda];
        A[i + (int64_t)mi * J.lda] = a;
      }
      __syncthreads();
      if (t == 0) {
        double c = J.cn[k];
        J.cn[k] = J.cn[mi];
        J.cn[mi] = c;
        int p = J.perm[k];
        J.perm[k] = J.perm[mi];
        J.perm[mi] = p;
      }
    }
    __syncthreads();
    // Householder: x = A[k:, k]; alpha = -phase(x0) ||x||; v = x - alpha e1; tau = 1 / (||x|| (||x|| + |x0|))
    if (t == 0) {
      double2 x0 = A[k + (int64_t)k * J.lda];
      double ax0 = sqrt(cabs2(x0));
      double2 ph = ax0 > 0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1, 0);
      double2 al = make_double2(-ph.x * nrm, -ph.y * nrm);
      s_alpha = al;
      A[k + (int64_t)k * J.lda] = csub(x0, al);
      s_tau = make_double2(1.0 / (nrm * (nrm + ax0)), 0);
      J.rdiag[k] = al;
      J.tau[k] = s_tau;
    }
    __syncthreads();
    const double tau = s_tau.x;
    const double2* v = A + (int64_t)k * J.lda;
    // apply (I - tau v v^H) to columns j > k, one warp per column; refresh trailing norms
    for (int j = k + 1 + w; j < n; j += nw) {
      double2* a = A + (int64_t)j * J.lda;
      double2 s = make_double2(0, 0);
      for (int i = k + lane; i < m; i += 32) cjfma(s, v[i], a[i]);
      s = warp_csum(s);
      s = cscale(s, tau);
      double nn = 0;
      for (int i = k + lane; i < m; i += 32) {
        double2 ai = a[i];
        cfma(ai, make_double2(-s.x, -s.y), v[i]);
        a[i] = ai;
        if (i > k) nn += cabs2(ai);
      }
      nn = warp_sum(nn);
      if (lane == 0) J.cn[j] = nn;
    }
    __syncthreads();
  }
  if (t == 0) *J.rank = k;
}

int pivoted_qr_batched(const std::vector<QRJob>& jobs, cudaStream_t s) {
  if (jobs.empty()) return FDA_OK;
  DBuf<QRJob> dj;
  FDA_TRY(dj.upload(jobs));
  for (size_t b0 = 0; b0 < jobs.size(); b0 += 65535) {
    size_t nb = std::min<size_t>(65535, jobs.size() - b0);
    k_pivqr<<<(unsigned)nb, QR_NT, 0, s>>>(dj.p + b0);
    FDA_LAUNCH_CHECK();
  }
  FDA_CUDA(cudaStreamSynchronize(s));
  return FDA_OK;
}

// Q_r = H_0 ... H_{r-1} [I_r; 0] (m x r, ldq) from the reflectors left in A by k_pivqr.
struct QFormJob {
  const double2* A;
  int m, lda, r;
  const double2* tau;
  double2* Q;
  int ldq;
};
static __global__ void __launch_bounds__(QR_NT) k_form_q(const QFormJob* jobs) {
  const QFormJob J = jobs[blockIdx.x];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = QR_NT / 32;
  for (int c = 0; c < J.r; ++c)
    for (int i = t; i < J.m; i += QR_NT) J.Q[i + (int64_t)c * J.ldq] = make_double2(i == c ? 1.0 : 0.0, 0);
  __syncthreads();
  for (int k = J.r - 1; k >= 0; --k) {
    const double2* v = J.A + (int64_t)k * J.lda;
    double tau = J.tau[k].x;
    for (int c = w; c < J.r; c += nw) {
      double2* q = J.Q + (int64_t)c * J.ldq;
      double2 s = make_double2(0, 0);
      for (int i = k + lane; i < J.m; i += 32) cjfma(s, v[i], q[i]);
      s = cscale(warp_csum(s), tau);
      for (int i = k + lane; i < J.m; i += 32) cfma(q[i], make_double2(-s.x, -s.y), v[i]);
    }
    __syncthreads();
  }
}

int form_q_batched(const std::vector<QFormJob>& jobs, cudaStream_t s) {
  if (jobs.empty()) return FDA_OK;
  DBuf<QFormJob> dj;
  FDA_TRY(dj.upload(jobs));
  for (size_t b0 = 0; b0 < jobs.size(); b0 += 65535) {
    size_t nb = std::min<size_t>(65535, jobs.size() - b0);
    k_form_q<<<(unsigned)nb, QR_NT, 0, s>>>(dj.p + b0);
    FDA_LAUNCH_CHECK();
  }
  FDA_CUDA(cudaStreamSynchronize(s));
  return FDA_OK;
}

// ------------------------------------------------------------------ Gaussian sketch matrices
// Entry q of a sketch is a standard normal variate (imaginary part 0) from a counter-based generator: two
// SplitMix64 outputs (Steele, Lea and Flood, 2014) of the counter 2q and 2q + 1 offset by the seed, mapped
// to (0, 1) and through the Box-Muller transform.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static __global__ void k_gaussian(double2* out, int64_t n, uint64_t seed) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(2 * q));
    const uint64_t b = splitmix64(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(2 * q + 1));
    const double u1 = ((double)(a >> 11) + 0.5) * 0x1.0p-53, u2 = ((double)(b >> 11) + 0.5) * 0x1.0p-53;
    out[q] = make_double2(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2), 0.0);
  }
}
int gaussian_fill(double2* out, int64_t n, uint64_t seed) {
  if (n <= 0) return FDA_OK;
  k_gaussian<<<(unsigned)std::min<int64_t>(4096, (n + 255) / 256), 256>>>(out, n, seed);
  FDA_LAUNCH_CHECK();
  return FDA_OK;
}

// ------------------------------------------------------------------ one-sided Jacobi SVD
// A (m x n) -> columns become U_j sigma_j; V (n x n) accumulates the rotations. After the sweeps the
// singular values are the column norms (sorted on the host).
struct SVDJob {
  double2* A;
  int m, n, lda;
  double2* V;
  int ldv;
  int* sweeps;
};

// Rounds of the round-robin pairing run as separate launches, one warp per column pair across many CTAs, all
// matrices of the batch in one launch (blockIdx.y): the rounds of a sweep are ordered by the stream, and every
// pair of a round is independent. A matrix whose last sweep rotated nothing is finished and skipped; the host
// reads the per-matrix rotation flags once per sweep (at most 40 sweeps).
static __global__ void k_jacobi_init(const SVDJob* jobs) {
  const SVDJob J = jobs[blockIdx.y];
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)J.n * J.n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % J.n), c = (int)(q / J.n);
    J.V[i + (int64_t)c * J.ldv] = make_double2(i == c ? 1.0 : 0.0, 0);
  }
}

#define JR_WARPS 8
static __global__ void __launch_bounds__(32 * JR_WARPS) k_jacobi_round(const SVDJob* jobs, int r, const int* active,
                                                                        int* rotated) {
  const int j = blockIdx.y;
  if (!active[j]) return;
  const SVDJob J = jobs[j];
  const int lane = threadIdx.x & 31, pr = blockIdx.x * JR_WARPS + (threadIdx.x >> 5);
  const int m = J.m, n = J.n, np = n + (n & 1);
  if (r >= np - 1 || pr >= np / 2) return;
  int p = (pr == 0) ? 0 : 1 + (r + pr - 1) % (np - 1);
  int q = 1 + (r + np - 2 - pr) % (np - 1);
  if (p >= n || q >= n) return;
  if (p > q) {
    const int tmp = p;
    p = q;
    q = tmp;
  }
  double2* ap = J.A + (int64_t)p * J.lda;
  double2* aq = J.A + (int64_t)q * J.lda;
  double al = 0, be = 0;
  double2 ga = make_double2(0, 0);
  for (int i = lane; i < m; i += 32) {
    double2 x = ap[i], y = aq[i];
    al += cabs2(x);
    be += cabs2(y);
    cjfma(ga, x, y);
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga = warp_csum(ga);
  const double ag = sqrt(cabs2(ga));
  if (ag <= 1e-15 * sqrt(al * be) || ag == 0.0) return;
  if (lane == 0) rotated[j] = 1;
  const double zeta = (be - al) / (2.0 * ag);
  const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + tt * tt), sn = c * tt;
  const double2 ph = make_double2(ga.x / ag, -ga.y / ag);  // conj(gamma)/|gamma|
  for (int i = lane; i < m; i += 32) {
    double2 x = ap[i], y = cmul(aq[i], ph);
    ap[i] = make_double2(c * x.x - sn * y.x, c * x.y - sn * y.y);
    aq[i] = make_double2(sn * x.x + c * y.x, sn * x.y + c * y.y);
  }
  double2* vp = J.V + (int64_t)p * J.ldv;
  double2* vq = J.V + (int64_t)q * J.ldv;
  for (int i = lane; i < n; i += 32) {
    double2 x = vp[i], y = cmul(vq[i], ph);
    vp[i] = make_double2(c * x.x - sn * y.x, c * x.y - sn * y.y);
    vq[i] = make_double2(sn * x.x + c * y.x, sn * x.y + c * y.y);
  }
}

int jacobi_svd_batched(const std::vector<SVDJob>& jobs, cudaStream_t s) {
  if (jobs.empty()) return FDA_OK;
  DBuf<SVDJob> dj;
  FDA_TRY(dj.upload(jobs));
  const int nj = (int)jobs.size();
  int npmax = 2, nmax = 1;
  for (const SVDJob& J : jobs) npmax = std::max(npmax, J.n + (J.n & 1)), nmax = std::max(nmax, J.n);
  k_jacobi_init<<<dim3(std::max(1, std::min(1024, (nmax * nmax + 255) / 256)), nj), 256, 0, s>>>(dj.p);
  FDA_LAUNCH_CHECK();
  std::vector<int> act(nj, 1), rot(nj, 0), sweeps(nj, 0);
  DBuf<int> dact, drot;
  FDA_TRY(dact.upload(act));
  FDA_TRY(drot.alloc(nj));
  const unsigned gx = (unsigned)((npmax / 2 + JR_WARPS - 1) / JR_WARPS);
  for (int sweep = 0; sweep < 40; ++sweep) {
    FDA_CUDA(cudaMemsetAsync(drot.p, 0, sizeof(int) * nj, s));
    for (int r = 0; r < npmax - 1; ++r) {
      k_jacobi_round<<<dim3(gx, nj), 32 * JR_WARPS, 0, s>>>(dj.p, r, dact.p, drot.p);
      FDA_LAUNCH_CHECK();
    }
    FDA_CUDA(cudaMemcpyAsync(rot.data(), drot.p, sizeof(int) * nj, cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    int live = 0;
    for (int j = 0; j < nj; ++j) {
      if (!act[j]) continue;
      sweeps[j] = sweep + 1;
      if (!rot[j]) act[j] = 0;
      live += act[j];
    }
    if (!live) break;
    FDA_CUDA(cudaMemcpyAsync(dact.p, act.data(), sizeof(int) * nj, cudaMemcpyHostToDevice, s));
  }
  for (int j = 0; j < nj; ++j)
    if (jobs[j].sweeps) FDA_CUDA(cudaMemcpyAsync(jobs[j].sweeps, &sweeps[j], sizeof(int), cudaMemcpyHostToDevice, s));
  FDA_CUDA(cudaStreamSynchronize(s));
  return FDA_OK;
}


}  // namespace fda
