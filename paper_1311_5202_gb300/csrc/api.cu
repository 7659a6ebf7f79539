// C ABI of the library (declared in include/fdbem.h): handle lifetime, argument checks, error strings.
#include <stdarg.h>

#include <new>

#include "plan.cuh"

#include <vector>

namespace fda {
static thread_local char g_err[1024] = "";
void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
const char* last_error() { return g_err; }

int nystrom_points(bm_problem_s* P);
int gmres_solve(fda_plan_s* P, const double2* b, double2* x, int nrhs, const bm_gmres_opts_t* o,
                bm_gmres_stats_t* st, cudaStream_t s, bm_precond_s* pc, bm_net_s* net);
int device_peaks(double* p64, double* p32);
}  // namespace fda

int fda_tree_build_impl(bm_problem_s* P, int leaf_max, fda_tree_s* T);

using namespace fda;

#define ARG_CHECK(cond, msg)          \
  do {                                \
    if (!(cond)) {                    \
      set_error("%s", msg);           \
      return FDA_E_INVALID_ARG;       \
    }                                 \
  } while (0)

static __global__ void k_check_elems(const int32_t* e, int64_t n, int64_t nn, int* bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (e[i] < 0 || e[i] >= nn)) atomicExch(bad, 1);
}

extern "C" {

const char* fda_last_error(void) { return last_error(); }

int bm_problem_create(const double* nodes, int64_t n_nodes, const int32_t* elems6, int64_t n_elems, double k,
                      double alpha_re, double alpha_im, bm_problem_t** out) {
  ARG_CHECK(out, "out is NULL");
  *out = nullptr;
  ARG_CHECK(nodes && elems6, "nodes/elems is NULL");
  ARG_CHECK(n_nodes >= 3 && n_elems >= 1, "empty mesh");
  ARG_CHECK(n_elems <= ((int64_t)1 << 31) / 6, "too many elements");
  ARG_CHECK(k > 0 && std::isfinite(k), "k must be positive and finite");
  bm_problem_s* P = new (std::nothrow) bm_problem_s();
  if (!P) {
    set_error("host allocation failed");
    return FDA_E_OOM;
  }
  P->ne = n_elems;
  P->N = 6 * n_elems;
  P->nn = n_nodes;
  P->k = k;
  P->alpha = make_double2(alpha_re, alpha_im);
  int rc = cudaGetDevice(&P->device) == cudaSuccess ? FDA_OK : FDA_E_CUDA;
  if (rc != FDA_OK) set_error("cudaGetDevice failed");
  if (rc == FDA_OK) rc = P->nodes.upload(nodes, 3 * n_nodes);
  if (rc == FDA_OK) rc = P->elems.upload(elems6, 6 * n_elems);
  if (rc == FDA_OK) {
    DBuf<int> bad;
    rc = bad.alloc(1);
    if (rc == FDA_OK) rc = bad.zero();
    if (rc == FDA_OK) {
      k_check_elems<<<cdiv(6 * n_elems, 256), 256>>>(P->elems.p, 6 * n_elems, n_nodes, bad.p);
      int hb = 0;
      if (cudaMemcpy(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("CUDA error while checking the element table");
        rc = FDA_E_CUDA;
      } else if (hb) {
        set_error("element table holds a node index outside [0, n_nodes)");
        rc = FDA_E_INVALID_ARG;
      }
    }
  }
  if (rc == FDA_OK) rc = nystrom_points(P);
  if (rc != FDA_OK) {
    delete P;
    return rc;
  }
  *out = P;
  return FDA_OK;
}

int bm_particles_create(const double* x, const double* n, int64_t N, double k, double alpha_re, double alpha_im,
                        bm_problem_t** out) {
  ARG_CHECK(out, "out is NULL");
  *out = nullptr;
  ARG_CHECK(x && n, "x/n is NULL");
  ARG_CHECK(N >= 2 && N <= ((int64_t)1 << 31), "N outside [2, 2^31]");
  ARG_CHECK(k > 0 && std::isfinite(k), "k must be positive and finite");
  for (int64_t i = 0; i < 3 * N; ++i) ARG_CHECK(std::isfinite(x[i]) && std::isfinite(n[i]), "non-finite coordinate");
  bm_problem_s* P = new (std::nothrow) bm_problem_s();
  if (!P) {
    set_error("host allocation failed");
    return FDA_E_OOM;
  }
  P->particles = 1;
  P->ne = 0;
  P->nn = 0;
  P->N = N;
  P->k = k;
  P->alpha = make_double2(alpha_re, alpha_im);
  std::vector<double> w((size_t)N, 1.0);
  int rc = cudaGetDevice(&P->device) == cudaSuccess ? FDA_OK : FDA_E_CUDA;
  if (rc != FDA_OK) set_error("cudaGetDevice failed");
  if (rc == FDA_OK) rc = P->x.upload(x, 3 * N);
  if (rc == FDA_OK) rc = P->n.upload(n, 3 * N);
  if (rc == FDA_OK) rc = P->w.upload(w);
  if (rc != FDA_OK) {
    delete P;
    return rc;
  }
  *out = P;
  return FDA_OK;
}

int bm_problem_geometry(const bm_problem_t* prob, double* x_dev, double* n_dev, double* w_dev) {
  ARG_CHECK(prob, "problem is NULL");
  if (x_dev) FDA_CUDA(cudaMemcpy(x_dev, prob->x.p, sizeof(double) * 3 * prob->N, cudaMemcpyDeviceToDevice));
  if (n_dev) FDA_CUDA(cudaMemcpy(n_dev, prob->n.p, sizeof(double) * 3 * prob->N, cudaMemcpyDeviceToDevice));
  if (w_dev) FDA_CUDA(cudaMemcpy(w_dev, prob->w.p, sizeof(double) * prob->N, cudaMemcpyDeviceToDevice));
  return FDA_OK;
}

void bm_problem_destroy(bm_problem_t* prob) { delete prob; }

static __global__ void k_plane_wave(const double* x, const double* n, int64_t N, const double* dirs, int nrhs,
                                    double k, double2 alpha, double2* b) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N * nrhs) return;
  int r = (int)(q / N);
  int64_t i = q - (int64_t)r * N;
  const double* d = dirs + 3 * r;
  double ph = k * (d[0] * x[3 * i] + d[1] * x[3 * i + 1] + d[2] * x[3 * i + 2]);
  double sn, cs;
  sincos(ph, &sn, &cs);
  double2 u = make_double2(cs, sn);
  double dn = d[0] * n[3 * i] + d[1] * n[3 * i + 1] + d[2] * n[3 * i + 2];
  double2 dudn = cmul(make_double2(0, k * dn), u);  // i k (d.n) u
  b[q] = cadd(u, cmul(alpha, dudn));
}

int bm_rhs_plane_wave(const bm_problem_t* prob, const double* dirs, int nrhs, void* b_dev, void* stream) {
  ARG_CHECK(prob && dirs && b_dev, "NULL argument");
  ARG_CHECK(nrhs >= 1, "nrhs must be >= 1");
  FDA_TRY(problem_device_current(prob));
  std::vector<double> d(3 * (size_t)nrhs);
  for (int r = 0; r < nrhs; ++r) {
    double l = sqrt(dirs[3 * r] * dirs[3 * r] + dirs[3 * r + 1] * dirs[3 * r + 1] + dirs[3 * r + 2] * dirs[3 * r + 2]);
    ARG_CHECK(l > 0 && std::isfinite(l), "direction of zero length");
    for (int c = 0; c < 3; ++c) d[3 * r + c] = dirs[3 * r + c] / l;
  }
  DBuf<double> dd;
  FDA_TRY(dd.upload(d));
  cudaStream_t s = (cudaStream_t)stream;
  k_plane_wave<<<cdiv(prob->N * nrhs, 256), 256, 0, s>>>(prob->x.p, prob->n.p, prob->N, dd.p, nrhs, prob->k,
                                                          prob->alpha, (double2*)b_dev);
  FDA_LAUNCH_CHECK();
  FDA_CUDA(cudaStreamSynchronize(s));
  return FDA_OK;
}

int fda_build_tree(bm_problem_t* prob, int leaf_max, fda_tree_t** out) {
  ARG_CHECK(out, "out is NULL");
  *out = nullptr;
  ARG_CHECK(prob, "problem is NULL");
  ARG_CHECK(leaf_max >= 1, "leaf_max must be >= 1");
  fda_tree_s* T = new (std::nothrow) fda_tree_s();
  if (!T) {
    set_error("host allocation failed");
    return FDA_E_OOM;
  }
  int rc = fda_tree_build_impl(prob, leaf_max, T);
  if (rc != FDA_OK) {
    delete T;
    return rc;
  }
  *out = T;
  return FDA_OK;
}

int fda_tree_export(const fda_tree_t* T, fda_tree_view_t* v) {
  ARG_CHECK(T && v, "NULL argument");
  v->n_points = T->N;
  v->n_boxes = T->nbox;
  v->n_levels = T->nlev;
  v->n_direct = T->ndir;
  v->n_m2l = T->nm2l;
  for (int d = 0; d < 3; ++d) v->corner[d] = T->corner[d];
  v->side = T->side;
  v->perm = T->h_perm.data();
  v->keys = T->h_keys.data();
  v->box_level = T->h_lev.data();
  v->box_ix = T->h_ix.data();
  v->box_iy = T->h_iy.data();
  v->box_iz = T->h_iz.data();
  v->box_nchild = T->h_nch.data();
  v->box_leaf = T->h_leaf.data();
  v->box_parent = T->h_par.data();
  v->box_child_begin = T->h_cbeg.data();
  v->box_pbeg = T->h_pb.data();
  v->box_pend = T->h_pe.data();
  v->level_hf = T->h_level_hf.data();
  v->level_T = T->h_level_T.data();
  v->level_n = T->h_level_n.data();
  v->direct = T->h_direct.data();
  v->m2l_box = T->h_m2l_box.data();
  v->m2l_info = T->h_m2l_info.data();
  return FDA_OK;
}

void fda_tree_destroy(fda_tree_t* T) { delete T; }

int fda_precompute_translations(fda_tree_t* tree, const fda_config_t* cfg, fda_plan_t** out) {
  ARG_CHECK(out, "out is NULL");
  *out = nullptr;
  ARG_CHECK(cfg, "cfg is NULL");
  ARG_CHECK(cfg->eps > 0 && cfg->eps < 1, "eps must lie in (0, 1)");
  ARG_CHECK(cfg->precision == FDA_PREC_FP64 || cfg->precision == FDA_PREC_FP32, "unknown precision");
  ARG_CHECK(cfg->nrhs_max >= 1 && cfg->nrhs_max <= 4096, "nrhs_max must lie in [1, 4096]");
  ARG_CHECK(cfg->m2l_tensor >= 0 && cfg->m2l_tensor <= 3, "m2l_tensor must be 0, 1, 2 or 3");
  ARG_CHECK(cfg->op >= 0 && cfg->op <= 2, "op must be 0, 1 or 2");
  ARG_CHECK(cfg->drop_fp64 == 0 || cfg->drop_fp64 == 1, "drop_fp64 must be 0 or 1");
  ARG_CHECK(cfg->near_form >= 0 && cfg->near_form <= 4, "near_form must be 0 to 4");
  ARG_CHECK(cfg->drop_fp64 == 0 || cfg->precision == FDA_PREC_FP32, "drop_fp64 needs precision FDA_PREC_FP32");
  ARG_CHECK(cfg->op != 2 || (std::isfinite(cfg->gamma_re) && std::isfinite(cfg->gamma_im)),
            "op = 2 needs a finite Robin coefficient gamma");
  ARG_CHECK(cfg->near_split >= 0 && cfg->near_split <= 2, "near_split must be 0, 1 or 2");
  ARG_CHECK(tree, "tree is NULL");
  fda_plan_s* P = new (std::nothrow) fda_plan_s();
  if (!P) {
    set_error("host allocation failed");
    return FDA_E_OOM;
  }
  int rc = plan_build(tree, cfg, P);
  if (rc != FDA_OK) {
    delete P;
    return rc;
  }
  *out = P;
  return FDA_OK;
}

int fda_matvec(fda_plan_t* plan, const void* x, void* y, int nrhs, int dtype, void* stream) {
  ARG_CHECK(plan && x && y, "NULL argument");
  ARG_CHECK(dtype == FDA_CPLX128 || dtype == FDA_CPLX64, "unknown dtype");
  ARG_CHECK(x != y, "x and y must not overlap");
  return plan_matvec(plan, plan->cfg.precision, x, y, nrhs, dtype, (cudaStream_t)stream, false);
}

int fda_matvec_ex(fda_plan_t* plan, int precision, const void* x, void* y, int nrhs, int dtype, void* stream) {
  ARG_CHECK(plan && x && y, "NULL argument");
  ARG_CHECK(dtype == FDA_CPLX128 || dtype == FDA_CPLX64, "unknown dtype");
  ARG_CHECK(precision == FDA_PREC_FP64 || precision == FDA_PREC_FP32 || precision == FDA_PREC_TF32,
            "unknown precision");
  ARG_CHECK(x != y, "x and y must not overlap");
  return plan_matvec(plan, precision, x, y, nrhs, dtype, (cudaStream_t)stream, false);
}

int fda_autotune(fda_plan_t* plan, int nrhs, void* stream, fda_tune_report_t* report) {
  ARG_CHECK(plan && report, "NULL argument");
  ARG_CHECK(nrhs >= 1 && nrhs <= plan->cfg.nrhs_max, "nrhs outside [1, nrhs_max]");
  if (plan->cfg.precision != FDA_PREC_FP32) {
    set_error("autotuning needs a plan built with FDA_PREC_FP32");
    return FDA_E_STATE;
  }
  return autotune(plan, nrhs, (cudaStream_t)stream, report);
}

int fda_m2l_force(fda_plan_t* plan, int variant) {
  ARG_CHECK(plan, "NULL plan");
  ARG_CHECK(variant >= -1 && variant <= 15, "variant outside [-1, 15]");
  if (variant > 0 && plan->cfg.precision != FDA_PREC_FP32) {
    set_error("tensor-core M2L variants need a plan built with FDA_PREC_FP32");
    return FDA_E_STATE;
  }
  if (variant == 2 && plan->cfg.m2l_tensor != 2) {
    set_error("variant 2 needs a plan built with m2l_tensor = 2");
    return FDA_E_STATE;
  }
  if (variant != 2 && variant > 0 && plan->cfg.m2l_tensor != 1 && plan->cfg.m2l_tensor != 3) {
    set_error("variants 1 and 3 to 9 need a plan built with m2l_tensor = 1 or 3");
    return FDA_E_STATE;
  }
  if (variant >= 3 && plan->cfg.m2l_tensor == 3 && variant != 6 && variant != 7) {  // 8 to 11: TF32 only
    set_error("a 3xTF32 plan (m2l_tensor = 3) runs variants 1, 6 and 7 only");
    return FDA_E_STATE;
  }
  for (int l = 0; l < FDA_MAXLEV; ++l)
    for (int st = 0; st < 2; ++st)
      plan->m2l_choice[l][st] = (st == 1 && (variant == 8 || variant == 9 || variant >= 12)) ? 6  // V^ only
                                                                                                 // (8, 9, 12-15)
                                : (st == 0 && variant == 10) ? 8                       // 10: U^ stage only
                                                             : variant;
  return FDA_OK;
}

int fda_overlap_force(fda_plan_t* plan, int mode, int evict_first, int far_levels) {
  ARG_CHECK(plan, "NULL plan");
  ARG_CHECK(mode >= 0 && mode <= 3, "mode outside [0, 3]");
  ARG_CHECK(evict_first == 0 || evict_first == 1, "evict_first outside [0, 1]");
  ARG_CHECK(far_levels == 0 || far_levels == 1, "far_levels outside [0, 1]");
  if ((mode > 0 || evict_first || far_levels) && plan->cfg.precision != FDA_PREC_FP32) {
    set_error("the product schedules need a plan built with FDA_PREC_FP32");
    return FDA_E_STATE;
  }
  plan->overlap = mode;
  plan->near_evict = evict_first;
  plan->far_par = far_levels;
  return FDA_OK;
}

int fda_plan_check(fda_plan_t* plan) {
  ARG_CHECK(plan, "NULL plan");
  FDA_CUDA(cudaDeviceSynchronize());
  int flag = 0;
  if (plan->tc_err.p) {
    FDA_CUDA(cudaMemcpy(&flag, plan->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    FDA_TRY(plan->tc_err.zero());
    FDA_CUDA(cudaDeviceSynchronize());
  }
  if (flag) {
    set_error("a bounded device wait gave up in an earlier product (results of that product are invalid)");
    return FDA_E_TIMEOUT;
  }
  return FDA_OK;
}

struct fda_graph_s {
  fda_plan_s* plan = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

int fda_matvec_graph_create(fda_plan_t* plan, int precision, const void* x, void* y, int nrhs, int dtype,
                            void* stream, fda_graph_t** out) {
  ARG_CHECK(plan && x && y && out, "NULL argument");
  ARG_CHECK(dtype == FDA_CPLX128 || dtype == FDA_CPLX64, "unknown dtype");
  ARG_CHECK(precision == FDA_PREC_FP64 || precision == FDA_PREC_FP32 || precision == FDA_PREC_TF32,
            "unknown precision");
  ARG_CHECK(x != y, "x and y must not overlap");
  *out = nullptr;
  // capture needs a stream other than the legacy default one; the internal stream does not wait for work that
  // the caller queued elsewhere on the plan's workspaces, so the device is drained first
  cudaStream_t s = (cudaStream_t)stream, own = nullptr;
  if (!s) {
    FDA_CUDA(cudaDeviceSynchronize());
    FDA_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
    s = own;
  }
  auto done = [&](int rc) {
    if (own) cudaStreamDestroy(own);
    return rc;
  };
  // one ordinary product first: one-time kernel attributes are set outside the capture
  int rc = plan_matvec(plan, precision, x, y, nrhs, dtype, s, false);
  if (rc != FDA_OK) return done(rc);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("matvec before capture failed");
    return done(FDA_E_CUDA);
  }
  fda_graph_s* G = new fda_graph_s;
  G->plan = plan;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    delete G;
    set_error("cudaStreamBeginCapture failed");
    return done(FDA_E_CUDA);
  }
  rc = plan_matvec(plan, precision, x, y, nrhs, dtype, s, false);
  cudaError_t e = cudaStreamEndCapture(s, &G->graph);
  if (rc == FDA_OK && e != cudaSuccess) {
    set_error("cudaStreamEndCapture: %s", cudaGetErrorString(e));
    rc = FDA_E_CUDA;
  }
  if (rc == FDA_OK && cudaGraphInstantiate(&G->exec, G->graph, 0) != cudaSuccess) {
    set_error("cudaGraphInstantiate failed");
    rc = FDA_E_CUDA;
  }
  if (rc != FDA_OK) {
    if (G->graph) cudaGraphDestroy(G->graph);
    delete G;
    cudaGetLastError();
    return done(rc);
  }
  *out = G;
  return done(FDA_OK);
}

int fda_graph_launch(fda_graph_t* g, void* stream) {
  ARG_CHECK(g && g->exec, "NULL graph");
  FDA_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  return FDA_OK;
}

int fda_graph_nodes(const fda_graph_t* g, int64_t* nodes) {
  ARG_CHECK(g && nodes, "NULL argument");
  size_t n = 0;
  FDA_CUDA(cudaGraphGetNodes(g->graph, nullptr, &n));
  *nodes = (int64_t)n;
  return FDA_OK;
}

void fda_graph_destroy(fda_graph_t* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

int fda_matvec_phases(fda_plan_t* plan, int precision, const void* x, void* y, int nrhs, int dtype, void* stream,
                      double* ms) {
  ARG_CHECK(plan && x && y && ms, "NULL argument");
  ARG_CHECK(precision == FDA_PREC_FP64 || precision == FDA_PREC_FP32 || precision == FDA_PREC_TF32,
            "unknown precision");
  ARG_CHECK(dtype == FDA_CPLX128 || dtype == FDA_CPLX64, "unknown dtype");
  cudaEvent_t ev[9];
  for (int q = 0; q < 9; ++q) FDA_CUDA(cudaEventCreate(&ev[q]));
  plan->phase_ev = ev;
  int rc = plan_matvec(plan, precision, x, y, nrhs, dtype, (cudaStream_t)stream, false);
  plan->phase_ev = nullptr;
  if (rc == FDA_OK) {
    FDA_CUDA(cudaEventSynchronize(ev[8]));
    float t = 0;
    double ph[9] = {0};
    for (int q = 0; q < 8; ++q) {
      cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
      ph[q] = t;
    }
    // phases: perm, near, S2M, M2M, M2L, L2L, L2T, assemble (event q+1 closes phase q)
    for (int q = 0; q < 8; ++q) ms[q] = ph[q];
  }
  for (int q = 0; q < 9; ++q) cudaEventDestroy(ev[q]);
  return rc;
}

int fda_device_peaks(double* fp64_tflops, double* fp32_tflops) {
  ARG_CHECK(fp64_tflops && fp32_tflops, "NULL argument");
  return device_peaks(fp64_tflops, fp32_tflops);
}

int fda_plan_info(const fda_plan_t* P, fda_plan_info_t* I) {
  ARG_CHECK(P && I, "NULL argument");
  memset(I, 0, sizeof(*I));
  I->n_levels = P->tree->nlev;
  I->lmin = P->lmin;
  I->precision = P->cfg.precision;
  I->lowrank = P->cfg.lowrank;
  for (int l = 0; l < FDA_MAXLEV && l < 32; ++l) {
    I->s[l] = P->lev[l].s;
    I->n_equiv[l] = P->lev[l].se;
    I->n_check[l] = P->lev[l].sc;
    I->n_wedges[l] = P->lev[l].used ? P->lev[l].nw : 0;
    I->m2l_pairs[l] = P->m2l_pairs[l];
    I->m2l_offsets[l] = P->m2l_offsets[l];
    I->m2l_lowrank[l] = P->m2l_lowrank[l];
  }
  I->n_leaves = (int64_t)P->h_leaves.size();
  I->n_direct_blocks = P->n_blocks;
  I->near_entries = P->near_entries;
  I->corr_entries = P->corr_entries;
  I->bytes_near = 16.0 * (double)(P->near_entries + P->corr_entries) + 4.0 * P->corr_entries;
  I->bytes_s2m_l2t = P->bytes_s2m_l2t;
  I->flops_m2l = P->flops_m2l;
  for (int l = 0; l < 32; ++l) {
    I->m2l_flops_lev[l] = l < FDA_MAXLEV ? P->m2l_flops_lev[l] : 0.0;
    I->m2l_op_bytes_lev[l] = l < FDA_MAXLEV ? P->m2l_op_bytes_lev[l] : 0.0;
  }
  I->flops_m2m_l2l = P->flops_m2m;
  I->flops_near = 8.0 * (double)(P->near_entries + P->corr_entries);
  double dev = 0;
  const fda::RunOps<double2>& a = P->op64;
  dev += a.S.bytes() + a.T.bytes() + a.M.bytes() + a.K.bytes() + a.near.bytes() + a.corr.bytes() + a.lr.bytes();
  const fda::RunOps<float2>& b = P->op32;
  dev += b.S.bytes() + b.T.bytes() + b.M.bytes() + b.K.bytes() + b.near.bytes() + b.corr.bytes() + b.lr.bytes();
  dev += P->tc_img.bytes();
  dev += P->corr_col.bytes() + P->cout64.bytes() + P->cin64.bytes() + P->cout32.bytes() + P->cin32.bytes();
  I->device_bytes = dev;
  for (int q = 0; q < 8; ++q) I->setup_ms[q] = P->setup_ms[q];
  I->launches_per_matvec = P->launches;
  return FDA_OK;
}

int fda_corrections_export(const fda_plan_t* P, const int64_t* rows, int64_t nrows, int64_t cap, int64_t* cnt,
                           int64_t* cols, double* vals) {
  ARG_CHECK(P && rows && cnt && cols && vals, "NULL argument");
  if (P->prob->particles) {
    set_error("a particle-summation problem has no locally corrected weights");
    return FDA_E_STATE;
  }
  const int64_t N = P->tree->N;
  for (int64_t r = 0; r < nrows; ++r) ARG_CHECK(rows[r] >= 0 && rows[r] < N, "row out of range");
  // the plan folds most corrections into its direct blocks, so recompute them (same kernels) for export
  DBuf<int64_t> di_ptr;
  DBuf<int32_t> di_cols;
  DBuf<double2> corr;
  FDA_TRY(near_corrections(P->prob, di_ptr, di_cols, corr, nullptr, P->cfg.op,
                           make_double2(P->cfg.gamma_re, P->cfg.gamma_im)));
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t rp[2];
    FDA_CUDA(cudaMemcpy(rp, di_ptr.p + rows[r], 2 * sizeof(int64_t), cudaMemcpyDeviceToHost));
    int64_t ne = rp[1] - rp[0];
    std::vector<int32_t> el(ne);
    std::vector<double2> v(6 * ne);
    if (ne) {
      FDA_CUDA(cudaMemcpy(el.data(), di_cols.p + rp[0], sizeof(int32_t) * ne, cudaMemcpyDeviceToHost));
      FDA_CUDA(cudaMemcpy(v.data(), corr.p + 6 * rp[0], sizeof(double2) * 6 * ne, cudaMemcpyDeviceToHost));
    }
    cnt[r] = 6 * ne;
    for (int64_t q = 0; q < 6 * ne && q < cap; ++q) {
      cols[r * cap + q] = 6 * (int64_t)el[q / 6] + q % 6;
      vals[2 * (r * cap + q)] = v[q].x;
      vals[2 * (r * cap + q) + 1] = v[q].y;
    }
  }
  return FDA_OK;
}

void fda_plan_destroy(fda_plan_t* plan) { delete plan; }

int bm_gmres_solve(fda_plan_t* plan, const void* b, void* x, int nrhs, const bm_gmres_opts_t* opts,
                   bm_gmres_stats_t* stats, void* stream) {
  ARG_CHECK(plan && b && x && opts, "NULL argument");
  ARG_CHECK(nrhs >= 1, "nrhs must be >= 1");
  ARG_CHECK(opts->tol > 0, "tol must be positive");
  ARG_CHECK(opts->restart >= 1, "restart must be >= 1");
  ARG_CHECK(opts->max_iter >= 1, "max_iter must be >= 1");
  return gmres_solve(plan, (const double2*)b, (double2*)x, nrhs, opts, stats, (cudaStream_t)stream, nullptr, nullptr);
}


}  // extern "C"
