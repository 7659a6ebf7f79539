// Plan layout: translation operators, near-field matrices and execution schedules.
#pragma once
#include <cuda.h>

#include "internal.cuh"

namespace fda {

struct QRJob;
struct QFormJob;
struct SVDJob;
int zgemm_batched(char opa, char opb, int M, int N, int K, double2 alpha, const double2* const* A, int lda,
                  const double2* const* B, int ldb, double2 beta, double2* const* C, int ldc, int64_t batch,
                  cudaStream_t s);
int near_corrections(bm_problem_s* P, DBuf<int64_t>& di_ptr, DBuf<int32_t>& di_cols, DBuf<double2>& corr,
                     double* ms, int op, double2 gamma);
int upload_geometry_constants();

// One level of the tree that carries outgoing/incoming representations.
struct LevelOps {
  bool used = false, hf = false;
  int n = 1, nw = 1;        // cells per face edge, wedges
  int s = 0, se = 0, sc = 0;  // compressed dim, selected equivalent / check points
  double w = 0;
  std::vector<double> b, a, Wa;   // canonical equivalent (se x 3), check (sc x 3), check weights
  std::vector<double> rot;        // nw x 9 rotations (row-major), e_x -> wedge centre direction
  DBuf<double> d_b, d_a, d_Wa, d_rot;
  DBuf<double2> P;    // sc x s : U~ Sigma~^-1
  DBuf<double2> Pc;   // sc x s : conj(P)
  DBuf<double2> V;    // se x s : V~
  std::vector<double> sigma;
  int64_t box_begin = 0, box_end = 0;  // boxes of this level
};

// One operator expanded into the tensor-core image (see m2l_tc.cu): the TF32 image, followed for split = 1
// by the image of the TF32 remainders (value - TF32(value)), so that three products hi*hi + hi*lo + lo*hi
// keep FP32 accuracy.
// One target leaf of the near-field stream: its first row (tree order), the first entry of its column list,
// the first entry of its matrix, its rows and its columns
struct alignas(16) NsMeta {
  int64_t tb, xb, nb;
  int32_t nr, ncol;
};

struct TcImgJob {
  const double2* src;  // the M x K operator: src[i + k ld], or src[k + i ld] when trans
  int M, K;
  int64_t img_off;     // first float of the image
  int64_t ld;
  int trans;
  int split;
};
__host__ __device__ inline int64_t tc3_image_floats(int M, int K) {
  const int MT = (2 * M + 127) / 128, nk = (2 * K + 31) / 32;
  const int rows_last = 2 * M - 128 * (MT - 1);
  const int last = ((rows_last < 128 ? rows_last : 128) + 7) / 8;
  return (int64_t)(MT - 1) * nk * 16 * 256 + (int64_t)nk * last * 256;
}
int tc3_build_images(const std::vector<TcImgJob>& jobs, float* img);

// A unit of grouped gather-GEMM-scatter work: Y[:, tgt(p)] (+)= A X[:, src(p)] for pairs p.
struct GemmUnit {
  int64_t a_off;      // offset of A (M x K, column-major, lda = M) in the matrix pool
  int32_t M, K;
  int64_t p_begin;    // first pair (index into pair arrays)
  int32_t p_count;
  int32_t m0;         // first output row of this unit's row tile
  int32_t mode;       // 0: coef_out -> coef_in (add), 1: coef_out -> mid (store), 2: mid -> coef_in (add)
  int32_t pad;
};

template <typename C>
struct RunOps {
  DBuf<C> S, T, M, K, near, corr, lr;  // operator pools
};

}  // namespace fda

struct fda_plan_s {
  fda_plan_s() {
    for (int l = 0; l < FDA_MAXLEV; ++l)
      m2l_choice[l][0] = m2l_choice[l][1] = m2l_choice_fast[l][0] = m2l_choice_fast[l][1] = -1;
  }
  ~fda_plan_s() {
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    for (int i = 0; i < 4; ++i) {
      if (lvs[i]) cudaStreamDestroy(lvs[i]);
      if (ev_lvj[i]) cudaEventDestroy(ev_lvj[i]);
    }
    for (int l = 0; l < FDA_MAXLEV; ++l)
      if (ev_lev[l]) cudaEventDestroy(ev_lev[l]);
  }
  // near field and far field of an FP32 product on two streams: the far field (S2M, M2M, M2L, L2L) on the
  // plan's side stream, forked after the permutation and joined before L2T; the near field on the caller's
  // stream with a smaller persistent grid, so that the far-field kernels find room on every SM.
  // overlap: -1 or 0 serial (the default until the autotuner or fda_overlap_force sets it), 1 two streams
  // with two near-field CTAs per SM, 2 two streams with one, 3 two streams with the full grid of three.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int overlap = -1;
  int near_grid_ov[2] = {0, 0};
  fda::DBuf<int32_t> near_part_ov[2];
  int near_sel = 0;    // the overlap code of the near-field launch being issued (0: the full grid)
  int near_evict = 0;  // 1: the near-field matrix copies carry an L2 evict-first policy
  // FP32 products with far_par = 1 run the M2L of each level on its own stream (lvs[(l - lmin) % 4]), forked
  // when that level's outgoing coefficients are complete (ev_lev[l], after S2M or its M2M step) and joined
  // (ev_lvj) before L2L
  int far_par = 0;
  cudaStream_t lvs[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_lvj[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_lev[FDA_MAXLEV] = {};
  fda_tree_s* tree = nullptr;
  bm_problem_s* prob = nullptr;
  fda_config_t cfg;
  int lmin = 0, lmax = 0;  // levels carrying representations
  fda::LevelOps lev[FDA_MAXLEV];
  // coefficient slots: per box (levels >= lmin) nw * s complex per RHS
  std::vector<int64_t> h_slot;  // per box: first coefficient index (or -1)
  int64_t n_coef = 0;
  fda::DBuf<int64_t> slot;
  // leaves carrying S2M / L2T (level >= lmin)
  std::vector<int64_t> h_leaves;
  fda::DBuf<int64_t> leaves, leaf_s_off, leaf_t_off;
  // near field: blocks per target leaf
  fda::DBuf<int64_t> near_tleaf;     // target leaves with at least one block
  fda::DBuf<int64_t> near_tptr;      // CSR over those leaves -> blocks
  fda::DBuf<int64_t> near_src;       // block -> source box
  fda::DBuf<int64_t> near_off;       // block -> entry offset
  fda::DBuf<int64_t> near_coff;      // block -> first column within its target leaf's matrix
  fda::DBuf<int64_t> near_nbase;     // target leaf -> first entry of its matrix (4-entry aligned)
  fda::DBuf<int32_t> near_ncol;      // target leaf -> number of columns
  fda::DBuf<int64_t> near_xbase;     // target leaf -> first entry of its column list in near_xcol
  fda::DBuf<int32_t> near_xcol;      // column -> tree position of its source point
  fda::DBuf<fda::NsMeta> near_meta;      // target leaf -> rows, columns and offsets, one 32-byte record
  // one right-hand side: 0 = three-stage ring, 1 = four-stage ring, 2 = packed FP32x2 FMAs on duplicated
  // densities (double-buffered windows only; autotuned)
  int near_form = 0;
  fda::DBuf<float4> xdup32;          // (x.x, x.x, x.y, x.y) per point for near_form = 2
  fda::DBuf<int32_t> near_part;      // persistent CTA -> first target leaf (grid + 1 entries)
  int near_grid = 0, near_max_nr = 0;
  int64_t corr_merged = 0;           // correction entries folded into the direct blocks
  int64_t n_near_tleaf = 0, n_blocks = 0, near_entries = 0;
  fda::DBuf<int64_t> corr_ptr;       // tree-order CSR of the correction matrix
  fda::DBuf<int32_t> corr_col;
  int64_t corr_entries = 0;
  // M2M / L2L: per level, parent boxes (non-leaf, level in [lmin, lmax-1])
  std::vector<int64_t> h_parents[FDA_MAXLEV];
  fda::DBuf<int64_t> parents[FDA_MAXLEV];
  int64_t m_off[FDA_MAXLEV] = {0};   // offset of M~(l, o, z) blocks in the M pool
  // M2L
  std::vector<fda::GemmUnit> h_units[FDA_MAXLEV][2];  // [level][0: dense or V^ stage, 1: U^ stage]
  fda::DBuf<fda::GemmUnit> units[FDA_MAXLEV][2];
  // tensor-core units: one per (group, pair chunk, block of up to 256 output rows)
  std::vector<fda::GemmUnit> h_tc_units[FDA_MAXLEV][2];
  fda::DBuf<fda::GemmUnit> tc_units[FDA_MAXLEV][2];
  int tc_max_rows[FDA_MAXLEV][2] = {{0}};
  // TF32 tensor-core form: operator images (canonical shared-memory layout) and units of up to 128 pairs
  fda::DBuf<float> tc_img;
  std::vector<fda::GemmUnit> h_tc3_units[FDA_MAXLEV][2];
  fda::DBuf<fda::GemmUnit> tc3_units[FDA_MAXLEV][2];
  int tc3_mt[FDA_MAXLEV][2] = {{0}};  // largest number of 128-row tiles of a unit
  int tc3_maxk[FDA_MAXLEV][2] = {{0}};  // largest complex K of a unit
  int64_t tc3_split[FDA_MAXLEV][2] = {{0}};  // units [0, split) have 2K <= 64
  // swapped-operand V^ kernel: the mode-1 units of stage 0 ordered by TMEM class (32, 64, 128, 256 columns);
  // class c covers units [vsw_cls[l][c], vsw_cls[l][c + 1])
  std::vector<fda::GemmUnit> h_vsw_units[FDA_MAXLEV];
  fda::DBuf<fda::GemmUnit> vsw_units[FDA_MAXLEV];
  int64_t vsw_cls[FDA_MAXLEV][5] = {{0}};
  // TMA-fed V^ kernel (one right-hand side): per level, a 2-D tensor map over the level's FP32 outgoing
  // coefficient vectors (rows of 2 s floats, 128-byte swizzle, boxes of 32 floats x 1 row for tile::gather4)
  alignas(64) CUtensorMap vtm_map[FDA_MAXLEV];
  bool vtm_ok[FDA_MAXLEV] = {false};
  int64_t vtm_base[FDA_MAXLEV] = {0};
  // persistent warp-specialised scatter kernel: the short-K U^-stage units (2 r <= 64), up to 512 pairs each
  std::vector<fda::GemmUnit> h_ws_units[FDA_MAXLEV];
  fda::DBuf<fda::GemmUnit> ws_units[FDA_MAXLEV];
  int ws_mt[FDA_MAXLEV] = {0};
  // the dense (mode 0) units of stage 0, run by the TF32 kernel beside the swapped V^ kernel
  std::vector<fda::GemmUnit> h_dn_units[FDA_MAXLEV];
  fda::DBuf<fda::GemmUnit> dn_units[FDA_MAXLEV];
  int dn_mt[FDA_MAXLEV] = {0}, dn_maxk[FDA_MAXLEV] = {0};
  // M2M / L2L on the same tensor-core kernel: per level (parent level l), units and pair arrays
  std::vector<fda::GemmUnit> h_mm_units[FDA_MAXLEV], h_ll_units[FDA_MAXLEV];
  fda::DBuf<fda::GemmUnit> mm_units[FDA_MAXLEV], ll_units[FDA_MAXLEV];
  fda::DBuf<int64_t> mm_src, mm_tgt, ll_src, ll_tgt;
  int mm_mt[FDA_MAXLEV] = {0}, ll_mt[FDA_MAXLEV] = {0};
  int fma_tm[FDA_MAXLEV][2] = {{0}};  // row tile of the FMA M2L units (16, 32 or 64)
  int m2l_choice[FDA_MAXLEV][2];      // autotuned M2L kernel per (level, stage), -1: from the plan options
  // products in FDA_PREC_TF32 on a plan with 3xTF32 images: single-pass TF32 kernels on the leading part of
  // each image, with their own autotuned choices
  int fast_tf32 = 0;
  int m2l_choice_fast[FDA_MAXLEV][2];
  int near_csep = -1;                 // near-field schedule: 0 per-leaf corrections, 1 split, 2 split + DB windows
  int near_wide = -1;                 // autotuned right-hand sides per near-field pass for wide batches
  fda::DBuf<int64_t> pair_src, pair_tgt;  // coefficient indices (slot + wedge * s)
  fda::DBuf<int64_t> pair_mid;            // low-rank intermediate index per pair (-1 if dense)
  int64_t n_pairs = 0, n_mid = 0;
  int64_t m2l_pairs[FDA_MAXLEV] = {0}, m2l_offsets[FDA_MAXLEV] = {0}, m2l_lowrank[FDA_MAXLEV] = {0};
  // operators
  fda::RunOps<double2> op64;
  fda::RunOps<float2> op32;
  // workspaces (sized for nrhs_max)
  fda::DBuf<double2> xt64, yt64, cout64, cin64, mid64;
  fda::DBuf<float2> xt32, yt32, cout32, cin32, mid32;
  fda::DBuf<int64_t> iperm;
  fda::DBuf<int> lev_s, lev_nw;  // per level: compressed dimension and wedge count
  int max_leaf = 1;
  double2 diag_c = {0.5, 0.0};   // y = diag_c x + ...: 1/2 (operator A), -alpha/2 (operator B), 0 (particle sums)
  int64_t launches = 0;          // kernels launched by the last matvec
  fda::DBuf<int> tc_err;         // set by a tensor-core kernel whose bounded wait gave up
  cudaEvent_t* phase_ev = nullptr;  // when set, 9 events recorded between the matvec phases
  double setup_ms[8] = {0};
  double flops_m2l = 0, flops_m2m = 0, bytes_s2m_l2t = 0;
  double m2l_flops_lev[FDA_MAXLEV] = {0}, m2l_op_bytes_lev[FDA_MAXLEV] = {0};
  // GMRES workspace (allocated on first solve)
  fda::DBuf<double2> gm_V, gm_w, gm_r, gm_x, gm_z, gm_b;
  fda::DBuf<double> gm_small;
};

namespace fda {
int plan_build(fda_tree_s* T, const fda_config_t* cfg, fda_plan_s* P);
int plan_matvec(fda_plan_s* P, int prec, const void* x, void* y, int nrhs, int io_dtype, cudaStream_t s,
                bool tree_order);
int autotune(fda_plan_s* P, int nrhs, cudaStream_t s, fda_tune_report_t* R);
}  // namespace fda
