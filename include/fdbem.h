/*
 * fdbem.h — C ABI of the GB300 fast directional Burton-Miller BEM library.
 *
 * The library solves the rigid-scatter Burton-Miller equation of Cao, Wen, Xiao & Liu,
 * "A fast directional BEM for large-scale acoustic problems based on the Burton-Miller
 * formulation" (Eng. Anal. Bound. Elem.):
 *     (1/2) u + (D + alpha H) u = u_inc + alpha du_inc/dn          (Eq. bm with q = 0)
 * discretised by the locally corrected Nystrom method on curved 6-node triangles (Sec. 2.2),
 * A x = b (Eq. Axb), solved by GMRES whose matrix-vector product is the kernel-independent
 * wideband fast directional algorithm (Sec. 3) with compressed and low-rank translation
 * matrices (Sec. 4).
 *
 * Conventions shared by every entry point:
 *  - Mesh: nodes (n_nodes x 3 doubles, row-major), elems (n_elems x 6 int32, node order
 *    v0, v1, v2, m01, m12, m20, counter-clockwise seen from outside the body).
 *  - Unknowns: N = 6 * n_elems Nystrom points; DOF index = 6 * element + j where j runs over
 *    the 6-point Gauss rule in the order (xi1, xi2) = (a1,a1),(b1,a1),(a1,b1),(a2,a2),(b2,a2),(a2,b2),
 *    a1 = 0.44594849091596488632, b1 = 1 - 2 a1, a2 = 0.09157621350977074346, b2 = 1 - 2 a2.
 *  - Normals: the paper's n points out of the fluid, i.e. into the scatterer.
 *  - Vectors: caller-owned DEVICE memory, interleaved complex (re, im), column-major N x nrhs,
 *    in the user's DOF order. dtype FDA_CPLX128 (double) or FDA_CPLX64 (float).
 *  - Streams: `stream` is a cudaStream_t (or NULL for the legacy default stream). Work is
 *    enqueued on it; the call returns once the work is enqueued unless stated otherwise.
 *  - Handles are library-owned and freed by the matching *_destroy. A handle must not be used
 *    from two host threads at once.
 *  - Every function returns FDA_OK (0) or a negative FDA_E_* code; fda_last_error() then
 *    describes the failure (thread-local string, valid until the next call on that thread).
 *    No C++ exception crosses this boundary.
 */
#ifndef FDBEM_H
#define FDBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FDA_OK = 0,
  FDA_E_INVALID_ARG = -1,   /* bad size, null pointer, unsupported option */
  FDA_E_OOM = -2,           /* device or host allocation failed */
  FDA_E_CUDA = -3,          /* a CUDA runtime call or kernel launch failed */
  FDA_E_NOT_CONVERGED = -4, /* GMRES hit max_iter before tol */
  FDA_E_BREAKDOWN = -5,     /* GMRES stagnated (residual did not decrease over a full restart cycle) */
  FDA_E_NAN = -6,           /* NaN or Inf detected in a vector */
  FDA_E_TIMEOUT = -7,       /* a bounded device-side wait gave up */
  FDA_E_STATE = -8          /* call not valid for this handle's state */
};

enum { FDA_CPLX128 = 0, FDA_CPLX64 = 1 };

/* Arithmetic of the matrix-vector product (near field and translations). */
enum {
  FDA_PREC_FP64 = 0, /* plain FP64 everywhere */
  FDA_PREC_FP32 = 1, /* near field and translations in FP32 with FP32 accumulation */
  FDA_PREC_TF32 = 2  /* products only (fda_matvec_ex): as FDA_PREC_FP32, with the tensor-core translations in one
                        TF32 pass also on a plan built with 3xTF32 images (m2l_tensor = 3: the leading TF32
                        part of each image is read, its remainder skipped); on other FP32 plans the same product
                        as FDA_PREC_FP32 */
};

typedef struct bm_problem_s bm_problem_t;
typedef struct fda_tree_s fda_tree_t;
typedef struct fda_plan_s fda_plan_t;

/* ------------------------------------------------------------------------------------------ */
/* Problem: mesh, wavenumber, Burton-Miller coupling (Sec. 2.1-2.2).                          */
/* ------------------------------------------------------------------------------------------ */

/* Create a particle-summation problem (Sec. 5.1, Eq. sum): N points x (host, N x 3) with unit normals n
 * (host, N x 3), on which fda_matvec evaluates p_i = sum_{j != i} [G(x_i, y_j) + alpha dG/dn_y(x_i, y_j)] q_j
 * with the same octree, translations and near field as the boundary-element operator, but plain kernel
 * values (no quadrature weights, no local corrections) and no 1/2 q_i term. Inputs are copied.
 * fda_corrections_export and bm_precond_create refuse such problems (FDA_E_STATE).
 * Errors: FDA_E_INVALID_ARG for N < 2, k <= 0 or a non-finite coordinate. */
int bm_particles_create(const double* x, const double* n, int64_t N, double k, double alpha_re, double alpha_im,
                        bm_problem_t** out);

/* Create a problem from a host mesh. Computes on the GPU the Nystrom points, the paper's
 * normals (into the body) and the quadrature weights w_j = Gauss weight * area Jacobian
 * (6-point rule, Sec. 2.2). alpha is the Burton-Miller coupling constant (the paper uses
 * alpha = i/k, Eq. bm). Inputs are host pointers, copied; the caller keeps ownership.
 * Errors: FDA_E_INVALID_ARG for n_elems < 1, k <= 0, a node index out of range. */
int bm_problem_create(const double* nodes, int64_t n_nodes, const int32_t* elems6, int64_t n_elems, double k,
                      double alpha_re, double alpha_im, bm_problem_t** out);

/* Copy the Nystrom points (N x 3), normals (N x 3) and weights (N) to caller DEVICE buffers
 * (any of them may be NULL). Synchronous. */
int bm_problem_geometry(const bm_problem_t* prob, double* x_dev, double* n_dev, double* w_dev);

/* Right-hand side of the rigid-scatter problem for plane waves u_inc = exp(i k d.x):
 * b = u_inc + alpha du_inc/dn_x (Eq. bm with q = 0; Sec. 5.3). dirs: host, nrhs x 3 (normalised
 * inside). b_dev: DEVICE, N x nrhs complex128, column-major. The problem's device must be the current
 * device (FDA_E_INVALID_ARG otherwise). Waits for its stream before it returns. */
int bm_rhs_plane_wave(const bm_problem_t* prob, const double* dirs, int nrhs, void* b_dev, void* stream);

/* The same right-hand side without any device allocation (the paper has no counterpart). It serves
 * callers that may issue CUDA calls but must not allocate device memory at the point they need a
 * right-hand side: codes that forbid allocation after start-up (every byte reserved up front), or code
 * that has handed the rest of the device to another allocator. The directions go through a fixed
 * file-scope device array of FDA_RHS_NOALLOC_MAX = 1024 directions (24 KiB, held by every GPU that loads
 * the library until the process exits); nrhs > 1024 fails with FDA_E_INVALID_ARG and writes nothing.
 * Set-up: the first call in a CUDA context of a device looks up that array's address there (a context
 * created later, e.g. after cudaDeviceReset, gets its own look-up); make that first call before any
 * stream capture begins. Every call shares the array and overwrites the entries it uses; calls that
 * overlap on the GPU (different streams without ordering) race on it. The problem's device must be the
 * current device (FDA_E_INVALID_ARG otherwise). The call waits for its stream before it returns. */
int bm_rhs_plane_wave_noalloc(const bm_problem_t* prob, const double* dirs, int nrhs, void* b_dev, void* stream);

void bm_problem_destroy(bm_problem_t* prob);

/* ------------------------------------------------------------------------------------------ */
/* Octree and interaction lists (Sec. 3.1.1), built by GPU kernels under integer rules:        */
/*  - root cube: bounding-box centre, side = largest extent * (1 + 2^-20); points quantised to */
/*    21-bit integer coordinates, 63-bit Morton keys, stable sort (ties by DOF index);          */
/*  - a box splits while it holds more than leaf_max points (N_p of Eq. npleaf);               */
/*  - level l (width w) is high-frequency iff k w >= 2 pi; near field: LF adjacent boxes, HF    */
/*    max-norm box offset m with m - 1 <= floor(k w / pi) (dist <= c_d k w^2, c_d = 1/pi);      */
/*  - interaction lists I^C = N^P \ N^C by a dual recursion over near pairs from (root, root);  */
/*    a near pair with a leaf on either side becomes a direct (near-field) block;              */
/*  - directional wedges: n x n cells on each face of [-1,1]^3, n = 2^(L_hf - l) where L_hf is */
/*    the finest HF level; a direction picks the face of its largest |component| (lowest axis  */
/*    on ties) and, along each remaining axis j, cell min(n-1, floor(n (d_j + m) / (2 m))).    */
/* ------------------------------------------------------------------------------------------ */
int fda_build_tree(bm_problem_t* prob, int leaf_max, fda_tree_t** out);

/* Host view of a tree, for tests and diagnostics. Arrays are owned by the tree handle and stay
 * valid until fda_tree_destroy. Boxes are ordered level by level, Morton order within a level;
 * children of a box are contiguous. Lists are sorted by (target box, source box). */
typedef struct {
  int64_t n_points, n_boxes, n_levels, n_direct, n_m2l;
  double corner[3], side;
  const int64_t* perm;        /* tree position -> DOF index (n_points) */
  const uint64_t* keys;       /* sorted Morton keys (n_points) */
  const int32_t* box_level;   /* n_boxes each */
  const int32_t* box_ix;
  const int32_t* box_iy;
  const int32_t* box_iz;
  const int32_t* box_nchild;
  const int32_t* box_leaf;
  const int64_t* box_parent;  /* -1 for the root */
  const int64_t* box_child_begin; /* -1 for leaves */
  const int64_t* box_pbeg;    /* point range [pbeg, pend) in tree order */
  const int64_t* box_pend;
  const int32_t* level_hf;    /* n_levels each */
  const int32_t* level_T;
  const int32_t* level_n;
  const int64_t* direct;      /* n_direct x 2: (target box, source box) */
  const int64_t* m2l_box;     /* n_m2l x 2: (target box, source box) */
  const int32_t* m2l_info;    /* n_m2l x 6: level, dx, dy, dz (source - target, box units),
                                 outgoing wedge of the source, incoming wedge of the target */
} fda_tree_view_t;

int fda_tree_export(const fda_tree_t* tree, fda_tree_view_t* view);
void fda_tree_destroy(fda_tree_t* tree);

/* ------------------------------------------------------------------------------------------ */
/* Plan: translation operators (Sec. 3.1.2, 3.2, 4) and near-field corrections (Sec. 2.2).    */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  double eps;        /* FDA accuracy: equivalent/check point selection and SVD truncation at
                        sigma_i >= eps sigma_1 (Eq. invr), low-rank M2L truncation (Eq. lrdk) */
  int precision;     /* FDA_PREC_FP64 or FDA_PREC_FP32: arithmetic of fda_matvec */
  int lowrank;       /* 1: factor compressed M2L matrices K~ = U^ V^ when rank < s/2 (Sec. 4.2) */
  int nrhs_max;      /* largest nrhs fda_matvec / bm_gmres_solve will be called with (>= 1) */
  int m2l_tensor;    /* FP32 plans: M2L (and its low-rank stages) on the tensor cores (tcgen05, TF32):
                        0 = FP32 FMA; 1 = TF32 with operators pre-expanded at plan time into their
                        shared-memory images (extra device memory about twice the FP32 M2L operators;
                        levels with s > 256 keep the FMA kernel); 2 = 3xTF32 split with the operators
                        expanded in the kernel (FP32-level accuracy); 3 = 3xTF32 from pre-expanded TF32 and
                        remainder images (twice the images of 1; the gathered coefficients are split in
                        shared memory; three products hi*hi + hi*lo + lo*hi; FP32-level accuracy for
                        products whose far field dominates) */
  int op;            /* operator of fda_matvec (boundary-element problems; particle problems ignore it):
                        0 = A = 1/2 I + Dbar + alpha Hbar (Eq. bm, the unknown u); 1 = B = Sbar + alpha Mbar
                        - alpha/2 I, which maps Neumann data q to the radiation right-hand side of Eq. bm
                        (same tree and translations; S2M from monopole sources, near field and local
                        corrections of G + alpha dG/dn_x); 2 = A + gamma B, the operator of Eq. bm under
                        Robin data a u + b q = g with gamma = a/b (q = (g - a u)/b eliminated; the right-hand
                        side is u_inc + alpha q_inc + (1/b) B g): S2M from dipole + gamma monopole sources,
                        near field and corrections of both kernel pairs, diagonal 1/2 - gamma alpha/2 */
  int near_split;    /* near-field schedule until fda_autotune chooses: 0 = the correction entries outside the
                        direct blocks are applied inside the near-field stream, per target leaf; 1 = by their
                        own CSR kernel (one warp per row) before the stream; 2 = as 1, with the stream's
                        density windows double-buffered for one right-hand side (the next window's densities
                        copied while the current one is used). Same sums, other order. */
  int drop_fp64;     /* FP32 plans: 1 = release every FP64 operator and near-field matrix once its FP32 copy
                        exists (about 60% of the device memory of a plan that keeps both). Such a plan serves
                        fda_matvec in FP32 only (FP64 requests fail with FDA_E_STATE), bm_gmres_solve with
                        refine = 0 (FP64 Krylov basis around the FP32 operator; with TF32 translations the
                        rounding stalls GMRES near a 1e-4 residual, with 3xTF32 ones, m2l_tensor = 3, it
                        reaches 1e-5 and below) and no preconditioner. */
  int near_form;      /* near-field stream (fda_autotune chooses it by timing): 0 = the FMA form with three ring
                        stages of 16 KB (one right-hand side); 1 = one right-hand side with four stages of about
                        14 KB; 2 = packed FP32x2 FMAs (FP32): one right-hand side with near_split = 2 on densities
                        kept twice over, (x.x, x.x, x.y, x.y); passes of 4 or 16 right-hand sides with each
                        matrix entry paired in registers; 3 = one right-hand side with near_split = 2 in a slim
                        CTA (three 12 KB stages, two 4 KB windows) that leaves shared memory to a far field
                        running beside it; 4 = products of 16 or more right-hand sides (FP32, leaves of at most
                        64 points) on the tensor cores in 3xTF32, up to 64 right-hand sides per pass over the
                        matrices, corrections outside the direct blocks by their own kernel. Same sums, other
                        order */
  double gamma_re, gamma_im;  /* op = 2: the Robin coefficient gamma = a/b (ignored otherwise) */
} fda_config_t;

/* Build every translation operator and the near-field matrices on the GPU (FP64 masters):
 *  - per level: equivalent points b and check points a selected by pivoted QR from candidate
 *    sets (LF: cube surfaces; HF: spheres around the box and a cone of far check points for
 *    the canonical wedge direction (1,0,0), rotated to every other wedge), R = G(a, b) and its
 *    truncated SVD (Eq. svdr, invr);
 *  - compressed S~ (with dG/dn_y check potentials, Eq. evas2mh), M~, K~, L~ = M~^T and T~
 *    (with E_dn = G + alpha dG/dn_x, Eq. eval2t) of Eq. cmps..cmpt;
 *  - optional low-rank factors of each K~;
 *  - the local regions D_i, the locally corrected weights (Eq. local correction; singular and
 *    hypersingular self-element moments in FP64), the direct near-field blocks and the
 *    correction matrix of Eq. kcorrection.
 * Synchronous (returns when the plan is complete). The tree and problem must outlive the plan.
 * Errors: FDA_E_INVALID_ARG (NULL cfg or out; a configuration field out of range, checked before the tree;
 * NULL tree), FDA_E_OOM, FDA_E_CUDA. On error *out is NULL. */
int fda_precompute_translations(fda_tree_t* tree, const fda_config_t* cfg, fda_plan_t** out);

/* y = A x with A = (1/2) I + Dbar + alpha Hbar (Eq. bm, q = 0; Eq. kcorrection), evaluated
 * as near field + FDA far field. x, y: DEVICE, N x nrhs complex (dtype), column-major, user
 * DOF order; x and y must not overlap. 1 <= nrhs <= cfg.nrhs_max. Asynchronous on `stream`. */
int fda_matvec(fda_plan_t* plan, const void* x, void* y, int nrhs, int dtype, void* stream);

/* fda_matvec with an explicit arithmetic: FDA_PREC_FP64 works on every plan that keeps its FP64 operators
 * (not drop_fp64); FDA_PREC_FP32 and FDA_PREC_TF32 need a plan built with cfg.precision = FDA_PREC_FP32 (else
 * FDA_E_STATE). */
int fda_matvec_ex(fda_plan_t* plan, int precision, const void* x, void* y, int nrhs, int dtype, void* stream);

/* Autotuner (no paper counterpart). For an FP32 plan and a batch width nrhs (1..nrhs_max), times on the
 * plan's own operators every M2L (level, stage) with the FP32 FMA kernel and with the plan's tensor-core
 * kernels (m2l_tensor 1: four tile shapes, two with a bulk-reduction epilogue, and for the V^ stage the
 * swapped-operand kernel; m2l_tensor 2: one), for nrhs >= 12 the near field at 4 and 16 right-hand sides per pass over
 * the near-field matrices, and the near field with its off-block correction entries inside the stream or as a
 * separate CSR kernel; the plan keeps the faster variant of each for all later products. Synchronous;
 * overwrites the plan's internal workspaces only. report (HOST) receives the timings and choices.
 * Errors: FDA_E_INVALID_ARG, FDA_E_STATE (FP64-only plan), FDA_E_OOM, FDA_E_CUDA. */
typedef struct {
  int32_t entries;        /* (level, stage) rows filled below */
  int32_t level[64];
  int32_t stage[64];      /* 0: dense K~ or V^ stage, 1: U^ stage */
  double ms_fma[64];      /* FP32 FMA kernel, best of 3 */
  double ms_tensor[64];   /* tensor-core kernel, best of 3 over its tile shapes (-1 when the plan holds none) */
  int32_t chosen[64];     /* 0: FMA kernel, 1: tensor-core kernel (default shape), 2 to 4: tensor-core kernel
                             (alternative shapes: other column width or stage count), 5 and 6: tensor-core
                             kernel with the bulk-reduction epilogue (default and single-stage shape), 7 and 8:
                             stage 0 with the swapped-operand V^ kernel (one and two pipeline stages), 9: stage
                             1 with the persistent warp-specialised scatter kernel, 10: bulk-reduction epilogue,
                             32 columns, exact row tiles, 11 and 12: stage 0 with the V^ kernel fed by TMA row
                             gathers (four and three stages), 13 and 14: stage 0 with the swapped V^ kernel in
                             16-wide K chunks (two and three in flight) */
  double near_ms[2];      /* near field at 4 and 16 right-hand sides per pass (nrhs >= 12; else 0) */
  int32_t near_rhs_per_pass;
  int32_t near_split;     /* near-field schedule kept: 0 = the correction entries outside the direct blocks inside
                             the stream, per target leaf; 1 = by their own CSR kernel before the stream; 2 = as 1,
                             and the stream's density windows double-buffered (one right-hand side) */
  double near_split_ms[2];  /* near field (at the chosen width) with schedules 0 and 1 */
  double near_window_ms;    /* schedule 2 (nrhs = 1; else -1) */
  int32_t overlap;          /* FP32 product schedule kept: 0 = serial; 1 to 3 = the far field (S2M, M2M, M2L,
                               L2L) on a stream of the plan, beside the near field on the caller's stream with two
                               (1), one (2) or three (3) near-field CTAs per SM */
  int32_t near_evict_first; /* 1: the near-field matrix copies carry an L2 evict-first policy */
  int32_t far_levels_concurrent; /* 1: the M2L of each level runs on its own stream of the plan */
  int32_t near_form;        /* near-field form kept (as fda_config_t.near_form; forms 1 and 3 serve one
                               right-hand side, form 4 batches) */
  double schedule_ms[16];   /* whole FP32 products, best of 5, at index overlap + 4 evict_first + 8 far_levels
                               (the three settings of fda_overlap_force); -1 where not timed (the setting needs
                               a near field in the stream form or a far field that the plan lacks) */
  double near_form_ms[3][3]; /* near field in form f (row) and schedule q (column) at the chosen width; -1 where
                                not timed (form 1: one right-hand side; form 2 with one right-hand side:
                                schedule 2 only) */
  int32_t m2l_rechosen;     /* M2L choices changed by the last pass: variants within 15% of the fastest of their
                               (level, stage) when timed alone, timed again inside whole products under the
                               chosen schedule (a change must gain at least 0.5%) */
  int32_t near_slim;        /* 1: the two-stream product runs the slim near-field CTA (near_form = 3: three
                               12 KB stages and two 4 KB windows, about 47 KB; one right-hand side, near_split 2) */
  double schedule_slim_ms[16]; /* schedule_ms with the slim near-field CTA (two-stream schedules only; else -1) */
  double product_ms;        /* the whole FP32 product with every choice made, best of 5 (-1 without far field) */
  double near_tc_ms;        /* the near field on the tensor cores (near_form = 4), best of 3; -1 when not timed
                               (fewer than 16 right-hand sides, leaves of more than 64 points) */
} fda_tune_report_t;
int fda_autotune(fda_plan_t* plan, int nrhs, void* stream, fda_tune_report_t* report);

/* Force one M2L kernel variant for every (level, stage) of an FP32 plan (diagnostic and testing; no paper
 * counterpart), replacing the autotuner's choices: -1 = the plan's default, 0 = FP32 FMA kernel, 1 = TF32
 * tensor cores from operator images (default shape), 2 = in-kernel expansion (plans with m2l_tensor = 2),
 * 3 to 5 = variant 1 in the alternative tile shapes, 6 and 7 = variant 1 with the bulk-reduction epilogue
 * (default and single-stage shape), 8 and 9 = the swapped-operand V^ kernel (one and two stages) for the V^
 * stage, with variant 6 for the U^ stage, 10 = the persistent warp-specialised scatter kernel for the U^ stage,
 * with variant 8 for the V^ stage, 11 = variant 1 with the bulk-reduction epilogue, 32 columns and exactly the
 * row tiles needed (the most CTAs per SM), 12 and 13 = the V^ kernel fed by TMA row gathers (four and three
 * stages; one right-hand side, else variant 8), 14 and 15 = the swapped V^ kernel with 16-wide K chunks (two
 * and three in flight), each with variant 6 for the U^ stage. A variant that does not apply to a (level, stage)
 * runs the FMA kernel there. Errors: FDA_E_INVALID_ARG (variant outside [-1, 15]), FDA_E_STATE (plan without
 * the kernel's operators). */
int fda_m2l_force(fda_plan_t* plan, int variant);

/* Set the schedule of FP32 products (no paper counterpart; fda_autotune chooses the three settings by timing
 * whole products). far_levels = 1 runs the M2L of each level on a stream of the plan of its own (four streams,
 * shared round-robin beyond four levels), forked when the level's outgoing coefficients are complete and joined
 * before L2L; 0 runs the levels in sequence. evict_first = 1 gives the near field's bulk copies of its matrices
 * an L2 evict-first policy (they are read once per pass), 0 the default policy. mode: 0 = the near field and
 * the far field in sequence on the caller's stream; 1 to 3 = S2M, M2M, M2L and L2L (which read x and write
 * only the expansion coefficients) on a stream the plan owns, forked after the permutation of x and joined
 * before L2T, while the near field streams on the caller's stream with two (1), one (2) or three (3)
 * persistent CTAs per SM. Products stay ordered on the caller's stream and
 * graph capture follows the fork and join. The two-stream forms apply only to FP32 products of plans whose
 * near field runs in the stream form; no stream but the caller's is used while phase events are recorded.
 * Errors: FDA_E_INVALID_ARG (mode outside [0, 3], evict_first or far_levels outside [0, 1]), FDA_E_STATE (plan
 * without FP32 operators). */
int fda_overlap_force(fda_plan_t* plan, int mode, int evict_first, int far_levels);

/* CUDA-graph form of one product (the batched matvec of many incident directions replayed without
 * per-kernel launch cost; no paper counterpart). fda_matvec_graph_create runs the product once on `stream`
 * (synchronously; a null stream means an internal one for the capture, used after the whole device has been
 * synchronised, so that no earlier work on the plan's workspaces is still running), then captures the same
 * product for these exact x, y (DEVICE, as fda_matvec_ex), nrhs, dtype and precision into a graph.
 * fda_graph_launch replays it on any stream: the caller refreshes x in place and reads y after the replay; the
 * graph keeps pointers to x, y and the plan, which must stay alive. fda_graph_nodes returns its kernel/memset node
 * count. Errors: FDA_E_INVALID_ARG, FDA_E_CUDA (capture or instantiation refused). */
typedef struct fda_graph_s fda_graph_t;
int fda_matvec_graph_create(fda_plan_t* plan, int precision, const void* x, void* y, int nrhs, int dtype,
                            void* stream, fda_graph_t** out);
int fda_graph_launch(fda_graph_t* g, void* stream);
int fda_graph_nodes(const fda_graph_t* g, int64_t* nodes);
void fda_graph_destroy(fda_graph_t* g);

/* Same product as fda_matvec_ex, with CUDA events recorded on `stream` between the phases; on return
 * (synchronous) phase_ms[0..7] holds the device time of: input permutation, near field (direct blocks +
 * corrections), S2M, M2M, M2L, L2L, L2T, output assembly. Diagnostic; no paper counterpart. */
int fda_matvec_phases(fda_plan_t* plan, int precision, const void* x, void* y, int nrhs, int dtype, void* stream,
                      double* phase_ms);

/* Plan statistics for measurement (sizes, algorithmic bytes and flops per matvec). */
typedef struct {
  int32_t n_levels, lmin, precision, lowrank;
  int32_t s[32];            /* compressed dimension per level (0 where unused) */
  int32_t n_equiv[32];      /* selected equivalent points per level */
  int32_t n_check[32];      /* selected check points per level */
  int32_t n_wedges[32];     /* wedges per level (1 in LF) */
  int64_t m2l_pairs[32];    /* M2L pairs per level */
  int64_t m2l_offsets[32];  /* distinct K~ per level */
  int64_t m2l_lowrank[32];  /* of which stored as U^ V^ */
  int64_t n_leaves, n_direct_blocks;
  int64_t near_entries;     /* stored complex entries of the direct near-field blocks */
  int64_t corr_entries;     /* stored complex entries of the correction matrix */
  double bytes_near;        /* algorithmic bytes of the near-field apply per RHS */
  double bytes_s2m_l2t;     /* algorithmic bytes of S2M + L2T per RHS */
  double flops_m2l;         /* algorithmic flops of M2L per RHS */
  double flops_m2m_l2l;     /* algorithmic flops of M2M + L2L per RHS */
  double flops_near;        /* 8 flops per stored complex entry per RHS */
  double device_bytes;      /* device memory held by the plan */
  double setup_ms[8];       /* point selection, SVD of R (Eq. svdr), S~T~, M~, K~, low-rank, corrections,
                               near blocks */
  int64_t launches_per_matvec; /* kernels launched by the last fda_matvec */
  double m2l_flops_lev[32];    /* algorithmic M2L flops per level per RHS */
  double m2l_op_bytes_lev[32]; /* FP64 bytes of the stored M2L operators per level (K~, or U^ and V^) */
} fda_plan_info_t;

int fda_plan_info(const fda_plan_t* plan, fda_plan_info_t* info);

/* Export the correction matrix of Eq. kcorrection for tests (recomputed on the GPU with the plan's
 * kernels, since the plan folds most entries into its direct blocks): for rows[r] (DOF indices, host),
 * fills cnt[r] (host) and, up to cap entries per row, cols[r*cap + q] (DOF index, host) and
 * vals[2*(r*cap + q)] (complex, host) with C_ij = wbar_ij - [j != i] K_H(x_i, y_j) w_j.
 * Synchronous. */
int fda_corrections_export(const fda_plan_t* plan, const int64_t* rows, int64_t nrows, int64_t cap, int64_t* cnt,
                           int64_t* cols, double* vals);

void fda_plan_destroy(fda_plan_t* plan);

/* ------------------------------------------------------------------------------------------ */
/* GMRES on A x = b (Eq. Axb; Sec. 2.2, 5.2).                                                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  double tol;          /* relative residual ||b - A x|| / ||b|| target */
  int restart;         /* Krylov dimension m of GMRES(m) (1..512) */
  int max_iter;        /* total matvec budget */
  int x0_given;        /* 1: x holds the initial guess on entry; 0: x0 = 0 */
  int refine;          /* 1: FP64 iterative refinement around an inner solve with FP32 products (their
                          translations in one TF32 pass, FDA_PREC_TF32); outer residual with the FP64
                          operator, or see refine_residual; 0: plain GMRES */
  int inner_restart;   /* inner Krylov dimension when refine = 1 */
  double inner_tol;    /* inner relative tolerance when refine = 1 */
  int refine_residual; /* refine = 1, plans built with m2l_tensor = 3: 1 = the outer residual with the plan's
                          FP32 product and its 3xTF32 translations (accurate to FP32 rounding, far below the eps
                          of the compressed operator; drop_fp64 plans too); 2 = as 1 until it meets tol, then
                          the residual with the FP64 operator, and FP64 residuals from there on until that
                          one meets tol too (the result is certified against the FP64 operator; plans that
                          keep it); 0 = the FP64 operator throughout */
  int reserved[5];
} bm_gmres_opts_t;

typedef struct {
  int iterations;      /* matvecs in the Krylov loops (inner + outer) */
  int outer_iterations;/* refinement steps (refine = 1) */
  double rel_residual; /* final true relative residual with the outer operator (FP64, or the 3xTF32 FP32
                          product when refine_residual = 1; with refine = 0 the operator of the solve) */
  double ms_total;
  double ms_matvec;
  int status;          /* same as the return code */
  int reserved[5];
} bm_gmres_stats_t;

/* Solve A x = b for nrhs right-hand sides (one Krylov space per column). b, x: DEVICE,
 * N x nrhs complex128, user DOF order. Synchronous (it reads back the Givens residual estimate
 * once per iteration). Returns FDA_E_NOT_CONVERGED / FDA_E_BREAKDOWN / FDA_E_NAN with x holding
 * the best iterate. The refine = 1 form needs a plan built with FDA_PREC_FP32 and uses the
 * plan's FP64 operator for the outer residual. With nrhs > 1 the columns advance in lockstep: every
 * step applies the operator once to the N x nrhs block (nrhs <= the plan's nrhs_max), each column keeps
 * its own Arnoldi basis and Givens rotations, and a column stops extending its basis once its own residual
 * estimate meets tol; stats->iterations then counts block steps and rel_residual is the worst column. */
int bm_gmres_solve(fda_plan_t* plan, const void* b, void* x, int nrhs, const bm_gmres_opts_t* opts,
                   bm_gmres_stats_t* stats, void* stream);

/* Measured FMA throughput of the current device (diagnostic; no paper counterpart): dependent-chain FMA
 * kernels over every SM, reported in TFLOP/s (2 flops per FMA). Synchronous. */
int fda_device_peaks(double* fp64_tflops, double* fp32_tflops);

/* ------------------------------------------------------------------------------------------ */
/* Learned leaf-block preconditioner for flexible GMRES (no paper counterpart; the method's own */
/* GMRES solves supply its training pairs).                                                    */
/* ------------------------------------------------------------------------------------------ */
typedef struct bm_net_s bm_net_t;
typedef struct bm_precond_s bm_precond_t;

/* Network 6 -> hidden -> hidden -> 4 (tanh), FP32 on the device, seeded splitmix64 initialisation; the
 * output layer starts at the identity preconditioner (z = r). 1 <= hidden <= 64. */
int bm_net_create(int hidden, uint64_t seed, bm_net_t** out);
/* Copy the parameters to get_host and/or from set_host (either may be NULL); *nparam = parameter count.
 * Layout: W1 (hidden x 6, row-major), b1, W2 (hidden x hidden), b2, W3 (4 x hidden), b3. Synchronous. */
int bm_net_params(bm_net_t* net, float* get_host, const float* set_host, int* nparam);
void bm_net_destroy(bm_net_t* net);

/* Per-leaf inverses of A_LL = (1/2) I + near-field self block (FP64 Gauss-Jordan, stored FP32) for the
 * plan's leaves of at most 64 points. The plan must outlive the preconditioner. Synchronous. */
int bm_precond_create(fda_plan_t* plan, bm_precond_t** out);
void bm_precond_destroy(bm_precond_t* precond);

/* z = M(r): per point z_i = w1_i r_i + w2_i y_i, y_L = A_LL^-1 r_L, (w1, w2) = net(r_i / s_L, y_i / s_L,
 * mean_L(y) / s_L), s_L the leaf's mean residual. r, z: DEVICE, N complex128, user order. Synchronous. */
int bm_precond_apply(bm_precond_t* precond, bm_net_t* net, const void* r, void* z, void* stream);

/* One training step on npairs residual/correction pairs (r_q, e_q), DEVICE N x npairs complex128 user
 * order: loss = mean_q |M(r_q) - e_q|^2 / |e_q|^2, gradient by the backward kernels, then an Adam update
 * with learning rate lr (lr <= 0: gradient only). *loss and grad_host (nparam floats, may be NULL) report
 * the loss and gradient before the update. Synchronous. */
int bm_precond_train_step(bm_precond_t* precond, bm_net_t* net, const void* r, const void* e, int npairs, double lr,
                          double* loss, float* grad_host, void* stream);

/* Training pair from a GMRES iterate: r = b - A x (FP64 operator) and e = xstar - x. All DEVICE, N
 * complex128, user order; r and e must not alias the inputs. Synchronous. */
int bm_residual_pair(fda_plan_t* plan, const void* b, const void* xstar, const void* x, void* r, void* e,
                     void* stream);

/* Flexible GMRES (right preconditioner M above) with the options and results of bm_gmres_solve. */
int bm_fgmres_solve(fda_plan_t* plan, bm_precond_t* precond, bm_net_t* net, const void* b, void* x, int nrhs,
                    const bm_gmres_opts_t* opts, bm_gmres_stats_t* stats, void* stream);

/* Failure detection (no paper counterpart). Every wait inside the library's kernels (bulk-copy and MMA
 * completion on mbarriers) has a wall-clock bound of 1 s; a wait that gives up records it in the plan's
 * device error flag and the kernel finishes without touching other memory. fda_plan_check synchronizes
 * the device, reads and clears that flag: FDA_OK, or FDA_E_TIMEOUT when some earlier product on this plan
 * had a wait give up (its results are invalid). bm_gmres_solve and bm_fgmres_solve check it before they
 * return. fda_wait_selftest launches one kernel that waits on an mbarrier nothing completes, bounded by
 * limit_ms (0 < limit_ms <= 1000), and reports *timed_out = 1 when the bound ran out (the expected
 * outcome); the context stays usable. */
int fda_plan_check(fda_plan_t* plan);
int fda_wait_selftest(double limit_ms, int* timed_out);

/* Self-test of the tensor-core M2L kernels (diagnostic; no paper counterpart): one complex M x K operator
 * (K <= 1024) applied to P gathered columns, against an FP64 host product of the same FP32 data.
 * split = 0: TF32 with operands expanded in the kernel (M = 64, P = 64); 1: 3xTF32 split (M = 64, P = 64);
 * 2..5: TF32 with the pre-expanded operator image of the m2l_tensor = 1 form (M = min(256, K), P = 100),
 * in its default tile shape (2) or the autotuner's alternatives (3, 4, 5); 6, 7: the same kernel with the
 * bulk-reduction epilogue (default and single-stage shape); 8, 9: the swapped-operand V^ kernel (one and
 * two stages; M = min(100, K), P = 100, results stored as the low-rank intermediate); 10, 11: 3xTF32 from the
 * TF32 and remainder images of the m2l_tensor = 3 form (atomic and bulk-reduction epilogue); 12, 13: the
 * swapped V^ kernel with 16-wide K chunks (two and three in flight).
 * *max_rel_err is the largest entrywise error relative to the sum of |a||x| over the row, *wait_failed is 1
 * when a bounded device wait gave up. Synchronous. */
int fda_tc_selftest(int K, int split, double* max_rel_err, int* wait_failed);

/* Last error message of the calling thread. */
const char* fda_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
