/*
 * lcq.h - C ABI of the GB300 locally corrected quadrature library (liblcq.so).
 *
 * Near-field quadrature corrections for Helmholtz layer potentials on surfaces
 * made of curved triangular patches, after Greengard, O'Neil, Rachh and Vico,
 * "Fast multipole methods for the evaluation of layer potentials with
 * locally-corrected quadratures" (arXiv 2006.02545).
 *
 * Conventions shared by every entry point
 *  - Degrees: a patch of degree d carries n_d = (d+1)(d+2)/2 discretization
 *    nodes (the paper's order p = d+1 with n_p = p(p+1)/2).  1 <= d <= 10.
 *  - Discretization nodes on T0 = {u,v >= 0, u+v <= 1} are the library's
 *    stand-in for the Vioreanu-Rokhlin nodes of Sec. 2.2; lcq_ref_nodes()
 *    returns them so that callers can sample their charts there.
 *  - Pointers documented "device" are CUDA device pointers on the context's
 *    device; pointers documented "host" are ordinary host memory.  The caller
 *    owns every pointer it passes; handles (lcq_ctx, lcq_near, lcq_corr) are
 *    owned by the library and released by the matching _destroy call.
 *  - Complex values are interleaved (re, im) doubles (complex128).
 *  - All device work is queued on the context's stream.  Calls that must size
 *    outputs synchronize that stream: lcq_build_near_lists three times (the grid box,
 *    followed by a read of the status word; the pair count; the per-patch sizes), plus
 *    once more the first time a context meets a patch degree (its tables are uploaded);
 *    a generation on fixed near lists can be replayed without any (lcq_plan).  Errors found
 *    on the device (depth cap, capacity) are latched in a device status word and
 *    returned by lcq_sync() or the next call that synchronizes.
 *  - No call aborts, traps or throws across the ABI; every failure is a status.  A call
 *    that fails part-way releases what it allocated: a creating call leaves its output
 *    handle NULL, and no work buffer of the call stays behind.
 *  - Results are deterministic: fixed orderings, no floating-point atomics.
 */
#ifndef LCQ_H
#define LCQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lcq_ctx lcq_ctx;
typedef struct lcq_near lcq_near;
typedef struct lcq_corr lcq_corr;
typedef struct lcq_plan lcq_plan;

typedef enum {
  LCQ_OK = 0,
  LCQ_ERR_ARG = 1,              /* invalid argument (null pointer, bad size or degree)  */
  LCQ_ERR_NONFINITE = 2,        /* NaN/Inf in node or target coordinates                 */
  LCQ_ERR_DEGENERATE_PATCH = 3, /* Jacobian <= 0 at a node of some patch                 */
  LCQ_ERR_MAX_DEPTH = 4,        /* adaptive refinement reached max_depth (result kept)   */
  LCQ_ERR_CAPACITY = 5,         /* internal work storage too small                       */
  LCQ_ERR_CUDA = 6,             /* CUDA runtime error                                    */
  LCQ_ERR_OOM = 7,              /* device allocation failed                              */
  LCQ_ERR_TABLES = 8,           /* reference tables could not be built                   */
  LCQ_ERR_TIMEOUT = 9           /* lcq_sync gave up waiting                              */
} lcq_status;

/* Layer potential kernels (Sec. 3, Eq. sldef / dldef / urep):
 *   LCQ_S    : G_k(x,y) = e^{ik|x-y|} / (4 pi |x-y|)
 *   LCQ_D    : n(y) . grad_y G_k(x,y)   (n outward)
 *   LCQ_CFIE : alpha D + beta S          (the paper's D - ik S is alpha = 1, beta = -ik)
 *   LCQ_SP   : S' = n(x) . grad_x G_k(x,y), the adjoint double layer of Neumann problems
 *              (Sec. 3).  n(x) is the target's unit normal: for an on-surface target the
 *              chart normal at its node, for an off-surface target the caller's
 *              (lcq_near_set_target_normals); far-order test points use the direction
 *              from the patch centroid.  LCQ_MIXED falls back to FP64 for S'. */
typedef enum { LCQ_S = 0, LCQ_D = 1, LCQ_CFIE = 2, LCQ_SP = 3 } lcq_kernel;

/* LCQ_FP64: every step in FP64 (the contraction of kernel values with basis values on the
 * tensor cores by an exact split of the FP64 operands).
 * LCQ_MIXED: the (target, node) kernel values of the adaptive near integration and of the
 * smooth-rule and annulus moments move to the FP32 pipe, always from the FP64 difference
 * x - X; the chart geometry, self rules, far orders, refinement tests (on the moments),
 * the values-to-coefficients contraction and the apply stay FP64.  By tolerance (per
 * surface in a batch):
 *   eps >= 1e-6          FP32 kernel values (r and the phase k r reduced in FP64),
 *                        contracted from 5 slices; the adaptive test's rounding floor is
 *                        raised to FP32's level; results move by about 1e-7 relative;
 *   1e-6 > eps >= 1e-11  two-float kernel values (pairs of FP32 numbers, about 48 bits),
 *                        contracted like FP64 values; results move by about 1e-14
 *                        relative; needs a real k and a real alpha (else FP64);
 *   eps < 1e-11          FP64.
 * S' always runs FP64.  lcq_counters reports the forms a generation used; the difference
 * from LCQ_FP64 is stated per result by the tests and the benchmark. */
typedef enum { LCQ_FP64 = 0, LCQ_MIXED = 1 } lcq_precision;

/* Surface: n_patches charts; patch j owns nodes node_off[j] .. node_off[j+1]-1,
 * sampled at lcq_ref_nodes(deg[j]) in that order (Sec. 5.2).
 *   deg      host   int32 [n_patches]
 *   node_off host   int64 [n_patches+1], node_off[0] = 0, node_off[j+1]-node_off[j] = n_{deg[j]}
 *   xyz      device double SoA [3][N], N = node_off[n_patches] (x row, then y, then z)
 * Charts must be oriented so that X_u x X_v points out of the body. */
typedef struct {
  int64_t n_patches;
  const int32_t* deg;
  const int64_t* node_off;
  const double* xyz;
} lcq_surface;

/* Parameters (Sec. 4.1-4.3, 5.2).  lcq_params_default() fills the defaults.
 *   eps        requested precision epsilon (> 0)
 *   eta        near-field radius factor; <= 0 selects the paper's default by order
 *              (2.75 for p <= 4, 2 for 4 < p <= 8, 1.25 for p > 8, p = d+1)
 *   eta1       adaptive radius factor (default 1.25); min(eta1, eta) is used
 *   eps_loosen factor on eps in the adaptive termination test (default 1)
 *   max_depth  deepest refinement level (default 24)
 *   m_max      largest smooth rule of the family (m^2 nodes, default 24, <= 32)
 *   self_order Gauss-Legendre order of the self rules (0: from eps)
 *   leaf_order smooth rule used on each subtriangle (0: the patch's far order q_j)
 *   test_dirs  host [n_test_dirs][3] unit vectors for the far-order test points
 *              (NULL: 15-point Fibonacci sphere) */
typedef struct {
  double eps;
  double eta;
  double eta1;
  double eps_loosen;
  int32_t max_depth;
  int32_t m_max;
  int32_t self_order;
  int32_t leaf_order;
  int32_t n_test_dirs;
  const double* test_dirs;
} lcq_params;

void lcq_params_default(lcq_params* p);

/* Context on one CUDA device (a library facility; the paper has no counterpart).
 * cuda_stream may be NULL (legacy default stream) or a cudaStream_t that the caller owns
 * and keeps alive while the context exists.  Allocates the device status word, the
 * per-device constants and the smooth-rule tables; *out receives the context.
 * Errors: LCQ_ERR_ARG (out NULL, device out of range), LCQ_ERR_CUDA, LCQ_ERR_OOM,
 * LCQ_ERR_TABLES; *out stays NULL.
 * lcq_destroy synchronizes the stream and frees everything the context allocated; the
 * near lists, corrections and plans made with it must be destroyed first.  NULL is a
 * no-op. */
lcq_status lcq_create(lcq_ctx** out, int device, void* cuda_stream);
void lcq_destroy(lcq_ctx* ctx);

/* Discretization nodes of degree deg (Sec. 2.1-2.2 stand-in): writes host
 * u[n], v[n] and interpolatory weights w[n], n = (deg+1)(deg+2)/2.  Host only. */
lcq_status lcq_ref_nodes(int deg, double* u, double* v, double* w);

/* Patch geometry and near lists (Sec. 4 N_eta definition; Sec. 5.2).
 *   tgt_xyz  device double SoA [3][NT]
 *   tgt_node device int64 [NT]: global node id of an on-surface target (it is
 *            then excluded from its own patch's near list and gets a self row),
 *            or -1 for an off-surface target.
 * Target t is near patch j iff |x_t - c_j|^2 <= (eta R_j)^2 and t is not on j;
 * it is adaptive iff |x_t - c_j|^2 <= (eta1 R_j)^2.  Synchronizes the stream. */
lcq_status lcq_build_near_lists(lcq_ctx* ctx, const lcq_surface* surf, const double* tgt_xyz,
                                const int64_t* tgt_node, int64_t n_targets,
                                const lcq_params* params, lcq_near** out);

/* Sizes of the near lists of Sec. 4 held by a near-list object: near pairs, self pairs,
 * adaptive pairs (inside N_eta1) and CSR entries, each to a host int64 (NULL skips it).
 * Host only, no synchronization.  LCQ_ERR_ARG for a NULL object. */
lcq_status lcq_near_info(const lcq_near* near, int64_t* n_pairs, int64_t* n_self,
                         int64_t* n_adaptive, int64_t* nnz);

/* Patch-major near lists N_eta(Gamma_j) of Sec. 4 to caller-owned host arrays:
 * pair_ptr[n_patches+1], tgt[n_pairs] (ascending per patch), adaptive[n_pairs] (0/1);
 * per-patch centroid c_j [3*n_patches] and radius R_j [n_patches] (Sec. 4, Eq. rjdef).
 * Any pointer may be NULL to skip it.  Synchronizes the stream; LCQ_ERR_ARG for a NULL
 * object, LCQ_ERR_CUDA if a copy fails. */
lcq_status lcq_near_export(lcq_near* near, int64_t* pair_ptr, int32_t* tgt, uint8_t* adaptive,
                           double* centroid, double* radius);

/* Normals n(x) of the targets for LCQ_SP (Sec. 3, S' = n(x) . grad_x S): device double
 * SoA [3][NT], copied (the caller keeps its buffer); only the off-surface targets'
 * columns are used, normalized by the library.  Required before an S' generation when the
 * near lists have off-surface targets.  LCQ_ERR_ARG for NULL arguments, LCQ_ERR_CUDA or
 * LCQ_ERR_OOM if the copy fails. */
lcq_status lcq_near_set_target_normals(lcq_near* near, const double* tgt_normal);

/* Frees a near-list object (stream-ordered; a library facility with no counterpart in
 * the paper); corrections made from it must be destroyed first.  NULL is a no-op. */
void lcq_near_destroy(lcq_near* near);

/* Net corrections (Sec. 4.2-4.3, 5.2-5.3), stored as a target-major CSR matrix: for
 * every near pair (t, j), c_{t,l} = a^j_l(x_t) - s^j_l(x_t), the quadrature weight
 * minus the weight the smooth rule q_j gives node l; for a self pair (t on patch j),
 * c_{t,l} = a^j_l(x_t), since apply masks the own patch out of the far sum.
 * k = k_re + i k_im (k_im >= 0); alpha, beta are the CFIE coefficients (ignored
 * for S and D). */
lcq_status lcq_gen_corrections(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                               lcq_kernel kernel, double k_re, double k_im, double alpha_re,
                               double alpha_im, double beta_re, double beta_im,
                               lcq_precision precision, const lcq_params* params,
                               lcq_corr** out);

/* ---- Batches of independent surfaces (no counterpart in the paper: many small
 * problems, e.g. a parameter study, generated together so that one launch per stage
 * covers all of them).  The surface lcq_surface is the concatenation of n_surfaces
 * surfaces; surface s owns patches [surface_patch_off[s], surface_patch_off[s+1])
 * (host int64 [n_surfaces+1], starting at 0, ending at n_patches, strictly
 * increasing).  A target is near only to patches of its own surface: an on-surface
 * target belongs to its patch's surface; an off-surface target to tgt_surface[t]
 * (device int32 [NT]; NULL puts every off-surface target in surface 0; a value
 * outside [0, n_surfaces) is LCQ_ERR_ARG).  Everything else is as for
 * lcq_build_near_lists. */
lcq_status lcq_build_near_lists_batched(lcq_ctx* ctx, const lcq_surface* surf, int n_surfaces,
                                        const int64_t* surface_patch_off, const double* tgt_xyz,
                                        const int64_t* tgt_node, const int32_t* tgt_surface,
                                        int64_t n_targets, const lcq_params* params,
                                        lcq_near** out);

/* Physics of one surface of a batch: wavenumber k (Im k >= 0), CFIE coefficients
 * (ignored for S and D) and the tolerance eps that replaces params->eps for it
 * (far order, adaptive tolerance eps * eps_loosen, default self-rule order). */
typedef struct {
  double k_re, k_im;
  double alpha_re, alpha_im;
  double beta_re, beta_im;
  double eps;
} lcq_surface_physics;

/* lcq_gen_corrections (Sec. 4.2-4.3, 5.2-5.3, per surface; the batch is an extension)
 * over near lists built by lcq_build_near_lists_batched, with physics[s] (host
 * [n_surfaces]) for surface s.  One launch per stage and patch
 * degree covers every surface.  The CSR and the apply functions work on the whole
 * batch: the far sum of a target runs over its own surface's sources with that
 * surface's kernel. */
lcq_status lcq_gen_corrections_batched(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                                       lcq_kernel kernel, int n_surfaces,
                                       const lcq_surface_physics* physics, lcq_precision precision,
                                       const lcq_params* params, lcq_corr** out);

/* nnz of the CSR, N_over = sum_j n_{q_j} (Sec. 5.2), value dtype (0 = complex128). */
lcq_status lcq_corr_info(const lcq_corr* corr, int64_t* nnz, int64_t* n_over, int* value_dtype);

/* The correction matrix of Sec. 5.3 (the near and self corrections, CSR by target) out
 * of the library: row_ptr[NT+1], col[nnz] (global node ids), val[2*nnz] (complex128),
 * each into caller-owned host or device memory of the context's device (copied with
 * unified addressing).  Synchronizes the stream.  Any pointer may be NULL.  LCQ_ERR_ARG
 * for a NULL object, LCQ_ERR_CUDA if a copy fails. */
lcq_status lcq_corr_export(lcq_corr* corr, int64_t* row_ptr, int32_t* col, double* val);

/* Per-patch far order q_j (Sec. 4.2, Eq. qj) and annulus order (0: no annulus targets)
 * to caller-owned host [n_patches]; per-near-pair number of accepted leaf triangles of the
 * adaptive integration (Sec. 4.3; 0 for annulus pairs) to host [n_pairs] in patch-major
 * order.  Any pointer may be NULL.  Synchronizes the stream; LCQ_ERR_ARG for a NULL
 * object, LCQ_ERR_CUDA if a copy fails. */
lcq_status lcq_corr_export_stats(lcq_corr* corr, int32_t* q, int32_t* q_near, int32_t* leaves);

/* Corrected layer potential (Sec. 5.3, subtract-and-add with a direct far sum; the
 * own patch of an on-surface target is masked out of the far sum):
 *   u(x_t) = sum_{j != own(t)} sum_{q in rule q_j} K(x_t, X_j(u_q)) J w_q sigma~_q
 *            + sum_row c sigma
 * sigma device complex128 [N] at the nodes, out device complex128 [NT].
 * jump != 0 adds jump * sigma(x_t) for on-surface targets (e.g. 0.5 for the
 * exterior limit of D).  The kernel must match the one the corrections were
 * generated for. */
lcq_status lcq_apply_corrected_S(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                                 const lcq_corr* corr, const double* sigma, double jump,
                                 double* out);
lcq_status lcq_apply_corrected_D(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                                 const lcq_corr* corr, const double* sigma, double jump,
                                 double* out);
lcq_status lcq_apply_corrected_CFIE(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                                    const lcq_corr* corr, const double* sigma, double jump,
                                    double* out);
lcq_status lcq_apply_corrected_Sp(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                                  const lcq_corr* corr, const double* sigma, double jump,
                                  double* out);

/* ---- Adjoint (no counterpart in the paper).  For a real functional L of the
 * corrected potential u = A(y) sigma with upstream gradient g = dL/d(conj u)
 * (device complex128 [NT]; PyTorch's convention, dL = Re sum_t conj(g_t) du_t):
 *
 * lcq_apply_adjoint: out = A^H g (device complex128 [N]), the density gradient, for the
 * operator of lcq_apply_corrected_* with the same jump (the far sum transposed per
 * source, the CSR transposed patch by patch: deterministic, no atomics).
 *
 * lcq_shape_gradient: out = dL/dy (device double SoA [3][N]) with respect to the node
 * coordinates, for the density sigma (device complex128 [N]), differentiating the
 * discrete method with every discrete choice frozen: near lists, far orders q_j,
 * annulus orders and refinement trees.  Each (target, patch) pair contributes through
 * the one rule that defines it (q_j, the annulus rule, or the accepted leaves); the
 * trees are recomputed by the adaptive kernel in gradient mode, not stored.  Targets
 * must be off the surface (a near list with self pairs is LCQ_ERR_ARG): on-surface
 * targets move with the nodes and use the self rules, which this does not cover. */
lcq_status lcq_apply_adjoint(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                             const lcq_corr* corr, const double* g, double jump, double* out);
lcq_status lcq_shape_gradient(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                              const lcq_corr* corr, const double* sigma, const double* g,
                              double* out);

/* The corrected potential of Sec. 5.3 as lcq_apply_corrected_S/D/CFIE/Sp, chosen by
 * kernel, for a density in either precision:
 * sigma_dtype 0 = complex128, 1 = complex64 (widened to complex128 on the device before
 * the FP64 sums).  out is complex128 [NT].  The kernel must match the corrections'. */
lcq_status lcq_apply_corrected(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                               const lcq_corr* corr, lcq_kernel kernel, const void* sigma,
                               int sigma_dtype, double jump, double* out);

/* Frees a correction object (stream-ordered; a library facility with no counterpart in
 * the paper); plans made on it must be destroyed first.  NULL is a no-op. */
void lcq_corr_destroy(lcq_corr* corr);

/* Captured regeneration (an extension: the paper has no counterpart).  lcq_plan_create
 * records, as one CUDA graph, the device work that regenerates corr in place from the
 * current contents of surf->xyz: the positions of the on-surface targets (their nodes),
 * the chart geometry of every patch (Sec. 3.2, Sec. 4; and for S' the target normals), then the far orders, the smooth, annulus and adaptive
 * moments, the self weights and the V contraction (Sec. 4.2-4.3, 5.3) with the kernel,
 * tolerance, precision, test directions and adaptive work-group sizes of corr's
 * generation.  lcq_plan_launch replays it on ctx's stream: no host synchronization and no
 * allocation, a few launches' worth of CPU time.  The near lists (pairs, adaptive flags,
 * CSR layout) are not rebuilt: between launches the caller may move the nodes (write new
 * coordinates into surf->xyz on the stream) only as far as the lists stay those of the
 * moved surface, as for lcq_shape_gradient.  Results equal those of lcq_gen_corrections on
 * the same coordinates and lists bit for bit.  lcq_stage_times are not recorded by a
 * launch; lcq_counters are.  The plan owns its work buffers (about the generation's
 * transient memory); ctx, near, corr and surf->xyz must outlive it.
 * Errors: LCQ_ERR_ARG when corr does not belong to near and surf, LCQ_ERR_CUDA when the
 * capture or instantiation fails (nothing is left allocated). */
lcq_status lcq_plan_create(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                           lcq_corr* corr, lcq_plan** out);
lcq_status lcq_plan_launch(lcq_plan* plan);
void lcq_plan_destroy(lcq_plan* plan);

/* Wait for the context's stream (a library facility; the paper has no counterpart):
 * polling, at most timeout_ms (< 0 waits without limit), then return and clear the
 * latched device status: LCQ_ERR_NONFINITE, LCQ_ERR_DEGENERATE_PATCH, LCQ_ERR_CAPACITY or
 * LCQ_ERR_MAX_DEPTH (results kept) as the device reported them, else LCQ_OK.  A wait that
 * runs out returns LCQ_ERR_TIMEOUT and leaves the work in flight and the status word
 * untouched, so a later call completes it.  LCQ_ERR_ARG for a NULL context, LCQ_ERR_CUDA
 * if the stream reports an error. */
lcq_status lcq_sync(lcq_ctx* ctx, int64_t timeout_ms);

/* Device-side work counters of the last lcq_gen_corrections on ctx (a measurement
 * facility with no counterpart in the paper; [1] is the evaluation count behind the
 * adaptive kernel's algorithmic FLOP rate), to caller-owned host out8[8]:
 * [0] adaptive tests, [1] adaptive leaf-rule node evaluations (target x node),
 * [2] self node evaluations, [3] smooth/annulus node evaluations (target x node),
 * [4] union-tree nodes walked by the adaptive kernel (each evaluates the chart geometry
 * at 4Q leaf nodes), [5] the largest number of adaptive targets per work item (the
 * group size the context's tuner chose), [6] adaptive work items, [7] the pair
 * evaluation forms the generation used, a bit mask (1: FP32, 2: two-float; 0: FP64 only;
 * see lcq_precision).  Synchronizes.
 * The adaptive walk takes its work in items of at most a group size of targets of one
 * patch; an online tuner in the context times each candidate size once per key (degree,
 * kernel, tolerance decade, precision, size of the adaptive work) on the generations that
 * use it and keeps the fastest; with at least 16 patches of adaptive targets per resident
 * block it takes whole patches without timing.  Every result is the same for every group
 * size. */
lcq_status lcq_counters(lcq_ctx* ctx, int64_t* out8);

/* Stage timings of the last lcq_build_near_lists and lcq_gen_corrections on ctx (a
 * measurement facility with no counterpart in the paper), from CUDA events recorded on the
 * streams that run them, to caller-owned host ms6[6] (milliseconds; NULL skips them):
 *   ms[0] near lists (geometry + both orientations)   ms[1] far order q_j
 *   ms[2] smooth-rule and annulus moments              ms[3] adaptive near moments
 *   ms[4] self weights (on an internal low-priority stream, concurrently with ms[1]-ms[3];
 *         the chain ms[1]-ms[3], ms[5] runs on an internal high-priority stream, forked
 *         from and joined back into the context's stream)
 *   ms[5] V contraction into the CSR
 * *launches receives the number of kernels those two calls launched.  Synchronizes. */
lcq_status lcq_stage_times(lcq_ctx* ctx, float* ms6, int64_t* launches);

/* Allocation-free variant for callers that cannot allocate device memory: code that
 * runs where cudaMalloc is unavailable or forbidden (inside a host callback or a
 * real-time loop that must not touch the allocator, or under a memory manager that owns
 * every byte of the device).  The paper has no counterpart; this is a library facility.
 *
 * Computes the adaptive near corrections of ONE patch for targets that are all treated
 * as adaptive, exactly as lcq_gen_corrections computes them for adaptive near pairs: out[t][l] = sum_nm V[nm][l] (I^adaptive_nm(x_t) - I^{rule q}_nm(x_t)).
 *   deg       patch degree, 1..8
 *   y         device double SoA [3][n] node coordinates, n = (deg+1)(deg+2)/2
 *   n_targets 1..128; tgt_xyz device double SoA [3][n_targets] (off-surface points)
 *   kernel, k, alpha, beta as for lcq_gen_corrections
 *   q         leaf / smooth rule order (the patch's far order q_j), 1..32
 *   eps       adaptive tolerance; max_depth 1..16
 *   out       device complex128 [n_targets][n] (interleaved re, im), caller-owned
 * All device storage (tables, geometry, moments, the union-tree workspace) lives in one
 * static 8 MiB device array that every GPU loading liblcq holds until process exit; no
 * call allocates or frees device memory.  The first call on a device, with that device
 * current, looks up the array's device address and uploads constant tables.  No call may
 * be made while cuda_stream is being captured (each copies host values and synchronizes
 * the stream): such a call returns LCQ_ERR_ARG and queues nothing.  Calls share the array
 * and keep the previous call's contents (each call rewrites what it reads): calls that
 * overlap on the GPU --
 * on different streams or from different threads -- race and must be serialized by the
 * caller.  Host-side set-up is safe when several host threads make their first calls at
 * once.  The call queues its work on cuda_stream (NULL: legacy default stream) and
 * synchronizes that stream before returning.  Returns LCQ_ERR_CAPACITY when deg,
 * n_targets or max_depth exceed the limits above, LCQ_ERR_MAX_DEPTH (result kept) or
 * LCQ_ERR_NONFINITE as lcq_gen_corrections does. */
lcq_status lcq_adaptive_corrections_noalloc(int deg, const double* y, int64_t n_targets,
                                            const double* tgt_xyz, lcq_kernel kernel,
                                            double k_re, double k_im, double alpha_re,
                                            double alpha_im, double beta_re, double beta_im,
                                            int q, double eps, int max_depth, void* cuda_stream,
                                            double* out);

/* Pipe-throughput microbenchmarks on `device` (no counterpart in the paper; the measured
 * denominators of the roofline fractions the benchmark reports).  Writes host out[n_out],
 * up to 8 values, each a rate measured by CUDA events over about 20 ms of one kernel that
 * keeps every SM busy with independent dependency chains:
 *   [0] FP64 FMA, TFLOP/s              [1] FP32 FMA, TFLOP/s
 *   [2] special-function unit (sin.approx.f32), 10^12 results/s
 *   [3] INT32 xor + add, 10^12 operations/s
 *   [4] mma.sync m8n8k4 f64, TFLOP/s   [5] mma.sync m16n8k16 f16 -> f32, TFLOP/s
 *   [6] mma.sync m16n8k16 bf16 -> f32, TFLOP/s   [7] mma.sync m16n8k8 tf32 -> f32, TFLOP/s
 * Allocates 32 KB of device memory and a private stream for the duration of the call;
 * takes about a second; LCQ_ERR_ARG for a null out or n_out < 1, LCQ_ERR_CUDA on any
 * CUDA failure (entries that were measured are kept). */
lcq_status lcq_pipe_peaks(int device, double* out, int n_out);

/* Device self-checks of the adaptive kernel's arithmetic (no counterpart in the paper).
 * Writes host out[n_out], up to 5 values (-1 where not measured):
 *   [0] max |sin - sin_ref|, |cos - cos_ref| of the table-driven sincos against CUDA's
 *       sincos over 4M arguments in [-3000, 3000] and around the table's breakpoints;
 *   [1] degree 6 and [2] degree 10: max over every output of |tensor-core contraction -
 *       FP64 contraction| / sum_q |a_q| |b_q| for random kernel-like rows (12 decades of
 *       magnitude, random phases) and basis-like columns at their bounds;
 *   [3] max |two-float kernel value - FP64 kernel value| relative to the sum of the
 *       magnitudes of its terms, S, D and CFIE at k = 1.3, 2 pi, 20, 2M near-singular and
 *       tangent-plane configurations (the mixed form below eps = 1e-6);
 *   [4] max |two-float sin, cos - CUDA's| / (1 + |th|) over |th| < 3000.
 * Allocates 64 bytes of device memory and a private stream for the call; LCQ_ERR_ARG for a
 * null out or n_out < 1, LCQ_ERR_CUDA on any CUDA failure. */
lcq_status lcq_selftest(int device, double* out, int n_out);

const char* lcq_status_string(lcq_status s);
const char* lcq_last_error(const lcq_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LCQ_H */
