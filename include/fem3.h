/*
 * fem3.h - C ABI of the GB300 (sm_103a) library for the fractional finite element
 * assembly of Yang, Nie, Yuan and Wang, "Finite Element Methods for Fractional PDEs in
 * Three Dimensions" (arXiv 1811.03339).
 *
 * Problem: the Riesz-type operator -sum_i K_i d^{alpha_i} u / d|x_i|^{alpha_i} = f on a
 * convex polyhedron meshed by linear tetrahedra, u = 0 outside the domain.  The
 * Galerkin matrix (Section 2.1, the uniform form (c D^a_i u, D^b_i v) with a = b =
 * alpha_i / 2 and the Riesz constant s_i = 1/(2 cos(pi alpha_i/2))) is
 *
 *     A = sum_i s_i K_i (L_i^T W R_i + R_i^T W L_i),
 *
 * where L_i[g, j] / R_i[g, j] is the left / right Riemann-Liouville derivative of
 * order alpha_i/2 of the P1 basis function of interior vertex j at Gauss point g along
 * axis i, and W = diag(Gauss weights).  The derivatives are summed over the path from
 * the Gauss point to the domain boundary (Section 2.2 path search).
 *
 * Conventions for every call:
 *   - Every call returns an int status: FEM3_OK (0) or a negative FEM3_E_* code.  The
 *     text of the last error of the calling thread is available from fem3_last_error.
 *     No exception crosses this interface.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Work is enqueued on it; results are ready when the stream reaches them.  Errors
 *     found by kernels (walk cap, template miss, non-SPD pivot) are reported by the
 *     next call that synchronises: fem3_sync, fem3_solve (which reads residual norms)
 *     and fem3_mesh_upload.
 *   - Pointers documented as "host or device" are inspected with
 *     cudaPointerGetAttributes; host memory is copied to the device inside the call
 *     (pinned host memory makes the copy asynchronous).  Pointers documented as
 *     "device" must be device (or managed) memory on the current device.
 *   - Dense matrices are row-major; multi-vector arguments are column-major
 *     [rows][nrhs] (column r starts at r * rows).
 *   - The library owns the memory behind a fem3_mesh handle until fem3_mesh_free.
 *     It never frees caller memory.
 */
#ifndef FEM3_H
#define FEM3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FEM3_OK 0
#define FEM3_E_ARG (-1)          /* invalid argument (null, size, range) */
#define FEM3_E_MESH (-2)         /* degenerate tet, non-manifold or non-conforming mesh */
#define FEM3_E_WALK (-3)         /* a path walk exceeded its step cap (no hang) */
#define FEM3_E_NOT_SPD (-4)      /* Cholesky met a non-positive pivot */
#define FEM3_E_NO_CONVERGE (-5)  /* iterative refinement did not reach the tolerance */
#define FEM3_E_CUDA (-6)         /* a CUDA runtime call failed */
#define FEM3_E_OOM (-7)          /* device allocation failed */
#define FEM3_E_STATE (-8)        /* call order violated (e.g. solve before assemble) */
#define FEM3_E_TEMPLATE (-9)     /* a path touched a dof outside its bin's template set */

/* arithmetic of the contraction and of the factorisation */
#define FEM3_FP64 0     /* FP64 tables, FP64 contraction (CUDA cores), FP64 Cholesky */
#define FEM3_TF32X3 1   /* FP64 tables split into TF32 hi/lo, 3 tensor-core products
                           (tcgen05 kind::tf32, FP32 accumulate); FP32 Cholesky;
                           FP64 iterative refinement against the FP64 tables */
#define FEM3_FP32 2     /* FP64 tables rounded to FP32, FP32 contraction (CUDA cores);
                           FP32 Cholesky; FP64 iterative refinement */
#define FEM3_BF16X3 3   /* FP64 tables split into BF16 hi/lo, 3 tensor-core products
                           (tcgen05 kind::f16 with BF16 A/B, FP32 accumulate; about
                           3 * 2^-16 relative per product); FP32 Cholesky; FP64 iterative
                           refinement against the FP64 tables (more sweeps than TF32X3) */

typedef struct fem3_mesh_s *fem3_mesh;

typedef struct fem3_options {
    double bin_scale;  /* transverse bin width in units of the mean cell size h
                          (h = (6 * mean tet volume)^(1/3)); <= 0 selects 0.5 */
    int32_t max_steps; /* cap on tets crossed by one walk; <= 0 selects
                          8 * n_tets^(1/3) + 64 */
    int32_t profile;   /* nonzero: record CUDA events around each stage (fem3_stage_ms) */
    int32_t tc_tile;   /* tile width (columns) of the tensor-core contraction: 128 or 256;
                          0 selects the tuner: the first contraction of a problem size class
                          in the process times both and later ones use the faster */
    int32_t chol_tc;   /* FP32 factorisation of the mixed forms: 0 by size (blocked with
                          tensor-core TF32 x 3 trailing updates from n_dof >= 4096, else the
                          one-launch tile-task factorisation), 1 always blocked, -1 never */
} fem3_options;

/*
 * fem3_mesh_upload - build the device records of a tetrahedral mesh.
 *
 * Section 2.2 ("Assume we have known the adjacent information of the triangulation"):
 * per tet the 4x4 barycentric (volume-coordinate) map, its volume and the four face
 * neighbours (hash matching of sorted face keys); per vertex the list of tets holding
 * it (the m-face star searched on edge and vertex exits); the boundary vertices (on a
 * face without neighbour) and the dof numbering (interior vertices in ascending node
 * order, u = 0 outside the domain, Section 3); the 4-point degree-2 Gauss rule per tet
 * (Section 2.1 quadrature); and, per axis, the transverse bins with their template dof
 * sets (Section 2.3 template matrix, read per axis as overlap of element-patch
 * bounding boxes in the coordinates other than the axis) that lay out the tables.
 *
 *   verts    host or device, float64 [n_nodes][3]; copied.
 *   tets     host or device, int32 [n_tets][4] node ids, any orientation; copied.
 *   opt      host, may be NULL (defaults).
 *   out      host; receives the handle.
 * Requires 4 <= n_nodes < 2^21 and 1 <= n_tets < 2^29.  Synchronises `stream`.
 * Errors: FEM3_E_ARG, FEM3_E_MESH (zero-volume tet, a face shared by > 2 tets),
 * FEM3_E_OOM, FEM3_E_CUDA.
 */
int fem3_mesh_upload(const double *verts, int64_t n_nodes, const int32_t *tets,
                     int64_t n_tets, const fem3_options *opt, void *stream, fem3_mesh *out);

/* Sizes of the mesh.  dof_of_node: host int32 [n_nodes] (dof index or -1), may be NULL.
 * Any output pointer may be NULL. */
int fem3_mesh_info(fem3_mesh m, int64_t *n_dof, int64_t *n_gp, int32_t *dof_of_node);

/*
 * fem3_assemble - path walk, derivative tables and contraction (Sections 2.1-2.3).
 *
 * For every Gauss point g and axis i the left and right paths are walked in FP64
 * across tets (Section 2.2: interval b~ + r d~ >= 0 per tet, exit m-face from the
 * zero pattern of the go-out volume coordinate).  On each segment the left/right
 * Riemann-Liouville derivative of order gamma = alpha_i/2 of every local P1 basis
 * function is added in closed form (integration by parts of eq. "def" on a segment
 * where the basis function is linear):
 *     L_i[g,j] += dphi_j/dx_i * (r_far^(1-gamma) - r_near^(1-gamma)) / Gamma(2-gamma)
 *     R_i[g,j] -= (same with the right path)
 * Then A = sum_i s_i K_i (L_i^T W R_i + R_i^T W L_i), s_i = 1/(2 cos(pi alpha_i/2)).
 *
 *   alpha    host float64[3], each in (1, 2] (alpha = 2 gives the P1 Laplacian).
 *   K        host float64[3], each > 0.
 *   precision  FEM3_FP64, FEM3_TF32X3, FEM3_BF16X3 or FEM3_FP32 (see above).
 *   A_out    device float64 [n_dof][n_dof] or NULL; when given, the assembled matrix
 *            (converted to FP64 for the mixed precisions) is written there.
 * The matrix and its precision stay in the handle for fem3_solve / fem3_adjoint.
 * Errors (FEM3_E_WALK, FEM3_E_TEMPLATE) are reported at the next synchronising call.
 */
int fem3_assemble(fem3_mesh m, const double alpha[3], const double K[3], int precision,
                  double *A_out, void *stream);

/*
 * fem3_assemble_part - one part of the matrix of fem3_assemble, for assembling one mesh
 * over several devices (each device one part, then a sum all-reduce of the parts).
 * The element sum of Section 2.1 is a sum over Gauss points, so the Gauss points of every
 * axis are split by transverse bins: part p of P walks and contracts the bins
 * [nb p / P, nb (p + 1) / P) of each axis (nb the axis's bin count), and the P parts sum to
 * the whole matrix (up to the order of floating-point additions).
 *   alpha, K, precision  as fem3_assemble.
 *   part, nparts         0 <= part < nparts.
 *   A_out    device float64 [n_dof][n_dof]: the part (symmetric, both triangles).
 * The handle then holds no operator for fem3_solve (FEM3_E_STATE until the next
 * fem3_assemble).  Not in the paper.
 */
int fem3_assemble_part(fem3_mesh m, const double alpha[3], const double K[3], int precision,
                       int part, int nparts, double *A_out, void *stream);

/*
 * fem3_assemble_form - one axis term of the general variational form of Section 2.1
 * (eq. "equ:varsss" and the element quadrature formula after it) with a variable
 * coefficient and unequal orders:
 *     K[k][l] = sum_g w_g c(x_g) (D^alpha psi_l)(x_g) (D^^beta psi_k)(x_g)
 * over the interior basis functions, D^alpha the left Riemann-Liouville operator along the
 * axis and D^^beta the right one when trial_left (else the other way round), orders in
 * [0, 1] (order 0: the function itself; order 1: the first derivative, with the one-sided
 * sign: D_L^1 = d/dx, D_R^1 = -d/dx).  The tables of the axis are walked with the two
 * orders (Section 2.2 paths, closed-form derivatives per segment), c multiplies the Gauss
 * weights, and the product runs on the bins of the axis (CUDA cores for FP64 and FP32, the
 * tensor cores for TF32X3 and BF16X3), without the symmetric fold of fem3_assemble.
 *   axis      0, 1 or 2.
 *   c         host or device float64 [n_gp] in Gauss-point order (4 t + q for the q-th
 *             point of tet t), or NULL for c = 1.
 *   K_out     device float64 [n_dof][n_dof] (row: test function k, column: trial l).
 * The call rewrites the axis's tables: the handle then holds no operator for fem3_solve
 * (FEM3_E_STATE until the next fem3_assemble).  Errors: FEM3_E_ARG, FEM3_E_OOM,
 * FEM3_E_CUDA; walk errors at the next synchronising call.
 */
int fem3_assemble_form(fem3_mesh m, int axis, double alpha, double beta, int trial_left,
                       const double *c, int precision, double *K_out, void *stream);

/*
 * fem3_assemble_divergence - Section 3's divergence-form operator (eq. "equ:sfde2"):
 *     a(u, v) = -sum_i ((p_i D_L^{beta_i} u, D_i v) - (q_i D_R^{beta_i} u, D_i v)),
 *     A[k][l] = a(psi_l, psi_k)   (not symmetric),
 * as the sum over the axes of two terms of the general form (fem3_assemble_form with order
 * 1 on the test side: D_L^1 = d/dx_i, D_R^1 = -d/dx_i), accumulated in FP64.
 *   beta     host float64[3], each in [0, 1].
 *   p, q     host or device float64 [3][n_gp]: the coefficients of each axis at the Gauss
 *            points (Gauss-point order as in fem3_assemble_form), positive for the solve.
 *   precision  the products of the terms (FEM3_FP64, FEM3_TF32X3, FEM3_BF16X3, FEM3_FP32);
 *            the operator fem3_solve uses is this matrix itself.
 *   A_out    device float64 [n_dof][n_dof] or NULL.
 * The matrix stays in the handle: fem3_solve then runs restarted GMRES (30 vectors, FP64)
 * right-preconditioned by the FP64 Cholesky factor of -(A + A^T)/2 (SPD for positive p, q;
 * FEM3_E_NOT_SPD otherwise), per column, until ||b - A u|| <= tol ||b|| (max_iter Arnoldi
 * steps, 300 when <= 0); iters_out reports the steps of the slowest column.  No adjoint.
 */
int fem3_assemble_divergence(fem3_mesh m, const double beta[3], const double *p,
                             const double *q, int precision, double *A_out, void *stream);

/*
 * fem3_assemble_integer - the integer-order special case alpha_i = 2 on every axis
 * (the right-hand columns of the paper's Table 4): -sum_i K_i d^2 u/dx_i^2, whose
 * Galerkin matrix is the P1 stiffness matrix
 *     A_jk = sum_i K_i sum_T |T| (d phi_j/dx_i)|_T (d phi_k/dx_i)|_T,
 * assembled tet by tet from the volume-coordinate gradients (no path walk, no tables).
 * fem3_assemble with alpha = (2, 2, 2) gives the same matrix through the walk.
 *   K        host float64[3], each > 0.
 *   A_out    device float64 [n_dof][n_dof] or NULL.
 * The matrix is FP64 and stays in the handle: fem3_solve runs the FP64 form, fem3_adjoint /
 * fem3_vjp take dA/dK_i from the same element formula; fem3_table_rows and
 * fem3_contract_work report FEM3_E_STATE (no tables).
 */
int fem3_assemble_integer(fem3_mesh m, const double K[3], double *A_out, void *stream);

/* Load vector b = M f, M the P1 mass matrix (rows: dofs, columns: all nodes), the
 * weak right-hand side (f, v) of Section 3.
 *   f    host or device float64 column-major [n_nodes][nrhs] (nodal values).
 *   b    device float64 column-major [n_dof][nrhs]. */
int fem3_load(fem3_mesh m, const double *f, int nrhs, double *b, void *stream);

/*
 * fem3_solve - u = A^{-1} M f for the last assembled A.
 *   FP64: FP64 Cholesky and triangular solves.
 *   TF32X3 / BF16X3 / FP32: FP32 Cholesky of the mixed-precision A, then iterative
 *   refinement: d = A32^{-1} r, u += d, r = M f - A u with A u applied from the tables
 *   in double-float FP32 arithmetic (FP64-accurate), until ||r||_2 <= tol ||M f||_2 for
 *   every column or max_iter corrections.  Once every column's residual is below
 *   1e4 tol, a sweep updates r -= A d instead, with A d in plain FP32 (about 1e-6
 *   relative; d is as small as r, so the update's error stays near tol / 100).
 *   f         host or device float64 column-major [n_nodes][nrhs].
 *   u         device float64 column-major [n_dof][nrhs].
 *   iters_out host int or NULL: refinement steps taken (0 for FP64).
 *   resid_out host float64 or NULL: largest final relative residual.
 * Synchronises `stream`.  Errors: FEM3_E_STATE (no matrix), FEM3_E_NOT_SPD,
 * FEM3_E_NO_CONVERGE (u then holds the last iterate), FEM3_E_WALK, FEM3_E_TEMPLATE.
 */
int fem3_solve(fem3_mesh m, const double *f, int nrhs, double tol, int max_iter, double *u,
               int *iters_out, double *resid_out, void *stream);

/*
 * fem3_adjoint - gradient of J = 0.5 ||u - u_obs||^2 with u = A(K)^{-1} M f.
 *   lambda = A^{-1} (u - u_obs)  (same factorisation and refinement as fem3_solve),
 *   dJ/dK_i = -s_i sum_g w_g ((L_i lambda)_g (R_i u)_g + (R_i lambda)_g (L_i u)_g),
 *   dJ/df   = M^T lambda (nodal).
 *   u, u_obs  device float64 [n_dof] (one right-hand side).
 *   dJ_dK     host float64[3].
 *   dJ_df     device float64 [n_nodes] or NULL.
 * Synchronises `stream`.  Not in the paper: the gradient of the discrete solve.
 */
int fem3_adjoint(fem3_mesh m, const double *u, const double *u_obs, double tol, int max_iter,
                 double *dJ_dK, double *dJ_df, void *stream);

/*
 * fem3_vjp - vector-Jacobian product of the solve u = A(K)^{-1} M f (the backward of an
 * autograd function): for an upstream gradient g = dL/du,
 *   lambda = A^{-1} g  (same factorisation and refinement as fem3_solve),
 *   dL/dK_i = -lambda^T (dA/dK_i) u = -s_i sum_g w_g ((L_i lambda)_g (R_i u)_g
 *                                                  + (R_i lambda)_g (L_i u)_g),
 *   dL/df   = M^T lambda (nodal).
 *   u, g    device float64 [n_dof] (one right-hand side; u the solution of the last
 *           fem3_solve of this handle).
 *   dK      host float64[3].   df  device float64 [n_nodes] or NULL.
 * fem3_adjoint is the case g = u - u_obs.  Synchronises `stream`.  Not in the paper.
 */
int fem3_vjp(fem3_mesh m, const double *u, const double *g, double tol, int max_iter,
             double *dK, double *df, void *stream);

/*
 * fem3_paths - export walks for parity checks (Section 2.2).
 *   For each Gauss point gps[l] (device int64 [n_lines]) along `axis` in direction
 *   dir (-1 left, +1 right): tet ids (device int32 [n_lines][cap]), segment ends
 *   r_in / r_out (device float64 [n_lines][cap]) and the segment count (device int32
 *   [n_lines]; -1 if the walk exceeded cap or its step limit).
 */
int fem3_paths(fem3_mesh m, int axis, int dir, const int64_t *gps, int64_t n_lines, int cap,
               int32_t *tet_out, double *r_in_out, double *r_out_out, int32_t *nseg_out,
               void *stream);

/*
 * fem3_table_rows - export rows of the FP64 derivative tables of the last assemble.
 *   rows: device float64 [n][n_dof]; row l = L_axis[gps[l], :] (dir = -1) or
 *   R_axis[gps[l], :] (dir = +1) scattered from the binned storage.
 */
int fem3_table_rows(fem3_mesh m, int axis, int dir, const int64_t *gps, int64_t n,
                    double *rows, void *stream);

/* Synchronise `stream` and report errors recorded by kernels since the last check. */
int fem3_sync(fem3_mesh m, void *stream);

/* Stage timings in milliseconds from the last profiled calls (opt.profile != 0).
 * Stages: 0 mesh geometry, 1 bins/template, 2 walk+tables, 3 contraction,
 * 4 load vector, 5 factorisation, 6 triangular solves + refinement. */
int fem3_stage_ms(fem3_mesh m, int stage, float *ms);

/* Counters: segments walked by the last assemble (all axes, both sides; read by
 * fem3_sync), flops of its contraction counted on the dense bin blocks (sum over bins of
 * 2 * D_b^2 * G_b), bytes of the FP64 tables, and the number of kernels this handle has
 * launched since upload.  Any output pointer may be NULL. */
int fem3_counters(fem3_mesh m, int64_t *segments, double *contract_flops,
                  int64_t *table_bytes, int64_t *launches);

/* Algorithmic flops of the last assemble's contraction (Section 2.1 element sum as sparse
 * outer products): sum over axes and Gauss points g of 2 * 2 * nnz(L_i[g]) * nnz(R_i[g]),
 * counted from the tables' nonzeros (one read of the tables; synchronises `stream`).
 * flops: host float64.  Errors: FEM3_E_ARG, FEM3_E_STATE (no assemble yet). */
int fem3_contract_work(fem3_mesh m, double *flops, void *stream);

/* Nonzeros of the last assemble's derivative tables (Section 2.1 tables, Section 2.3
 * layout), L and R of every axis together: sum over axes and Gauss points g of
 * nnz(L_i[g]) + nnz(R_i[g]); the operator apply A u from the tables takes two
 * multiply-adds per nonzero and vector.  One read of the tables; synchronises `stream`.
 * nnz: host int64.  Errors: FEM3_E_ARG, FEM3_E_STATE (no fractional assemble yet). */
int fem3_table_nnz(fem3_mesh m, int64_t *nnz, void *stream);

/* Kernel classes timed launch by launch when the handle profiles (opt.profile != 0):
 * CUDA events on the launch stream around every launch of the class, summed over the
 * launches since the last fem3_assemble and collected by the next synchronising call
 * (fem3_solve, fem3_sync).  Classes: 0 walk + derivative tables (one launch, three axes),
 * 1 operand split of the tables, 2 contraction GEMMs, 3 Cholesky factorisation,
 * 4 triangular-solve chains, 5 refinement operator apply.  Any output pointer may be NULL. */
int fem3_kernel_ms(fem3_mesh m, int kclass, float *ms, int32_t *launches);

/* Transverse bins of one axis (Section 2.3 template, per axis): number of bins, template
 * rows summed over the bins, and the largest template dof set and Gauss-point count of a
 * bin.  axis in 0..2; any output pointer may be NULL. */
int fem3_bin_stats(fem3_mesh m, int axis, int64_t *n_bins, int64_t *n_tmpl, int32_t *max_dof,
                   int32_t *max_gp);

/* Tile width (128 or 256 columns) of the last tensor-core contraction of this handle, 0 if
 * none, and whether that contraction ran the tuner (1) or used a forced or cached width
 * (0).  Any output pointer may be NULL. */
int fem3_tc_tile(fem3_mesh m, int32_t *tile_n, int32_t *tuned);

/* Which form the refinement's operator apply A u (Section 2.3 tables) takes for this mesh:
 * *lists = 1 from the nonzero lists of the tables (the bins' template rows and Gauss-point
 * sums of 17 vectors fit the list kernel's 112 KB of shared memory and its threads' items),
 * 0 from the dense table blocks of the bins.  Decided by the bins alone, so known once the
 * mesh is uploaded.  lists: host int32.  Errors: FEM3_E_ARG. */
int fem3_apply_lists(fem3_mesh m, int32_t *lists);

/*
 * Batches of meshes (not in the paper, which assembles one mesh at a time).
 *
 * fem3_batch_create - upload n_meshes meshes; arrays as in fem3_mesh_upload, one
 *   pointer and size per mesh (host arrays of pointers to host or device data).
 *   Synchronises `stream`.
 * fem3_batch_mesh - the handle of mesh i (owned by the batch: do not free it); use it
 *   for fem3_mesh_info, fem3_paths or fem3_table_rows.
 * fem3_batch_run - assemble and solve every mesh of the batch (see also the graph note
 *   after the declarations).
 *   One launch walks every Gauss-point line of every mesh (Section 2.2, 2.1 tables);
 *   contraction, load vector and factorisation of each mesh run on internal streams;
 *   each refinement sweep solves all meshes in one batched triangular solve.
 *   alpha, K  host float64 [n_meshes][3].
 *   f         host array of n_meshes device pointers, each column-major [n_nodes_i][nrhs].
 *   u         host array of n_meshes device pointers, each column-major [n_dof_i][nrhs].
 *   nrhs      1..16.  iters, resid: host [n_meshes] or NULL (refinement sweeps and the
 *             largest final relative residual of each mesh; FP64 solves directly).
 *   Synchronises `stream`; work is ordered after earlier work on `stream`.
 *   Errors: as fem3_assemble / fem3_solve, the text names the mesh.
 * fem3_batch_free - release the batch and its meshes.
 */
typedef struct fem3_batch_s *fem3_batch;

int fem3_batch_create(int n_meshes, const double *const *verts, const int64_t *n_nodes,
                      const int32_t *const *tets, const int64_t *n_tets, const fem3_options *opt,
                      void *stream, fem3_batch *out);
int fem3_batch_mesh(fem3_batch b, int i, fem3_mesh *out);
int fem3_batch_run(fem3_batch b, const double *alpha, const double *K, int precision,
                   const double *const *f, int nrhs, double tol, int max_iter, double *const *u,
                   int *iters, double *resid, void *stream);
/* The assembly and factorisation of a run (walk, contractions, load vectors, factorisations:
 * everything before the first refinement sweep) is captured as one CUDA graph by the second
 * run with the same alpha, K, precision, nrhs and f pointers and replayed as one graph launch
 * by later runs with them (the first run goes eagerly; a change of any of them captures
 * again).  The refinement sweeps are host-driven.  fem3_batch_graph_launches reports the
 * graph launches so far, the capturing run's own launch included (host int64). */
int fem3_batch_graph_launches(fem3_batch b, int64_t *n);
void fem3_batch_free(fem3_batch b);

/*
 * fem3_spd_solve_static - solve A x = b for a dense symmetric positive definite matrix
 * without allocating any device memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc where they need a solve
 * (latency-critical loops that must not enter the allocator, host applications or plugin
 * hosts that own every device allocation and hand the library only the problem's
 * buffers).
 *
 *   A       device float64 row-major [n][n], SPD; read only (the lower triangle is used).
 *   b       device float64 [n]; read only.
 *   x       device float64 [n]; receives the solution.
 *   n       1 <= n <= 512; larger systems are rejected with FEM3_E_ARG.
 * A, b and x must be device (or managed) memory of the current device; any other pointer
 * is rejected with FEM3_E_ARG before a kernel runs.
 * Working memory is one static device array of about 2.1 MB (a 512 x 512 FP64 factor,
 * one 64 x 64 block inverse and an error word) that every GPU which loads the library
 * holds until the process exits.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current.  All calls share the
 * array and it keeps the last call's
 * contents: each call clears the error word and rewrites the factor, so calls that
 * overlap on the GPU (other streams, other host threads) race and must be serialised
 * by the caller.  Synchronises `stream`.  Errors: FEM3_E_ARG, FEM3_E_NOT_SPD,
 * FEM3_E_CUDA.
 */
int fem3_spd_solve_static(const double *A, int64_t n, const double *b, double *x,
                          void *stream);

/* Text of the last error of the calling thread. */
int fem3_last_error(char *buf, size_t len);

void fem3_mesh_free(fem3_mesh m);

#ifdef __cplusplus
}
#endif
#endif /* FEM3_H */
