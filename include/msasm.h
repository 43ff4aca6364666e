/*
 * msasm.h -- multiscale lookup-table stiffness assembly on one GB300 (sm_103a).
 *
 * C ABI of the data-parallel hot path of "Fast and Multiscale Formation of
 * Isogeometric Matrices of Microstructured Geometric Models" (Hirschler, Antolin,
 * Buffa; arXiv 2107.09568):
 *
 *   (step 2)  build the stiffness lookup table mat[K] of the reference tile
 *             (Sec. 3.2.3, eq. 51-52, 56-57)                -> msasm_build_tables
 *   (step 1)  pull back the elasticity tensor through each macro element and
 *             interpolate it at the (q+1)^3 nodes, or (q1+1)(q2+1)(q3+1) with a degree per
 *             direction (eq. 37, 42, 79-97)
 *   (step 3)  contract the table with the coefficients, one GEMM (eq. 58)
 *   (step 4)  add the tile blocks into a global CSR matrix (Sec. 3.2.4)
 *                                                           -> msasm_assemble
 *   compliance sensitivity u^T (dK/dP) u (Sec. 4.1.2, eq. 69-73) -> msasm_assemble_grad
 *
 * Conventions shared by every call:
 *  - Every function returns an msasm_status; none aborts, exits or traps.  On an
 *    error, msasm_last_error() returns a thread-local message.
 *  - Pointers named d_* are device pointers on the current CUDA device, owned by
 *    the caller; pointers named h_* (and descriptor arrays) are host memory, read
 *    only during the call.  Opaque handles own library-allocated device memory
 *    and are released by the matching *_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is queued on it and the call returns without synchronising, except
 *    where a call is documented to read a result back to the host.
 *  - A plan holds scratch (coefficients, nzdata, slices) that its calls reuse, so
 *    one plan serves one stream at a time.  Tables make their sliced copies for a
 *    precision form at the first call that needs them; after that they are only
 *    read and may be shared by plans on different streams.
 *  - Tile t = (ix, iy, iz) of an nx x ny x nz macro mesh has linear index
 *    ix + nx*(iy + ny*iz).  Interpolation node C = c1 + (q+1)*(c2 + (q+1)*c3)
 *    with the q+1 Gauss-Legendre points of [0,1] ascending per direction.
 *  - Table layout: T[m][C][i][j] (row m = pair (A,B) of eq. 56 in lexicographic
 *    order, A <= B, local ids of the reference tile), i.e. mat[K] of eq. 57 with
 *    column k = 9*C + 3*i + j.
 *  - Coefficient layout (mat[<A>] of eq. 58, stored transposed): coef[n][k] with
 *    n = 9*t + 3*alpha + beta and k = 9*C + 3*i + j, value A_ij(xi_C)[alpha][beta].
 *  - nzdata layout (eq. 58, the tile matrices K_t block by block): nz[t][m][3*alpha + beta],
 *    the 3x3 block of pair m = (A,B) of tile t, value K_t[(A,alpha),(B,beta)], at
 *    9*(t*n_nz + m) + 3*alpha + beta; the block of (B,A) is its transpose and is not stored.
 *  - Global stiffness: DOF 3*g + alpha of global control point g; CSR with int64
 *    row pointer, int32 ascending column indices, full symmetric storage.
 */
#ifndef MSASM_H
#define MSASM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MSASM_OK = 0,
  MSASM_EINVAL = -1,        /* null pointer, bad size, unsupported degree/shape */
  MSASM_ECUDA = -2,         /* a CUDA runtime/driver call failed */
  MSASM_ENOMEM = -3,        /* device or host allocation failed */
  MSASM_EDEGENERATE = -4,   /* |det J| <= tol at some node: degenerate macro element (Sec. 3.3.4) */
  MSASM_EUNSUPPORTED = -5,  /* precision/feature not available for this shape */
  MSASM_EIO = -6            /* a file cannot be opened, read or written, or is not a valid file of its kind */
} msasm_status;

typedef enum {
  MSASM_F64 = 0,            /* FP64 contraction (CUDA-core DFMA) */
  MSASM_F32 = 1,            /* tensor cores, FP32 values: each operand row cut into 4 exact BF16 slices (28
                               bits), the 10 slice products with i+j <= 3 summed exactly, one rounding to
                               FP32 (CUDA-core FFMA for tables with 9 n_pi > 576) */
  MSASM_SPLIT_F16 = 2,      /* tensor cores, FP16 hi/lo operands, FP32 accumulation, FP32 values */
  MSASM_SPLIT_BF16 = 3,     /* tensor cores, BF16 hi/lo operands, FP32 accumulation, FP32 values */
  MSASM_TF32 = 4,           /* tensor cores, TF32 operands, FP32 accumulation, FP32 values */
  MSASM_TF32X3 = 5,         /* tensor cores, TF32 hi/lo (3 products), FP32 values */
  MSASM_F64_EMU = 6         /* tensor cores, FP64 emulated by exact BF16 slices, FP64 values */
} msasm_precision;

/* flags for msasm_assemble */
#define MSASM_FLAG_CHECK_DEGENERATE 1u  /* synchronise `stream` and fail with EDEGENERATE if any |det J| <= tol */
#define MSASM_FLAG_STAGE_TIMES 2u       /* record CUDA events around each stage on `stream` (msasm_stage_times) */

/* Reference tile T^r (eq. 3): axis-aligned box patches in [0,1]^3, each an
 * open-uniform B-spline with its control points at the Greville abscissae
 * (an affine patch map).  Patches are glued by coincident control points.
 * Arrays are host memory of length 3*n_patches, patch-major.  Neighbouring tiles
 * are glued through the points on the faces xi_d = 0, 1; a control point on faces
 * of two directions (an edge or corner of [0,1]^3, shared by more than two tiles)
 * is not supported: msasm_build_tables returns MSASM_EUNSUPPORTED. */
typedef struct {
  int32_t n_patches;
  const int32_t* degree;    /* per patch and direction, 1..4 */
  const int32_t* n_elem;    /* per patch and direction, >= 1 */
  const double* box_lo;     /* box lower corner */
  const double* box_hi;     /* box upper corner */
} msasm_micro_desc;

/* Macro B-spline map M (eq. 4): degrees and open knot vectors (host memory).
 * The control net is passed to each assemble call because it changes during
 * shape optimisation: d_ctrl[(i + n1*(j + n2*k))*3 + p], n_d = n_knots[d]-degree[d]-1. */
typedef struct {
  int32_t degree[3];        /* 1..5 */
  int32_t n_knots[3];
  const double* knots[3];   /* non-decreasing, open (first/last value repeated degree+1 times) */
} msasm_macro_desc;

typedef struct msasm_tables msasm_tables;   /* opaque: tile topology + table in device memory */
typedef struct msasm_plan msasm_plan;       /* opaque: macro mesh, numbering, CSR pattern, scratch */

/* ---------------------------------------------------------------- tables (step 2) */

/* Build mat[K] (eq. 52, 57) in FP64 on the GPU for interpolation degree q (0..5),
 * using n_gauss points per direction per micro element (<= 0: exact rule
 * ceil((2 p_T + q + 1)/2)).  Synchronises `stream` before returning.
 * Errors: EINVAL (bad descriptor, q out of range), ENOMEM, ECUDA. */
msasm_status msasm_build_tables(const msasm_micro_desc* micro, int32_t q, int32_t n_gauss,
                                void* stream, msasm_tables** out);

/* The same with a projection degree per direction, q3 = (q1, q2, q3) (host int32[3], each 0..5):
 * the anisotropic space Q_(q1,q2,q3) of Sec. 3.3.4 (e.g. a higher degree along a twist), n_pi =
 * (q1+1)(q2+1)(q3+1) nodes C = c1 + (q1+1)(c2 + (q2+1) c3) at each direction's Gauss-Legendre
 * points.  Every call that takes these tables uses that space (the FP64-accurate tensor-core
 * contraction needs 9 n_pi <= 576). */
msasm_status msasm_build_tables_q3(const msasm_micro_desc* micro, const int32_t* q3, int32_t n_gauss,
                                   void* stream, msasm_tables** out);

/* The tables' degree per direction into q3 (host int32[3]). */
msasm_status msasm_tables_degrees(const msasm_tables* tab, int32_t* q3);

/* Sizes of a table: n_T control points, n_nz pairs (eq. 56), n_pi = (q1+1)(q2+1)(q3+1). */
msasm_status msasm_tables_info(const msasm_tables* tab, int32_t* n_T, int32_t* n_nz, int32_t* n_pi);

/* Copy the FP64 table (n_nz * 9 * n_pi values, layout above) to d_table, and the
 * pair list (2*n_nz int32, A then B per row) to h_pairs if non-NULL (host). */
msasm_status msasm_tables_copy(const msasm_tables* tab, double* d_table, int32_t* h_pairs, void* stream);

void msasm_tables_destroy(msasm_tables* tab);

/* Store the tables of a reference tile in a file and read them back (Sec. 3.1.1, 3.2.3: the
 * lookup tables of a microstructure are computed once and kept, and an assembly only reads
 * them).  The file holds the micro descriptor, the projection degrees and every FP64 table
 * (stiffness eq. 57, load eq. 55, volume eq. 18, faces eq. 55 with F >= 1), followed by a 64-bit
 * FNV-1a checksum; numbers are little-endian.  msasm_tables_load rebuilds the tile topology
 * from the stored descriptor, checks that it gives the stored sizes, and uploads the tables
 * without recomputing them: every call then behaves bit for bit as with the saved object.
 * Both synchronise `stream`.  Errors: EINVAL (NULL argument), EIO (the file cannot be opened,
 * read or written, has another kind tag, format version or byte order, is truncated, fails its
 * checksum, or describes a tile whose topology does not match its sizes), ENOMEM, ECUDA. */
msasm_status msasm_tables_save(const msasm_tables* tab, const char* path, void* stream);
msasm_status msasm_tables_load(const char* path, void* stream, msasm_tables** out);

/* ---------------------------------------------------------------- plan (integer work, once per mesh) */

/* Number the global control points of the tiled structure and build the CSR pattern of the
 * stiffness: the union over tiles of the pairs of eq. 56 (two control points interact when they
 * share a micro element of a tile; the pattern is the sparse structure of K that Sec. 3.2.4's
 * step 4 fills), the per-(tile, pair) index map of each tile block into it, and allocate scratch for
 * `max_tiles_per_pass` tiles (<= 0: all tiles in one pass).  The plan keeps a
 * reference to `tab`, which must outlive it.  Writes n_rows = 3 * n_points and
 * nnz (host).  Synchronises `stream`.  Errors: EINVAL, ENOMEM, ECUDA. */
msasm_status msasm_plan_create(const msasm_tables* tab, const msasm_macro_desc* macro,
                               int32_t max_tiles_per_pass, void* stream, msasm_plan** out,
                               int64_t* n_rows, int64_t* nnz);

/* Sizes: tiles, global points, rows, nnz, control points of the macro net. */
msasm_status msasm_plan_info(const msasm_plan* plan, int64_t* n_tiles, int64_t* n_points,
                             int64_t* n_rows, int64_t* nnz, int64_t* n_ctrl);

/* Copy the CSR pattern of eq. 56 (every (A, B) pair of every tile, in global numbering, with full
 * symmetric storage): d_rowptr (n_rows+1 int64) and d_col (nnz int32, ascending within a row). */
msasm_status msasm_plan_csr(const msasm_plan* plan, int64_t* d_rowptr, int32_t* d_col, void* stream);

/* Copy the global numbering gmap[t][A] (n_tiles * n_T int32) to d_gmap. */
msasm_status msasm_plan_numbering(const msasm_plan* plan, int32_t* d_gmap, void* stream);

void msasm_plan_destroy(msasm_plan* plan);

/* ---------------------------------------------------------------- assembly (steps 1, 3, 4) */

/* K = sum over tiles of the lookup-form tile matrices (eq. 50, 58) scattered into
 * the CSR pattern of the plan.  d_ctrl: macro control net (n_ctrl*3 FP64).
 * E, nu: isotropic material (Lame constants as in eq. 84).  d_values: nnz values,
 * FP64 for MSASM_F64 / MSASM_F64_EMU, FP32 otherwise; overwritten.  The
 * Jacobian, its determinant and inverse are FP64 in every precision.
 * Errors: EINVAL, EUNSUPPORTED, ECUDA; EDEGENERATE only with
 * MSASM_FLAG_CHECK_DEGENERATE (otherwise degenerate nodes are counted, see
 * msasm_degenerate_count, and the values are still written). */
msasm_status msasm_assemble(msasm_plan* plan, const double* d_ctrl, double E, double nu,
                            msasm_precision prec, void* d_values, uint32_t flags, void* stream);

/* Same as msasm_assemble but with host buffers: h_ctrl (n_ctrl*3 FP64) is copied
 * to the device and the nnz values are copied back into h_values (FP64 or FP32
 * as above) before the call returns (it synchronises `stream`).  Pinned host
 * memory gives full copy bandwidth. */
msasm_status msasm_assemble_host(msasm_plan* plan, const double* h_ctrl, double E, double nu,
                                 msasm_precision prec, void* h_values, uint32_t flags, void* stream);

/* Gradient of L with respect to the macro control net (Sec. 4.1.2, eq. 69-73), through the
 * lookup form of msasm_assemble.  Give exactly one of
 *   d_u           (n_rows values): L = u^T K u, the internal-work term of eq. 69-70
 *                 (with f fixed and u = K^-1 f the compliance gradient is -dL/dP);
 *   d_grad_values (nnz values): dL/dvalues of an arbitrary L (the chain through step 4).
 * Both are FP64 for MSASM_F64 / MSASM_F64_EMU and FP32 otherwise.  The contraction of the
 * table with u (W = mat[K]^T G, eq. 73) runs in FP64 on the CUDA cores (MSASM_F64), as
 * sliced BF16 products on the tensor cores in chunks of 576 pairs summed in FP64
 * (MSASM_F64_EMU: each row of G is kept to 49 bits of its largest entry, about 1e-11
 * relative on a bending state), or in FP32 (other precisions); the chain rule through
 * |det J| and J^-1 to the control points is FP64.
 * d_grad_ctrl (n_ctrl*3 FP64) is overwritten.  Errors: EINVAL, EUNSUPPORTED, ECUDA. */
msasm_status msasm_assemble_grad(msasm_plan* plan, const double* d_ctrl, double E, double nu,
                                 msasm_precision prec, const void* d_u, const void* d_grad_values,
                                 double* d_grad_ctrl, void* stream);

/* ---------------------------------------------------------------- one mesh across GPUs (tile ranges)
 *
 * The tile matrices of eq. 58 are independent per tile, and the tile-major numbering makes the
 * rows owned by a contiguous tile range [t0, t1) one contiguous range of rows and of CSR values.
 * A rank assembles the complete rows its tiles own by also recomputing the halo: the tiles of
 * the next layer above the range (up to t1 + nx*ny), whose blocks on their glued lower faces
 * land in those rows.  No data moves between ranks for the assembly; the gradient of a range is
 * a partial sum, added across ranks by one all-reduce (the caller's). */

/* The rows [*row0, *row1) and CSR values [*v0, *v1) owned by tiles [t0, t1) (0 <= t0 <= t1 <=
 * n_tiles), and the end of the tiles that reach them (*halo_end: t1 plus the next layer, at most
 * n_tiles).  Any output may be NULL.  Host only.  Errors: EINVAL. */
msasm_status msasm_plan_range(const msasm_plan* plan, int64_t t0, int64_t t1, int64_t* row0, int64_t* row1,
                              int64_t* v0, int64_t* v1, int64_t* halo_end);

/* msasm_assemble for the rows owned by tiles [t0, t1): d_values holds the values [v0, v1) of
 * msasm_plan_range (its first element is value v0), and receives exactly the values a whole-mesh
 * msasm_assemble writes there (bit for bit: the same kernels, the same sums).  Tiles [t0,
 * halo_end) are computed; the blocks of tiles outside [t0, t1) are written only where they land
 * in the window.  t0 == t1 does nothing.  Errors: as msasm_assemble. */
msasm_status msasm_assemble_range(msasm_plan* plan, const double* d_ctrl, double E, double nu,
                                  msasm_precision prec, int64_t t0, int64_t t1, void* d_values, uint32_t flags,
                                  void* stream);

/* msasm_assemble_grad restricted to the tiles [t0, t1): d_grad_ctrl (n_ctrl*3, overwritten) gets
 * the part of dL/dP that those tiles' blocks contribute (eq. 69-73 summed over the range); the
 * sum over a partition of the tiles is the whole gradient.  d_u (n_rows) or d_grad_values (nnz)
 * are the whole-mesh arrays, as in msasm_assemble_grad.  Errors: as msasm_assemble_grad. */
msasm_status msasm_assemble_grad_range(msasm_plan* plan, const double* d_ctrl, double E, double nu,
                                       msasm_precision prec, int64_t t0, int64_t t1, const void* d_u,
                                       const void* d_grad_values, double* d_grad_ctrl, void* stream);

/* Global control points on macro face `face` = 2 d + s (the face xi_d = s of the macro
 * parameter cube), ascending, into h_points (host; *count in: capacity, out: number).
 * With h_points NULL only the count is returned. */
msasm_status msasm_face_points(const msasm_plan* plan, int32_t face, int32_t* h_points, int64_t* count);

/* Load vector of a uniform traction t (force per unit physical area, host double[3]) on
 * macro face `face`: f_{3g+c} = t_c int_Gamma R_g dGamma (eq. 29, 33), by Gauss quadrature on
 * the micro patch faces lying on the face, for the control net h_ctrl (host, n_ctrl*3).
 * h_f: n_rows doubles (host), overwritten.  Runs on the host (set-up data). */
msasm_status msasm_traction_load(const msasm_plan* plan, int32_t face, const double* traction,
                                 const double* h_ctrl, double* h_f);

/* ---------------------------------------------------------------- learned surrogate (graded lattices) */

/* A surrogate of the lookup table for a family of reference tiles with one parameter w
 * (the strut width): T(w) ~ U V(w)^T, U (n_nz x r, orthonormal columns) fitted once, V(w)
 * (9 n_pi x r) predicted by an MLP.  Not in the paper: an interface addition for graded
 * lattices, where the paper's method needs one quadrature table per distinct tile. */
typedef struct msasm_mlp msasm_mlp;               /* opaque: 1 -> H -> H -> n_out tanh MLP */
typedef struct msasm_surrogate msasm_surrogate;   /* opaque: basis U + MLP + target scaling */

/* MLP with FP16 weights (FP32 master copy and Adam state), FP32 accumulation; Glorot-uniform
 * weights from `seed`, zero biases.  Parameter vector layout (FP32, n_params values):
 * W1[H], b1[H], W2[H][H], b2[H], W3[n_out][H], b3[n_out]; tanh after layers 1 and 2. */
msasm_status msasm_mlp_create(int32_t n_out, int32_t hidden, uint64_t seed, msasm_mlp** out);
msasm_status msasm_mlp_info(const msasm_mlp* mlp, int64_t* n_params, int32_t* n_out, int32_t* hidden);
/* Set the FP32 master parameters (device) and refresh the FP16 copy. */
msasm_status msasm_mlp_set_params(msasm_mlp* mlp, const float* d_params, void* stream);
/* Copy the FP32 master parameters and/or the FP16 compute copy (n_params __half) to device buffers. */
msasm_status msasm_mlp_get_params(const msasm_mlp* mlp, float* d_master, void* d_half, void* stream);
/* y = MLP(x) for B scalar inputs: d_y (B x n_out) FP32. */
msasm_status msasm_mlp_forward(msasm_mlp* mlp, const float* d_x, int32_t B, float* d_y, void* stream);

/* The same forward pass with the output layer on the tensor cores (split FP16: the last hidden
 * layer as hi + 2^-11 lo per row-scaled slice, three products, FP32 accumulation; the FP16 output
 * weights are exact in the slices, made once per set of weights): about 1e-7 relative to
 * msasm_mlp_forward.  The surrogate's predictions and assembly use this form. */
msasm_status msasm_mlp_forward_tc(msasm_mlp* mlp, const float* d_x, int32_t B, float* d_y, void* stream);
/* Loss L = mean over B x n_out of (y - t)^2 and dL/dparams (w.r.t. the FP16 weights, FP32 result,
 * n_params values into d_grad if non-NULL).  Synchronises `stream`. */
msasm_status msasm_mlp_loss_grad(msasm_mlp* mlp, const float* d_x, const float* d_t, int32_t B, float* h_loss,
                                 float* d_grad, void* stream);
/* `steps` full-batch Adam steps (beta 0.9 / 0.999, eps 1e-8) at learning rate lr, one step
 * replayed as a CUDA graph; h_loss (optional, steps floats) gets the loss before each step. */
msasm_status msasm_mlp_train(msasm_mlp* mlp, const float* d_x, const float* d_t, int32_t B, int32_t steps, float lr,
                             float* h_loss, void* stream);
void msasm_mlp_destroy(msasm_mlp* mlp);

/* Fit the surrogate from n_tables quadrature tables T(w_k) (msasm_build_tables of the tile at
 * width widths[k], host array) and coefficient rows of the workload (d_coef_samples,
 * n_sample_rows x 9 n_pi FP64, e.g. rows of msasm_pullback): U spans the dominant left singular
 * subspace of [T(w_k) C^T] (randomized range finder with `power_iters` power iterations, FP64),
 * the MLP (hidden width `hidden`, output r x 9 n_pi) is initialised from `seed` and its
 * training targets are V_k^T = U^T T(w_k), centred and scaled.  Synchronises `stream`. */
msasm_status msasm_surrogate_create(const msasm_tables* const* tables, const double* widths, int32_t n_tables,
                                    const double* d_coef_samples, int64_t n_sample_rows, int32_t rank,
                                    int32_t hidden, int32_t power_iters, uint64_t seed, void* stream,
                                    msasm_surrogate** out);
msasm_status msasm_surrogate_info(const msasm_surrogate* sur, int32_t* rank, int32_t* K, int32_t* n_nz);
/* Train the MLP on the fitted targets (msasm_mlp_train semantics). */
msasm_status msasm_surrogate_train(msasm_surrogate* sur, int32_t steps, float lr, float* h_loss, void* stream);
/* The surrogate's MLP (owned by the surrogate). */
msasm_status msasm_surrogate_mlp(msasm_surrogate* sur, msasm_mlp** mlp);
/* U as n_nz x r FP32 (row-major) into d_U. */
msasm_status msasm_surrogate_basis(const msasm_surrogate* sur, float* d_U, void* stream);
/* V(w)^T for n widths (device FP64): d_Vt (n x r x 9 n_pi) FP32. */
msasm_status msasm_surrogate_predict(msasm_surrogate* sur, const double* d_widths, int64_t n, float* d_Vt,
                                     void* stream);
/* Low-rank eq. 58 with the factor U (d_U, n_nz x rank FP32 row-major): for n_tiles tiles,
 * nz[t][m][ab] = sum_r (sum_k Vt_t[r][k] coef[9t+ab][k]) U[m][r], Vt (n_tiles x rank x K FP32),
 * coef (9 n_tiles x K FP64); d_nz (n_tiles x n_nz x 9 FP32, the nzdata layout above).  Z in FP32, the product with U on the
 * tensor cores in split FP16 (about 6e-7 relative); synchronises `stream`. */
msasm_status msasm_lowrank_contract(const float* d_U, int32_t n_nz, int32_t rank, int32_t K, const float* d_Vt,
                                    const double* d_coef, int64_t n_tiles, float* d_nz, void* stream);
/* K of a graded lattice: per-tile widths d_widths (n_tiles FP64, device); pullback, MLP,
 * low-rank contraction and scatter into d_values (nnz FP32). */
msasm_status msasm_surrogate_assemble(msasm_plan* plan, msasm_surrogate* sur, const double* d_ctrl, double E,
                                      double nu, const double* d_widths, float* d_values, void* stream);
void msasm_surrogate_destroy(msasm_surrogate* sur);

/* Store a fitted (and possibly trained) surrogate in a file and read it back: the basis U, the
 * width normalisation, the normalised training targets, and the MLP with its Adam state, so that
 * a loaded surrogate predicts and assembles bit for bit as the saved one and continues training
 * from the same step.  File format and errors as msasm_tables_save / msasm_tables_load (EIO also
 * for sizes outside the limits of msasm_surrogate_create).  Both synchronise `stream`. */
msasm_status msasm_surrogate_save(const msasm_surrogate* sur, const char* path, void* stream);
msasm_status msasm_surrogate_load(const char* path, void* stream, msasm_surrogate** out);

/* Number of interpolation nodes with |det J| <= tol found by the last assemble
 * on this plan (reads back from the device; synchronises `stream`). */
msasm_status msasm_degenerate_count(const msasm_plan* plan, int64_t* count, void* stream);

/* Device time of each stage of the last assemble run with MSASM_FLAG_STAGE_TIMES,
 * summed over its passes (CUDA events on the call's stream): ms[0] pullback,
 * ms[1] contraction, ms[2] scatter (both kernels); launches[0..2] the kernel
 * launches of each stage.  Synchronises on the recorded events.  EINVAL if the
 * last assemble did not record times. */
msasm_status msasm_stage_times(const msasm_plan* plan, double* ms, int32_t* launches);

/* ---------------------------------------------------------------- stages (tests / composition) */

/* Step 1 only: pulled-back macro field at the nodes (eq. 37, 42), written as the
 * FP64 coefficient matrix d_coef[9*n_tiles][9*n_pi] (layout above). */
msasm_status msasm_pullback(msasm_plan* plan, const double* d_ctrl, double E, double nu,
                            double* d_coef, void* stream);

/* Step 1 with the L2 projection onto Q_q of eq. 20-24 instead of interpolation: the coefficients
 * (same layout as msasm_pullback, q the tables' degree) of the Lagrange basis at the q+1 Gauss-
 * Legendre nodes that minimise the L2 norm of A_bar - <A_bar> over each tile, with the load
 * integrals int N_C A_bar taken by the n_gauss-point Gauss rule per direction (1..9).  In that basis
 * the mass matrix is diagonal (the nodes' rule integrates it exactly), so no system is solved;
 * n_gauss = q + 1 gives the interpolant exactly.  The result feeds msasm_contract and msasm_scatter
 * unchanged (the table of eq. 52 does not depend on how the coefficients were obtained).
 * Synchronises `stream`.  Errors: EINVAL, EUNSUPPORTED (macro degree and n_gauss beyond the
 * kernel's shared memory), ECUDA. */
msasm_status msasm_pullback_l2(msasm_plan* plan, const double* d_ctrl, double E, double nu, int32_t n_gauss,
                               double* d_coef, void* stream);

/* Step 3 only: nz[t][m][3a+b] = sum_k coef[9t+3a+b][k] T[m][k] (eq. 58) for `n_tiles` tiles
 * of FP64 coefficients d_coef (layout above).  d_nz: n_tiles*n_nz*9 values in the nzdata
 * layout above, FP64 for MSASM_F64 / MSASM_F64_EMU, FP32 otherwise. */
msasm_status msasm_contract(const msasm_tables* tab, msasm_precision prec, const double* d_coef,
                            int64_t n_tiles, void* d_nz, void* stream);

/* The FP64 contraction of msasm_contract for callers that cannot let the
 * library allocate device memory (an application that has reserved the GPU's
 * memory for its own pool, or a service that may not call cudaMalloc/cudaFree,
 * which synchronise the device, after start-up).  The paper has no counterpart:
 * it is an interface addition, not a step of the method.  Same arguments and
 * result as msasm_contract with MSASM_F64 (d_nz: n_tiles x n_nz x 9 FP64, the nzdata
 * layout above), but the padded intermediate lives in a fixed 32 MiB file-scope device
 * array: n_tiles * 9 * round_up(n_nz, 8) * 8 bytes must fit, otherwise EINVAL (for
 * n_nz = 23286 that is 20 tiles per call).  The first call on a device, made
 * with that device current, looks up the array's address; make it before any
 * stream capture.  Calls share the array: calls that overlap on the GPU race and
 * must be serialised by the caller.  Nothing is allocated and nothing needs
 * clearing between calls. */
msasm_status msasm_contract_noalloc(const msasm_tables* tab, const double* d_coef, int64_t n_tiles,
                                   double* d_nz, void* stream);

/* Step 4 only: CSR values from nzdata of all tiles of the plan (d_nz as written by
 * msasm_contract for all plan tiles, same precision family). */
msasm_status msasm_scatter(msasm_plan* plan, msasm_precision prec, const void* d_nz,
                           void* d_values, void* stream);

/* ---------------------------------------------------------------- matrix-free operator */

/* y = K u without the global CSR values (Sec. 4.2, eq. 74): the tile matrices are formed on the
 * fly from the lookup table and the projection coefficients d_coef (9 n_tiles x 9 n_pi FP64, as
 * written by msasm_pullback) by the contraction of eq. 58 in precision `prec`, and applied to u.
 * d_u, d_y: n_rows FP64 (y overwritten).
 *  - Tensor-core forms MSASM_F64_EMU (FP64 products) and MSASM_SPLIT_F16, _SPLIT_BF16, _TF32,
 *    _TF32X3 (FP32 products): the contraction's epilogue applies each tile block to u as it leaves
 *    the accumulators, with FP64 atomic additions into y: no tile matrix is ever stored, no nzdata
 *    scratch is used, and the last bits of every row may vary between calls (the order of the
 *    atomic additions).
 *  - MSASM_F64 and MSASM_F32: pass by pass in the plan's nzdata scratch; every row is written by the tile that
 *    owns it, then the glued-face blocks are added with atomics (so the last bits of those rows may
 *    vary between calls); the first such call builds per-type column maps and synchronises `stream`.
 * Errors: EINVAL, EUNSUPPORTED, ECUDA. */
msasm_status msasm_linop_apply(msasm_plan* plan, const double* d_coef, msasm_precision prec, const double* d_u,
                               double* d_y, void* stream);

/* ---------------------------------------------------------------- projection error */

/* Relative projection error of the macro field (eq. 59, the quantity of eq. 47-48) for the
 * interpolation degree q (0..7; independent of the plan's own q): per tile, the largest over the
 * sample points xi_s = (s + 1/2)/n_samples (n_samples per direction, 1..8) of
 * ||A_bar - Pi A_bar||_F / ||A_bar||_F over the 81 components, into d_err_tiles (n_tiles FP64,
 * may be NULL) and the largest over the tiles into d_err_max (one FP64, may be NULL; not both).
 * The degree of eq. 65 is the smallest q whose error is below a tolerance.  Synchronises `stream`.
 * Errors: EINVAL, EUNSUPPORTED, ECUDA. */
msasm_status msasm_projection_error(const msasm_plan* plan, const double* d_ctrl, int32_t q, int32_t n_samples,
                                    double E, double nu, double* d_err_tiles, double* d_err_max, void* stream);

/* The same error for a degree per direction, q3 = (q1, q2, q3) (host int32[3], each 0..7). */
msasm_status msasm_projection_error_q3(const msasm_plan* plan, const double* d_ctrl, const int32_t* q3,
                                       int32_t n_samples, double E, double nu, double* d_err_tiles, double* d_err_max,
                                       void* stream);

/* The same error for the L2 projection of degree q (msasm_pullback_l2, load rule of n_gauss points
 * per direction, 1..9) in place of the interpolant. */
msasm_status msasm_projection_error_l2(const msasm_plan* plan, const double* d_ctrl, int32_t q, int32_t n_gauss,
                                       int32_t n_samples, double E, double nu, double* d_err_tiles, double* d_err_max,
                                       void* stream);

/* The degree of eq. 65 (Sec. 3.3.1): the smallest q in [q0, q_max] (0 <= q0 <= q_max <= 7) whose
 * E_proj (msasm_projection_error with n_samples per direction) is at most tol, else q_max; into
 * *q_out, and its E_proj into *err_out (may be NULL).  An error within a relative 1e-9 above tol
 * counts as meeting it, so that rounding differences between implementations of E_proj cannot
 * decide the degree.  Synchronises `stream`.  Errors: EINVAL, EUNSUPPORTED, ECUDA. */
msasm_status msasm_select_degree(const msasm_plan* plan, const double* d_ctrl, double tol, int32_t q0, int32_t q_max,
                                 int32_t n_samples, double E, double nu, int32_t* q_out, double* err_out,
                                 void* stream);

/* A projection degree per direction (the anisotropic space of Sec. 3.3.4), from q_init (host
 * int32[3], e.g. the macro map's degrees; each in 0..q_max, q_max <= 7): while E_proj > tol, raise
 * the one direction whose increase lowers E_proj most; then, while possible, lower the direction
 * whose decrease keeps E_proj lowest and still within tol.  Errors within a relative 1e-9 of each
 * other are ties, which go to the lowest direction, and within 1e-9 above tol meet it.  The
 * degrees into q_out (host int32[3]), their E_proj into *err_out (may be NULL).  Synchronises
 * `stream`.  Errors: EINVAL, EUNSUPPORTED, ECUDA. */
msasm_status msasm_select_degrees(const msasm_plan* plan, const double* d_ctrl, double tol, const int32_t* q_init,
                                  int32_t q_max, int32_t n_samples, double E, double nu, int32_t* q_out,
                                  double* err_out, void* stream);

/* ---------------------------------------------------------------- volume and loads */

/* The load lookup table of eq. 54-55 (body term, F = 0): d_F[A][C] = int_{Omega_T} R_A N_C
 * (n_T x n_pi FP64, row-major), and the volume table of eq. 18: d_vol[C] = int_{Omega_T} N_C
 * (n_pi FP64); either may be NULL.  Both are built with the stiffness table. */
msasm_status msasm_load_table_copy(const msasm_tables* tab, double* d_F, double* d_vol, void* stream);

/* Volume of the lattice (Sec. 3.1, eq. 14-19) through the volume table: per tile
 * V^(t) = t^h . d^(t), d_C^(t) = |det J^(t)(xi_C)| at the interpolation nodes, into
 * d_tile_volume (n_tiles FP64, may be NULL), and the total (summed in a fixed order) into
 * d_total (one FP64, may be NULL; not both NULL).  Errors: EINVAL, EUNSUPPORTED, ECUDA. */
msasm_status msasm_volume(const msasm_plan* plan, const double* d_ctrl, double* d_tile_volume, double* d_total,
                          void* stream);

/* Gradient of the volume with respect to the macro control net (Sec. 4.1.1, eq. 66-67): the
 * adjoint field t^h times d|det J|/dP at the nodes, summed back to the control points;
 * d_grad_ctrl (n_ctrl*3 FP64) is overwritten.  Errors: EINVAL, EUNSUPPORTED, ECUDA. */
msasm_status msasm_volume_grad(const msasm_plan* plan, const double* d_ctrl, double* d_grad_ctrl, void* stream);

/* Load vector of a constant body force b = (bx, by, bz) (eq. 39-40 and the F = 0 term of eq. 53):
 * f_{3g+a} = b_a sum over the tiles holding point g of sum_C F[A][C] |det J^(t)(xi_C)|;
 * d_f (n_rows FP64) is overwritten.  Errors: EINVAL, EUNSUPPORTED, ECUDA. */
msasm_status msasm_body_load(const msasm_plan* plan, const double* d_ctrl, double bx, double by, double bz,
                             double* d_f, void* stream);

/* Load vector of a uniform traction t = (tx, ty, tz) (force per unit physical area) on macro face
 * `face` = 2 d + s (the tiles' boundary parts on xi_d = s), through the face tables (the F >= 1
 * terms of eq. 53-55): per tile on the face, t |det I_M| (eq. 87-88, the macro surface element
 * |dM/dxi_a x dM/dxi_b| on that face) interpolated at the face's (q_a+1)(q_b+1) Gauss-Legendre nodes,
 * times the table: f_{3g+c} = t_c sum_C2 Ff[A][C2] |det I_M|(node C2).  Equals the direct
 * quadrature (msasm_traction_load) to roundoff when the surface element is a polynomial of degree
 * <= q per direction (an affine map), and converges with q otherwise.  d_f (n_rows FP64) is
 * overwritten.  Points shared by face tiles receive one addition per tile (FP64 atomics).
 * Synchronises `stream`.  Errors: EINVAL, EUNSUPPORTED, ECUDA. */
msasm_status msasm_traction_load_lookup(const msasm_plan* plan, const double* d_ctrl, int32_t face, double tx,
                                        double ty, double tz, double* d_f, void* stream);

/* Copy the face load table of `face` (n_T x (q_a+1)(q_b+1) FP64, row A, column C2 = c_a + (q_a+1) c_b
 * over the two in-face directions a < b) to d_Ff. */
msasm_status msasm_face_table_copy(const msasm_tables* tab, int32_t face, double* d_Ff, void* stream);

/* ---------------------------------------------------------------- diagnostics */

const char* msasm_last_error(void);
const char* msasm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MSASM_H */
