/*
 * dg.h -- C ABI of libdg: GPU assembly of the symmetric interior-penalty
 * discontinuous Galerkin (SIPG) matrix and load vector for linear
 * diffusion-advection-reaction problems on polygonal (2D) and polyhedral (3D)
 * meshes, after Dong, Georgoulis & Kappas, "GPU-accelerated discontinuous
 * Galerkin methods on polytopic meshes" (arXiv 2007.04881).
 *
 * Problem (Sec. 2.1, Eq. (2.1)):  -div(a grad u) + b . grad u + c u = f,
 * with a > 0 piecewise constant per element (A = a I), b and c constant (or,
 * through dg_assemble_varcoef, an affine b and a cubic c such as the fields
 * of Sec. 4.2), u = g_D on the Dirichlet boundary and a grad u . n = g_N on
 * the Neumann boundary (Eq. (2.2); sides marked in dg_mesh_desc.neumann, the
 * whole boundary Dirichlet by default).
 * Discretisation (Sec. 2.2): B(u_h, v) = l(v) with the bilinear form of
 * Eq. (2.4) and the load functional of Eq. (2.5); the local space on element
 * k is P_{p_k}, spanned by tensorised orthonormal Legendre polynomials of
 * total degree p_k on the element's bounding box (Sec. 3.1).
 * Quadrature (Sec. 3 intro, Sec. 3.1): each element is split into simplices
 * (2D: triangles (centroid, v_i, v_{i+1}) of the CCW vertex loop; 3D: the
 * element's tetrahedra) carrying collapsed Gauss-Legendre rules with p+2
 * points per direction; faces carry Gauss rules with max(p_1, p_2) + 1 points
 * per direction (2D edges; 3D triangles, collapsed).
 * Penalty (Appendix A, simplified): sigma_F = C_sigma * max over the face's
 * elements of a_k p_k^2 / h_k, h_k the element diameter.
 *
 * Output: a variable-block BSR matrix.  Block row r = element r; the columns
 * of row r are r and every element sharing a face with r, ascending.  Block
 * (r, c) is n_r x n_c, row-major (row = test function of r, column = trial
 * function of c), n_k = C(p_k + d, d).  One block per element pair, however
 * many faces the two elements share (the unique-index idea of Sec. 3.4).
 * Entries are written without atomics in a fixed order, so results are
 * bitwise reproducible.
 *
 * Conventions for every entry point:
 *   - returns DG_OK (0) or a negative DG_ERR_* code; dg_last_error() gives a
 *     message (thread-local).  No C++ exception crosses this ABI.
 *   - "device" pointers are CUDA device memory on the context's device,
 *     allocated and owned by the caller; "host" pointers are CPU memory.
 *   - assembly calls are asynchronous on the context's stream; results are
 *     valid once the stream (or dg_sync) completes.
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DG_OK 0
#define DG_ERR_ARG (-1)     /* invalid argument (null pointer, bad size/flag) */
#define DG_ERR_MESH (-2)    /* invalid mesh (non-manifold, bad orientation, zero area, p range) */
#define DG_ERR_CUDA (-3)    /* a CUDA runtime call failed */
#define DG_ERR_OOM (-4)     /* device or host allocation failed */
#define DG_ERR_ORDER (-5)   /* dg_assemble_faces called before dg_assemble_volume */
#define DG_ERR_TIMEOUT (-6) /* a bounded device-side wait ran out */
#define DG_ERR_BOUNDS (-7)  /* builds with DG_CHECK_BOUNDS: a kernel found an output range outside its array */

/* precision flags (prec argument) */
#define DG_PREC_FP64 0 /* everything in FP64; vals are double */
#define DG_PREC_FP32 1 /* basis evaluation and contractions in FP32 on geometry
                          records (maps, Jacobians, normals, penalty) equal to the
                          FP64 geometry's rounded to FP32; vals are float.  A pass
                          that recomputes the geometry (dg_assemble_step,
                          dg_assemble_host, graphs) builds them in FP32 from the
                          coordinates split into float pairs; the FP64 geometry
                          runs at upload, dg_geometry and dg_mesh_update. */
/* Tensor-core forms: geometry, points, weights and basis values as
 * DG_PREC_FP32; the local contractions U^T V (and the load vector, as one
 * more column of V) run on the tensor cores with FP32 accumulation, every
 * operand split as x = hi + lo and each product taken as hi*hi + hi*lo +
 * lo*hi.  Degree-1 elements use the FP32 form.  vals and rhs are float. */
#define DG_PREC_BF16X3 2 /* hi, lo in bfloat16 */
#define DG_PREC_TF32X3 3 /* hi, lo in TF32 */
/* Flag OR-ed into the precision of the entry points that recompute the
 * geometry each pass (dg_assemble_step, dg_assemble_host, dg_graph_create)
 * for the FP32 and tensor-core forms: the pass runs the FP64 geometry
 * kernels (maps, Jacobians, normals, penalties in FP64, stored in FP64 and
 * rounded to FP32 for the contraction) instead of the reduced-precision
 * ones on float-pair coordinates.  No effect on DG_PREC_FP64. */
#define DG_GEOM_FP64 16

/* source / boundary data */
#define DG_SRC_ZERO 0    /* f = 0, g_D = 0 */
#define DG_SRC_SINPROD 1 /* u = prod_d sin(pi x_d): f = a d pi^2 u + b.grad u + c u, g_D = u */
#define DG_SRC_POLY 2    /* u = sum_k poly[k] m_k(x), graded monomials of degree <= 3
                            (2D: 1,x,y,x^2,xy,y^2,x^3,x^2y,xy^2,y^3; 3D: the 20 monomials
                            ordered as: degree k, then z-power l, then y-power j);
                            f = -a Lap u + b.grad u + c u, g_D = u */

#define DG_PMAX_2D 6
#define DG_PMAX_3D 4

typedef struct dg_ctx dg_ctx;
typedef struct dg_mesh dg_mesh;

/* Mesh description.  All pointers are HOST memory and are copied by
 * dg_mesh_upload; the caller keeps ownership.
 *   2D: elem_ptr[ne+1] and elem_idx[] list each element's vertex loop,
 *       counter-clockwise; neighbouring elements share vertex ids (conforming).
 *   3D: elem_ptr[ne+1] indexes tetrahedra; elem_idx[4*ntet] holds the 4 vertex
 *       ids of each tetrahedron, grouped by element.  Faces between tetrahedra
 *       of the same element are interior to it.
 * Faces are derived from the elements: a 2D loop edge / 3D tetrahedron
 * triangle seen by two elements is an interior face, seen by one a boundary
 * face. */
typedef struct {
  int dim;                 /* 2 or 3 */
  int nv;                  /* vertices */
  const double *x, *y, *z; /* vertex coordinates (z unused in 2D) */
  int ne;                  /* elements */
  const int *elem_ptr;     /* [ne+1] */
  const int *elem_idx;     /* 2D: loop vertex ids; 3D: 4 vertex ids per tetrahedron */
  const int8_t *p;         /* [ne] polynomial degree, 1 <= p <= DG_PMAX_{2D,3D} */
  const double *a;         /* [ne] diffusion coefficient, a > 0 */
  double b[3];             /* constant advection field */
  double c;                /* constant reaction, c >= 0 (c - div b / 2 = c >= 0, Sec. 2.1) */
  int source;              /* DG_SRC_* */
  double poly[20];         /* coefficients for DG_SRC_POLY */
  double c_sigma;          /* penalty constant C_sigma (> 0; the configs use 10) */
  int neumann;             /* Neumann part of the boundary (Eq. (2.2)): bit 2d + s marks the
                              side x_d = min (s = 0) or x_d = max (s = 1) of the bounding box
                              of the vertices.  A boundary face all of whose vertices lie on a
                              marked side (coordinates compared exactly) is a Neumann face:
                              it adds no term to the matrix (Eq. (2.4)) and g_N v, g_N = a
                              grad u . n of the manufactured u, to the load vector (Eq.
                              (2.5)); every other boundary face is a Dirichlet face.  0: the
                              whole boundary is Dirichlet.  Bits past 2 dim are an error. */
} dg_mesh_desc;

/* Sizes of the block-sparse layout of a mesh. */
typedef struct {
  int ne;           /* block rows = elements */
  int nnzb;         /* stored blocks */
  int64_t nvals;    /* stored scalar entries = sum over blocks of n_r * n_c */
  int64_t ndofs;    /* sum of n_k = length of the load vector */
  int nfaces;       /* faces (interior + boundary) */
  int ninterfaces;  /* element pairs sharing at least one face */
  int nbfaces;      /* boundary faces */
  int nsub;         /* sub-simplices (2D triangles, 3D tetrahedra) */
  int64_t nqvol;    /* volume quadrature points */
  int64_t nqface;   /* face quadrature points (interior faces counted once) */
} dg_bsr_info;

/* Create a context on CUDA device `device` that issues all work on
 * `stream` (a cudaStream_t; NULL = the legacy default stream).  The stream
 * stays owned by the caller. */
int dg_create(dg_ctx **ctx, int device, void *stream);
void dg_destroy(dg_ctx *ctx);
const char *dg_last_error(void);

/* Validate and upload a mesh, derive faces and interfaces, build the BSR
 * pattern and work lists (host), and run the geometry kernels (device,
 * Sec. 3 intro: subdivision data, bounding boxes, normals, penalties).
 * Returns DG_ERR_MESH for: index out of range, a 2D loop with fewer than 3
 * vertices or non-positive area, a zero-volume tetrahedron, a face seen by
 * more than two elements, two neighbouring 2D loops traversing their common
 * edge in the same direction, p out of range, a <= 0, c < 0, C_sigma <= 0. */
int dg_mesh_upload(dg_ctx *ctx, const dg_mesh_desc *desc, dg_mesh **out);
int dg_mesh_free(dg_mesh *mesh);

/* on != 0: the context's later dg_mesh_upload calls build the block pattern
 * on the device (the paper builds its pattern with Thrust on the GPU, Sec. 3.4
 * and Sec. 4.2, "indices" in Tables 1, 2, 5, 6): half faces keyed by their
 * sorted vertex ids and matched after a stable LSD radix sort, faces ordered
 * by (boundary, e0, e1), interfaces as runs of equal element pairs, block rows
 * from a stable sort of the interfaces by their second element, offsets by
 * exclusive scans, the work lists by stable radix sorts.  The descriptor's
 * scalar checks stay on the host; the geometric checks (2D loop and fan
 * areas, 3D tetrahedron volumes) and the face checks run on the device and
 * give the same DG_ERR_MESH cases.  The arrays are bitwise those of the host
 * build.  Partitions (dg_mesh_upload_part) and batches keep the host build.
 * Off by default. */
int dg_set_pattern_device(dg_ctx *ctx, int on);

/* Wall times of the mesh's upload: the pattern build (host plan or device
 * build, including its host copies) and the whole upload, in ms; on_device
 * 1 when the pattern was built on the device.  Any output may be NULL. */
int dg_mesh_timings(const dg_mesh *mesh, double *pattern_ms, double *upload_ms, int *on_device);

/* Copy one of the mesh's internal arrays to host memory: "row_ptr", "col",
 * "blk_off", "dof_off", "blk_if", "diag_blk", "blk_rec" (int4 per block),
 * "f_e0", "f_e1", "f_v", "f_flip" (int8), "f_nq", "f_hf" ([2][nf]),
 * "hf_ptr", "hf_face", "hf_side" (int8), "hf_qoff", "e_nqf", "if_e0",
 * "if_e1", "if_fptr", "if_slot01", "if_slot10", "elem_perm", "if_perm",
 * "sub_elem", "uvptr", "uvidx", "elem_pstart", "if_pstart" (9 ints each).
 * *bytes (may be NULL) gets the array's size; host may be NULL to query it;
 * DG_ERR_ARG for an unknown name or cap_bytes too small.  Synchronous. */
int dg_mesh_array(const dg_mesh *mesh, const char *name, void *host, int64_t cap_bytes, int64_t *bytes);

/* Host-only dry run of dg_mesh_upload: the same validation, face derivation
 * and BSR pattern, without touching a GPU.  Fills *info (may be NULL) and,
 * for non-NULL arrays sized from a previous call's info, row_ptr[ne+1],
 * col[nnzb] and blk_off[nnzb+1].  Same error codes as dg_mesh_upload. */
int dg_mesh_check(const dg_mesh_desc *desc, dg_bsr_info *info, int *row_ptr, int *col,
                  int64_t *blk_off);

/* Replace vertex coordinates (host, same topology) and per-element
 * diffusion coefficients (host, may be NULL to keep them); re-runs the
 * geometry kernels on the context stream. */
int dg_mesh_update(dg_ctx *ctx, dg_mesh *mesh, const double *x, const double *y, const double *z,
                   const double *a);

/* Re-run the geometry kernels (bounding boxes, sub-simplex maps, face data,
 * penalties) from the uploaded coordinates, on the context stream. */
int dg_geometry(dg_ctx *ctx, dg_mesh *mesh);

int dg_bsr_layout(const dg_mesh *mesh, dg_bsr_info *out);
/* Copy the pattern to HOST arrays: row_ptr[ne+1], col[nnzb], blk_off[nnzb+1]
 * (offsets of blocks in vals, in entries), dof_off[ne+1] (offsets of each
 * element's entries in the load vector). Any pointer may be NULL. */
int dg_bsr_pattern(const dg_mesh *mesh, int *row_ptr, int *col, int64_t *blk_off, int64_t *dof_off);

/* Volume integrals (first line of Eq. (2.4)) of every element: OVERWRITES
 * each element's diagonal block in vals (device, nvals entries of double for
 * DG_PREC_FP64, float for the other forms).  Off-diagonal blocks are untouched. */
int dg_assemble_volume(dg_ctx *ctx, const dg_mesh *mesh, int prec, void *vals);

/* Face integrals (second and third lines of Eq. (2.4)): ADDS each element's
 * own-face contributions to its diagonal block (each element reduces its own
 * faces in a fixed order; no atomics) and OVERWRITES the off-diagonal blocks
 * of every interface.  Must follow dg_assemble_volume on the same vals
 * (DG_ERR_ORDER otherwise). */
int dg_assemble_faces(dg_ctx *ctx, const dg_mesh *mesh, int prec, void *vals);

/* Load vector of Eq. (2.5) into rhs (device, ndofs entries of double /
 * float by prec), OVERWRITTEN. */
int dg_assemble_rhs(dg_ctx *ctx, const dg_mesh *mesh, int prec, void *rhs);

/* Whole system in one pass: every block of vals and, if rhs is not NULL,
 * the load vector; equal up to rounding to volume + faces (+ rhs). */
int dg_assemble(dg_ctx *ctx, const dg_mesh *mesh, int prec, void *vals, void *rhs);

/* End-to-end from host memory: copies x,y,z (host, nv each; may be NULL to
 * keep the uploaded coordinates) and a (host, ne; may be NULL) to the
 * device, recomputes the geometry in the pass's precision (as
 * dg_assemble_step), assembles the system into library-owned device
 * buffers and copies vals (host, nvals entries) and rhs (host, ndofs
 * entries; may be NULL) back.  The launch shape is the one dg_graph_create
 * last tuned for this mesh and precision (under the context's current
 * volume-path setting), else concurrent degree groups.  Synchronous. */
int dg_assemble_host(dg_ctx *ctx, dg_mesh *mesh, int prec, const double *x, const double *y,
                     const double *z, const double *a, void *vals_host, void *rhs_host);

/* Pipelined form of dg_assemble_host, for a sequence of independent
 * assemblies on one mesh (new coefficients a or coordinates each time):
 * the system of Eq. (2.4) and the load vector of Eq. (2.5), as
 * dg_assemble_host computes them, with the copy back of one assembly
 * running beside the next one's pass.
 *
 * dg_assemble_host_submit queues, on the context's stream, the copies of
 * x, y, z, a (host; NULL keeps the device copy) and the pass into one of
 * two library-owned device slots. On a copy stream of the mesh it then
 * queues the copy of vals (host, nvals entries) and rhs (host, ndofs
 * entries, or NULL) back. It returns without waiting, with *ticket (0, 1,
 * 2, ...) naming the submission.
 *
 * dg_assemble_host_wait blocks until that submission's vals and rhs are in
 * host memory.
 *
 * Ownership: the caller keeps x, y, z, a, vals_host and rhs_host valid and
 * unchanged until the ticket's wait returns. Page-locked host buffers let
 * the copies run asynchronously.
 *
 * Ordering: submissions run in order. A slot is reused two submissions
 * later, after its copy back. A change of prec between submissions waits
 * for every queued copy and reallocates the slots.
 *
 * Errors: DG_ERR_ARG for a null argument, or a ticket not submitted on this
 * mesh; DG_ERR_OOM or DG_ERR_CUDA as in dg_assemble_host. */
int dg_assemble_host_submit(dg_ctx *ctx, dg_mesh *mesh, int prec, const double *x, const double *y,
                            const double *z, const double *a, void *vals_host, void *rhs_host,
                            long long *ticket);
int dg_assemble_host_wait(dg_ctx *ctx, dg_mesh *mesh, long long ticket);

/* One pass of the whole hot path on device-resident inputs: the geometry
 * kernels in the pass's precision followed by the row kernels, in the
 * launch shape of dg_assemble_host.  Asynchronous.
 *
 * Concurrent degree groups run on four forked streams per context (and
 * four per graph, captured).  A process that uses more streams than the
 * driver's hardware work queues (CUDA_DEVICE_MAX_CONNECTIONS, 8 by default)
 * can see two groups serialised on one queue; set that variable to 32
 * before the CUDA context is created. */
int dg_assemble_step(dg_ctx *ctx, dg_mesh *mesh, int prec, void *vals, void *rhs);

/* Batches (many independent meshes in one pass).  dg_batch_upload merges n
 * descriptors (same dim and problem data b, c, source, poly, C_sigma) into
 * one mesh, their disjoint union: its block-sparse matrix is the
 * block-diagonal concatenation of the members' matrices, member k owning
 * element rows elem_off[k] .. elem_off[k+1], values val_off[k] ..
 * val_off[k+1] and load-vector entries dof_off[k] .. dof_off[k+1]
 * (dg_batch_offsets; arrays of n+1 entries, any may be NULL).  All degree
 * groups of all members are then assembled by the same launches. */
int dg_batch_upload(dg_ctx *ctx, const dg_mesh_desc *const *descs, int n, dg_mesh **out);

/* The other form of a batch: nmesh meshes uploaded separately (each by
 * dg_mesh_upload or dg_batch_upload), each assembled into its own buffers in
 * one call.  vals[k] (device, nvals of mesh k, double for DG_PREC_FP64 else
 * float) is OVERWRITTEN with every block; rhs (may be NULL, or hold NULL
 * entries) with the load vectors.  Each member runs its whole pass as
 * dg_assemble_step does (geometry in the pass's precision, then the row
 * kernels in the launch shape last tuned for that mesh, degree groups one
 * after the other); members run concurrently on four forked streams of the
 * context.  use_graph != 0 records the whole batch as one CUDA graph,
 * launches it and frees it (for repeated passes over the same meshes, record
 * once: dg_batch_upload + dg_graph_create).  prec may carry DG_GEOM_FP64.
 * Asynchronous on the context stream; each member's result equals its own
 * dg_assemble_step bit for bit. */
int dg_assemble_batch(dg_ctx *ctx, dg_mesh *const *meshes, int nmesh, int prec, void *const *vals, void *const *rhs,
                      int use_graph);
int dg_batch_offsets(const dg_mesh *mesh, int *nmesh, int *elem_off, int64_t *val_off, int64_t *dof_off);

/* How the row passes evaluate the volume terms of Eq. (2.4):
 *   path 1 (default): the quadrature sums over each element's rule (the
 *     sub-simplex rules of Sec. 3, or its learned rule) are accumulated as
 *     weighted Legendre-product moments sum_q W_q P_c(xi_q) P_d(eta_q)
 *     (P_e(zeta_q)), c + d (+ e) <= 2p, and every block entry is formed from
 *     them through the exact Legendre linearisation of the basis products:
 *     the same rule and points, the sums taken in another order.  Used for
 *     degrees whose moments fit in registers (2D p >= 3 in FP32, p = 3, 4
 *     in FP64; 3D p = 2, 3 in FP32, p = 2 in FP64) in the FP32 and FP64
 *     forms; the diagonal block is then written by a separate moment
 *     launch and the row kernel adds the face terms to it.
 *   path 2: as path 1, but the moments are exact, from the element's
 *     boundary (Sec. 1 and Sec. 3: integrals of homogeneous functions moved
 *     to the boundary).  2D, by Green's theorem along the loop: mu_cd =
 *     (L_1 L_2 / 4) times the closed integral of Q_c(xi) P_d(eta) d eta, Q_c
 *     an antiderivative of P_c, with the (p + 1)-point Gauss rule on each
 *     edge (exact: degree <= 2p + 1).  3D, by the divergence theorem with
 *     the field (L_1 / 2) Q_c P_d P_e e_1 over the element's boundary
 *     triangles, with the collapsed rule of p + 2 points per direction
 *     (exact: degree <= 2p + 2).  For the polynomial volume integrands of
 *     constant coefficients this is the sub-simplex rule's value up to
 *     rounding; the load vector (a general source) keeps the rule's points.
 *   path 0: the per-point block contraction in the row kernels throughout.
 * The tensor-core forms always take their own contraction.  A mesh with
 * learned rules installed (28 points per element) takes the per-point path
 * in the calls; dg_graph_create's autotuner times both.  Applies to later
 * calls and recorded passes made after it; DG_ERR_ARG for another path. */
int dg_set_volume_path(dg_ctx *ctx, int path);

/* Register-tile variant (0..2) of each degree's row kernel (variants[p], 9
 * entries, p = 0..8; NULL: all defaults) for the calls that have no tuned
 * launch shape: the direct calls, and dg_assemble_step / dg_assemble_host /
 * dg_assemble_batch on a mesh and precision dg_graph_create has not tuned.
 * A degree without that variant (see dg_graph_tiles) takes its default.
 * Every variant sums each block entry over the same points in the same
 * order, so the results are bitwise those of the default tiles. */
int dg_set_tile_variants(dg_ctx *ctx, const int *variants);

/* on != 0: NVTX ranges (host markers read by profilers) around the later
 * calls of this context that upload, assemble, tune or record, and around
 * their stages (host or device pattern, geometry).  Off by default. */
int dg_set_nvtx(dg_ctx *ctx, int on);

/* Parts of each degree group (split[p], 9 entries, 1..4; NULL: all 1) for
 * the calls without a tuned launch shape that run the degree groups
 * concurrently (dg_assemble_step / dg_assemble_host on an untuned mesh,
 * the slab step's spatial pass).  A group in k parts is k contiguous runs
 * of equal element count, each with its own moment launch and row launch on
 * a stream of its own, so that the chains of the largest groups run side by
 * side instead of one after the other.  Every element is computed by the
 * same kernel as without parts: the results are bitwise the same.
 * DG_ERR_ARG for a value outside 1..4. */
int dg_set_group_split(dg_ctx *ctx, const int *split);

/* Partitions (Sec. 4.2: the elements are split across GPUs, each GPU builds
 * and assembles its own rows, faces on a cut are computed by both owners, and
 * assembly needs no communication).
 *
 * dg_partition (host only) writes part[e] in 0..nparts-1 for every element
 * of desc: elements are ordered along a space-filling curve through their
 * vertex means (Hilbert in 2D, Morton in 3D) and cut into nparts contiguous
 * runs of about equal cost, the cost of an element being its volume
 * quadrature points times n^2.  Deterministic.  DG_ERR_ARG if nparts is
 * outside 1..ne.
 *
 * dg_mesh_upload_part uploads the part my_part of desc (host arrays of the
 * whole mesh; part as written by dg_partition or by any other partitioner):
 * its owned elements (part[e] == my_part) plus the halo, the elements that
 * share a face with an owned one.  Local elements and vertices keep the
 * increasing order of their global ids.  Only owned elements have block
 * rows (halo rows are empty; column indices are local ids) and load-vector
 * entries (halo elements have none), and only they are assembled.  Each
 * owned block row, mapped to global ids, is bitwise equal to the same row of
 * the whole mesh assembled by dg_mesh_upload.  dg_mesh_update and
 * dg_assemble_host then take arrays in the local numbering.
 *
 * dg_part_map returns the local -> global element map (elem_global[ne]),
 * owned flags (owned[ne]), and the local -> global vertex map
 * (vert_global[nv_local]); any output may be NULL.  DG_ERR_ARG for a mesh
 * not made by dg_mesh_upload_part.
 *
 * dg_part_check is the host part of dg_mesh_upload_part (no GPU): the local
 * layout (info, nowned, row_ptr[ne+1], col[nnzb], blk_off[nnzb+1],
 * elem_global[ne], owned[ne]; sizes from info, any output may be NULL). */
int dg_partition(const dg_mesh_desc *desc, int nparts, int *part);
int dg_mesh_upload_part(dg_ctx *ctx, const dg_mesh_desc *desc, const int *part, int my_part, dg_mesh **out);
int dg_part_map(const dg_mesh *mesh, int *nowned, int *nv_local, int *elem_global, int8_t *owned,
                int *vert_global);
int dg_part_check(const dg_mesh_desc *desc, const int *part, int my_part, dg_bsr_info *info, int *nowned,
                  int *row_ptr, int *col, int64_t *blk_off, int *elem_global, int8_t *owned);

/* CUDA graphs.  dg_graph_create records one whole pass (geometry kernels and
 * the row kernels, as dg_assemble_step) of mesh into vals / rhs (device,
 * fixed for the graph's life) as a CUDA graph.  With autotune != 0 it first
 * times the candidate launch shapes (co-resident CTAs per SM capped at 1, 2
 * or the occupancy limit; degree groups serial on one stream or concurrent
 * on forked streams; for the FP32 and FP64 forms, when the context's volume
 * path is 1, also the moment and the per-point volume paths) and records
 * the fastest.  Without autotuning the context's path is used (the per-point
 * one for a mesh with learned rules installed).  The first call must precede
 * any stream capture by the caller.  dg_graph_launch replays the pass on the
 * context stream.  dg_graph_info: the recorded shape (any output may be
 * NULL; vol_path 0 per-point, 1 moments). */
typedef struct dg_graph dg_graph;
int dg_graph_create(dg_ctx *ctx, dg_mesh *mesh, int prec, void *vals, void *rhs, int autotune, dg_graph **out);
int dg_graph_launch(dg_ctx *ctx, dg_graph *graph);
int dg_graph_info(const dg_graph *graph, int *occ_cap, int *concurrent, float *tuned_ms, int *launches,
                  int *vol_path);
/* The register tiles the recorded pass uses: tile_tm[p] (9 entries, p =
 * 0..8) is the tile edge of the degree-p row kernel (-1 for the tensor-core
 * forms' fixed fragment layout, 0 where the mesh has no element of degree p);
 * trials: passes the autotuner timed (0 without autotuning); persistent: 1
 * when the pass's row work is the persistent launch.  Any output may be
 * NULL.  With autotuning, dg_graph_create first times the launch shapes
 * above with the default tiles, then, for each degree present, every other
 * tile variant of its row kernel (FP32: 2D degree 3 {5, 4}, degree 4
 * {8, 5, 4}, degree 5 {7, 6, 5}, degree 6 {7, 6}; 3D degree 2 {5, 4},
 * degree 3 {4, 5, 7}; the first is the default) against the best pass so
 * far, keeping a variant only where it makes the pass faster; then, for the
 * FP32 form (2D degrees <= 5, 3D degrees <= 3), the persistent pass on each
 * volume path tried.
 *
 * The persistent pass is one launch with as many CTAs as fit on the GPU at
 * once; each warp takes the next tile of a work list (an atomic counter)
 * until the list is done.  A tile is G elements of one degree: a moment tile
 * (the volume terms through the Legendre-product moments) or a row tile (the
 * face terms and off-diagonal blocks, and, off the moment path, the volume
 * terms; one element per thread degrees get warp tiles of half the block's
 * edge).  The list holds every moment tile first, then every row tile, each
 * part ordered by estimated work, largest first; it is built on the host at
 * the first persistent pass of a mesh and volume path (a synchronous upload,
 * done by the autotuner before the graph is recorded).  A row tile adds to
 * the diagonal blocks and load vector its elements' moment tiles wrote: it
 * waits for their flags, a wait bounded in wall time (dg_set_wait_limit); a
 * wait that runs out skips those additions and makes the next dg_sync return
 * DG_ERR_TIMEOUT.  The work list of each volume path is kept with the mesh
 * (recorded graphs refer to it); the flags are the mesh's, so persistent
 * passes of one mesh must not overlap on the GPU (one stream, or events). */
int dg_graph_tiles(const dg_graph *graph, int *tile_tm, int *trials, int *persistent);
/* The parts per degree group of a recorded pass (split[9]; all 1 for a
 * serial or persistent pass): the autotuner tries 2..4 parts for each degree
 * present, from the highest, after the tiles (see dg_set_group_split). */
int dg_graph_splits(const dg_graph *graph, int *split);
int dg_graph_free(dg_graph *graph);

/* Learned reduced volume rules (2D).  For each element mapped to its
 * bounding box [-1,1]^2, a rule of 28 points and weights that reproduces
 * the 28 moments of P_6 (so the p <= 3 volume integrands with constant
 * coefficients are integrated exactly) replaces the sub-triangle rule.  The
 * paper notes that tailored polytope rules need a costly optimisation per
 * element (Sec. 1); here a small network proposes the rule and a few FP64
 * Gauss-Newton steps finish it, with the sub-triangle rule as the fallback.
 *   dg_quad_prepare: exact moments of the normalised element by the
 *     divergence theorem (FP64) and the network input: the vertex loop in
 *     bounding-box coordinates from the vertex of largest x, zero-padded to
 *     12 vertices, as 24 bfloat16 values per element.
 *   dg_quad_fit: minimum-norm Gauss-Newton, iters steps from init (device,
 *     [ne][84] network outputs (x[28], y[28], 28 w / area - 1), or NULL for
 *     a fixed 4 x 7 tensor rule); an element is accepted when the monomial
 *     moment residual / area < 1e-10 and every point lies in the bounding
 *     box; install != 0 makes accepted rules the elements' volume rules for
 *     the following assembly calls.  stats may be NULL.
 *   dg_quad_targets: the current rules encoded as network targets (device,
 *     [ne][84] float).
 *   dg_quad_buffers: library-owned device arrays (features [ne][24] bf16,
 *     rules [ne][84] double in bounding-box coordinates and weights,
 *     residuals [ne] float, accepted flags [ne] int, Legendre-product moments
 *     [ne][28] double).  Any output may be NULL.
 *   dg_quad_clear: back to the sub-triangle rules. */
typedef struct {
  int elements;
  int eligible;  /* elements with at most 12 vertices */
  int accepted;
  float max_accepted_residual;
} dg_quad_stats;
int dg_quad_prepare(dg_ctx *ctx, dg_mesh *mesh);
int dg_quad_fit(dg_ctx *ctx, dg_mesh *mesh, const float *init, int iters, int install, dg_quad_stats *stats);
int dg_quad_targets(dg_ctx *ctx, dg_mesh *mesh, float *targets);
int dg_quad_buffers(const dg_mesh *mesh, const void **feat, const double **rules, const float **resid, const int **ok,
                    const double **moments);
int dg_quad_clear(dg_ctx *ctx, dg_mesh *mesh);

/* The proposal network: 24 -> 128 -> 128 -> 84, tanh hidden layers, linear
 * output; bfloat16 operands with FP32 accumulation on the tensor cores, FP32
 * master parameters and Adam (beta 0.9 / 0.999, eps 1e-8).  Loss: mean over
 * rows of |out - target|^2 / 2.  Parameters are one flat FP32 array of
 * dg_mlp_num_params() values: W1 [24][128], b1, W2 [128][128], b2,
 * W3 [128][84], b3 (weights row-major, input index first).  x_bf16 are
 * device arrays [n][24] of bfloat16, target / out / grad device FP32.
 * dg_mlp_get/set_params and get/set_state (Adam moments) copy to and from
 * HOST arrays for checkpoints. */
typedef struct dg_mlp dg_mlp;
int dg_mlp_create(dg_ctx *ctx, int seed, dg_mlp **out);
int dg_mlp_free(dg_mlp *net);
int64_t dg_mlp_num_params(void);
int dg_mlp_get_params(const dg_mlp *net, float *host, int64_t *step);
int dg_mlp_set_params(dg_mlp *net, const float *host, int64_t step);
int dg_mlp_get_state(const dg_mlp *net, float *m1, float *m2);
int dg_mlp_set_state(dg_mlp *net, const float *m1, const float *m2);
int dg_mlp_forward(dg_ctx *ctx, dg_mlp *net, const void *x_bf16, int n, float *out);
int dg_mlp_grad(dg_ctx *ctx, dg_mlp *net, const void *x_bf16, const float *target, int n, float *grad, float *loss);
int dg_mlp_train_step(dg_ctx *ctx, dg_mlp *net, const void *x_bf16, const float *target, int n, float lr,
                      float *loss);

/* Checkpoints of a training run.  dg_mlp_save writes, after waiting for the
 * context stream, one file holding the FP32 parameters, both Adam moment
 * arrays, the step count, and two values of the caller's training loop that
 * it needs to resume where it stopped: the seed of its data order and its
 * data cursor (opaque to the library).  Format (host byte order): "DGMLPCK1",
 * u32 version 1, u32 dg_mlp_num_params(), i64 step, u64 seed, i64 cursor,
 * f32 params[], f32 m1[], f32 m2[], u64 FNV-1a checksum of the preceding
 * bytes.  It is written to "<path>.tmp" and renamed over path.
 * dg_mlp_load restores parameters, moments and step into net (the bfloat16
 * operand copy is refreshed) and returns seed and cursor (either pointer may
 * be NULL); DG_ERR_ARG for a missing, foreign, truncated or corrupted file.
 * Training resumed from a checkpoint on the same GPU reproduces the loss
 * curve of the uninterrupted run bit for bit: every training kernel sums in a
 * fixed order. */
int dg_mlp_save(dg_ctx *ctx, const dg_mlp *net, const char *path, uint64_t seed, int64_t cursor);
int dg_mlp_load(dg_ctx *ctx, dg_mlp *net, const char *path, uint64_t *seed, int64_t *cursor);

/* Learned rules for a mesh in one call (Sec. 1 and Sec. 3: a reduced rule
 * per element in place of the sub-triangle rules): dg_quad_prepare, the
 * network's proposal for every element (net NULL: the fixed 4 x 7 start),
 * iters Gauss-Newton steps, and installation of the accepted rules, which
 * the following assembly calls then use; the other elements keep their
 * sub-triangle rules.  The proposals go to a library-owned buffer of
 * ne x 84 floats (allocated at the first call, freed with the mesh).
 * stats may be NULL.  2D meshes; asynchronous except for the statistics and
 * the work-list update, which wait for the context stream. */
int dg_quad_learn(dg_ctx *ctx, dg_mesh *mesh, dg_mlp *net, int iters, dg_quad_stats *stats);

/* Per-launch timing.  When enabled, every kernel launch of the following
 * calls is bracketed by CUDA events on the context stream.  dg_kernel_stats
 * waits for the stream and copies up to cap records of the most recent call
 * (dg_geometry, dg_assemble*, dg_assemble_step) into out, returning their
 * number.  flops / bytes are the launch's algorithmic work: FMA = 2 flops;
 * per quadrature point, element of n dofs in dimension d: volume
 * d n(n+1)/2 + [b or c != 0](n^2 + n(d+1)) + basis (n d^2 + 5 d p) + n (load);
 * own interior-face point 3 n^2 + [b != 0] n^2/2 + basis; boundary-face
 * point 3 n^2 + [b != 0] n^2 + basis + 2n (load); off-diagonal block, per
 * interface point 3 n_e n_k + [b != 0] n_e n_k / 2.  Bytes: values written
 * once plus geometry records read once, in the precision's element size.
 * With the moment path (dg_set_volume_path), a degree group is two launches
 * ("row2d_vol_p<p>_<t>" for the volume terms, then the faces); the volume
 * launch is credited with the volume terms' work above.  When the call
 * issued row kernels, two more records follow: "row_pass", the span from
 * the first row-kernel start to the last row-kernel end (degree groups may
 * run concurrently) with their summed flops and bytes, and
 * "row_pass_executed", the same span with the flops the launches executed
 * (the moment form executes fewer: per volume point 2 d (2p-1) + (2p+1) +
 * one per moment (+ (2p+1)(2p+2)/2 in 3D) + n d FMAs, per element 3 per
 * moment combination of each block entry (+ 3 per (c, d) pair in 3D) and
 * 3 d (p+1)^2 (2p+1) for the coefficient tables). */
typedef struct {
  char name[48];
  float ms;
  double flops;
  double bytes;
} dg_kernel_stat;
int dg_set_timing(dg_ctx *ctx, int enable);
int dg_kernel_stats(dg_ctx *ctx, dg_kernel_stat *out, int cap);

/* Volume blocks without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (code running inside another framework's memory pool or under a
 * fixed memory budget, processes that must not grow their device footprint
 * after start-up).  The caller passes every input and output as its own
 * device buffers:
 *   x, y [nv] vertex coordinates; elem_ptr [ne+1], elem_idx [nsub] CCW vertex
 *   loops (nsub = elem_ptr[ne], the number of fan triangles); a [ne];
 *   blocks [ne * n * n] output, element-major, each n x n block row-major,
 *   n = (p+1)(p+2)/2, double for DG_PREC_FP64, float for DG_PREC_FP32;
 *   status (one int, may be NULL): set to DG_OK, or to DG_ERR_MESH when
 *   elem_ptr is not a list from 0 to nsub with at least 3 vertices per loop
 *   or a vertex id lies outside 0..nv-1.  The lists are checked on the GPU,
 *   and a bad list is replaced by a stand-in of the same sizes, so no access
 *   leaves the caller's buffers; the blocks of such a call are meaningless.
 * It computes, for every element of uniform degree p, the volume part of
 * Eq. (2.4) with advection (bx, by) and reaction c, exactly as
 * dg_assemble_volume does for the element's diagonal block.  Intermediate
 * records live in one file-scope device array of 16 MiB that every GPU
 * loading the library keeps until exit; ne <= 16384 and nsub <= 131072, and
 * larger meshes are rejected with DG_ERR_ARG before any CUDA call.  The first
 * call on a device looks up the array's device address and writes the
 * reference rules into it (synchronous copies): make that first call before
 * any stream capture.  Calls that overlap on the GPU share the array and
 * race; serialise them (one stream, or events).  Asynchronous on stream
 * (a cudaStream_t, NULL = legacy default stream) on device `device`; the
 * calling thread's current device is restored before the call returns. */
int dg_volume_noalloc(void *stream, int device, int prec, int p, int nv, const double *x, const double *y,
                      int ne, int nsub, const int *elem_ptr, const int *elem_idx, const double *a, double bx,
                      double by, double c, void *blocks, int *status);

/* Advection and reaction fields for dg_assemble_varcoef: an affine b and a
 * cubic c,
 *   b_d(x) = b0[d] + sum_e bx[d][e] x_e,   c(x) = sum_k c[k] m_k(x),
 * m_k the graded monomials of total degree <= 3 in the order of DG_SRC_POLY
 * (2D: the first 10; the z entries are ignored).  The fields of the paper's
 * multi-GPU test problem (Sec. 4.2) are b0 = (1, 1, 1), bx = I and c = 3 +
 * prod_d x_d (c[0] = 3, and c[4] = 1 in 2D, c[15] = 1 in 3D). */
typedef struct {
  double b0[3];
  double bx[3][3];
  double c[20];
} dg_fields;

/* The fields dg_assemble_varcoef uses on this mesh (copied; NULL: the Sec.
 * 4.2 fields, the default).  DG_ERR_ARG for a non-finite coefficient. */
int dg_mesh_set_fields(dg_mesh *mesh, const dg_fields *fields);

/* Variable advection and reaction: the mesh's fields (dg_mesh_set_fields)
 * evaluated at every quadrature point, with the inflow part of each face
 * decided point by point (b . n < 0; b . n = 0 is outflow) and no inflow
 * term on Neumann faces (Eq. (2.4)).  The mesh must be uploaded with b = 0
 * and c = 0 (DG_ERR_ARG otherwise): its a, C_sigma, Neumann sides and source
 * (DG_SRC_ZERO, DG_SRC_SINPROD or DG_SRC_POLY, with f = -a Lap u + b(x) .
 * grad u + c(x) u, g_D = u, g_N = a grad u . n) apply, and the call supplies
 * b(x) and c(x).  vals (device, nvals values) and rhs (device, ndofs values,
 * may be NULL) are OVERWRITTEN with the whole system in prec (DG_PREC_FP64,
 * or DG_PREC_FP32: FP32 geometry records, field table, basis and
 * accumulation): the row kernels write every term without b and c, then one
 * warp per element row adds the b and c terms of its blocks and load-vector
 * entries.  Each lane of that warp stages one quadrature point of a chunk of
 * 32 (basis values, weighted field row, load term) in shared memory; 25
 * lanes then contract the chunk into register tiles of the block.  2D and
 * 3D meshes from dg_mesh_upload or dg_batch_upload without learned rules;
 * DG_ERR_ARG otherwise.  Asynchronous on the context stream. */
int dg_assemble_varcoef_form(dg_ctx *ctx, dg_mesh *mesh, int prec, void *vals, void *rhs);
/* dg_assemble_varcoef_form with DG_PREC_FP64. */
int dg_assemble_varcoef(dg_ctx *ctx, dg_mesh *mesh, void *vals, void *rhs);

/* Space-time slabs (Sec. 2.3).  The slab (t0, t1] x D over an uploaded mesh
 * is cut into prisms kappa x (t0, t1].  A prism of degree p carries the
 * basis T_k(t) phi_j(x): T_k = sqrt((2k+1)/tau) P_k(2 (t - t0)/tau - 1), the
 * Legendre polynomials orthonormal on the slab (tau = t1 - t0), times the
 * element's spatial basis phi_j.  Its dofs i = (k, j) run k-major:
 *   DG_SPACE_P:  k = 0..p, j < nbasis(dim, p - k)  (space-time total degree <= p)
 *   DG_SPACE_PQ: k = 0..p, j < nbasis(dim, p)      (degree <= p in t and in x)
 * nbasis(2, q) = (q+1)(q+2)/2, nbasis(3, q) = (q+1)(q+2)(q+3)/6, and j follows
 * the spatial order, so j < nbasis(dim, q) is exactly the degree <= q part.
 *
 * The slab system is the time-discontinuous Galerkin form of Sec. 2.3 for
 * u_t - div(a grad u) + b.grad u + c u = f with the mesh's coefficients,
 * source and Dirichlet data (all constant in time):
 *   int_(t0,t1] [(U_t, W) + B(U, W)] dt + (U(t0+), W(t0+))
 *     = int_(t0,t1] l(W) dt + (u_prev, W(t0+)),
 * B and l the spatial forms of Eqs. (2.4) and (2.5); a lateral face
 * F x (t0, t1] takes F's spatial penalty.  Its block pattern is the mesh's;
 * block (r, s) holds nt_r x nt_s entries, row-major, rows the test
 * functions of r, nt the dofs of a prism.
 *
 * HOST arithmetic only, no GPU: the slab offsets of a block pattern.
 * row_ptr [ne+1], col [nnzb] (the layout of dg_bsr_pattern), p [ne] degrees
 * (1..DG_PMAX_2D / DG_PMAX_3D); out: blk_off [nnzb+1] (offsets of the slab
 * blocks in vals) and dof_off [ne+1] (of each prism's entries in the load
 * vector), caller-owned host arrays, either may be NULL.  DG_ERR_ARG on a
 * bad dim, space, degree, row_ptr or column. */
#define DG_SPACE_P 0
#define DG_SPACE_PQ 1
int dg_slab_offsets(int dim, int ne, const int *row_ptr, const int *col, const int *p, int space,
                    int64_t *blk_off, int64_t *dof_off);

/* Sizes of the mesh's slab system: nvals block values, ndofs load-vector
 * entries (either pointer may be NULL).  Meshes from dg_mesh_upload and
 * dg_batch_upload; DG_ERR_ARG for a partition mesh or a bad space. */
int dg_slab_layout(const dg_mesh *mesh, int space, int64_t *nvals, int64_t *ndofs);

/* Assemble the slab system of (t0, t1] (t0 < t1, both finite):
 *   vals (device, the slab layout's nvals entries, double for DG_PREC_FP64,
 *     float for DG_PREC_FP32; OVERWRITTEN) the block values;
 *   rhs (device, ndofs entries of the same type, OVERWRITTEN; may be NULL)
 *     the load vector  rhs(k, j) = [k = 0] sqrt(tau) l_j + T_k(t0+) (M u_prev)_j,
 *     l the element's spatial load vector (constant-in-time data against
 *     T_k integrate to sqrt(tau) for k = 0 and to 0 otherwise) and M its
 *     spatial mass matrix;
 *   u_prev (device, the mesh's spatial ndofs entries in the same type; NULL
 *     = zero): the spatial coefficients of U(t0-), the previous slab's
 *     trace (dg_slab_trace) or the initial value's coefficients.
 * How: with the orthonormal T_k every block is
 *   A[(k, j), (l, m)] = [k = l] B[j, m] + [r = s] D_kl M[j, m],
 *   D_kl = int T_l' T_k dt + T_l(t0+) T_k(t0+)
 *        = sqrt((2k+1)(2l+1)) / tau (2 [k < l, k + l odd] + (-1)^(k+l)),
 * B the spatial block of Eq. (2.4).  The call runs the row kernels for B
 * and l, and once more for M (the volume pass with a = 0, b = 0, c = 1), into
 * library-owned device scratch of 2 nvals + ndofs entries of the spatial
 * layout (allocated at the first call, freed with the mesh), then one
 * expansion kernel writes vals and one writes rhs.  The volume path is the
 * context's (dg_set_volume_path).  DG_PREC_BF16X3 / DG_PREC_TF32X3:
 * DG_ERR_ARG.  Asynchronous on the context stream. */
int dg_assemble_slab(dg_ctx *ctx, dg_mesh *mesh, int prec, int space, double t0, double t1,
                     const void *u_prev, void *vals, void *rhs);

/* The slab step of dg_assemble_slab (same arguments; vals, rhs and u_prev
 * fixed for the graph's life) recorded as one CUDA graph: the spatial and
 * mass passes with their degree groups on forked streams, the expansion and
 * the load vector.  Replay with dg_graph_launch, free with dg_graph_free.
 * The scratch of the slab pass is allocated before the capture, so the call
 * must precede any stream capture by the caller. */
int dg_slab_graph_create(dg_ctx *ctx, dg_mesh *mesh, int prec, int space, double t0, double t1, const void *u_prev,
                         void *vals, void *rhs, dg_graph **out);

/* The trace U(t1-) of a slab solution in the spatial basis:
 *   u_end_j = sum_k U(k, j) T_k(t1),  T_k(t1) = sqrt((2k+1)/tau),
 * over the k that carry j.  U: device, the slab layout's ndofs entries;
 * u_end: device, the mesh's spatial ndofs entries, OVERWRITTEN; double for
 * DG_PREC_FP64, float for DG_PREC_FP32.  Asynchronous on the context stream. */
int dg_slab_trace(dg_ctx *ctx, const dg_mesh *mesh, int prec, int space, double t0, double t1, const void *U,
                  void *u_end);

/* Wait for all work on the context stream; reports device-side errors:
 * DG_ERR_CUDA for a failed launch, DG_ERR_TIMEOUT when a bounded device wait
 * (the persistent pass's, or dg_wait_probe's) ran out since the last
 * dg_sync (the context's status word, cleared by the call). */
int dg_sync(dg_ctx *ctx);

/* on != 0: the calls without a tuned launch shape (dg_assemble_step,
 * dg_assemble_host and dg_assemble_batch on a mesh and precision that
 * dg_graph_create has not tuned, and dg_graph_create without autotuning)
 * take the persistent pass where it serves the mesh (FP32; 2D degrees <= 5,
 * 3D degrees <= 3), else their usual launches.  Off by default. */
int dg_set_persistent(dg_ctx *ctx, int on);

/* Bound of each device-side wait of the context's passes, in seconds of
 * wall time (default 2; (0, 60]). */
int dg_set_wait_limit(dg_ctx *ctx, double seconds);

/* One launch of the persistent pass's bounded wait on flag (device, one int,
 * owned by the caller): it returns once *flag != 0 or after seconds of wall
 * time, in which case the next dg_sync returns DG_ERR_TIMEOUT.  A check of
 * the timeout path that needs no fault: a flag that nothing sets makes the
 * wait run out.  Asynchronous on the context stream. */
int dg_wait_probe(dg_ctx *ctx, const int *flag, double seconds);

/* Number of kernel launches issued by the last assembly call (for
 * accounting in benchmarks). */
int dg_last_launch_count(const dg_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
