/*
 * msgfem.h -- C ABI of the GB300 (sm_103a) MS-GFEM local stage.
 *
 * Multiscale-spectral GFEM for 3-D anisotropic linear elasticity on a
 * laminated beam (Benezech et al., arXiv 2211.13893).  The library computes,
 * for every overlapping subdomain Omega_j with oversampling domain Omega*_j:
 *   - the subdomain stiffness a_{Omega*_j} of trilinear hexahedra with
 *     ply-rotated orthotropic tensors (Sec. 2, Eqs. eq-hooke, weak_form,
 *     element_stiffness, restricted_bilinear_form);
 *   - the n_loc smallest eigenpairs of the A-harmonic local eigenproblem
 *     (Sec. 3.3, Eq. AHarmonicGeneralizeEigenProblem; matrix form
 *     Eq. algebraicAharmonic) and the local particular function (Eq. up_r);
 *   - the partition-of-unity weighted basis and its Galerkin contribution to
 *     the coarse problem (Eq. AHarmonic_coarse_space, Sec. 4.3-4.4,
 *     Eq. GFEM_coarse_approximation), and the coarse solution u^G.
 *
 * Geometry and numbering.  The mesh is a box of nx * ny * nz bricks of size
 * hx * hy * hz, or a structured mesh with given node coordinates (see
 * msgfem_mesh); node (i, j, k) sits at (i hx, j hy, k hz) and has global id
 * (i (ny+1) + j)(nz+1) + k; DoF 3 id + c holds displacement component c.
 * Element (i, j, k) has index (i ny + j) nz + k; layer k is ply k.  The x = 0
 * face is clamped (Gamma_D, zero displacement); the x = L face carries a
 * uniform compressive traction (-traction, 0, 0); the other faces are free.
 *
 * Decomposition.  The non-overlapping subdomains are an sx * sy box partition
 * in (x, y) over the full thickness (Sec. 3.1), subdomain (a, b) having index
 * j = a sy + b, or a list of element boxes (msgfem_partition.boxes).
 * Omega_j grows the box by `overlap` element layers, Omega*_j by
 * `oversampling` layers, both counted from the non-overlapping box and
 * clipped to the mesh (Secs. 3.3, 4.2).
 *
 * Memory and ownership.  All pointers passed in are owned by the caller and
 * are read (and copied where needed) during the call only.  Output arrays are
 * caller-allocated; an output pointer may be host or device memory (the
 * library checks with cudaPointerGetAttributes).  Device memory used by the
 * computation is owned by the handle: it is allocated by msgfem_setup with
 * cudaMalloc and released by msgfem_destroy.  Work is issued on the stream
 * given in msgfem_options (NULL = legacy default stream); every call returns
 * only after its results are complete on that stream.
 *
 * Errors.  Every call returns a status; msgfem_last_error gives a message.
 * Calls must come in the order setup -> local_spaces -> coarse_assemble ->
 * solve (MSGFEM_ESTATE otherwise); local_spaces may be repeated after
 * msgfem_update_angles.  Repeating a step discards the later ones: once a
 * repeated local_spaces (or coarse_assemble) call has accepted its
 * arguments, coarse_assemble (or solve) has to run again, also if the call
 * then fails.  A handle is not thread-safe.
 */
#ifndef MSGFEM_H
#define MSGFEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct msgfem* msgfem_h;

typedef enum {
  MSGFEM_OK = 0,
  MSGFEM_EINVAL = 1,    /* invalid argument or descriptor */
  MSGFEM_ENOMEM = 2,    /* device or host allocation failed */
  MSGFEM_ECUDA = 3,     /* a CUDA call failed */
  MSGFEM_ENOTSPD = 4,   /* a local matrix lost positive definiteness in a pivot */
  MSGFEM_ENOCONV = 5,   /* eigensolver hit max_iter; results are the last iterate */
  MSGFEM_ESTATE = 6     /* call out of order */
} msgfem_status;

/* Hexahedral mesh (Sec. 5.1: one element per ply through the thickness).
 *
 * kind 0, structured: nx * ny * nz elements.  With xyz == NULL it is the box of
 * bricks hx * hy * hz described above.  Otherwise xyz holds the coordinates of
 * every node, 3 doubles per node in the global node order (host or device
 * pointer, copied during msgfem_setup), hx, hy, hz are ignored, and each
 * element is the trilinear map of its 8 nodes (curved laminates such as a
 * C-section spar: index j then runs along the arc of the cross-section and k
 * through the thickness).  The boundary faces stay the index faces: i = 0
 * clamped, i = nx loaded.
 *
 * kind 1, hexahedron list (the general input of Sec. 3.1 / Sec. 4.1): n_nodes
 * nodes with coordinates node_xyz [n_nodes][3] and n_elems elements hex8
 * [n_elems][8] (0-based node ids, host pointers, copied) in the standard local
 * order: nodes 0-3 counterclockwise around the face zeta = 0 seen from zeta > 0,
 * nodes 4-7 above them, so that local directions 0->1, 0->3, 0->4 form a
 * right-handed frame.  The list may come in any node and element order, but the
 * layer-block factorisation of the local stage needs a structured block: the
 * elements must form an nx x ny x nz block and share one orientation, and the
 * 0->4 direction runs through the thickness (the plies).  msgfem_setup recovers
 * the (i, j, k) numbering (i along 0->1, j along 0->3, k along 0->4, from the
 * corner node that precedes no other; EINVAL with the reason otherwise) and
 * then nx, ny, nz, hx, hy, hz and xyz are ignored.  Every per-node or
 * per-element array of the calls (loads, angles, frames, elem_part, the
 * solutions of msgfem_solve, msgfem_schwarz_solve, msgfem_energy_error_noalloc
 * and msgfem_solution_errors) is in the list's own order; the local layouts
 * of msgfem_get_basis / msgfem_export_local and the element fields of the
 * warm start use the recovered structured numbering (msgfem_get_numbering).
 *
 * dirichlet_node (either kind; NULL = the face i = 0): per node 1 where all
 * three displacement components are clamped (Gamma_D, zero displacement),
 * 0 elsewhere.  The DoF classes and rigid-mode pins of the local stage assume
 * that Gamma_D is the face i = 0 of the structured numbering: flags that mark
 * anything else are refused (EINVAL). */
typedef struct {
  int nx, ny, nz;
  double hx, hy, hz;
  double traction;      /* magnitude of the compressive traction on x = L (MPa): the load is
                           the consistent nodal force of (-traction, 0, 0) over the i = nx face */
  const double* xyz;    /* NULL (box) or [(nx+1)(ny+1)(nz+1)][3] node coordinates */
  const double* load;   /* NULL: the traction above.  Else the right-hand side b of Eq.
                           fe_matrix_system as nodal forces, [(nx+1)(ny+1)(nz+1)][3] in the
                           global node order (host or device pointer, copied during
                           msgfem_setup; traction ignored); entries on the clamped face have
                           no effect.  A subdomain gets a particular function (Eq. up_r)
                           when the load has a non-zero entry on its B1 DoFs. */
  int kind;             /* 0 structured, 1 hexahedron list */
  int n_nodes, n_elems; /* kind 1 */
  const double* node_xyz;   /* kind 1: [n_nodes][3] */
  const int* hex8;      /* kind 1: [n_elems][8] */
  const unsigned char* dirichlet_node;   /* NULL or [nodes] 0 / 1 */
} msgfem_mesh;

/* Orthotropic ply material and fibre angles (Sec. 5.1).
 * E9 = {E11, E22, E33, G12, G13, G23, nu12, nu13, nu23} in the ply axes.
 * elem_angle_deg[(i ny + j) nz + k] is the fibre angle of element (i, j, k)
 * (host or device pointer).  The angle is measured in the element's ply
 * frame: elem_frame[9 e .. 9 e + 8] holds three orthonormal, right-handed
 * unit vectors a0, a1, a2 (row-major 3 x 3, global coordinates); the fibre is
 * cos(theta) a0 + sin(theta) a1 and a2 is the laminate normal.  NULL means
 * a0, a1, a2 = x, y, z for every element (theta from x toward y about +z).
 * The frames are copied during msgfem_setup (host or device pointer). */
typedef struct {
  const double* E9;
  const double* elem_angle_deg;
  const double* elem_frame;   /* NULL or [nx ny nz][9] */
} msgfem_plies;

/* Non-overlapping subdomains (Sec. 3.1): with n_boxes == 0 the regular
 * sx * sy box partition described above; otherwise n_boxes element boxes
 * boxes[4 j .. 4 j + 3] = {x0, x1, y0, y1} (elements [x0, x1) x [y0, y1) x
 * all k) that must tile the nx * ny element grid exactly (EINVAL otherwise);
 * subdomain j is box j and sx, sy are ignored.  Or elem_part: the part id
 * (0 .. P - 1, every id used) of every element, as a graph partitioner such as
 * ParMETIS gives it (Sec. 4.1); subdomain j is part j, and each part must be
 * an (i, j) box of the structured numbering through the full thickness (the
 * layer-block storage spans whole node layers; EINVAL naming the part
 * otherwise); n_boxes, boxes, sx and sy are then ignored.  Host pointers,
 * copied. */
typedef struct {
  int sx, sy;           /* subdomains along x and y */
  int n_boxes;          /* 0 or the number of explicit boxes */
  const int* boxes;     /* NULL or [n_boxes][4] */
  const int* elem_part; /* NULL or [elements] part ids */
} msgfem_partition;

/* MSGFEM_FP64: all arithmetic in FP64.  MSGFEM_MIXED: layer blocks, their
 * factorisation and the block solves in FP32, every solve refined to FP64
 * accuracy with FP64 stencil residuals; Gram products, Rayleigh-Ritz,
 * CholeskyQR2, residual checks and the coarse problem stay FP64. */
typedef enum { MSGFEM_FP64 = 0, MSGFEM_MIXED = 1 } msgfem_precision;

typedef struct {
  int precision;        /* msgfem_precision */
  int block;            /* subspace iteration block size p; 0 = n_loc + max(8, n_loc / 2) */
  int max_iter;         /* cap on the eigensolver's steps: subspace iterations, or block Krylov
                           block steps (thick restarts of the 96-column basis included: 12 steps
                           fill it, each restart adds 8); 0 = 100.  A capped run returns ENOCONV
                           with the last Rayleigh-Ritz pairs */
  double tol;           /* stop when ||theta E S^-1 T x - x||_T <= tol per wanted pair (or the
                           decrease stalls below 1e2 tol); 0 = 1e-7 */
  unsigned long long seed;  /* seed of the counter-based start-block generator */
  void* stream;         /* cudaStream_t to issue work on; NULL = default stream */
  int profile;          /* 1: time the phases with CUDA events (msgfem_get_profile) */
  int solver;           /* 0: block Krylov (block width 8, basis <= 96), 1: subspace iteration */
  int streams;          /* independent task groups run on their own streams (1..32); 0 = 16, and
                           msgfem_autotune may then choose up to 32 */
  int refine;           /* MSGFEM_MIXED: most FP64 correction steps after each FP32 solve: for
                           K, preconditioned CG steps with the FP32 factor as preconditioner;
                           for A11, refinement steps.  A subdomain stops once its relative
                           residual is below 1e-11 (CG) or 1e-13 (refinement, also when it
                           stops falling); 0 = 10 */
  int instances;        /* batch of S >= 1 copies of the mesh and partition, each with its own
                           element angles (elem_angle_deg holds S consecutive fields);
                           subdomain j of copy i is subdomain i N0 + j of the handle.  With
                           S > 1 the handle runs the local stage only (msgfem_coarse_assemble
                           returns EINVAL).  0 = 1 */
  int solve_kernel;     /* kernel of the 8-column block solves: 0 = build default (FP32: cp.async
                           ring, FP64: register streaming), 1 = cp.async ring (FP32 only),
                           2 = register streaming, one CTA per 64-row task, 3 = two-CTA
                           cluster per task (inner dimension split), 4 = the ring of 1 filled
                           by tensor-memory-accelerator copies, one 64 x 64 tile per copy
                           (FP32 only; a copy that does not arrive within a second makes the
                           call return MSGFEM_ECUDA); msgfem_autotune sets it */
  int factor_schedule;  /* layer-block factorisation: 0 = right-looking (per tile column: POTRF,
                           TRMM, update of the trailing matrix), 1 = left-looking (update of the
                           column by all finished columns, then POTRF, TRMM); same work, fewer
                           and longer tasks; msgfem_autotune sets it */
  int direct_launch;    /* 0: factorisation and block-solve schedules are captured once as CUDA
                           graphs and replayed; 1: their kernels are launched one by one (the
                           same kernels and order; for kernel profilers) */
  double wave_mb;       /* device memory (MiB) for the layer blocks, factors and block-solve
                           buffers.  Subdomains whose storage does not fit at once are processed
                           in waves that share one pool of this size (largest first, a wave
                           closed when the next subdomain no longer fits); results do not
                           depend on the grouping.  0 = 80 % of the device memory free at
                           set-up less room for the element matrices (one wave when everything
                           fits).  ENOMEM if one subdomain alone exceeds it */
  /* Device memory of the handle from the caller's allocator: dev_alloc(bytes, alloc_ctx)
     returns device memory of the current device, at least 256-byte aligned, or NULL
     (ENOMEM); dev_free(p, bytes, alloc_ctx) takes back a block (bytes as allocated).  Both
     are called on the thread of the API call, during msgfem_setup, msgfem_update_angles,
     msgfem_local_spaces, msgfem_autotune, msgfem_get_basis and msgfem_destroy; the
     library synchronises its stream before it frees a block.  Both NULL: cudaMalloc and
     cudaFree.  One of them NULL: EINVAL.  (The network handles of msgfem_warm.h and the
     fixed scratch array of msgfem_energy_error_noalloc do not use them.) */
  void* (*dev_alloc)(size_t bytes, void* alloc_ctx);
  void (*dev_free)(void* p, size_t bytes, void* alloc_ctx);
  void* alloc_ctx;
  int method;           /* local eigenproblem: MSGFEM_METHOD_MSGFEM (0) the A-harmonic problem on the
                           oversampling domain (Eq. AHarmonicGeneralizeEigenProblem) with the
                           particular functions; MSGFEM_METHOD_GENEO (1) the GenEO problem of
                           Eq. bilinearGeneralizeEigenProblem, the paper's comparison (Sec. 2.3):
                           a_{Omega_j}(phi, v) = lambda a_{Omega_j}(Xi_j phi, Xi_j v) on Omega_j
                           itself (oversampling must equal overlap, EINVAL otherwise) over all its
                           free DoFs, no A-harmonic constraint, no particular function; the coarse
                           space is span{R_j^T Xi_j phi_{j,k}} with the Galerkin projection (Sec. 2.4).
                           GenEO runs the block Krylov solver only (solver = 0) and takes no
                           start blocks (msgfem_set_start_block) */
  int factor_kernel;    /* MSGFEM_MIXED, kernel of the FP32 layer-block factorisation's tile GEMMs:
                           0 = FP32 FMA on the CUDA cores; 1 = the tensor cores (tcgen05.mma,
                           operands staged by TMA, each FP32 operand split exactly into three TF32
                           parts hi + mid + lo, the six products of weight down to 2^-22 summed
                           smallest first, FP32 accumulation in tensor memory); msgfem_autotune
                           sets it (1 only when its factor agrees with kernel 0's) */
  int tile_chol;        /* MSGFEM_MIXED: precision of the 64 x 64 tile Cholesky and inverse inside
                           the FP32 factorisation: 0 = FP64 (default), 1 = FP32 (a wave whose FP32
                           tile Cholesky meets a non-positive pivot is factorised again with FP64
                           tiles, and so are the later waves of the call).  FP32 tiles shorten
                           the factorisation's critical path (each of its steps waits on one
                           tile Cholesky), but their inverses are less accurate: on small
                           clamped subdomains the A11 refinement then stalls above its target
                           and the final eigen-residuals rise to 1e-4 */
  int factor_persistent;  /* MSGFEM_MIXED: 1 runs the FP32 factorisation of a wave as one persistent
                           cooperative launch (FMA tile kernel; every CTA takes tasks in a
                           topological order and waits, bounded by two seconds, on the
                           completion counter of the previous step of the task's chain)
                           instead of the graph-captured step schedule; the factors are the
                           same bit for bit.  0 = the step schedule.  msgfem_autotune sets it */
} msgfem_options;

enum { MSGFEM_METHOD_MSGFEM = 0, MSGFEM_METHOD_GENEO = 1 };

/* Phase timers (CUDA events on the handle's stream, milliseconds, summed over
 * calls since msgfem_setup or the last msgfem_reset_profile) and algorithmic
 * work of the last local stage.  Flop counts use the unpadded layer sizes n of
 * the nL node layers: factorisation of the block-tridiagonal matrix, per
 * matrix, sum_l n^3/3 [diagonal Cholesky] + (nL - 1) 2 n^3 [coupling block,
 * update of the next diagonal block]; one block solve (4 (nL - 1) + 2 nL) n^2 p. */
typedef struct {
  double assemble_ms;   /* element stiffness, stencils, layer blocks */
  double factor_ms;     /* layer-block Cholesky + inverses of K and A11 */
  double solve_ms;      /* all block triangular solves of the iteration */
  double iterate_ms;    /* the whole eigen-iteration including solves */
  double coarse_ms;     /* coarse_assemble + solve */
  double factor_flops;  /* per local stage */
  double solve_flops;   /* per local stage, all solve calls */
  long long launches;   /* kernel launches issued by the library (all calls) */
  int solve_calls;      /* block solves in the last local stage */
  double solve_bytes;   /* per local stage, all solve calls: factor blocks read (the
                           inverse diagonal blocks as triangles, the coupling blocks whole,
                           forward and backward) in the factor's precision, plus the FP64
                           right-hand side read and solution written */
  double stencil_ms;    /* stencil products (K, B, K + sigma B) inside the iteration */
  double ortho_ms;      /* Gram, block updates, CholeskyQR, basis rotations */
  double stencil_flops; /* per local stage: 18 flop per (node, neighbour) pair and column, 24 for the
                           fused K + sigma B pass */
  int waves;            /* waves of subdomains per local stage (msgfem_options.wave_mb) */
  double pool_mb;       /* size of the shared layer-block / factor / solve-buffer pool (MiB) */
  double factor_flops_inverse;   /* factor_flops plus the n^3/3 per layer of the explicit
                                    inverses of the diagonal factors that the solves use */
  double factor_flops_executed;  /* flops the factorisation's 64 x 64 tile tasks execute
                                    (padding, whole diagonal tiles and inverses included) */
} msgfem_profile;

/* Launch shapes chosen by msgfem_autotune and what it measured. */
typedef struct {
  int factor_schedule;  /* msgfem_options.factor_schedule chosen */
  int factor_streams;   /* stream groups of the factorisation schedules chosen (16 or 32) */
  double factor_ms[2][2];  /* factorisation of the measured wave: [right-, left-looking][16, 32
                              groups]; -1 = not run */
  int streams;          /* stream groups of the block-solve schedules (4, 8, 16 or 32) */
  int solve_kernel;     /* msgfem_options.solve_kernel value chosen (1 to 4) */
  double best_ms;       /* time of one application of the shift-invert operator to an 8-column
                           block of the measured wave (solves, refinement and stencils) */
  double solve_ms[4][4];   /* [streams 4, 8, 16, 32][kernel 1, 2, 3, 4]; -1 = not applicable or not run */
  int factor_kernel;    /* msgfem_options.factor_kernel chosen (mixed precision) */
  double factor_ms_tc[2][2];   /* as factor_ms with the tensor-core tile kernel; -1 = not run */
  double tc_factor_diff;       /* ||L_tc - L_fma||_F / ||L_fma||_F on the measured wave's subdomain
                                  with the widest K layer, both with the fastest FMA schedule;
                                  -1 = not run */
  double fma_factor_diff;      /* the same between the FMA kernel's two schedules (two summation orders:
                                  the factor's FP32 rounding level); the tensor-core kernel is adopted
                                  only when tc_factor_diff <= 2 fma_factor_diff and it is faster */
  int factor_persistent;       /* msgfem_options.factor_persistent chosen (mixed precision) */
  double factor_ms_persistent[2];   /* the persistent FMA factorisation, [right-, left-looking];
                                       -1 = not run */
} msgfem_tuning;

/* Per-subdomain diagnostics filled by msgfem_get_info. */
typedef struct {
  int n_star_dof;       /* DoFs of Omega*_j */
  int n1, n2, n3;       /* sizes of the DoF classes B1, B2, B3 (Sec. 4.3) */
  int floating;         /* 1 if Omega*_j does not touch the clamped face */
  int iterations;       /* eigensolver iterations used: block Krylov steps (thick restarts
                           included; a warm start that fell back to a cold one counts the cold
                           run) or subspace iterations */
  int basis_size;       /* coarse basis functions contributed (n_loc [+1]) */
  double residual;      /* max relative eigen-residual over the subdomain's n_loc pairs */
  int threshold_reached;   /* msgfem_coarse_assemble_threshold: 0 if every one of the n_loc
                              eigenvalues was below 1 / t (the basis may need a larger n_loc) */
  int cold_restart;     /* 1 if the subdomain's registered start block (msgfem_set_start_block)
                           did not lead to convergence and the block Krylov solver was run
                           again from the cold (seeded random) start */
  int n_loc;            /* eigenpairs of the subdomain in the last local stage (or import),
                           0 before the first */
} msgfem_subinfo;

/* Partition, DoF classes (Sec. 4.3) and partition of unity (Sec. 4.2) on the
 * host; copies the angles and allocates all device memory.  The handle is
 * written to *out.  Errors: EINVAL (sizes <= 0, overlap < 1, oversampling <
 * overlap, a subdomain without interior, boxes that do not tile the mesh,
 * non-finite coordinates or frames), ENOMEM, ECUDA. */
msgfem_status msgfem_setup(const msgfem_mesh* mesh, const msgfem_plies* plies,
                           const msgfem_partition* part, int overlap, int oversampling,
                           const msgfem_options* opt, msgfem_h* out);

/* Device storage that a problem needs, planned on the host without a handle
 * and without any CUDA call (node coordinates must then be a host pointer):
 * the same decomposition as msgfem_setup (Secs. 3.1, 4.2, 4.3: subdomains,
 * oversampling domains, DoF classes), the layer blocks, factors and
 * block-solve buffers of every subdomain in the precision of opt (NULL:
 * FP64), and their grouping into waves for opt->wave_mb (0: one wave, the
 * budget msgfem_setup derives from the free device memory is unknown here). */
typedef struct {
  int n_subdomains;     /* N (all instances) */
  int waves;            /* waves for the budget */
  double pool_mb;       /* pool of the largest wave (MiB), what msgfem_setup allocates for it */
  double blocks_mb;     /* storage of all subdomains together (MiB) */
  double largest_mb;    /* storage of the largest subdomain (MiB); a budget below it is ENOMEM */
  long long n_dof;      /* 3 (nx+1)(ny+1)(nz+1) */
  int max_star_dof;     /* largest oversampling domain (DoFs) */
} msgfem_plan_info;

/* Errors: EINVAL (as msgfem_setup), ENOMEM (one subdomain exceeds wave_mb;
 * *info still filled but waves = 0). */
msgfem_status msgfem_plan(const msgfem_mesh* mesh, const msgfem_partition* part, int overlap, int oversampling,
                          const msgfem_options* opt, msgfem_plan_info* info);

/* Replace the element angles (same layout as msgfem_plies.elem_angle_deg). */
msgfem_status msgfem_update_angles(msgfem_h h, const double* elem_angle_deg);

/* The local stage: element stiffness and subdomain matrices (Eqs.
 * element_stiffness, restricted_bilinear_form), the n_loc smallest eigenpairs
 * of Eq. AHarmonicGeneralizeEigenProblem per subdomain (block Krylov, or
 * subspace iteration with msgfem_options.solver = 1; shift-invert at zero,
 * Rayleigh-Ritz in FP64; the six rigid modes of a floating subdomain are
 * exact zero eigenpairs and count in n_loc) and the particular functions
 * (Eq. up_r), wave by wave when the factors do not fit at once
 * (msgfem_options.wave_mb).  lambda_out (N * n_loc doubles, subdomain-major,
 * ascending; may be NULL; host or device) receives the eigenvalues.  Errors:
 * EINVAL (n_loc outside 1 .. 31 (a subdomain's eigenvectors and its
 * particular function fill at most 32 basis columns) or larger than the
 * A-harmonic space of a subdomain),
 * ENOTSPD, ENOCONV (results are the last iterate; msgfem_subinfo gives each
 * subdomain's residual), ECUDA. */
msgfem_status msgfem_local_spaces(msgfem_h h, int n_loc, double* lambda_out);

/* msgfem_local_spaces with its own n_loc for every subdomain: the local basis
 * sizes m_j of Eq. AHarmonic_coarse_space, which differ between subdomains
 * (Sec. 5.3: interior subdomains need more eigenvectors for the same local
 * error; Sec. 5.5: m_j from 60 to 170 on the C-spar).  n_loc: N ints
 * (host or device, copied), n_loc[j] eigenpairs of subdomain j, each within the limits of
 * msgfem_local_spaces.  lambda_out (may be NULL; host or device) receives
 * N * n_max doubles, n_max the largest n_loc[j], subdomain-major; entries
 * c >= n_loc[j] of row j are NaN.  msgfem_get_basis and msgfem_export_local
 * then give n_max columns per subdomain, columns c >= n_loc[j] zero (and
 * NaN eigenvalues); msgfem_coarse_assemble keeps the n_loc[j] eigenvectors
 * of subdomain j, msgfem_coarse_assemble_threshold at most as many.
 * msgfem_local_spaces(h, n, out) is this call with every n_loc[j] = n.
 * Errors as msgfem_local_spaces; EINVAL also for n_loc NULL. */
msgfem_status msgfem_local_spaces_var(msgfem_h h, const int* n_loc, double* lambda_out);

/* PoU-weighted basis with Gram-Schmidt and the appended particular function
 * (Sec. 4.3-4.4), coarse matrix A^H_{ij} = V_i^T A V_j and load b^H
 * (Eq. GFEM_coarse_approximation).  *coarse_dim_out receives dim V_H. */
msgfem_status msgfem_coarse_assemble(msgfem_h h, int* coarse_dim_out);

/* msgfem_coarse_assemble with local basis sizes chosen by an eigenvalue
 * threshold (Sec. 5.5, Sec. 5.6; the error bound of Thm. error_bound is driven
 * by 1 / lambda_{j, m_j + 1}): subdomain j keeps its eigenvectors with
 * 1 / lambda > t (rigid modes always), m_j <= the subdomain's n_loc in the
 * last local stage; t = 0 keeps all of them (msgfem_coarse_assemble).  When all
 * of a subdomain's eigenvalues are below 1 / t its
 * msgfem_subinfo.threshold_reached is 0.
 * Errors: EINVAL (t < 0), ESTATE, ENOTSPD. */
msgfem_status msgfem_coarse_assemble_threshold(msgfem_h h, double t, int* coarse_dim_out);

/* Coarse solve A^H c = b^H (FP64 Cholesky) and u^G = sum_j V_j c_j.
 * u_out receives u^G on all 3 (nx+1)(ny+1)(nz+1) DoFs (may be NULL).  If
 * u_ref is not NULL (fine solution u_h, same layout), *energy_err_out
 * receives ||u_ref - u^G||_a / ||u_ref||_a (Theorem 1). */
msgfem_status msgfem_solve(msgfem_h h, double* u_out, const double* u_ref, double* energy_err_out);

/* Eigenvectors of subdomain j on the DoFs of Omega*_j, column-major
 * n_star_dof * n_loc, normalised phi^T B phi = 1 (B as in Eq.
 * algebraicAharmonic).  Node (i, j, k) of the Omega*_j node box
 * [i0, i1] x [j0, j1] x [0, nz] has local id ((i - i0)(j1 - j0 + 1) + (j - j0))(nz + 1) + k
 * and local DoFs 3 id + c; DoFs in B3 are zero.  *rows and *cols receive the
 * shape; phi_out may be NULL to query it (also before msgfem_local_spaces;
 * *cols is then the n_loc of the last local stage, 0 before the first).  box_out (may be NULL) receives the
 * Omega*_j node box {i0, i1, j0, j1}. */
msgfem_status msgfem_get_basis(msgfem_h h, int j, double* phi_out, int* rows, int* cols, int* box_out);

/* Checkpoint of the local stage (the offline / online reuse of local bases
 * the paper suggests, Sec. 6): subdomain j's n_loc eigenpairs and its
 * particular function (Eq. up_r).  phi_out (may be NULL): n_star_dof *
 * (n_loc + 1) doubles, column-major in the layout of msgfem_get_basis, the
 * n_loc eigenvectors followed by psi_j (zero when the load does not reach
 * B1); lambda_out (may be NULL): n_loc doubles.  Host or device pointers.
 * Errors: EINVAL, ESTATE (before msgfem_local_spaces), ENOMEM, ECUDA. */
msgfem_status msgfem_export_local(msgfem_h h, int j, double* phi_out, double* lambda_out);

/* Resume from exported local spaces: on a handle set up like the exporting one
 * (same mesh, angles, partition, loads), assembles the element and subdomain
 * matrices as msgfem_local_spaces does and takes the eigenpairs and particular
 * functions from lambda (N * n_loc doubles, subdomain-major) and phi (N
 * pointers, each as phi_out of msgfem_export_local) instead of solving for
 * them; the handle is then ready for msgfem_coarse_assemble.  A row of lambda
 * may end in NaN entries, as msgfem_local_spaces_var writes them: subdomain j
 * then keeps the eigenpairs before its first NaN.  Host or device pointers,
 * copied.  Errors: EINVAL (NULL, n_loc outside 1 .. 31 or above a
 * subdomain's B2 size, an infinite eigenvalue, a NaN followed by a number, a
 * row without eigenvalues), ESTATE (before msgfem_setup), ENOMEM, ECUDA. */
msgfem_status msgfem_import_local(msgfem_h h, int n_loc, const double* lambda, const double* const* phi);

/* Energy error ||u_ref - u||_a / ||u_ref||_a of two caller-owned device
 * vectors (3 (nx+1)(ny+1)(nz+1) doubles each, the layout of msgfem_solve), the
 * same quantity msgfem_solve reports, computed without allocating any memory.
 * The paper has no counterpart: this is a library convenience.
 *
 * Why it exists: some callers cannot call cudaMalloc at the point where they
 * evaluate a solution -- for example an application whose device memory is
 * already committed to another framework's memory pool, or a latency-bound loop
 * that must not enter the driver's allocator, which can synchronise the device.
 * msgfem_solve needs its handle-owned staging buffer for u_ref; this entry point
 * reads the caller's device vectors in place and keeps its partial sums in a
 * fixed 64 KiB array in device global memory that every GPU loading the library
 * holds until the process exits.  It calls no allocating routine.
 *
 * Limits and behaviour: the mesh may have at most 4,194,304 elements (EINVAL
 * with a message otherwise); u and u_ref must be device pointers (EINVAL);
 * the handle must have run msgfem_local_spaces (ESTATE), whose element
 * stiffness is reused.  energy_err_out may be a host pointer (the call then
 * copies the result back and waits for it; ESTATE while the handle's stream is
 * being captured) or a device pointer (written on the handle's stream).
 * msgfem_setup looks up the device address of the array on the device current
 * during set-up (the handle's device); this call must be made with that device
 * current (EINVAL otherwise) and has nothing left to look up or load.  All
 * calls share the one array and each call overwrites every slot it reads, so
 * consecutive calls are independent, but calls whose kernels overlap on the
 * GPU (other streams, other threads, other handles) race on the array and
 * must be serialised by the caller. */
msgfem_status msgfem_energy_error_noalloc(msgfem_h h, const double* u, const double* u_ref, double* energy_err_out);

/* Relative L2 errors (Sec. 5.4) of the coarse solution u^G of the last
 * msgfem_solve against a reference u_ref ([3 n_nodes] doubles, node-major as
 * u_out of msgfem_solve; host or device; copied):
 *   errors_out[0] = e_d   = ||u_ref - u^G|| / ||u_ref||,
 *   errors_out[1] = e_eps = ||eps(u_ref - u^G)|| / ||eps(u_ref)||,
 * with the norms of L2(Omega) of the finite element fields, integrated over
 * every element by 2x2x2 Gauss quadrature through its trilinear map (node
 * coordinates or the box), and eps : eps (tensor components) as the strain's
 * pointwise square.  The paper writes ||.||_2 without saying whether the
 * vector or the field norm is meant; the field norm is taken.  errors_out: 2
 * doubles, host.  A reference with zero norm gives 0.  Errors: EINVAL (NULL
 * argument), ESTATE (no msgfem_solve since the last local stage or coarse
 * assembly), ECUDA. */
msgfem_status msgfem_solution_errors(msgfem_h h, const double* u_ref, double* errors_out);

/* Autotuner of the factorisation and block-solve launches (not in the paper:
 * a library convenience for batches of uneven subdomains).  On the subdomains
 * of the last wave of the previous msgfem_local_spaces call it first times the
 * layer-block factorisation with the right- and the left-looking schedule,
 * dealt into 16 or 32 stream groups (re-assembling the layer blocks before
 * each run), in mixed precision with the FMA and with the tensor-core tile
 * kernel (msgfem_options.factor_kernel; the latter only when its factor passes
 * the accuracy gate of msgfem_tuning.fma_factor_diff), and keeps the fastest;
 * then, for every combination of stream groups {4, 8, 16, 32} (at most
 * msgfem_options.streams) and solve kernel (register streaming, two-CTA
 * cluster, and in mixed precision the cp.async ring and the TMA-filled ring),
 * it times `reps` (0 = 3) applications of the shift-invert operator as the
 * eigensolver makes them, back to back on a fresh random block each (the
 * N-product stencil, the 8-column K solve with, in mixed precision, its PCG
 * refinement, and the A-harmonic extension by A11 solves), after one untimed
 * application, then regroups the solve schedules of every wave and sets the
 * kernel to the fastest combination; later calls use it.  The working blocks
 * the timing reads and writes are scratch of the eigensolver; results of the
 * previous local stage, the phase timers and the launch count are kept.
 * tuning (may be NULL) receives the choice and the measured times.  Errors:
 * ESTATE before msgfem_local_spaces, ECUDA. */
msgfem_status msgfem_autotune(msgfem_h h, int reps, msgfem_tuning* tuning);

/* Two-level additive Schwarz preconditioned conjugate gradients for the fine
 * problem A u = b (Eq. fe_matrix_system) on the free DoFs: the solver that a
 * coarse space preconditions (Sec. 2.3, Eq. condition_bound) and the paper's
 * reference solver for u_h (Sec. 5.3-5.4).  The preconditioner is
 *   M^{-1} r = sum_j R_j^T A_j^{-1} R_j r + V A_0^{-1} V^T r,
 * R_j the restriction to the DoFs of Omega_j off its cut boundary and off the
 * clamped face, A_j = R_j A R_j^T (Dirichlet problems on the overlapping
 * subdomains), V the coarse basis and A_0 = V^T A V.
 *   local: a handle set up with oversampling equal to overlap (Omega*_j =
 *          Omega_j, so its A11 factors are the A_j), one instance, one wave;
 *          its layer blocks are assembled and factored here unless its last
 *          msgfem_local_spaces left them in place (a GenEO handle's do).
 *   coarse: a handle of the same mesh after msgfem_coarse_assemble (MS-GFEM or
 *          GenEO coarse space; may be `local` itself), or NULL for the
 *          one-level method.  Its coarse right-hand side is restored on exit.
 *   b:     all 3 n_nodes DoFs (host or device; clamped entries ignored), or
 *          NULL for the local handle's own load.
 *   u0:    start vector (all DoFs, host or device), or NULL for zero; the
 *          coarse solution u^G of msgfem_solve is a good one.
 *   rtol:  stop when ||b - A u||_2 <= rtol ||b||_2 over the free DoFs (0 = 1e-10);
 *   max_iter: 0 = 2000.  u_out (all DoFs, host or device) receives u.
 *   info (may be NULL): iterations, final relative residual and the extreme
 *          eigenvalues of M^{-1} A estimated from the CG coefficients (the
 *          Lanczos matrix), and their ratio.
 * Runs on the local handle's stream; uses the working blocks of both handles'
 * eigensolvers as scratch (their local spaces and coarse problems are kept).
 * Errors: EINVAL, ESTATE (no coarse problem on `coarse`), ENOCONV (max_iter
 * reached; u_out holds the last iterate), ENOTSPD (CG broke down), ENOMEM,
 * ECUDA. */
typedef struct {
  int iterations;
  double residual;
  double lambda_min, lambda_max, kappa;
} msgfem_pcg_info;

msgfem_status msgfem_schwarz_solve(msgfem_h local, msgfem_h coarse, const double* b, const double* u0, double rtol,
                                   int max_iter, double* u_out, msgfem_pcg_info* info);

/* Arithmetic throughput probe (not in the paper: the measured counterpart of
 * the ALU peaks that bound the layer-block factorisation): dependent-chain FMA
 * loops on every SM of the current device, FP64 (precision MSGFEM_FP64) or
 * FP32 (MSGFEM_MIXED), timed with CUDA events on the default stream after a
 * warm-up launch, best of three.  *tflops receives the rate in TFLOP/s (2 flops per FMA),
 * *sm_count_out (may be NULL) the SM count.  Uses a small cudaMalloc'ed
 * buffer of its own.  Errors: EINVAL, ENOMEM, ECUDA. */
msgfem_status msgfem_probe_fma(int precision, double* tflops, double* sm_count_out);

/* The structured numbering the handle works in (see msgfem_mesh): dims (may be
 * NULL) receives {nx, ny, nz}; node_of_user[u] (may be NULL; n_nodes ints) the
 * structured id (i (ny+1) + j)(nz+1) + k of node u of the caller's mesh and
 * elem_of_user[e] (may be NULL; n_elems ints) the structured index
 * (i ny + j) nz + k of element e; identities for a structured mesh.  Host
 * pointers.  Errors: EINVAL. */
msgfem_status msgfem_get_numbering(msgfem_h h, int* dims, int* node_of_user, int* elem_of_user);

msgfem_status msgfem_get_info(msgfem_h h, int j, msgfem_subinfo* info);
/* Copy the phase timers (requires msgfem_options.profile = 1 for times). */
msgfem_status msgfem_get_profile(msgfem_h h, msgfem_profile* out);
msgfem_status msgfem_reset_profile(msgfem_h h);
int msgfem_num_subdomains(msgfem_h h);
const char* msgfem_last_error(msgfem_h h);
void msgfem_destroy(msgfem_h h);

#ifdef __cplusplus
}
#endif
#endif
