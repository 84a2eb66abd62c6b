/*
 * ufe.h -- C ABI of the GB300 BDDC-PCG solver for unfitted (cut-cell) Q1
 * finite elements on a Cartesian background mesh (Badia & Verdugo,
 * "Robust and scalable domain decomposition solvers for unfitted finite
 * element methods").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Grid: nx*ny*nz cubic cells on the box [lo, hi]; nodes are numbered
 *    i + (nx+1)*(j + (ny+1)*k), cells i + nx*(j + ny*k) (x fastest).
 *  * The physical domain is {phi < 0} (Sect. 2.1: the boundary is the zero
 *    level set); phi == 0 counts as outside.
 *  * Array arguments are caller-owned and only borrowed for the duration of
 *    the call.  Each call that takes arrays also takes `mem`: UFE_MEM_HOST
 *    (pageable or pinned host memory; the library copies) or UFE_MEM_DEVICE
 *    (CUDA device pointers on the current device, read on the handle's stream).
 *  * Handles are opaque and library-owned; release them with *_destroy.
 *    A system borrows its mesh and a bddc borrows its system: destroy in the
 *    reverse order of creation.
 *  * All work is issued on the stream given to ufe_mesh_create (NULL = the
 *    legacy default stream) and every call returns after its results are
 *    complete (the calls synchronise that stream).
 *  * Errors: a negative ufe_status; ufe_last_error() returns a message for the
 *    calling thread.  Outputs are unspecified after an error, except
 *    UFE_ERR_NO_CONVERGENCE, after which x holds the last iterate and the
 *    info struct is filled.
 *  * Every kernel behind these calls is a hand-written sm_103a kernel; there
 *    is no host or library fallback for any step.
 */
#ifndef UFE_H
#define UFE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ufe_status;

#define UFE_OK                   0
#define UFE_ERR_INVALID_ARG     -1
#define UFE_ERR_OUT_OF_MEMORY   -2
#define UFE_ERR_CUDA            -3
#define UFE_ERR_SINGULAR_LOCAL  -4   /* a local Dirichlet or constrained-Neumann matrix is not SPD */
#define UFE_ERR_SINGULAR_COARSE -5   /* the assembled coarse matrix is not SPD */
#define UFE_ERR_BREAKDOWN       -6   /* PCG: p.Ap <= 0 */
#define UFE_ERR_NO_CONVERGENCE  -7   /* PCG: maxit reached; x holds the last iterate */
#define UFE_ERR_UNSUPPORTED     -8
#define UFE_ERR_TIMEOUT         -9   /* a bounded device-side loop hit its iteration limit */

#define UFE_MEM_HOST   0
#define UFE_MEM_DEVICE 1

/* cell types (Sect. 2.1) */
#define UFE_CELL_EXTERNAL 0
#define UFE_CELL_CUT      1
#define UFE_CELL_INTERNAL 2

/* object kinds (Sect. 3.2) */
#define UFE_OBJ_CORNER 0
#define UFE_OBJ_EDGE   1
#define UFE_OBJ_FACE   2

/* ufe_bddc_opts.weighting */
#define UFE_WEIGHT_STIFFNESS   0   /* Eq. alge-weighting (Sect. 4.3) */
#define UFE_WEIGHT_TOPOLOGICAL 1   /* Eq. weighting (Sect. 3.3) */
/* ufe_bddc_opts.objects */
#define UFE_OBJECTS_STANDARD 0     /* Sect. 3.2 */
#define UFE_OBJECTS_VARIANT1 1     /* Sect. 4.4: cut coarse edges split */
#define UFE_OBJECTS_VARIANT2 2     /* Sect. 4.5: coarse edges split into runs of equal stiffness weights
                                      (two weights equal when they differ by at most 1e-8); Poisson */
/* ufe_bddc_opts.coarse: which objects carry a coarse DOF (Sect. 3.2) */
#define UFE_COARSE_C   0
#define UFE_COARSE_CE  1
#define UFE_COARSE_CEF 2
/* ufe_bddc_opts.precision */
#define UFE_PREC_FP64  0           /* every local factor and product in FP64 */
#define UFE_PREC_MIXED 1           /* Jacobi-scaled FP32 local operators; FP64 PCG, weights, coarse */

/* ufe_bddc_opts.coarse_solver: how u_c = A_c^-1 r_c is computed (no paper counterpart;
 * both are exact FP64 solves of the same coarse problem) */
#define UFE_COARSE_SOLVER_AUTO  0  /* dense inverse up to 2048 coarse DOFs, else cyclic reduction */
#define UFE_COARSE_SOLVER_DENSE 1  /* explicit FP64 inverse of A_c (n_coarse up to ~28,000: r_c in one CTA's shared memory) */
#define UFE_COARSE_SOLVER_CR    2  /* FP64 block cyclic reduction over the z layers of subdomain blocks */
#define UFE_COARSE_SOLVER_BDDC  3  /* three-level method: the coarse problem is not solved but
                                      preconditioned by BDDC over groups of coarse_group^3 blocks of
                                      subdomains, whose own coarse problem is inverted in FP64 */

#define UFE_PIN_NONE -1
#define UFE_PIN_AUTO -2

typedef struct ufe_mesh ufe_mesh;
typedef struct ufe_system ufe_system;
typedef struct ufe_bddc ufe_bddc;

/* Message describing the last error of the calling thread ("" if none). */
const char* ufe_last_error(void);

/* ABI version of this header (major * 100 + minor). */
int ufe_version(void);

/* Number of library kernels launched by this process so far (every kernel node
 * of a launched CUDA graph counts once).  Instrumentation only; no paper
 * counterpart. */
int64_t ufe_kernel_launches(void);

/* Kernel timing (instrumentation only; no paper counterpart).  While enabled, the
 * library brackets every launch of the named set-up kernels with CUDA events on
 * the stream it launches them on:
 *   "gj_update_f64"  FP64 Gauss-Jordan update step (coarse matrix; local matrices in FP64 mode)
 *   "gj_update_f32"  FP32 Gauss-Jordan update step (local matrices in mixed precision)
 *   "gj_lookahead_f64", "gj_lookahead_f32"  block row / column K+1 of each step with the
 *                    next diagonal-block inverse
 *   "gj_panel_f64", "gj_panel_f32"  the row panel of each Gauss-Jordan step
 *   "gj_diag_f64", "gj_diag_f32"  the first diagonal-block inverse
 *   "integrate_cut"  marching-tetrahedra cut-cell integration
 * the per-iteration kernels when they run outside a CUDA graph (ufe_system_apply,
 * ufe_bddc_apply and the first preconditioner application of ufe_pcg_solve):
 *   "apply"          operator apply y = A x
 *   "prec_interior"  y_I = A_II^-1 r_I, t_G = A_GI y_I
 *   "prec_neumann"   weighted restriction, constrained Neumann solve, coarse residual parts
 *   "coarse_solve"   u_c = A_c^-1 r_c
 *   "prec_prolong"   coarse prolongation Phi u_c
 *   "prec_final"     weighted average and harmonic extension
 * and the phases "phase_mesh", "phase_assemble", "phase_objects", "phase_local",
 * "phase_factor", "phase_coarse", "phase_solve" (events around the host code of
 * each phase, so they include its synchronisations and host work).
 * ufe_timing_get sums the elapsed device time (ms) and the launch count of one
 * name since the last reset (it synchronises on the recorded events).
 * Unknown names return UFE_ERR_INVALID_ARG. */
void ufe_timing_enable(int on);
void ufe_timing_reset(void);
ufe_status ufe_timing_get(const char* kernel, double* total_ms, int64_t* launches);

/* Measured FMA rate of the current device (instrumentation only; no paper
 * counterpart): an FMA-loop kernel with eight independent chains per thread and
 * four 256-thread CTAs per SM, timed by CUDA events on `stream` (NULL: the legacy
 * default stream) after one warm-up launch.  kind 0: FP64, 1: FP32 (SIMT pipes).
 * *tflops receives 2 flops per FMA over the elapsed time, in TFLOP/s; it is the
 * denominator of the ALU rooflines the benchmark reports. */
ufe_status ufe_probe_fma_rate(int kind, void* stream, double* tflops);

typedef struct {
  int64_t n_nodes, n_cells;
  int64_t n_active_cells, n_cut_cells;
  int64_t n_dof;               /* free DOFs */
  int64_t n_subdomains;
  int64_t n_interface_dofs;    /* DOFs with |neigh| >= 2 */
  int64_t pinned_node;         /* node id of the pinned node, -1 if none */
  int64_t n_constrained;       /* box-face Dirichlet nodes plus the pinned node */
  int32_t max_interior, max_interface;   /* largest local interior / interface sizes */
} ufe_mesh_info;

/*
 * ufe_mesh_create -- background mesh, cell classification, DOFs and subdomains.
 *
 * Sect. 2.1 (cell partition: internal / external / cut, active = internal or
 * cut; subdomains by aggregation of active cells) and Sect. 5.1 (strong
 * Dirichlet on box faces; one pinned node when no box face is Dirichlet).
 *
 *  box_lo, box_hi   3 doubles each (host); cells must be cubes (equal spacing).
 *  cells            3 ints (host): nx, ny, nz >= 1.
 *  sub_cells        3 ints (host): cells per subdomain block edge, 1..16, dividing cells.
 *  phi_nodes        (nx+1)(ny+1)(nz+1) doubles, nodal level set; memory per `mem`.
 *  dirichlet_face_mask  bit f set = strong Dirichlet on box face f (x-,x+,y-,y+,z-,z+).
 *  pin_node         UFE_PIN_NONE, UFE_PIN_AUTO (pin the node whose 8 cells are
 *                   internal with the smallest phi, ties -> lowest id, only if no
 *                   box-face node is constrained), or an explicit active node id.
 *  stream           cudaStream_t used by every call on this mesh and its children.
 *  out              receives the new handle.
 * DOFs are the nodes of active cells minus the constrained ones, numbered in node
 * order.  A subdomain is a connected component (cells sharing a DOF) of the
 * active cells of one block, ordered by (block, smallest cell id).
 * Errors: INVALID_ARG for bad sizes / pin, CUDA, OUT_OF_MEMORY, TIMEOUT.
 */
ufe_status ufe_mesh_create(const double box_lo[3], const double box_hi[3], const int32_t cells[3],
                           const int32_t sub_cells[3], const double* phi_nodes, int mem,
                           uint32_t dirichlet_face_mask, int64_t pin_node, void* stream,
                           ufe_mesh** out);
ufe_status ufe_mesh_get_info(const ufe_mesh* mesh, ufe_mesh_info* info);
/* cell_types: n_cells bytes (UFE_CELL_*). */
ufe_status ufe_mesh_get_cell_types(const ufe_mesh* mesh, uint8_t* cell_types, int mem);
/* dof_of_node: n_nodes int32, -1 for nodes that are not free DOFs. */
ufe_status ufe_mesh_get_dof_map(const ufe_mesh* mesh, int32_t* dof_of_node, int mem);
/* sub_of_cell: n_cells int32, -1 for external cells. */
ufe_status ufe_mesh_get_subdomains(const ufe_mesh* mesh, int32_t* sub_of_cell, int mem);
/* neigh: n_dof * 8 int32: sorted subdomain ids of neigh(xi) (Sect. 3.3), padded with -1. */
ufe_status ufe_mesh_get_neighbours(const ufe_mesh* mesh, int32_t* neigh, int mem);
void ufe_mesh_destroy(ufe_mesh* mesh);

/*
 * ufe_assemble -- cut-cell integration and the global right-hand side.
 *
 * Sect. 2.2 bulk form A_e(u,v) = int_{e cap Omega} kappa_e grad u . grad v with
 * Neumann data on the unfitted boundary; the cut part of each cut cell is
 * integrated by marching tetrahedra (6 Kuhn tets per cube, phi linear on each)
 * with degree-7 Grundmann-Moeller rules; internal cells use the closed-form Q1
 * matrices.  b = int f_h phi_a + int_{Gamma cap e} (q_h . n) phi_a minus the
 * strong Dirichlet lift (Sect. 2.2, 5.1).
 *
 *  kappa_cells       n_cells doubles (per-cell coefficient) or NULL for 1.
 *  f_nodes           n_nodes doubles: nodal source (Q1 interpolated), or NULL for 0.
 *  flux_nodes        n_nodes*3 doubles (x,y,z per node): nodal flux q, Neumann
 *                    data g = q . n on the cut boundary; NULL for g = 0.
 *  dirichlet_values  n_nodes doubles read at the constrained nodes; NULL for 0.
 * All arrays live in memory `mem`.  The system keeps a pointer to the mesh.
 */
ufe_status ufe_assemble(ufe_mesh* mesh, const double* kappa_cells, const double* f_nodes,
                        const double* flux_nodes, const double* dirichlet_values, int mem,
                        ufe_system** out);
/*
 * ufe_assemble_nitsche -- Poisson with weak Dirichlet data on the unfitted boundary
 * (Sect. 2.2, Nitsche's method; the boundary condition of the paper's Dirichlet
 * experiments, Sect. 5.1).  Each cut cell's form gains
 *   int_{Gamma cap e} ( beta_e u v - v (n . grad u) - u (n . grad v) ) dS
 * and its load int_{Gamma cap e} ( beta_e v g - (n . grad v) g ) dS, with g the Q1
 * interpolant of dirichlet_values, n the outward normal of the marching-tetrahedra
 * boundary and beta_e = 2 C_e, C_e the largest eigenvalue of the cell's generalised
 * eigenproblem B_e x = C D_e x (Eq. local-eigenvals; D_e the cut-cell stiffness, B_e
 * the boundary form of the normal derivatives; both vanish on the constants).  Box
 * faces of the mesh's dirichlet_face_mask keep strong Dirichlet values; use
 * ufe_mesh_create with pin_node = -1 (the weak condition fixes the constant).
 *
 *  f_nodes           n_nodes doubles: nodal source (Q1 interpolated), or NULL for 0.
 *  dirichlet_values  n_nodes doubles: the Dirichlet data, weak on the unfitted
 *                    boundary and strong at the constrained box nodes (required).
 * Errors: INVALID_ARG, SINGULAR_LOCAL (a cell's eigenproblem has no positive
 * largest eigenvalue), CUDA, OUT_OF_MEMORY.
 */
ufe_status ufe_assemble_nitsche(ufe_mesh* mesh, const double* f_nodes, const double* dirichlet_values, int mem,
                                ufe_system** out);
/* beta: n_cut doubles, the Nitsche coefficient beta_e of each cut cell in cut-cell order
 * (physical units, 0 for a cell without boundary area); INVALID_ARG for a system
 * assembled without weak Dirichlet data. */
ufe_status ufe_system_get_nitsche_beta(const ufe_system* sys, double* beta, int mem);
/*
 * ufe_assemble_elastic -- the vector-valued (Q1^3) variant: isotropic linear
 * elasticity on the same unfitted mesh (no counterpart in the paper, which treats
 * the Poisson problem; same bulk-form integration, natural boundary condition on
 * the unfitted boundary).
 *   a_e(u,v) = int_{e cap Omega} s_e (lambda div u div v + 2 mu eps(u) : eps(v)),
 *   lambda = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu)).
 * The system has 3 DOFs per free node d, numbered 3 d + c (component c = x, y, z);
 * element DOF 3 a + c of vertex a.  The Dirichlet box faces of the mesh clamp all
 * three components; use ufe_mesh_create with pin_node = -1 (no pinned node).
 *
 *  E, nu             material (E > 0, -1 < nu < 1/2).
 *  E_scale_cells     n_cells doubles s_e scaling the element matrix, or NULL for 1.
 *  f_nodes           n_nodes*3 doubles: nodal body force (Q1 interpolated).
 *  stress_nodes      n_nodes*9 doubles: nodal stress sigma (row-major), the boundary
 *                    traction is sigma n on the cut boundary; NULL for traction-free.
 *  dirichlet_values  n_nodes*3 doubles read at the constrained nodes; NULL for 0.
 * Errors: INVALID_ARG, CUDA, OUT_OF_MEMORY.
 */
ufe_status ufe_assemble_elastic(ufe_mesh* mesh, double E, double nu, const double* E_scale_cells,
                                const double* f_nodes, const double* stress_nodes,
                                const double* dirichlet_values, int mem, ufe_system** out);
/* ncomp: 1 (Poisson) or 3 (elasticity); n = ncomp * n_dof, the length of every
 * solution / right-hand-side vector of this system. */
ufe_status ufe_system_get_info(const ufe_system* sys, int32_t* ncomp, int64_t* n);
/* b: n doubles (the assembled right-hand side, n from ufe_system_get_info). */
ufe_status ufe_system_get_rhs(const ufe_system* sys, double* b, int mem);
/* y = A x over the free DOFs (element-by-element apply); x, y of length n. */
ufe_status ufe_system_apply(const ufe_system* sys, const double* x, double* y, int mem);
/*
 * ufe_system_set_kappa -- replace the per-cell coefficient of a Poisson system
 * (A = sum_e kappa_e K_e) and rebuild its right-hand side (the Dirichlet lifting
 * depends on kappa).  No paper counterpart: an inverse-problem step (finite
 * differences, line searches) that keeps the set-up.  A preconditioner built on this
 * system stays valid and keeps the coefficient it was built with: ufe_pcg_solve still
 * converges to the solution of the updated system (BDDC of the old coefficient as
 * the preconditioner).
 *  kappa_cells  n_cells doubles (> 0 on active cells); the system must have been
 *               assembled with a coefficient (INVALID_ARG otherwise).
 * Errors: INVALID_ARG, UNSUPPORTED (elasticity), CUDA.
 */
ufe_status ufe_system_set_kappa(ufe_system* sys, const double* kappa_cells, int mem);
/* Cut-cell data in cut-cell order (ascending cell id): cut_cells n_cut int32,
 * K n_cut*ne*ne doubles (ne x ne row-major with ne = 8 ncomp, element DOF
 * ncomp a + c, vertex a = x + 2y + 4z, without kappa / E_scale), load n_cut*ne
 * doubles, eta n_cut doubles (volume fraction). Any may be NULL. */
ufe_status ufe_system_get_cut_data(const ufe_system* sys, int32_t* cut_cells, double* K, double* load,
                                   double* eta, int mem);
void ufe_system_destroy(ufe_system* sys);

typedef struct {
  int32_t weighting;   /* UFE_WEIGHT_* */
  int32_t objects;     /* UFE_OBJECTS_* */
  int32_t coarse;      /* UFE_COARSE_* */
  int32_t precision;   /* UFE_PREC_* */
  int32_t coarse_solver;   /* UFE_COARSE_SOLVER_* (DENSE and CR solve the coarse problem exactly in FP64,
                              BDDC preconditions it one level up) */
  int32_t coarse_group;    /* UFE_COARSE_SOLVER_BDDC: blocks per level-2 subdomain edge (0: 2); read
                              only with that solver */
  int32_t coarse_keep_corners;   /* UFE_COARSE_SOLVER_BDDC: 1 keeps every coarse DOF of a first-level
                                    corner (Sect. 3.2, 4.4) as a level-2 corner instead of merging it
                                    into the level-2 edge or face means; read only with that solver */
} ufe_bddc_opts;

typedef struct {
  int64_t n_objects, n_corners, n_edges, n_faces;
  int64_t n_coarse;               /* coarse DOFs (objects in Lambda_O) */
  int32_t max_local_coarse;       /* largest number of coarse DOFs of one subdomain */
  double setup_ms;                /* device time of ufe_bddc_setup */
  double inverse_flops_local;     /* sum of n^3 over the inverted local matrices (A_II, S', S_c) */
  double inverse_flops_coarse;    /* sum of n^3 over the inverted coarse matrices (n_coarse^3 for the
                                     dense solver, the layer blocks for cyclic reduction) */
  /* storage read by the per-iteration kernels (bytes): A_II^-1, the constrained
   * Neumann operator K, the coarse basis Phi (FP32 in mixed precision), the A_GI and
   * A_IG stencils (index + value per slot), the FP64 coarse solver's matrices */
  double bytes_interior_inverse, bytes_neumann, bytes_coarse_basis, bytes_offdiag, bytes_coarse_inverse;
  int64_t interior_slots, interface_slots;   /* sum over subdomains of local interior / interface DOFs */
  int32_t fp64_refactor;   /* mixed precision requested: 1 when no subdomain could keep FP32 local
                              operators (see fp64_subdomains), so the whole problem is factored and
                              applied in FP64 (classical PCG) */
  int32_t coarse_solver;   /* the coarse solver used: UFE_COARSE_SOLVER_DENSE, _CR or _BDDC */
  double cphi_error;       /* mixed precision requested: max |C Phi - I| of the FP32 coarse basis (Sect.
                              3.2 defines Phi by C Phi = I) over the subdomains that keep FP32
                              operators; a subdomain above 1e-2 gets FP64 operators */
  int32_t coarse_layers, coarse_levels;   /* cyclic reduction: non-empty z layers, reduction levels */
  int32_t local_tensor_cores;   /* 1 when the FP32 local inversions ran their Gauss-Jordan updates on the
                                   tensor cores (3xTF32 split products, tcgen05), 0 otherwise */
  int32_t prec_cluster, prec_stages;   /* launch shape of the per-iteration preconditioner kernels: CTAs per
                                          subdomain cluster and row-stream stages per CTA (0: from the
                                          shared-memory budget), chosen by timing the candidates once per
                                          size class and process (Poisson, 128 subdomains or more; otherwise
                                          and with UFE_AUTOTUNE=0: 4 and 0; UFE_PREC_SHAPE="cl,stages" fixes
                                          them) */
  int32_t fp64_subdomains;   /* mixed precision requested: subdomains whose local operators are FP64 --
                                those whose Jacobi-scaled A_II or S' had an FP32 pivot below 1e-3 (or
                                not positive), or whose FP32 coarse basis missed C Phi = I by more
                                than 1e-2 (tiny cut fractions); they are factored and applied in
                                FP64, the others in FP32 */
  int32_t level2_subdomains;   /* UFE_COARSE_SOLVER_BDDC: level-2 subdomains (groups of blocks split
                                  into components linked by shared coarse DOFs); 0 otherwise */
  int32_t level3_coarse;       /* UFE_COARSE_SOLVER_BDDC: level-2 objects, the DOFs of the inverted
                                  level-3 problem; 0 otherwise */
} ufe_bddc_info;

/*
 * ufe_bddc_setup -- the BDDC preconditioner of Eq. bddc for this system.
 *
 * Sect. 3.1 sub-assembled local Neumann matrices; Sect. 3.2 objects and coarse
 * DOFs (object means, Eq. coarse-dofs); Sect. 4.4 variant-1 objects; Sect. 3.3
 * topological weighting (Eq. weighting) or Sect. 4.3 stiffness weighting
 * (Eq. alge-weighting); harmonic extension with local Dirichlet problems.
 * Local operators are formed explicitly: A_II^-1, the constrained Neumann
 * inverse restricted to the interface and the interface rows of the coarse
 * basis; the coarse matrix sum_w Phi^T A^w Phi is assembled in FP64 and solved
 * exactly in FP64: explicit inverse, or block cyclic reduction over the z layers of
 * subdomain blocks, in which order A_c is block tridiagonal (opts.coarse_solver).
 * With UFE_COARSE_SOLVER_BDDC (Sect. 6 points to multilevel BDDC beyond one coarse
 * factorisation) A_c is instead preconditioned by BDDC one level up: level-2
 * subdomains group coarse_group^3 blocks (split into components linked by shared
 * coarse DOFs), level-2 objects are the coarse DOFs of one type (Poisson: one; elasticity:
 * a component mean or a rotation moment about one axis) shared by equal sets of level-2
 * subdomains (split into components; corners / edges / faces by opts.coarse), their
 * means are the level-3 DOFs, weights are stiffness weights of the level-2 matrices,
 * and the level-3 matrix is inverted in FP64.
 * Errors: SINGULAR_LOCAL (e.g. a floating subdomain with no coarse DOF),
 * SINGULAR_COARSE, INVALID_ARG, UNSUPPORTED, CUDA, OUT_OF_MEMORY, TIMEOUT.
 */
ufe_status ufe_bddc_setup(ufe_system* sys, const ufe_bddc_opts* opts, ufe_bddc** out);
ufe_status ufe_bddc_get_info(const ufe_bddc* bddc, ufe_bddc_info* info);
/* object_of_dof: n_dof int32 (object id, -1 off the interface; objects are sets of
 * free nodes); object_kind: n_objects int32 (UFE_OBJ_*); coarse_of_object:
 * n_objects int32, the first coarse DOF of the object (-1 if the object carries
 * none). Objects are ordered by their smallest DOF id.  Poisson: one coarse DOF
 * per object, its nodal mean (Eq. coarse-dofs).  Elasticity: consecutive coarse
 * DOFs per object -- the mean of each component, then the mean rotation moments
 * (1/n) sum (y x u)_k about each axis k (y the node's grid position relative to
 * the object's centroid) except about the axis of an object lying on one grid
 * line; corners carry 3, edges 5, faces 6. */
ufe_status ufe_bddc_get_objects(const ufe_bddc* bddc, int32_t* object_of_dof, int32_t* object_kind,
                                int32_t* coarse_of_object, int mem);
/* z = M r for one vector (n = ncomp n_dof doubles), Eq. bddc. */
ufe_status ufe_bddc_apply(ufe_bddc* bddc, const double* r, double* z, int mem);

/*
 * ufe_bddc_apply_noalloc -- the same z = M r as ufe_bddc_apply, for callers that
 * must not allocate device memory while they run: a serving loop that reserved
 * its memory budget up front, or host code called back from another framework
 * that owns the device allocator.  The paper has no counterpart; this is a
 * deployment variant.  It launches the same kernels, in the launch shape the set-up
 * chose, as ufe_bddc_apply.
 *
 *  r, z   n doubles each (n = ncomp n_dof), DEVICE pointers on the current device (host
 *         pointers are not accepted: staging them would need an allocation).
 *
 * The preconditioner's intermediate vectors live in one file-scope device array
 * of fixed size (688,128 doubles, about 5.5 MB, held by every device that loads the
 * library until the process exits) instead of the buffers ufe_bddc_setup made; with
 * UFE_COARSE_SOLVER_BDDC the level-2 vectors stay in the handle's own buffers, which
 * set-up allocated and the call reuses.
 * Problems beyond its limits -- more than 262,144 interface slots (the sum over
 * subdomains of their interface DOFs, counted per component), 65,536 subdomain coarse slots or 32,768
 * coarse DOFs -- are rejected with UFE_ERR_INVALID_ARG and a message naming the
 * limit.  The call allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.  ufe_bddc_setup (which does allocate) looks up the array's
 * device address (cudaGetSymbolAddress) on the device current at set-up and loads
 * every kernel this call launches, so no module or kernel loading, which takes
 * device memory, happens inside the call.  The call must be made with the set-up's
 * device current and with r and z in that device's memory; otherwise it returns
 * UFE_ERR_INVALID_ARG.  All calls share the array and it keeps the last call's
 * contents, so calls that overlap on the GPU (other streams or threads using any
 * ufe_bddc handle) race; serialise them.  The call waits on the preconditioner's
 * stream and returns after z is complete.
 */
ufe_status ufe_bddc_apply_noalloc(ufe_bddc* bddc, const double* r, double* z);
void ufe_bddc_destroy(ufe_bddc* bddc);

typedef struct {
  double rtol;          /* stop when |r|_2 < rtol |b|_2 (Sect. 5.1); e.g. 1e-8 */
  int32_t maxit;        /* iteration cap */
  int32_t flexible;     /* 0 classical beta, 1 flexible beta, -1 auto (flexible iff mixed) */
  int32_t check_every;  /* unused: the iterations run in a device-side loop (kept for layout) */
  int32_t reserved;
} ufe_solve_opts;

typedef struct {
  int32_t iterations;        /* operator applications to search directions */
  int32_t converged;
  double rel_residual;       /* |r|_2 / |b|_2 of the recursively updated residual */
  double true_rel_residual;  /* |b - A x|_2 / |b|_2 recomputed at the end */
  double solve_ms;           /* device time of the solve */
} ufe_solve_info;

/*
 * ufe_pcg_solve -- BDDC-preconditioned CG (Sect. 5.1), all on the device.
 * The solve runs as one CUDA graph built at the first call and reused: initial
 * residual and preconditioner, a conditional while node around one iteration whose
 * last kernel decides from the device-side state whether to run again (bounded by
 * maxit + 1 passes), and the true residual; the host waits once.
 *  b     n doubles (n = ncomp n_dof) or NULL for the assembled right-hand side.
 *  x     n doubles: initial guess in, solution out.
 *  info  may be NULL.
 * Errors: BREAKDOWN, NO_CONVERGENCE (x holds the last iterate), CUDA, INVALID_ARG.
 */
ufe_status ufe_pcg_solve(ufe_system* sys, ufe_bddc* bddc, const double* b, double* x, int mem,
                         const ufe_solve_opts* opts, ufe_solve_info* info);

/*
 * ufe_pcg_solve_batched -- n independent solves at once (many problems of uneven
 * size, e.g. a serving queue; no counterpart in the paper).  Each problem's solve
 * graph (as in ufe_pcg_solve) is launched on one of 16 library-owned streams after
 * that problem's own stream, so the GPU runs the problems side by side; later work
 * on each problem's stream waits for its solve.  Returns when all are done.
 *  systems, bddcs  n handles; bddcs[i] set up on systems[i]; no handle twice.
 *  b               NULL, or n pointers (each NULL for the assembled right-hand side).
 *  x               n pointers: initial guesses in, solutions out (length ncomp n_dof each).
 *  infos           n entries or NULL.
 * Every problem is solved and reported; the return value is the first non-OK
 * status among them (BREAKDOWN, NO_CONVERGENCE), or an argument / CUDA error.
 */
ufe_status ufe_pcg_solve_batched(int32_t n, ufe_system* const* systems, ufe_bddc* const* bddcs,
                                 const double* const* b, double* const* x, int mem,
                                 const ufe_solve_opts* opts, ufe_solve_info* infos);

/*
 * ufe_adjoint -- gradient of J(u) = 1/2 |u - u_d|^2 over the free DOFs with
 * respect to the per-cell coefficients kappa (no counterpart in the paper).
 * Solves A lambda = dJdu with the same BDDC-PCG (A is SPD, so A^T = A) and
 * contracts dJ/dkappa_e = -u_e^T Khat_e lambda_e per active cell, Khat_e the
 * coefficient-free cell matrix (b does not depend on kappa).
 *  u          n_dof doubles: the forward solution.
 *  dJdu       n_dof doubles: the adjoint right-hand side (u - u_d for this J).
 *  lambda     n_dof doubles: adjoint solution out (initial guess in).
 *  dJdkappa   n_cells doubles out (0 on external cells).
 * Poisson systems only (UFE_ERR_UNSUPPORTED for an elasticity system).
 */
ufe_status ufe_adjoint(ufe_system* sys, ufe_bddc* bddc, const double* u, const double* dJdu,
                       double* lambda, double* dJdkappa, int mem, const ufe_solve_opts* opts,
                       ufe_solve_info* info);

#ifdef __cplusplus
}
#endif

#endif /* UFE_H */
