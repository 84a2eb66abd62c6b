// BDDC preconditioner state shared by the set-up (bddc.cu) and the solver (pcg.cu).
#pragma once

#include "ufe_internal.cuh"

namespace ufe {

// metadata the per-subdomain solve kernels read (all device pointers)
// Index spaces: a node-level list (I_list, G_list: free-node DOF ids) holds ncomp
// vector DOFs per entry; vector DOF ncomp d + c of node DOF d, local vector index
// ncomp p + c of local node p, and vector CSR pointers vI_ptr = ncomp I_ptr,
// vG_ptr = ncomp G_ptr.  Poisson has ncomp = 1 and both spaces coincide.
struct SubMeta {
  GridGeom g;
  int n_sub;
  int ncomp;
  const int32_t* vI_ptr;    // vector CSR pointers of the interior / interface DOFs
  const int32_t* vG_ptr;
  const double* Kref;       // elasticity: h Khat_el
  const int32_t* sub_block;
  const int32_t* sub_of_cell;
  const uint8_t* cell_type;
  const int32_t* cut_index;
  const double* K_cut;
  const double* kappa;      // may be null
  const int32_t* dof_of_node;
  const int32_t* lmap;
  const int32_t* I_ptr;
  const int32_t* I_list;
  const int32_t* G_ptr;
  const int32_t* G_list;
  const int32_t* C_ptr;
  const int32_t* C_list;
  const int32_t* neigh;
  const uint8_t* n_neigh;
  const int32_t* gpos;
  const int64_t* off_II;    // element offset of A_II^-1 (nI x ldI)
  const int64_t* off_GG;    // element offset of K (nG x ldG)
  const int64_t* off_GC;    // element offset of Phi (nG x ldC)
  const double* w;          // weight per interface slot
  const int32_t* gi_k;      // A_GI in ELL form (27 slots, slot-major per subdomain)
  const double* gi_v;
  const int32_t* ig_k;      // A_IG in ELL form
  const double* ig_v;
  int* status;              // DEV_* flags raised by bounded device waits
  const double* sI;         // scale of each local interior / interface vector slot: the stored
  const double* sG;         // operators are those of the scaled problem (D^-1/2 A D^-1/2)
};

struct PcgScalars {
  double rtol;         // relative residual target (set by the host before a solve)
  double pq;           // p . A p
  double rr;           // r . r after the update
  double rz;           // r_k . z_k of the previous iteration
  double rz_next;      // r . z of the freshly preconditioned residual
  double rzold_next;   // r . z_old (flexible beta)
  double bb;           // |b|^2
  double tol2;         // (rtol |b|)^2
  int iter;            // completed x/r updates
  int done;            // 0 running, 1 converged, 2 max iterations, 3 breakdown
  int first;           // first search direction (beta = 0)
  int maxit;
  int flexible;
  unsigned passes;     // passes of the device-side loop (bounds it at maxit + 1)
  unsigned int counter[8];   // last-block-done counters per kernel
};

// coarse solver (coarse.cu): block cyclic reduction of the block-tridiagonal coarse
// matrix over the z layers of subdomain blocks; every solve step is a list of tasks
//   V[y + i] = (base >= 0 ? V[base + i] : 0) + sum_t sign_t (M_t V[x_t + .])_i
struct CoarseTerm {
  int64_t off;   // matrix offset in the store (row-major, leading dimension ld)
  int ld, cols;
  int64_t x;     // input offset in the work vector
  double sign;
};
struct CoarseTask {
  int64_t y, base;   // output / base offsets in the work vector (base -1: none)
  int64_t row0;      // first row of the task within its launch
  int n, term0, nterm;
};
struct CoarseStep {
  int task0, ntask;
  int64_t rows;
};
struct CoarseCR {
  int64_t n = 0;               // coarse DOFs
  int nlayers = 0, nlevels = 0;
  DBuf<int32_t> perm;          // CR position -> coarse DOF
  DBuf<double> store;          // X, T1, T2, W1, W2 and coupling blocks
  DBuf<CoarseTask> tasks;
  DBuf<CoarseTerm> terms;
  std::vector<CoarseStep> steps;
  DBuf<double> work;           // r (CR order) then u, 2 n
  double bytes = 0.0;          // matrix bytes one solve reads
  double inv_flops = 0.0;      // sum of n_j^3 over the inverted layer blocks
};

// three-level method (multilevel.cu): the coarse problem preconditioned by BDDC over
// groups of subdomains ("level 2"), whose own coarse problem ("level 3") is inverted
struct MultiLevel {
  int n2 = 0;                   // level-2 subdomains (0: the three-level method is not in use)
  int n3 = 0, ld3 = 4;          // level-3 coarse DOFs (level-2 objects)
  int n_obj2 = 0;
  int64_t n_slots = 0;          // sum over level-2 subdomains of their coarse DOFs
  int max_n = 0, max_nI = 0, max_nG = 0, max_nC = 0;
  DBuf<int32_t> dof_ptr, nI, dofs, slot_J, gpos2, c_ptr, c_list, cpos3;
  DBuf<uint8_t> owner, nn2, nn3;
  DBuf<int64_t> offA, offK, offP;
  DBuf<double> store;           // every level-2 operator (FP64)
  DBuf<double> A3inv;           // level-3 inverse (n3 x ld3)
  DBuf<double> w2, y2, rc2, t2, vw2, g3, u3;
  double bytes = 0.0, inv_flops = 0.0;
};

struct Bddc {
  System* sys = nullptr;
  Mesh* mesh = nullptr;
  cudaStream_t stream = nullptr;
  int device = -1;              // device current at set-up (its stream and buffers live there)
  ufe_bddc_opts opts{};
  bool mixed = false;

  // objects (Sect. 3.2, Sect. 4.4)
  int ncomp = 1;
  int64_t n_obj = 0, n_corner = 0, n_edge = 0, n_face = 0, n_coarse = 0, n_Cloc = 0;
  int max_nC = 0;
  int max_nIv = 0, max_nGv = 0;         // largest vector interior / interface sizes
  int64_t n_vIloc = 0, n_vGloc = 0;     // vector local slots
  DBuf<int32_t> vI_ptr, vG_ptr;
  DBuf<int32_t> obj_nrows;              // coarse rows (coarse DOFs) per object
  DBuf<int32_t> obj_rot;                // elasticity: bit k = rotation row about axis k kept
  DBuf<long long> obj_sum;              // sum of the node grid coordinates of each object (3 per object)
  DBuf<int32_t> obj_lo, obj_hi;         // coordinate bounds of each object (3 per object)
  DBuf<int32_t> obj_of_dof, obj_kind, obj_rep, obj_size, coarse_of_obj, coarse_obj, coarse_rep;
  // coarse_of_obj: first coarse row of an object (-1 if not a coarse object);
  // coarse_obj / coarse_rep / coarse_nn are per coarse row
  DBuf<uint8_t> coarse_nn;      // |neigh| of each coarse DOF
  DBuf<int32_t> C_ptr, C_list, cpos;
  std::vector<int32_t> h_nI, h_nG, h_nC;

  // per-iteration operators
  DBuf<int64_t> off_II, off_GG, off_GC;
  DBuf<double> dII, dGG, dGC;   // FP64 operators
  DBuf<float> fII, fGG, fGC;    // FP32 operators (mixed)
  DBuf<double> w;               // n_Gloc weights
  DBuf<double> sI, sG;          // Jacobi scales of the local slots (operators stored scaled)
  DBuf<int32_t> gi_k, ig_k;     // A_GI / A_IG in ELL form (local indices)
  DBuf<double> gi_v, ig_v;
  int coarse_solver = 0;        // requested UFE_COARSE_SOLVER_*
  int coarse_group = 2;         // three-level method: blocks per level-2 subdomain edge
  bool coarse_keep_corners = false;   // three-level method: first-level corners stay level-2 corners
  bool coarse_dense = true;     // resolved: explicit inverse (else cyclic reduction)
  DBuf<double> Ac_inv;          // dense: n_coarse x ldc, FP64
  int ldc = 0;
  CoarseCR cr;                  // cyclic reduction over the z layers of subdomain blocks
  MultiLevel ml;                // three-level method (coarse_solver UFE_COARSE_SOLVER_BDDC)
  DBuf<int> coarse_status;      // dense coarse inversion in flight: its pivot flags (coarse_check reads them)

  // solver work space
  DBuf<double> tG, vw, gC, uc;
  DBuf<double> x, r, b, z, q, p0, p1;
  DBuf<double> part;            // per-block partial sums
  DBuf<PcgScalars> sc;
  DBuf<int> status;             // DEV_* flags of the per-iteration kernels
  PcgScalars* h_sc = nullptr;   // pinned mirror
  // the whole solve as one instantiated graph: initial residual and preconditioner,
  // a conditional while node whose body is one PCG iteration, the true residual
  cudaGraphExec_t solve_exec = nullptr;
  cudaStream_t cap_stream = nullptr;    // library-owned streams used only for graph capture
  cudaStream_t cap_stream2 = nullptr;
  long long k_init = 0, k_body = 0, k_final = 0;   // kernel nodes per part of the graph
  DBuf<double> tres;                    // |b - A x|^2, |b|^2 after the solve
  int64_t part_blocks = 0;
  double setup_ms = 0.0;
  double inv_flops_local = 0.0, inv_flops_coarse = 0.0;
  double bytes_II = 0.0, bytes_GG = 0.0, bytes_GC = 0.0, bytes_off = 0.0, bytes_Ac = 0.0;
  int fp64_refactor = 0;                // mixed precision requested, FP64 local operators kept (FP32 too ill-conditioned)
  // mixed precision with some subdomains in FP64: their ids (wl64, n_sub64 of them; the
  // FP64 operators dII, dGG, dGC hold those subdomains) and the FP32 ones (wl32)
  int n_sub64 = 0;
  DBuf<int32_t> wl32, wl64;
  double cphi_error = 0.0;              // mixed: max |C Phi - I| of the FP32 operators
  int local_tc = 0;                     // FP32 local inversions ran the tensor-core update
  int prec_cl = 4;                      // CTAs per subdomain cluster in the preconditioner kernels (tuned)
  int prec_stages = 0;                  // row-stream stages per CTA (tuned; 0: from the shared-memory budget)

  SubMeta meta() const;
  ~Bddc();
};

void bddc_build(Bddc& B);
// coarse solver: set-up from the assembled dense A_c (n_coarse x ldc, symmetric; the
// dense solver takes ownership of the buffer), and u_c = A_c^-1 r_c with r_c gathered
// from the subdomain parts gC (work: 2 n_coarse doubles)
void coarse_setup(Bddc& B, DBuf<double>& Ac, int ldc, cudaStream_t s);
// SINGULAR_COARSE if the dense coarse inversion queued by coarse_setup met a bad pivot
void coarse_check(Bddc& B);
// records the solve graph during the set-up when the launch shape is already known
// (fixed, cached for the size class, or not tuned); returns whether it did
bool solve_graph_early(Bddc& B);
// drops a solve graph recorded for operators that the set-up then replaced
void solve_graph_reset(Bddc& B);
void coarse_solve(const Bddc& B, const double* gC, double* uc, double* work, const PcgScalars* sc, cudaStream_t s);
// u = A^-1 r with r gathered from up to eight parts per row (parts[cpos[8 l + k]], k < cnn[l])
// checks that r of n values fits one CTA's shared memory and raises the kernel's limit
void dense_coarse_prepare(int64_t n, int ld);
void dense_coarse_gemv(int64_t n, int ld, const double* Ainv, const int32_t* cpos, const uint8_t* cnn,
                       const double* parts, double* u, const PcgScalars* sc, cudaStream_t s);
// three-level method: level-2 set-up from the subdomains' coarse matrices A_c^w (offsets
// oCC, host) with groups of `group`^3 blocks, and one application u_c = M_2 r_c
void ml_setup(Bddc& B, const DBuf<double>& Acw, const std::vector<int64_t>& oCC, int group, cudaStream_t s);
void ml_coarse_solve(const Bddc& B, const double* gC, double* uc, const PcgScalars* sc, cudaStream_t s);
void bddc_apply(Bddc& B, const double* r_dev, double* z_dev);
void bddc_apply_noalloc(Bddc& B, const double* r_dev, double* z_dev);
// made by the set-up: loads the device code and looks up the static array the
// allocation-free apply uses, so that the apply itself takes no device memory
void bddc_noalloc_prepare(Bddc& B);
// launch shape of the per-iteration preconditioner kernels, timed per size class (pcg.cu)
void tune_preconditioner(Bddc& B);
// UFE_ERR_UNSUPPORTED if a subdomain's vectors and one operator row do not fit one CTA's shared memory
void check_local_sizes(const Bddc& B);
// loads the coarse solver's kernels (cudaFuncGetAttributes), once per device
void coarse_prepare();
void pcg_solve(Bddc& B, const double* b_dev, double* x_dev, const ufe_solve_opts& o, ufe_solve_info* info);
ufe_status pcg_solve_batched(int n, Bddc* const* Bs, const double* const* b_dev, double* const* x_dev,
                             const ufe_solve_opts& o, ufe_solve_info* infos);

}  // namespace ufe
