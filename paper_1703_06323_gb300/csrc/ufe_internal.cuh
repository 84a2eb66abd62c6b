// Internal declarations shared by the CUDA translation units of libufe.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/ufe.h"

namespace ufe {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);

struct Error {
  ufe_status code;
  std::string msg;
};

#define UFE_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t _e = (call);                                                                 \
    if (_e != cudaSuccess)                                                                   \
      throw ::ufe::Error{UFE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)}; \
  } while (0)

// kernel launch accounting: launches issued directly count at once; launches
// recorded into a graph count once per graph launch (see pcg.cu)
void note_launch();

#define UFE_CHECK_LAUNCH()         \
  do {                             \
    UFE_CUDA(cudaGetLastError());  \
    ::ufe::note_launch();          \
  } while (0)

#define UFE_REQUIRE(cond, code, msg)                     \
  do {                                                   \
    if (!(cond)) throw ::ufe::Error{(code), (msg)};      \
  } while (0)

// device status bits written by bounded device loops / factorisations
enum DevStatus : int {
  DEV_OK = 0,
  DEV_SINGULAR = 1,
  DEV_TIMEOUT = 2,
  DEV_ILLCOND = 4,   // a pivot of a Jacobi-scaled matrix fell below the precision's floor
};

// ---------------------------------------------------------------------------
// stream-ordered device buffers
// ---------------------------------------------------------------------------
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void alloc(size_t count, cudaStream_t stream) {
    release();
    s = stream;
    n = count;
    if (count) {
      cudaError_t e = cudaMallocAsync((void**)&p, count * sizeof(T), stream);
      if (e != cudaSuccess) {
        p = nullptr;
        n = 0;
        throw Error{UFE_ERR_OUT_OF_MEMORY, std::string("cudaMallocAsync: ") + cudaGetErrorString(e)};
      }
    }
  }
  void zero() {
    if (n) UFE_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
  void fill_bytes(int v) {
    if (n) UFE_CUDA(cudaMemsetAsync(p, v, n * sizeof(T), s));
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
};

// copy helpers honouring the UFE_MEM_* convention
void copy_in(void* dst_dev, const void* src, size_t bytes, int mem, cudaStream_t s);
void copy_out(void* dst, const void* src_dev, size_t bytes, int mem, cudaStream_t s);
template <typename T>
std::vector<T> to_host(const T* dev, size_t n, cudaStream_t s) {
  std::vector<T> h(n);
  if (n) UFE_CUDA(cudaMemcpyAsync(h.data(), dev, n * sizeof(T), cudaMemcpyDeviceToHost, s));
  UFE_CUDA(cudaStreamSynchronize(s));
  return h;
}
template <typename T>
T scalar_to_host(const T* dev, cudaStream_t s) {
  T v;
  UFE_CUDA(cudaMemcpyAsync(&v, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
  UFE_CUDA(cudaStreamSynchronize(s));
  return v;
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }
__host__ __device__ inline int pad4(int n) { return (n + 3) & ~3; }

// ---------------------------------------------------------------------------
// grid geometry passed by value to kernels
// ---------------------------------------------------------------------------
struct GridGeom {
  int nx, ny, nz;      // cells
  int sx, sy, sz;      // cells per block edge
  int bx, by, bz;      // blocks per axis
  int lnx, lny, lnz;   // local nodes per block edge (s + 1)
  int n_local_nodes;   // lnx * lny * lnz
  double lo[3];
  double h;
  __host__ __device__ int64_t node(int i, int j, int k) const {
    return (int64_t)i + (int64_t)(nx + 1) * ((int64_t)j + (int64_t)(ny + 1) * k);
  }
  __host__ __device__ int64_t cell(int i, int j, int k) const {
    return (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k);
  }
  __host__ __device__ int64_t n_nodes() const { return (int64_t)(nx + 1) * (ny + 1) * (nz + 1); }
  __host__ __device__ int64_t n_cells() const { return (int64_t)nx * ny * nz; }
  __host__ __device__ int n_blocks() const { return bx * by * bz; }
};

// The operator apply works on boxes of kApplyTX x kApplyTY x kApplyTZ grid nodes
// ("node tiles", numbered x fastest); only tiles that hold a free DOF are launched.
constexpr int kApplyTX = 8, kApplyTY = 8, kApplyTZ = 4;
__host__ __device__ inline int apply_tiles_x(const GridGeom& g) { return (g.nx + kApplyTX) / kApplyTX; }
__host__ __device__ inline int apply_tiles_y(const GridGeom& g) { return (g.ny + kApplyTY) / kApplyTY; }
__host__ __device__ inline int apply_tiles_z(const GridGeom& g) { return (g.nz + kApplyTZ) / kApplyTZ; }
__host__ __device__ inline int64_t apply_tile_of_node(const GridGeom& g, int i, int j, int k) {
  return (int64_t)(i / kApplyTX) +
         (int64_t)apply_tiles_x(g) * ((int64_t)(j / kApplyTY) + (int64_t)apply_tiles_y(g) * (k / kApplyTZ));
}

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
struct Mesh {
  cudaStream_t stream = nullptr;
  GridGeom g{};
  uint32_t face_mask = 0;
  int64_t pin = -1;
  int64_t n_dof = 0, n_sub = 0, n_active = 0, n_cut = 0, n_gamma = 0, n_constrained = 0, n_apply_tiles = 0;
  int64_t n_Iloc = 0, n_Gloc = 0;   // sum over subdomains of interior / interface sizes
  int max_nI = 0, max_nG = 0;

  DBuf<double> phi;            // n_nodes
  DBuf<uint8_t> cell_type;     // n_cells
  DBuf<uint8_t> node_flags;    // n_nodes: bit0 active, bit1 constrained, bit2 pin candidate
  DBuf<int32_t> dof_of_node;   // n_nodes
  DBuf<int32_t> node_of_dof;   // n_dof
  DBuf<int32_t> apply_tiles;   // n_apply_tiles: node tiles of the operator apply holding a free DOF
  DBuf<int32_t> cut_index;     // n_cells: index into cut arrays or -1
  DBuf<int32_t> cut_cells;     // n_cut
  DBuf<int32_t> sub_of_cell;   // n_cells
  DBuf<int32_t> sub_block;     // n_sub
  DBuf<int32_t> neigh;         // n_dof * 8
  DBuf<uint8_t> n_neigh;       // n_dof
  DBuf<int32_t> gpos;          // n_dof * 8: slot of (xi, k-th neighbour) in the interface-local arrays
  DBuf<int32_t> lmap;          // n_sub * n_local_nodes: (kind << 24) | local index
  DBuf<int32_t> I_ptr, I_list; // CSR interior DOFs per subdomain
  DBuf<int32_t> G_ptr, G_list; // CSR interface DOFs per subdomain
  std::vector<int32_t> h_I_ptr, h_G_ptr;
};

// lmap codes
enum : int { LKIND_NONE = 0, LKIND_I = 1, LKIND_G = 2 };
__host__ __device__ inline int lmap_kind(int32_t code) { return (code >> 24) & 0xff; }
__host__ __device__ inline int lmap_index(int32_t code) { return code & 0xffffff; }

// Poisson (ncomp = 1) or linear elasticity (ncomp = 3, DOF 3 d + c of free node d).
// Element matrices have ne = 8 ncomp rows (element DOF ncomp a + c of vertex a).
struct System {
  Mesh* mesh = nullptr;
  cudaStream_t stream = nullptr;
  int ncomp = 1;
  double lam = 0.0, mu = 0.0;   // elasticity: Lame parameters
  bool has_kappa = false;
  DBuf<double> kappa;       // n_cells (only if has_kappa): scales the element matrix
  DBuf<double> Kref;        // elasticity: h Khat_el (24 x 24)
  DBuf<double> K_cut;       // n_cut * ne^2
  DBuf<double> load_cut;    // n_cut * ne
  DBuf<double> eta;         // n_cut
  DBuf<double> b;           // ncomp * n_dof
  DBuf<double> gnode;       // ncomp * n_nodes: Dirichlet values read at constrained nodes (zeros if none given)
  DBuf<double> fnode;       // Poisson: nodal source (zeros if none given), kept to rebuild b after a kappa update
  bool nitsche = false;     // weak Dirichlet data on the unfitted boundary (Nitsche terms in K_cut, load_cut)
  DBuf<double> beta;        // n_cut Nitsche coefficients beta_e (physical units; 0 without boundary)
  int64_t n_vec() const { return (int64_t)ncomp * mesh->n_dof; }
};

struct Bddc;   // defined in bddc.cu

// ---------------------------------------------------------------------------
// building blocks implemented in the .cu files
// ---------------------------------------------------------------------------
// exclusive scan of predicate flags (uint8 0/1) -> index (-1 where flag == 0); returns the count
int64_t scan_flags(const uint8_t* flags, int64_t n, int32_t* index_out, cudaStream_t s);
// exclusive scan of int32 counts -> offsets (n+1 entries, offsets[n] = total); returns total
int64_t scan_counts(const int32_t* counts, int64_t n, int32_t* offsets_out, cudaStream_t s);

void mesh_build(Mesh& m, const double* phi_dev, int64_t pin_node);
void system_build(System& sys, const double* kappa, const double* f, const double* q, const double* g,
                  bool weak_dirichlet = false);
// Poisson: b rebuilt from the kept source, cut loads and Dirichlet values after sys.kappa changed
void system_rebuild_rhs(System& sys);
// elasticity: f 3 values per node, sigma 9 per node (may be null), g 3 per node (may be null)
void system_build_elastic(System& sys, const double* kappa, const double* f, const double* sigma, const double* g);
void system_apply(const System& sys, const double* x_dev, double* y_dev, cudaStream_t s);
// dJ/dkappa_e = -ubar_e^T Khat_e lambda_e per cell (ubar: u with the Dirichlet values)
void kappa_gradient(const System& sys, const double* u_dev, const double* lambda_dev, double* out_dev, cudaStream_t s);

// constant tables (Q1 reference matrices, quadrature) uploaded once
void ensure_constants();

// whether ufe_timing_enable is on (the launch-shape tuner switches it off around its runs)
bool timing_enabled();
void set_timing_enabled(bool on);

// optional event timing of named kernels (see ufe_timing_enable)
struct TimedLaunch {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void begin(const char* name, cudaStream_t s);
  void end(cudaStream_t s);
  const char* name = nullptr;
};

// launch accounting state
extern std::atomic<long long> g_kernel_launches;
extern thread_local long long* g_capture_counter;   // non-null while a graph is being captured

}  // namespace ufe
