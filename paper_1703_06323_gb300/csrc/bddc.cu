// BDDC set-up (Sect. 3, Sect. 4): geometric objects and coarse DOFs, weights,
// local matrices, the explicit local operators applied at every iteration and
// the coarse matrix.
//
// Per subdomain w with interior DOFs I and interface DOFs G the preconditioner
// (Eq. bddc) needs only
//   * A_II^-1                       (interior / harmonic-extension solves),
//   * K = S'^-1 - S'^-1 C^T (C S'^-1 C^T)^-1 C S'^-1   restricted to G,
//     the constrained Neumann inverse, where S' = S + C^T rho C and
//     S = A_GG - A_GI A_II^-1 A_IG is the Schur complement (the constraint rows C
//     live on G only, so eliminating I is exact; adding C^T rho C leaves the
//     constrained solution unchanged because C v = 0 there),
//   * Phi_G = S'^-1 C^T (C S'^-1 C^T)^-1, the interface rows of the energy-
//     minimising coarse basis (C Phi = I), and
//   * A_c^w = Phi^T A^w Phi = (C S'^-1 C^T)^-1 - rho   (coarse contribution).
// All local matrices are Jacobi-scaled (D^-1/2 A D^-1/2) before inversion; in
// mixed precision the scaled matrices are inverted and stored in FP32.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <mutex>

#include "bddc.cuh"
#include "dense.cuh"
#include "q1.cuh"

namespace ufe {

Bddc::~Bddc() {
  if (solve_exec) cudaGraphExecDestroy(solve_exec);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  if (cap_stream2) cudaStreamDestroy(cap_stream2);
  if (h_sc) cudaFreeHost(h_sc);
}

SubMeta Bddc::meta() const {
  const Mesh& m = *mesh;
  SubMeta s;
  s.g = m.g;
  s.n_sub = (int)m.n_sub;
  s.ncomp = ncomp;
  s.vI_ptr = vI_ptr.p;
  s.vG_ptr = vG_ptr.p;
  s.Kref = sys->Kref.p;
  s.sub_block = m.sub_block.p;
  s.sub_of_cell = m.sub_of_cell.p;
  s.cell_type = m.cell_type.p;
  s.cut_index = m.cut_index.p;
  s.K_cut = sys->K_cut.p;
  s.kappa = sys->has_kappa ? sys->kappa.p : nullptr;
  s.dof_of_node = m.dof_of_node.p;
  s.lmap = m.lmap.p;
  s.I_ptr = m.I_ptr.p;
  s.I_list = m.I_list.p;
  s.G_ptr = m.G_ptr.p;
  s.G_list = m.G_list.p;
  s.C_ptr = C_ptr.p;
  s.C_list = C_list.p;
  s.neigh = m.neigh.p;
  s.n_neigh = m.n_neigh.p;
  s.gpos = m.gpos.p;
  s.off_II = off_II.p;
  s.off_GG = off_GG.p;
  s.off_GC = off_GC.p;
  s.w = w.p;
  s.gi_k = gi_k.p;
  s.gi_v = gi_v.p;
  s.ig_k = ig_k.p;
  s.ig_v = ig_v.p;
  s.status = status.p;
  s.sI = sI.p;
  s.sG = sG.p;
  return s;
}

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------
// grid edge from node (i,j,k) to its +axis neighbour belongs to an active cell
__device__ __forceinline__ bool fe_edge(const GridGeom& g, const uint8_t* __restrict__ cell_type, int i, int j, int k,
                                        int axis) {
  for (int a = -1; a <= 0; ++a)
    for (int b = -1; b <= 0; ++b) {
      int ci = i, cj = j, ck = k;
      if (axis == 0) { cj += a; ck += b; }
      else if (axis == 1) { ci += a; ck += b; }
      else { ci += a; cj += b; }
      if (ci < 0 || cj < 0 || ck < 0 || ci >= g.nx || cj >= g.ny || ck >= g.nz) continue;
      if (cell_type[g.cell(ci, cj, ck)] != UFE_CELL_EXTERNAL) return true;
    }
  return false;
}

__device__ __forceinline__ bool same_neigh(const int32_t* __restrict__ neigh, const uint8_t* __restrict__ nn,
                                           int64_t d, int64_t e) {
  if (nn[d] != nn[e]) return false;
  for (int t = 0; t < 8; ++t)
    if (neigh[d * 8 + t] != neigh[e * 8 + t]) return false;
  return true;
}

// calls f(e, inside_e) for every axis neighbour DOF e of DOF d joined to d by an FE edge
template <typename F>
__device__ __forceinline__ void for_fe_neighbours(const GridGeom& g, const int32_t* __restrict__ node_of_dof,
                                                  const int32_t* __restrict__ dof_of_node,
                                                  const uint8_t* __restrict__ cell_type, int64_t d, F f) {
  const int64_t v = node_of_dof[d];
  const int i = (int)(v % (g.nx + 1)), j = (int)((v / (g.nx + 1)) % (g.ny + 1));
  const int k = (int)(v / ((int64_t)(g.nx + 1) * (g.ny + 1)));
  const int lim[3] = {g.nx, g.ny, g.nz};
  const int c[3] = {i, j, k};
  for (int axis = 0; axis < 3; ++axis)
    for (int dir = -1; dir <= 1; dir += 2) {
      int cc[3] = {c[0], c[1], c[2]};
      cc[axis] += dir;
      if (cc[axis] < 0 || cc[axis] > lim[axis]) continue;
      const int64_t wv = g.node(cc[0], cc[1], cc[2]);
      const int32_t e = dof_of_node[wv];
      if (e < 0) continue;
      int lo[3] = {c[0], c[1], c[2]};
      if (dir < 0) lo[axis] -= 1;
      if (!fe_edge(g, cell_type, lo[0], lo[1], lo[2], axis)) continue;
      f((int64_t)e, wv);
    }
}

// min-label propagation; mode 0: interface DOFs with equal neigh sets (standard
// objects); mode 1: non-corner DOFs of one edge object joined by uncut FE edges
constexpr double kV2WeightTol = 1e-8;

__global__ void k_obj_propagate(GridGeom g, int64_t n_dof, const int32_t* __restrict__ node_of_dof,
                                const int32_t* __restrict__ dof_of_node, const uint8_t* __restrict__ cell_type,
                                const int32_t* __restrict__ neigh, const uint8_t* __restrict__ nn,
                                const double* __restrict__ phi, const int32_t* __restrict__ std_obj,
                                const uint8_t* __restrict__ active, int mode, const double* __restrict__ wv2,
                                int32_t* label, int* changed) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dof || !active[d]) return;
  int32_t m = label[d];
  const bool in_d = phi[node_of_dof[d]] < 0.0;
  for_fe_neighbours(g, node_of_dof, dof_of_node, cell_type, d, [&](int64_t e, int64_t wv) {
    if (!active[e]) return;
    if (mode == 0) {
      if (!same_neigh(neigh, nn, d, e)) return;
    } else if (mode == 1) {
      if (std_obj[e] != std_obj[d]) return;
      if ((phi[wv] < 0.0) != in_d) return;
    } else {
      if (std_obj[e] != std_obj[d]) return;
      for (int t = 0; t < nn[d]; ++t)   // d and e share one neigh list (same object)
        if (fabs(wv2[d * 8 + t] - wv2[e * 8 + t]) > kV2WeightTol) return;
    }
    const int32_t l = label[e];
    if (l < m) m = l;
  });
  const int32_t mm = label[m];
  if (mm < m) m = mm;
  if (m < label[d]) {
    label[d] = m;
    *changed = 1;
  }
}

// variant 2 (Sect. 4.5): stiffness weight of every (interface DOF, neigh slot), the slot's
// subdomain's diagonal A^w_dd (sum over its active cells containing the node, kappa
// included) over the sum of all neigh slots' diagonals
__global__ void k_v2_weights(GridGeom g, int64_t n_dof, const int32_t* __restrict__ node_of_dof,
                             const uint8_t* __restrict__ cell_type, const int32_t* __restrict__ sub_of_cell,
                             const int32_t* __restrict__ cut_index, const double* __restrict__ K_cut,
                             const double* __restrict__ kappa, const int32_t* __restrict__ neigh,
                             const uint8_t* __restrict__ nn, double* __restrict__ w) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dof || nn[d] < 2) return;
  const int64_t v = node_of_dof[d];
  const int i = (int)(v % (g.nx + 1)), j = (int)((v / (g.nx + 1)) % (g.ny + 1));
  const int k = (int)(v / ((int64_t)(g.nx + 1) * (g.ny + 1)));
  double diag[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int a = 0; a < 8; ++a) {   // the cell whose vertex a is this node
    const int ci = i - (a & 1), cj = j - ((a >> 1) & 1), ck = k - (a >> 2);
    if (ci < 0 || cj < 0 || ck < 0 || ci >= g.nx || cj >= g.ny || ck >= g.nz) continue;
    const int64_t c = ci + (int64_t)g.nx * (cj + (int64_t)g.ny * ck);
    if (cell_type[c] == UFE_CELL_EXTERNAL) continue;
    const int32_t idx = cut_index[c];
    double kaa = idx >= 0 ? K_cut[(int64_t)idx * 64 + a * 9] : g.h * q1_khat(a, a);
    if (kappa) kaa *= kappa[c];
    const int32_t sub = sub_of_cell[c];
    for (int t = 0; t < nn[d]; ++t)
      if (neigh[d * 8 + t] == sub) diag[t] += kaa;
  }
  double sum = 0.0;
  for (int t = 0; t < nn[d]; ++t) sum += diag[t];
  for (int t = 0; t < nn[d]; ++t) w[d * 8 + t] = diag[t] / sum;
}

// variant 2: every DOF of an edge object takes part in the relabelling, from its own id
__global__ void k_v2_prepare(int64_t n_dof, const int32_t* __restrict__ obj_of_dof, const int32_t* __restrict__ obj_kind,
                             uint8_t* __restrict__ corner, uint8_t* __restrict__ active, int32_t* __restrict__ label2,
                             const int32_t* __restrict__ label) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dof) return;
  const int32_t o = obj_of_dof[d];
  const bool is_edge = o >= 0 && obj_kind[o] == UFE_OBJ_EDGE;
  corner[d] = 0;
  active[d] = is_edge ? 1 : 0;
  label2[d] = is_edge ? (int32_t)d : label[d];
}

// variant 1: DOFs of edge objects incident to a cut FE edge of the same object
__global__ void k_v1_corners(GridGeom g, int64_t n_dof, const int32_t* __restrict__ node_of_dof,
                             const int32_t* __restrict__ dof_of_node, const uint8_t* __restrict__ cell_type,
                             const double* __restrict__ phi, const int32_t* __restrict__ obj_of_dof,
                             const int32_t* __restrict__ obj_kind, uint8_t* __restrict__ corner,
                             uint8_t* __restrict__ active, int32_t* __restrict__ label2,
                             const int32_t* __restrict__ label) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dof) return;
  const int32_t o = obj_of_dof[d];
  bool is_edge = o >= 0 && obj_kind[o] == UFE_OBJ_EDGE;
  bool cut = false;
  if (is_edge) {
    const bool in_d = phi[node_of_dof[d]] < 0.0;
    for_fe_neighbours(g, node_of_dof, dof_of_node, cell_type, d, [&](int64_t e, int64_t wv) {
      if (obj_of_dof[e] != o) return;
      if ((phi[wv] < 0.0) != in_d) cut = true;
    });
  }
  corner[d] = cut ? 1 : 0;
  active[d] = (is_edge && !cut) ? 1 : 0;
  label2[d] = is_edge ? (int32_t)d : label[d];
}

__global__ void k_rep_flags(int64_t n, const int32_t* __restrict__ label, uint8_t* __restrict__ f) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d < n) f[d] = (label[d] >= 0 && label[d] == d) ? 1 : 0;
}

__global__ void k_obj_assign(int64_t n, const int32_t* __restrict__ label, const int32_t* __restrict__ rep_index,
                             int32_t* __restrict__ obj_of_dof, int32_t* __restrict__ obj_size,
                             int32_t* __restrict__ obj_rep) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const int32_t l = label[d];
  if (l < 0) {
    obj_of_dof[d] = -1;
    return;
  }
  const int32_t o = rep_index[l];
  obj_of_dof[d] = o;
  atomicAdd(obj_size + o, 1);
  if (l == d) obj_rep[o] = (int32_t)d;
}

// kinds: |neigh| = 2 -> face; else 1 DOF -> corner, more -> edge.  With prev_kind
// (variant 1) faces and corners keep their kind and split edges follow the rule
// above, a DOF on a cut FE edge being a corner.
__global__ void k_obj_kind(int64_t n_obj, const int32_t* __restrict__ obj_rep, const int32_t* __restrict__ obj_size,
                           const uint8_t* __restrict__ nn, const int32_t* __restrict__ prev_obj,
                           const int32_t* __restrict__ prev_kind, const uint8_t* __restrict__ corner,
                           int32_t* __restrict__ kind) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  const int32_t rep = obj_rep[o];
  int k;
  if (nn[rep] == 2)
    k = UFE_OBJ_FACE;
  else
    k = obj_size[o] == 1 ? UFE_OBJ_CORNER : UFE_OBJ_EDGE;
  if (prev_kind) {
    const int pk = prev_kind[prev_obj[rep]];
    if (pk == UFE_OBJ_FACE) k = UFE_OBJ_FACE;
    else if (pk == UFE_OBJ_CORNER) k = UFE_OBJ_CORNER;
    else if (corner[rep]) k = UFE_OBJ_CORNER;
  }
  kind[o] = k;
}

__global__ void k_coarse_list(int64_t n_obj, const int32_t* __restrict__ coarse_of_obj, const int32_t* __restrict__ obj_rep,
                              const int32_t* __restrict__ nrows, const uint8_t* __restrict__ nn,
                              int32_t* __restrict__ coarse_obj, int32_t* __restrict__ coarse_rep,
                              uint8_t* __restrict__ coarse_nn, const int32_t* __restrict__ neigh,
                              int32_t* __restrict__ nC) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  const int32_t c = coarse_of_obj[o];
  if (c < 0) return;
  const int32_t rep = obj_rep[o];
  for (int t = 0; t < nrows[o]; ++t) {
    coarse_obj[c + t] = (int32_t)o;
    coarse_rep[c + t] = rep;
    coarse_nn[c + t] = nn[rep];
  }
  for (int k = 0; k < nn[rep]; ++k) atomicAdd(nC + neigh[(int64_t)rep * 8 + k], nrows[o]);
}

// coarse DOFs of subdomain w in increasing order
__global__ void k_sub_coarse_fill(int64_t n_coarse, const int32_t* __restrict__ coarse_rep,
                                  const uint8_t* __restrict__ coarse_nn, const int32_t* __restrict__ neigh,
                                  const int32_t* __restrict__ C_ptr, int32_t* __restrict__ C_list) {
  const int w = blockIdx.x;
  __shared__ int warp_tot[32];
  int base = C_ptr[w];
  for (int64_t c0 = 0; c0 < n_coarse; c0 += blockDim.x) {
    const int64_t c = c0 + threadIdx.x;
    int mem = 0;
    if (c < n_coarse) {
      const int32_t rep = coarse_rep[c];
      for (int k = 0; k < coarse_nn[c]; ++k)
        if (neigh[(int64_t)rep * 8 + k] == w) mem = 1;
    }
    // block exclusive scan of mem (blockDim = 256)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = mem;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    int woff = 0, tot = 0;
    for (int x = 0; x < (int)(blockDim.x >> 5); ++x) {
      if (x < wid) woff += warp_tot[x];
      tot += warp_tot[x];
    }
    if (mem) C_list[base + woff + inc - 1] = (int32_t)c;
    base += tot;
    __syncthreads();
  }
}

__global__ void k_cpos(const int32_t* __restrict__ C_ptr, const int32_t* __restrict__ C_list,
                       const int32_t* __restrict__ coarse_rep, const uint8_t* __restrict__ coarse_nn,
                       const int32_t* __restrict__ neigh, int32_t* __restrict__ cpos) {
  const int w = blockIdx.x;
  for (int i = C_ptr[w] + threadIdx.x; i < C_ptr[w + 1]; i += blockDim.x) {
    const int32_t c = C_list[i];
    const int32_t rep = coarse_rep[c];
    for (int k = 0; k < coarse_nn[c]; ++k)
      if (neigh[(int64_t)rep * 8 + k] == w) cpos[(int64_t)c * 8 + k] = i;
  }
}

// subdomains touching a constrained (Dirichlet / pinned) node
__global__ void k_touch_constrained(GridGeom g, const int32_t* __restrict__ sub_block,
                                    const int32_t* __restrict__ sub_of_cell, const int32_t* __restrict__ dof_of_node,
                                    const uint8_t* __restrict__ node_flags, int* __restrict__ touches) {
  const int w = blockIdx.x;
  const int b = sub_block[w];
  const int bi = b % g.bx, bj = (b / g.bx) % g.by, bk = b / (g.bx * g.by);
  int t = 0;
  for (int lc = threadIdx.x; lc < g.sx * g.sy * g.sz; lc += blockDim.x) {
    const int li = lc % g.sx, lj = (lc / g.sx) % g.sy, lk = lc / (g.sx * g.sy);
    const int gi = bi * g.sx + li, gj = bj * g.sy + lj, gk = bk * g.sz + lk;
    if (sub_of_cell[g.cell(gi, gj, gk)] != w) continue;
    for (int a = 0; a < 8; ++a) {
      const int64_t v = g.node(gi + (a & 1), gj + ((a >> 1) & 1), gk + (a >> 2));
      if ((node_flags[v] & 1) && dof_of_node[v] < 0) t = 1;
    }
  }
  t = __syncthreads_or(t);
  if (threadIdx.x == 0) touches[w] = t;
}

// ---------------------------------------------------------------------------
// local matrices (Sect. 3.1): A^w from the cells of w, split into II, IG, GG
// ---------------------------------------------------------------------------
// entry A^w((node1, c1), (node2, c2)) of two local nodes of subdomain w: sum over the
// cells of w containing both (kappa h Khat for internal cells, the cut-cell matrix
// otherwise; element DOF ncomp a + c)
__device__ double local_entry(const SubMeta& sm, int w, int bi, int bj, int bk, int lx, int ly, int lz, int lx2,
                              int ly2, int lz2, int c1, int c2) {
  const GridGeom& g = sm.g;
  const int nc = sm.ncomp, ne = 8 * nc;
  double val = 0.0;
  for (int cz = max(lz, lz2) - 1; cz <= min(lz, lz2); ++cz) {
    if (cz < 0 || cz >= g.sz) continue;
    for (int cy = max(ly, ly2) - 1; cy <= min(ly, ly2); ++cy) {
      if (cy < 0 || cy >= g.sy) continue;
      for (int cx = max(lx, lx2) - 1; cx <= min(lx, lx2); ++cx) {
        if (cx < 0 || cx >= g.sx) continue;
        const int64_t c = g.cell(bi * g.sx + cx, bj * g.sy + cy, bk * g.sz + cz);
        if (sm.sub_of_cell[c] != w) continue;
        const int a = (lx - cx) + 2 * (ly - cy) + 4 * (lz - cz);
        const int bb = (lx2 - cx) + 2 * (ly2 - cy) + 4 * (lz2 - cz);
        const int ra = nc * a + c1, rb = nc * bb + c2;
        const double kap = sm.kappa ? sm.kappa[c] : 1.0;
        double kab;
        if (sm.cell_type[c] == UFE_CELL_INTERNAL)
          kab = nc == 1 ? g.h * q1_khat(a, bb) : sm.Kref[ra * 24 + rb];
        else
          kab = sm.K_cut[(int64_t)sm.cut_index[c] * ne * ne + ra * ne + rb];
        val += kap * kab;
      }
    }
  }
  return val;
}

// CTAs per subdomain for the stencil-by-stencil set-up kernels (9^3 nodes x 27
// neighbours of work per subdomain: one CTA alone is latency bound)
constexpr int kLocalSplit = 8;

// dense A_II and A_GG of every subdomain (Sect. 3.1: Neumann matrix over the cells of w);
// local vector index NC p + c
template <int NC>
__global__ void k_local_assemble(SubMeta sm, const int64_t* __restrict__ oII, const int64_t* __restrict__ oGG,
                                 double* __restrict__ AII, double* __restrict__ AGG) {
  const GridGeom& g = sm.g;
  const int w = blockIdx.x;
  const int b = sm.sub_block[w];
  const int bi = b % g.bx, bj = (b / g.bx) % g.by, bk = b / (g.bx * g.by);
  const int nI = sm.vI_ptr[w + 1] - sm.vI_ptr[w], nG = sm.vG_ptr[w + 1] - sm.vG_ptr[w];
  const int ldI = pad4(nI), ldG = pad4(nG);
  const int32_t* lm = sm.lmap + (int64_t)w * g.n_local_nodes;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < g.n_local_nodes * 27; e += blockDim.x * gridDim.y) {
    const int ln = e / 27, o = e % 27;
    const int32_t c1 = lm[ln];
    const int k1 = lmap_kind(c1);
    if (k1 == LKIND_NONE) continue;
    const int lx = ln % g.lnx, ly = (ln / g.lnx) % g.lny, lz = ln / (g.lnx * g.lny);
    const int lx2 = lx + (o % 3) - 1, ly2 = ly + ((o / 3) % 3) - 1, lz2 = lz + (o / 9) - 1;
    if (lx2 < 0 || ly2 < 0 || lz2 < 0 || lx2 >= g.lnx || ly2 >= g.lny || lz2 >= g.lnz) continue;
    const int32_t c2 = lm[lx2 + g.lnx * (ly2 + g.lny * lz2)];
    const int k2 = lmap_kind(c2);
    if (k2 != k1) continue;
    const int p1 = lmap_index(c1), p2 = lmap_index(c2);
    for (int a1 = 0; a1 < NC; ++a1)
      for (int a2 = 0; a2 < NC; ++a2) {
        const double val = local_entry(sm, w, bi, bj, bk, lx, ly, lz, lx2, ly2, lz2, a1, a2);
        const int64_t r = NC * p1 + a1, q = NC * p2 + a2;
        if (k1 == LKIND_I)
          AII[oII[w] + r * ldI + q] = val;
        else
          AGG[oGG[w] + r * ldG + q] = val;
      }
  }
}

// Off-diagonal blocks in ELL form.  A_GI: for each interface vector DOF j of w, the
// interior vector DOFs k among the 27 neighbouring nodes (slot o NC + c2, -1 when
// empty) and A^w_jk; layout per subdomain slot-major (entry KS g0 + slot nG + j, KS =
// 27 NC, g0 = vG_ptr[w]) so that rows are read coalesced.  A_IG likewise over the
// interior rows (entry KS i0 + slot nI + p).
template <int NC>
__global__ void k_off_ell(SubMeta sm, int rows_kind, int32_t* __restrict__ ell_k, double* __restrict__ ell_v) {
  const GridGeom& g = sm.g;
  const int w = blockIdx.x;
  const int b = sm.sub_block[w];
  const int bi = b % g.bx, bj = (b / g.bx) % g.by, bk = b / (g.bx * g.by);
  const int col_kind = rows_kind == LKIND_G ? LKIND_I : LKIND_G;
  const int32_t* vptr = rows_kind == LKIND_G ? sm.vG_ptr : sm.vI_ptr;
  const int nR = vptr[w + 1] - vptr[w];
  const int64_t base = 27 * NC * (int64_t)vptr[w];
  const int32_t* lm = sm.lmap + (int64_t)w * g.n_local_nodes;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < g.n_local_nodes * 27; e += blockDim.x * gridDim.y) {
    const int ln = e / 27, o = e % 27;
    const int32_t c1 = lm[ln];
    if (lmap_kind(c1) != rows_kind) continue;
    const int lx = ln % g.lnx, ly = (ln / g.lnx) % g.lny, lz = ln / (g.lnx * g.lny);
    const int lx2 = lx + (o % 3) - 1, ly2 = ly + ((o / 3) % 3) - 1, lz2 = lz + (o / 9) - 1;
    int p2 = -1;
    if (lx2 >= 0 && ly2 >= 0 && lz2 >= 0 && lx2 < g.lnx && ly2 < g.lny && lz2 < g.lnz) {
      const int32_t c2 = lm[lx2 + g.lnx * (ly2 + g.lny * lz2)];
      if (lmap_kind(c2) == col_kind) p2 = lmap_index(c2);
    }
    for (int a1 = 0; a1 < NC; ++a1)
      for (int a2 = 0; a2 < NC; ++a2) {
        const int64_t slot = base + (int64_t)(o * NC + a2) * nR + NC * lmap_index(c1) + a1;
        ell_k[slot] = p2 >= 0 ? NC * p2 + a2 : -1;
        ell_v[slot] = p2 >= 0 ? local_entry(sm, w, bi, bj, bk, lx, ly, lz, lx2, ly2, lz2, a1, a2) : 0.0;
      }
  }
}

// scaled A^_GI entries: s_G[j] A_GI[j][k] s_I[k]  (KS = 27 NC slots per row)
template <typename T>
__global__ void k_ell_scale(SubMeta sm, int KS, const int32_t* __restrict__ ell_k, const double* __restrict__ ell_v,
                            const double* __restrict__ sI, const double* __restrict__ sG, T* __restrict__ ell_s,
                            const int32_t* __restrict__ wl) {
  const int w = wl ? wl[blockIdx.y] : (int)blockIdx.y;
  const int nG = sm.vG_ptr[w + 1] - sm.vG_ptr[w];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nG * KS; e += gridDim.x * blockDim.x) {
    const int64_t slot = (int64_t)sm.vG_ptr[w] * KS + e;
    const int32_t k = ell_k[slot];
    ell_s[slot] = k < 0 ? T(0) : (T)(ell_v[slot] * sG[sm.vG_ptr[w] + e % nG] * sI[sm.vI_ptr[w] + k]);
  }
}

// X^T = (A^_II^-1 A^_IG)^T, row j = sum_k A^_GI[j][k] A^_II^-1[k][:]  (A^_II^-1 symmetric)
constexpr int kMaxKS = 81;
template <typename T>
__global__ void __launch_bounds__(256)
k_xt(SubMeta sm, int KS, const int64_t* __restrict__ oII, const int64_t* __restrict__ oGI,
     const int32_t* __restrict__ ell_k, const T* __restrict__ ell_s, const T* __restrict__ IIinv, T* __restrict__ Xt,
     const int32_t* __restrict__ wl) {
  __shared__ int32_t sk[8][kMaxKS];
  __shared__ T sv[8][kMaxKS];
  const int w = wl ? wl[blockIdx.y] : (int)blockIdx.y;
  const int nI = sm.vI_ptr[w + 1] - sm.vI_ptr[w], nG = sm.vG_ptr[w + 1] - sm.vG_ptr[w];
  const int ldI = pad4(nI);
  const int j0 = blockIdx.x * 8;
  if (j0 >= nG) return;
  for (int e = threadIdx.x; e < 8 * KS; e += blockDim.x) {
    const int jj = e / KS, o = e % KS;
    const bool ok = j0 + jj < nG;
    const int64_t slot = KS * (int64_t)sm.vG_ptr[w] + (int64_t)o * nG + j0 + jj;
    sk[jj][o] = ok ? ell_k[slot] : -1;
    sv[jj][o] = ok ? ell_s[slot] : T(0);
  }
  __syncthreads();
  const T* Ainv = IIinv + oII[w];
  for (int jj = 0; jj < 8 && j0 + jj < nG; ++jj) {
    for (int c = threadIdx.x; c < ldI; c += blockDim.x) {
      T acc = T(0);
      for (int o = 0; o < KS; ++o) {
        const int32_t k = sk[jj][o];
        if (k >= 0) acc += sv[jj][o] * Ainv[(int64_t)k * ldI + c];
      }
      Xt[oGI[w] + (int64_t)(j0 + jj) * ldI + c] = acc;
    }
  }
}

// S^ = A^_GG - A^_GI X^ ; row j of the result is written from column j of the product
// (S^ is symmetric): S^[j][i] -= sum_k A^_GI[i][k] X^T[j][k]
template <typename T>
__global__ void __launch_bounds__(256)
k_schur(SubMeta sm, int KS, const int64_t* __restrict__ oGG, const int64_t* __restrict__ oGI,
        const int32_t* __restrict__ ell_k, const T* __restrict__ ell_s, const T* __restrict__ Xt, T* __restrict__ GG,
        const int32_t* __restrict__ wl) {
  extern __shared__ __align__(16) char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  const int w = wl ? wl[blockIdx.y] : (int)blockIdx.y, j = blockIdx.x;
  const int nI = sm.vI_ptr[w + 1] - sm.vI_ptr[w], nG = sm.vG_ptr[w + 1] - sm.vG_ptr[w];
  if (j >= nG) return;
  const int ldI = pad4(nI), ldG = pad4(nG);
  for (int c = threadIdx.x; c < nI; c += blockDim.x) xs[c] = Xt[oGI[w] + (int64_t)j * ldI + c];
  __syncthreads();
  for (int i = threadIdx.x; i < nG; i += blockDim.x) {
    const int64_t base = KS * (int64_t)sm.vG_ptr[w] + i;
    T acc = T(0);
    for (int o0 = 0; o0 < KS; o0 += 27) {
      int32_t kk[27];
      T vv[27];
#pragma unroll
      for (int o = 0; o < 27; ++o) {
        kk[o] = ell_k[base + (int64_t)(o0 + o) * nG];
        vv[o] = ell_s[base + (int64_t)(o0 + o) * nG];
      }
#pragma unroll
      for (int o = 0; o < 27; ++o)
        if (kk[o] >= 0) acc += vv[o] * xs[kk[o]];
    }
    GG[oGG[w] + (int64_t)j * ldG + i] -= acc;
  }
}

// Jacobi scales s = diag^-1/2 and the raw interface diagonal (stiffness weights).  For
// elasticity the interface scale is s = (max(diag, tau max_w diag))^-1/2 with tau a
// small fraction of the largest interface diagonal of the subdomain: DOFs whose
// support in the cut cells is tiny (diagonals down to 1e-30 of their neighbours)
// would otherwise carry constraint-row entries (C D^-1/2) of up to 1e15 and, with
// several coarse rows per object, make S_c = C S'^-1 C^T numerically singular.  Any
// positive scaling is an exact change of variables; Poisson (one row per object)
// keeps the plain Jacobi scale (tau = 0).
__global__ void k_local_diag(SubMeta sm, double tau, const int64_t* __restrict__ oII, const int64_t* __restrict__ oGG,
                             const double* __restrict__ AII, const double* __restrict__ AGG, double* __restrict__ sI,
                             double* __restrict__ sG, double* __restrict__ dGraw) {
  __shared__ double red[32];
  const int w = blockIdx.x;
  const int nI = sm.vI_ptr[w + 1] - sm.vI_ptr[w], nG = sm.vG_ptr[w + 1] - sm.vG_ptr[w];
  const int ldI = pad4(nI), ldG = pad4(nG);
  for (int p = threadIdx.x; p < nI; p += blockDim.x) sI[sm.vI_ptr[w] + p] = 1.0 / sqrt(AII[oII[w] + (int64_t)p * ldI + p]);
  double mx = 0.0;
  for (int p = threadIdx.x; p < nG; p += blockDim.x) mx = fmax(mx, AGG[oGG[w] + (int64_t)p * ldG + p]);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const double floor_d = tau * red[0];
  for (int p = threadIdx.x; p < nG; p += blockDim.x) {
    const double d = AGG[oGG[w] + (int64_t)p * ldG + p];
    dGraw[sm.vG_ptr[w] + p] = d;
    sG[sm.vG_ptr[w] + p] = 1.0 / sqrt(fmax(d, floor_d));
  }
}

// weights per interface vector slot: stiffness A^w_xx / sum_w' A^w'_xx (Eq. alge-weighting,
// per component) or 1/|neigh| (Eq. weighting)
__global__ void k_weights(int64_t n_dof, int nc, const uint8_t* __restrict__ nn, const int32_t* __restrict__ gpos,
                          const double* __restrict__ dGraw, int topological, double* __restrict__ w) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dof || nn[d] < 2) return;
  const int cnt = nn[d];
  for (int c = 0; c < nc; ++c) {
    double sum = 0.0;
    for (int k = 0; k < cnt; ++k) sum += dGraw[(int64_t)nc * gpos[d * 8 + k] + c];
    for (int k = 0; k < cnt; ++k) {
      const int64_t s = (int64_t)nc * gpos[d * 8 + k] + c;
      w[s] = topological ? 1.0 / cnt : dGraw[s] / sum;
    }
  }
}

// scale and convert: dst[i][j] = src[i][j] * sr_i * sc_j  (FP64 -> T); grid (row chunks, subdomain)
template <typename T>
__global__ void k_scale_block(const double* __restrict__ src, T* __restrict__ dst, const int64_t* __restrict__ off,
                              const int32_t* __restrict__ rptr, const int32_t* __restrict__ cptr,
                              const double* __restrict__ sr, const double* __restrict__ scl,
                              const int32_t* __restrict__ wl) {
  const int w = wl ? wl[blockIdx.y] : (int)blockIdx.y;
  const int nr = rptr[w + 1] - rptr[w], nc = cptr[w + 1] - cptr[w];
  const int ld = pad4(nc);
  const int64_t o = off[w];
  // the local matrices are sparse (at most 27 nonzeros per row of a few hundred): only
  // nonzeros are scaled, which keeps this pass at memory speed on the scarce FP64 pipe
  for (int i = blockIdx.x; i < nr; i += gridDim.x) {
    const double ri = sr[rptr[w] + i];
    for (int j = threadIdx.x; j < ld; j += blockDim.x) {
      const double a = j < nc ? src[o + (int64_t)i * ld + j] : 0.0;
      dst[o + (int64_t)i * ld + j] = (T)(a != 0.0 ? a * ri * scl[cptr[w] + j] : 0.0);
    }
  }
}

// scaled constraint rows C^ = C D_G^-1/2, C_rho = diag(rho) C^ with rho_l = 1 / |C^_l|^2.
// The rows of an object (consecutive coarse ids from coarse_of_obj[o]): Poisson, the
// uniform nodal mean (Eq. coarse-dofs); elasticity, the mean of each component and
// the kept rotation moments (1/n) sum (y x u)_k with y the node's grid position
// relative to the object's centroid (bit k of obj_rot).
template <typename T, int NC>
__global__ void k_constraints(SubMeta sm, const int32_t* __restrict__ node_of_dof,
                              const int32_t* __restrict__ obj_of_dof, const int32_t* __restrict__ coarse_of_obj,
                              const int32_t* __restrict__ obj_size, const int32_t* __restrict__ obj_rot,
                              const long long* __restrict__ obj_sum, const double* __restrict__ sG,
                              const int64_t* __restrict__ oCG, T* __restrict__ Cs, T* __restrict__ Crho,
                              double* __restrict__ rho, const int32_t* __restrict__ wl) {
  const int w = wl ? wl[blockIdx.x] : (int)blockIdx.x;
  const int nGn = sm.G_ptr[w + 1] - sm.G_ptr[w];
  const int nG = sm.vG_ptr[w + 1] - sm.vG_ptr[w];
  const int c0 = sm.C_ptr[w], nC = sm.C_ptr[w + 1] - c0;
  const int ldG = pad4(nG);
  const int g0 = sm.vG_ptr[w];
  T* Cw = Cs + oCG[w];
  for (int j = threadIdx.x; j < nGn; j += blockDim.x) {
    const int32_t d = sm.G_list[sm.G_ptr[w] + j];
    const int32_t o = obj_of_dof[d];
    const int32_t c = coarse_of_obj[o];
    if (c < 0 || nC == 0) continue;
    int lo = 0, hi = nC - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sm.C_list[c0 + mid] < c) lo = mid + 1; else hi = mid;
    }
    const double inv_n = 1.0 / obj_size[o];
    for (int a = 0; a < NC; ++a) Cw[(int64_t)(lo + a) * ldG + NC * j + a] = (T)(sG[g0 + NC * j + a] * inv_n);
    if (NC == 3 && obj_rot[o]) {
      const int64_t v = node_of_dof[d];
      const GridGeom& g = sm.g;
      const int64_t ijk[3] = {v % (g.nx + 1), (v / (g.nx + 1)) % (g.ny + 1), v / ((int64_t)(g.nx + 1) * (g.ny + 1))};
      double y[3];
      for (int k = 0; k < 3; ++k) y[k] = (double)ijk[k] - (double)obj_sum[3 * (int64_t)o + k] * inv_n;
      int t = 0;
      for (int k = 0; k < 3; ++k) {
        if (!((obj_rot[o] >> k) & 1)) continue;
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        T* row = Cw + (int64_t)(lo + 3 + t) * ldG + NC * j;
        row[k2] = (T)(y[k1] * inv_n * sG[g0 + NC * j + k2]);
        row[k1] = (T)(-y[k2] * inv_n * sG[g0 + NC * j + k1]);
        ++t;
      }
    }
  }
  __syncthreads();
  // rho_l = 1 / |C^_l|^2, each row summed in order by one thread (deterministic)
  for (int i = threadIdx.x; i < nC; i += blockDim.x) {
    double nrm = 0.0;
    for (int j = 0; j < nG; ++j) {
      const double v = (double)Cw[(int64_t)i * ldG + j];
      nrm += v * v;
    }
    rho[c0 + i] = 1.0 / nrm;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nC * ldG; e += blockDim.x) {
    const int i = e / ldG;
    Crho[oCG[w] + e] = (T)((double)Cw[e] * rho[c0 + i]);
  }
}

// object geometry for the elastic rows: sums and bounds of the node grid coordinates
__global__ void k_obj_geom(GridGeom g, int64_t n_dof, const int32_t* __restrict__ node_of_dof,
                           const int32_t* __restrict__ obj_of_dof, long long* __restrict__ sum,
                           int32_t* __restrict__ lo, int32_t* __restrict__ hi) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dof) return;
  const int32_t o = obj_of_dof[d];
  if (o < 0) return;
  const int64_t v = node_of_dof[d];
  const int c[3] = {(int)(v % (g.nx + 1)), (int)((v / (g.nx + 1)) % (g.ny + 1)),
                    (int)(v / ((int64_t)(g.nx + 1) * (g.ny + 1)))};
  for (int k = 0; k < 3; ++k) {
    atomicAdd(reinterpret_cast<unsigned long long*>(sum + 3 * (int64_t)o + k), (unsigned long long)c[k]);
    atomicMin(lo + 3 * (int64_t)o + k, c[k]);
    atomicMax(hi + 3 * (int64_t)o + k, c[k]);
  }
}

// coarse rows of every object: 1 (Poisson); 3 component means plus a rotation row
// about each axis k unless all nodes share coordinates k+1 and k+2 (elasticity);
// counts[o] = rows of the kept (coarse) objects, 0 otherwise
__global__ void k_obj_rows(int64_t n_obj, int nc, const int32_t* __restrict__ kind, int coarse,
                           const int32_t* __restrict__ size, const int32_t* __restrict__ lo,
                           const int32_t* __restrict__ hi, int32_t* __restrict__ nrows, int32_t* __restrict__ rot,
                           int32_t* __restrict__ counts) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  int r = 1, bits = 0;
  if (nc == 3) {
    r = 3;
    if (size[o] > 1)
      for (int k = 0; k < 3; ++k) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        if (lo[3 * o + k1] != hi[3 * o + k1] || lo[3 * o + k2] != hi[3 * o + k2]) {
          bits |= 1 << k;
          ++r;
        }
      }
  }
  nrows[o] = r;
  rot[o] = bits;
  const int k = kind[o];
  const bool keep = (k == UFE_OBJ_CORNER) || (k == UFE_OBJ_EDGE && coarse >= UFE_COARSE_CE) ||
                    (k == UFE_OBJ_FACE && coarse >= UFE_COARSE_CEF);
  counts[o] = keep ? r : 0;
}

__global__ void k_coarse_first(int64_t n_obj, const int32_t* __restrict__ counts, const int32_t* __restrict__ offs,
                               int32_t* __restrict__ coarse_of_obj) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o < n_obj) coarse_of_obj[o] = counts[o] > 0 ? offs[o] : -1;
}

// A_c^w = (C S'^-1 C^T)^-1 - rho  (FP64)
template <typename T>
__global__ void k_coarse_local(const int32_t* __restrict__ C_ptr, const int64_t* __restrict__ oCC,
                               const T* __restrict__ invSc, const double* __restrict__ rho, double* __restrict__ Acw,
                               const int32_t* __restrict__ wl) {
  const int w = wl ? wl[blockIdx.x] : (int)blockIdx.x;
  const int c0 = C_ptr[w], nC = C_ptr[w + 1] - c0, ldC = pad4(nC);
  for (int e = threadIdx.x; e < nC * nC; e += blockDim.x) {
    const int i = e / nC, j = e % nC;
    double v = (double)invSc[oCC[w] + (int64_t)i * ldC + j];
    if (i == j) v -= rho[c0 + i];
    Acw[oCC[w] + (int64_t)i * ldC + j] = v;
  }
}

// accuracy of the coarse basis of each subdomain: E = C Phi (computed from the stored
// operators) must be the identity (Sect. 3.2: Phi^w is defined by C Phi = I); err[w] =
// max |E - I|, and a subdomain above tol is flagged DEV_ILLCOND
template <typename T>
__global__ void k_cphi_error(const int32_t* __restrict__ C_ptr, const int64_t* __restrict__ oCC,
                             const T* __restrict__ E, double tol, double* __restrict__ err, int* status,
                             const int32_t* __restrict__ wl) {
  const int w = wl ? wl[blockIdx.x] : (int)blockIdx.x;
  const int nC = C_ptr[w + 1] - C_ptr[w], ldC = pad4(nC);
  double m = 0.0;
  for (int e = threadIdx.x; e < nC * nC; e += blockDim.x) {
    const int i = e / nC, j = e % nC;
    const double v = (double)E[oCC[w] + (int64_t)i * ldC + j] - (i == j ? 1.0 : 0.0);
    m = fmax(m, isfinite(v) ? fabs(v) : INFINITY);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, red[k]);
    m = fmax(m, red[0]);
    err[w] = m;
    if (!(m <= tol)) atomicOr(status + w, DEV_ILLCOND);
  }
}

// coarse matrix: row l gathers A_c^w of every subdomain w in neigh(l), in neigh order
__global__ void k_coarse_assemble(int64_t n_coarse, int ldc, const int32_t* __restrict__ coarse_rep,
                                  const uint8_t* __restrict__ coarse_nn, const int32_t* __restrict__ neigh,
                                  const int32_t* __restrict__ cpos, const int32_t* __restrict__ C_ptr,
                                  const int32_t* __restrict__ C_list, const int64_t* __restrict__ oCC,
                                  const double* __restrict__ Acw, double* __restrict__ Ac) {
  const int64_t l = blockIdx.x;
  const int32_t rep = coarse_rep[l];
  for (int k = 0; k < coarse_nn[l]; ++k) {
    const int w = neigh[(int64_t)rep * 8 + k];
    const int c0 = C_ptr[w], nC = C_ptr[w + 1] - c0, ldC = pad4(nC);
    const int i = cpos[l * 8 + k] - c0;
    for (int j = threadIdx.x; j < nC; j += blockDim.x)
      Ac[l * ldc + C_list[c0 + j]] += Acw[oCC[w] + (int64_t)i * ldC + j];
    __syncthreads();
  }
}

__global__ void k_symmetrize(double* A, int n, int ld) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (j <= i) return;
  const double v = 0.5 * (A[(int64_t)i * ld + j] + A[(int64_t)j * ld + i]);
  A[(int64_t)i * ld + j] = v;
  A[(int64_t)j * ld + i] = v;
}

__global__ void k_scale_ptr(int64_t n, int nc, const int32_t* __restrict__ in, int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = nc * in[i];
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static void propagate(const Mesh& m, cudaStream_t s, const uint8_t* active, int mode, const int32_t* std_obj,
                      int32_t* label, const double* wv2 = nullptr) {
  DBuf<int> changed;
  changed.alloc(1, s);
  for (int round = 0; round < 512; ++round) {
    changed.zero();
    for (int rep = 0; rep < 4; ++rep) {
      k_obj_propagate<<<grid_for(m.n_dof, 256), 256, 0, s>>>(m.g, m.n_dof, m.node_of_dof.p, m.dof_of_node.p,
                                                             m.cell_type.p, m.neigh.p, m.n_neigh.p, m.phi.p, std_obj,
                                                             active, mode, wv2, label, changed.p);
      UFE_CHECK_LAUNCH();
    }
    if (scalar_to_host(changed.p, s) == 0) return;
  }
  throw Error{UFE_ERR_TIMEOUT, "object labelling did not converge"};
}

__global__ void k_init_labels(int64_t n, const uint8_t* __restrict__ nn, int32_t* __restrict__ label,
                              uint8_t* __restrict__ active) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const bool g = nn[d] >= 2;
  label[d] = g ? (int32_t)d : -1;
  active[d] = g ? 1 : 0;
}

// Steps 8, 9 and the C Phi = I test of an FP32 pass, run on a second stream beside the
// coarse set-up (which needs only A_c^w, step 10): `pending` once they are queued,
// `done` recorded after them, `err` the per-subdomain |C Phi - I| (finish_deferred).
struct DeferredCheck {
  bool pending = false;
  cudaEvent_t done = nullptr;
  DBuf<double> err;
  ~DeferredCheck() {
    if (done) cudaEventDestroy(done);
  }
};

static cudaStream_t objects_stream();

// scaled A_II in precision T and its inverse (step 1 of the local factorisations; it
// needs only the mesh, so it runs while the objects are found); the pivot flags land
// in status and are checked with the later steps.  ws lists the subdomains to factor
// (wl: the same list on the device, or null when ws holds every subdomain).
template <typename T>
static void factor_interior(Bddc& B, const std::vector<int64_t>& oII, int64_t nII, DBuf<double>& AII,
                            DBuf<double>& sI, DBuf<T>& II, DBuf<int>& status, const std::vector<int>& ws,
                            const int32_t* wl) {
  cudaStream_t s = B.stream;
  const int nw = (int)ws.size();
  status.zero();
  DBuf<int64_t> dII;
  dII.alloc(std::max<size_t>(oII.size(), 1), s);
  UFE_CUDA(cudaMemcpyAsync(dII.p, oII.data(), oII.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  II.alloc(std::max<int64_t>(nII, 1), s);
  if (nw > 0)
    k_scale_block<T><<<dim3(64, nw), 128, 0, s>>>(AII.p, II.p, dII.p, B.vI_ptr.p, B.vI_ptr.p, sI.p, sI.p, wl);
  UFE_CHECK_LAUNCH();
  std::vector<InvDesc> inv;
  for (int w : ws) inv.push_back({B.h_nI[w], pad4(B.h_nI[w]), oII[w]});
  batched_inverse<T>(inv, II.p, status.p, s, sizeof(T) == 4 ? T(1e-3) : T(0));
}

template <typename T>
static void factor_pipeline(Bddc& B, const std::vector<int64_t>& oII, const std::vector<int64_t>& oIG,
                            const std::vector<int64_t>& oGG, const std::vector<int64_t>& oCG,
                            const std::vector<int64_t>& oGC, const std::vector<int64_t>& oCC, int64_t nII, int64_t nIG,
                            int64_t nGG, int64_t nCG, int64_t nGC, int64_t nCC, DBuf<double>& AII, DBuf<double>& AIG,
                            DBuf<double>& AGG, DBuf<double>& sI, DBuf<double>& sG, DBuf<int32_t>& ell_k,
                            DBuf<double>& ell_v, DBuf<T>& II, DBuf<T>& GG,
                            DBuf<T>& GC, DBuf<double>& Acw, DBuf<double>& rho, DBuf<int>& status,
                            bool interior_ready, const std::vector<int>& ws, const int32_t* wl,
                            std::vector<char>* bad, DeferredCheck* later = nullptr) {
  if (!interior_ready) factor_interior<T>(B, oII, nII, AII, sI, II, status, ws, wl);
  Mesh& m = *B.mesh;
  cudaStream_t s = B.stream;
  const int ns = (int)m.n_sub;
  const int nw = (int)ws.size();
  const SubMeta sm = B.meta();
  auto up = [&](const std::vector<int64_t>& v) {
    DBuf<int64_t>* d = new DBuf<int64_t>();
    d->alloc(v.size(), s);
    UFE_CUDA(cudaMemcpyAsync(d->p, v.data(), v.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    return std::unique_ptr<DBuf<int64_t>>(d);
  };
  auto dII = up(oII), dIG = up(oIG), dGG = up(oGG), dCG = up(oCG), dCC = up(oCC);
  // scaled blocks in precision T (A_II: factor_interior)
  DBuf<T> Cs, Crho, X, Y, Sc;
  GG.alloc(std::max<int64_t>(nGG, 1), s);
  k_scale_block<T><<<dim3(64, nw), 128, 0, s>>>(AGG.p, GG.p, dGG->p, B.vG_ptr.p, B.vG_ptr.p, sG.p, sG.p, wl);
  UFE_CHECK_LAUNCH();
  Cs.alloc(std::max<int64_t>(nCG, 1), s);
  Crho.alloc(std::max<int64_t>(nCG, 1), s);
  Cs.zero();
  if (!wl) rho.alloc(std::max<int64_t>(B.n_Cloc, 1), s);   // a subset pass keeps the others' rho
  if (B.ncomp == 3)
    k_constraints<T, 3><<<nw, 256, 0, s>>>(sm, m.node_of_dof.p, B.obj_of_dof.p, B.coarse_of_obj.p, B.obj_size.p,
                                           B.obj_rot.p, B.obj_sum.p, sG.p, dCG->p, Cs.p, Crho.p, rho.p, wl);
  else
    k_constraints<T, 1><<<nw, 256, 0, s>>>(sm, m.node_of_dof.p, B.obj_of_dof.p, B.coarse_of_obj.p, B.obj_size.p,
                                           B.obj_rot.p, B.obj_sum.p, sG.p, dCG->p, Cs.p, Crho.p, rho.p, wl);
  UFE_CHECK_LAUNCH();

  // a non-positive pivot in one of the local inversions (in FP32 also a pivot of a
  // Jacobi-scaled matrix below 1e-3: the operators of such a subdomain are too
  // ill-conditioned to be stored and applied in FP32).  With `bad` (the FP32 pass) the
  // subdomain is marked for FP64 operators and the pass goes on (its later products
  // are not used); otherwise the matrix and subdomain are named in the error.
  auto check = [&](const char* what) {
    std::vector<int> st = to_host(status.p, ns, s);
    for (int w : ws)
      UFE_REQUIRE(!(st[w] & DEV_TIMEOUT), UFE_ERR_TIMEOUT,
                  std::string(what) + " of subdomain " + std::to_string(w) + ": a tensor-core copy or product did not "
                  "complete in time");
    for (int w : ws) {
      if (bad) {
        if (st[w] != 0) (*bad)[w] = 1;
        continue;
      }
      UFE_REQUIRE(st[w] == 0, UFE_ERR_SINGULAR_LOCAL,
                  std::string(what) + " of subdomain " + std::to_string(w) +
                      ((st[w] & DEV_SINGULAR) ? " is not positive definite" : " is too ill-conditioned"));
    }
  };
  const T floor = sizeof(T) == 4 ? T(1e-3) : T(0);
  std::vector<InvDesc> inv;
  std::vector<GemmDesc> g;
  // 1. A_II^-1 (factor_interior)
  check("A_II");
  // 2. X^T = (A_II^-1 A_IG)^T and 3. S = A_GG - A_GI X, both from the sparse A_GI
  X.alloc(std::max<int64_t>(nIG, 1), s);
  {
    int nGmax = 1;
    for (int w = 0; w < ns; ++w) nGmax = std::max(nGmax, B.h_nG[w]);
    int nImax = 4;
    for (int w = 0; w < ns; ++w) nImax = std::max(nImax, pad4(B.h_nI[w]));
    const int KS = 27 * B.ncomp;
    DBuf<T> ell_s;
    ell_s.alloc(std::max<int64_t>(B.n_vGloc, 1) * KS, s);
    k_ell_scale<T><<<dim3(8, std::max(nw, 1)), 256, 0, s>>>(sm, KS, ell_k.p, ell_v.p, sI.p, sG.p, ell_s.p, wl);
    UFE_CHECK_LAUNCH();
    k_xt<T><<<dim3((nGmax + 7) / 8, std::max(nw, 1)), 256, 0, s>>>(sm, KS, dII->p, dIG->p, ell_k.p, ell_s.p, II.p, X.p,
                                                                   wl);
    UFE_CHECK_LAUNCH();
    if (nImax * sizeof(T) > 48 * 1024)   // interiors of large blocks
      UFE_CUDA(cudaFuncSetAttribute(k_schur<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(nImax * sizeof(T))));
    k_schur<T><<<dim3(nGmax, std::max(nw, 1)), 256, nImax * sizeof(T), s>>>(sm, KS, dGG->p, dIG->p, ell_k.p, ell_s.p,
                                                                          X.p, GG.p, wl);
    UFE_CHECK_LAUNCH();
  }
  X.release();
  // 4. S' = S + C^T rho C
  g.clear();
  for (int w : ws)
    g.push_back({B.h_nG[w], B.h_nG[w], B.h_nC[w], pad4(B.h_nG[w]), pad4(B.h_nG[w]), pad4(B.h_nG[w]), oCG[w], oCG[w], oGG[w]});
  batched_gemm<T>(true, false, g, Cs.p, Crho.p, GG.p, T(1), T(1), s);
  Crho.release();
  // 5. S'^-1
  inv.clear();
  for (int w : ws) inv.push_back({B.h_nG[w], pad4(B.h_nG[w]), oGG[w]});
  batched_inverse<T>(inv, GG.p, status.p, s, floor);
  check("S' = S + C^T rho C");
  // 6. Y = S'^-1 C^T
  Y.alloc(std::max<int64_t>(nGC, 1), s);
  g.clear();
  for (int w : ws)
    g.push_back({B.h_nG[w], B.h_nC[w], B.h_nG[w], pad4(B.h_nG[w]), pad4(B.h_nG[w]), pad4(B.h_nC[w]), oGG[w], oCG[w], oGC[w]});
  batched_gemm<T>(false, true, g, GG.p, Cs.p, Y.p, T(1), T(0), s);
  // 7. S_c = C Y, then S_c^-1
  Sc.alloc(std::max<int64_t>(nCC, 1), s);
  g.clear();
  for (int w : ws)
    g.push_back({B.h_nC[w], B.h_nC[w], B.h_nG[w], pad4(B.h_nG[w]), pad4(B.h_nC[w]), pad4(B.h_nC[w]), oCG[w], oGC[w], oCC[w]});
  batched_gemm<T>(false, false, g, Cs.p, Y.p, Sc.p, T(1), T(0), s);
  inv.clear();
  for (int w : ws) inv.push_back({B.h_nC[w], pad4(B.h_nC[w]), oCC[w]});
  batched_inverse<T>(inv, Sc.p, status.p, s);
  check("S_c = C S'^-1 C^T");
  // 10. A_c^w = S_c^-1 - rho (FP64), first: the coarse set-up needs nothing else
  if (!wl) Acw.alloc(std::max<int64_t>(nCC, 1), s);   // a subset pass overwrites only its subdomains
  if (nw > 0) k_coarse_local<T><<<nw, 256, 0, s>>>(B.C_ptr.p, dCC->p, Sc.p, rho.p, Acw.p, wl);
  UFE_CHECK_LAUNCH();
  GC.alloc(std::max<int64_t>(nGC, 1), s);
  GC.zero();
  DBuf<double> err;
  if (sizeof(T) == 4) {
    err.alloc(ns, s);
    err.zero();
  }
  // an FP32 pass with no failed pivot so far runs the rest on a second stream beside
  // the coarse set-up, and its C Phi = I test is read after both (finish_deferred)
  bool defer = later && bad && sizeof(T) == 4;
  if (defer)
    for (int w : ws) defer = defer && !(*bad)[w];
  cudaStream_t sx = s;
  if (defer) {
    UFE_CUDA(cudaEventCreateWithFlags(&later->done, cudaEventDisableTiming));
    UFE_CUDA(cudaEventRecord(later->done, s));
    sx = objects_stream();
    UFE_CUDA(cudaStreamWaitEvent(sx, later->done, 0));
  }
  // 8. Phi^ = Y S_c^-1
  g.clear();
  for (int w : ws)
    g.push_back({B.h_nG[w], B.h_nC[w], B.h_nC[w], pad4(B.h_nC[w]), pad4(B.h_nC[w]), pad4(B.h_nC[w]), oGC[w], oCC[w], oGC[w]});
  batched_gemm<T>(false, false, g, Y.p, Sc.p, GC.p, T(1), T(0), sx);
  // 9. K^ = S'^-1 - Phi^ Y^T
  g.clear();
  for (int w : ws)
    g.push_back({B.h_nG[w], B.h_nG[w], B.h_nC[w], pad4(B.h_nC[w]), pad4(B.h_nC[w]), pad4(B.h_nG[w]), oGC[w], oGC[w], oGG[w]});
  batched_gemm<T>(false, true, g, GC.p, Y.p, GG.p, T(-1), T(1), sx);
  if (sizeof(T) == 4) {
    // FP32 operators: the coarse basis must still satisfy C Phi = I to 1e-2, else the
    // subdomain gets FP64 local operators (S_c = C S'^-1 C^T can be too ill-conditioned
    // for FP32, e.g. the rotation rows of small elasticity objects)
    g.clear();
    for (int w : ws)
      g.push_back({B.h_nC[w], B.h_nC[w], B.h_nG[w], pad4(B.h_nG[w]), pad4(B.h_nC[w]), pad4(B.h_nC[w]), oCG[w], oGC[w], oCC[w]});
    batched_gemm<T>(false, false, g, Cs.p, GC.p, Sc.p, T(1), T(0), sx);
    if (nw > 0) k_cphi_error<T><<<nw, 256, 0, sx>>>(B.C_ptr.p, dCC->p, Sc.p, 1e-2, err.p, status.p, wl);
    UFE_CHECK_LAUNCH();
    if (defer) {
      UFE_CUDA(cudaEventRecord(later->done, sx));
      later->pending = true;
      std::swap(later->err.p, err.p);
      std::swap(later->err.n, err.n);
      std::swap(later->err.s, err.s);
      // the buffers the second stream reads are released on it, after its work
      Y.s = Sc.s = Cs.s = sx;
      dCC->s = sx;
    } else {
      const std::vector<double> he = to_host(err.p, ns, s);
      check("the coarse basis (C Phi = I)");
      // the largest error over the subdomains that keep FP32 operators
      B.cphi_error = 0.0;
      for (int w : ws)
        if (!bad || !(*bad)[w]) B.cphi_error = std::max(B.cphi_error, he[w]);
    }
  }
  // 11. the operators stay in the scaled variables: the iterations apply
  //     A_II^-1 = S_I Ahat_II^-1 S_I, K = S_G Khat S_G and Phi = S_G Phihat with the FP64
  //     scale vectors, so the stored entries are O(1) whatever the cut fractions (the
  //     unscaled entries of a DOF with a 1e-40 diagonal would overflow FP32)
}

// Objects (Sect. 3.2, 4.4, 4.5), coarse DOFs and the per-subdomain coarse lists, on
// stream s.  They depend on the mesh (and, for variant 2, on the assembled cut cells)
// only, so bddc_build runs them on a stream of their own next to the local matrices
// and the interior inversions; the host waits here at every count it needs.
static void build_objects(Bddc& B, cudaStream_t s) {
  Mesh& m = *B.mesh;
  const int T = 256;
  const int64_t nd = m.n_dof;
  const int ns = (int)m.n_sub;
  const int NC = B.ncomp;
  TimedLaunch ph_obj;
  ph_obj.begin("phase_objects", s);
  // ---- standard objects
  DBuf<int32_t> label;
  DBuf<uint8_t> active, flags;
  label.alloc(nd, s);
  active.alloc(nd, s);
  flags.alloc(nd, s);
  k_init_labels<<<grid_for(nd, T), T, 0, s>>>(nd, m.n_neigh.p, label.p, active.p);
  UFE_CHECK_LAUNCH();
  propagate(m, s, active.p, 0, nullptr, label.p);
  DBuf<int32_t> rep_index;
  rep_index.alloc(nd, s);
  k_rep_flags<<<grid_for(nd, T), T, 0, s>>>(nd, label.p, flags.p);
  UFE_CHECK_LAUNCH();
  int64_t n_obj = scan_flags(flags.p, nd, rep_index.p, s);
  B.obj_of_dof.alloc(nd, s);
  B.obj_size.alloc(std::max<int64_t>(n_obj, 1), s);
  B.obj_rep.alloc(std::max<int64_t>(n_obj, 1), s);
  B.obj_kind.alloc(std::max<int64_t>(n_obj, 1), s);
  B.obj_size.zero();
  k_obj_assign<<<grid_for(nd, T), T, 0, s>>>(nd, label.p, rep_index.p, B.obj_of_dof.p, B.obj_size.p, B.obj_rep.p);
  UFE_CHECK_LAUNCH();
  if (n_obj) {
    k_obj_kind<<<grid_for(n_obj, T), T, 0, s>>>(n_obj, B.obj_rep.p, B.obj_size.p, m.n_neigh.p, nullptr, nullptr,
                                                nullptr, B.obj_kind.p);
    UFE_CHECK_LAUNCH();
  }

  // ---- variant 1 (Sect. 4.4): split the edge objects at their cut FE edges;
  //      variant 2 (Sect. 4.5): split them into runs of equal stiffness weights
  if ((B.opts.objects == UFE_OBJECTS_VARIANT1 || B.opts.objects == UFE_OBJECTS_VARIANT2) && n_obj) {
    DBuf<uint8_t> corner;
    DBuf<int32_t> label2;
    DBuf<double> wv2;
    corner.alloc(nd, s);
    label2.alloc(nd, s);
    if (B.opts.objects == UFE_OBJECTS_VARIANT1) {
      k_v1_corners<<<grid_for(nd, T), T, 0, s>>>(m.g, nd, m.node_of_dof.p, m.dof_of_node.p, m.cell_type.p, m.phi.p,
                                                 B.obj_of_dof.p, B.obj_kind.p, corner.p, active.p, label2.p, label.p);
      UFE_CHECK_LAUNCH();
      propagate(m, s, active.p, 1, B.obj_of_dof.p, label2.p);
    } else {
      wv2.alloc(std::max<int64_t>(nd, 1) * 8, s);
      k_v2_weights<<<grid_for(nd, T), T, 0, s>>>(m.g, nd, m.node_of_dof.p, m.cell_type.p, m.sub_of_cell.p,
                                                 m.cut_index.p, B.sys->K_cut.p,
                                                 B.sys->has_kappa ? B.sys->kappa.p : nullptr, m.neigh.p, m.n_neigh.p,
                                                 wv2.p);
      UFE_CHECK_LAUNCH();
      k_v2_prepare<<<grid_for(nd, T), T, 0, s>>>(nd, B.obj_of_dof.p, B.obj_kind.p, corner.p, active.p, label2.p,
                                                 label.p);
      UFE_CHECK_LAUNCH();
      propagate(m, s, active.p, 2, B.obj_of_dof.p, label2.p, wv2.p);
    }
    k_rep_flags<<<grid_for(nd, T), T, 0, s>>>(nd, label2.p, flags.p);
    UFE_CHECK_LAUNCH();
    const int64_t n_obj2 = scan_flags(flags.p, nd, rep_index.p, s);
    DBuf<int32_t> obj2, size2, rep2, kind2;
    obj2.alloc(nd, s);
    size2.alloc(n_obj2, s);
    rep2.alloc(n_obj2, s);
    kind2.alloc(n_obj2, s);
    size2.zero();
    k_obj_assign<<<grid_for(nd, T), T, 0, s>>>(nd, label2.p, rep_index.p, obj2.p, size2.p, rep2.p);
    UFE_CHECK_LAUNCH();
    k_obj_kind<<<grid_for(n_obj2, T), T, 0, s>>>(n_obj2, rep2.p, size2.p, m.n_neigh.p, B.obj_of_dof.p, B.obj_kind.p,
                                                 corner.p, kind2.p);
    UFE_CHECK_LAUNCH();
    std::swap(B.obj_of_dof.p, obj2.p);
    std::swap(B.obj_size.p, size2.p);
    std::swap(B.obj_rep.p, rep2.p);
    std::swap(B.obj_kind.p, kind2.p);
    std::swap(B.obj_size.n, size2.n);
    std::swap(B.obj_rep.n, rep2.n);
    std::swap(B.obj_kind.n, kind2.n);
    n_obj = n_obj2;
  }
  B.n_obj = n_obj;
  {
    std::vector<int32_t> kinds = to_host(B.obj_kind.p, n_obj, s);
    B.n_corner = std::count(kinds.begin(), kinds.end(), (int32_t)UFE_OBJ_CORNER);
    B.n_edge = std::count(kinds.begin(), kinds.end(), (int32_t)UFE_OBJ_EDGE);
    B.n_face = std::count(kinds.begin(), kinds.end(), (int32_t)UFE_OBJ_FACE);
  }

  // ---- coarse DOFs (rows per object) and the per-subdomain coarse lists
  B.coarse_of_obj.alloc(std::max<int64_t>(n_obj, 1), s);
  B.obj_nrows.alloc(std::max<int64_t>(n_obj, 1), s);
  B.obj_rot.alloc(std::max<int64_t>(n_obj, 1), s);
  B.obj_sum.alloc(std::max<int64_t>(n_obj, 1) * 3, s);
  B.obj_lo.alloc(std::max<int64_t>(n_obj, 1) * 3, s);
  B.obj_hi.alloc(std::max<int64_t>(n_obj, 1) * 3, s);
  B.obj_sum.zero();
  B.obj_lo.fill_bytes(0x7f);
  B.obj_hi.zero();
  if (n_obj) {
    k_obj_geom<<<grid_for(nd, T), T, 0, s>>>(m.g, nd, m.node_of_dof.p, B.obj_of_dof.p, B.obj_sum.p, B.obj_lo.p,
                                             B.obj_hi.p);
    UFE_CHECK_LAUNCH();
    DBuf<int32_t> counts, offs;
    counts.alloc(n_obj, s);
    offs.alloc(n_obj + 1, s);
    k_obj_rows<<<grid_for(n_obj, T), T, 0, s>>>(n_obj, NC, B.obj_kind.p, B.opts.coarse, B.obj_size.p, B.obj_lo.p,
                                                B.obj_hi.p, B.obj_nrows.p, B.obj_rot.p, counts.p);
    UFE_CHECK_LAUNCH();
    B.n_coarse = scan_counts(counts.p, n_obj, offs.p, s);
    k_coarse_first<<<grid_for(n_obj, T), T, 0, s>>>(n_obj, counts.p, offs.p, B.coarse_of_obj.p);
    UFE_CHECK_LAUNCH();
  } else {
    B.n_coarse = 0;
  }
  const int64_t nco = B.n_coarse;
  B.coarse_obj.alloc(std::max<int64_t>(nco, 1), s);
  B.coarse_rep.alloc(std::max<int64_t>(nco, 1), s);
  B.coarse_nn.alloc(std::max<int64_t>(nco, 1), s);
  DBuf<int32_t> nC;
  nC.alloc(ns, s);
  nC.zero();
  if (n_obj) {
    k_coarse_list<<<grid_for(n_obj, T), T, 0, s>>>(n_obj, B.coarse_of_obj.p, B.obj_rep.p, B.obj_nrows.p, m.n_neigh.p,
                                                   B.coarse_obj.p, B.coarse_rep.p, B.coarse_nn.p, m.neigh.p, nC.p);
    UFE_CHECK_LAUNCH();
  }
  B.C_ptr.alloc(ns + 1, s);
  B.n_Cloc = scan_counts(nC.p, ns, B.C_ptr.p, s);
  B.C_list.alloc(std::max<int64_t>(B.n_Cloc, 1), s);
  B.cpos.alloc(std::max<int64_t>(nco, 1) * 8, s);
  B.cpos.fill_bytes(0xff);
  if (nco) {
    k_sub_coarse_fill<<<ns, 256, 0, s>>>(nco, B.coarse_rep.p, B.coarse_nn.p, m.neigh.p, B.C_ptr.p, B.C_list.p);
    UFE_CHECK_LAUNCH();
    k_cpos<<<ns, 256, 0, s>>>(B.C_ptr.p, B.C_list.p, B.coarse_rep.p, B.coarse_nn.p, m.neigh.p, B.cpos.p);
    UFE_CHECK_LAUNCH();
  }
  std::vector<int32_t> hC = to_host(B.C_ptr.p, ns + 1, s);
  B.h_nC.resize(ns);
  B.max_nC = 0;
  for (int w = 0; w < ns; ++w) {
    B.h_nC[w] = hC[w + 1] - hC[w];
    B.max_nC = std::max(B.max_nC, B.h_nC[w]);
  }
  UFE_REQUIRE(B.max_nC <= 1024, UFE_ERR_UNSUPPORTED, "more than 1024 coarse DOFs in one subdomain");
  B.inv_flops_local = 0.0;
  for (int w = 0; w < ns; ++w)
    B.inv_flops_local += std::pow((double)B.h_nI[w], 3) + std::pow((double)B.h_nG[w], 3) + std::pow((double)B.h_nC[w], 3);

  // structural singularity: a floating subdomain (no constrained node) without coarse DOFs
  {
    DBuf<int> touch;
    touch.alloc(ns, s);
    k_touch_constrained<<<ns, 256, 0, s>>>(m.g, m.sub_block.p, m.sub_of_cell.p, m.dof_of_node.p, m.node_flags.p,
                                           touch.p);
    UFE_CHECK_LAUNCH();
    std::vector<int> t = to_host(touch.p, ns, s);
    for (int w = 0; w < ns; ++w)
      UFE_REQUIRE(t[w] || B.h_nC[w] > 0, UFE_ERR_SINGULAR_LOCAL,
                  "subdomain " + std::to_string(w) + " floats and has no coarse DOF");
  }

  ph_obj.end(s);
}

// the objects' stream (one per device, like the Gauss-Jordan look-ahead stream)
static cudaStream_t objects_stream() {
  static std::mutex mu;
  static cudaStream_t st[128] = {};
  int dev = 0;
  UFE_CUDA(cudaGetDevice(&dev));
  UFE_REQUIRE(dev >= 0 && dev < 128, UFE_ERR_UNSUPPORTED, "device ordinal beyond 127");
  std::lock_guard<std::mutex> lock(mu);
  if (!st[dev]) UFE_CUDA(cudaStreamCreateWithFlags(&st[dev], cudaStreamNonBlocking));
  return st[dev];
}

void bddc_build(Bddc& B) {
  Mesh& m = *B.mesh;
  cudaStream_t s = B.stream;
  const int T = 256;
  const int64_t nd = m.n_dof;
  const int ns = (int)m.n_sub;
  cudaEvent_t e0, e1;
  UFE_CUDA(cudaEventCreate(&e0));
  UFE_CUDA(cudaEventCreate(&e1));
  UFE_CUDA(cudaEventRecord(e0, s));
  B.status.alloc(1, s);
  B.status.zero();
  B.ncomp = B.sys->ncomp;
  const int NC = B.ncomp;
  B.vI_ptr.alloc(ns + 1, s);
  B.vG_ptr.alloc(ns + 1, s);
  k_scale_ptr<<<grid_for(ns + 1, T), T, 0, s>>>(ns + 1, NC, m.I_ptr.p, B.vI_ptr.p);
  UFE_CHECK_LAUNCH();
  k_scale_ptr<<<grid_for(ns + 1, T), T, 0, s>>>(ns + 1, NC, m.G_ptr.p, B.vG_ptr.p);
  UFE_CHECK_LAUNCH();
  B.n_vIloc = NC * m.n_Iloc;
  B.n_vGloc = NC * m.n_Gloc;
  B.max_nIv = NC * m.max_nI;
  B.max_nGv = NC * m.max_nG;
  // the per-iteration kernels hold a subdomain's vectors in one CTA's shared memory:
  // refuse local sizes beyond that before any local operator is allocated
  check_local_sizes(B);

  B.h_nI.resize(ns);
  B.h_nG.resize(ns);
  for (int w = 0; w < ns; ++w) {
    B.h_nI[w] = NC * (m.h_I_ptr[w + 1] - m.h_I_ptr[w]);
    B.h_nG[w] = NC * (m.h_G_ptr[w + 1] - m.h_G_ptr[w]);
  }
  // the objects (build_objects) need only the mesh: they start on their own stream once
  // the local matrices and the interior inversions are queued on this one
  cudaStream_t so = objects_stream();
  cudaEvent_t fork_ev, join_ev;
  UFE_CUDA(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
  UFE_CUDA(cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming));
  UFE_CUDA(cudaEventRecord(fork_ev, s));
  struct EventsGuard {
    cudaEvent_t a, b;
    ~EventsGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } events_guard{fork_ev, join_ev};

  TimedLaunch ph_loc;
  ph_loc.begin("phase_local", s);
  // ---- storage offsets (the coarse ones once the objects are known)
  std::vector<int64_t> oII(ns), oIG(ns), oGG(ns), oCG(ns), oGC(ns), oCC(ns);
  int64_t nII = 0, nIG = 0, nGG = 0, nCG = 0, nGC = 0, nCC = 0;
  for (int w = 0; w < ns; ++w) {
    const int nI = B.h_nI[w], nG = B.h_nG[w];
    oII[w] = nII; nII += (int64_t)nI * pad4(nI);
    oIG[w] = nIG; nIG += (int64_t)nG * pad4(nI);   // X^T (interface rows x interior columns)
    oGG[w] = nGG; nGG += (int64_t)nG * pad4(nG);
  }
  auto upload = [&](DBuf<int64_t>& d, const std::vector<int64_t>& v) {
    d.alloc(v.size(), s);
    UFE_CUDA(cudaMemcpyAsync(d.p, v.data(), v.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  };
  upload(B.off_II, oII);
  upload(B.off_GG, oGG);
  {
    const double tm = B.mixed ? 4.0 : 8.0;
    B.bytes_II = tm * nII;
    B.bytes_GG = tm * nGG;
    B.bytes_off = 12.0 * 27 * NC * (double)(B.n_vGloc + B.n_vIloc);
  }

  // ---- local matrices, scales, weights
  DBuf<double> AII, AIG, AGG, dGraw;
  DBuf<double>& sI = B.sI;
  DBuf<double>& sG = B.sG;
  AII.alloc(std::max<int64_t>(nII, 1), s);
  AGG.alloc(std::max<int64_t>(nGG, 1), s);
  AII.zero();
  AGG.zero();
  DBuf<int32_t>& ell_k = B.gi_k;
  DBuf<double>& ell_v = B.gi_v;
  const int KS = 27 * NC;
  ell_k.alloc(std::max<int64_t>(B.n_vGloc, 1) * KS, s);
  ell_v.alloc(std::max<int64_t>(B.n_vGloc, 1) * KS, s);
  B.ig_k.alloc(std::max<int64_t>(B.n_vIloc, 1) * KS, s);
  B.ig_v.alloc(std::max<int64_t>(B.n_vIloc, 1) * KS, s);
  sI.alloc(std::max<int64_t>(B.n_vIloc, 1), s);
  sG.alloc(std::max<int64_t>(B.n_vGloc, 1), s);
  dGraw.alloc(std::max<int64_t>(B.n_vGloc, 1), s);
  const SubMeta sm = B.meta();
  if (NC == 3) {
    k_local_assemble<3><<<dim3(ns, kLocalSplit), 256, 0, s>>>(sm, B.off_II.p, B.off_GG.p, AII.p, AGG.p);
    UFE_CHECK_LAUNCH();
    k_off_ell<3><<<dim3(ns, kLocalSplit), 256, 0, s>>>(sm, LKIND_G, ell_k.p, ell_v.p);
    UFE_CHECK_LAUNCH();
    k_off_ell<3><<<dim3(ns, kLocalSplit), 256, 0, s>>>(sm, LKIND_I, B.ig_k.p, B.ig_v.p);
    UFE_CHECK_LAUNCH();
  } else {
    k_local_assemble<1><<<dim3(ns, kLocalSplit), 256, 0, s>>>(sm, B.off_II.p, B.off_GG.p, AII.p, AGG.p);
    UFE_CHECK_LAUNCH();
    k_off_ell<1><<<dim3(ns, kLocalSplit), 256, 0, s>>>(sm, LKIND_G, ell_k.p, ell_v.p);
    UFE_CHECK_LAUNCH();
    k_off_ell<1><<<dim3(ns, kLocalSplit), 256, 0, s>>>(sm, LKIND_I, B.ig_k.p, B.ig_v.p);
    UFE_CHECK_LAUNCH();
  }
  k_local_diag<<<ns, 256, 0, s>>>(sm, NC == 3 ? 1e-8 : 0.0, B.off_II.p, B.off_GG.p, AII.p, AGG.p, sI.p, sG.p,
                                  dGraw.p);
  UFE_CHECK_LAUNCH();
  B.w.alloc(std::max<int64_t>(B.n_vGloc, 1), s);
  k_weights<<<grid_for(nd, T), T, 0, s>>>(nd, NC, m.n_neigh.p, m.gpos.p, dGraw.p,
                                          B.opts.weighting == UFE_WEIGHT_TOPOLOGICAL, B.w.p);
  UFE_CHECK_LAUNCH();

  ph_loc.end(s);
  TimedLaunch ph_fac;
  ph_fac.begin("phase_factor", s);
  // ---- factorisations and explicit local operators; step 1 (A_II^-1) is queued
  // before the objects are found
  DBuf<int> status;
  status.alloc(ns, s);
  std::vector<int> all_subs(ns);
  for (int w = 0; w < ns; ++w) all_subs[w] = w;
  if (B.mixed) {
    B.local_tc = fp32_tensor_cores() ? 1 : 0;
    factor_interior<float>(B, oII, nII, AII, sI, B.fII, status, all_subs, nullptr);
  } else {
    factor_interior<double>(B, oII, nII, AII, sI, B.dII, status, all_subs, nullptr);
  }
  UFE_CUDA(cudaStreamWaitEvent(so, fork_ev, 0));
  build_objects(B, so);
  UFE_CUDA(cudaEventRecord(join_ev, so));
  UFE_CUDA(cudaStreamWaitEvent(s, join_ev, 0));
  // the object buffers are used (and released) on this stream from here on
  B.obj_of_dof.s = B.obj_size.s = B.obj_rep.s = B.obj_kind.s = B.coarse_of_obj.s = B.obj_nrows.s = B.obj_rot.s = s;
  B.obj_lo.s = B.obj_hi.s = B.coarse_obj.s = B.coarse_rep.s = B.C_ptr.s = B.C_list.s = B.cpos.s = s;
  B.obj_sum.s = s;
  B.coarse_nn.s = s;
  for (int w = 0; w < ns; ++w) {
    const int nG = B.h_nG[w], nc = B.h_nC[w];
    oCG[w] = nCG; nCG += (int64_t)nc * pad4(nG);
    oGC[w] = nGC; nGC += (int64_t)nG * pad4(nc);
    oCC[w] = nCC; nCC += (int64_t)nc * pad4(nc);
  }
  upload(B.off_GC, oGC);
  B.bytes_GC = (B.mixed ? 4.0 : 8.0) * nGC;
  const int64_t nco = B.n_coarse;
  DBuf<double> Acw, rho;
  TimedLaunch ph_co;
  // ---- coarse matrix (FP64), assembled densely, then inverted (small problems) or
  // factored by block cyclic reduction over the z layers of subdomain blocks (coarse.cu)
  auto do_coarse = [&]() {
    ph_co.begin("phase_coarse", s);
    if (nco && B.coarse_solver == UFE_COARSE_SOLVER_BDDC) {
      // three-level method: the coarse problem is never assembled; BDDC over groups of
      // subdomains is built from the A_c^w (multilevel.cu)
      B.coarse_dense = false;
      ml_setup(B, Acw, oCC, B.coarse_group, s);
      B.cr.bytes = B.ml.bytes;
      B.cr.inv_flops = B.ml.inv_flops;
    } else if (nco) {
      const int ldc = pad4((int)nco);
      DBuf<double> Ac;
      Ac.alloc((size_t)nco * ldc, s);
      Ac.zero();
      DBuf<int64_t> dCC;
      upload(dCC, oCC);
      k_coarse_assemble<<<(unsigned)nco, 128, 0, s>>>(nco, ldc, B.coarse_rep.p, B.coarse_nn.p, m.neigh.p, B.cpos.p,
                                                      B.C_ptr.p, B.C_list.p, dCC.p, Acw.p, Ac.p);
      UFE_CHECK_LAUNCH();
      k_symmetrize<<<grid_for(nco * nco, T), T, 0, s>>>(Ac.p, (int)nco, ldc);
      UFE_CHECK_LAUNCH();
      B.Ac_inv.release();   // a second set-up (after the FP64 pass of some subdomains) replaces the first
      coarse_setup(B, Ac, ldc, s);
    } else {
      DBuf<double> none;
      coarse_setup(B, none, 4, s);
    }
    B.bytes_Ac = B.cr.bytes;
    B.inv_flops_coarse = B.cr.inv_flops;
    ph_co.end(s);
  };
  // ---- solver work space (before the coarse set-up: the solve graph can then be
  // recorded while the GPU inverts the coarse matrix)
  B.tG.alloc(std::max<int64_t>(B.n_vGloc, 1), s);
  B.vw.alloc(std::max<int64_t>(B.n_vGloc, 1), s);
  B.gC.alloc(std::max<int64_t>(B.n_Cloc, 1), s);
  B.uc.alloc(std::max<int64_t>(nco, 1), s);
  for (DBuf<double>* v : {&B.x, &B.r, &B.b, &B.z, &B.q, &B.p0, &B.p1}) {
    v->alloc(NC * nd, s);
    v->zero();
  }
  // per-CTA partial sums (the preconditioner runs up to eight CTAs per subdomain)
  B.part_blocks = std::max<int64_t>(std::max<int64_t>(grid_for(NC * nd, 256), B.sys->mesh->n_apply_tiles),
                                    16 * (int64_t)ns) + 8;
  B.part.alloc(B.part_blocks * 2, s);
  B.sc.alloc(1, s);
  B.sc.zero();
  B.tres.alloc(2, s);
  B.tres.zero();
  if (!B.h_sc) UFE_CUDA(cudaMallocHost((void**)&B.h_sc, sizeof(PcgScalars)));

  bool coarse_done = false;
  if (B.mixed) {
    // FP32 local operators where they are accurate enough; a subdomain whose FP32 pivots
    // or coarse basis fail the tests (tiny cut fractions) gets FP64 operators, factored
    // in a second pass over those subdomains only, and the iterations apply each
    // subdomain in its own precision
    std::vector<char> bad(ns, 0);
    DeferredCheck later;
    factor_pipeline<float>(B, oII, oIG, oGG, oCG, oGC, oCC, nII, nIG, nGG, nCG, nGC, nCC, AII, AIG, AGG, sI, sG,
                           ell_k, ell_v, B.fII, B.fGG, B.fGC, Acw, rho, status, true, all_subs, nullptr, &bad, &later);
    if (later.pending) {
      // every pivot passed: the coarse set-up runs while the last FP32 products and the
      // C Phi = I test finish on the second stream, then the test is read
      ph_fac.end(s);
      do_coarse();
      coarse_done = true;
      // the solve graph for the all-FP32 outcome, recorded while the GPU works (the
      // host is free); dropped below if a subdomain fails the tests
      solve_graph_early(B);
      UFE_CUDA(cudaStreamWaitEvent(s, later.done, 0));
      const std::vector<double> he = to_host(later.err.p, ns, s);
      const std::vector<int> st = to_host(status.p, ns, s);
      for (int w = 0; w < ns; ++w)
        UFE_REQUIRE(!(st[w] & DEV_TIMEOUT), UFE_ERR_TIMEOUT,
                    "the coarse basis of subdomain " + std::to_string(w) + ": a device wait did not complete in time");
      B.cphi_error = 0.0;
      for (int w = 0; w < ns; ++w) {
        if (st[w]) bad[w] = 1;
        if (!bad[w]) B.cphi_error = std::max(B.cphi_error, he[w]);
      }
    }
    std::vector<int> sub64, sub32;
    for (int w = 0; w < ns; ++w) (bad[w] ? sub64 : sub32).push_back(w);
    if (!sub64.empty()) {
      coarse_done = false;   // A_c^w of those subdomains changes
      solve_graph_reset(B);  // and so do the operators and the launch groups
    }
    if (sub32.empty()) {
      // no subdomain keeps FP32: the problem is factored and applied in FP64 throughout
      B.local_tc = 0;
      B.fII.release();
      B.fGG.release();
      B.fGC.release();
      B.mixed = false;
      B.fp64_refactor = 1;
      B.bytes_II *= 2.0;
      B.bytes_GG *= 2.0;
      B.bytes_GC *= 2.0;
      factor_pipeline<double>(B, oII, oIG, oGG, oCG, oGC, oCC, nII, nIG, nGG, nCG, nGC, nCC, AII, AIG, AGG, sI, sG,
                              ell_k, ell_v, B.dII, B.dGG, B.dGC, Acw, rho, status, false, all_subs, nullptr, nullptr);
    } else if (!sub64.empty()) {
      B.n_sub64 = (int)sub64.size();
      B.wl64.alloc(sub64.size(), s);
      B.wl32.alloc(sub32.size(), s);
      UFE_CUDA(cudaMemcpyAsync(B.wl64.p, sub64.data(), sub64.size() * 4, cudaMemcpyHostToDevice, s));
      UFE_CUDA(cudaMemcpyAsync(B.wl32.p, sub32.data(), sub32.size() * 4, cudaMemcpyHostToDevice, s));
      factor_pipeline<double>(B, oII, oIG, oGG, oCG, oGC, oCC, nII, nIG, nGG, nCG, nGC, nCC, AII, AIG, AGG, sI, sG,
                              ell_k, ell_v, B.dII, B.dGG, B.dGC, Acw, rho, status, false, sub64, B.wl64.p, nullptr);
      // the host lists go out of scope: the copies above must have read them
      UFE_CUDA(cudaStreamSynchronize(s));
    }
  } else
    factor_pipeline<double>(B, oII, oIG, oGG, oCG, oGC, oCC, nII, nIG, nGG, nCG, nGC, nCC, AII, AIG, AGG, sI, sG, ell_k,
                            ell_v, B.dII, B.dGG, B.dGC, Acw, rho, status, true, all_subs, nullptr, nullptr);
  AII.release();
  AIG.release();
  AGG.release();

  if (!coarse_done) {
    ph_fac.end(s);
    do_coarse();
  }
  // the solve graph is recorded while the GPU finishes the set-up (the host is free),
  // then the coarse inversion's pivots are read
  solve_graph_early(B);
  coarse_check(B);

  UFE_CUDA(cudaEventRecord(e1, s));
  UFE_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  UFE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  B.setup_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

}  // namespace ufe
