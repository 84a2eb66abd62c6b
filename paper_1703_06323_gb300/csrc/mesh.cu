// Mesh set-up kernels: cell classification, DOF numbering, subdomain aggregation,
// neighbour sets and subdomain-local numbering (Sect. 2.1, Sect. 3.1, Sect. 5.1).
//
// Every result here is integer and must be identical to the oracle's, so every
// kernel is written to be order independent: scans produce lexicographic
// numberings, component labels are minima, reductions break ties by index.
#include <climits>

#include "ufe_internal.cuh"

namespace ufe {

// ---------------------------------------------------------------------------
// block-wide exclusive scan (blockDim.x a multiple of 32, <= 1024)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// returns the exclusive prefix of v over the block; *total receives the sum
__device__ int block_excl_scan(int v, int* total) {
  __shared__ int warp_tot[32];
  __shared__ int s_total;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  int inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? warp_tot[lane] : 0;
    int wi = warp_incl_scan(w);
    if (lane < nw) warp_tot[lane] = wi - w;
    if (lane == nw - 1) s_total = wi;
  }
  __syncthreads();
  int res = inc - v + warp_tot[wid];
  int t = s_total;
  __syncthreads();
  *total = t;
  return res;
}

// ---------------------------------------------------------------------------
// device-wide scans (tile = 1024 items, 256 threads x 4)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

template <typename Src>
__global__ void k_tile_sums(Src src, int64_t n, int32_t* tile_sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t)
    if (base + t < n) v += src(base + t);
  int total;
  block_excl_scan(v, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// single block: exclusive scan of the tile sums in place; tile_sums[n_tiles] = total
__global__ void k_scan_tile_sums(int32_t* tile_sums, int64_t n_tiles) {
  int carry = 0;
  for (int64_t base = 0; base < n_tiles; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int v = i < n_tiles ? tile_sums[i] : 0;
    int total;
    int ex = block_excl_scan(v, &total);
    if (i < n_tiles) tile_sums[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) tile_sums[n_tiles] = carry;
}

struct FlagSrc {
  const uint8_t* f;
  __device__ int operator()(int64_t i) const { return f[i] ? 1 : 0; }
};
struct CountSrc {
  const int32_t* c;
  __device__ int operator()(int64_t i) const { return c[i]; }
};

template <typename Src, bool kFlags>
__global__ void k_scan_apply(Src src, int64_t n, const int32_t* tile_offsets, int32_t* out) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int vals[kScanItems];
  int v = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    vals[t] = (base + t < n) ? src(base + t) : 0;
    v += vals[t];
  }
  int total;
  int ex = block_excl_scan(v, &total) + tile_offsets[blockIdx.x];
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    if (base + t < n) {
      if (kFlags)
        out[base + t] = vals[t] ? ex : -1;
      else
        out[base + t] = ex;
    }
    ex += vals[t];
  }
}

template <typename Src, bool kFlags>
static int64_t scan_impl(Src src, int64_t n, int32_t* out, int32_t* total_dev, cudaStream_t s) {
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 0) tiles = 1;
  DBuf<int32_t> sums;
  sums.alloc(tiles + 1, s);
  k_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(src, n, sums.p);
  UFE_CHECK_LAUNCH();
  k_scan_tile_sums<<<1, 1024, 0, s>>>(sums.p, tiles);
  UFE_CHECK_LAUNCH();
  if (n > 0) {
    k_scan_apply<Src, kFlags><<<(unsigned)tiles, kScanThreads, 0, s>>>(src, n, sums.p, out);
    UFE_CHECK_LAUNCH();
  }
  if (total_dev)
    UFE_CUDA(cudaMemcpyAsync(total_dev, sums.p + tiles, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  return scalar_to_host(sums.p + tiles, s);
}

int64_t scan_flags(const uint8_t* flags, int64_t n, int32_t* index_out, cudaStream_t s) {
  return scan_impl<FlagSrc, true>(FlagSrc{flags}, n, index_out, nullptr, s);
}

int64_t scan_counts(const int32_t* counts, int64_t n, int32_t* offsets_out, cudaStream_t s) {
  // offsets_out has n+1 entries; the last receives the total
  return scan_impl<CountSrc, false>(CountSrc{counts}, n, offsets_out, offsets_out + n, s);
}

// ---------------------------------------------------------------------------
// Sect. 2.1: classification (internal / external / cut) by vertex signs
// ---------------------------------------------------------------------------
__global__ void k_classify(GridGeom g, const double* __restrict__ phi, uint8_t* __restrict__ cell_type) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.n_cells()) return;
  int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((int64_t)g.nx * g.ny));
  int cnt = 0;
#pragma unroll
  for (int a = 0; a < 8; ++a) cnt += phi[g.node(i + (a & 1), j + ((a >> 1) & 1), k + (a >> 2))] < 0.0;
  cell_type[c] = cnt == 0 ? UFE_CELL_EXTERNAL : (cnt == 8 ? UFE_CELL_INTERNAL : UFE_CELL_CUT);
}

// node flags: bit0 active (vertex of an active cell), bit1 on a Dirichlet box face
// (and active), bit2 pin candidate (all 8 incident cells internal)
__global__ void k_node_flags(GridGeom g, uint32_t face_mask, const uint8_t* __restrict__ cell_type,
                             uint8_t* __restrict__ flags, uint8_t* __restrict__ cons) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.n_nodes()) return;
  int i = (int)(v % (g.nx + 1)), j = (int)((v / (g.nx + 1)) % (g.ny + 1));
  int k = (int)(v / ((int64_t)(g.nx + 1) * (g.ny + 1)));
  bool act = false;
  int n_int = 0;
  for (int dk = -1; dk <= 0; ++dk)
    for (int dj = -1; dj <= 0; ++dj)
      for (int di = -1; di <= 0; ++di) {
        int ci = i + di, cj = j + dj, ck = k + dk;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= g.nx || cj >= g.ny || ck >= g.nz) continue;
        uint8_t t = cell_type[g.cell(ci, cj, ck)];
        act |= (t != UFE_CELL_EXTERNAL);
        n_int += (t == UFE_CELL_INTERNAL);
      }
  bool face = ((face_mask & 1) && i == 0) || ((face_mask & 2) && i == g.nx) || ((face_mask & 4) && j == 0) ||
              ((face_mask & 8) && j == g.ny) || ((face_mask & 16) && k == 0) || ((face_mask & 32) && k == g.nz);
  uint8_t f = (act ? 1 : 0) | ((act && face) ? 2 : 0) | (n_int == 8 ? 4 : 0);
  flags[v] = f;
  cons[v] = (act && face) ? 1 : 0;
}

// arg-min of phi over pin candidates; ties -> lowest node id (deterministic)
__device__ __forceinline__ bool key_less(double a, long long ia, double b, long long ib) {
  return (a < b) || (a == b && ia < ib);
}

__global__ void k_argmin_candidates(int64_t n, const double* __restrict__ phi, const uint8_t* __restrict__ flags,
                                    double* blk_val, long long* blk_idx) {
  __shared__ double sv[256];
  __shared__ long long si[256];
  double best = INFINITY;
  long long bi = LLONG_MAX;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (flags[v] & 4) {
      double p = phi[v];
      if (key_less(p, v, best, bi)) { best = p; bi = v; }
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s && key_less(sv[threadIdx.x + s], si[threadIdx.x + s], sv[threadIdx.x], si[threadIdx.x])) {
      sv[threadIdx.x] = sv[threadIdx.x + s];
      si[threadIdx.x] = si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { blk_val[blockIdx.x] = sv[0]; blk_idx[blockIdx.x] = si[0]; }
}

__global__ void k_argmin_final(int nb, const double* blk_val, const long long* blk_idx, long long* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double best = INFINITY;
  long long bi = LLONG_MAX;
  for (int b = 0; b < nb; ++b)
    if (key_less(blk_val[b], blk_idx[b], best, bi)) { best = blk_val[b]; bi = blk_idx[b]; }
  *out = (bi == LLONG_MAX) ? -1 : bi;
}

__global__ void k_free_flags(int64_t n, const uint8_t* __restrict__ flags, int64_t pin, uint8_t* __restrict__ freef) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint8_t f = flags[v];
  freef[v] = ((f & 1) && !(f & 2) && v != pin) ? 1 : 0;
}

__global__ void k_node_of_dof(int64_t n, const int32_t* __restrict__ dof_of_node, int32_t* __restrict__ node_of_dof) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int32_t d = dof_of_node[v];
  if (d >= 0) node_of_dof[d] = (int32_t)v;
}

// node tiles of the operator apply that hold a free DOF (flags, then the list in tile order)
__global__ void k_apply_tile_flags(GridGeom g, int64_t n_dof, const int32_t* __restrict__ node_of_dof,
                                   uint8_t* __restrict__ flags) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dof) return;
  const int64_t v = node_of_dof[d];
  const int i = (int)(v % (g.nx + 1)), j = (int)((v / (g.nx + 1)) % (g.ny + 1));
  const int k = (int)(v / ((int64_t)(g.nx + 1) * (g.ny + 1)));
  flags[apply_tile_of_node(g, i, j, k)] = 1;
}
__global__ void k_apply_tile_list(int64_t n, const int32_t* __restrict__ index, int32_t* __restrict__ list) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && index[t] >= 0) list[index[t]] = (int32_t)t;
}

// ---------------------------------------------------------------------------
// Sect. 2.1: subdomains = connected components (cells sharing a DOF) of the
// active cells of each block.  One CTA per block (up to 16^3 cells), each thread
// walking the block's cells with a stride; labels converge to the smallest cell
// index of the component (min propagation with pointer jumping; bounded).
// ---------------------------------------------------------------------------
constexpr int kMaxBlockCells = 16 * 16 * 16;
constexpr int kBlockThreads = 1024;
constexpr unsigned kCellActive = 0x100;   // vm bit: the cell is active (low 8 bits: vertices holding a DOF)

__global__ void __launch_bounds__(kBlockThreads)
k_block_components(GridGeom g, const uint8_t* __restrict__ cell_type, const int32_t* __restrict__ dof_of_node,
                   int32_t* __restrict__ comp_rank, int32_t* __restrict__ n_comp, int* status) {
  __shared__ int lab[kMaxBlockCells];
  __shared__ int rank_of[kMaxBlockCells];
  __shared__ uint16_t vm[kMaxBlockCells];
  const int b = blockIdx.x;
  const int bi = b % g.bx, bj = (b / g.bx) % g.by, bk = b / (g.bx * g.by);
  const int ncb = g.sx * g.sy * g.sz;
  for (int lc = threadIdx.x; lc < ncb; lc += blockDim.x) {
    const int li = lc % g.sx, lj = (lc / g.sx) % g.sy, lk = lc / (g.sx * g.sy);
    const int gi = bi * g.sx + li, gj = bj * g.sy + lj, gk = bk * g.sz + lk;
    unsigned m = 0;
    if (cell_type[g.cell(gi, gj, gk)] != UFE_CELL_EXTERNAL) {
      m = kCellActive;
      for (int a = 0; a < 8; ++a)
        if (dof_of_node[g.node(gi + (a & 1), gj + ((a >> 1) & 1), gk + (a >> 2))] >= 0) m |= 1u << a;
    }
    vm[lc] = (uint16_t)m;
    lab[lc] = m ? lc : INT_MAX;
  }
  __syncthreads();
  int it = 0;
  for (; it < 4 * kMaxBlockCells; ++it) {
    int changed = 0;
    for (int lc = threadIdx.x; lc < ncb; lc += blockDim.x) {
      const unsigned vmask = vm[lc];
      if (!vmask) continue;
      const int li = lc % g.sx, lj = (lc / g.sx) % g.sy, lk = lc / (g.sx * g.sy);
      int m = lab[lc];
      for (int a = 0; a < 8; ++a) {
        if (!(vmask & (1u << a))) continue;
        const int vx = li + (a & 1), vy = lj + ((a >> 1) & 1), vz = lk + (a >> 2);
        for (int oz = vz - 1; oz <= vz; ++oz) {
          if (oz < 0 || oz >= g.sz) continue;
          for (int oy = vy - 1; oy <= vy; ++oy) {
            if (oy < 0 || oy >= g.sy) continue;
            for (int ox = vx - 1; ox <= vx; ++ox) {
              if (ox < 0 || ox >= g.sx) continue;
              int l = lab[ox + g.sx * (oy + g.sy * oz)];
              if (l < m) m = l;
            }
          }
        }
      }
      int mm = lab[m];
      if (mm < m) m = mm;
      if (m < lab[lc]) {
        lab[lc] = m;
        changed = 1;
      }
    }
    if (!__syncthreads_or(changed)) break;
  }
  if (it >= 4 * kMaxBlockCells && threadIdx.x == 0) atomicOr(status, DEV_TIMEOUT);
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 0;
    for (int x = 0; x < ncb; ++x) {
      rank_of[x] = -1;
      if (lab[x] == x) rank_of[x] = r++;
    }
    n_comp[b] = r;
  }
  __syncthreads();
  for (int lc = threadIdx.x; lc < ncb; lc += blockDim.x) {
    const int li = lc % g.sx, lj = (lc / g.sx) % g.sy, lk = lc / (g.sx * g.sy);
    comp_rank[g.cell(bi * g.sx + li, bj * g.sy + lj, bk * g.sz + lk)] = vm[lc] ? rank_of[lab[lc]] : -1;
  }
}

__global__ void k_sub_of_cell(GridGeom g, const int32_t* __restrict__ comp_rank, const int32_t* __restrict__ sub_base,
                              int32_t* __restrict__ sub_of_cell) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.n_cells()) return;
  int r = comp_rank[c];
  if (r < 0) {
    sub_of_cell[c] = -1;
    return;
  }
  int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((int64_t)g.nx * g.ny));
  int b = (i / g.sx) + g.bx * ((j / g.sy) + g.by * (k / g.sz));
  sub_of_cell[c] = sub_base[b] + r;
}

__global__ void k_sub_block(int nblocks, const int32_t* __restrict__ sub_base, int32_t* __restrict__ sub_block) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  for (int s = sub_base[b]; s < sub_base[b + 1]; ++s) sub_block[s] = b;
}

// ---------------------------------------------------------------------------
// neigh(xi): sorted subdomain ids owning an active cell that contains xi
// ---------------------------------------------------------------------------
__global__ void k_neigh(GridGeom g, int64_t n_dof, const int32_t* __restrict__ node_of_dof,
                        const int32_t* __restrict__ sub_of_cell, int32_t* __restrict__ neigh,
                        uint8_t* __restrict__ n_neigh) {
  int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dof) return;
  int64_t v = node_of_dof[d];
  int i = (int)(v % (g.nx + 1)), j = (int)((v / (g.nx + 1)) % (g.ny + 1));
  int k = (int)(v / ((int64_t)(g.nx + 1) * (g.ny + 1)));
  int ids[8];
  int cnt = 0;
  for (int dk = -1; dk <= 0; ++dk)
    for (int dj = -1; dj <= 0; ++dj)
      for (int di = -1; di <= 0; ++di) {
        int ci = i + di, cj = j + dj, ck = k + dk;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= g.nx || cj >= g.ny || ck >= g.nz) continue;
        int s = sub_of_cell[g.cell(ci, cj, ck)];
        if (s < 0) continue;
        // insert into the sorted unique list
        int p = 0;
        while (p < cnt && ids[p] < s) ++p;
        if (p < cnt && ids[p] == s) continue;
        for (int q = cnt; q > p; --q) ids[q] = ids[q - 1];
        ids[p] = s;
        ++cnt;
      }
  for (int t = 0; t < 8; ++t) neigh[d * 8 + t] = t < cnt ? ids[t] : -1;
  n_neigh[d] = (uint8_t)cnt;
}

// ---------------------------------------------------------------------------
// subdomain-local numbering: the DOFs of subdomain w are the DOF nodes of its
// cells, in node order, split into interior (|neigh| = 1) and interface.
// One CTA per subdomain, walking the local nodes of its block in chunks of one node
// per thread (the running counts carry the order from chunk to chunk).
// ---------------------------------------------------------------------------
constexpr int kLocalThreads = 1024;

__device__ __forceinline__ bool node_in_sub(const GridGeom& g, int bi, int bj, int bk, int lx, int ly, int lz, int w,
                                            const int32_t* __restrict__ sub_of_cell) {
  for (int oz = lz - 1; oz <= lz; ++oz) {
    if (oz < 0 || oz >= g.sz) continue;
    for (int oy = ly - 1; oy <= ly; ++oy) {
      if (oy < 0 || oy >= g.sy) continue;
      for (int ox = lx - 1; ox <= lx; ++ox) {
        if (ox < 0 || ox >= g.sx) continue;
        if (sub_of_cell[g.cell(bi * g.sx + ox, bj * g.sy + oy, bk * g.sz + oz)] == w) return true;
      }
    }
  }
  return false;
}

__global__ void __launch_bounds__(kLocalThreads)
k_local_count(GridGeom g, const int32_t* __restrict__ sub_block, const int32_t* __restrict__ sub_of_cell,
              const int32_t* __restrict__ dof_of_node, const uint8_t* __restrict__ n_neigh,
              int32_t* __restrict__ lmap, int32_t* __restrict__ nI, int32_t* __restrict__ nG) {
  const int w = blockIdx.x;
  const int b = sub_block[w];
  const int bi = b % g.bx, bj = (b / g.bx) % g.by, bk = b / (g.bx * g.by);
  int baseI = 0, baseG = 0;
  for (int l0 = 0; l0 < g.n_local_nodes; l0 += blockDim.x) {
    const int ln = l0 + (int)threadIdx.x;
    int kind = LKIND_NONE;
    if (ln < g.n_local_nodes) {
      const int lx = ln % g.lnx, ly = (ln / g.lnx) % g.lny, lz = ln / (g.lnx * g.lny);
      const int64_t v = g.node(bi * g.sx + lx, bj * g.sy + ly, bk * g.sz + lz);
      const int32_t d = dof_of_node[v];
      if (d >= 0 && node_in_sub(g, bi, bj, bk, lx, ly, lz, w, sub_of_cell))
        kind = n_neigh[d] >= 2 ? LKIND_G : LKIND_I;
    }
    int totI, totG;
    const int pI = block_excl_scan(kind == LKIND_I, &totI);
    const int pG = block_excl_scan(kind == LKIND_G, &totG);
    if (ln < g.n_local_nodes) {
      const int idx = kind == LKIND_I ? baseI + pI : (kind == LKIND_G ? baseG + pG : 0);
      lmap[(int64_t)w * g.n_local_nodes + ln] = (kind << 24) | idx;
    }
    baseI += totI;
    baseG += totG;
  }
  if (threadIdx.x == 0) {
    nI[w] = baseI;
    nG[w] = baseG;
  }
}

__global__ void k_local_fill(GridGeom g, const int32_t* __restrict__ sub_block, const int32_t* __restrict__ dof_of_node,
                             const int32_t* __restrict__ lmap, const int32_t* __restrict__ I_ptr,
                             const int32_t* __restrict__ G_ptr, int32_t* __restrict__ I_list,
                             int32_t* __restrict__ G_list) {
  const int w = blockIdx.x;
  const int b = sub_block[w];
  const int bi = b % g.bx, bj = (b / g.bx) % g.by, bk = b / (g.bx * g.by);
  for (int ln = threadIdx.x; ln < g.n_local_nodes; ln += blockDim.x) {
    int32_t code = lmap[(int64_t)w * g.n_local_nodes + ln];
    int kind = lmap_kind(code);
    if (kind == LKIND_NONE) continue;
    const int lx = ln % g.lnx, ly = (ln / g.lnx) % g.lny, lz = ln / (g.lnx * g.lny);
    int32_t d = dof_of_node[g.node(bi * g.sx + lx, bj * g.sy + ly, bk * g.sz + lz)];
    if (kind == LKIND_I)
      I_list[I_ptr[w] + lmap_index(code)] = d;
    else
      G_list[G_ptr[w] + lmap_index(code)] = d;
  }
}

// slot of (interface DOF xi, k-th entry of neigh(xi)) in the interface-local arrays
__global__ void k_gpos(const int32_t* __restrict__ G_ptr, const int32_t* __restrict__ G_list,
                       const int32_t* __restrict__ neigh, const uint8_t* __restrict__ n_neigh, int32_t* __restrict__ gpos) {
  const int w = blockIdx.x;
  for (int j = G_ptr[w] + threadIdx.x; j < G_ptr[w + 1]; j += blockDim.x) {
    int32_t d = G_list[j];
    for (int k = 0; k < n_neigh[d]; ++k)
      if (neigh[(int64_t)d * 8 + k] == w) gpos[(int64_t)d * 8 + k] = j;
  }
}

__global__ void k_count_flag(int64_t n, const uint8_t* __restrict__ f, uint8_t mask, unsigned long long* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool hit = i < n && (f[i] & mask);
  unsigned ballot = __ballot_sync(0xffffffffu, hit);
  if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(out, (unsigned long long)__popc(ballot));
}

__global__ void k_cut_flags(int64_t n, const uint8_t* __restrict__ t, uint8_t* __restrict__ f) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) f[c] = t[c] == UFE_CELL_CUT;
}
void launch_cut_flags(int64_t n, const uint8_t* t, uint8_t* f, cudaStream_t s) {
  k_cut_flags<<<grid_for(n, 256), 256, 0, s>>>(n, t, f);
  UFE_CHECK_LAUNCH();
}

__global__ void k_count_ge2(int64_t n, const uint8_t* __restrict__ nn, unsigned long long* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool hit = i < n && nn[i] >= 2;
  unsigned ballot = __ballot_sync(0xffffffffu, hit);
  if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(out, (unsigned long long)__popc(ballot));
}
void launch_count_ge2(int64_t n, const uint8_t* nn, unsigned long long* out, cudaStream_t s) {
  k_count_ge2<<<grid_for(n, 256), 256, 0, s>>>(n, nn, out);
  UFE_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
void mesh_build(Mesh& m, const double* phi_dev, int64_t pin_node) {
  cudaStream_t s = m.stream;
  GridGeom& g = m.g;
  const int64_t nn = g.n_nodes(), nc = g.n_cells();
  const int T = 256;

  m.cell_type.alloc(nc, s);
  k_classify<<<grid_for(nc, T), T, 0, s>>>(g, phi_dev, m.cell_type.p);
  UFE_CHECK_LAUNCH();

  m.node_flags.alloc(nn, s);
  DBuf<uint8_t> cons;
  cons.alloc(nn, s);
  k_node_flags<<<grid_for(nn, T), T, 0, s>>>(g, m.face_mask, m.cell_type.p, m.node_flags.p, cons.p);
  UFE_CHECK_LAUNCH();

  DBuf<unsigned long long> cnt;
  cnt.alloc(2, s);
  cnt.zero();
  k_count_flag<<<grid_for(nn, T), T, 0, s>>>(nn, m.node_flags.p, 2, cnt.p);
  UFE_CHECK_LAUNCH();
  k_count_flag<<<grid_for(nc, T), T, 0, s>>>(nc, m.cell_type.p, 0xff, cnt.p + 1);
  UFE_CHECK_LAUNCH();
  std::vector<unsigned long long> hc = to_host(cnt.p, 2, s);
  const int64_t n_face_cons = (int64_t)hc[0];
  m.n_active = (int64_t)hc[1];

  // pinned node (Sect. 5.1): only when no box face constrains a node
  m.pin = -1;
  if (pin_node == UFE_PIN_AUTO) {
    if (n_face_cons == 0) {
      const int nb = 304;
      DBuf<double> bv;
      DBuf<long long> bidx, res;
      bv.alloc(nb, s);
      bidx.alloc(nb, s);
      res.alloc(1, s);
      k_argmin_candidates<<<nb, 256, 0, s>>>(nn, phi_dev, m.node_flags.p, bv.p, bidx.p);
      UFE_CHECK_LAUNCH();
      k_argmin_final<<<1, 32, 0, s>>>(nb, bv.p, bidx.p, res.p);
      UFE_CHECK_LAUNCH();
      m.pin = scalar_to_host(res.p, s);
      UFE_REQUIRE(m.pin >= 0, UFE_ERR_INVALID_ARG, "no node with 8 internal cells to pin");
    }
  } else if (pin_node >= 0) {
    UFE_REQUIRE(pin_node < nn, UFE_ERR_INVALID_ARG, "pin_node out of range");
    uint8_t f = scalar_to_host(m.node_flags.p + pin_node, s);
    UFE_REQUIRE(f & 1, UFE_ERR_INVALID_ARG, "pin_node is not an active node");
    m.pin = pin_node;
  } else {
    UFE_REQUIRE(pin_node == UFE_PIN_NONE, UFE_ERR_INVALID_ARG, "invalid pin_node");
  }
  m.n_constrained = n_face_cons;
  if (m.pin >= 0 && !(scalar_to_host(m.node_flags.p + m.pin, s) & 2)) m.n_constrained += 1;

  // DOFs = active nodes that are not constrained, numbered in node order
  DBuf<uint8_t> freef;
  freef.alloc(nn, s);
  k_free_flags<<<grid_for(nn, T), T, 0, s>>>(nn, m.node_flags.p, m.pin, freef.p);
  UFE_CHECK_LAUNCH();
  m.dof_of_node.alloc(nn, s);
  m.n_dof = scan_flags(freef.p, nn, m.dof_of_node.p, s);
  UFE_REQUIRE(m.n_dof > 0, UFE_ERR_INVALID_ARG, "the level set leaves no free DOF");
  m.node_of_dof.alloc(m.n_dof, s);
  k_node_of_dof<<<grid_for(nn, T), T, 0, s>>>(nn, m.dof_of_node.p, m.node_of_dof.p);
  UFE_CHECK_LAUNCH();
  {
    const int64_t nt = (int64_t)apply_tiles_x(g) * apply_tiles_y(g) * apply_tiles_z(g);
    DBuf<uint8_t> tf;
    DBuf<int32_t> tidx;
    tf.alloc(nt, s);
    tf.zero();
    tidx.alloc(nt, s);
    k_apply_tile_flags<<<grid_for(m.n_dof, T), T, 0, s>>>(g, m.n_dof, m.node_of_dof.p, tf.p);
    UFE_CHECK_LAUNCH();
    m.n_apply_tiles = scan_flags(tf.p, nt, tidx.p, s);
    m.apply_tiles.alloc(std::max<int64_t>(m.n_apply_tiles, 1), s);
    k_apply_tile_list<<<grid_for(nt, T), T, 0, s>>>(nt, tidx.p, m.apply_tiles.p);
    UFE_CHECK_LAUNCH();
  }

  // cut cells, in cell order
  {
    DBuf<uint8_t> cutf;
    cutf.alloc(nc, s);
    m.cut_index.alloc(nc, s);
    launch_cut_flags(nc, m.cell_type.p, cutf.p, s);
    m.n_cut = scan_flags(cutf.p, nc, m.cut_index.p, s);
  }

  // subdomains
  const int nblocks = g.n_blocks();
  DBuf<int32_t> comp_rank, n_comp, sub_base, status;
  comp_rank.alloc(nc, s);
  n_comp.alloc(nblocks, s);
  sub_base.alloc(nblocks + 1, s);
  status.alloc(1, s);
  status.zero();
  const int ncb = g.sx * g.sy * g.sz;
  UFE_REQUIRE(ncb <= kMaxBlockCells, UFE_ERR_INVALID_ARG, "more than 16^3 cells in one subdomain block");
  k_block_components<<<nblocks, ncb <= 512 ? 512 : kBlockThreads, 0, s>>>(g, m.cell_type.p, m.dof_of_node.p,
                                                                          comp_rank.p, n_comp.p, status.p);
  UFE_CHECK_LAUNCH();
  m.n_sub = scan_counts(n_comp.p, nblocks, sub_base.p, s);
  UFE_REQUIRE(scalar_to_host(status.p, s) == 0, UFE_ERR_TIMEOUT, "subdomain labelling did not converge");
  UFE_REQUIRE(m.n_sub > 0, UFE_ERR_INVALID_ARG, "no active cell");
  m.sub_of_cell.alloc(nc, s);
  k_sub_of_cell<<<grid_for(nc, T), T, 0, s>>>(g, comp_rank.p, sub_base.p, m.sub_of_cell.p);
  UFE_CHECK_LAUNCH();
  m.sub_block.alloc(m.n_sub, s);
  k_sub_block<<<grid_for(nblocks, T), T, 0, s>>>(nblocks, sub_base.p, m.sub_block.p);
  UFE_CHECK_LAUNCH();

  // neighbour sets and the interface
  m.neigh.alloc(m.n_dof * 8, s);
  m.n_neigh.alloc(m.n_dof, s);
  k_neigh<<<grid_for(m.n_dof, T), T, 0, s>>>(g, m.n_dof, m.node_of_dof.p, m.sub_of_cell.p, m.neigh.p, m.n_neigh.p);
  UFE_CHECK_LAUNCH();

  // local numbering
  m.lmap.alloc((size_t)m.n_sub * g.n_local_nodes, s);
  DBuf<int32_t> nI, nG;
  nI.alloc(m.n_sub, s);
  nG.alloc(m.n_sub, s);
  k_local_count<<<(unsigned)m.n_sub, kLocalThreads, 0, s>>>(g, m.sub_block.p, m.sub_of_cell.p, m.dof_of_node.p,
                                                             m.n_neigh.p, m.lmap.p, nI.p, nG.p);
  UFE_CHECK_LAUNCH();
  m.I_ptr.alloc(m.n_sub + 1, s);
  m.G_ptr.alloc(m.n_sub + 1, s);
  m.n_Iloc = scan_counts(nI.p, m.n_sub, m.I_ptr.p, s);
  m.n_Gloc = scan_counts(nG.p, m.n_sub, m.G_ptr.p, s);
  m.I_list.alloc(m.n_Iloc > 0 ? m.n_Iloc : 1, s);
  m.G_list.alloc(m.n_Gloc > 0 ? m.n_Gloc : 1, s);
  k_local_fill<<<(unsigned)m.n_sub, 256, 0, s>>>(g, m.sub_block.p, m.dof_of_node.p, m.lmap.p, m.I_ptr.p, m.G_ptr.p,
                                                  m.I_list.p, m.G_list.p);
  UFE_CHECK_LAUNCH();
  m.gpos.alloc(m.n_dof * 8, s);
  m.gpos.fill_bytes(0xff);
  k_gpos<<<(unsigned)m.n_sub, 256, 0, s>>>(m.G_ptr.p, m.G_list.p, m.neigh.p, m.n_neigh.p, m.gpos.p);
  UFE_CHECK_LAUNCH();
  m.h_I_ptr = to_host(m.I_ptr.p, m.n_sub + 1, s);
  m.h_G_ptr = to_host(m.G_ptr.p, m.n_sub + 1, s);
  m.max_nI = m.max_nG = 0;
  for (int64_t w = 0; w < m.n_sub; ++w) {
    m.max_nI = std::max(m.max_nI, m.h_I_ptr[w + 1] - m.h_I_ptr[w]);
    m.max_nG = std::max(m.max_nG, m.h_G_ptr[w + 1] - m.h_G_ptr[w]);
  }
  // interface DOF count = DOFs with |neigh| >= 2
  {
    DBuf<unsigned long long> c2;
    c2.alloc(1, s);
    c2.zero();
    launch_count_ge2(m.n_dof, m.n_neigh.p, c2.p, s);
    m.n_gamma = (int64_t)scalar_to_host(c2.p, s);
  }
}

}  // namespace ufe
